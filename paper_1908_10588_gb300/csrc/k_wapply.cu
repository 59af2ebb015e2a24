// Sparse application of one MPO site tensor (Eq. MPO) to a stacked tensor.
// The operators of the nonzero blocks are themselves sparse (q tridiagonal,
// b^+b diagonal, |i><j| a single entry) and are read row-compressed.
//
// The vibronic MPO is block sparse: most (w_in, w_out) blocks of a site are
// zero and many of the rest are identities that only carry a channel
// through the site. The middle legs of H_eff (Eq. two-site Hamiltonian) and
// of the environment updates therefore run here as a loop over the nonzero
// blocks of the site instead of a dense GEMM over w x d.
#include "common.h"

namespace vb {
namespace {

template <class R>
__global__ void wapply_kernel(const int *__restrict__ rp, const int *__restrict__ col, const R *__restrict__ val,
                              const int *__restrict__ ptr, const int *__restrict__ ent, int d, int Wp,
                              const cplx<R> *__restrict__ X, WStrides xs, cplx<R> *__restrict__ Y, WStrides ys,
                              int P, int Q) {
  long long total = (long long)P * d * Wp * Q;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int q = (int)(idx % Q);
    long long r = idx / Q;
    int wo = (int)(r % Wp);
    r /= Wp;
    int so = (int)(r % d);
    int p = (int)(r / d);
    R ax = 0, ay = 0;
    const cplx<R> *xb = X + p * xs.p + q * xs.q;
    for (int e = ptr[wo]; e < ptr[wo + 1]; ++e) {
      int wi = ent[3 * e], ident = ent[3 * e + 1], off = ent[3 * e + 2];
      const cplx<R> *xw = xb + wi * xs.w;
      if (ident) {
        cplx<R> v = xw[so * xs.s];
        ax += v.x;
        ay += v.y;
      } else {
        for (int k = rp[off + so]; k < rp[off + so + 1]; ++k) {
          const R c = val[k];
          const cplx<R> v = xw[col[k] * xs.s];
          ax = fma(c, v.x, ax);
          ay = fma(c, v.y, ay);
        }
      }
    }
    Y[p * ys.p + so * ys.s + wo * ys.w + q * ys.q] = mkc<R>(ax, ay);
  }
}

}  // namespace

template <class R>
vb_status wapply(const MpoSite &site, int dir, const cplx<R> *X, WStrides xs, long long x_size,
                 cplx<R> *Y, WStrides ys, long long y_size, int P, int Q, cudaStream_t st) {
  const int d = site.d;
  const int Wp = dir == 0 ? site.wr : site.wl;
  const int Wc = dir == 0 ? site.wl : site.wr;
  long long total = (long long)P * d * Wp * Q;
  if (total == 0) return VB_OK;
  if (P < 0 || Q < 0 || xs.p < 0 || xs.w < 0 || xs.s < 0 || xs.q < 0 || ys.p < 0 || ys.w < 0 ||
      ys.s < 0 || ys.q < 0)
    return fail(VB_EINVAL, "wapply: negative size or stride");
  const long long xmax = (P - 1) * xs.p + (Wc - 1) * xs.w + (d - 1) * xs.s + (Q - 1) * xs.q;
  const long long ymax = (P - 1) * ys.p + (Wp - 1) * ys.w + (d - 1) * ys.s + (Q - 1) * ys.q;
  if (xmax >= x_size || ymax >= y_size)
    return fail(VB_EINVAL, "wapply: view exceeds its buffer (x " + std::to_string(xmax) + " >= " +
                               std::to_string(x_size) + " or y " + std::to_string(ymax) + " >= " +
                               std::to_string(y_size) + ")");
  int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  const R *vals;
  if constexpr (sizeof(R) == 8)
    vals = reinterpret_cast<const R *>(site.d_csr_val);
  else
    vals = reinterpret_cast<const R *>(site.d_csr_val32);
  wapply_kernel<R><<<(int)blocks, threads, 0, st>>>(site.d_csr_ptr, site.d_csr_col, vals,
                                                 dir == 0 ? site.d_fwd_ptr : site.d_bwd_ptr,
                                                 dir == 0 ? site.d_fwd_ent : site.d_bwd_ent, d, Wp,
                                                 X, xs, Y, ys, P, Q);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

template vb_status wapply<double>(const MpoSite &, int, const cd *, WStrides, long long, cd *, WStrides,
                                  long long, int, int, cudaStream_t);
template vb_status wapply<float>(const MpoSite &, int, const cf *, WStrides, long long, cf *, WStrides,
                                 long long, int, int, cudaStream_t);

}  // namespace vb
