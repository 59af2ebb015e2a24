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
#include <climits>

namespace vb {
namespace {

// A block covers RB output rows (p, s', w') and TQ * QPT consecutive q of
// each; every warp stays inside one row, so the loops over the row's nonzero
// blocks and operator entries are uniform and the q accesses of a warp are
// coalesced. Index arithmetic is 32-bit and done once per row.
template <class R, int QPT>
__global__ void __launch_bounds__(128) wapply_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                                     const R *__restrict__ val, const int *__restrict__ ptr,
                                                     const int *__restrict__ ent, int d, int Wp, int rows, int TQ,
                                                     const cplx<R> *__restrict__ X, WStrides xs,
                                                     cplx<R> *__restrict__ Y, WStrides ys, int Q) {
  const int RB = blockDim.x / TQ;
  const int tq = threadIdx.x % TQ, rb = threadIdx.x / TQ;
  const int q0 = blockIdx.x * TQ * QPT + tq;
  const int xq = (int)xs.q, yq = (int)ys.q;
  for (int row = blockIdx.y * RB + rb; row < rows; row += gridDim.y * RB) {
    const int wo = row % Wp, t = row / Wp;
    const int so = t % d, p = t / d;
    R ax[QPT], ay[QPT];
#pragma unroll
    for (int j = 0; j < QPT; ++j) ax[j] = ay[j] = 0;
    const cplx<R> *xb = X + p * xs.p;
    const int e1 = ptr[wo + 1];
    for (int e = ptr[wo]; e < e1; ++e) {
      const int wi = ent[3 * e], ident = ent[3 * e + 1], off = ent[3 * e + 2];
      const cplx<R> *xw = xb + wi * xs.w;
      if (ident) {
        const cplx<R> *xr = xw + so * xs.s;
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
          const int q = q0 + j * TQ;
          if (q < Q) {
            const cplx<R> v = xr[q * xq];
            ax[j] += v.x;
            ay[j] += v.y;
          }
        }
      } else {
        const int k1 = rp[off + so + 1];
        for (int k = rp[off + so]; k < k1; ++k) {
          const R c = val[k];
          const cplx<R> *xr = xw + col[k] * xs.s;
#pragma unroll
          for (int j = 0; j < QPT; ++j) {
            const int q = q0 + j * TQ;
            if (q < Q) {
              const cplx<R> v = xr[q * xq];
              ax[j] = fma(c, v.x, ax[j]);
              ay[j] = fma(c, v.y, ay[j]);
            }
          }
        }
      }
    }
    cplx<R> *yr = Y + p * ys.p + so * ys.s + wo * ys.w;
#pragma unroll
    for (int j = 0; j < QPT; ++j) {
      const int q = q0 + j * TQ;
      if (q < Q) yr[q * yq] = mkc<R>(ax[j], ay[j]);
    }
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
  if (xs.q > INT_MAX / 4 || ys.q > INT_MAX / 4 || (long long)Q * std::max(xs.q, ys.q) > INT_MAX ||
      (long long)P * d * Wp > INT_MAX)
    return fail(VB_EINVAL, "wapply: sizes or strides out of range");
  const int rows = P * d * Wp;
  // q tiling: wide rows take 128 threads x 4 q each; narrow rows share a block
  int TQ, qpt;
  if (Q >= 512) {
    TQ = 128; qpt = 4;
  } else if (Q > 128) {
    TQ = 128; qpt = (Q + 127) / 128;
    if (qpt == 3) qpt = 4;
  } else {
    TQ = std::max(32, (Q + 31) / 32 * 32); qpt = 1;
    if (TQ == 96) TQ = 128;
  }
  const int RB = 128 / TQ;
  const long long gx = (Q + (long long)TQ * qpt - 1) / ((long long)TQ * qpt);
  const long long gy = std::min<long long>((rows + RB - 1) / RB, 65535);
  dim3 grid((unsigned)gx, (unsigned)gy);
  const R *vals;
  if constexpr (sizeof(R) == 8)
    vals = reinterpret_cast<const R *>(site.d_csr_val);
  else
    vals = reinterpret_cast<const R *>(site.d_csr_val32);
  const int *pt = dir == 0 ? site.d_fwd_ptr : site.d_bwd_ptr, *en = dir == 0 ? site.d_fwd_ent : site.d_bwd_ent;
  if (qpt == 4)
    wapply_kernel<R, 4><<<grid, 128, 0, st>>>(site.d_csr_ptr, site.d_csr_col, vals, pt, en, d, Wp, rows, TQ, X, xs,
                                              Y, ys, Q);
  else if (qpt == 2)
    wapply_kernel<R, 2><<<grid, 128, 0, st>>>(site.d_csr_ptr, site.d_csr_col, vals, pt, en, d, Wp, rows, TQ, X, xs,
                                              Y, ys, Q);
  else
    wapply_kernel<R, 1><<<grid, 128, 0, st>>>(site.d_csr_ptr, site.d_csr_col, vals, pt, en, d, Wp, rows, TQ, X, xs,
                                              Y, ys, Q);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

template vb_status wapply<double>(const MpoSite &, int, const cd *, WStrides, long long, cd *, WStrides,
                                  long long, int, int, cudaStream_t);
template vb_status wapply<float>(const MpoSite &, int, const cf *, WStrides, long long, cf *, WStrides,
                                 long long, int, int, cudaStream_t);

}  // namespace vb
