// Leading eigenpairs of the Hermitian reduced density matrix used to split
// and truncate the two-site tensor (Sec. 2.1.1: truncation by fixed M or by
// DBSS, which both keep the largest Schmidt weights).
//
// Pipeline (templated on the real type; the FP64 path runs it in double):
//  1. Householder reduction rho = Q T Q^+ (T Hermitian tridiagonal), one
//     column per step: reflector, Hermitian matrix-vector product, the
//     rank-2 update of the trailing block. Reflectors are kept row-wise in a
//     separate n x n buffer for coalesced back-transformation.
//  2. A diagonal unitary D makes T real: T' = D^+ T D with |e_j| off the
//     diagonal.
//  3. Bisection with Sturm counts gives the k_want largest eigenvalues.
//  4. Inverse iteration (tridiagonal LU with partial pivoting), run for all
//     requested vectors in parallel, alternated with an in-order block
//     Gram-Schmidt (two passes) so that clustered eigenvalues get an
//     orthonormal basis of their invariant subspace.
//  5. Back-transformation z = Q D y.
#include <algorithm>

#include <atomic>

#include "common.h"

namespace vb {
namespace {

constexpr int INVIT_ROUNDS = 3;

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <class R>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double eps = 2.220446049250313e-16, tiny = 2.2250738585072014e-308, big = 1e150,
                          huge = 1e300;
};
template <>
struct Eps<float> {
  static constexpr float eps = 1.1920929e-07f, tiny = 1.1754944e-38f, big = 1e18f, huge = 1e37f;
};

// block-wide sum, result broadcast to all threads
template <class R>
__device__ R block_sum_all(R v, R *sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double r = lane < nw ? sh[lane] : 0.0;
    r = warp_sum(r);
    if (lane == 0) sh[32] = r;
  }
  __syncthreads();
  return sh[32];
}

struct EigLayout {
  size_t off_vref, off_tau, off_dg, off_ec, off_eabs, off_delta, off_p, off_y, off_lu, off_part, off_bar, total;
  EigLayout(int n, int k, int rb) {
    const size_t cb = 2 * (size_t)rb;
    size_t o = 0;
    auto take = [&](size_t bytes) {
      size_t r = o;
      o += (bytes + 255) / 256 * 256;
      return r;
    };
    off_vref = take((size_t)n * n * cb);
    off_tau = take((size_t)n * rb);
    off_dg = take((size_t)n * rb);
    off_ec = take((size_t)n * cb);
    off_eabs = take((size_t)n * rb);
    off_delta = take((size_t)n * cb);
    off_p = take((size_t)2 * n * cb);
    off_y = take((size_t)k * n * rb);
    off_lu = take((size_t)k * n * 5 * rb + (size_t)k * n * sizeof(int));
    off_part = take((size_t)2 * 1024 * rb);
    off_bar = take(256);  // barrier count, generation, error flag
    total = o;
  }
};

// ---- 1. Householder reduction, one column j (trailing size m = n - j - 1 >= 2)
template <class R>
__global__ void hh_vector(cplx<R> *A, int n, int j, cplx<R> *vref, R *tau, R *dg, cplx<R> *ec) {
  typedef cplx<R> cd;
  __shared__ R sh[33];
  const int m = n - j - 1;
  R s = 0;
  for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) s += cabs2(A[(long long)(j + 1 + i) * n + j]);
  const R sigma = block_sum_all<R>(s, sh);
  const cd alpha = A[(long long)(j + 1) * n + j];
  cd *v = vref + (long long)j * n + j + 1;
  if (sigma == R(0)) {
    if (threadIdx.x == 0) {
      tau[j] = 0;
      ec[j] = alpha;
      dg[j] = A[(long long)j * n + j].x;
    }
    return;
  }
  const R aa = sqrt(cabs2(alpha));
  const R nx = sqrt(aa * aa + sigma);
  const cd ph = aa > R(0) ? mkc<R>(alpha.x / aa, alpha.y / aa) : mkc<R>(1, 0);
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    v[i] = (i == 0) ? cscale(ph, aa + nx) : A[(long long)(j + 1 + i) * n + j];
  if (threadIdx.x == 0) {
    tau[j] = R(1) / (nx * (nx + aa));
    ec[j] = cscale(ph, -nx);
    dg[j] = A[(long long)j * n + j].x;
  }
}

// p = tau A22 v (one warp per row of the trailing block)
template <class R>
__global__ void hh_symv(const cplx<R> *A, int n, int j, const cplx<R> *vref, const R *tau, cplx<R> *p) {
  typedef cplx<R> cd;
  const R t = tau[j];
  const int m = n - j - 1;
  const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (r >= m || t == R(0)) return;
  const cd *row = A + (long long)(j + 1 + r) * n + j + 1;
  const cd *v = vref + (long long)j * n + j + 1;
  R sx = 0, sy = 0;
  for (int c = lane; c < m; c += 32) {
    cd a = row[c], b = v[c];
    sx = fma(a.x, b.x, fma(-a.y, b.y, sx));
    sy = fma(a.x, b.y, fma(a.y, b.x, sy));
  }
  sx = warp_sum<R>(sx);
  sy = warp_sum<R>(sy);
  if (lane == 0) p[r] = mkc<R>(t * sx, t * sy);
}

// w = p - (tau/2) (v^+ p) v, in place in p
template <class R>
__global__ void hh_wvec(int n, int j, const cplx<R> *vref, const R *tau, cplx<R> *p) {
  typedef cplx<R> cd;
  __shared__ R sh[33];
  const R t = tau[j];
  if (t == R(0)) return;
  const int m = n - j - 1;
  const cd *v = vref + (long long)j * n + j + 1;
  R s = 0;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    cd a = v[c], b = p[c];
    s += a.x * b.x + a.y * b.y;  // Re(conj(v) p)
  }
  const R K = R(0.5) * t * block_sum_all<R>(s, sh);
  for (int c = threadIdx.x; c < m; c += blockDim.x) p[c] = csub(p[c], cscale(v[c], K));
}

// A22 -= v w^+ + w v^+
template <class R>
__global__ void hh_rank2(cplx<R> *A, int n, int j, const cplx<R> *vref, const R *tau, const cplx<R> *w) {
  typedef cplx<R> cd;
  if (tau[j] == R(0)) return;
  const int m = n - j - 1;
  const int r = blockIdx.y;
  const cd *v = vref + (long long)j * n + j + 1;
  const cd vr = v[r], wr = w[r];
  cd *row = A + (long long)(j + 1 + r) * n + j + 1;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    cd vc = v[c], wc = w[c];
    cd x = cadd(cmul(vr, cconj(wc)), cmul(wr, cconj(vc)));
    row[c] = csub(row[c], x);
  }
}

// ---- 2. last diagonal / off-diagonal entries, |e| and the phases of D
template <class R>
__global__ void tri_finish(const cplx<R> *A, int n, R *tau, R *dg, cplx<R> *ec, R *eabs,
                           cplx<R> *delta) {
  if (threadIdx.x != 0) return;
  if (n >= 2) {
    dg[n - 2] = A[(long long)(n - 2) * n + n - 2].x;
    ec[n - 2] = A[(long long)(n - 1) * n + n - 2];
    tau[n - 2] = 0;
  }
  dg[n - 1] = A[(long long)(n - 1) * n + n - 1].x;
  tau[n - 1] = 0;
  delta[0] = mkc<R>(1, 0);
  for (int j = 0; j + 1 < n; ++j) {
    R a = sqrt(cabs2(ec[j]));
    eabs[j] = a;
    delta[j + 1] = a > R(0) ? cmul(delta[j], mkc<R>(ec[j].x / a, ec[j].y / a)) : delta[j];
  }
  eabs[n - 1] = 0;
}

// after hh_tridiag_fused: dg[0..n-2], ec[0..n-2] are already set; only the
// last diagonal element is read from A
template <class R>
__global__ void tri_finish_fused(const cplx<R> *A, int n, R *tau, R *dg, cplx<R> *ec, R *eabs, cplx<R> *delta) {
  if (threadIdx.x != 0) return;
  dg[n - 1] = A[(long long)(n - 1) * n + n - 1].x;
  tau[n - 2] = 0;
  tau[n - 1] = 0;
  delta[0] = mkc<R>(1, 0);
  for (int j = 0; j + 1 < n; ++j) {
    R a = sqrt(cabs2(ec[j]));
    eabs[j] = a;
    delta[j + 1] = a > R(0) ? cmul(delta[j], mkc<R>(ec[j].x / a, ec[j].y / a)) : delta[j];
  }
  eabs[n - 1] = 0;
}

// ---- 3. bisection: evals[t] = (t)-th largest eigenvalue of T'
template <class R>
__device__ int sturm_count(const R *dg, const R *e, int n, R x, R pivmin) {
  // number of eigenvalues < x
  int cnt = 0;
  R q = dg[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < R(0)) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = dg[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < R(0)) ++cnt;
  }
  return cnt;
}

template <class R>
__global__ void bisect_kernel(const R *dg, const R *e, int n, int k_want, R *evals) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k_want) return;
  const R eps = Eps<R>::eps, tiny = Eps<R>::tiny;
  R lo = Eps<R>::huge, hi = -Eps<R>::huge, emax = 0;
  for (int i = 0; i < n; ++i) {
    R r = (i > 0 ? e[i - 1] : R(0)) + (i + 1 < n ? e[i] : R(0));
    lo = fmin(lo, dg[i] - r);
    hi = fmax(hi, dg[i] + r);
    emax = fmax(emax, fabs(dg[i]) + r);
  }
  const R tnorm = fmax(emax, tiny);
  const R pivmin = tiny * fmax(R(1), tnorm * tnorm);
  lo -= R(2) * eps * tnorm * n + tiny;
  hi += R(2) * eps * tnorm * n + tiny;
  const int target = n - 1 - t;  // ascending index
  for (int it = 0; it < 200; ++it) {
    R mid = R(0.5) * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (hi - lo <= R(2) * eps * fmax(fabs(lo), fabs(hi)) + R(1e-18) * tnorm) break;
    int c = sturm_count<R>(dg, e, n, mid, pivmin);
    if (c > target)
      hi = mid;
    else
      lo = mid;
  }
  evals[t] = R(0.5) * (lo + hi);
}

// ---- 4. inverse iteration, one thread per vector
__device__ __forceinline__ double hash_unit(int t, int i) {
  unsigned int h = (unsigned int)(t * 7919 + 17) * 2654435761u ^ (unsigned int)(i + 1) * 2246822519u;
  h ^= h >> 15;
  h *= 2654435761u;
  h ^= h >> 13;
  return (double)(h & 0xFFFFFF) / (double)0x1000000 * 2.0 - 1.0;
}

template <class R>
__global__ void invit_round(const R *dg, const R *e, int n, int k_vec, const R *evals, R *Y, R *lu,
                            int *piv, int round) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k_vec) return;
  R *y = Y + (long long)t * n;
  R *dl = lu + (long long)t * n * 4;
  R *dd = dl + n, *du = dd + n, *du2 = du + n;
  int *pv = piv + (long long)t * n;
  R tnorm = 0;
  for (int i = 0; i < n; ++i)
    tnorm = fmax(tnorm, fabs(dg[i]) + (i > 0 ? e[i - 1] : R(0)) + (i + 1 < n ? e[i] : R(0)));
  const R pivmin = fmax(tnorm * Eps<R>::eps, Eps<R>::tiny);
  const R lam = evals[t];
  if (round == 0) {
    // factor T' - lam I = P L U once
    for (int i = 0; i < n; ++i) {
      dd[i] = dg[i] - lam;
      if (i + 1 < n) {
        dl[i] = e[i];
        du[i] = e[i];
      }
      du2[i] = 0;
      pv[i] = 0;
    }
    for (int i = 0; i + 1 < n; ++i) {
      if (fabs(dd[i]) >= fabs(dl[i])) {
        if (dd[i] == R(0)) dd[i] = pivmin;
        R l = dl[i] / dd[i];
        dl[i] = l;
        dd[i + 1] -= l * du[i];
        pv[i] = 0;
      } else {
        R l = dd[i] / dl[i];
        dd[i] = dl[i];
        dl[i] = l;
        R tmp = du[i];
        du[i] = dd[i + 1];
        dd[i + 1] = tmp - l * dd[i + 1];
        if (i + 2 < n) {
          du2[i] = du[i + 1];
          du[i + 1] = -l * du[i + 1];
        }
        pv[i] = 1;
      }
    }
    if (dd[n - 1] == R(0)) dd[n - 1] = pivmin;
    for (int i = 0; i < n; ++i) y[i] = R(hash_unit(t, i));
  }
  // solve (T' - lam I) y_new = y
  for (int i = 0; i + 1 < n; ++i) {
    if (pv[i]) {
      R tmp = y[i];
      y[i] = y[i + 1];
      y[i + 1] = tmp;
    }
    y[i + 1] -= dl[i] * y[i];
  }
  // back substitution; the system is linear, so the whole vector may be
  // rescaled whenever a component grows large (near-singular shifts)
  for (int i = n - 1; i >= 0; --i) {
    R v = y[i];
    if (i + 1 < n) v -= du[i] * y[i + 1];
    if (i + 2 < n) v -= du2[i] * y[i + 2];
    v /= dd[i];
    y[i] = v;
    if (fabs(v) > Eps<R>::big)
      for (int q = 0; q < n; ++q) y[q] *= R(1) / Eps<R>::big;
  }
  // normalise (guard against overflow by scaling with the max first)
  R mx = 0;
  for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(y[i]));
  if (mx == R(0)) mx = 1;
  R s = 0;
  for (int i = 0; i < n; ++i) {
    y[i] /= mx;
    s += y[i] * y[i];
  }
  s = R(1) / sqrt(s);
  for (int i = 0; i < n; ++i) y[i] *= s;
}

// in-order two-pass Gram-Schmidt of the rows of Y (descending eigenvalues)
template <class R>
__global__ void cgs2_rows(R *Y, int n, int k) {
  __shared__ R sh[33];
  __shared__ R coef[128];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = 0; t < k; ++t) {
    R *yt = Y + (long long)t * n;
    for (int pass = 0; pass < 2; ++pass) {
      for (int s = wid; s < t; s += nw) {
        const R *ys = Y + (long long)s * n;
        R d = 0;
        for (int i = lane; i < n; i += 32) d += ys[i] * yt[i];
        d = warp_sum<R>(d);
        if (lane == 0) coef[s] = d;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        R v = yt[i];
        for (int s = 0; s < t; ++s) v -= coef[s] * Y[(long long)s * n + i];
        yt[i] = v;
      }
      __syncthreads();
    }
    R ss = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) ss += yt[i] * yt[i];
    ss = block_sum_all<R>(ss, sh);
    const R inv = ss > R(0) ? R(1) / sqrt(ss) : R(0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) yt[i] *= inv;
    __syncthreads();
  }
}

// ---- 4'. block Gram-Schmidt of the rows of Y in panels of BGS_PANEL rows:
// every panel is projected twice against all earlier rows (multi-block
// kernels), then orthonormalised in order inside the panel (one block)
constexpr int BGS_PANEL = 16;

// C[s][p] = <Y_s, Y_{p0+p}>, s < p0, p < b: one warp per pair
template <class R>
__global__ void bgs_dots(const R *Y, int n, int p0, int b, R *C) {
  const int pair = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (pair >= p0 * b) return;
  const int s = pair / b, p = pair % b;
  const R *ys = Y + (long long)s * n, *yp = Y + (long long)(p0 + p) * n;
  R d = 0;
  for (int i = lane; i < n; i += 32) d += ys[i] * yp[i];
  d = warp_sum<R>(d);
  if (lane == 0) C[s * b + p] = d;
}

// Y_{p0+p} -= sum_{s < p0} C[s][p] Y_s
template <class R>
__global__ void bgs_update(R *Y, int n, int p0, int b, const R *C) {
  const long long total = (long long)b * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(e / n), i = (int)(e % n);
    R v = Y[(long long)(p0 + p) * n + i];
    for (int s = 0; s < p0; ++s) v -= C[s * b + p] * Y[(long long)s * n + i];
    Y[(long long)(p0 + p) * n + i] = v;
  }
}

// in-panel two-pass Gram-Schmidt and normalisation of rows [p0, p0 + b)
template <class R>
__global__ void bgs_panel(R *Y, int n, int p0, int b) {
  __shared__ R sh[33];
  __shared__ R coef[BGS_PANEL];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = p0; t < p0 + b; ++t) {
    R *yt = Y + (long long)t * n;
    for (int pass = 0; pass < 2; ++pass) {
      for (int s = p0 + wid; s < t; s += nw) {
        const R *ys = Y + (long long)s * n;
        R d = 0;
        for (int i = lane; i < n; i += 32) d += ys[i] * yt[i];
        d = warp_sum<R>(d);
        if (lane == 0) coef[s - p0] = d;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        R v = yt[i];
        for (int s = p0; s < t; ++s) v -= coef[s - p0] * Y[(long long)s * n + i];
        yt[i] = v;
      }
      __syncthreads();
    }
    R ss = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) ss += yt[i] * yt[i];
    ss = block_sum_all<R>(ss, sh);
    const R inv = ss > R(0) ? R(1) / sqrt(ss) : R(0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) yt[i] *= inv;
    __syncthreads();
  }
}

// ---- 5. z_t = Q D y_t, one block per vector
template <class R>
__global__ void backtransform(const cplx<R> *vref, const R *tau, const cplx<R> *delta, const R *Y, int n,
                              cplx<R> *Z) {
  typedef cplx<R> cd;
  __shared__ R sh[33];
  const int t = blockIdx.x;
  const R *y = Y + (long long)t * n;
  cd *z = Z + (long long)t * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = cscale(delta[i], y[i]);
  __syncthreads();
  for (int j = n - 3; j >= 0; --j) {
    const R tj = tau[j];
    if (tj == R(0)) continue;
    const cd *v = vref + (long long)j * n;
    R sx = 0, sy = 0;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      cd a = v[i], b = z[i];
      sx += a.x * b.x + a.y * b.y;
      sy += a.x * b.y - a.y * b.x;
    }
    sx = block_sum_all<R>(sx, sh);
    sy = block_sum_all<R>(sy, sh);
    const cd f = mkc<R>(tj * sx, tj * sy);
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) z[i] = csub(z[i], cmul(v[i], f));
    __syncthreads();
  }
}


// ---- 1'. the whole Householder reduction in one cooperative launch
//
// One block per SM; the blocks meet at a bounded grid barrier twice per
// column. Every block recomputes the reflector of column j from row j
// (contiguous: A is kept Hermitian in both triangles, so row j holds the
// conjugated column), so no barrier is needed for it.
constexpr long long GB_LIMIT = 1LL << 27;  // polls before a barrier is declared failed (well over a second)

__device__ bool grid_barrier(unsigned int *count, volatile unsigned int *gen, unsigned int nblocks, int *err,
                             int *sh_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (*(volatile int *)err) {
      ok = 0;
    } else {
      const unsigned int g = *gen;
      __threadfence();
      const unsigned int arrived = atomicAdd(count, 1u);
      if (arrived == nblocks - 1) {
        atomicExch(count, 0u);
        __threadfence();
        atomicAdd((unsigned int *)gen, 1u);
      } else {
        long long i = 0;
        while (*gen == g) {
          if (++i > GB_LIMIT || ((i & 1023) == 0 && *(volatile int *)err)) {
            atomicExch(err, 1);
            ok = 0;
            break;
          }
        }
      }
      __threadfence();
    }
    *sh_ok = ok;
  }
  __syncthreads();
  return *sh_ok != 0;
}

template <class R>
__global__ void __launch_bounds__(512) hh_tridiag_coop(cplx<R> *A, int n, cplx<R> *vref, R *tau, R *dg,
                                                       cplx<R> *ec, cplx<R> *p, R *partial, unsigned int *bar,
                                                       int *err) {
  typedef cplx<R> cd;
  __shared__ R sh[33];
  __shared__ R shw[16];
  __shared__ int sh_ok;
  const unsigned int nb = gridDim.x;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + wib, GW = nb * wpb;
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    const cd *rowj = A + (long long)j * n + j + 1;  // conj of column j below the diagonal
    R s = 0;
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) s += cabs2(rowj[i]);
    const R sigma = block_sum_all<R>(s, sh);
    const cd alpha = cconj(rowj[0]);
    if (sigma == R(0)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        tau[j] = 0;
        ec[j] = alpha;
        dg[j] = A[(long long)j * n + j].x;
      }
      continue;  // identical decision in every block: no barrier needed
    }
    const R aa = sqrt(cabs2(alpha));
    const R nx = sqrt(aa * aa + sigma);
    const cd ph = aa > R(0) ? mkc<R>(alpha.x / aa, alpha.y / aa) : mkc<R>(1, 0);
    const cd v0 = cscale(ph, aa + nx);
    const R t = R(1) / (nx * (nx + aa));
    if (blockIdx.x == 0) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) vref[(long long)j * n + j + 1 + i] = i == 0 ? v0 : cconj(rowj[i]);
      if (threadIdx.x == 0) {
        tau[j] = t;
        ec[j] = cscale(ph, -nx);
        dg[j] = A[(long long)j * n + j].x;
      }
    }
    // p = t A22 v (one warp per row), with the partial sums of Re(v^+ p)
    R wsum = 0;
    for (int r = gw; r < m; r += GW) {
      const cd *row = A + (long long)(j + 1 + r) * n + j + 1;
      R sx = 0, sy = 0;
      for (int c = lane; c < m; c += 32) {
        const cd a = row[c];
        const cd v = c == 0 ? v0 : cconj(rowj[c]);
        sx = fma(a.x, v.x, fma(-a.y, v.y, sx));
        sy = fma(a.x, v.y, fma(a.y, v.x, sy));
      }
      sx = warp_sum<R>(sx);
      sy = warp_sum<R>(sy);
      if (lane == 0) {
        const cd pr = mkc<R>(t * sx, t * sy);
        p[r] = pr;
        const cd vr = r == 0 ? v0 : cconj(rowj[r]);
        wsum += vr.x * pr.x + vr.y * pr.y;
      }
    }
    if (lane == 0) shw[wib] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      R b = 0;
      for (int w = 0; w < wpb; ++w) b += shw[w];
      partial[blockIdx.x] = b;
    }
    if (!grid_barrier(bar, bar + 1, nb, err, &sh_ok)) return;
    // K = (t/2) Re(v^+ p); w = p - K v; A22 -= v w^+ + w v^+
    R tot = 0;
    for (unsigned int b = 0; b < nb; ++b) tot += partial[b];
    const R K = R(0.5) * t * tot;
    for (int r = gw; r < m; r += GW) {
      cd *row = A + (long long)(j + 1 + r) * n + j + 1;
      const cd vr = r == 0 ? v0 : cconj(rowj[r]);
      const cd wr = csub(p[r], cscale(vr, K));
      for (int c = lane; c < m; c += 32) {
        const cd vc = c == 0 ? v0 : cconj(rowj[c]);
        const cd wc = csub(p[c], cscale(vc, K));
        const cd x = cadd(cmul(vr, cconj(wc)), cmul(wr, cconj(vc)));
        row[c] = csub(row[c], x);
      }
    }
    if (!grid_barrier(bar, bar + 1, nb, err, &sh_ok)) return;
  }
}

// ---- 1''. the reduction with one grid barrier per column (look-ahead)
//
// Invariant at the top of iteration j: the trailing block A22_j = A[j+1:, j+1:]
// is stored up to date; every block holds the reflector v_j (shared memory);
// p_j = tau_j A22_j v_j and the block partials of Re(v_j^+ p_j) are in
// global memory. After the barrier each block forms w_j = p_j - K_j v_j,
// recomputes the updated row j+1 on its own and derives reflector j+1 from
// it, then one fused pass over its rows of A22_j applies the rank-2 update
// and dots each updated row with v_{j+1}, producing p_{j+1}. Column j+1 and
// row j+1 are not written back (their content lives in v_{j+1}, dg, ec).
template <class R>
__global__ void __launch_bounds__(512) hh_tridiag_fused(cplx<R> *A, int n, cplx<R> *vref, R *tau, R *dg,
                                                        cplx<R> *ec, cplx<R> *p, R *partial, unsigned int *bar,
                                                        int *err) {
  typedef cplx<R> cd;
  extern __shared__ __align__(16) unsigned char fsm[];
  cd *vbuf0 = reinterpret_cast<cd *>(fsm);
  cd *vbuf1 = vbuf0 + n;
  cd *wbuf = vbuf1 + n;  // w_j = p_j - K_j v_j of the current column
  __shared__ R sh[33];
  __shared__ R shw[16];
  __shared__ int sh_ok;
  __shared__ R s_tau;
  const unsigned int nb = gridDim.x;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + wib, GW = nb * wpb;
  cd *vcur = vbuf0, *vnext = vbuf1;
  // double-buffered p and block partials: iteration j reads one, writes the other
  cd *pcur = p, *pnext = p + n;
  R *partcur = partial, *partnext = partial + 1024;
  // reflector 0 from row 0 (redundantly in every block)
  {
    const int m = n - 1;
    const cd *row0 = A + 1;
    R s = 0;
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) s += cabs2(row0[i]);
    const R sigma = block_sum_all<R>(s, sh);
    const cd alpha = cconj(row0[0]);
    R t = 0;
    cd beta = alpha;
    if (sigma != R(0)) {
      const R aa = sqrt(cabs2(alpha));
      const R nx = sqrt(aa * aa + sigma);
      const cd ph = aa > R(0) ? mkc<R>(alpha.x / aa, alpha.y / aa) : mkc<R>(1, 0);
      t = R(1) / (nx * (nx + aa));
      beta = cscale(ph, -nx);
      for (int i = threadIdx.x; i < m; i += blockDim.x) vcur[i] = i == 0 ? cscale(ph, aa + nx) : cconj(row0[i]);
    } else {
      for (int i = threadIdx.x; i < m; i += blockDim.x) vcur[i] = mkc<R>(0, 0);
    }
    if (threadIdx.x == 0) s_tau = t;
    __syncthreads();
    if (blockIdx.x == 0) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) vref[1 + i] = vcur[i];
      if (threadIdx.x == 0) {
        tau[0] = t;
        ec[0] = beta;
        dg[0] = A[0].x;
      }
    }
    // p_0 = t A22_0 v_0
    R wsum = 0;
    for (int r = gw; r < m; r += GW) {
      const cd *row = A + (long long)(1 + r) * n + 1;
      R sx = 0, sy = 0;
      for (int c = lane; c < m; c += 32) {
        const cd a = row[c], v = vcur[c];
        sx = fma(a.x, v.x, fma(-a.y, v.y, sx));
        sy = fma(a.x, v.y, fma(a.y, v.x, sy));
      }
      sx = warp_sum<R>(sx);
      sy = warp_sum<R>(sy);
      if (lane == 0) {
        const cd pr = mkc<R>(t * sx, t * sy);
        pcur[r] = pr;
        wsum += vcur[r].x * pr.x + vcur[r].y * pr.y;
      }
    }
    if (lane == 0) shw[wib] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      R b = 0;
      for (int w = 0; w < wpb; ++w) b += shw[w];
      partcur[blockIdx.x] = b;
    }
  }
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;  // size of A22_j
    if (!grid_barrier(bar, bar + 1, nb, err, &sh_ok)) return;
    const R t = s_tau;
    if (wib == 0) {
      R ps = 0;
      for (unsigned int b = lane; b < nb; b += 32) ps += partcur[b];
      ps = warp_sum<R>(ps);
      if (lane == 0) sh[32] = ps;
    }
    __syncthreads();
    const R K = R(0.5) * t * sh[32];
    for (int c = threadIdx.x; c < m; c += blockDim.x) wbuf[c] = csub(pcur[c], cscale(vcur[c], K));
    __syncthreads();
    // look-ahead: updated row 0 of A22_j, u(c) = A22_j[0][c] - (v_0 conj(w_c) + w_0 conj(v_c))
    const cd *row0 = A + (long long)(j + 1) * n + (j + 1);
    const cd v0 = vcur[0];
    const cd w0 = wbuf[0];
    const bool last = (j + 1 == n - 2);  // no reflector after this one
    R s = 0;
    for (int c = 1 + threadIdx.x; c < m; c += blockDim.x) {
      const cd vc = vcur[c], wc = wbuf[c];
      const cd u = csub(row0[c], cadd(cmul(v0, cconj(wc)), cmul(w0, cconj(vc))));
      vnext[c - 1] = cconj(u);  // column j+1 below the diagonal
      if (c >= 2) s += cabs2(u);
    }
    const R sigma = block_sum_all<R>(s, sh);  // includes a __syncthreads: vnext complete
    const cd u0 = csub(row0[0], cadd(cmul(v0, cconj(w0)), cmul(w0, cconj(v0))));
    R tn = 0;
    if (!last) {
      const cd alpha = vnext[0];
      cd beta = alpha;
      if (sigma != R(0)) {
        const R aa = sqrt(cabs2(alpha));
        const R nx = sqrt(aa * aa + sigma);
        const cd ph = aa > R(0) ? mkc<R>(alpha.x / aa, alpha.y / aa) : mkc<R>(1, 0);
        tn = R(1) / (nx * (nx + aa));
        beta = cscale(ph, -nx);
        __syncthreads();
        if (threadIdx.x == 0) vnext[0] = cscale(ph, aa + nx);
      } else {
        __syncthreads();
        for (int i = threadIdx.x; i < m - 1; i += blockDim.x) vnext[i] = mkc<R>(0, 0);
      }
      __syncthreads();
      if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < m - 1; i += blockDim.x) vref[(long long)(j + 1) * n + (j + 2) + i] = vnext[i];
        if (threadIdx.x == 0) {
          tau[j + 1] = tn;
          ec[j + 1] = beta;
          dg[j + 1] = u0.x;
        }
      }
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
      tau[j + 1] = 0;
      ec[j + 1] = vnext[0];
      dg[j + 1] = u0.x;
    }
    // fused pass: update rows r >= 1 of A22_j (columns c >= 1) and dot with v_{j+1}
    R wsum = 0;
    for (int r = 1 + gw; r < m; r += GW) {
      cd *row = A + (long long)(j + 1 + r) * n + (j + 1);
      const cd vr = vcur[r], wr = wbuf[r];
      R sx = 0, sy = 0;
#pragma unroll 4
      for (int c = 1 + lane; c < m; c += 32) {
        const cd vc = vcur[c], wc = wbuf[c];
        const cd a = csub(row[c], cadd(cmul(vr, cconj(wc)), cmul(wr, cconj(vc))));
        row[c] = a;
        if (!last) {
          const cd v = vnext[c - 1];
          sx = fma(a.x, v.x, fma(-a.y, v.y, sx));
          sy = fma(a.x, v.y, fma(a.y, v.x, sy));
        }
      }
      if (!last) {
        sx = warp_sum<R>(sx);
        sy = warp_sum<R>(sy);
        if (lane == 0) {
          const cd pr = mkc<R>(tn * sx, tn * sy);
          pnext[r - 1] = pr;
          wsum += vnext[r - 1].x * pr.x + vnext[r - 1].y * pr.y;
        }
      }
    }
    if (lane == 0) shw[wib] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      R b = 0;
      for (int w = 0; w < wpb; ++w) b += shw[w];
      partnext[blockIdx.x] = b;  // read by every block after the next barrier only
      s_tau = tn;
    }
    cd *tv = vcur;
    vcur = vnext;
    vnext = tv;
    cd *tp = pcur;
    pcur = pnext;
    pnext = tp;
    R *tq = partcur;
    partcur = partnext;
    partnext = tq;
  }
}

// ---- 3'. multisection: one warp per eigenvalue, 32 Sturm counts per step
template <class R>
__global__ void multisect_kernel(const R *dg, const R *e, int n, int k_want, R *evals) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= k_want) return;
  const R eps = Eps<R>::eps, tiny = Eps<R>::tiny;
  R lo = Eps<R>::huge, hi = -Eps<R>::huge, emax = 0;
  for (int i = 0; i < n; ++i) {
    R r = (i > 0 ? e[i - 1] : R(0)) + (i + 1 < n ? e[i] : R(0));
    lo = fmin(lo, dg[i] - r);
    hi = fmax(hi, dg[i] + r);
    emax = fmax(emax, fabs(dg[i]) + r);
  }
  const R tnorm = fmax(emax, tiny);
  const R pivmin = tiny * fmax(R(1), tnorm * tnorm);
  lo -= R(2) * eps * tnorm * n + tiny;
  hi += R(2) * eps * tnorm * n + tiny;
  const int target = n - 1 - t;  // ascending index: count(lo) <= target < count(hi)
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= R(2) * eps * fmax(fabs(lo), fabs(hi)) + R(1e-18) * tnorm) break;
    const R x = lo + (hi - lo) * R(lane + 1) / R(33);
    const int c = sturm_count<R>(dg, e, n, x, pivmin);
    // largest lane whose point still has count <= target -> new lo; next point -> new hi
    const unsigned int below = __ballot_sync(0xffffffffu, c <= target);
    const int kb = below ? 31 - __clz(below) : -1;  // highest lane with c <= target
    const R nlo = kb >= 0 ? __shfl_sync(0xffffffffu, x, kb) : lo;
    const R nhi = kb < 31 ? __shfl_sync(0xffffffffu, x, kb + 1 > 31 ? 31 : kb + 1) : hi;
    if (!(nlo > lo || nhi < hi)) break;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) evals[t] = R(0.5) * (lo + hi);
}

}  // namespace

size_t EigWork::bytes(int n, int k_want, int real_bytes) { return EigLayout(n, k_want, real_bytes).total; }

vb_status EigWork::check(int n, int k_want, int real_bytes, const void *work, cudaStream_t st) {
  EigLayout lay(n, k_want, real_bytes);
  const int *err = reinterpret_cast<const int *>(static_cast<const char *>(work) + lay.off_bar) + 2;
  int h = 0;
  VB_TRY_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  VB_TRY_CUDA(cudaStreamSynchronize(st));
  if (h) return fail(VB_ETIMEOUT, "eigensolver: a grid barrier of the tridiagonal reduction ran out");
  return VB_OK;
}

template <class R>
vb_status eig_values(int n, cplx<R> *rho, int k_want, R *evals, void *work, cudaStream_t st) {
  typedef cplx<R> C_;
  if (n < 1 || k_want < 1 || k_want > n) return fail(VB_EINVAL, "eig_values: bad n / k_want");
  EigLayout lay(n, k_want, sizeof(R));
  char *w = static_cast<char *>(work);
  C_ *vref = reinterpret_cast<C_ *>(w + lay.off_vref);
  R *tau = reinterpret_cast<R *>(w + lay.off_tau);
  R *dg = reinterpret_cast<R *>(w + lay.off_dg);
  C_ *ec = reinterpret_cast<C_ *>(w + lay.off_ec);
  R *eabs = reinterpret_cast<R *>(w + lay.off_eabs);
  C_ *delta = reinterpret_cast<C_ *>(w + lay.off_delta);
  C_ *p = reinterpret_cast<C_ *>(w + lay.off_p);
  if (n <= 64 || (sizeof(R) == 8 && n > 256)) {
    // small matrices, and large FP64 ones: four launches per column. (A large
    // FP64 reduction is bound by GB300's FP64 issue rate, where these
    // per-column kernels spread the rank-2 update over every SM; the
    // cooperative kernel wins in FP32 and for small FP64 matrices, where
    // barriers and launches dominate.)
    VB_TRY_CUDA(cudaMemsetAsync(w + lay.off_bar, 0, 3 * sizeof(unsigned int), st));
    // small matrices: four launches per column are cheaper than a grid-wide launch
    for (int j = 0; j + 2 < n; ++j) {
      const int m = n - j - 1;
      hh_vector<R><<<1, 256, 0, st>>>(rho, n, j, vref, tau, dg, ec);
      VB_CHECK_LAUNCH();
      hh_symv<R><<<(m + 7) / 8, 256, 0, st>>>(rho, n, j, vref, tau, p);
      VB_CHECK_LAUNCH();
      hh_wvec<R><<<1, 256, 0, st>>>(n, j, vref, tau, p);
      VB_CHECK_LAUNCH();
      dim3 g2((m + 255) / 256, m);
      hh_rank2<R><<<g2, 256, 0, st>>>(rho, n, j, vref, tau, p);
      VB_CHECK_LAUNCH();
    }
  } else if (n > 2) {
    R *part = reinterpret_cast<R *>(w + lay.off_part);
    unsigned int *bar = reinterpret_cast<unsigned int *>(w + lay.off_bar);
    int *err = reinterpret_cast<int *>(bar + 2);
    VB_TRY_CUDA(cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned int), st));
    int dev = 0, sms = 0, per_sm = 0;
    VB_TRY_CUDA(cudaGetDevice(&dev));
    VB_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    VB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hh_tridiag_coop<R>, 512, 0));
    if (per_sm < 1) return fail(VB_ECUDA, "eig_values: cooperative kernel does not fit on an SM");
    // one block per SM at most; for small matrices fewer blocks (16 warps
    // each) make the grid barrier cheaper without idling rows. FP64 runs at
    // two FMA per clock and SM on this part, so there the blocks are 4 warps
    // (one per scheduler) and each warp owns about one row.
    const int bt = sizeof(R) == 8 ? 128 : 512;
    int nb = sizeof(R) == 8 ? std::min(sms, std::max(8, (n + 3) / 4)) : std::min(sms, std::max(8, (n + 15) / 16));
    if (nb > 1024) nb = 1024;
    void *args[] = {(void *)&rho, (void *)&n, (void *)&vref, (void *)&tau, (void *)&dg, (void *)&ec,
                    (void *)&p, (void *)&part, (void *)&bar, (void *)&err};
    const size_t vsm = (size_t)3 * n * sizeof(C_);
    if (vsm <= 44 * 1024) {
      // one barrier per column; the reflectors stay in shared memory
      VB_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)hh_tridiag_fused<R>, dim3(nb), dim3(bt), args, vsm, st));
      count_launch();
      tri_finish_fused<R><<<1, 32, 0, st>>>(rho, n, tau, dg, ec, eabs, delta);
      VB_CHECK_LAUNCH();
      goto values;
    }
    VB_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)hh_tridiag_coop<R>, dim3(nb), dim3(512), args, 0, st));
    count_launch();
  }
  tri_finish<R><<<1, 32, 0, st>>>(rho, n, tau, dg, ec, eabs, delta);
  VB_CHECK_LAUNCH();
values:
  {
    // FP64: one warp per block, so the warps (one per eigenvalue) land on
    // separate SMs and do not share an FP64 pipe
    const int mt = sizeof(R) == 8 ? 32 : 256;
    multisect_kernel<R><<<(k_want * 32 + mt - 1) / mt, mt, 0, st>>>(dg, eabs, n, k_want, evals);
  }
  VB_CHECK_LAUNCH();
  return VB_OK;
}

template <class R>
vb_status eig_vectors(int n, const cplx<R> *rho, int k_want, int k_vec, const R *evals, cplx<R> *evecs,
                      void *work, cudaStream_t st, int rounds_in) {
  typedef cplx<R> C_;
  (void)rho;
  if (k_vec < 1 || k_vec > k_want) return fail(VB_EINVAL, "eig_vectors: bad k_vec");
  // the panelled Gram-Schmidt keeps p0 * b <= 128 * 16 coefficients (off_part)
  if (k_vec > 144) return fail(VB_EINVAL, "eig_vectors: at most 144 vectors");
  EigLayout lay(n, k_want, sizeof(R));
  char *w = static_cast<char *>(work);
  C_ *vref = reinterpret_cast<C_ *>(w + lay.off_vref);
  R *tau = reinterpret_cast<R *>(w + lay.off_tau);
  R *dg = reinterpret_cast<R *>(w + lay.off_dg);
  R *eabs = reinterpret_cast<R *>(w + lay.off_eabs);
  C_ *delta = reinterpret_cast<C_ *>(w + lay.off_delta);
  R *Y = reinterpret_cast<R *>(w + lay.off_y);
  R *lu = reinterpret_cast<R *>(w + lay.off_lu);
  int *piv = reinterpret_cast<int *>(lu + (size_t)k_want * n * 4);
  // FP32 vectors only seed an FP64 Rayleigh-Ritz step: two rounds suffice there
  const int rounds = rounds_in > 0 ? std::min(rounds_in, INVIT_ROUNDS) : (sizeof(R) == 8 ? INVIT_ROUNDS : 2);
  for (int r = 0; r < rounds; ++r) {
    prof_begin(PH_INVIT, st);
    invit_round<R><<<(k_vec + 31) / 32, 32, 0, st>>>(dg, eabs, n, k_vec, evals, Y, lu, piv, r);
    VB_CHECK_LAUNCH();
    prof_end(PH_INVIT, st, 0.0);
    prof_begin(PH_CGS, st);
    if (k_vec <= BGS_PANEL) {
      cgs2_rows<R><<<1, 512, 0, st>>>(Y, n, k_vec);
      VB_CHECK_LAUNCH();
    } else {
      R *C = reinterpret_cast<R *>(w + lay.off_part);  // 2048 reals; p0 * b <= 128 * 16 for k_vec <= 144
      for (int p0 = 0; p0 < k_vec; p0 += BGS_PANEL) {
        const int b = std::min(BGS_PANEL, k_vec - p0);
        if (p0 > 0) {
          for (int pass = 0; pass < 2; ++pass) {
            const int pairs = p0 * b;
            bgs_dots<R><<<(pairs * 32 + 255) / 256, 256, 0, st>>>(Y, n, p0, b, C);
            VB_CHECK_LAUNCH();
            const long long tot = (long long)b * n;
            bgs_update<R><<<(int)std::min<long long>((tot + 255) / 256, 152LL * 8), 256, 0, st>>>(Y, n, p0, b, C);
            VB_CHECK_LAUNCH();
          }
        }
        bgs_panel<R><<<1, 512, 0, st>>>(Y, n, p0, b);
        VB_CHECK_LAUNCH();
      }
    }
    prof_end(PH_CGS, st, 0.0);
  }
  prof_begin(PH_BACKT, st);
  backtransform<R><<<k_vec, 256, 0, st>>>(vref, tau, delta, Y, n, evecs);
  VB_CHECK_LAUNCH();
  prof_end(PH_BACKT, st, 0.0);
  return VB_OK;
}

template vb_status eig_values<double>(int, cd *, int, double *, void *, cudaStream_t);
template vb_status eig_values<float>(int, cf *, int, float *, void *, cudaStream_t);
template vb_status eig_vectors<double>(int, const cd *, int, int, const double *, cd *, void *, cudaStream_t, int);
template vb_status eig_vectors<float>(int, const cf *, int, int, const float *, cf *, void *, cudaStream_t, int);

}  // namespace vb

// ---------------------------------------------------------------------------
// Allocation-free variant of vb_herm_eig_top.
//
// Some callers cannot allocate device memory at the point where they need
// the split: a host framework that owns every byte of device memory through
// its own pool, or a latency-critical loop that must not pay for the
// device-wide synchronisation cudaMalloc implies. For them the eigensolver's
// workspace lives in a fixed file-scope device array instead of a caller
// buffer. The array is part of the library image, so every GPU that loads
// the library keeps it until the process exits.
namespace vb {
namespace {

constexpr int NOALLOC_MAX_N = 256;       // largest matrix dimension
constexpr int NOALLOC_MAX_KWANT = 128;   // largest number of eigenvalues
constexpr size_t NOALLOC_SCRATCH_BYTES = 3u << 20;  // 3 MiB

static __device__ __align__(256) unsigned char g_eig_scratch[NOALLOC_SCRATCH_BYTES];

// device address of g_eig_scratch, looked up once per device; atomic so that
// host threads making their first call on one device at the same time do not
// race (they look up and store the same address)
constexpr int NOALLOC_MAX_DEVICES = 64;
std::atomic<void *> g_scratch_addr[NOALLOC_MAX_DEVICES];

vb_status scratch_address(void **out) {
  int dev = -1;
  VB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(VB_EINVAL, "noalloc eig: device ordinal out of range");
  void *addr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!addr) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_eig_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(VB_ECUDA, std::string("noalloc eig: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    }
    g_scratch_addr[dev].store(p, std::memory_order_release);
    addr = p;
  }
  *out = addr;
  return VB_OK;
}

}  // namespace
}  // namespace vb

extern "C" vb_status vb_herm_eig_top_noalloc(int n, double *rho, int k_want, int k_vec, double *evals,
                                             double *evecs, void *stream) {
  using namespace vb;
  if (n < 1 || !rho || k_want < 1 || k_want > n || k_vec < 0 || k_vec > k_want || !evals ||
      (k_vec > 0 && !evecs))
    return fail(VB_EINVAL, "vb_herm_eig_top_noalloc: bad argument");
  if (n > NOALLOC_MAX_N || k_want > NOALLOC_MAX_KWANT)
    return fail(VB_EINVAL, "vb_herm_eig_top_noalloc: n must be <= " + std::to_string(NOALLOC_MAX_N) +
                               " and k_want <= " + std::to_string(NOALLOC_MAX_KWANT) +
                               " (fixed workspace); use vb_herm_eig_top with a caller buffer");
  if (EigWork::bytes(n, k_want) > NOALLOC_SCRATCH_BYTES)
    return fail(VB_EINVAL, "vb_herm_eig_top_noalloc: workspace exceeds the fixed scratch array");
  void *work = nullptr;
  VB_TRY(scratch_address(&work));
  // every workspace entry the solver reads is written earlier in the same
  // call, so nothing needs clearing between calls
  cudaStream_t st = (cudaStream_t)stream;
  VB_TRY(eig_values(n, (cd *)rho, k_want, evals, work, st));
  if (k_vec > 0) VB_TRY(eig_vectors(n, (cd *)rho, k_want, k_vec, evals, (cd *)evecs, work, st));
  // a grid barrier of the reduction that ran out leaves its error word in the
  // scratch array: report it before the next call clears it
  return EigWork::check(n, k_want, sizeof(double), work, st);
}

