// Krylov-space kernels of the local exponential (Eq. Krylov subspace):
// block inner products against all basis vectors, the matching update, norms,
// scaling, the final combination theta' = |theta| sum_k u_k v_k, and the
// exponential of the small tridiagonal Lanczos matrix. All in FP64 with
// deterministic (fixed-order) reductions.
#include "common.h"

namespace vb {
namespace {

constexpr int RT = 256;  // threads per reduction block

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of one double per thread; result valid in thread 0
__device__ double block_sum(double v, double *sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// partial[b * nv + j] = sum over block b's chunk of conj(V_j[i]) w[i].
// blockIdx.y picks a group of up to DOT_JB vectors; each thread keeps the
// group's partial sums in registers (independent FMA chains) and reads w[i]
// once per group. The group size is a template parameter, so a short last
// group issues no predicated-off FP64 instructions.
constexpr int DOT_JB = 8;
template <int JB>
__device__ __forceinline__ void dot_group(const cd *__restrict__ Vg, long long ldv, const cd *__restrict__ w,
                                          long long i0, long long i1, double *sh, double *out2) {
  double sx[JB], sy[JB];
#pragma unroll
  for (int j = 0; j < JB; ++j) sx[j] = sy[j] = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += RT) {
    const cd b = w[i];
#pragma unroll
    for (int j = 0; j < JB; ++j) {
      const cd a = Vg[j * ldv + i];
      sx[j] = fma(a.x, b.x, fma(a.y, b.y, sx[j]));
      sy[j] = fma(a.x, b.y, fma(-a.y, b.x, sy[j]));
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < JB; ++j) {
    const double rx = warp_sum(sx[j]), ry = warp_sum(sy[j]);
    if (lane == 0) {
      sh[wid * 2 * DOT_JB + 2 * j] = rx;
      sh[wid * 2 * DOT_JB + 2 * j + 1] = ry;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * JB) {
    double s = 0.0;
    for (int w2 = 0; w2 < RT / 32; ++w2) s += sh[w2 * 2 * DOT_JB + threadIdx.x];
    out2[threadIdx.x] = s;
  }
}

// With cnt != nullptr (one zeroed counter per vector group), the last block
// of a group to finish sums the group's partials over all blocks, in block
// order (the same order as reduce_parts_cd), writes out[j] and re-zeroes its
// counter: no separate reduction launch.
__global__ void __launch_bounds__(RT) multi_dot_part(const cd *__restrict__ V, long long ldv, int nv,
                                                     const cd *__restrict__ w, long long n,
                                                     cd *__restrict__ partial, unsigned int *cnt, cd *out) {
  __shared__ double sh[(RT / 32) * 2 * DOT_JB];
  __shared__ unsigned int s_ticket;
  const int j0 = blockIdx.y * DOT_JB;
  const int jn = min(DOT_JB, nv - j0);
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  const cd *Vg = V + j0 * ldv;
  double *out2 = reinterpret_cast<double *>(partial + (long long)blockIdx.x * nv + j0);
  switch (jn) {
    case 8: dot_group<8>(Vg, ldv, w, i0, i1, sh, out2); break;
    case 7: dot_group<7>(Vg, ldv, w, i0, i1, sh, out2); break;
    case 6: dot_group<6>(Vg, ldv, w, i0, i1, sh, out2); break;
    case 5: dot_group<5>(Vg, ldv, w, i0, i1, sh, out2); break;
    case 4: dot_group<4>(Vg, ldv, w, i0, i1, sh, out2); break;
    case 3: dot_group<3>(Vg, ldv, w, i0, i1, sh, out2); break;
    case 2: dot_group<2>(Vg, ldv, w, i0, i1, sh, out2); break;
    default: dot_group<1>(Vg, ldv, w, i0, i1, sh, out2); break;
  }
  if (!cnt) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(&cnt[blockIdx.y], 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = wid; j < jn; j += RT / 32) {
    double sx = 0.0, sy = 0.0;
#pragma unroll 4
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const double2 p = __ldcg(reinterpret_cast<const double2 *>(partial + (long long)b * nv + j0 + j));
      sx += p.x;
      sy += p.y;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) out[j0 + j] = mkc(sx, sy);
  }
  if (threadIdx.x == 0) cnt[blockIdx.y] = 0u;
}

__global__ void reduce_parts_cd(const cd *__restrict__ partial, int n_part, int nv, cd *out) {
  // one warp per output j
  int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (j >= nv) return;
  double sx = 0.0, sy = 0.0;
  for (int b = lane; b < n_part; b += 32) {
    cd p = partial[(long long)b * nv + j];
    sx += p.x;
    sy += p.y;
  }
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  if (lane == 0) out[j] = mkc(sx, sy);
}

// w[i] += sign * sum_j c[j] V_j[i], two elements per thread (four
// independent FMA chains). With partial != nullptr each block also writes
// the sum of |w_new[i]|^2 over its elements to partial[blockIdx.x].
// With w32 != nullptr the kernel also writes the FP32 copy of w_new.
__global__ void __launch_bounds__(256) multi_axpy_kernel(const cd *__restrict__ V, long long ldv, int nv,
                                                         const cd *__restrict__ c, double sign, cd *__restrict__ w,
                                                         long long n, double *__restrict__ partial,
                                                         unsigned int *cnt, double *nrm_out, cf *__restrict__ w32) {
  __shared__ cd cs[128];
  __shared__ double sh[8];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) cs[j] = cscale(c[j], sign);
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  double nn = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
    const long long i2 = i + stride;
    const bool two = i2 < n;
    double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
    for (int j = 0; j < nv; ++j) {
      const cd cj = cs[j];
      const cd v = V[j * ldv + i];
      ax = fma(cj.x, v.x, fma(-cj.y, v.y, ax));
      ay = fma(cj.x, v.y, fma(cj.y, v.x, ay));
      if (two) {
        const cd u = V[j * ldv + i2];
        bx = fma(cj.x, u.x, fma(-cj.y, u.y, bx));
        by = fma(cj.x, u.y, fma(cj.y, u.x, by));
      }
    }
    const cd o = w[i];
    const cd r = mkc(o.x + ax, o.y + ay);
    w[i] = r;
    if (w32) w32[i] = mkc((float)r.x, (float)r.y);
    if (partial) nn = fma(r.x, r.x, fma(r.y, r.y, nn));
    if (two) {
      const cd o2 = w[i2];
      const cd r2 = mkc(o2.x + bx, o2.y + by);
      w[i2] = r2;
      if (w32) w32[i2] = mkc((float)r2.x, (float)r2.y);
      if (partial) nn = fma(r2.x, r2.x, fma(r2.y, r2.y, nn));
    }
  }
  if (partial) {
    nn = warp_sum(nn);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = nn;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) s += sh[w2];
      partial[blockIdx.x] = s;
    }
    if (cnt) {
      // the last block sums the block partials in block order (as
      // norm2_final does) and writes |w|
      __shared__ unsigned int s_ticket;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_ticket = atomicAdd(cnt, 1u);
      __syncthreads();
      if (s_ticket == gridDim.x - 1 && threadIdx.x < 32) {
        __threadfence();
        double s = 0.0;
#pragma unroll 4
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += __ldcg(partial + b);
        s = warp_sum(s);
        if (threadIdx.x == 0) {
          nrm_out[0] = sqrt(s);
          cnt[0] = 0u;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(RT) norm2_part(const cd *__restrict__ x, long long n,
                                                 double *__restrict__ partial) {
  __shared__ double sh[RT / 32];
  long long chunk = (n + gridDim.x - 1) / gridDim.x;
  long long i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += RT) {
    cd a = x[i];
    s = fma(a.x, a.x, fma(a.y, a.y, s));
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void norm2_final(const double *__restrict__ partial, int n_part, double *out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < n_part; b += 32) s += partial[b];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[0] = sqrt(s);
}

__global__ void scale_inv_kernel(cd *x, long long n, const double *nrm, double *keep, const cd *c, const cd *c2,
                                 double *alpha_k, cf *shadow) {
  // a zero norm (Lanczos breakdown, zero input) gives a zero vector
  const double s = nrm[0] > 0.0 ? 1.0 / nrm[0] : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (keep) keep[0] = nrm[0];
    if (alpha_k) alpha_k[0] = c[0].x + c2[0].x;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cd a = x[i];
    const cd r = mkc(a.x * s, a.y * s);
    x[i] = r;
    if (shadow) shadow[i] = mkc((float)r.x, (float)r.y);
  }
}

// ---- the Gram-Schmidt passes of the mixed form on FP32 copies of the
// Krylov vectors. w = H v_k comes from the FP32 tensor-core product and is
// itself only FP32-accurate, so its inner products need no more: products and
// per-thread sums in FP32, the block and final sums in FP64, and the
// correction sum_j c_j v_j formed in FP32 and added to the FP64 vector. Half
// the bytes of the FP64 passes, no FP64 arithmetic beyond the sums and the
// norm. w is read either as its FP32 copy or as the FP64 vector rounded on
// load (as_cf), from global or shared memory (index i - woff).
__device__ __forceinline__ cf as_cf(const cf &v) { return v; }
__device__ __forceinline__ cf as_cf(const cd &v) { return mkc((float)v.x, (float)v.y); }

template <int JB, typename WT>
__device__ __forceinline__ void dot32_group(const cf *__restrict__ Vg, long long ldv, const WT *__restrict__ w,
                                            long long woff, long long i0, long long i1, double *sh,
                                            double *out2) {
  float sx[JB], sy[JB];
#pragma unroll
  for (int j = 0; j < JB; ++j) sx[j] = sy[j] = 0.f;
  // two elements per iteration with all their loads issued before the
  // products (more bytes in flight); the accumulation order is unchanged
  long long i = i0 + threadIdx.x;
  for (; i + RT < i1; i += 2 * RT) {
    const cf b0 = as_cf(w[i - woff]), b1 = as_cf(w[i + RT - woff]);
    cf a0[JB], a1[JB];
#pragma unroll
    for (int j = 0; j < JB; ++j) {
      a0[j] = Vg[j * ldv + i];
      a1[j] = Vg[j * ldv + i + RT];
    }
#pragma unroll
    for (int j = 0; j < JB; ++j) {
      sx[j] = fmaf(a0[j].x, b0.x, fmaf(a0[j].y, b0.y, sx[j]));
      sy[j] = fmaf(a0[j].x, b0.y, fmaf(-a0[j].y, b0.x, sy[j]));
      sx[j] = fmaf(a1[j].x, b1.x, fmaf(a1[j].y, b1.y, sx[j]));
      sy[j] = fmaf(a1[j].x, b1.y, fmaf(-a1[j].y, b1.x, sy[j]));
    }
  }
  if (i < i1) {
    const cf b = as_cf(w[i - woff]);
#pragma unroll
    for (int j = 0; j < JB; ++j) {
      const cf a = Vg[j * ldv + i];
      sx[j] = fmaf(a.x, b.x, fmaf(a.y, b.y, sx[j]));
      sy[j] = fmaf(a.x, b.y, fmaf(-a.y, b.x, sy[j]));
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < JB; ++j) {
    const double rx = warp_sum((double)sx[j]), ry = warp_sum((double)sy[j]);
    if (lane == 0) {
      sh[wid * 2 * DOT_JB + 2 * j] = rx;
      sh[wid * 2 * DOT_JB + 2 * j + 1] = ry;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * JB) {
    double s = 0.0;
    for (int w2 = 0; w2 < RT / 32; ++w2) s += sh[w2 * 2 * DOT_JB + threadIdx.x];
    out2[threadIdx.x] = s;
  }
}

template <typename WT>
__device__ __forceinline__ void dot32_any(int jn, const cf *Vg, long long ldv, const WT *w, long long woff,
                                          long long i0, long long i1, double *sh, double *out2) {
  switch (jn) {
    case 8: dot32_group<8>(Vg, ldv, w, woff, i0, i1, sh, out2); break;
    case 7: dot32_group<7>(Vg, ldv, w, woff, i0, i1, sh, out2); break;
    case 6: dot32_group<6>(Vg, ldv, w, woff, i0, i1, sh, out2); break;
    case 5: dot32_group<5>(Vg, ldv, w, woff, i0, i1, sh, out2); break;
    case 4: dot32_group<4>(Vg, ldv, w, woff, i0, i1, sh, out2); break;
    case 3: dot32_group<3>(Vg, ldv, w, woff, i0, i1, sh, out2); break;
    case 2: dot32_group<2>(Vg, ldv, w, woff, i0, i1, sh, out2); break;
    default: dot32_group<1>(Vg, ldv, w, woff, i0, i1, sh, out2); break;
  }
}

// out[j] = vs[j] <V_j, w> (vs nullable: 1) for the group of blockIdx.y, the
// partial sums over each block's chunk of w summed by the group's last block
template <typename WT>
__global__ void __launch_bounds__(RT) multi_dot32_part(const cf *__restrict__ V, long long ldv, int nv,
                                                       const WT *__restrict__ w, long long n,
                                                       cd *__restrict__ partial, unsigned int *cnt, cd *out,
                                                       const double *__restrict__ vs) {
  __shared__ double sh[(RT / 32) * 2 * DOT_JB];
  __shared__ unsigned int s_ticket;
  const int j0 = blockIdx.y * DOT_JB;
  const int jn = min(DOT_JB, nv - j0);
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  const cf *Vg = V + j0 * ldv;
  double *out2 = reinterpret_cast<double *>(partial + (long long)blockIdx.x * nv + j0);
  dot32_any(jn, Vg, ldv, w, 0, i0, i1, sh, out2);
  // the last block of the group sums the partials in block order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(&cnt[blockIdx.y], 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = wid; j < jn; j += RT / 32) {
    double sx = 0.0, sy = 0.0;
#pragma unroll 4
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const double2 p = __ldcg(reinterpret_cast<const double2 *>(partial + (long long)b * nv + j0 + j));
      sx += p.x;
      sy += p.y;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) {
      const double f = vs ? vs[j0 + j] : 1.0;
      out[j0 + j] = mkc(sx * f, sy * f);
    }
  }
  if (threadIdx.x == 0) cnt[blockIdx.y] = 0u;
}

// The first pass's update fused with the full pass's inner products (one
// read of the data instead of two): each block takes one chunk of w,
// w <- w + sign * sum_{j<n1} c1_j V1_j (FP32 correction, FP64 w, as in
// multi_axpy32_norm_kernel), keeps the FP32 copy of the new w in shared
// memory, then forms partial[b * nv + j] = <V_j, w32> over its chunk for all
// nv vectors in groups of DOT_JB (as multi_dot32_part); the last block sums
// the partials in block order. vs1 / vs (nullable): factors of the stored
// copies V1 / V (coefficients and inner products are those of the normalised
// vectors). Dynamic shared memory: chunk FP32 elements.
__global__ void __launch_bounds__(RT, 4) axpy_dot32_kernel(const cf *__restrict__ V1, int n1,
                                                        const cd *__restrict__ c1, double sign,
                                                        cd *__restrict__ w, long long n, const cf *__restrict__ V,
                                                        long long ldv, int nv, cd *__restrict__ partial,
                                                        unsigned int *cnt, cd *out, const double *__restrict__ vs1,
                                                        const double *__restrict__ vs) {
  extern __shared__ __align__(16) unsigned char adsm[];
  cf *ws = reinterpret_cast<cf *>(adsm);
  __shared__ double sh[(RT / 32) * 2 * DOT_JB];
  __shared__ cf cs[2];
  __shared__ unsigned int s_ticket;
  if (threadIdx.x < n1) {
    const double f = sign * (vs1 ? vs1[threadIdx.x] : 1.0);
    cs[threadIdx.x] = mkc((float)(f * c1[threadIdx.x].x), (float)(f * c1[threadIdx.x].y));
  }
  __syncthreads();
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  for (long long i = i0 + threadIdx.x; i < i1; i += 2 * RT) {
    const long long i2 = i + RT;
    const bool two = i2 < i1;
    const cd o = w[i];
    const cd o2 = two ? w[i2] : mkc(0.0, 0.0);
    float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
    for (int j = 0; j < n1; ++j) {
      const cf cj = cs[j];
      const cf v = V1[j * ldv + i];
      const cf u = two ? V1[j * ldv + i2] : mkc(0.f, 0.f);
      ax = fmaf(cj.x, v.x, fmaf(-cj.y, v.y, ax));
      ay = fmaf(cj.x, v.y, fmaf(cj.y, v.x, ay));
      bx = fmaf(cj.x, u.x, fmaf(-cj.y, u.y, bx));
      by = fmaf(cj.x, u.y, fmaf(cj.y, u.x, by));
    }
    const cd r = mkc(o.x + (double)ax, o.y + (double)ay);
    w[i] = r;
    ws[i - i0] = mkc((float)r.x, (float)r.y);
    if (two) {
      const cd r2 = mkc(o2.x + (double)bx, o2.y + (double)by);
      w[i2] = r2;
      ws[i2 - i0] = mkc((float)r2.x, (float)r2.y);
    }
  }
  __syncthreads();
  for (int j0 = 0; j0 < nv; j0 += DOT_JB) {
    double *out2 = reinterpret_cast<double *>(partial + (long long)blockIdx.x * nv + j0);
    dot32_any(min(DOT_JB, nv - j0), V + j0 * ldv, ldv, ws, i0, i0, i1, sh, out2);
    __syncthreads();  // sh is reused by the next group
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(cnt, 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = wid; j < nv; j += RT / 32) {
    double sx = 0.0, sy = 0.0;
#pragma unroll 4
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const double2 p = __ldcg(reinterpret_cast<const double2 *>(partial + (long long)b * nv + j));
      sx += p.x;
      sy += p.y;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) {
      const double f = vs ? vs[j] : 1.0;
      out[j] = mkc(sx * f, sy * f);
    }
  }
  if (threadIdx.x == 0) cnt[0] = 0u;
}

// w[i] += sign * sum_j c[j] vs[j] V32_j[i] (correction in FP32, w in FP64;
// vs nullable: 1); with w32 != nullptr the FP32 copy of the new w is written
// too; with partial != nullptr |w| in FP64 by the last block (cnt: one zeroed
// counter), which also writes the Lanczos record (1/|w|, |w|, alpha_k)
__global__ void __launch_bounds__(256) multi_axpy32_norm_kernel(const cf *__restrict__ V, long long ldv, int nv,
                                                                const cd *__restrict__ c, double sign,
                                                                cd *__restrict__ w, long long n,
                                                                double *__restrict__ partial, unsigned int *cnt,
                                                                double *nrm_out, cf *__restrict__ w32,
                                                                const double *__restrict__ vs, LanczosRecord rec) {
  __shared__ cf cs[128];
  __shared__ double sh[8];
  __shared__ unsigned int s_ticket;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    const double f = sign * (vs ? vs[j] : 1.0);
    cs[j] = mkc((float)(f * c[j].x), (float)(f * c[j].y));
  }
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  double nn = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
    const long long i2 = i + stride;
    const bool two = i2 < n;
    float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
    for (int j = 0; j < nv; ++j) {
      const cf cj = cs[j];
      const cf v = V[j * ldv + i];
      ax = fmaf(cj.x, v.x, fmaf(-cj.y, v.y, ax));
      ay = fmaf(cj.x, v.y, fmaf(cj.y, v.x, ay));
      if (two) {
        const cf u = V[j * ldv + i2];
        bx = fmaf(cj.x, u.x, fmaf(-cj.y, u.y, bx));
        by = fmaf(cj.x, u.y, fmaf(cj.y, u.x, by));
      }
    }
    const cd o = w[i];
    const cd r = mkc(o.x + (double)ax, o.y + (double)ay);
    w[i] = r;
    if (w32) w32[i] = mkc((float)r.x, (float)r.y);
    nn = fma(r.x, r.x, fma(r.y, r.y, nn));
    if (two) {
      const cd o2 = w[i2];
      const cd r2 = mkc(o2.x + (double)bx, o2.y + (double)by);
      w[i2] = r2;
      if (w32) w32[i2] = mkc((float)r2.x, (float)r2.y);
      nn = fma(r2.x, r2.x, fma(r2.y, r2.y, nn));
    }
  }
  if (!partial) return;
  nn = warp_sum(nn);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = nn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += sh[w2];
    partial[blockIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(cnt, 1u);
  __syncthreads();
  if (s_ticket == gridDim.x - 1 && threadIdx.x < 32) {
    __threadfence();
    double t = 0.0;
#pragma unroll 4
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) t += __ldcg(partial + b);
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      const double nr = sqrt(t);
      nrm_out[0] = nr;
      if (rec.vs_next) rec.vs_next[0] = nr > 0.0 ? 1.0 / nr : 0.0;
      if (rec.beta_k) rec.beta_k[0] = nr;
      if (rec.alpha_k) rec.alpha_k[0] = rec.ck[0].x + rec.c2k[0].x;
      cnt[0] = 0u;
    }
  }
}

__global__ void copy_kernel(const cd *x, cd *y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i];
}

__global__ void combine_kernel(const cd *__restrict__ V, long long ldv, int nv,
                               const cd *__restrict__ u, const double *nrm, cd *__restrict__ y,
                               long long n, const double *__restrict__ vs) {
  __shared__ cd cs[128];
  double s = nrm[0];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) cs[j] = cscale(u[j], vs ? s * vs[j] : s);
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double ax = 0.0, ay = 0.0;
    for (int j = 0; j < nv; ++j) {
      cd v = V[j * ldv + i];
      ax = fma(cs[j].x, v.x, fma(-cs[j].y, v.y, ax));
      ay = fma(cs[j].x, v.y, fma(cs[j].y, v.x, ay));
    }
    y[i] = mkc(ax, ay);
  }
}

// ---------------------------------------------------------------------------
// u = exp(-i T tau) e_1 for the symmetric tridiagonal Lanczos matrix T
// (alpha on the diagonal, beta off it), kdim <= 64, one warp; row r lives in
// lane r % 32, slot r / 32. Chebyshev expansion (Jacobi-Anger identity):
// with T's Gershgorin interval [mu - D, mu + D] and H = (T - mu) / D,
//   exp(-i z H) = J_0(z) + 2 sum_{n >= 1} (-i)^n J_n(z) T_n(H),   z = D tau,
// T_n(H) v from the three-term recurrence v_{n+1} = 2 H v_n - v_{n-1}, and
// exp(-i T tau) = exp(-i mu tau) exp(-i z H). The Bessel values come from
// Miller's backward recurrence normalised by J_0 + 2 sum_k J_2k = 1; terms
// stop at the last n > |z| with |J_n(z)| >= 1e-18 (at most |z| + 30; J_n
// falls super-exponentially beyond |z|); larger |z| is cut into substeps of
// |z| <= 40. With c != nullptr the kernel first sets the newest diagonal
// entry alpha[kdim - 1] = Re c[kdim - 1] + Re c2[kdim - 1]. Writes
// out[0] = bnext |u_{kdim-1}| (the Lanczos error estimate), out[1] = bnext.
constexpr int TRI_ZMAX = 40;                 // largest |z| per substep
constexpr int TRI_NMAX = TRI_ZMAX + 30;      // terms per substep
constexpr int TRI_MILLER = TRI_NMAX + 40;    // start of the backward recurrence (even)

__device__ __forceinline__ void tri_matvec(const double *d, const double *bl, const double *br, const cd *v, cd *w,
                                           int lane) {
  // neighbours row - 1 and row + 1 of both slots
  double u0x = __shfl_up_sync(0xffffffffu, v[0].x, 1), u0y = __shfl_up_sync(0xffffffffu, v[0].y, 1);
  double u1x = __shfl_up_sync(0xffffffffu, v[1].x, 1), u1y = __shfl_up_sync(0xffffffffu, v[1].y, 1);
  const double c0x = __shfl_sync(0xffffffffu, v[0].x, 31), c0y = __shfl_sync(0xffffffffu, v[0].y, 31);
  double d0x = __shfl_down_sync(0xffffffffu, v[0].x, 1), d0y = __shfl_down_sync(0xffffffffu, v[0].y, 1);
  double d1x = __shfl_down_sync(0xffffffffu, v[1].x, 1), d1y = __shfl_down_sync(0xffffffffu, v[1].y, 1);
  const double c1x = __shfl_sync(0xffffffffu, v[1].x, 0), c1y = __shfl_sync(0xffffffffu, v[1].y, 0);
  if (lane == 0) {
    u0x = u0y = 0.0;
    u1x = c0x;
    u1y = c0y;
  }
  if (lane == 31) {
    d0x = c1x;
    d0y = c1y;
    d1x = d1y = 0.0;
  }
  w[0] = mkc(d[0] * v[0].x + bl[0] * u0x + br[0] * d0x, d[0] * v[0].y + bl[0] * u0y + br[0] * d0y);
  w[1] = mkc(d[1] * v[1].x + bl[1] * u1x + br[1] * d1x, d[1] * v[1].y + bl[1] * u1y + br[1] * d1y);
}

// real vectors (ns row slots in use)
__device__ __forceinline__ void tri_matvec_r(int ns, const double *d, const double *bl, const double *br,
                                             const double *v, double *w, int lane) {
  double u0 = __shfl_up_sync(0xffffffffu, v[0], 1), dn0 = __shfl_down_sync(0xffffffffu, v[0], 1);
  if (ns == 1) {
    if (lane == 0) u0 = 0.0;
    if (lane == 31) dn0 = 0.0;
    w[0] = d[0] * v[0] + bl[0] * u0 + br[0] * dn0;
    w[1] = 0.0;
    return;
  }
  double u1 = __shfl_up_sync(0xffffffffu, v[1], 1), dn1 = __shfl_down_sync(0xffffffffu, v[1], 1);
  const double c0 = __shfl_sync(0xffffffffu, v[0], 31), c1 = __shfl_sync(0xffffffffu, v[1], 0);
  if (lane == 0) {
    u0 = 0.0;
    u1 = c0;
  }
  if (lane == 31) {
    dn0 = c1;
    dn1 = 0.0;
  }
  w[0] = d[0] * v[0] + bl[0] * u0 + br[0] * dn0;
  w[1] = d[1] * v[1] + bl[1] * u1 + br[1] * dn1;
}

// one-slot form (kdim <= 32)
__device__ __forceinline__ void tri_matvec1(double d, double bl, double br, cd v, cd &w, int lane) {
  double ux = __shfl_up_sync(0xffffffffu, v.x, 1), uy = __shfl_up_sync(0xffffffffu, v.y, 1);
  double dx = __shfl_down_sync(0xffffffffu, v.x, 1), dy = __shfl_down_sync(0xffffffffu, v.y, 1);
  if (lane == 0) ux = uy = 0.0;
  if (lane == 31) dx = dy = 0.0;
  w = mkc(d * v.x + bl * ux + br * dx, d * v.y + bl * uy + br * dy);
}

__global__ void tridiag_expm_kernel(const cd *c, const cd *c2, double *alpha, const double *__restrict__ beta,
                                    int kdim, double tau, const double *bnext, cd *u, double *out) {
  __shared__ double jn[TRI_NMAX + 1];
  __shared__ int s_nt;
  const int lane = threadIdx.x;
  // the newest diagonal entry: sum of the two Gram-Schmidt passes' <v_k, H v_k>
  if (c && lane == 0) alpha[kdim - 1] = c[kdim - 1].x + c2[kdim - 1].x;
  __syncwarp();
  double lo = 1e300, hi = -1e300;
  for (int r = lane; r < kdim; r += 32) {
    const double rad = (r > 0 ? fabs(beta[r - 1]) : 0.0) + (r + 1 < kdim ? fabs(beta[r]) : 0.0);
    lo = fmin(lo, alpha[r] - rad);
    hi = fmax(hi, alpha[r] + rad);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const double mu = 0.5 * (lo + hi);
  const double D = 0.5 * (hi - lo);
  const double ztot = D * fabs(tau);
  int steps = (int)ceil(ztot / TRI_ZMAX);
  if (steps < 1) steps = 1;
  const double ts = tau / steps;
  const double z = D * fabs(ts);
  // Bessel values J_n(z), n <= nt (lane 0)
  const int nt = z > 0.0 ? min(TRI_NMAX, (int)ceil(z) + 30) : 0;
  if (lane == 0) {
    for (int n = 0; n <= TRI_NMAX; ++n) jn[n] = 0.0;
    if (z > 0.0) {
      double fp = 0.0, f = 1e-280, norm = 0.0;  // f_{n+1}, f_n
      const double tz = 2.0 / z;
      for (int n = min(TRI_MILLER, nt + 40) & ~1; n >= 0; --n) {
        if (n <= nt) jn[n] = f;
        if (n % 2 == 0) norm += (n == 0 ? 1.0 : 2.0) * f;
        if (n > 0) {
          const double fm = (n * tz) * f - fp;
          fp = f;
          f = fm;
        }
        if (fabs(f) > 1e250) {  // rescale everything computed so far
          f *= 1e-250;
          fp *= 1e-250;
          norm *= 1e-250;
          for (int q = n; q <= nt; ++q) jn[q] *= 1e-250;
        }
      }
      const double s = 1.0 / norm;
      for (int n = 0; n <= nt; ++n) jn[n] *= s;
      // last term needed: beyond z the values fall super-exponentially
      int last = nt;
      while (last > 1 && last > z + 1.0 && fabs(jn[last]) < 1e-18) --last;
      s_nt = last;
    } else {
      jn[0] = 1.0;
      s_nt = 0;
    }
  }
  __syncwarp();
  const int nu = s_nt;
  // H = (T - mu) / D for this lane's rows; the zero rows beyond kdim stay zero
  double d[2], bl[2], br[2];
  const double inv = D > 0.0 ? 1.0 / D : 0.0;
  for (int sl = 0; sl < 2; ++sl) {
    const int r = lane + 32 * sl;
    const bool ok = r < kdim;
    d[sl] = ok ? (alpha[r] - mu) * inv : 0.0;
    bl[sl] = (ok && r > 0) ? beta[r - 1] * inv : 0.0;
    br[sl] = (ok && r + 1 < kdim) ? beta[r] * inv : 0.0;
  }
  // (-i)^n for ts >= 0, (+i)^n for ts < 0 (J_n(-z) = (-1)^n J_n(z))
  const double sg = ts >= 0.0 ? -1.0 : 1.0;
  double ps, pc;
  sincos(-mu * ts, &ps, &pc);
  cd x[2] = {mkc(lane == 0 ? 1.0 : 0.0, 0.0), mkc(0.0, 0.0)};
  const int ns = kdim > 32 ? 2 : 1;  // row slots in use
  if (steps == 1) {
    // from e_1 every T_n(H) e_1 is real and every coefficient is real or
    // imaginary, so one real recurrence and one real update per term
    double r0[2] = {lane == 0 ? 1.0 : 0.0, 0.0}, r1[2], r2[2];
    double ar[2], ai[2];
    tri_matvec_r(ns, d, bl, br, r0, r1, lane);
    for (int sl = 0; sl < 2; ++sl) {
      ar[sl] = jn[0] * r0[sl];
      ai[sl] = 2.0 * jn[1] * sg * r1[sl];
    }
    for (int n = 2; n <= nu; ++n) {
      tri_matvec_r(ns, d, bl, br, r1, r2, lane);
      const double cj = 2.0 * jn[n];
      const int m = n & 3;
      const double cr = m == 0 ? cj : (m == 2 ? -cj : 0.0);
      const double ci = m == 1 ? cj * sg : (m == 3 ? -cj * sg : 0.0);
      for (int sl = 0; sl < ns; ++sl) {
        r2[sl] = 2.0 * r2[sl] - r0[sl];
        if (m & 1)
          ai[sl] = fma(ci, r2[sl], ai[sl]);
        else
          ar[sl] = fma(cr, r2[sl], ar[sl]);
        r0[sl] = r1[sl];
        r1[sl] = r2[sl];
      }
    }
    for (int sl = 0; sl < 2; ++sl) x[sl] = mkc(pc * ar[sl] - ps * ai[sl], pc * ai[sl] + ps * ar[sl]);
  }
  for (int st = 0; st < (steps == 1 ? 0 : steps); ++st) {
    cd v0[2] = {x[0], x[1]}, v1[2], acc[2];
    if (ns == 2)
      tri_matvec(d, bl, br, v0, v1, lane);
    else
      tri_matvec1(d[0], bl[0], br[0], v0[0], v1[0], lane), v1[1] = mkc(0.0, 0.0);
    // n = 0 and n = 1 terms: J_0 v0 + 2 (sg i) J_1 v1
    const double j0 = jn[0], j1 = 2.0 * jn[1] * sg;
    for (int sl = 0; sl < 2; ++sl)
      acc[sl] = mkc(j0 * v0[sl].x - j1 * v1[sl].y, j0 * v0[sl].y + j1 * v1[sl].x);
    for (int n = 2; n <= nu; ++n) {
      cd v2[2];
      if (ns == 2)
        tri_matvec(d, bl, br, v1, v2, lane);
      else
        tri_matvec1(d[0], bl[0], br[0], v1[0], v2[0], lane), v2[1] = mkc(0.0, 0.0);
      // c_n = 2 (sg i)^n J_n: n % 4 = 0 -> 2J, 1 -> 2 sg i J, 2 -> -2J, 3 -> -2 sg i J
      const double cj = 2.0 * jn[n];
      const int m = n & 3;
      for (int sl = 0; sl < ns; ++sl) {
        v2[sl] = mkc(2.0 * v2[sl].x - v0[sl].x, 2.0 * v2[sl].y - v0[sl].y);
        if (m == 0)
          acc[sl] = mkc(acc[sl].x + cj * v2[sl].x, acc[sl].y + cj * v2[sl].y);
        else if (m == 2)
          acc[sl] = mkc(acc[sl].x - cj * v2[sl].x, acc[sl].y - cj * v2[sl].y);
        else {
          const double c = (m == 1 ? cj : -cj) * sg;  // times i
          acc[sl] = mkc(acc[sl].x - c * v2[sl].y, acc[sl].y + c * v2[sl].x);
        }
        v0[sl] = v1[sl];
        v1[sl] = v2[sl];
      }
    }
    for (int sl = 0; sl < 2; ++sl) x[sl] = mkc(pc * acc[sl].x - ps * acc[sl].y, pc * acc[sl].y + ps * acc[sl].x);
  }
  for (int sl = 0; sl < 2; ++sl) {
    const int r = lane + 32 * sl;
    if (r < kdim) u[r] = x[sl];
  }
  __syncwarp();
  if (lane == 0) {
    const cd last = u[kdim - 1];
    out[0] = bnext[0] * sqrt(cabs2(last));
    out[1] = bnext[0];
  }
}

inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

int reduce_parts(long long n) {
  long long p = (n + 4095) / 4096;
  if (p > 304) p = 304;
  if (p < 1) p = 1;
  return (int)p;
}

vb_status vec_multi_dot(const cd *V, long long ldv, int nv, const cd *w, long long n, cd *out,
                        cd *partial, int n_part, cudaStream_t st, unsigned int *cnt) {
  if (nv <= 0) return VB_OK;
  if (nv > 128 || (long long)n_part * nv > 512LL * 128) return fail(VB_EINVAL, "multi_dot: too many vectors");
  multi_dot_part<<<dim3(n_part, (nv + DOT_JB - 1) / DOT_JB), RT, 0, st>>>(V, ldv, nv, w, n, partial, cnt, out);
  VB_CHECK_LAUNCH();
  if (!cnt) {
    reduce_parts_cd<<<(nv + 7) / 8, 256, 0, st>>>(partial, n_part, nv, out);
    VB_CHECK_LAUNCH();
  }
  return VB_OK;
}

vb_status vec_multi_axpy(const cd *V, long long ldv, int nv, const cd *c, double sign, cd *w,
                         long long n, cudaStream_t st, cf *w32) {
  if (nv <= 0 || n == 0) return VB_OK;
  if (nv > 128) return fail(VB_EINVAL, "multi_axpy: more than 128 vectors");
  multi_axpy_kernel<<<grid_for((n + 1) / 2, 256), 256, 0, st>>>(V, ldv, nv, c, sign, w, n, nullptr, nullptr,
                                                                 nullptr, w32);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

template <typename WT>
static vb_status multi_dot32_launch(const cf *V, long long ldv, int nv, const WT *w, long long n, cd *out,
                                    cd *partial, int n_part, cudaStream_t st, unsigned int *cnt,
                                    const double *vs) {
  if (nv <= 0) return VB_OK;
  if (nv > 128 || n_part < 1 || (long long)n_part * nv > 512LL * 128 || !cnt)
    return fail(VB_EINVAL, "multi_dot32: too many vectors or no counters");
  multi_dot32_part<WT><<<dim3(n_part, (nv + DOT_JB - 1) / DOT_JB), RT, 0, st>>>(V, ldv, nv, w, n, partial, cnt,
                                                                                out, vs);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status vec_multi_dot32(const cf *V, long long ldv, int nv, const cf *w, long long n, cd *out, cd *partial,
                          int n_part, cudaStream_t st, unsigned int *cnt, const double *vs) {
  return multi_dot32_launch(V, ldv, nv, w, n, out, partial, n_part, st, cnt, vs);
}

vb_status vec_multi_dot32(const cf *V, long long ldv, int nv, const cd *w, long long n, cd *out, cd *partial,
                          int n_part, cudaStream_t st, unsigned int *cnt, const double *vs) {
  return multi_dot32_launch(V, ldv, nv, w, n, out, partial, n_part, st, cnt, vs);
}

int axpy_dot32_blocks(long long n, int nv, long long partial_elems) {
  if (n <= 0 || nv <= 0 || nv > 128) return 0;
  // AXPY_DOT_CHUNK elements per block on large vectors; on smaller ones at
  // least four blocks per SM while a block still gets 1024 elements
  const long long nb = std::min<long long>(
      AXPY_DOT_MAX_BLOCKS, std::max<long long>((n + AXPY_DOT_CHUNK - 1) / AXPY_DOT_CHUNK,
                                               std::min<long long>((n + 1023) / 1024, 4 * 152)));
  if ((n + nb - 1) / nb > AXPY_DOT_MAX_CHUNK || nb * nv > partial_elems) return 0;
  return (int)nb;
}

vb_status vec_axpy_dot32(const cf *V1, int n1, const cd *c1, double sign, cd *w, long long n, const cf *V,
                         long long ldv, int nv, cd *out, cd *partial, long long partial_elems, cudaStream_t st,
                         unsigned int *cnt, const double *vs1, const double *vs) {
  const int nb = axpy_dot32_blocks(n, nv, partial_elems);
  if (!nb || n1 < 1 || n1 > 2 || !cnt) return fail(VB_EINVAL, "axpy_dot32: sizes out of range");
  // the attribute is per device; setting it twice from two threads is harmless
  static std::atomic<bool> attr_set[64];
  int dev = 0;
  VB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(VB_EINVAL, "axpy_dot32: device ordinal out of range");
  if (!attr_set[dev].load()) {
    VB_TRY_CUDA(cudaFuncSetAttribute(axpy_dot32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(AXPY_DOT_MAX_CHUNK * sizeof(cf))));
    attr_set[dev].store(true);
  }
  const long long chunk = (n + nb - 1) / nb;
  axpy_dot32_kernel<<<nb, RT, (size_t)chunk * sizeof(cf), st>>>(V1, n1, c1, sign, w, n, V, ldv, nv, partial, cnt,
                                                                out, vs1, vs);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status vec_multi_axpy32_norm(const cf *V, long long ldv, int nv, const cd *c, double sign, cd *w, long long n,
                                double *out, double *partial, cudaStream_t st, unsigned int *cnt,
                                const double *vs, cf *w32, const LanczosRecord &rec) {
  if (nv > 128 || nv <= 0 || n <= 0 || !cnt)
    return fail(VB_EINVAL, "multi_axpy32: 1..128 vectors, a nonempty w and a counter needed");
  const int blocks = (int)std::min<long long>(512, std::max<long long>(1, (n + 511) / 512));
  multi_axpy32_norm_kernel<<<blocks, 256, 0, st>>>(V, ldv, nv, c, sign, w, n, partial, cnt, out, w32, vs, rec);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status vec_multi_axpy32(const cf *V, long long ldv, int nv, const cd *c, double sign, cd *w, long long n,
                           cf *w32, cudaStream_t st, const double *vs) {
  if (nv > 128) return fail(VB_EINVAL, "multi_axpy32: more than 128 vectors");
  if (nv <= 0 || n == 0) return VB_OK;
  const int blocks = (int)std::min<long long>(152LL * 8, std::max<long long>(1, (n + 511) / 512));
  multi_axpy32_norm_kernel<<<blocks, 256, 0, st>>>(V, ldv, nv, c, sign, w, n, nullptr, nullptr, nullptr, w32, vs,
                                                   LanczosRecord{});
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status vec_multi_axpy_norm(const cd *V, long long ldv, int nv, const cd *c, double sign, cd *w, long long n,
                              double *out, double *partial, cudaStream_t st, unsigned int *cnt) {
  if (nv > 128) return fail(VB_EINVAL, "multi_axpy: more than 128 vectors");
  if (nv <= 0 || n == 0) return vec_norm2(w, n, out, partial, reduce_parts(n), st);
  const int blocks = (int)std::min<long long>(512, std::max<long long>(1, (n + 511) / 512));
  multi_axpy_kernel<<<blocks, 256, 0, st>>>(V, ldv, nv, c, sign, w, n, partial, cnt, out, nullptr);
  VB_CHECK_LAUNCH();
  if (!cnt) {
    norm2_final<<<1, 32, 0, st>>>(partial, blocks, out);
    VB_CHECK_LAUNCH();
  }
  return VB_OK;
}

vb_status vec_norm2(const cd *x, long long n, double *out, double *partial, int n_part,
                    cudaStream_t st) {
  norm2_part<<<n_part, RT, 0, st>>>(x, n, partial);
  VB_CHECK_LAUNCH();
  norm2_final<<<1, 32, 0, st>>>(partial, n_part, out);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status vec_scale_inv(cd *x, long long n, const double *nrm, cudaStream_t st, double *keep, const cd *c,
                        const cd *c2, double *alpha_k, cf *shadow) {
  if (n == 0) return VB_OK;
  scale_inv_kernel<<<grid_for(n, 256), 256, 0, st>>>(x, n, nrm, keep, c, c2, alpha_k, shadow);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status vec_copy_scaled(const cd *x, cd *y, long long n, cudaStream_t st) {
  if (n == 0) return VB_OK;
  copy_kernel<<<grid_for(n, 256), 256, 0, st>>>(x, y, n);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status vec_combine(const cd *V, long long ldv, int nv, const cd *u, const double *nrm, cd *y,
                      long long n, cudaStream_t st, const double *vs) {
  if (nv > 128) return fail(VB_EINVAL, "combine: more than 128 vectors");
  combine_kernel<<<grid_for(n, 256), 256, 0, st>>>(V, ldv, nv, u, nrm, y, n, vs);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status tridiag_expm(const cd *c, const cd *c2, double *alpha, const double *beta, int kdim, double tau,
                       const double *bnext, cd *u, double *out, cudaStream_t st) {
  if (kdim < 1 || kdim > 64) return fail(VB_EINVAL, "tridiag_expm: kdim must be in 1..64");
  tridiag_expm_kernel<<<1, 32, 0, st>>>(c, c2, alpha, beta, kdim, tau, bnext, u, out);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

}  // namespace vb
