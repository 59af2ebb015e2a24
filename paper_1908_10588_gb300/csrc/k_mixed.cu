// Mixed-precision H_eff products (the mixed form of the 2TDVP path).
//
// The Krylov vectors, environments and every step other than the H_eff
// products stay in complex double. One product y = H_eff x (Eq. two-site
// Hamiltonian, or Eq. one-site Hamiltonian 1) runs its two dense legs on the
// tensor cores (tcgen05 kind::tf32 in three split-TF32 products, FP32
// accumulation, k_tc.cu) and its
// sparse MPO legs in FP32 on the CUDA cores:
//
//   L leg   T1 = L x        real embedding: [[Re L, -Im L], [Im L, Re L]] (2M x 2K)
//                           times [Re x; Im x] (stored transposed, K-major),
//                           output planar (real rows, then imaginary rows)
//   W legs  T2, T3          planar FP32, sum over the nonzero MPO blocks
//   R leg   y = T3 R^T      A = [Re T3 | Im T3] per row (K-major), B rows
//                           [Re R, -Im R] and [Im R, Re R]; the epilogue
//                           writes y directly as complex double
//
// K dimensions are zero-padded to multiples of 32 (one 128-byte swizzle
// atom of fp32). The conversion kernels write every padding element.
#include <algorithm>

#include "common.h"
#include <climits>
#include <cstdint>

namespace vb {

vb_status tc_gemm_tf32(const float *A, long long lda, const float *B, long long ldb, int M, int N, int K,
                       int mode, float *D, long long ldd, double *Y, int nh, int *err, cudaStream_t st,
                       bool split, float *ws = nullptr, long long ws_elems = 0, const float *Alo = nullptr,
                       const float *Blo = nullptr);
// split-K workspace of the tensor-core legs (floats): enough for every slice
// count the GEMM picks (fewer than 76 tiles, at most 2 x 152 + 76 items)
constexpr long long TC_WS_ELEMS = 380LL * 128 * 128;

namespace {

inline long long pad32(long long k) { return (k + 31) / 32 * 32; }

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  return (int)std::max(1LL, b);
}

// AL[i][k]: rows i < M: [Re L[i,:], -Im L[i,:], 0...]; rows M + i: [Im L, Re L, 0...]
// x = hi + lo with hi = x truncated to tf32 (low 13 mantissa bits cleared,
// exact in tf32) and lo = x - hi (exact in fp32): the operand split of the
// three-product TF32 GEMM, done where the operand is produced
__device__ __forceinline__ void tf32_split_store(float v, float *hi, float *lo, long long e) {
  const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
  hi[e] = h;
  lo[e] = v - h;
}

__global__ void prep_left_env(const cd *__restrict__ L, long long M, int K, long long ld, float *__restrict__ AL,
                              float *__restrict__ ALlo) {
  const long long total = 2 * M * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / ld;
    const int col = (int)(e % ld);
    float v = 0.f;
    if (col < 2 * K) {
      const bool imrow = row >= M;
      const long long i = imrow ? row - M : row;
      const int a = col < K ? col : col - K;
      const cd z = L[i * K + a];
      if (!imrow)
        v = col < K ? (float)z.x : (float)(-z.y);
      else
        v = col < K ? (float)z.y : (float)z.x;
    }
    tf32_split_store(v, AL, ALlo, e);
  }
}

// BR[n][k]: rows n < N: [Re R[n,:], -Im R[n,:], 0...]; rows N + n: [Im R, Re R, 0...]
__global__ void prep_right_env(const cd *__restrict__ R, int N, long long K, long long ld, float *__restrict__ BR,
                               float *__restrict__ BRlo) {
  const long long total = 2LL * N * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / ld;
    const long long col = e % ld;
    float v = 0.f;
    if (col < 2 * K) {
      const bool imrow = row >= N;
      const long long n = imrow ? row - N : row;
      const long long k = col < K ? col : col - K;
      const cd z = R[n * K + k];
      if (!imrow)
        v = col < K ? (float)z.x : (float)(-z.y);
      else
        v = col < K ? (float)z.y : (float)z.x;
    }
    tf32_split_store(v, BR, BRlo, e);
  }
}

// BX[n][k] = [Re x[k][n] (k < K), Im x[k-K][n] (K <= k < 2K), 0...]: a tiled
// transpose of x (K x Ncols complex double) into K-major fp32 rows; x is
// multiplied by *xs on load where xs is given (a vector stored unnormalised)
__global__ void prep_vector_T(const cd *__restrict__ x, int K, long long Ncols, long long ld, float *__restrict__ BX,
                              float *__restrict__ BXlo, const double *__restrict__ xs) {
  __shared__ float tr[32][33], ti[32][33];
  const long long n0 = (long long)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  // the factor is applied in FP32 (GB300's FP64 pipe is narrow); the
  // operand is FP32-accurate either way
  const float f = xs ? (float)xs[0] : 1.f;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r;
    const long long n = n0 + tx;
    cd z = mkc(0.0, 0.0);
    if (k < K && n < Ncols) z = x[(long long)k * Ncols + n];
    tr[r][tx] = (float)z.x * f;
    ti[r][tx] = (float)z.y * f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const long long n = n0 + r;
    const int k = k0 + tx;
    if (n < Ncols && k < K) {
      tf32_split_store(tr[tx][r], BX, BXlo, n * ld + k);
      tf32_split_store(ti[tx][r], BX, BXlo, n * ld + K + k);
    }
  }
}

// zero the K padding columns [from, ld) of BX rows
__global__ void zero_cols(float *__restrict__ X, long long rows, long long ld, long long from) {
  const long long w = ld - from;
  const long long total = rows * w;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    X[(e / w) * ld + from + e % w] = 0.f;
}

// Sparse MPO leg of the mixed-precision H_eff product (FP32, CUDA cores), real
// and imaginary parts in separate planes of X and Y. A block covers RB output
// rows (p, s', w') and TQ * QPT consecutive q of each; every warp stays inside
// one row, so the loops over the row's nonzero blocks and operator entries are
// uniform, and the q reads of a warp are coalesced. Index arithmetic is 32-bit
// and done once per row.
template <int QPT>
__global__ void __launch_bounds__(128) wapply_planar_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                                            const float *__restrict__ val, const int *__restrict__ ptr,
                                                            const int *__restrict__ ent, int d, int Wp, int rows,
                                                            int TQ, const float *__restrict__ X, long long xplane,
                                                            WStrides xs, float *__restrict__ Y, long long yplane,
                                                            WStrides ys, int Q) {
  const int RB = blockDim.x / TQ;
  const int tq = threadIdx.x % TQ, rb = threadIdx.x / TQ;
  const int q0 = blockIdx.x * TQ * QPT + tq;
  const int xq = (int)xs.q, yq = (int)ys.q;
  for (int row = blockIdx.y * RB + rb; row < rows; row += gridDim.y * RB) {
    const int wo = row % Wp, t = row / Wp;
    const int so = t % d, p = t / d;
    float ax[QPT], ay[QPT];
#pragma unroll
    for (int j = 0; j < QPT; ++j) ax[j] = ay[j] = 0.f;
    const float *xb = X + p * xs.p;
    const int e1 = ptr[wo + 1];
    for (int e = ptr[wo]; e < e1; ++e) {
      const int wi = ent[3 * e], ident = ent[3 * e + 1], off = ent[3 * e + 2];
      const float *xw = xb + wi * xs.w;
      if (ident) {
        const float *xr = xw + so * xs.s;
#pragma unroll
        for (int j = 0; j < QPT; ++j) {
          const int q = q0 + j * TQ;
          if (q < Q) {
            ax[j] += xr[q * xq];
            ay[j] += xr[q * xq + xplane];
          }
        }
      } else {
        const int k1 = rp[off + so + 1];
        for (int k = rp[off + so]; k < k1; ++k) {
          const float c = val[k];
          const float *xr = xw + col[k] * xs.s;
#pragma unroll
          for (int j = 0; j < QPT; ++j) {
            const int q = q0 + j * TQ;
            if (q < Q) {
              ax[j] = fmaf(c, xr[q * xq], ax[j]);
              ay[j] = fmaf(c, xr[q * xq + xplane], ay[j]);
            }
          }
        }
      }
    }
    float *yr = Y + p * ys.p + so * ys.s + wo * ys.w;
#pragma unroll
    for (int j = 0; j < QPT; ++j) {
      const int q = q0 + j * TQ;
      if (q < Q) {
        yr[q * yq] = ax[j];
        yr[q * yq + yplane] = ay[j];
      }
    }
  }
}

// Vectorised form of the leg for unit q stride, Q % 4 == 0 and 16-byte
// aligned rows: a block takes one output pair (s', w') and a chunk of
// 128 * WV4_J consecutive (p, q/4) positions, so all its threads walk the same
// nonzero blocks and operator entries; each thread moves four q per load.
// Blocks are ordered with the chunk slowest, so the (s', w') blocks of one
// chunk run together and share its input rows in L2.
constexpr int WV4_J = 2;
// 32-bit element offsets (both buffers are below 2^31 elements; checked on
// the host), so the per-thread row offsets take one register each
struct V4Strides {
  int xp, xw, xs, xplane, yp, yw, ys, yplane;
};
__global__ void __launch_bounds__(128, 12) wapply_planar_v4_kernel(
    const int *__restrict__ rp, const int *__restrict__ col, const float *__restrict__ val,
    const int *__restrict__ ptr, const int *__restrict__ ent, int d, int Wp, int P, int Q4,
    const float *__restrict__ X, float *__restrict__ Y, V4Strides s) {
  const int b = blockIdx.x;
  const int wo = b % Wp, t = b / Wp;
  const int so = t % d, chunk = t / d;
  const int npair = P * Q4;
  int xo[WV4_J], yo[WV4_J];
  bool ok[WV4_J];
#pragma unroll
  for (int j = 0; j < WV4_J; ++j) {
    const int i = chunk * (128 * WV4_J) + threadIdx.x + 128 * j;
    ok[j] = i < npair;
    const int p = ok[j] ? i / Q4 : 0, q4 = ok[j] ? i % Q4 : 0;
    xo[j] = p * s.xp + 4 * q4;
    yo[j] = p * s.yp + so * s.ys + wo * s.yw + 4 * q4;
  }
  float4 ar[WV4_J], ai[WV4_J];
#pragma unroll
  for (int j = 0; j < WV4_J; ++j) ar[j] = ai[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int e1 = ptr[wo + 1];
  for (int e = ptr[wo]; e < e1; ++e) {
    const int wi = ent[3 * e], ident = ent[3 * e + 1], off = ent[3 * e + 2];
    const int ow = wi * s.xw;
    if (ident) {
      const float *xr = X + (ow + so * s.xs);
#pragma unroll
      for (int j = 0; j < WV4_J; ++j) {
        if (!ok[j]) continue;
        const float4 vr = *reinterpret_cast<const float4 *>(xr + xo[j]);
        const float4 vi = *reinterpret_cast<const float4 *>(xr + xo[j] + s.xplane);
        ar[j].x += vr.x; ar[j].y += vr.y; ar[j].z += vr.z; ar[j].w += vr.w;
        ai[j].x += vi.x; ai[j].y += vi.y; ai[j].z += vi.z; ai[j].w += vi.w;
      }
    } else {
      const int k1 = rp[off + so + 1];
      for (int kk = rp[off + so]; kk < k1; ++kk) {
        const float c = val[kk];
        const float *xr = X + (ow + col[kk] * s.xs);
#pragma unroll
        for (int j = 0; j < WV4_J; ++j) {
          if (!ok[j]) continue;
          const float4 vr = *reinterpret_cast<const float4 *>(xr + xo[j]);
          const float4 vi = *reinterpret_cast<const float4 *>(xr + xo[j] + s.xplane);
          ar[j].x = fmaf(c, vr.x, ar[j].x); ar[j].y = fmaf(c, vr.y, ar[j].y);
          ar[j].z = fmaf(c, vr.z, ar[j].z); ar[j].w = fmaf(c, vr.w, ar[j].w);
          ai[j].x = fmaf(c, vi.x, ai[j].x); ai[j].y = fmaf(c, vi.y, ai[j].y);
          ai[j].z = fmaf(c, vi.z, ai[j].z); ai[j].w = fmaf(c, vi.w, ai[j].w);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < WV4_J; ++j) {
    if (!ok[j]) continue;
    *reinterpret_cast<float4 *>(Y + yo[j]) = ar[j];
    *reinterpret_cast<float4 *>(Y + yo[j] + s.yplane) = ai[j];
  }
}

vb_status wapply_planar(const MpoSite &S, const float *X, long long xplane, WStrides xs, long long x_size,
                        float *Y, long long yplane, WStrides ys, long long y_size, int P, int Q, cudaStream_t st) {
  const int d = S.d, Wp = S.wr, Wc = S.wl;
  const long long total = (long long)P * d * Wp * Q;
  if (total == 0) return VB_OK;
  if (P < 0 || Q < 0 || xs.q < 0 || ys.q < 0 || xs.q > INT_MAX / 4 || ys.q > INT_MAX / 4 ||
      (long long)Q * std::max(xs.q, ys.q) > INT_MAX || (long long)P * d * Wp > INT_MAX)
    return fail(VB_EINVAL, "wapply_planar: sizes or strides out of range");
  const long long xmax = (P - 1) * xs.p + (Wc - 1) * xs.w + (d - 1) * xs.s + (Q - 1) * xs.q + xplane;
  const long long ymax = (P - 1) * ys.p + (Wp - 1) * ys.w + (d - 1) * ys.s + (Q - 1) * ys.q + yplane;
  if (xmax >= x_size || ymax >= y_size) return fail(VB_EINVAL, "wapply_planar: view exceeds its buffer");
  auto al16 = [](long long v) { return (v & 3) == 0; };
  if (xs.q == 1 && ys.q == 1 && Q % 4 == 0 && al16(xs.p) && al16(xs.w) && al16(xs.s) && al16(xplane) &&
      al16(ys.p) && al16(ys.w) && al16(ys.s) && al16(yplane) && ((uintptr_t)X & 15) == 0 &&
      ((uintptr_t)Y & 15) == 0 && x_size <= INT_MAX && y_size <= INT_MAX) {
    const long long chunks = ((long long)P * (Q / 4) + 128 * WV4_J - 1) / (128 * WV4_J);
    const long long blocks = chunks * d * Wp;
    if (blocks <= INT_MAX) {
      const V4Strides sv{(int)xs.p, (int)xs.w, (int)xs.s, (int)xplane, (int)ys.p, (int)ys.w, (int)ys.s, (int)yplane};
      wapply_planar_v4_kernel<<<(unsigned)blocks, 128, 0, st>>>(S.d_csr_ptr, S.d_csr_col, S.d_csr_val32, S.d_fwd_ptr,
                                                                S.d_fwd_ent, d, Wp, P, Q / 4, X, Y, sv);
      VB_CHECK_LAUNCH();
      return VB_OK;
    }
  }
  const int rows = P * d * Wp;
  // q tiling: wide rows take 128 threads x 4 q each; narrow rows share a block
  int TQ, qpt;
  if (Q >= 512) {
    TQ = 128; qpt = 4;
  } else if (Q > 128) {
    TQ = 128; qpt = (Q + 127) / 128;  // 2..4
    if (qpt == 3) qpt = 4;
  } else {
    TQ = std::max(32, (Q + 31) / 32 * 32); qpt = 1;
    if (TQ == 96) TQ = 128;
  }
  const int RB = 128 / TQ;
  const long long gx = (Q + (long long)TQ * qpt - 1) / ((long long)TQ * qpt);
  const long long gy = std::min<long long>((rows + RB - 1) / RB, 65535);
  dim3 grid((unsigned)gx, (unsigned)gy);
  const int *rp = S.d_csr_ptr, *cl = S.d_csr_col, *pt = S.d_fwd_ptr, *en = S.d_fwd_ent;
  const float *vl = S.d_csr_val32;
  if (qpt == 4)
    wapply_planar_kernel<4><<<grid, 128, 0, st>>>(rp, cl, vl, pt, en, d, Wp, rows, TQ, X, xplane, xs, Y, yplane, ys, Q);
  else if (qpt == 2)
    wapply_planar_kernel<2><<<grid, 128, 0, st>>>(rp, cl, vl, pt, en, d, Wp, rows, TQ, X, xplane, xs, Y, yplane, ys, Q);
  else
    wapply_planar_kernel<1><<<grid, 128, 0, st>>>(rp, cl, vl, pt, en, d, Wp, rows, TQ, X, xplane, xs, Y, yplane, ys, Q);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

struct TcLayout {
  long long ML, KL, ldL, NL;  // L leg: (2 ML) x ldL times NL x ldL
  long long MR, KR, ld3;      // R leg: MR x ld3 times (2 mR) x ld3
  long long nT1, nT2;
  size_t oAL, oBX, oT1, oT2, oT3, oBR, oWs, oALlo, oBXlo, oBRlo, oErr, total;
  TcLayout(const vb_mpo *mpo, int site, int two_site, int mL, int mR) {
    const MpoSite &S = mpo->sites[site];
    const MpoSite &S2 = two_site ? mpo->sites[site + 1] : S;
    const long long d1 = S.d, d2 = two_site ? S2.d : 1;
    const long long wL = S.wl, wM = S.wr, wR = two_site ? S2.wr : S.wr;
    ML = (long long)mL * wL;
    KL = mL;
    ldL = pad32(2 * KL);
    NL = d1 * d2 * mR;
    MR = (long long)mL * d1 * d2;
    KR = wR * mR;
    ld3 = pad32(2 * KR);
    nT1 = 2 * ML * NL;
    nT2 = two_site ? 2LL * mL * d1 * wM * d2 * mR : 0;
    size_t o = 0;
    auto take = [&](size_t bytes) {
      size_t r = o;
      o += (bytes + 255) / 256 * 256;
      return r;
    };
    oAL = take((size_t)2 * ML * ldL * 4);
    oBX = take((size_t)NL * ldL * 4);
    oT1 = take((size_t)nT1 * 4);
    oT2 = take((size_t)std::max<long long>(nT2, 1) * 4);
    oT3 = take((size_t)MR * ld3 * 4);
    oBR = take((size_t)2 * mR * ld3 * 4);
    oWs = take((size_t)TC_WS_ELEMS * 4);
    oALlo = take((size_t)2 * ML * ldL * 4);
    oBXlo = take((size_t)NL * ldL * 4);
    oBRlo = take((size_t)2 * mR * ld3 * 4);
    oErr = take(256);
    total = o;
  }
};

}  // namespace

size_t heff_mixed_work_bytes(const vb_mpo *mpo, int site, int two_site, int mL, int mR) {
  if (!mpo || site < 0 || site >= mpo->n || (two_site && site + 1 >= mpo->n) || mL < 1 || mR < 1) return 0;
  return TcLayout(mpo, site, two_site, mL, mR).total;
}

// device address of the tensor-core error flag inside a mixed workspace
int *heff_mixed_err_flag(const vb_mpo *mpo, int site, int two_site, int mL, int mR, void *work) {
  TcLayout lay(mpo, site, two_site, mL, mR);
  return reinterpret_cast<int *>(static_cast<char *>(work) + lay.oErr);
}

vb_status heff_mixed_apply(const vb_mpo *mpo, int site, int two_site, int mL, int mR, const cd *L,
                           const cd *R, const cd *x, cd *y, void *work, size_t work_bytes, int *err,
                           cudaStream_t st, const double *x_scale) {
  TcLayout lay(mpo, site, two_site, mL, mR);
  if (work_bytes < lay.total) return fail(VB_EINVAL, "heff_mixed_apply: workspace too small");
  char *w = static_cast<char *>(work);
  float *AL = reinterpret_cast<float *>(w + lay.oAL);
  float *BX = reinterpret_cast<float *>(w + lay.oBX);
  float *T1 = reinterpret_cast<float *>(w + lay.oT1);
  float *T2 = reinterpret_cast<float *>(w + lay.oT2);
  float *T3 = reinterpret_cast<float *>(w + lay.oT3);
  float *BR = reinterpret_cast<float *>(w + lay.oBR);
  float *ALlo = reinterpret_cast<float *>(w + lay.oALlo);
  float *BXlo = reinterpret_cast<float *>(w + lay.oBXlo);
  float *BRlo = reinterpret_cast<float *>(w + lay.oBRlo);
  const MpoSite &S = mpo->sites[site];
  const double theta_elems = (double)lay.NL * mL;  // complex elements of x
  // operands of the L leg
  prof_begin(PH_PREP, st);
  prep_left_env<<<grid_for(2 * lay.ML * lay.ldL), 256, 0, st>>>(L, lay.ML, (int)lay.KL, lay.ldL, AL, ALlo);
  VB_CHECK_LAUNCH();
  {
    dim3 g((unsigned)((lay.NL + 31) / 32), (unsigned)((lay.KL + 31) / 32));
    prep_vector_T<<<g, 256, 0, st>>>(x, (int)lay.KL, lay.NL, lay.ldL, BX, BXlo, x_scale);
    VB_CHECK_LAUNCH();
    if (lay.ldL > 2 * lay.KL) {
      zero_cols<<<grid_for(lay.NL * (lay.ldL - 2 * lay.KL)), 256, 0, st>>>(BX, lay.NL, lay.ldL, 2 * lay.KL);
      VB_CHECK_LAUNCH();
      zero_cols<<<grid_for(lay.NL * (lay.ldL - 2 * lay.KL)), 256, 0, st>>>(BXlo, lay.NL, lay.ldL, 2 * lay.KL);
      VB_CHECK_LAUNCH();
    }
  }
  prep_right_env<<<grid_for(2LL * mR * lay.ld3), 256, 0, st>>>(R, mR, lay.KR, lay.ld3, BR, BRlo);
  VB_CHECK_LAUNCH();
  prof_end(PH_PREP, st, 0.0);
  // L leg: T1 planar (2 ML) x NL (both operands split by the prep kernels;
  // K = 2 mL <= 128 takes the resident-B form of the GEMM)
  prof_begin(PH_TC, st);
  VB_TRY(tc_gemm_tf32(AL, lay.ldL, BX, lay.ldL, (int)(2 * lay.ML), (int)lay.NL, (int)lay.ldL, 0, T1, lay.NL,
                      nullptr, 0, err, st, true, nullptr, 0, ALlo, BXlo));
  prof_end(PH_TC, st, 8.0 * theta_elems * (double)lay.ML);
  const long long P1 = lay.ML * lay.NL;  // plane offset of T1
  if (two_site) {
    const MpoSite &S2 = mpo->sites[site + 1];
    const long long d1 = S.d, d2 = S2.d, wL = S.wl, wM = S.wr, Q1 = d2 * mR;
    const long long P2 = lay.nT2 / 2;
    // T2[a'][s'][w1][(t b)] planar
    prof_begin(PH_WLEG, st);
    VB_TRY(wapply_planar(S, T1, P1, WS(/*p*/ wL * d1 * Q1, /*w*/ d1 * Q1, /*s*/ Q1, /*q*/ 1), lay.nT1, T2, P2,
                         WS(/*p*/ d1 * wM * Q1, /*w*/ Q1, /*s*/ wM * Q1, /*q*/ 1), lay.nT2, mL, (int)Q1, st));
    prof_end(PH_WLEG, st, 0.0, 4.0 * (double)(lay.nT1 + lay.nT2));
    // T3 row (a' s' t'): [Re (w2 b) | Im (w2 b) | 0]
    prof_begin(PH_WLEG, st);
    VB_TRY(wapply_planar(S2, T2, P2, WS(/*p*/ wM * d2 * mR, /*w*/ d2 * mR, /*s*/ mR, /*q*/ 1), lay.nT2, T3,
                         lay.KR, WS(/*p*/ d2 * lay.ld3, /*w*/ mR, /*s*/ lay.ld3, /*q*/ 1), lay.MR * lay.ld3,
                         (int)(mL * d1), mR, st));
    prof_end(PH_WLEG, st, 0.0, 4.0 * (double)(lay.nT2 + 2 * lay.MR * lay.KR));
  } else {
    const long long d = S.d, wL = S.wl;
    prof_begin(PH_WLEG, st);
    VB_TRY(wapply_planar(S, T1, P1, WS(/*p*/ wL * d * mR, /*w*/ d * mR, /*s*/ mR, /*q*/ 1), lay.nT1, T3, lay.KR,
                         WS(/*p*/ d * lay.ld3, /*w*/ mR, /*s*/ lay.ld3, /*q*/ 1), lay.MR * lay.ld3, mL, mR, st));
    prof_end(PH_WLEG, st, 0.0, 4.0 * (double)(lay.nT1 + 2 * lay.MR * lay.KR));
  }
  if (lay.ld3 > 2 * lay.KR) {
    prof_begin(PH_PREP, st);
    zero_cols<<<grid_for(lay.MR * (lay.ld3 - 2 * lay.KR)), 256, 0, st>>>(T3, lay.MR, lay.ld3, 2 * lay.KR);
    VB_CHECK_LAUNCH();
    prof_end(PH_PREP, st, 0.0);
  }
  // R leg: y (complex double) = T3 BR^T
  prof_begin(PH_TC, st);
  VB_TRY(tc_gemm_tf32(T3, lay.ld3, BR, lay.ld3, (int)lay.MR, 2 * mR, (int)lay.ld3, 1, nullptr, 0,
                      reinterpret_cast<double *>(y), mR, err, st, true, reinterpret_cast<float *>(w + lay.oWs),
                      TC_WS_ELEMS, nullptr, BRlo));
  prof_end(PH_TC, st, 8.0 * theta_elems * (double)lay.KR);
  return VB_OK;
}

}  // namespace vb
