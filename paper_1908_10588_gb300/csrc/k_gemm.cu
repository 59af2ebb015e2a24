// Strided batched complex GEMM on the CUDA cores (complex double on the FP64
// path; complex float where the mixed path needs a SIMT product).
//
// Every dense contraction of the FP64 2TDVP path (the L and R legs of
// H_eff, the environment updates, the merge of two sites, the reduced
// density matrix and the split) is one call of this kernel with the right
// operand views. GB300 has no FP64 tensor-core MMA kind, so this path runs
// on the FP64 FMA units; the mixed-precision path replaces the H_eff legs
// with tensor-core products.
#include <algorithm>

#include "common.h"

namespace vb {
namespace {

constexpr int BM = 64, BN = 64, BK = 8, NT = 256;

template <class R>
__device__ __forceinline__ cplx<R> ldA(const cplx<R> *A, int op, long long lda, int i, int k) {
  // op(A)[i,k]
  cplx<R> v;
  if (op == OP_N || op == OP_R)
    v = A[(long long)i * lda + k];
  else
    v = A[(long long)k * lda + i];
  if (op == OP_C || op == OP_R) v.y = -v.y;
  return v;
}

template <class R>
__device__ __forceinline__ cplx<R> ldB(const cplx<R> *B, int op, long long ldb, int k, int j) {
  // op(B)[k,j]
  cplx<R> v;
  if (op == OP_N || op == OP_R)
    v = B[(long long)k * ldb + j];
  else
    v = B[(long long)j * ldb + k];
  if (op == OP_C || op == OP_R) v.y = -v.y;
  return v;
}

template <class R>
__global__ void __launch_bounds__(NT) zgemm_kernel(GemmArgsT<R> g) {
  typedef cplx<R> C_;
  __shared__ C_ As[BK][BM + 1];
  __shared__ C_ Bs[BK][BN + 1];
  const int b = blockIdx.z;
  const C_ *A = g.A + (long long)b * g.sA;
  const C_ *B = g.B + (long long)b * g.sB;
  C_ *C = g.C + (long long)b * g.sC;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  // split-K chunk: only k < Kb of this batch entry
  const int Kb = g.kc > 0 ? (int)min((long long)g.K, g.kfull - (long long)b * g.kc) : g.K;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const bool a_kfast = (g.opA == OP_N || g.opA == OP_R);
  const bool b_jfast = (g.opB == OP_N || g.opB == OP_R);
  C_ acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = mkc<R>(0, 0);
  // rows of this thread: i0 + ty + 16 r; a warp holds ty = 2w, 2w + 1, so
  // the number of row groups r with a valid row is the same for the warp
  const int wrow = i0 + 2 * (tid >> 5);
  const int rwarp = max(0, min(4, (g.M - wrow + 15) / 16));
  const bool rfull = i0 + BM <= g.M;

  for (int k0 = 0; k0 < Kb; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int l = tid + r * NT;
      int ii, kk;
      if (a_kfast) {
        kk = l % BK;
        ii = l / BK;
      } else {
        ii = l % BM;
        kk = l / BM;
      }
      int gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < g.M && gk < Kb) ? ldA<R>(A, g.opA, g.lda, gi, gk) : mkc<R>(0, 0);
      int jj;
      if (b_jfast) {
        jj = l % BN;
        kk = l / BN;
      } else {
        kk = l % BK;
        jj = l / BK;
      }
      int gj = j0 + jj;
      gk = k0 + kk;
      Bs[kk][jj] = (gj < g.N && gk < Kb) ? ldB<R>(B, g.opB, g.ldb, gk, gj) : mkc<R>(0, 0);
    }
    __syncthreads();
    if (rfull) {
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        C_ a[4], bb[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bb[c] = Bs[kk][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            acc[r][c].x = fma(a[r].x, bb[c].x, acc[r][c].x);
            acc[r][c].x = fma(-a[r].y, bb[c].y, acc[r][c].x);
            acc[r][c].y = fma(a[r].x, bb[c].y, acc[r][c].y);
            acc[r][c].y = fma(a[r].y, bb[c].x, acc[r][c].y);
          }
      }
    } else if (rwarp > 0) {
      // ragged last row tile: only the warp-uniform row groups that hold
      // valid rows do arithmetic (FP64 issue slots are the scarce resource)
      for (int kk = 0; kk < BK; ++kk) {
        C_ bb[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) bb[c] = Bs[kk][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (r >= rwarp) break;
          const C_ a = As[kk][ty + 16 * r];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            acc[r][c].x = fma(a.x, bb[c].x, acc[r][c].x);
            acc[r][c].x = fma(-a.y, bb[c].y, acc[r][c].x);
            acc[r][c].y = fma(a.x, bb[c].y, acc[r][c].y);
            acc[r][c].y = fma(a.y, bb[c].x, acc[r][c].y);
          }
        }
      }
    }
    __syncthreads();
  }
  const bool beta0 = (g.beta.x == R(0) && g.beta.y == R(0));
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int gi = i0 + ty + 16 * r;
    if (gi >= g.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int gj = j0 + tx + 16 * c;
      if (gj >= g.N) continue;
      C_ v = cmul(g.alpha, acc[r][c]);
      long long o = (long long)gi * g.ldc + gj;
      if (!beta0) v = cadd(v, cmul(g.beta, C[o]));
      C[o] = v;
    }
  }
}

// C = alpha sum_b ws[b] + beta C, summed in chunk order (deterministic)
template <class R>
__global__ void splitk_reduce(const cplx<R> *__restrict__ ws, int chunks, int M, int N, cplx<R> *C, long long ldc,
                              cplx<R> alpha, cplx<R> beta) {
  const long long MN = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MN;
       e += (long long)gridDim.x * blockDim.x) {
    cplx<R> s = mkc<R>(0, 0);
    for (int b = 0; b < chunks; ++b) s = cadd(s, ws[(long long)b * MN + e]);
    const long long o = (e / N) * ldc + e % N;
    cplx<R> v = cmul(alpha, s);
    if (!(beta.x == R(0) && beta.y == R(0))) v = cadd(v, cmul(beta, C[o]));
    C[o] = v;
  }
}

}  // namespace

template <class R>
vb_status gemm(const GemmArgsT<R> &g, cudaStream_t st) {
  if (g.M < 0 || g.N < 0 || g.K < 0 || g.batch < 0)
    return fail(VB_EINVAL, "zgemm: negative size");
  if (g.M == 0 || g.N == 0 || g.batch == 0) return VB_OK;
  if (g.batch > 65535) return fail(VB_EINVAL, "zgemm: batch > 65535");
  if ((g.M + BM - 1) / BM > 65535) return fail(VB_EINVAL, "zgemm: M too large");
  {
    const bool at = !(g.opA == OP_N || g.opA == OP_R), bt = !(g.opB == OP_N || g.opB == OP_R);
    const long long amax = (long long)(g.batch - 1) * g.sA +
                           (at ? (long long)(g.K - 1) * g.lda + (g.M - 1) : (long long)(g.M - 1) * g.lda + (g.K - 1));
    const long long bmax = (long long)(g.batch - 1) * g.sB +
                           (bt ? (long long)(g.N - 1) * g.ldb + (g.K - 1) : (long long)(g.K - 1) * g.ldb + (g.N - 1));
    const long long cmax = (long long)(g.batch - 1) * g.sC + (long long)(g.M - 1) * g.ldc + (g.N - 1);
    if ((g.K > 0 && g.a_size > 0 && amax >= g.a_size) || (g.K > 0 && g.b_size > 0 && bmax >= g.b_size) ||
        (g.c_size > 0 && cmax >= g.c_size))
      return fail(VB_EINVAL, "zgemm: operand view exceeds its buffer");
    if (g.a_size <= 0 || g.b_size <= 0 || g.c_size <= 0)
      return fail(VB_EINVAL, "zgemm: buffer sizes must be given");
  }
  const long long tiles = (long long)((g.N + BN - 1) / BN) * ((g.M + BM - 1) / BM) * g.batch;
  if (g.ws && g.batch == 1 && tiles < 76 && g.K >= 4 * BK * 8) {
    // split K so that the launch fills the GPU
    long long chunks = std::min<long long>((152 * 2 + tiles - 1) / tiles, g.K / (8 * BK));
    chunks = std::max<long long>(chunks, 2);
    long long kc = (g.K + chunks - 1) / chunks;
    kc = (kc + BK - 1) / BK * BK;
    chunks = (g.K + kc - 1) / kc;
    if (chunks * (long long)g.M * g.N <= g.ws_elems && chunks <= 65535) {
      GemmArgsT<R> h = g;
      const bool a_kfast = (g.opA == OP_N || g.opA == OP_R), b_kslow = (g.opB == OP_N || g.opB == OP_R);
      h.batch = (int)chunks;
      h.sA = a_kfast ? kc : kc * g.lda;
      h.sB = b_kslow ? kc * g.ldb : kc;
      h.C = g.ws;
      h.ldc = g.N;
      h.sC = (long long)g.M * g.N;
      h.alpha = mkc<R>(1, 0);
      h.beta = mkc<R>(0, 0);
      h.K = (int)kc;
      h.kc = kc;
      h.kfull = g.K;
      dim3 grid2((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, (unsigned)chunks);
      zgemm_kernel<R><<<grid2, NT, 0, st>>>(h);
      VB_CHECK_LAUNCH();
      const long long MN = (long long)g.M * g.N;
      long long blocks = std::min<long long>((MN + 255) / 256, 152LL * 8);
      splitk_reduce<R><<<(int)std::max(1LL, blocks), 256, 0, st>>>(g.ws, (int)chunks, g.M, g.N, g.C, g.ldc, g.alpha,
                                                                  g.beta);
      VB_CHECK_LAUNCH();
      return VB_OK;
    }
  }
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
  zgemm_kernel<R><<<grid, NT, 0, st>>>(g);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

template vb_status gemm<double>(const GemmArgsT<double> &, cudaStream_t);
template vb_status gemm<float>(const GemmArgsT<float> &, cudaStream_t);

}  // namespace vb
