// Leading eigenvectors of a reduced density matrix by subspace iteration, for
// the mixed form of the truncated split (Sec. 2.1.1: the kept Schmidt
// directions of theta are the leading eigenvectors of rho = M M^+ or M^+ M).
// The iteration works on theta itself, never on rho: each step applies M and
// then M^+ in complex FP32, and re-orthonormalises the r basis rows with a
// row-scaled Cholesky QR (twice). The basis starts from the bond tensor of the
// previous state, whose span is already close to the wanted one after a short
// time step, topped up with counter-based random rows.
#include "common.h"

namespace vb {
namespace {

// splitmix64 finaliser (Steele, Lea, Flood 2014), mapped to [-1, 1)
__device__ __forceinline__ float urand(unsigned long long seed, unsigned long long idx) {
  unsigned long long z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(z >> 40) * (2.0f / 16777216.0f) - 1.0f;
}

// Q (r x n): rows j < m_warm from the old bond tensor, the rest random.
// left:  old tensor is n x m_old (row-major), row j of Q = its column j
// right: old tensor is m_old x n, row j of Q = its row j
__global__ void init_rows_kernel(cf *__restrict__ Q, int r, int n, const cd *__restrict__ warm, int m_old,
                                 int m_warm, int left, unsigned long long seed) {
  const long long tot = (long long)r * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), x = (int)(e % n);
    cf v;
    if (j < m_warm) {
      const cd a = left ? warm[(long long)x * m_old + j] : warm[(long long)j * n + x];
      v = mkc((float)a.x, (float)a.y);
    } else {
      v = mkc(urand(seed, 2ull * e), urand(seed, 2ull * e + 1));
    }
    Q[e] = v;
  }
}

// rows i with flag[i] != 0 get fresh random entries
__global__ void fill_flagged_kernel(cf *__restrict__ Q, int r, int n, const int *__restrict__ flag,
                                    unsigned long long seed) {
  const long long tot = (long long)r * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / n);
    if (flag[j]) Q[e] = mkc(urand(seed, 2ull * e), urand(seed, 2ull * e + 1));
  }
}

// One CTA. G = A A^+ (r x r). With D = diag(G)^(-1/2), factor D G D = L L^+
// (lower) and write W = L^-1 D (r x r), so that W A has orthonormal rows. A
// row whose scaled pivot is <= tau (its part orthogonal to the rows before it
// is below sqrt(tau) of its length) gets a zero row in W and flag 1;
// flag[r] counts them. Shared memory: r*r complex + 2 r words; the strictly
// upper triangle of L holds the strictly lower triangle of L^-1, transposed.
constexpr int CHOL_THREADS = 512;
__global__ void __launch_bounds__(CHOL_THREADS) chol_rows_kernel(const cf *__restrict__ G, int r, float tau,
                                                                 cf *__restrict__ W, int *__restrict__ flag) {
  extern __shared__ __align__(16) unsigned char chol_smem[];
  cf *L = reinterpret_cast<cf *>(chol_smem);
  float *dsc = reinterpret_cast<float *>(L + (size_t)r * r);
  int *bad = reinterpret_cast<int *>(dsc + r);
  __shared__ float dinv[128];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < r; i += nt) {
    const float g = G[(long long)i * r + i].x;
    dsc[i] = g > 0.f ? 1.0f / sqrtf(g) : 0.f;
    bad[i] = 0;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, j = e % r;
    if (j <= i) {
      const cf g = G[e];
      const float s = dsc[i] * dsc[j];
      L[e] = mkc(g.x * s, g.y * s);
    }
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    const float p = L[j * r + j].x;
    const bool fail = !(p > tau);
    __syncthreads();
    if (fail) {
      for (int i = j + tid; i < r; i += nt) L[i * r + j] = mkc(0.f, 0.f);
      if (tid == 0) bad[j] = 1;
      __syncthreads();
      continue;
    }
    const float ljj = sqrtf(p), inv = 1.0f / ljj;
    for (int i = j + 1 + tid; i < r; i += nt) {
      const cf v = L[i * r + j];
      L[i * r + j] = mkc(v.x * inv, v.y * inv);
    }
    if (tid == 0) L[j * r + j] = mkc(ljj, 0.f);
    __syncthreads();
    const int m = r - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int ii = e / m, cc = e % m;
      if (cc > ii) continue;
      const int i = j + 1 + ii, c = j + 1 + cc;
      const cf a = L[i * r + j], b = L[c * r + j];
      const cf cur = L[i * r + c];
      L[i * r + c] = mkc(cur.x - (a.x * b.x + a.y * b.y), cur.y - (a.y * b.x - a.x * b.y));
    }
    __syncthreads();
  }
  // inverse by forward substitution, one thread per column c:
  // x_i = (delta_ic - sum_{c<=k<i} L_ik x_k) / L_ii, x_c kept in dinv[c]
  for (int c = tid; c < r; c += nt) {
    const float xc = bad[c] ? 0.f : 1.0f / L[c * r + c].x;
    dinv[c] = xc;
    for (int i = c + 1; i < r; ++i) {
      cf s = mkc(0.f, 0.f);
      if (!bad[i]) {
        {
          const cf a = L[i * r + c];
          s = mkc(-a.x * xc, -a.y * xc);
        }
        for (int k = c + 1; k < i; ++k) {
          const cf a = L[i * r + k], x = L[c * r + k];
          s.x -= a.x * x.x - a.y * x.y;
          s.y -= a.x * x.y + a.y * x.x;
        }
        const float li = 1.0f / L[i * r + i].x;
        s = mkc(s.x * li, s.y * li);
      }
      L[c * r + i] = s;
    }
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, c = e % r;
    cf w = mkc(0.f, 0.f);
    if (i == c)
      w = mkc(dinv[c], 0.f);
    else if (i > c)
      w = L[c * r + i];
    if (bad[i]) w = mkc(0.f, 0.f);
    const float s = dsc[c];
    W[e] = mkc(w.x * s, w.y * s);
  }
  if (tid == 0) {
    int cnt = 0;
    for (int i = 0; i < r; ++i) cnt += bad[i];
    flag[r] = cnt;
  }
  for (int i = tid; i < r; i += nt) flag[i] = bad[i];
}

__global__ void __launch_bounds__(256) norm2_f32_part(const cf *__restrict__ x, long long n,
                                                      double *__restrict__ partial) {
  __shared__ double sh[8];
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += 256) {
    const cf a = x[i];
    s += (double)a.x * a.x + (double)a.y * a.y;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

__global__ void sum_parts_kernel(const double *__restrict__ partial, int n_part, double *out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < n_part; b += 32) s += partial[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[0] = s;
}

__global__ void status_kernel(const double *capt, const int *cnt, double *out) {
  out[0] = capt[0];
  out[1] = (double)cnt[0];
}

inline int grid_of(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)); }

}  // namespace

size_t subspace_chol_smem(int r) { return (size_t)r * r * sizeof(cf) + 2 * (size_t)r * sizeof(float); }

vb_status subspace_init(cf *Q, int r, int n, const cd *warm, int m_old, int m_warm, bool left,
                        unsigned long long seed, cudaStream_t st) {
  if (r < 1 || n < r || m_warm < 0 || m_warm > r || (m_warm > 0 && (!warm || m_old < m_warm)))
    return fail(VB_EINVAL, "subspace_init: bad sizes");
  init_rows_kernel<<<grid_of((long long)r * n), 256, 0, st>>>(Q, r, n, warm, m_old, m_warm, left ? 1 : 0, seed);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

// one scaled Cholesky QR pass: T = W A with W from A A^+; flagged rows of T
// are refilled at random
static vb_status orth_pass(const cf *A, cf *T, int r, int n, const SubspaceWork &w, unsigned long long seed,
                           cudaStream_t st) {
  GemmArgsF g{};
  g.M = r; g.N = r; g.K = n; g.batch = 1;
  g.opA = OP_N; g.opB = OP_C;
  g.A = A; g.lda = n; g.B = A; g.ldb = n; g.C = w.G; g.ldc = r;
  g.alpha = mkc(1.f, 0.f); g.beta = mkc(0.f, 0.f);
  g.a_size = (long long)r * n; g.b_size = (long long)r * n; g.c_size = (long long)r * r;
  g.ws = w.ws; g.ws_elems = w.ws_elems;
  VB_TRY(gemm<float>(g, st));
  chol_rows_kernel<<<1, CHOL_THREADS, subspace_chol_smem(r), st>>>(w.G, r, 1e-4f, w.W, w.flag);
  VB_CHECK_LAUNCH();
  GemmArgsF h{};
  h.M = r; h.N = n; h.K = r; h.batch = 1;
  h.opA = OP_N; h.opB = OP_N;
  h.A = w.W; h.lda = r; h.B = A; h.ldb = n; h.C = T; h.ldc = n;
  h.alpha = mkc(1.f, 0.f); h.beta = mkc(0.f, 0.f);
  h.a_size = (long long)r * r; h.b_size = (long long)r * n; h.c_size = (long long)r * n;
  VB_TRY(gemm<float>(h, st));
  fill_flagged_kernel<<<grid_of((long long)r * n), 256, 0, st>>>(T, r, n, w.flag, seed);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status subspace_orth(cf *Q, int r, int n, const SubspaceWork &w, unsigned long long seed, cudaStream_t st) {
  if (r < 1 || r > 128 || n < r) return fail(VB_EINVAL, "subspace_orth: needs 1 <= r <= min(n, 128)");
  static int smem_set[64] = {0};
  int dev = 0;
  VB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !smem_set[dev]) {
    VB_TRY_CUDA(cudaFuncSetAttribute(chol_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)subspace_chol_smem(128)));
    smem_set[dev] = 1;
  }
  VB_TRY(orth_pass(Q, w.T, r, n, w, seed, st));
  VB_TRY(orth_pass(w.T, Q, r, n, w, seed ^ 0x5bd1e995ull, st));
  return VB_OK;
}

vb_status subspace_status(const double *capt, const int *cnt, double *out, cudaStream_t st) {
  status_kernel<<<1, 1, 0, st>>>(capt, cnt, out);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status norm2_sq_f32(const cf *x, long long n, double *out, double *partial, int n_part, cudaStream_t st) {
  if (n_part < 1 || n_part > 1024) return fail(VB_EINVAL, "norm2_sq_f32: bad partial count");
  norm2_f32_part<<<n_part, 256, 0, st>>>(x, n, partial);
  VB_CHECK_LAUNCH();
  sum_parts_kernel<<<1, 32, 0, st>>>(partial, n_part, out);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

}  // namespace vb
