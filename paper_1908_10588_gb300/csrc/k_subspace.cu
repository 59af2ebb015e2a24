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

// One CTA. G = A A^+ (r x r). With D = diag(G)^(-1/2), factor
// D G D = L P L^+ (L unit lower triangular, P = diag(p_j)) and write
// W = P^(-1/2) L^-1 D, so that W A has orthonormal rows. A row whose pivot
// p_j is <= tau (its part orthogonal to the rows before it is below
// sqrt(tau) of its length) gets a zero row in W and flag 1; flag[r] counts
// them.
// Step j eliminates column j and at the same time applies the same row
// operation to M = L^-1 (M_ic -= l_ij M_jc for c < j, M_ij = -l_ij), so each
// step needs a single barrier. The lower triangle holds the elimination,
// the strictly upper triangle holds M transposed.
constexpr int CHOL_THREADS = 1024;
template <class R>
__global__ void __launch_bounds__(CHOL_THREADS) chol_rows_kernel(const cplx<R> *__restrict__ G, int r, R tau,
                                                                 cplx<R> *__restrict__ W, int *__restrict__ flag) {
  typedef cplx<R> C_;
  extern __shared__ __align__(16) unsigned char chol_smem[];
  C_ *S = reinterpret_cast<C_ *>(chol_smem);
  R *dsc = reinterpret_cast<R *>(S + (size_t)r * r);
  R *piv = dsc + r;  // p_j, 0 for a rejected row
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const R zero = R(0), one = R(1);
  for (int i = tid; i < r; i += nt) {
    const R g = G[(long long)i * r + i].x;
    dsc[i] = g > zero ? one / sqrt(g) : zero;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, j = e % r;
    if (j <= i) {
      const C_ g = G[e];
      const R s = dsc[i] * dsc[j];
      S[e] = mkc<R>(g.x * s, g.y * s);
    }
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    const R p = S[j * r + j].x;
    const bool ok = p > tau;
    const R inv = ok ? one / p : zero;
    // warps take rows i > j, lanes the columns c <= i
    for (int i = j + 1 + wid; i < r; i += nw) {
      const C_ a = S[i * r + j];
      const R lx = a.x * inv, ly = a.y * inv;
      for (int c = lane; c <= i; c += 32) {
        if (!ok) {
          if (c == j) S[j * r + i] = mkc<R>(zero, zero);
          continue;
        }
        if (c > j) {  // trailing update of the lower triangle
          const C_ b = S[c * r + j];
          const C_ cur = S[i * r + c];
          S[i * r + c] = mkc<R>(cur.x - (lx * b.x + ly * b.y), cur.y - (ly * b.x - lx * b.y));
        } else if (c < j) {  // M_ic -= l_ij M_jc
          const C_ mj = S[c * r + j];
          const C_ cur = S[c * r + i];
          S[c * r + i] = mkc<R>(cur.x - (lx * mj.x - ly * mj.y), cur.y - (lx * mj.y + ly * mj.x));
        } else {  // M_ij = -l_ij
          S[j * r + i] = mkc<R>(-lx, -ly);
        }
      }
    }
    if (tid == 0) piv[j] = ok ? p : zero;
    __syncthreads();
  }
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, c = e % r;
    C_ w = mkc<R>(zero, zero);
    if (piv[i] > zero && c <= i) {
      const C_ mv = c == i ? mkc<R>(one, zero) : S[c * r + i];
      const R s = dsc[c] / sqrt(piv[i]);
      w = mkc<R>(mv.x * s, mv.y * s);
    }
    W[e] = w;
  }
  if (tid == 0) {
    int cnt = 0;
    for (int i = 0; i < r; ++i) cnt += piv[i] > zero ? 0 : 1;
    flag[r] = cnt;
  }
  for (int i = tid; i < r; i += nt) flag[i] = piv[i] > zero ? 0 : 1;
}

// One-CTA Jacobi eigensolver for the small Hermitian Rayleigh-Ritz matrix
// S (n x n, n <= JAC_MAX_N), all in shared memory: parallel (round-robin)
// ordering, n/2 disjoint rotations per round; every 2 x 2 block of A and
// every row pair of V is updated independently, so a round costs two
// barriers. A rotation U = diag(1, e^{-i phi}) R(theta) zeroes |A_pq| (phase
// phi of A_pq; theta from the real Jacobi rule tan 2 theta = 2|A_pq|/(A_pp - A_qq),
// smaller root). Sweeps stop when no off-diagonal element exceeds
// 1e-7 max(sqrt(A_pp A_qq), |A_pp - A_qq|) + 1e-12 tr A (nor after 20
// sweeps; the sweep count goes to info[0]). Writes the k largest eigenvalues
// (descending) and their eigenvectors as rows W[t][0..n).
constexpr int JAC_THREADS = 1024;
constexpr int JAC_MAX_N = 112;
constexpr int JAC_SWEEPS = 20;
__global__ void __launch_bounds__(JAC_THREADS) ritz_jacobi_kernel(const cf *__restrict__ S, int n, int k,
                                                                  float *__restrict__ evals, cf *__restrict__ W,
                                                                  int *__restrict__ info) {
  extern __shared__ __align__(16) unsigned char jsm[];
  const int np = n + (n & 1), h = np / 2;
  cf *A = reinterpret_cast<cf *>(jsm);
  cf *V = A + np * np;
  cf *ph = V + np * np;  // e^{-i phi} per pair
  float *cs = reinterpret_cast<float *>(ph + h);
  float *sn = cs + h;
  int *pp = reinterpret_cast<int *>(sn + h);
  int *qq = pp + h;
  __shared__ int s_any;
  __shared__ float s_scale;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < np * np; e += nt) {
    const int i = e / np, j = e % np;
    cf a = mkc(0.f, 0.f);
    if (i < n && j < n) {
      const cf u = S[(long long)i * n + j], v = S[(long long)j * n + i];
      a = mkc(0.5f * (u.x + v.x), 0.5f * (u.y - v.y));  // Hermitian part
    }
    A[e] = a;
    V[e] = mkc(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += fabsf(A[i * np + i].x);
    s_scale = s;
  }
  __syncthreads();
  const float floor_abs = 1e-12f * s_scale;
  int sweep = 0;
  for (; sweep < JAC_SWEEPS; ++sweep) {
    if (tid == 0) s_any = 0;
    __syncthreads();
    for (int rd = 0; rd < np - 1; ++rd) {
      for (int t = tid; t < h; t += nt) {
        // circle method: slot 0 fixed, slots 1..np-1 rotate by rd
        const int s0 = t, s1 = np - 1 - t;
        int p = s0 == 0 ? 0 : 1 + (s0 - 1 + rd) % (np - 1);
        int q = 1 + (s1 - 1 + rd) % (np - 1);
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        pp[t] = p;
        qq[t] = q;
        float c_ = 1.f, s_ = 0.f;
        cf e = mkc(1.f, 0.f);
        if (q < n) {
          const float a = A[p * np + p].x, b = A[q * np + q].x;
          const cf c = A[p * np + q];
          const float ac = sqrtf(c.x * c.x + c.y * c.y);
          // rotate while the coupling is above FP32 resolution both relative
          // to the pair's scale and as a rotation angle (|c| / |a - b|): on
          // a graded matrix the rounding noise of the large entries (~eps
          // max(a, b)) stays above 1e-7 sqrt(ab) and would keep every sweep
          // busy with rotations by angles below FP32 precision
          if (ac > 1e-7f * fmaxf(sqrtf(fabsf(a * b)), fabsf(b - a)) + floor_abs) {
            const float tau = (b - a) / (2.f * ac);
            const float tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c_ = 1.f / sqrtf(1.f + tt * tt);
            s_ = tt * c_;
            e = mkc(c.x / ac, -c.y / ac);
            s_any = 1;
          }
        }
        cs[t] = c_;
        sn[t] = s_;
        ph[t] = e;
      }
      __syncthreads();
      // A <- U^H A U, block by block; V <- V U
      for (int e2 = tid; e2 < h * h; e2 += nt) {
        const int bi = e2 / h, bj = e2 % h;
        const float si = sn[bi], sj = sn[bj];
        // a pair that does not rotate has U = I (c = 1, s = 0, phase 1): a
        // block between two such pairs is left exactly as it is
        if (si == 0.f && sj == 0.f && ph[bi].x == 1.f && ph[bi].y == 0.f && ph[bj].x == 1.f && ph[bj].y == 0.f)
          continue;
        const int pi = pp[bi], qi = qq[bi], pj = pp[bj], qj = qq[bj];
        const float ci = cs[bi], cj = cs[bj];
        const cf ei = ph[bi], ej = ph[bj];
        const cf b00 = A[pi * np + pj], b01 = A[pi * np + qj], b10 = A[qi * np + pj], b11 = A[qi * np + qj];
        // left: rows (pi, qi) by U_i^H = [[c, -s conj(e)], [s, c conj(e)]]
        const cf ce = mkc(ei.x, -ei.y);
        const cf t10 = mkc(ce.x * b10.x - ce.y * b10.y, ce.x * b10.y + ce.y * b10.x);
        const cf t11 = mkc(ce.x * b11.x - ce.y * b11.y, ce.x * b11.y + ce.y * b11.x);
        const cf l00 = mkc(ci * b00.x - si * t10.x, ci * b00.y - si * t10.y);
        const cf l01 = mkc(ci * b01.x - si * t11.x, ci * b01.y - si * t11.y);
        const cf l10 = mkc(si * b00.x + ci * t10.x, si * b00.y + ci * t10.y);
        const cf l11 = mkc(si * b01.x + ci * t11.x, si * b01.y + ci * t11.y);
        // right: columns (pj, qj) by U_j = [[c, s], [-s e, c e]]
        const cf u01 = mkc(ej.x * l01.x - ej.y * l01.y, ej.x * l01.y + ej.y * l01.x);
        const cf u11 = mkc(ej.x * l11.x - ej.y * l11.y, ej.x * l11.y + ej.y * l11.x);
        cf r00 = mkc(cj * l00.x - sj * u01.x, cj * l00.y - sj * u01.y);
        cf r01 = mkc(sj * l00.x + cj * u01.x, sj * l00.y + cj * u01.y);
        cf r10 = mkc(cj * l10.x - sj * u11.x, cj * l10.y - sj * u11.y);
        cf r11 = mkc(sj * l10.x + cj * u11.x, sj * l10.y + cj * u11.y);
        if (bi == bj) {
          // diagonal block: real diagonal, the rotated coupling is zero
          r00.y = 0.f;
          r11.y = 0.f;
          if (si != 0.f) r01 = r10 = mkc(0.f, 0.f);
        }
        A[pi * np + pj] = r00;
        A[pi * np + qj] = r01;
        A[qi * np + pj] = r10;
        A[qi * np + qj] = r11;
      }
      for (int e2 = tid; e2 < np * h; e2 += nt) {
        const int x = e2 / h, bj = e2 % h;
        const float sj = sn[bj];
        if (sj == 0.f && ph[bj].x == 1.f && ph[bj].y == 0.f) continue;  // U = I
        const int pj = pp[bj], qj = qq[bj];
        const float cj = cs[bj];
        const cf ej = ph[bj];
        const cf v0 = V[x * np + pj], v1 = V[x * np + qj];
        const cf w1 = mkc(ej.x * v1.x - ej.y * v1.y, ej.x * v1.y + ej.y * v1.x);
        V[x * np + pj] = mkc(cj * v0.x - sj * w1.x, cj * v0.y - sj * w1.y);
        V[x * np + qj] = mkc(sj * v0.x + cj * w1.x, sj * v0.y + cj * w1.y);
      }
      __syncthreads();
    }
    const int any = s_any;
    __syncthreads();
    if (!any) break;
  }
  // k largest eigenvalues, descending (ties by index), and their vectors
  for (int i = tid; i < n; i += nt) {
    const float di = A[i * np + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const float dj = A[j * np + j].x;
      rank += (dj > di || (dj == di && j < i)) ? 1 : 0;
    }
    if (rank < k) {
      evals[rank] = di;
      for (int x = 0; x < n; ++x) W[(long long)rank * n + x] = V[x * np + i];
    }
  }
  if (tid == 0) info[0] = sweep;
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
  prof_begin(PH_ORTHGEMM, st);
  VB_TRY(gemm<float>(g, st));
  prof_end(PH_ORTHGEMM, st, 0.0);
  prof_begin(PH_CHOL, st);
  chol_rows_kernel<float><<<1, CHOL_THREADS, subspace_chol_smem(r), st>>>(w.G, r, 1e-4f, w.W, w.flag);
  VB_CHECK_LAUNCH();
  prof_end(PH_CHOL, st, 0.0);
  GemmArgsF h{};
  h.M = r; h.N = n; h.K = r; h.batch = 1;
  h.opA = OP_N; h.opB = OP_N;
  h.A = w.W; h.lda = r; h.B = A; h.ldb = n; h.C = T; h.ldc = n;
  h.alpha = mkc(1.f, 0.f); h.beta = mkc(0.f, 0.f);
  h.a_size = (long long)r * r; h.b_size = (long long)r * n; h.c_size = (long long)r * n;
  prof_begin(PH_ORTHGEMM, st);
  VB_TRY(gemm<float>(h, st));
  prof_end(PH_ORTHGEMM, st, 0.0);
  fill_flagged_kernel<<<grid_of((long long)r * n), 256, 0, st>>>(T, r, n, w.flag, seed);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status subspace_orth(cf *Q, int r, int n, const SubspaceWork &w, unsigned long long seed, cudaStream_t st) {
  if (r < 1 || r > SUBSPACE_MAX_R || n < r)
    return fail(VB_EINVAL, "subspace_orth: needs 1 <= r <= min(n, " + std::to_string(SUBSPACE_MAX_R) + ")");
  static std::atomic<bool> smem_set[64];  // per device; setting it twice is harmless
  int dev = 0;
  VB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(VB_EINVAL, "subspace_orth: device ordinal out of range");
  if (!smem_set[dev].load()) {
    VB_TRY_CUDA(cudaFuncSetAttribute(chol_rows_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)subspace_chol_smem(SUBSPACE_MAX_R)));
    smem_set[dev].store(true);
  }
  VB_TRY(orth_pass(Q, w.T, r, n, w, seed, st));
  VB_TRY(orth_pass(w.T, Q, r, n, w, seed ^ 0x5bd1e995ull, st));
  return VB_OK;
}

// ---- FP64 Cholesky factor for the orthonormalisations of the one-site sweep
// W (r x r) with W G W^+ = I on the accepted rows, from G (r x r, r <= 112):
// the same row-scaled elimination in FP64; only rows without a resolvable
// independent part (scaled pivot <= 1e-28, i.e. zero rows and exact
// dependencies) are rejected (zero row in W, flag[i] = 1, flag[r] = count):
// a row with any independent part keeps it, so that span(W A) contains every
// row of A (the caller's second pass restores orthogonality)
constexpr int CHOL64_MAX_R = 112;
size_t chol64_smem(int r) { return (size_t)r * r * sizeof(cd) + 2 * (size_t)r * sizeof(double); }

vb_status chol_w64(const cd *G, int r, cd *W, int *flag, cudaStream_t st) {
  if (r < 1 || r > CHOL64_MAX_R) return fail(VB_EINVAL, "chol_w64: needs 1 <= r <= 112");
  static std::atomic<bool> smem_set[64];  // per device; setting it twice is harmless
  int dev = 0;
  VB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(VB_EINVAL, "chol_w64: device ordinal out of range");
  if (!smem_set[dev].load()) {
    VB_TRY_CUDA(cudaFuncSetAttribute(chol_rows_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)chol64_smem(CHOL64_MAX_R)));
    smem_set[dev].store(true);
  }
  chol_rows_kernel<double><<<1, CHOL_THREADS, chol64_smem(r), st>>>(G, r, 1e-28, W, flag);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status subspace_status(const double *capt, const int *cnt, double *out, cudaStream_t st) {
  status_kernel<<<1, 1, 0, st>>>(capt, cnt, out);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

size_t ritz_jacobi_smem(int n) {
  const size_t np = n + (n & 1), h = np / 2;
  return 2 * np * np * sizeof(cf) + h * (sizeof(cf) + 2 * sizeof(float) + 2 * sizeof(int));
}

vb_status ritz_eig_small(const cf *S, int n, int k, float *evals, cf *W, int *info, cudaStream_t st) {
  if (n < 2 || n > JAC_MAX_N || k < 1 || k > n) return fail(VB_EINVAL, "ritz_eig_small: needs 2 <= n <= 112");
  static std::atomic<bool> smem_set[64];  // per device; setting it twice is harmless
  int dev = 0;
  VB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(VB_EINVAL, "ritz_eig_small: device ordinal out of range");
  if (!smem_set[dev].load()) {
    VB_TRY_CUDA(cudaFuncSetAttribute(ritz_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ritz_jacobi_smem(JAC_MAX_N)));
    smem_set[dev].store(true);
  }
  ritz_jacobi_kernel<<<1, JAC_THREADS, ritz_jacobi_smem(n), st>>>(S, n, k, evals, W, info);
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
