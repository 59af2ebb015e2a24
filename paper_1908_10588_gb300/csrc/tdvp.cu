// Two-site TDVP time stepping (Sec. 2.1.2) on the GPU: host orchestration
// of the kernels and the C ABI declared in include/vibtdvp.h.
//
// Data layout in device memory (all complex double, row-major):
//   site tensor A[p]      [m_{p-1}][d_p][m_p]          capacity bcap_{p} d_p bcap_{p+1}
//   left block  L[p]      [m_{p-1}][w_in(p)][m_{p-1}]  sites 0..p-1, first index bra
//   right block R[p]      [m_{p-1}][w_in(p)][m_{p-1}]  sites p..n-1, first index bra
//   two-site tensor       [m_{i-1}][d_i][d_{i+1}][m_{i+1}]
//   Krylov basis          (krylov_cap + 1) vectors of the largest two-site size
// bcap_b = min(m_cap, full dimension of bond b) bounds every bond.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include <thread>

#include "common.h"

using namespace vb;

namespace vb {
constexpr double HBAR_EV_FS = 0.6582119569;
constexpr double MULTIPLET_RTOL = 1e-10;
constexpr int MIXED_SPLIT_MIN_N = 192;
// subspace iteration of the mixed split: at most this many applications of
// rho; stop once the captured weight changes by less than this fraction
constexpr int SUBSPACE_MAXIT = 30;
constexpr double SUBSPACE_RTOL = 3e-7;

// H_eff products in split-TF32 on the tensor cores (k_mixed.cu); x_scale
// (nullable, device): x is multiplied by *x_scale on load
vb_status heff_mixed_apply(const vb_mpo *mpo, int site, int two_site, int mL, int mR, const cd *L,
                           const cd *R, const cd *x, cd *y, void *work, size_t work_bytes, int *err,
                           cudaStream_t st, const double *x_scale);
size_t heff_mixed_work_bytes(const vb_mpo *mpo, int site, int two_site, int mL, int mR);
int *heff_mixed_err_flag(const vb_mpo *mpo, int site, int two_site, int mL, int mR, void *work);

namespace {

__global__ void trace_kernel(const cd *rho, int n, double *out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += rho[(long long)i * n + i].x;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    out[0] = t;
  }
}

// dst[i*k + a] = src[a*n + i]
__global__ void transpose_kernel(const cd *src, int k, int n, cd *dst) {
  long long tot = (long long)k * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / k), a = (int)(e % k);
    dst[e] = src[(long long)a * n + i];
  }
}

// y += a x (a real)
__global__ void add_scaled_kernel(cd *__restrict__ y, const cd *__restrict__ x, double a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = mkc(y[i].x + a * x[i].x, y[i].y + a * x[i].y);
}

// x *= exp(-i phi)
__global__ void phase_kernel(cd *x, long long n, double phi) {
  double sn, cs;
  sincos(phi, &sn, &cs);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = mkc(cs * x[i].x + sn * x[i].y, cs * x[i].y - sn * x[i].x);
}

__global__ void conj_copy_kernel(const cd *src, long long n, cd *dst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = cconj(src[e]);
}

__global__ void c64_to_c32(const cd *__restrict__ x, cf *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = mkc<float>((float)x[i].x, (float)x[i].y);
}

__global__ void c32_to_c64(const cf *__restrict__ x, cd *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = mkc<double>((double)x[i].x, (double)x[i].y);
}

// G <- (3 I - G) / 2 (one Lowdin step towards G^{-1/2} for G close to I)
__global__ void lowdin_kernel(cd *G, int r) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
    const int i = e / r, j = e % r;
    cd g = G[e];
    G[e] = mkc((i == j ? 1.5 : 0.0) - 0.5 * g.x, -0.5 * g.y);
  }
}

// w[i] = |row i of X|^2 (X is kws x len, or len x kws when rows == 0: columns)
__global__ void ritz_weights_kernel(const cd *__restrict__ X, int kws, int len, int rows, double *w) {
  __shared__ double sh[8];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int x = threadIdx.x; x < len; x += blockDim.x) s += cabs2(rows ? X[(long long)i * len + x] : X[(long long)x * kws + i]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += sh[j];
    w[i] = t;
  }
}

// rows perm[0..k) of src (rows of length len): mode 0 writes them as the
// columns of dst (len x k), mode 1 as rows (k x len), mode 2 as conjugated rows
__global__ void ritz_gather_kernel(const cd *__restrict__ src, int len, const int *__restrict__ perm, int k, int mode,
                                   cd *__restrict__ dst) {
  const long long tot = (long long)k * len;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    if (mode == 0) {
      const int x = (int)(e / k), j = (int)(e % k);
      dst[e] = src[(long long)perm[j] * len + x];
    } else {
      const int j = (int)(e / len), x = (int)(e % len);
      const cd v = src[(long long)perm[j] * len + x];
      dst[e] = mode == 2 ? cconj(v) : v;
    }
  }
}

// entries of the rows (cols == 0) or columns (cols == 1) flagged in flag[] of
// an r x n (rows) or n x r (columns) row-major matrix get counter-based random
// values (splitmix64 finaliser) in [-1, 1)
__device__ __forceinline__ double urand64(unsigned long long seed, unsigned long long idx) {
  unsigned long long z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void fill_flagged64(cd *__restrict__ Q, int r, long long n, int cols, const int *__restrict__ flag,
                               unsigned long long seed) {
  const long long tot = (long long)r * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int j = cols ? (int)(e % r) : (int)(e / n);
    if (flag[j]) Q[e] = mkc(urand64(seed, 2ull * e), urand64(seed, 2ull * e + 1));
  }
}

// FP64 copy of the FP32 basis rows, conjugated when conj != 0
__global__ void subspace_rows_c64(const cf *__restrict__ q, cd *__restrict__ out, long long n, int conj) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cf a = q[i];
    out[i] = mkc((double)a.x, conj ? -(double)a.y : (double)a.y);
  }
}

__global__ void populations_kernel(const cd *C, int d, int mR, double *out) {
  // C[0][s][b]: P_s = sum_b |C[s,b]|^2 / sum |C|^2 ; one warp per s, then normalise
  __shared__ double ps[64];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int s = w; s < d; s += nw) {
    double a = 0.0;
    for (int b = lane; b < mR; b += 32) a += cabs2(C[(long long)s * mR + b]);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) ps[s] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int s = 0; s < d; ++s) t += ps[s];
    for (int s = 0; s < d; ++s) out[s] = ps[s] / t;
  }
}

__global__ void populations_proj_kernel(const cd *A, const cd *X, int me, int d, int mr, double *out) {
  // P_k = Re sum_{x', y} conj(A[x', k, y]) X[x', k, y] / sum over k; one warp per k
  __shared__ double ps[64];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long rows = (long long)me * mr;
  for (int k = w; k < d; k += nw) {
    double a = 0.0;
    for (long long r = lane; r < rows; r += 32) {
      const long long o = (r / mr) * d * mr + (long long)k * mr + r % mr;
      const cd u = A[o], v = X[o];
      a += u.x * v.x + u.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) ps[k] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < d; ++k) t += ps[k];
    for (int k = 0; k < d; ++k) out[k] = ps[k] / t;
  }
}

inline int grid1(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  return (int)std::max(1LL, b);
}

long long full_dim(const std::vector<int> &dims, int lo, int hi, long long cap) {
  // product of dims[lo..hi) saturated at cap
  long long p = 1;
  for (int i = lo; i < hi; ++i) {
    p *= dims[i];
    if (p >= cap) return cap;
  }
  return p;
}

}  // namespace
}  // namespace vb

struct vb_mps {
  int n = 0;
  int dtype = VB_FP64;
  int m_cap = 0;
  int kcap = 40;
  int device = -1;
  cudaStream_t st = nullptr;
  vb::Alloc alloc;
  const vb_mpo *mpo = nullptr;
  std::vector<int> dims;
  std::vector<int> bond;   // bond[p] = left bond of site p; bond[0] = bond[n] = 1
  std::vector<int> bcap;   // capacity per bond
  std::vector<cd *> A, L, R;
  cd *theta = nullptr, *V = nullptr, *T1 = nullptr, *T2 = nullptr, *rho = nullptr, *Z = nullptr;
  cf *V32 = nullptr, *w32 = nullptr;  // mixed form: FP32 copies of the Krylov vectors and of w
  void *eigw = nullptr;
  void *mixw = nullptr;
  size_t mixw_bytes = 0;
  long long theta_cap = 0, inter_cap = 0, nrho_cap = 0;
  int kw_cap = 0;
  // device scalars
  double *d_vs = nullptr;  // mixed Lanczos: factors that normalise the stored basis vectors
  double *d_nrm = nullptr, *d_alpha = nullptr, *d_beta = nullptr, *d_bnext = nullptr,
         *d_evals = nullptr, *d_trace = nullptr, *d_part = nullptr, *d_pop = nullptr;
  cd *d_c = nullptr, *d_c2 = nullptr, *d_u = nullptr, *d_partc = nullptr;
  double *h_flag = nullptr, *d_flag = nullptr;  // mapped: [0] err, [1] beta_next
  int *d_tcerr = nullptr;                        // raised by a tensor-core kernel whose wait ran out
  unsigned int *d_cnt = nullptr;                 // zeroed block counters of the last-block reductions
  std::vector<int> khint;                        // Krylov steps of the last call per operator
  // one-site sweep (allocated on its first use)
  bool t1_ready = false;
  cd *q_G = nullptr, *q_W = nullptr, *q_Q = nullptr, *q_Rm = nullptr, *q_ws = nullptr;
  long long q_ws_elems = 0;
  int *q_flag = nullptr;
  // subspace iteration of the mixed split
  cf *subZ = nullptr, *subT = nullptr, *subG = nullptr, *subW = nullptr, *skws32 = nullptr;
  long long skws32_elems = 0;
  int *subflag = nullptr, *d_perm = nullptr;
  double *d_capt = nullptr;
  float *ev32 = nullptr;
  void *eigw32 = nullptr;
  unsigned long long split_calls = 0;
  // mixed split: FP32 subspace iteration and Ritz vectors, FP64 basis, projection and weights
  int rcap = 0;
  cf *M32 = nullptr, *Q32 = nullptr;
  cd *Q64 = nullptr, *Qo = nullptr, *G = nullptr, *X = nullptr;
  cd *skws = nullptr;  // split-K workspace of the FP64 projection products
  long long skws_elems = 0;
  // mixed form: environment updates in complex FP32
  cf *envA32 = nullptr, *envE32 = nullptr, *envO32 = nullptr, *envT1 = nullptr, *envT2 = nullptr;
  cf *mrgB32 = nullptr;  // mixed merge: FP32 copy of the right site tensor (the left one goes to envA32)
  long long env_site_cap = 0, env_blk_cap = 0;
  std::vector<void *> owned;
  int center = 0;
};

namespace vb {
namespace {

vb_status mps_alloc(vb_mps *s, void **p, size_t bytes) {
  VB_TRY(s->alloc.get(p, bytes));
  s->owned.push_back(*p);
  return VB_OK;
}

struct Ctx {
  vb_mps *s;
  const vb_mpo *mpo;
  cudaStream_t st;
};

// ---- H_eff,2 theta (Eq. two-site Hamiltonian), FP64 path
// T1 and T2 each hold at least max(w_in(i), w_out(i), w_out(i+1)) * |theta| elements.
vb_status heff2_fp64(const vb_mpo *mpo, int i, int mL, int mR, const cd *L, const cd *R,
                     const cd *x, cd *y, cd *T1, cd *T2, long long t_cap, cudaStream_t st) {
  const MpoSite &Si = mpo->sites[i], &Sj = mpo->sites[i + 1];
  const long long d1 = Si.d, d2 = Sj.d, wL = Si.wl, wM = Si.wr, wR = Sj.wr;
  const long long th = mL * d1 * d2 * mR, Q1 = d2 * mR;
  // T1[(a' w0), (s t b)] = L[(a' w0), a] x[a, (s t b)]
  GemmArgs g{};
  g.M = (int)(mL * wL); g.N = (int)(d1 * Q1); g.K = mL; g.batch = 1;
  g.opA = OP_N; g.opB = OP_N;
  g.A = L; g.lda = mL; g.B = x; g.ldb = g.N; g.C = T1; g.ldc = g.N;
  g.alpha = mkc(1.0, 0.0); g.beta = mkc(0.0, 0.0);
  g.a_size = mL * wL * mL; g.b_size = th; g.c_size = t_cap;
  VB_TRY(zgemm(g, st));
  // T2[a'][s'][w1][(t b)] = W_i applied to T1[a'][w0][s][(t b)]
  VB_TRY(wapply(Si, 0, T1, WS(/*p*/ wL * d1 * Q1, /*w*/ d1 * Q1, /*s*/ Q1, /*q*/ 1), t_cap, T2,
                WS(/*p*/ d1 * wM * Q1, /*w*/ Q1, /*s*/ wM * Q1, /*q*/ 1), t_cap, mL, (int)Q1, st));
  // T3[(a' s')][t'][w2][b] = W_{i+1} applied to T2[(a' s')][w1][t][b]   (T3 reuses T1)
  VB_TRY(wapply(Sj, 0, T2, WS(/*p*/ wM * d2 * mR, /*w*/ d2 * mR, /*s*/ mR, /*q*/ 1), t_cap, T1,
                WS(/*p*/ d2 * wR * mR, /*w*/ mR, /*s*/ wR * mR, /*q*/ 1), t_cap, (int)(mL * d1), mR, st));
  // y[(a' s' t'), b'] = T3[(a' s' t'), (w2 b)] R[b', (w2 b)]^T
  GemmArgs h{};
  h.M = (int)(mL * d1 * d2); h.N = mR; h.K = (int)(wR * mR); h.batch = 1;
  h.opA = OP_N; h.opB = OP_T;
  h.A = T1; h.lda = h.K; h.B = R; h.ldb = h.K; h.C = y; h.ldc = mR;
  h.alpha = mkc(1.0, 0.0); h.beta = mkc(0.0, 0.0);
  h.a_size = t_cap; h.b_size = (long long)mR * wR * mR; h.c_size = th;
  return zgemm(h, st);
}

// ---- H_eff,1 C (Eq. one-site Hamiltonian 1), FP64 path
vb_status heff1_fp64(const vb_mpo *mpo, int j, int mL, int mR, const cd *L, const cd *R,
                     const cd *x, cd *y, cd *T1, cd *T2, long long t_cap, cudaStream_t st) {
  const MpoSite &S = mpo->sites[j];
  const long long d = S.d, wL = S.wl, wR = S.wr;
  GemmArgs g{};
  g.M = (int)(mL * wL); g.N = (int)(d * mR); g.K = mL; g.batch = 1;
  g.opA = OP_N; g.opB = OP_N;
  g.A = L; g.lda = mL; g.B = x; g.ldb = g.N; g.C = T1; g.ldc = g.N;
  g.alpha = mkc(1.0, 0.0); g.beta = mkc(0.0, 0.0);
  g.a_size = mL * wL * mL; g.b_size = mL * d * mR; g.c_size = t_cap;
  VB_TRY(zgemm(g, st));
  // T2[a'][t'][w1][b] = W applied to T1[a'][w0][t][b]
  VB_TRY(wapply(S, 0, T1, WS(/*p*/ wL * d * mR, /*w*/ d * mR, /*s*/ mR, /*q*/ 1), t_cap, T2,
                WS(/*p*/ d * wR * mR, /*w*/ mR, /*s*/ wR * mR, /*q*/ 1), t_cap, mL, mR, st));
  GemmArgs h{};
  h.M = (int)(mL * d); h.N = mR; h.K = (int)(wR * mR); h.batch = 1;
  h.opA = OP_N; h.opB = OP_T;
  h.A = T2; h.lda = h.K; h.B = R; h.ldb = h.K; h.C = y; h.ldc = mR;
  h.alpha = mkc(1.0, 0.0); h.beta = mkc(0.0, 0.0);
  h.a_size = t_cap; h.b_size = (long long)mR * wR * mR; h.c_size = mL * d * mR;
  return zgemm(h, st);
}

// ---- environment updates (the blocks of Eq. one-site Hamiltonian 1)
template <class R>
vb_status env_left(const vb_mpo *mpo, int p, int mL, int mR, const cplx<R> *L, const cplx<R> *A, cplx<R> *Lnew,
                   cplx<R> *T1, cplx<R> *T2, long long t_cap, cudaStream_t st) {
  const MpoSite &S = mpo->sites[p];
  const long long d = S.d, wL = S.wl, wR = S.wr;
  // T1[(x w), (s y)] = L[(x w), z] A[z, (s y)]
  GemmArgsT<R> g{};
  g.M = (int)(mL * wL); g.N = (int)(d * mR); g.K = mL; g.batch = 1;
  g.opA = OP_N; g.opB = OP_N;
  g.A = L; g.lda = mL; g.B = A; g.ldb = g.N; g.C = T1; g.ldc = g.N;
  g.alpha = mkc<R>(1, 0); g.beta = mkc<R>(0, 0);
  g.a_size = mL * wL * mL; g.b_size = mL * d * mR; g.c_size = t_cap;
  VB_TRY(gemm<R>(g, st));
  // T2[x][s'][v][y] = W applied to T1[x][w][s][y]
  VB_TRY(wapply<R>(S, 0, T1, WS(/*p*/ wL * d * mR, /*w*/ d * mR, /*s*/ mR, /*q*/ 1), t_cap, T2,
                WS(/*p*/ d * wR * mR, /*w*/ mR, /*s*/ wR * mR, /*q*/ 1), t_cap, mL, mR, st));
  // Lnew[y', (v y)] = sum_{(x s')} conj(A[(x s'), y']) T2[(x s'), (v y)]
  GemmArgsT<R> h{};
  h.M = mR; h.N = (int)(wR * mR); h.K = (int)(mL * d); h.batch = 1;
  h.opA = OP_C; h.opB = OP_N;
  h.A = A; h.lda = mR; h.B = T2; h.ldb = h.N; h.C = Lnew; h.ldc = h.N;
  h.alpha = mkc<R>(1, 0); h.beta = mkc<R>(0, 0);
  h.a_size = mL * d * mR; h.b_size = t_cap; h.c_size = (long long)mR * wR * mR;
  return gemm<R>(h, st);
}

template <class Rt>
vb_status env_right(const vb_mpo *mpo, int p, int mL, int mR, const cplx<Rt> *R, const cplx<Rt> *B, cplx<Rt> *Rnew,
                    cplx<Rt> *T1, cplx<Rt> *T2, long long t_cap, cudaStream_t st) {
  const MpoSite &S = mpo->sites[p];
  const long long d = S.d, wL = S.wl, wR = S.wr;
  // T1[(a t)][v][y] = sum_z B[(a t), z] R[y, v, z]   (batched over v)
  GemmArgsT<Rt> g{};
  g.M = (int)(mL * d); g.N = mR; g.K = mR; g.batch = (int)wR;
  g.opA = OP_N; g.opB = OP_T;
  g.A = B; g.lda = mR; g.sA = 0;
  g.B = R; g.ldb = wR * mR; g.sB = mR;
  g.C = T1; g.ldc = wR * mR; g.sC = mR;
  g.alpha = mkc<Rt>(1, 0); g.beta = mkc<Rt>(0, 0);
  g.a_size = mL * d * mR; g.b_size = (long long)mR * wR * mR; g.c_size = t_cap;
  VB_TRY(gemm<Rt>(g, st));
  // T2[a][w][t'][y] = sum_{t, v} W[w, t', t, v] T1[a][t][v][y]
  VB_TRY(wapply<Rt>(S, 1, T1, WS(/*p*/ d * wR * mR, /*w*/ mR, /*s*/ wR * mR, /*q*/ 1), t_cap, T2,
                WS(/*p*/ wL * d * mR, /*w*/ d * mR, /*s*/ mR, /*q*/ 1), t_cap, mL, mR, st));
  // Rnew[a', w, a] = sum_k conj(B[a', k]) T2[a, w, k]   (batched over w)
  GemmArgsT<Rt> h{};
  h.M = mL; h.N = mL; h.K = (int)(d * mR); h.batch = (int)wL;
  h.opA = OP_R; h.opB = OP_T;
  h.A = B; h.lda = d * mR; h.sA = 0;
  h.B = T2; h.ldb = wL * d * mR; h.sB = d * mR;
  h.C = Rnew; h.ldc = wL * mL; h.sC = mL;
  h.alpha = mkc<Rt>(1, 0); h.beta = mkc<Rt>(0, 0);
  h.a_size = mL * d * mR; h.b_size = t_cap; h.c_size = (long long)mL * wL * mL;
  return gemm<Rt>(h, st);
}

// ---- operator applied inside the Krylov loop
struct HeffOp {
  int two_site;  // 1: two-site, 0: one-site, -1: zero-site (bond between site and site + 1)
  int site;
  int mL, mR;
  const cd *L, *R;
};

// algorithmic floating-point operations of one W-site application to
// `outer` stacked vectors: a non-identity d x d block costs 4 d^2 per vector
// (real operator times complex data), an identity block 2 d
double wsite_flops(const MpoSite &S, double outer) {
  double f = 0.0;
  for (const MpoBlock &B : S.blocks) f += B.ident ? 2.0 * S.d : 4.0 * S.d * S.d;
  return f * outer;
}

double heff_flops(const vb_mpo *mpo, int site, int two_site, int mL, int mR) {
  const MpoSite &S = mpo->sites[site];
  if (two_site) {
    const MpoSite &S2 = mpo->sites[site + 1];
    return heff2_flops_of(mL, mR, S.d, S2.d, S.wl, S2.wr, S.nnz_ops, S.n_ident, S2.nnz_ops, S2.n_ident);
  }
  const double c = (double)mL * S.d * mR;
  return 8.0 * c * mL * S.wl + wsite_flops(S, (double)mL * mR) + 8.0 * c * S.wr * mR;
}

// ---- H_eff,0 X for the bond matrix X (m_a x m_b) between site and site + 1
// (zero-site Hamiltonian of the one-site sweep): T[(a' w), b] = L[(a' w), a] X[a, b],
// y[a', b'] = sum_{(w b)} T[a', (w b)] R[b', (w b)]; two complex FP64 GEMMs
vb_status heff0_fp64(const vb_mpo *mpo, int site, int ma, int mb, const cd *L, const cd *R, const cd *x, cd *y,
                     cd *T, long long t_cap, cd *ws, long long ws_elems, cudaStream_t st) {
  const long long w = mpo->sites[site].wr;
  GemmArgs g{};
  g.M = (int)(ma * w); g.N = mb; g.K = ma; g.batch = 1;
  g.opA = OP_N; g.opB = OP_N;
  g.A = L; g.lda = ma; g.B = x; g.ldb = mb; g.C = T; g.ldc = mb;
  g.alpha = mkc(1.0, 0.0); g.beta = mkc(0.0, 0.0);
  g.a_size = ma * w * ma; g.b_size = (long long)ma * mb; g.c_size = t_cap;
  VB_TRY(zgemm(g, st));
  GemmArgs h{};
  h.M = ma; h.N = mb; h.K = (int)(w * mb); h.batch = 1;
  h.opA = OP_N; h.opB = OP_T;
  h.A = T; h.lda = w * mb; h.B = R; h.ldb = w * mb; h.C = y; h.ldc = mb;
  h.alpha = mkc(1.0, 0.0); h.beta = mkc(0.0, 0.0);
  h.a_size = t_cap; h.b_size = (long long)mb * w * mb; h.c_size = (long long)ma * mb;
  h.ws = ws; h.ws_elems = ws_elems;  // one output tile, K = w m: split-K
  return zgemm(h, st);
}

// The mixed form's FP32 operators leave out the zero-point constant e_zpe of
// the Hamiltonian (vb_mpo::e_zpe); a mixed sweep of length dt restores it as
// the exact global phase exp(-i e_zpe dt / hbar) on the center (site 0).
vb_status zero_point_phase(vb_mps *s, double dt_fs) {
  if (s->dtype != VB_MIXED || s->mpo->e_zpe == 0.0) return VB_OK;
  const long long el = (long long)s->bond[0] * s->dims[0] * s->bond[1];
  phase_kernel<<<grid1(el), 256, 0, s->st>>>(s->A[0], el, s->mpo->e_zpe * dt_fs / HBAR_EV_FS);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

// Reads the flag a mixed-form tensor-core kernel raises when one of its
// bounded waits runs out, and clears it once reported, so that the error is
// neither lost nor blamed on a later call. Synchronises the handle's stream.
vb_status take_wait_flag(vb_mps *s, const char *who) {
  if (s->dtype != VB_MIXED) return VB_OK;
  int flag = 0;
  VB_TRY_CUDA(cudaMemcpyAsync(&flag, s->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  VB_TRY_CUDA(cudaStreamSynchronize(s->st));
  if (!flag) return VB_OK;
  VB_TRY_CUDA(cudaMemsetAsync(s->d_tcerr, 0, sizeof(int), s->st));
  VB_TRY_CUDA(cudaStreamSynchronize(s->st));
  return fail(VB_ETIMEOUT, std::string(who) + ": a tensor-core kernel's wait ran out (results invalid)");
}

// x_scale (nullable, device; mixed two- and one-site products only): x is
// stored unnormalised and multiplied by *x_scale on load
vb_status apply_heff(vb_mps *s, const HeffOp &op, const cd *x, cd *y, const double *x_scale = nullptr) {
  if (op.two_site < 0)  // zero-site (bond) Hamiltonian: FP64 in both forms
    return x_scale ? fail(VB_EINVAL, "apply_heff: no input scale for the zero-site product")
                   : heff0_fp64(s->mpo, op.site, op.mL, op.mR, op.L, op.R, x, y, s->T1, s->inter_cap, s->q_ws,
                                s->q_ws_elems, s->st);
  const int ph = op.two_site ? PH_HEFF2 : PH_HEFF1;
  prof_begin(ph, s->st);
  vb_status r;
  if (s->dtype == VB_MIXED)
    r = heff_mixed_apply(s->mpo, op.site, op.two_site, op.mL, op.mR, op.L, op.R, x, y, s->mixw,
                         s->mixw_bytes, s->d_tcerr, s->st, x_scale);
  else if (x_scale)
    r = fail(VB_EINVAL, "apply_heff: input scale only in the mixed form");
  else if (op.two_site)
    r = heff2_fp64(s->mpo, op.site, op.mL, op.mR, op.L, op.R, x, y, s->T1, s->T2, s->inter_cap, s->st);
  else
    r = heff1_fp64(s->mpo, op.site, op.mL, op.mR, op.L, op.R, x, y, s->T1, s->T2, s->inter_cap, s->st);
  prof_end(ph, s->st, prof_on() ? heff_flops(s->mpo, op.site, op.two_site, op.mL, op.mR) : 0.0);
  return r;
}

// ---- x <- exp(-i H dt/hbar) x by Lanczos with full re-orthogonalisation
vb_status krylov_expm(vb_mps *s, const HeffOp &op, cd *x, long long N, double dt_fs, int kmax,
                      double tol, int *iters, int *converged) {
  cudaStream_t st = s->st;
  // convergence is checked (small exponential + host wait) from two steps
  // before the count the previous call for the same operator needed; the
  // steps before run without a host wait. Checking later only adds steps,
  // which makes the result more accurate, never less.
  const size_t hk = (size_t)(op.two_site + 1) * (s->n + 1) + op.site;
  if (s->khint.size() < (size_t)3 * (s->n + 1)) s->khint.assign((size_t)3 * (s->n + 1), 0);
  const int check_from = std::max(1, s->khint[hk] - 2);
  const int np = reduce_parts(N);
  const long long ldv = s->theta_cap;
  cd *V = s->V;
  kmax = (int)std::min<long long>(std::min(kmax, s->kcap), N);
  const double tau = dt_fs / HBAR_EV_FS;
  const bool mixed = s->dtype == VB_MIXED;
  cf *V32 = mixed ? s->V32 : nullptr;
  // mixed two- and one-site products: v_{k+1} is kept as the unnormalised w
  // (FP64 and FP32 copy) and vs[k+1] = 1/|w|; the H_eff product, the
  // Gram-Schmidt kernels and the final combination apply the factor, so no
  // pass rescales the vector (vs[0] = 1: v_0 is normalised explicitly)
  const bool defer = mixed && op.two_site >= 0;
  const double *vs = defer ? s->d_vs : nullptr;
  prof_begin(PH_KRYLOV, st);
  VB_TRY(vec_norm2(x, N, s->d_nrm, s->d_part, np, st));
  VB_TRY(vec_copy_scaled(x, V, N, st));
  VB_TRY(vec_scale_inv(V, N, s->d_nrm, st, nullptr, nullptr, nullptr, nullptr, V32));
  // algorithmic FP64 flops: a complex multiply-add counts 8, |z|^2 counts 4
  const double Nd = (double)N;
  prof_end(PH_KRYLOV, st, 4.0 * Nd + 2.0 * Nd);
  int kdim = 0;
  *converged = 0;
  for (int k = 0; k < kmax; ++k) {
    cd *w = V + (k + 1) * ldv;
    VB_TRY(apply_heff(s, op, V + k * ldv, w, defer ? s->d_vs + k : nullptr));
    prof_begin(PH_KRYLOV, st);
    double kbytes = 0.0;
    if (mixed) {
      // Gram-Schmidt on the FP32 copies of the vectors (FP32 products, FP64
      // sums, FP32 corrections added to the FP64 w): w = H v_k comes from the
      // FP32 tensor-core product and is only FP32-accurate itself, so FP32
      // arithmetic here adds no error beyond it. A first pass against v_{k-1},
      // v_k (the three-term recurrence: alpha_k, beta_k), then one full pass,
      // which only removes components of the size of that FP32 error and so
      // loses no orthogonality to cancellation.
      const int j0 = k > 0 ? k - 1 : 0;
      const int n1 = k + 1 - j0;
      // bandwidth-bound: more, smaller partial blocks than the FP64 dots use
      const int np32 = (int)std::min<long long>(608, std::max<long long>(1, (N + 1023) / 1024));
      const double *vs1 = vs ? vs + j0 : nullptr;
      // first pass: inner products with w rounded to FP32 on load
      VB_TRY(vec_multi_dot32(V32 + j0 * ldv, ldv, n1, w, N, s->d_c + j0, s->d_partc, np32, st, s->d_cnt, vs1));
      if (axpy_dot32_blocks(N, k + 1, PARTC_ELEMS)) {
        // its update fused with the full pass's inner products
        VB_TRY(vec_axpy_dot32(V32 + j0 * ldv, n1, s->d_c + j0, -1.0, w, N, V32, ldv, k + 1, s->d_c2, s->d_partc,
                              PARTC_ELEMS, st, s->d_cnt, vs1, vs));
      } else {
        VB_TRY(vec_multi_axpy32(V32 + j0 * ldv, ldv, n1, s->d_c + j0, -1.0, w, N, s->w32, st, vs1));
        VB_TRY(vec_multi_dot32(V32, ldv, k + 1, s->w32, N, s->d_c2, s->d_partc, np32, st, s->d_cnt, vs));
      }
      // full-pass update and |w|; deferred: also the FP32 copy of w as the
      // stored copy of v_{k+1}, its factor 1/|w|, beta and alpha of step k
      LanczosRecord rec{};
      if (defer) rec = LanczosRecord{s->d_vs + k + 1, s->d_beta + k, s->d_alpha + k, s->d_c + k, s->d_c2 + k};
      VB_TRY(vec_multi_axpy32_norm(V32, ldv, k + 1, s->d_c2, -1.0, w, N, s->d_bnext, s->d_part, st,
                                   s->d_cnt + 32, vs, defer ? V32 + (k + 1) * ldv : nullptr, rec));
      // algorithmic bytes: first-pass inner products (w read, copies of
      // v_{k-1}, v_k read), fused update + inner products (w read and
      // written, the two copies and all k+1 copies read), full-pass update
      // (copies read, w read and written, deferred: the FP32 copy written)
      kbytes = (double)N * (16.0 + 8.0 * n1 + 32.0 + 8.0 * n1 + 8.0 * (k + 1) + 8.0 * (k + 1) + 32.0 +
                            (defer ? 8.0 : 0.0));
    } else {
      // FP64-pipe-bound: one partial block per 512 elements up to four per SM
      const int np64 = (int)std::min<long long>(608, std::max<long long>(1, (N + 511) / 512));
      VB_TRY(vec_multi_dot(V, ldv, k + 1, w, N, s->d_c, s->d_partc, np64, st, s->d_cnt));
      VB_TRY(vec_multi_axpy(V, ldv, k + 1, s->d_c, -1.0, w, N, st));
      VB_TRY(vec_multi_dot(V, ldv, k + 1, w, N, s->d_c2, s->d_partc, np64, st, s->d_cnt));
      VB_TRY(vec_multi_axpy_norm(V, ldv, k + 1, s->d_c2, -1.0, w, N, s->d_bnext, s->d_part, st, s->d_cnt + 32));
    }

    const bool check = k + 1 >= check_from || k + 1 == kmax;
    if (check)
      VB_TRY(tridiag_expm(s->d_c, s->d_c2, s->d_alpha, s->d_beta, k + 1, tau, s->d_bnext, s->d_u, s->d_flag, st));
    {
      const double nv1 = mixed ? (double)(k > 0 ? 2 : 1) : (double)(k + 1);
      prof_end(PH_KRYLOV, st, Nd * (16.0 * (nv1 + k + 1) + 4.0), kbytes);
    }
    kdim = k + 1;
    if (check) {
      VB_TRY_CUDA(cudaStreamSynchronize(st));
      const double err = s->h_flag[0], b = s->h_flag[1];
      if (!(err == err) || !(b == b)) return fail(VB_ECUDA, "krylov: NaN in the Lanczos recurrence");
      if (err < tol || b <= 1e-300 || k + 1 == N) {
        *converged = 1;
        break;
      }
    }
    if (!defer) {
      prof_begin(PH_KRYLOV, st);
      // v_{k+1} = w / beta_{k+1}; also records beta_{k+1} and alpha_k
      VB_TRY(vec_scale_inv(w, N, s->d_bnext, st, s->d_beta + k, s->d_c + k, s->d_c2 + k, s->d_alpha + k,
                           mixed ? V32 + (k + 1) * ldv : nullptr));
      prof_end(PH_KRYLOV, st, 2.0 * Nd);
    }
  }
  *iters = kdim;
  if (*converged) s->khint[hk] = kdim;
  prof_begin(PH_KRYLOV, st);
  VB_TRY(vec_combine(V, ldv, kdim, s->d_u, s->d_nrm, x, N, st, vs));
  prof_end(PH_KRYLOV, st, 8.0 * Nd * kdim);
  return VB_OK;
}

struct TruncOpts {
  int m_max;
  double eps, floor;
};

// number of kept Schmidt directions (DBSS / fixed M, Sec. 2.1.1) from the
// kw largest eigenvalues lam (descending) of an n x n reduced density matrix
// with trace tot; rank_bound bounds the Schmidt rank. Sets *disc to the
// relative discarded weight.
int choose_rank(const std::vector<double> &lam, int n, double tot, int rank_bound,
                const TruncOpts &o, double *disc) {
  const int kw = (int)lam.size();
  int k = std::min(n, rank_bound);
  if (o.floor > 0.0) {
    int c = 0;
    while (c < kw && lam[c] > o.floor * tot) ++c;
    if (c < kw || kw == n) k = std::min(k, c);
  }
  std::vector<double> prefix(kw + 1, 0.0);
  for (int j = 0; j < kw; ++j) prefix[j + 1] = prefix[j] + lam[j];
  if (o.eps > 0.0) {
    int kk = n;
    for (int j = 0; j <= kw; ++j)
      if (tot - prefix[j] <= o.eps * tot) {
        kk = j;
        break;
      }
    k = std::min(k, kk);
  }
  k = std::min(k, o.m_max);
  k = std::max(k, 1);
  while (k > 1 && k < n && k < kw && (lam[k - 1] - lam[k]) < MULTIPLET_RTOL * lam[k - 1]) --k;
  *disc = tot > 0.0 ? (tot - prefix[std::min(k, kw)]) / tot : 0.0;
  if (*disc < 0.0) *disc = 0.0;
  return k;
}

// theta (mL d1 x d2 mR) -> left-orthonormal A_i (into dstA) and C (into dstC),
// or (right) C (dstA) and right-orthonormal B (dstC). Returns the new bond.
vb_status split_mixed(vb_mps *s, bool left, int mL, int d1, int d2, int mR, int m_old, const TruncOpts &o,
                      cd *dstA, cd *dstC, int *k_out, double *disc);
vb_status qr_cols(vb_mps *s, const cd *M, long long n1, int m, cd *Q, cd *Rm, unsigned long long seed);
vb_status lq_rows(vb_mps *s, const cd *Cm, int m, long long n2, cd *Q, cd *Rm, unsigned long long seed);
vb_status tdvp1_setup(vb_mps *s);

// The same split from the Gram matrix of the other, smaller side (FP64),
// for pairs whose two sides differ much in size (a small-basis site next to
// a large one): the Schmidt vectors of the small side come from its
// eigenvectors, the large side's are theta applied to them, orthonormalised
// by Cholesky QR done twice, and the bond tensor is theta projected on those.
// Mathematically the same truncation as the eigenvectors of the large side's
// rho; the eigenproblem is only min(n1, n2) wide.
vb_status split_small_side(vb_mps *s, bool left, int n1, int n2, const TruncOpts &o, cd *dstA, cd *dstC,
                           int *k_out, double *disc) {
  cudaStream_t st = s->st;
  const int ns = left ? n2 : n1;
  const cd *M = s->theta;
  const cd one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  auto G64 = [&](int Mm, int Nn, int Kk, int opA, const cd *A, long long lda, long long asz, int opB, const cd *B,
                 long long ldb, long long bsz, cd *C, long long ldc, long long csz) {
    GemmArgs g{};
    g.M = Mm; g.N = Nn; g.K = Kk; g.batch = 1; g.opA = opA; g.opB = opB;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    g.alpha = one; g.beta = zero; g.a_size = asz; g.b_size = bsz; g.c_size = csz;
    g.ws = s->skws; g.ws_elems = s->skws_elems;
    return zgemm(g, st);
  };
  const long long nm = (long long)n1 * n2, rs = (long long)s->nrho_cap * s->nrho_cap;
  prof_begin(PH_RHO, st);
  if (left)  // rho_s = M^+ M (n2 x n2)
    VB_TRY(G64(ns, ns, n1, OP_C, M, n2, nm, OP_N, M, n2, nm, s->rho, ns, rs));
  else  // rho_s = M M^+ (n1 x n1)
    VB_TRY(G64(ns, ns, n2, OP_N, M, n2, nm, OP_C, M, n2, nm, s->rho, ns, rs));
  trace_kernel<<<1, 256, 0, st>>>(s->rho, ns, s->d_trace);
  VB_CHECK_LAUNCH();
  prof_end(PH_RHO, st, 0.0);
  const int kw = std::min(ns, o.m_max + 1);
  prof_begin(PH_EIGVAL, st);
  VB_TRY(eig_values(ns, s->rho, kw, s->d_evals, s->eigw, st));
  prof_end(PH_EIGVAL, st, 0.0);
  std::vector<double> lam(kw);
  double tot = 0.0;
  VB_TRY_CUDA(cudaMemcpyAsync(lam.data(), s->d_evals, kw * sizeof(double), cudaMemcpyDeviceToHost, st));
  VB_TRY_CUDA(cudaMemcpyAsync(&tot, s->d_trace, sizeof(double), cudaMemcpyDeviceToHost, st));
  VB_TRY_CUDA(cudaStreamSynchronize(st));
  VB_TRY(EigWork::check(ns, kw, sizeof(double), s->eigw, st));
  const int k = choose_rank(lam, ns, tot, ns, o, disc);
  prof_begin(PH_EIGVEC, st);
  VB_TRY(eig_vectors(ns, s->rho, kw, k, s->d_evals, s->Z, s->eigw, st));
  prof_end(PH_EIGVEC, st, 0.0);
  prof_begin(PH_SPLITOUT, st);
  const unsigned long long seed = 0x452821E638D01377ull + 0x9E3779B97F4A7C15ull * (++s->split_calls);
  cd *Y = s->X;
  if (left) {
    // rows z_j of Z: right vectors conj(z_j); Y = M Z^T (n1 x k) has columns
    // sigma_j u_j; A = Q of Y, C = A^+ M
    VB_TRY(G64(n1, k, n2, OP_N, M, n2, nm, OP_T, s->Z, ns, (long long)k * ns, Y, k, (long long)n1 * k));
    VB_TRY(qr_cols(s, Y, n1, k, dstA, s->q_Rm, seed));
    VB_TRY(G64(k, n2, n1, OP_C, dstA, k, (long long)n1 * k, OP_N, M, n2, nm, dstC, n2, (long long)k * n2));
    const long long nc = (long long)k * n2;
    VB_TRY(vec_norm2(dstC, nc, s->d_nrm, s->d_part, reduce_parts(nc), st));
    VB_TRY(vec_scale_inv(dstC, nc, s->d_nrm, st));
  } else {
    // rows z_j of Z: left vectors u_j = z_j; Y = conj(Z) M (k x n2) has rows
    // sigma_j v_j^+; B = the LQ factor of Y with orthonormal rows, C = M B^+
    VB_TRY(G64(k, n2, n1, OP_R, s->Z, ns, (long long)k * ns, OP_N, M, n2, nm, Y, n2, (long long)k * n2));
    VB_TRY(lq_rows(s, Y, k, n2, dstC, s->q_Rm, seed));
    VB_TRY(G64(n1, k, n2, OP_N, M, n2, nm, OP_C, dstC, n2, (long long)k * n2, dstA, k, (long long)n1 * k));
    const long long nc = (long long)n1 * k;
    VB_TRY(vec_norm2(dstA, nc, s->d_nrm, s->d_part, reduce_parts(nc), st));
    VB_TRY(vec_scale_inv(dstA, nc, s->d_nrm, st));
  }
  prof_end(PH_SPLITOUT, st, 0.0);
  *k_out = k;
  return VB_OK;
}

// m_old: the bond dimension between the two sites before this split; dstA
// (left) or dstC (right) still holds the old tensor on entry
vb_status split(vb_mps *s, bool left, int mL, int d1, int d2, int mR, int m_old, const TruncOpts &o,
                cd *dstA, cd *dstC, int *k_out, double *disc) {
  cudaStream_t st = s->st;
  const int n1 = mL * d1, n2 = d2 * mR;
  const int n = left ? n1 : n2;
  // mixed form: FP32 subspace iteration + FP64 projection once the matrix is
  // large enough for the FP64 reduction to matter
  if (s->dtype == VB_MIXED && n > MIXED_SPLIT_MIN_N) {
    // the other side small: its FP64 eigenproblem, then theta maps the
    // vectors across (bond capacities within the one-site QR buffers' 112)
    if ((left ? n2 : n1) <= MIXED_SPLIT_MIN_N && *std::max_element(s->bcap.begin(), s->bcap.end()) <= 112) {
      VB_TRY(tdvp1_setup(s));
      return split_small_side(s, left, n1, n2, o, dstA, dstC, k_out, disc);
    }
    if (o.m_max + 1 + 8 <= s->rcap) return split_mixed(s, left, mL, d1, d2, mR, m_old, o, dstA, dstC, k_out, disc);
  }
  const cd *M = s->theta;
  GemmArgs g{};
  g.M = n; g.N = n; g.batch = 1;
  g.alpha = mkc(1.0, 0.0); g.beta = mkc(0.0, 0.0);
  if (left) {  // rho = M M^+
    g.K = n2; g.opA = OP_N; g.opB = OP_C;
    g.A = M; g.lda = n2; g.B = M; g.ldb = n2;
  } else {  // rho = M^+ M
    g.K = n1; g.opA = OP_C; g.opB = OP_N;
    g.A = M; g.lda = n2; g.B = M; g.ldb = n2;
  }
  g.C = s->rho; g.ldc = n;
  g.a_size = (long long)n1 * n2; g.b_size = (long long)n1 * n2; g.c_size = s->nrho_cap * s->nrho_cap;
  prof_begin(PH_RHO, st);
  VB_TRY(zgemm(g, st));
  trace_kernel<<<1, 256, 0, st>>>(s->rho, n, s->d_trace);
  VB_CHECK_LAUNCH();
  prof_end(PH_RHO, st, 0.0);
  const int kw = std::min(n, o.m_max + 1);
  prof_begin(PH_EIGVAL, st);
  VB_TRY(eig_values(n, s->rho, kw, s->d_evals, s->eigw, st));
  prof_end(PH_EIGVAL, st, 0.0);
  std::vector<double> lam(kw);
  double tot = 0.0;
  VB_TRY_CUDA(cudaMemcpyAsync(lam.data(), s->d_evals, kw * sizeof(double), cudaMemcpyDeviceToHost, st));
  VB_TRY_CUDA(cudaMemcpyAsync(&tot, s->d_trace, sizeof(double), cudaMemcpyDeviceToHost, st));
  VB_TRY_CUDA(cudaStreamSynchronize(st));
  VB_TRY(EigWork::check(n, kw, sizeof(double), s->eigw, st));
  const int k = choose_rank(lam, n, tot, std::min(n1, n2), o, disc);
  prof_begin(PH_EIGVEC, st);
  VB_TRY(eig_vectors(n, s->rho, kw, k, s->d_evals, s->Z, s->eigw, st));
  prof_end(PH_EIGVEC, st, 0.0);
  prof_begin(PH_SPLITOUT, st);
  if (left) {
    transpose_kernel<<<grid1((long long)k * n1), 256, 0, st>>>(s->Z, k, n1, dstA);
    VB_CHECK_LAUNCH();
    GemmArgs h{};
    h.M = k; h.N = n2; h.K = n1; h.batch = 1;
    h.opA = OP_R; h.opB = OP_N;
    h.A = s->Z; h.lda = n1; h.B = M; h.ldb = n2; h.C = dstC; h.ldc = n2;
    h.alpha = mkc(1.0, 0.0); h.beta = mkc(0.0, 0.0);
    h.a_size = (long long)k * n1; h.b_size = (long long)n1 * n2; h.c_size = (long long)k * n2;
    VB_TRY(zgemm(h, st));
    const long long nc = (long long)k * n2;
    VB_TRY(vec_norm2(dstC, nc, s->d_nrm, s->d_part, reduce_parts(nc), st));
    VB_TRY(vec_scale_inv(dstC, nc, s->d_nrm, st));
  } else {
    conj_copy_kernel<<<grid1((long long)k * n2), 256, 0, st>>>(s->Z, (long long)k * n2, dstC);
    VB_CHECK_LAUNCH();
    GemmArgs h{};
    h.M = n1; h.N = k; h.K = n2; h.batch = 1;
    h.opA = OP_N; h.opB = OP_T;
    h.A = M; h.lda = n2; h.B = s->Z; h.ldb = n2; h.C = dstA; h.ldc = k;
    h.alpha = mkc(1.0, 0.0); h.beta = mkc(0.0, 0.0);
    h.a_size = (long long)n1 * n2; h.b_size = (long long)k * n2; h.c_size = (long long)n1 * k;
    VB_TRY(zgemm(h, st));
    const long long nc = (long long)n1 * k;
    VB_TRY(vec_norm2(dstA, nc, s->d_nrm, s->d_part, reduce_parts(nc), st));
    VB_TRY(vec_scale_inv(dstA, nc, s->d_nrm, st));
  }
  prof_end(PH_SPLITOUT, st, 0.0);
  *k_out = k;
  return VB_OK;
}

// Mixed form of the split (Sec. 2.1.1 truncation). The kept Schmidt
// directions are found in FP32: subspace iteration on theta for the
// r = min(n, m_max + 9, 144) leading eigenvectors of rho, then a
// Rayleigh-Ritz step on their span (S = Q^* rho Q^T diagonalised in FP32) for
// the kws = min(r, m_max + 1) leading Ritz vectors. Everything that defines
// the new tensors is FP64: the Ritz basis is re-orthonormalised (one Lowdin
// step), theta is projected on it, and the weights that the truncation rule
// sees are the FP64 Rayleigh quotients |X_i|^2, so the discarded weight
// reported is exactly the weight the chosen tensors drop.
vb_status split_mixed(vb_mps *s, bool left, int mL, int d1, int d2, int mR, int m_old, const TruncOpts &o,
                      cd *dstA, cd *dstC, int *k_out, double *disc) {
  cudaStream_t st = s->st;
  const int n1 = mL * d1, n2 = d2 * mR;
  const int n = left ? n1 : n2;
  const long long nm = (long long)n1 * n2;
  const cd *M = s->theta;
  const int kw = std::min(n, o.m_max + 1);
  const int r = std::min(n, std::min(kw + 8, s->rcap));
  const cd one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  auto G64 = [&](int Mm, int Nn, int Kk, int opA, const cd *A, long long lda, long long asz, int opB, const cd *B,
                 long long ldb, long long bsz, cd *C, long long ldc, long long csz) {
    GemmArgs g{};
    g.M = Mm; g.N = Nn; g.K = Kk; g.batch = 1; g.opA = opA; g.opB = opB;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    g.alpha = one; g.beta = zero; g.a_size = asz; g.b_size = bsz; g.c_size = csz;
    g.ws = s->skws; g.ws_elems = s->skws_elems;
    return zgemm(g, st);
  };
  // ---- FP32 subspace iteration for the r leading eigenvectors of rho
  prof_begin(PH_RHO, st);
  c64_to_c32<<<grid1(nm), 256, 0, st>>>(M, s->M32, nm);
  VB_CHECK_LAUNCH();
  VB_TRY(vec_norm2(M, nm, s->d_trace, s->d_part, reduce_parts(nm), st));
  prof_end(PH_RHO, st, 0.0);
  prof_begin(PH_EIGVAL, st);
  // rows of Q: left, u_j^T (rho = M M^+); right, conj(v_j)^T (rho = M^+ M).
  // Z = conj(Q) op1(M) and Q <- conj(Z) op2(M) apply rho once (left: op1 = N,
  // op2 = T; right: op1 = T, op2 = N); |Z|^2 is the weight the span captures
  const int nother = left ? n2 : n1;
  const unsigned long long seed = 0x243F6A8885A308D3ull + 0x9E3779B97F4A7C15ull * (++s->split_calls);
  const SubspaceWork sw{s->subG, s->subW, s->subT, s->subflag, s->skws32, s->skws32_elems};
  const int m_warm = std::min(std::max(m_old, 0), r);
  prof_begin(PH_SUBORTH, st);
  VB_TRY(subspace_init(s->Q32, r, n, left ? dstA : dstC, m_old, m_warm, left, seed, st));
  VB_TRY(subspace_orth(s->Q32, r, n, sw, seed + 1, st));
  prof_end(PH_SUBORTH, st, 0.0);
  const cf onef = mkc(1.f, 0.f), zerof = mkc(0.f, 0.f);
  double prev = -1.0;
  for (int it = 0; it < SUBSPACE_MAXIT; ++it) {
    prof_begin(PH_SUBPROD, st);
    GemmArgsF g{};
    g.M = r; g.N = nother; g.K = n; g.batch = 1;
    g.opA = OP_R; g.A = s->Q32; g.lda = n;
    g.opB = left ? OP_N : OP_T; g.B = s->M32; g.ldb = n2;
    g.C = s->subZ; g.ldc = nother;
    g.alpha = onef; g.beta = zerof;
    g.a_size = (long long)r * n; g.b_size = nm; g.c_size = (long long)r * nother;
    g.ws = s->skws32; g.ws_elems = s->skws32_elems;
    VB_TRY(gemm<float>(g, st));
    const long long nz = (long long)r * nother;
    VB_TRY(norm2_sq_f32(s->subZ, nz, s->d_capt, s->d_part, reduce_parts(nz), st));
    GemmArgsF h{};
    h.M = r; h.N = n; h.K = nother; h.batch = 1;
    h.opA = OP_R; h.A = s->subZ; h.lda = nother;
    h.opB = left ? OP_T : OP_N; h.B = s->M32; h.ldb = n2;
    h.C = s->Q32; h.ldc = n;
    h.alpha = onef; h.beta = zerof;
    h.a_size = nz; h.b_size = nm; h.c_size = (long long)r * n;
    h.ws = s->skws32; h.ws_elems = s->skws32_elems;
    VB_TRY(gemm<float>(h, st));
    prof_end(PH_SUBPROD, st, 0.0);
    prof_begin(PH_SUBORTH, st);
    VB_TRY(subspace_orth(s->Q32, r, n, sw, seed + 2 + it, st));
    VB_TRY(subspace_status(s->d_capt, s->subflag + r, s->d_flag + 2, st));
    prof_end(PH_SUBORTH, st, 0.0);
    VB_TRY_CUDA(cudaStreamSynchronize(st));
    const double capt = s->h_flag[2], nbad = s->h_flag[3];
    if (!(capt == capt)) return fail(VB_ECUDA, "split: NaN in the subspace iteration");
    if (nbad > 0.0) VB_TRY(subspace_orth(s->Q32, r, n, sw, seed + 0x1000 + it, st));
    if (it >= 1 && std::fabs(capt - prev) <= SUBSPACE_RTOL * capt) break;
    prev = capt;
  }
  // ---- Rayleigh-Ritz in FP32: rotate the basis to the kws leading Ritz vectors
  const int kws = std::min(r, kw);
  prof_begin(PH_RR, st);
  prof_begin(PH_RR32, st);
  {
    GemmArgsF g{};
    g.M = r; g.N = nother; g.K = n; g.batch = 1;
    g.opA = OP_R; g.A = s->Q32; g.lda = n;
    g.opB = left ? OP_N : OP_T; g.B = s->M32; g.ldb = n2;
    g.C = s->subZ; g.ldc = nother;
    g.alpha = onef; g.beta = zerof;
    g.a_size = (long long)r * n; g.b_size = nm; g.c_size = (long long)r * nother;
    g.ws = s->skws32; g.ws_elems = s->skws32_elems;
    VB_TRY(gemm<float>(g, st));
    GemmArgsF h{};  // S32 = Z Z^+ = conj(Q) rho Q^T
    h.M = r; h.N = r; h.K = nother; h.batch = 1;
    h.opA = OP_N; h.A = s->subZ; h.lda = nother;
    h.opB = OP_C; h.B = s->subZ; h.ldb = nother;
    h.C = s->subG; h.ldc = r;
    h.alpha = onef; h.beta = zerof;
    h.a_size = (long long)r * nother; h.b_size = (long long)r * nother; h.c_size = (long long)r * r;
    h.ws = s->skws32; h.ws_elems = s->skws32_elems;
    VB_TRY(gemm<float>(h, st));
  }
  const bool jacobi = r <= 112;
  if (jacobi) {
    prof_begin(PH_JACOBI, st);
    VB_TRY(ritz_eig_small(s->subG, r, kws, s->ev32, s->subW, s->subflag, st));
    prof_end(PH_JACOBI, st, 0.0);
  } else {
    VB_TRY(eig_values<float>(r, s->subG, kws, s->ev32, s->eigw32, st));
    VB_TRY(eig_vectors<float>(r, s->subG, kws, kws, s->ev32, s->subW, s->eigw32, st));
  }
  {
    GemmArgsF g{};  // Ritz basis: rows of W Q (kws x n)
    g.M = kws; g.N = n; g.K = r; g.batch = 1;
    g.opA = OP_N; g.A = s->subW; g.lda = r;
    g.opB = OP_N; g.B = s->Q32; g.ldb = n;
    g.C = s->subT; g.ldc = n;
    g.alpha = onef; g.beta = zerof;
    g.a_size = (long long)kws * r; g.b_size = (long long)r * n; g.c_size = (long long)kws * n;
    VB_TRY(gemm<float>(g, st));
  }
  prof_end(PH_RR32, st, 0.0);
  // ---- FP64: orthonormal Ritz basis Qo, X = theta projected on it, and the
  // kept weights as FP64 Rayleigh quotients |X_i|^2
  prof_begin(PH_RR64, st);
  subspace_rows_c64<<<grid1((long long)kws * n), 256, 0, st>>>(s->subT, s->Q64, (long long)kws * n, left ? 0 : 1);
  VB_CHECK_LAUNCH();
  const long long rn = (long long)kws * n, rr = (long long)kws * kws;
  VB_TRY(G64(kws, kws, n, OP_N, s->Q64, n, rn, OP_C, s->Q64, n, rn, s->G, kws, rr));  // G = Q Q^+
  lowdin_kernel<<<grid1(rr), 256, 0, st>>>(s->G, kws);
  VB_CHECK_LAUNCH();
  VB_TRY(G64(kws, n, kws, OP_N, s->G, kws, rr, OP_N, s->Q64, n, rn, s->Qo, n, rn));  // Qo = (3I - G)/2 Q
  if (left)  // X = conj(Qo) M  (kws x n2)
    VB_TRY(G64(kws, n2, n1, OP_R, s->Qo, n1, rn, OP_N, M, n2, nm, s->X, n2, (long long)kws * n2));
  else  // X^T = Qo M^T  (kws x n1), rows for the GEMM's sake
    VB_TRY(G64(kws, n1, n2, OP_N, s->Qo, n2, rn, OP_T, M, n2, nm, s->X, n1, (long long)kws * n1));
  ritz_weights_kernel<<<kws, 256, 0, st>>>(s->X, kws, left ? n2 : n1, 1, s->d_evals);
  VB_CHECK_LAUNCH();
  prof_end(PH_RR64, st, 0.0);
  prof_end(PH_RR, st, 0.0);
  std::vector<double> w(kws);
  double nrm = 0.0;
  VB_TRY_CUDA(cudaMemcpyAsync(w.data(), s->d_evals, kws * sizeof(double), cudaMemcpyDeviceToHost, st));
  VB_TRY_CUDA(cudaMemcpyAsync(&nrm, s->d_trace, sizeof(double), cudaMemcpyDeviceToHost, st));
  int jac_sweeps = 0;  // sweeps of the Jacobi eigensolver, for the profiler
  if (jacobi && prof_on())
    VB_TRY_CUDA(cudaMemcpyAsync(&jac_sweeps, s->subflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  VB_TRY_CUDA(cudaStreamSynchronize(st));
  if (jacobi) prof_note(PH_JACOBI, (double)jac_sweeps);
  if (r > 112) VB_TRY(EigWork::check(r, kws, 4, s->eigw32, st));
  prof_end(PH_EIGVAL, st, 0.0);
  for (double v : w)
    if (!(v == v)) return fail(VB_ECUDA, "split: NaN in the Ritz weights");
  std::vector<int> perm(kws);
  for (int i = 0; i < kws; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return w[a] > w[b]; });
  std::vector<double> lam(kws);
  for (int i = 0; i < kws; ++i) lam[i] = w[perm[i]];
  const int k = choose_rank(lam, n, nrm * nrm, std::min(n1, n2), o, disc);
  prof_begin(PH_SPLITOUT, st);
  VB_TRY_CUDA(cudaMemcpyAsync(s->d_perm, perm.data(), k * sizeof(int), cudaMemcpyHostToDevice, st));
  if (left) {
    // A[x][j] = Qo[perm_j][x];  C[j][y] = X[perm_j][y]
    ritz_gather_kernel<<<grid1((long long)k * n1), 256, 0, st>>>(s->Qo, n1, s->d_perm, k, 0, dstA);
    VB_CHECK_LAUNCH();
    ritz_gather_kernel<<<grid1((long long)k * n2), 256, 0, st>>>(s->X, n2, s->d_perm, k, 1, dstC);
    VB_CHECK_LAUNCH();
    const long long nc = (long long)k * n2;
    VB_TRY(vec_norm2(dstC, nc, s->d_nrm, s->d_part, reduce_parts(nc), st));
    VB_TRY(vec_scale_inv(dstC, nc, s->d_nrm, st));
  } else {
    // B[j][y] = conj(Qo[perm_j][y]);  C[x][j] = X^T[perm_j][x]
    ritz_gather_kernel<<<grid1((long long)k * n2), 256, 0, st>>>(s->Qo, n2, s->d_perm, k, 2, dstC);
    VB_CHECK_LAUNCH();
    ritz_gather_kernel<<<grid1((long long)n1 * k), 256, 0, st>>>(s->X, n1, s->d_perm, k, 0, dstA);
    VB_CHECK_LAUNCH();
    const long long nc = (long long)n1 * k;
    VB_TRY(vec_norm2(dstA, nc, s->d_nrm, s->d_part, reduce_parts(nc), st));
    VB_TRY(vec_scale_inv(dstA, nc, s->d_nrm, st));
  }
  prof_end(PH_SPLITOUT, st, 0.0);
  *k_out = k;
  return VB_OK;
}

// environment update of the sweep: FP64, or complex FP32 in the mixed form
// (inputs converted from and the result converted back to the FP64 storage)
vb_status env_update(vb_mps *s, bool left, int p, int mL, int mR, const cd *E, const cd *A, cd *Enew) {
  const vb_mpo *mpo = s->mpo;
  if (s->dtype != VB_MIXED) {
    if (left) return env_left<double>(mpo, p, mL, mR, E, A, Enew, s->T1, s->T2, s->inter_cap, s->st);
    return env_right<double>(mpo, p, mL, mR, E, A, Enew, s->T1, s->T2, s->inter_cap, s->st);
  }
  const MpoSite &S = mpo->sites[p];
  const long long na = (long long)mL * S.d * mR;
  const long long ne = left ? (long long)mL * S.wl * mL : (long long)mR * S.wr * mR;
  const long long no = left ? (long long)mR * S.wr * mR : (long long)mL * S.wl * mL;
  c64_to_c32<<<grid1(na), 256, 0, s->st>>>(A, s->envA32, na);
  VB_CHECK_LAUNCH();
  c64_to_c32<<<grid1(ne), 256, 0, s->st>>>(E, s->envE32, ne);
  VB_CHECK_LAUNCH();
  if (left)
    VB_TRY(env_left<float>(mpo, p, mL, mR, s->envE32, s->envA32, s->envO32, s->envT1, s->envT2, s->inter_cap, s->st));
  else
    VB_TRY(env_right<float>(mpo, p, mL, mR, s->envE32, s->envA32, s->envO32, s->envT1, s->envT2, s->inter_cap, s->st));
  c32_to_c64<<<grid1(no), 256, 0, s->st>>>(s->envO32, Enew, no);
  VB_CHECK_LAUNCH();
  return VB_OK;
}

vb_status merge(vb_mps *s, int i) {
  const int mL = s->bond[i], mM = s->bond[i + 1], mR = s->bond[i + 2];
  const int d1 = s->dims[i], d2 = s->dims[i + 1];
  if (s->dtype == VB_MIXED) {
    // complex FP32 (FP32 products, K = mM terms per element): theta is the
    // start of an exponential whose products are FP32-accurate themselves
    const long long na = (long long)mL * d1 * mM, nb = (long long)mM * d2 * mR, nt = (long long)mL * d1 * d2 * mR;
    if (na > s->env_site_cap || nb > s->env_site_cap || nt > s->theta_cap)
      return fail(VB_EINVAL, "merge: tensors exceed their FP32 buffers");
    c64_to_c32<<<grid1(na), 256, 0, s->st>>>(s->A[i], s->envA32, na);
    VB_CHECK_LAUNCH();
    c64_to_c32<<<grid1(nb), 256, 0, s->st>>>(s->A[i + 1], s->mrgB32, nb);
    VB_CHECK_LAUNCH();
    GemmArgsF g{};
    g.M = mL * d1; g.N = d2 * mR; g.K = mM; g.batch = 1;
    g.opA = OP_N; g.opB = OP_N;
    g.A = s->envA32; g.lda = mM; g.B = s->mrgB32; g.ldb = g.N; g.C = s->M32; g.ldc = g.N;
    g.alpha = mkc(1.f, 0.f); g.beta = mkc(0.f, 0.f);
    g.a_size = na; g.b_size = nb; g.c_size = s->theta_cap;
    g.ws = s->skws32; g.ws_elems = s->skws32_elems;
    VB_TRY(gemm<float>(g, s->st));
    c32_to_c64<<<grid1(nt), 256, 0, s->st>>>(s->M32, s->theta, nt);
    VB_CHECK_LAUNCH();
    return VB_OK;
  }
  GemmArgs g{};
  g.M = mL * d1; g.N = d2 * mR; g.K = mM; g.batch = 1;
  g.opA = OP_N; g.opB = OP_N;
  g.A = s->A[i]; g.lda = mM; g.B = s->A[i + 1]; g.ldb = g.N; g.C = s->theta; g.ldc = g.N;
  g.alpha = mkc(1.0, 0.0); g.beta = mkc(0.0, 0.0);
  g.a_size = (long long)mL * d1 * mM; g.b_size = (long long)mM * d2 * mR; g.c_size = s->theta_cap;
  return zgemm(g, s->st);
}

vb_status set_device_of(vb_mps *s) {
  int dev = -1;
  VB_TRY_CUDA(cudaGetDevice(&dev));
  if (dev != s->device) VB_TRY_CUDA(cudaSetDevice(s->device));
  return VB_OK;
}

// allocate all buffers of a new MPS handle
vb_status mps_setup(const vb_mpo *mpo, const vb_mps_opts *opts, vb_mps **out) {
  if (!mpo || !opts || !out) return fail(VB_EINVAL, "mps: null argument");
  if (opts->m_cap < 1) return fail(VB_EINVAL, "mps: m_cap must be >= 1");
  if (opts->dtype != VB_FP64 && opts->dtype != VB_MIXED) return fail(VB_EINVAL, "mps: bad dtype");
  int kcap = opts->krylov_cap > 0 ? opts->krylov_cap : 40;
  if (kcap > 64) return fail(VB_EINVAL, "mps: krylov_cap must be <= 64");
  VB_TRY(mpo_upload(mpo));
  vb_mps *s = new vb_mps();
  s->n = mpo->n;
  s->dtype = opts->dtype;
  s->m_cap = opts->m_cap;
  s->kcap = kcap;
  s->st = (cudaStream_t)opts->cuda_stream;
  s->alloc.user = opts->alloc;
  s->alloc.stream = s->st;
  s->mpo = mpo;
  s->dims = mpo->dims;
  cudaGetDevice(&s->device);
  const int n = s->n;
  s->bond.assign(n + 1, 1);
  s->bcap.assign(n + 1, 1);
  for (int b = 1; b < n; ++b) {
    long long l = full_dim(s->dims, 0, b, opts->m_cap), r = full_dim(s->dims, b, n, opts->m_cap);
    s->bcap[b] = (int)std::min<long long>(std::min(l, r), opts->m_cap);
  }
  auto fail_free = [&](vb_status st) {
    for (void *p : s->owned) s->alloc.put(p);
    delete s;
    return st;
  };
  s->A.assign(n, nullptr);
  s->L.assign(n + 1, nullptr);
  s->R.assign(n + 1, nullptr);
  long long inter = 0;
  for (int p = 0; p < n; ++p) {
    const MpoSite &S = mpo->sites[p];
    size_t sa = (size_t)s->bcap[p] * S.d * s->bcap[p + 1];
    vb_status e = mps_alloc(s, (void **)&s->A[p], sa * sizeof(cd));
    if (e != VB_OK) return fail_free(e);
    size_t se = (size_t)s->bcap[p] * S.wl * s->bcap[p];
    e = mps_alloc(s, (void **)&s->L[p], se * sizeof(cd));
    if (e != VB_OK) return fail_free(e);
    e = mps_alloc(s, (void **)&s->R[p], se * sizeof(cd));
    if (e != VB_OK) return fail_free(e);
    // one-site intermediates
    long long one = (long long)s->bcap[p] * S.d * s->bcap[p + 1] * std::max(S.wl, S.wr);
    inter = std::max(inter, one);
    s->nrho_cap = std::max<long long>(s->nrho_cap, (long long)s->bcap[p] * S.d);
    s->nrho_cap = std::max<long long>(s->nrho_cap, (long long)S.d * s->bcap[p + 1]);
    if (p + 1 < n) {
      const MpoSite &S2 = mpo->sites[p + 1];
      long long th = (long long)s->bcap[p] * S.d * S2.d * s->bcap[p + 2];
      s->theta_cap = std::max(s->theta_cap, th);
      int wmax = std::max(S.wl, std::max(S.wr, S2.wr));
      inter = std::max(inter, th * wmax);
    }
  }
  if (n == 1) s->theta_cap = std::max<long long>(s->theta_cap, s->dims[0]);
  s->theta_cap = std::max<long long>(s->theta_cap, 1);
  for (int p = 0; p < n; ++p)
    s->theta_cap = std::max<long long>(s->theta_cap, (long long)s->bcap[p] * s->dims[p] * s->bcap[p + 1]);
  s->theta_cap = (s->theta_cap + 31) / 32 * 32;
  s->inter_cap = std::max<long long>(inter, 1);
  {
    vb_status e = VB_OK;
    auto A2 = [&](void **p, size_t b) {
      if (e == VB_OK) e = mps_alloc(s, p, b);
    };
    A2((void **)&s->L[n], sizeof(cd));
    A2((void **)&s->R[n], sizeof(cd));
    A2((void **)&s->theta, s->theta_cap * sizeof(cd));
    A2((void **)&s->V, (size_t)(kcap + 1) * s->theta_cap * sizeof(cd));
    if (s->dtype == VB_MIXED) {
      A2((void **)&s->V32, (size_t)(kcap + 1) * s->theta_cap * sizeof(cf));
      A2((void **)&s->w32, (size_t)s->theta_cap * sizeof(cf));
    }
    A2((void **)&s->T1, s->inter_cap * sizeof(cd));
    A2((void **)&s->T2, s->inter_cap * sizeof(cd));
    const int nr = (int)s->nrho_cap;
    s->kw_cap = std::min(nr, opts->m_cap + 1);
    A2((void **)&s->rho, (size_t)nr * nr * sizeof(cd));
    A2((void **)&s->Z, (size_t)(s->kw_cap) * nr * sizeof(cd));
    A2(&s->eigw, EigWork::bytes(nr, s->kw_cap));
    A2((void **)&s->d_nrm, 256);
    A2((void **)&s->d_alpha, 128 * sizeof(double));
    A2((void **)&s->d_beta, 128 * sizeof(double));
    A2((void **)&s->d_bnext, 256);
    A2((void **)&s->d_evals, (size_t)(s->kw_cap + 1) * sizeof(double));
    A2((void **)&s->d_trace, 256);
    A2((void **)&s->d_part, 512 * sizeof(double));
    A2((void **)&s->d_pop, 64 * sizeof(double));
    A2((void **)&s->d_c, 128 * sizeof(cd));
    A2((void **)&s->d_c2, 128 * sizeof(cd));
    A2((void **)&s->d_u, 128 * sizeof(cd));
    A2((void **)&s->d_partc, (size_t)PARTC_ELEMS * sizeof(cd));
    A2((void **)&s->d_tcerr, 256);
    A2((void **)&s->d_cnt, 64 * sizeof(unsigned int));
    A2((void **)&s->d_vs, 128 * sizeof(double));
    if (e != VB_OK) return fail_free(e);
    static const double one = 1.0;  // vs[0]: v_0 is stored normalised
    if (cudaMemsetAsync(s->d_tcerr, 0, sizeof(int), s->st) != cudaSuccess ||
        cudaMemsetAsync(s->d_cnt, 0, 64 * sizeof(unsigned int), s->st) != cudaSuccess ||
        cudaMemcpyAsync(s->d_vs, &one, sizeof(double), cudaMemcpyHostToDevice, s->st) != cudaSuccess) {
      cudaGetLastError();
      return fail_free(fail(VB_ECUDA, "mps: memset failed"));
    }
    if (s->dtype == VB_MIXED) {
      size_t mb = 0;
      for (int p = 0; p < n; ++p) {
        mb = std::max(mb, heff_mixed_work_bytes(mpo, p, 0, s->bcap[p], s->bcap[p + 1]));
        if (p + 1 < n) mb = std::max(mb, heff_mixed_work_bytes(mpo, p, 1, s->bcap[p], s->bcap[p + 2]));
      }
      s->mixw_bytes = mb;
      A2(&s->mixw, mb);
      const long long nr2 = s->nrho_cap;
      s->rcap = (int)std::min<long long>(nr2, std::min(opts->m_cap + 1 + 32, SUBSPACE_MAX_R));
      const long long rc = std::max(s->rcap, 1);
      A2((void **)&s->M32, s->theta_cap * sizeof(cf));
      A2((void **)&s->subZ, (size_t)rc * nr2 * sizeof(cf));
      A2((void **)&s->subT, (size_t)rc * nr2 * sizeof(cf));
      A2((void **)&s->subG, (size_t)rc * rc * sizeof(cf));
      A2((void **)&s->subW, (size_t)rc * rc * sizeof(cf));
      A2((void **)&s->subflag, (size_t)(rc + 1) * sizeof(int));
      A2((void **)&s->d_capt, 256);
      A2((void **)&s->d_perm, (size_t)rc * sizeof(int));
      A2((void **)&s->ev32, (size_t)rc * sizeof(float));
      A2(&s->eigw32, EigWork::bytes((int)rc, (int)rc, 4));
      s->skws32_elems = 48LL * rc * nr2;
      A2((void **)&s->skws32, (size_t)s->skws32_elems * sizeof(cf));
      A2((void **)&s->Q32, (size_t)rc * nr2 * sizeof(cf));
      A2((void **)&s->Q64, (size_t)rc * nr2 * sizeof(cd));
      A2((void **)&s->Qo, (size_t)rc * nr2 * sizeof(cd));
      A2((void **)&s->X, (size_t)rc * nr2 * sizeof(cd));
      A2((void **)&s->G, (size_t)rc * rc * sizeof(cd));
      s->skws_elems = 48LL * rc * nr2;
      A2((void **)&s->skws, (size_t)s->skws_elems * sizeof(cd));
      for (int p = 0; p <= n; ++p) {
        const int w = p < n ? mpo->sites[p].wl : 1;
        s->env_blk_cap = std::max<long long>(s->env_blk_cap, (long long)s->bcap[p] * w * s->bcap[p]);
        if (p < n)
          s->env_site_cap = std::max<long long>(s->env_site_cap, (long long)s->bcap[p] * s->dims[p] * s->bcap[p + 1]);
      }
      A2((void **)&s->envA32, (size_t)s->env_site_cap * sizeof(cf));
      A2((void **)&s->mrgB32, (size_t)s->env_site_cap * sizeof(cf));
      A2((void **)&s->envE32, (size_t)s->env_blk_cap * sizeof(cf));
      A2((void **)&s->envO32, (size_t)s->env_blk_cap * sizeof(cf));
      A2((void **)&s->envT1, (size_t)s->inter_cap * sizeof(cf));
      A2((void **)&s->envT2, (size_t)s->inter_cap * sizeof(cf));
      if (e != VB_OK) return fail_free(e);
    }
  }
  if (cudaHostAlloc((void **)&s->h_flag, 4 * sizeof(double), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void **)&s->d_flag, s->h_flag, 0) != cudaSuccess) {
    cudaGetLastError();
    return fail_free(fail(VB_ECUDA, "mps: cudaHostAlloc (mapped) failed"));
  }
  // boundary environments = 1
  cd one = mkc(1.0, 0.0);
  if (cudaMemcpyAsync(s->L[0], &one, sizeof(cd), cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
      cudaMemcpyAsync(s->R[n], &one, sizeof(cd), cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(s->h_flag);
    return fail_free(fail(VB_ECUDA, "mps: boundary upload failed"));
  }
  *out = s;
  return VB_OK;
}

// build R[p] for p = n-1 .. 1 from the right-canonical tensors
vb_status build_right_envs(vb_mps *s) {
  for (int p = s->n - 1; p >= 1; --p)
    VB_TRY(env_right<double>(s->mpo, p, s->bond[p], s->bond[p + 1], s->R[p + 1], s->A[p], s->R[p], s->T1,
                             s->T2, s->inter_cap, s->st));
  return VB_OK;
}

// ---- observables of whole states

// temporaries of one observable call, from the handle's allocator
struct Scratch {
  vb::Alloc *al;
  std::vector<void *> held;
  explicit Scratch(vb::Alloc *a) : al(a) {}
  vb_status get(void **p, size_t bytes) {
    VB_TRY(al->get(p, std::max<size_t>(bytes, 256)));
    held.push_back(*p);
    return VB_OK;
  }
  ~Scratch() {
    for (void *p : held) al->put(p);
  }
};

// transfer matrix of sites 0 .. p_end-1: E_p[y', y] =
// sum_{x, x', s} conj(A_p[x', s, y']) E_{p-1}[x', x] B_p[x, s, y], E_0 = 1
// (two complex FP64 GEMMs per site), on a's stream; result left on the device
vb_status transfer_left(const vb_mps *a, const vb_mps *b, int p_end, Scratch &sc, cd **res) {
  long long e_cap = 1, x_cap = 1;
  for (int p = 0; p <= p_end; ++p) e_cap = std::max<long long>(e_cap, (long long)a->bond[p] * b->bond[p]);
  for (int p = 0; p < p_end; ++p)
    x_cap = std::max<long long>(x_cap, (long long)a->bond[p] * a->dims[p] * b->bond[p + 1]);
  cd *E0 = nullptr, *E1 = nullptr, *X = nullptr;
  VB_TRY(sc.get((void **)&E0, e_cap * sizeof(cd)));
  VB_TRY(sc.get((void **)&E1, e_cap * sizeof(cd)));
  VB_TRY(sc.get((void **)&X, x_cap * sizeof(cd)));
  const cd one = mkc(1.0, 0.0);
  VB_TRY_CUDA(cudaMemcpyAsync(E0, &one, sizeof(cd), cudaMemcpyHostToDevice, a->st));
  for (int p = 0; p < p_end; ++p) {
    const int xa = a->bond[p], ya = a->bond[p + 1], xb = b->bond[p], yb = b->bond[p + 1], d = a->dims[p];
    GemmArgs g{};  // X[x', (s y)] = E[x', x] B[x, (s y)]
    g.M = xa; g.N = d * yb; g.K = xb; g.batch = 1;
    g.opA = OP_N; g.opB = OP_N;
    g.A = E0; g.lda = xb; g.B = b->A[p]; g.ldb = (long long)d * yb; g.C = X; g.ldc = (long long)d * yb;
    g.alpha = one; g.beta = mkc(0.0, 0.0);
    g.a_size = (long long)xa * xb; g.b_size = (long long)xb * d * yb; g.c_size = x_cap;
    VB_TRY(zgemm(g, a->st));
    GemmArgs h{};  // E'[y', y] = sum_{(x' s)} conj(A[(x' s), y']) X[(x' s), y]
    h.M = ya; h.N = yb; h.K = xa * d; h.batch = 1;
    h.opA = OP_C; h.opB = OP_N;
    h.A = a->A[p]; h.lda = ya; h.B = X; h.ldb = yb; h.C = E1; h.ldc = yb;
    h.alpha = one; h.beta = mkc(0.0, 0.0);
    h.a_size = (long long)xa * d * ya; h.b_size = x_cap; h.c_size = e_cap;
    VB_TRY(zgemm(h, a->st));
    std::swap(E0, E1);
  }
  *res = E0;
  return VB_OK;
}

// <a|b>: the transfer matrix of the whole chain (1 x 1)
vb_status overlap_dev(const vb_mps *a, const vb_mps *b, Scratch &sc, cd **res) {
  return transfer_left(a, b, a->n, sc, res);
}

// <psi|H|psi> through the left environments of the whole chain, FP64
vb_status energy_dev(const vb_mps *s, Scratch &sc, cd **res) {
  const vb_mpo *mpo = s->mpo;
  const int n = s->n;
  long long e_cap = 1, t_cap = 1;
  for (int p = 0; p < n; ++p) {
    const MpoSite &S = mpo->sites[p];
    const long long mL = s->bond[p], mR = s->bond[p + 1];
    e_cap = std::max(e_cap, std::max(mL * S.wl * mL, mR * S.wr * mR));
    t_cap = std::max(t_cap, std::max(mL * S.wl * S.d * mR, mL * S.d * S.wr * mR));
  }
  cd *E0 = nullptr, *E1 = nullptr, *T1 = nullptr, *T2 = nullptr;
  VB_TRY(sc.get((void **)&E0, e_cap * sizeof(cd)));
  VB_TRY(sc.get((void **)&E1, e_cap * sizeof(cd)));
  VB_TRY(sc.get((void **)&T1, t_cap * sizeof(cd)));
  VB_TRY(sc.get((void **)&T2, t_cap * sizeof(cd)));
  const cd one = mkc(1.0, 0.0);
  VB_TRY_CUDA(cudaMemcpyAsync(E0, &one, sizeof(cd), cudaMemcpyHostToDevice, s->st));
  for (int p = 0; p < n; ++p) {
    VB_TRY(env_left<double>(mpo, p, s->bond[p], s->bond[p + 1], E0, s->A[p], E1, T1, T2, t_cap, s->st));
    std::swap(E0, E1);
  }
  *res = E0;
  return VB_OK;
}

// ---- orthonormalisations of the one-site sweep (Cholesky QR, twice, FP64)
// QR of M (n1 x m, row-major): Q (n1 x m) with orthonormal columns, Rm = Q^+ M
// (m x m), M = Q Rm. Columns that depend on earlier ones get random
// orthonormal completions (their rows of Rm vanish).
vb_status qr_cols(vb_mps *s, const cd *M, long long n1, int m, cd *Q, cd *Rm, unsigned long long seed) {
  cudaStream_t st = s->st;
  const cd one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  const long long nm = n1 * m, mm = (long long)m * m;
  auto G = [&](int Mm, int Nn, int Kk, int opA, const cd *A, long long lda, long long asz, int opB, const cd *B,
               long long ldb, long long bsz, cd *C, long long ldc, long long csz) {
    GemmArgs g{};
    g.M = Mm; g.N = Nn; g.K = Kk; g.batch = 1; g.opA = opA; g.opB = opB;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    g.alpha = one; g.beta = zero; g.a_size = asz; g.b_size = bsz; g.c_size = csz;
    g.ws = s->q_ws; g.ws_elems = s->q_ws_elems;  // split-K for the m x m products with long K
    return zgemm(g, st);
  };
  VB_TRY(G(m, m, (int)n1, OP_C, M, m, nm, OP_N, M, m, nm, s->q_G, m, mm));  // G = M^+ M
  VB_TRY(chol_w64(s->q_G, m, s->q_W, s->q_flag, st));
  VB_TRY(G((int)n1, m, m, OP_N, M, m, nm, OP_C, s->q_W, m, mm, s->q_Q, m, nm));  // Q1 = M W^+
  fill_flagged64<<<grid1(nm), 256, 0, st>>>(s->q_Q, m, n1, 1, s->q_flag, seed);
  VB_CHECK_LAUNCH();
  VB_TRY(G(m, m, (int)n1, OP_C, s->q_Q, m, nm, OP_N, s->q_Q, m, nm, s->q_G, m, mm));  // G2 = Q1^+ Q1
  VB_TRY(chol_w64(s->q_G, m, s->q_W, s->q_flag, st));
  VB_TRY(G((int)n1, m, m, OP_N, s->q_Q, m, nm, OP_C, s->q_W, m, mm, Q, m, nm));  // Q = Q1 W2^+
  return G(m, m, (int)n1, OP_C, Q, m, nm, OP_N, M, m, nm, Rm, m, mm);  // Rm = Q^+ M
}

// LQ of C (m x n2): Q (m x n2) with orthonormal rows, Rm = C Q^+ (m x m), C = Rm Q
vb_status lq_rows(vb_mps *s, const cd *Cm, int m, long long n2, cd *Q, cd *Rm, unsigned long long seed) {
  cudaStream_t st = s->st;
  const cd one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  const long long nm = n2 * m, mm = (long long)m * m;
  auto G = [&](int Mm, int Nn, int Kk, int opA, const cd *A, long long lda, long long asz, int opB, const cd *B,
               long long ldb, long long bsz, cd *C, long long ldc, long long csz) {
    GemmArgs g{};
    g.M = Mm; g.N = Nn; g.K = Kk; g.batch = 1; g.opA = opA; g.opB = opB;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    g.alpha = one; g.beta = zero; g.a_size = asz; g.b_size = bsz; g.c_size = csz;
    g.ws = s->q_ws; g.ws_elems = s->q_ws_elems;  // split-K for the m x m products with long K
    return zgemm(g, st);
  };
  VB_TRY(G(m, m, (int)n2, OP_N, Cm, n2, nm, OP_C, Cm, n2, nm, s->q_G, m, mm));  // G = C C^+
  VB_TRY(chol_w64(s->q_G, m, s->q_W, s->q_flag, st));
  VB_TRY(G(m, (int)n2, m, OP_N, s->q_W, m, mm, OP_N, Cm, n2, nm, s->q_Q, n2, nm));  // Q1 = W C
  fill_flagged64<<<grid1(nm), 256, 0, st>>>(s->q_Q, m, n2, 0, s->q_flag, seed);
  VB_CHECK_LAUNCH();
  VB_TRY(G(m, m, (int)n2, OP_N, s->q_Q, n2, nm, OP_C, s->q_Q, n2, nm, s->q_G, m, mm));  // G2 = Q1 Q1^+
  VB_TRY(chol_w64(s->q_G, m, s->q_W, s->q_flag, st));
  VB_TRY(G(m, (int)n2, m, OP_N, s->q_W, m, mm, OP_N, s->q_Q, n2, nm, Q, n2, nm));  // Q = W2 Q1
  return G(m, m, (int)n2, OP_N, Cm, n2, nm, OP_C, Q, n2, nm, Rm, m, mm);  // Rm = C Q^+
}

vb_status tdvp1_setup(vb_mps *s) {
  if (s->t1_ready) return VB_OK;
  int mmax = 1;
  for (int b : s->bcap) mmax = std::max(mmax, b);
  if (mmax > 112) return fail(VB_EINVAL, "tdvp1_sweep: bond capacity above 112");
  const size_t mm = (size_t)mmax * mmax;
  VB_TRY(mps_alloc(s, (void **)&s->q_G, mm * sizeof(cd)));
  VB_TRY(mps_alloc(s, (void **)&s->q_W, mm * sizeof(cd)));
  VB_TRY(mps_alloc(s, (void **)&s->q_Rm, mm * sizeof(cd)));
  VB_TRY(mps_alloc(s, (void **)&s->q_Q, (size_t)s->theta_cap * sizeof(cd)));
  VB_TRY(mps_alloc(s, (void **)&s->q_flag, (size_t)(mmax + 2) * sizeof(int)));
  s->q_ws_elems = 320LL * 64 * 64;  // split-K chunks x one 64 x 64 tile (chunks <= 2 x 152 / tiles)
  s->q_ws_elems = std::max<long long>(s->q_ws_elems, 320LL * mm);
  VB_TRY(mps_alloc(s, (void **)&s->q_ws, (size_t)s->q_ws_elems * sizeof(cd)));
  s->t1_ready = true;
  return VB_OK;
}

}  // namespace
}  // namespace vb

extern "C" {

vb_status mps_create(const vb_mpo *mpo, const int *init_index, const vb_mps_opts *opts,
                     vb_mps **out) {
  if (!mpo || !init_index || !opts || !out) return fail(VB_EINVAL, "mps_create: null argument");
  *out = nullptr;
  for (int p = 0; p < mpo->n; ++p)
    if (init_index[p] < 0 || init_index[p] >= mpo->dims[p])
      return fail(VB_EINVAL, "mps_create: init_index out of range at site " + std::to_string(p));
  vb_mps *s = nullptr;
  VB_TRY(mps_setup(mpo, opts, &s));
  const int n = s->n;
  // bond dimensions: 1, or the padded full dimensions (bounded by m_cap)
  for (int b = 1; b < n; ++b) s->bond[b] = opts->pad_full ? s->bcap[b] : 1;
  // right-orthonormal padded product state: first row carries the product
  // state, the remaining rows are distinct unit vectors
  for (int p = 0; p < n; ++p) {
    const int dl = s->bond[p], d = s->dims[p], dr = s->bond[p + 1];
    std::vector<cd> h((size_t)dl * d * dr, mkc(0.0, 0.0));
    if (p == 0) {
      h[(size_t)init_index[0] * dr] = mkc(1.0, 0.0);
    } else {
      const int cols = d * dr, first = init_index[p] * dr;
      h[first] = mkc(1.0, 0.0);
      int c = 0;
      for (int r = 1; r < dl; ++r) {
        if (c == first) ++c;
        h[(size_t)r * cols + c] = mkc(1.0, 0.0);
        ++c;
      }
    }
    if (cudaMemcpyAsync(s->A[p], h.data(), h.size() * sizeof(cd), cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
        cudaStreamSynchronize(s->st) != cudaSuccess) {
      mps_destroy(s);
      return fail(VB_ECUDA, "mps_create: upload failed");
    }
  }
  vb_status e = build_right_envs(s);
  if (e == VB_OK && cudaStreamSynchronize(s->st) != cudaSuccess) e = fail(VB_ECUDA, "mps_create: env build failed");
  if (e != VB_OK) {
    mps_destroy(s);
    return e;
  }
  *out = s;
  return VB_OK;
}

vb_status mps_create_from_tensors(const vb_mpo *mpo, const int *bond_dims,
                                  const double *const *host_tensors, const vb_mps_opts *opts,
                                  vb_mps **out) {
  if (!mpo || !host_tensors || !opts || !out || (mpo->n > 1 && !bond_dims))
    return fail(VB_EINVAL, "mps_create_from_tensors: null argument");
  *out = nullptr;
  vb_mps *s = nullptr;
  VB_TRY(mps_setup(mpo, opts, &s));
  const int n = s->n;
  for (int b = 1; b < n; ++b) {
    if (bond_dims[b - 1] < 1 || bond_dims[b - 1] > s->bcap[b]) {
      mps_destroy(s);
      return fail(VB_EINVAL, "mps_create_from_tensors: bond " + std::to_string(b - 1) +
                                 " outside 1..min(m_cap, full dimension)");
    }
    s->bond[b] = bond_dims[b - 1];
  }
  for (int p = 0; p < n; ++p) {
    size_t el = (size_t)s->bond[p] * s->dims[p] * s->bond[p + 1];
    if (!host_tensors[p] ||
        cudaMemcpyAsync(s->A[p], host_tensors[p], el * sizeof(cd), cudaMemcpyHostToDevice, s->st) != cudaSuccess) {
      mps_destroy(s);
      return fail(VB_EINVAL, "mps_create_from_tensors: upload of site " + std::to_string(p) + " failed");
    }
  }
  vb_status e = build_right_envs(s);
  if (e == VB_OK && cudaStreamSynchronize(s->st) != cudaSuccess) e = fail(VB_ECUDA, "env build failed");
  if (e != VB_OK) {
    mps_destroy(s);
    return e;
  }
  *out = s;
  return VB_OK;
}

vb_status mps_destroy(vb_mps *s) {
  if (!s) return VB_OK;
  cudaStreamSynchronize(s->st);
  for (void *p : s->owned) s->alloc.put(p);
  if (s->h_flag) cudaFreeHost(s->h_flag);
  delete s;
  return VB_OK;
}

int mps_n_sites(const vb_mps *s) { return s ? s->n : -1; }

vb_status mps_bond_dims(const vb_mps *s, int *host_out) {
  if (!s || !host_out) return fail(VB_EINVAL, "mps_bond_dims: null argument");
  for (int b = 1; b < s->n; ++b) host_out[b - 1] = s->bond[b];
  return VB_OK;
}

vb_status mps_get_site(const vb_mps *s, int site, double *host_out) {
  if (!s || !host_out || site < 0 || site >= s->n) return fail(VB_EINVAL, "mps_get_site: bad argument");
  size_t el = (size_t)s->bond[site] * s->dims[site] * s->bond[site + 1];
  VB_TRY_CUDA(cudaMemcpyAsync(host_out, s->A[site], el * sizeof(cd), cudaMemcpyDeviceToHost, s->st));
  VB_TRY_CUDA(cudaStreamSynchronize(s->st));
  return VB_OK;
}

vb_status mps_get_tensor(const vb_mps *s, int site, double *dev_out, void *stream) {
  if (!s || !dev_out || site < 0 || site >= s->n) return fail(VB_EINVAL, "mps_get_tensor: bad argument");
  VB_TRY(set_device_of(const_cast<vb_mps *>(s)));
  size_t el = (size_t)s->bond[site] * s->dims[site] * s->bond[site + 1];
  cudaStream_t dst = (cudaStream_t)stream;
  VB_TRY_CUDA(cudaMemcpyAsync(dev_out, s->A[site], el * sizeof(cd), cudaMemcpyDeviceToDevice, s->st));
  if (dst != s->st) VB_TRY_CUDA(cudaStreamSynchronize(s->st));
  return VB_OK;
}

vb_status vb_test_raise_wait_flag(vb_mps *s) {
  if (!s) return fail(VB_EINVAL, "vb_test_raise_wait_flag: null argument");
  if (s->dtype != VB_MIXED) return fail(VB_EINVAL, "vb_test_raise_wait_flag: only mixed-form handles have the flag");
  VB_TRY(set_device_of(s));
  const int one = 1;
  VB_TRY_CUDA(cudaMemcpyAsync(s->d_tcerr, &one, sizeof(int), cudaMemcpyHostToDevice, s->st));
  VB_TRY_CUDA(cudaStreamSynchronize(s->st));
  return VB_OK;
}

vb_status tdvp2_sweep(vb_mps *s, const vb_mpo *mpo, double dt_fs, const vb_tdvp_opts *o,
                      vb_sweep_stats *stats) {
  if (!s || !mpo || !o) return fail(VB_EINVAL, "tdvp2_sweep: null argument");
  if (mpo != s->mpo) return fail(VB_EINVAL, "tdvp2_sweep: MPS was created for another MPO");
  if (s->center != 0) return fail(VB_ESTATE, "tdvp2_sweep: center is not on site 0");
  if (o->m_max < 1 || o->m_max > s->m_cap) return fail(VB_EINVAL, "tdvp2_sweep: m_max outside 1..m_cap");
  if (o->krylov_max < 1 || o->krylov_max > s->kcap)
    return fail(VB_EINVAL, "tdvp2_sweep: krylov_max outside 1..krylov_cap");
  if (o->eps < 0 || o->zero_floor < 0 || !(o->krylov_tol > 0))
    return fail(VB_EINVAL, "tdvp2_sweep: eps, zero_floor must be >= 0 and krylov_tol > 0");
  if (s->n < 2) return fail(VB_EINVAL, "tdvp2_sweep: needs at least two sites");
  VB_TRY(set_device_of(s));
  const int n = s->n;
  const double tau = 0.5 * dt_fs;
  TruncOpts to{o->m_max, o->eps, o->zero_floor};
  vb_sweep_stats st{};
  auto evolve = [&](const HeffOp &op, cd *x, long long N, double dt) -> vb_status {
    int it = 0, conv = 0;
    VB_TRY(krylov_expm(s, op, x, N, dt, o->krylov_max, o->krylov_tol, &it, &conv));
    st.krylov_iters_max = std::max(st.krylov_iters_max, it);
    st.krylov_iters_total += it;
    if (!conv) {
      st.noconv++;
      if (o->on_noconv) return fail(VB_ENOCONV, "Krylov exponential did not converge");
    }
    return VB_OK;
  };
  // left to right, tau = dt/2
  for (int i = 0; i + 1 < n; ++i) {
    const int mL = s->bond[i], mR = s->bond[i + 2], d1 = s->dims[i], d2 = s->dims[i + 1];
    prof_begin(PH_MERGE, s->st);
    VB_TRY(merge(s, i));
    prof_end(PH_MERGE, s->st, 0.0);
    HeffOp op{1, i, mL, mR, s->L[i], s->R[i + 2]};
    VB_TRY(evolve(op, s->theta, (long long)mL * d1 * d2 * mR, tau));
    int k = 0;
    double disc = 0.0;
    prof_begin(PH_SPLIT, s->st);
    VB_TRY(split(s, true, mL, d1, d2, mR, s->bond[i + 1], to, s->A[i], s->A[i + 1], &k, &disc));
    prof_end(PH_SPLIT, s->st, 0.0);
    st.discarded_weight += disc;
    s->bond[i + 1] = k;
    prof_begin(PH_ENV, s->st);
    VB_TRY(env_update(s, true, i, mL, k, s->L[i], s->A[i], s->L[i + 1]));
    prof_end(PH_ENV, s->st, 0.0);
    if (i + 2 < n) {
      HeffOp op1{0, i + 1, k, mR, s->L[i + 1], s->R[i + 2]};
      VB_TRY(evolve(op1, s->A[i + 1], (long long)k * d2 * mR, -tau));
    }
  }
  // right to left, tau = dt/2
  for (int i = n - 2; i >= 0; --i) {
    const int mL = s->bond[i], mR = s->bond[i + 2], d1 = s->dims[i], d2 = s->dims[i + 1];
    prof_begin(PH_MERGE, s->st);
    VB_TRY(merge(s, i));
    prof_end(PH_MERGE, s->st, 0.0);
    HeffOp op{1, i, mL, mR, s->L[i], s->R[i + 2]};
    VB_TRY(evolve(op, s->theta, (long long)mL * d1 * d2 * mR, tau));
    int k = 0;
    double disc = 0.0;
    prof_begin(PH_SPLIT, s->st);
    VB_TRY(split(s, false, mL, d1, d2, mR, s->bond[i + 1], to, s->A[i], s->A[i + 1], &k, &disc));
    prof_end(PH_SPLIT, s->st, 0.0);
    st.discarded_weight += disc;
    s->bond[i + 1] = k;
    prof_begin(PH_ENV, s->st);
    VB_TRY(env_update(s, false, i + 1, k, mR, s->R[i + 2], s->A[i + 1], s->R[i + 1]));
    prof_end(PH_ENV, s->st, 0.0);
    if (i > 0) {
      HeffOp op1{0, i, mL, k, s->L[i], s->R[i + 1]};
      VB_TRY(evolve(op1, s->A[i], (long long)mL * d1 * k, -tau));
    }
  }
  VB_TRY(zero_point_phase(s, dt_fs));
  VB_TRY_CUDA(cudaStreamSynchronize(s->st));
  prof_collect();
  VB_TRY(take_wait_flag(s, "tdvp2_sweep"));
  for (int b = 1; b < n; ++b) st.max_bond = std::max(st.max_bond, s->bond[b]);
  if (stats) *stats = st;
  return VB_OK;
}

vb_status tdvp1_sweep(vb_mps *s, const vb_mpo *mpo, double dt_fs, const vb_tdvp_opts *o, vb_sweep_stats *stats) {
  if (!s || !mpo || !o) return fail(VB_EINVAL, "tdvp1_sweep: null argument");
  if (mpo != s->mpo) return fail(VB_EINVAL, "tdvp1_sweep: MPS was created for another MPO");
  if (s->center != 0) return fail(VB_ESTATE, "tdvp1_sweep: center is not on site 0");
  if (o->krylov_max < 1 || o->krylov_max > s->kcap)
    return fail(VB_EINVAL, "tdvp1_sweep: krylov_max outside 1..krylov_cap");
  if (!(o->krylov_tol > 0)) return fail(VB_EINVAL, "tdvp1_sweep: krylov_tol must be > 0");
  for (int b = 1; b < s->n; ++b)
    if ((long long)s->bond[b] > (long long)s->bond[b - 1] * s->dims[b - 1] ||
        (long long)s->bond[b] > (long long)s->dims[b] * s->bond[b + 1])
      return fail(VB_ESTATE, "tdvp1_sweep: a bond dimension exceeds what its neighbours can carry");
  VB_TRY(set_device_of(s));
  VB_TRY(tdvp1_setup(s));
  const int n = s->n;
  const double tau = 0.5 * dt_fs;
  cudaStream_t st = s->st;
  vb_sweep_stats ss{};
  auto evolve = [&](const HeffOp &op, cd *x, long long N, double dt) -> vb_status {
    int it = 0, conv = 0;
    VB_TRY(krylov_expm(s, op, x, N, dt, o->krylov_max, o->krylov_tol, &it, &conv));
    ss.krylov_iters_max = std::max(ss.krylov_iters_max, it);
    ss.krylov_iters_total += it;
    if (!conv) {
      ss.noconv++;
      if (o->on_noconv) return fail(VB_ENOCONV, "Krylov exponential did not converge");
    }
    return VB_OK;
  };
  const unsigned long long seed = 0x6A09E667F3BCC909ull + 0x9E3779B97F4A7C15ull * (++s->split_calls);
  // left to right: C_i forward, C_i = A_i Rm, Rm backward, C_{i+1} = Rm B_{i+1}
  for (int i = 0; i < n; ++i) {
    const int mL = s->bond[i], mR = s->bond[i + 1], d = s->dims[i];
    HeffOp op1{0, i, mL, mR, s->L[i], s->R[i + 1]};
    VB_TRY(evolve(op1, s->A[i], (long long)mL * d * mR, tau));
    if (i == n - 1) break;
    const long long n1 = (long long)mL * d;
    VB_TRY(qr_cols(s, s->A[i], n1, mR, s->theta, s->q_Rm, seed + 2 * i));
    VB_TRY_CUDA(cudaMemcpyAsync(s->A[i], s->theta, n1 * mR * sizeof(cd), cudaMemcpyDeviceToDevice, st));
    prof_begin(PH_ENV, st);
    VB_TRY(env_update(s, true, i, mL, mR, s->L[i], s->A[i], s->L[i + 1]));
    prof_end(PH_ENV, st, 0.0);
    HeffOp op0{-1, i, mR, mR, s->L[i + 1], s->R[i + 1]};
    VB_TRY(evolve(op0, s->q_Rm, (long long)mR * mR, -tau));
    // C_{i+1} = Rm B_{i+1}
    const long long n2 = (long long)s->dims[i + 1] * s->bond[i + 2];
    GemmArgs g{};
    g.M = mR; g.N = (int)n2; g.K = mR; g.batch = 1; g.opA = OP_N; g.opB = OP_N;
    g.A = s->q_Rm; g.lda = mR; g.B = s->A[i + 1]; g.ldb = n2; g.C = s->theta; g.ldc = n2;
    g.alpha = mkc(1.0, 0.0); g.beta = mkc(0.0, 0.0);
    g.a_size = (long long)mR * mR; g.b_size = mR * n2; g.c_size = s->theta_cap;
    VB_TRY(zgemm(g, st));
    VB_TRY_CUDA(cudaMemcpyAsync(s->A[i + 1], s->theta, mR * n2 * sizeof(cd), cudaMemcpyDeviceToDevice, st));
  }
  // right to left: C_i forward, C_i = Rm Q_i, Rm backward, C_{i-1} = A_{i-1} Rm
  for (int i = n - 1; i >= 0; --i) {
    const int mL = s->bond[i], mR = s->bond[i + 1], d = s->dims[i];
    HeffOp op1{0, i, mL, mR, s->L[i], s->R[i + 1]};
    VB_TRY(evolve(op1, s->A[i], (long long)mL * d * mR, tau));
    if (i == 0) break;
    const long long n2 = (long long)d * mR;
    VB_TRY(lq_rows(s, s->A[i], mL, n2, s->theta, s->q_Rm, seed + 2 * i + 1));
    VB_TRY_CUDA(cudaMemcpyAsync(s->A[i], s->theta, (long long)mL * n2 * sizeof(cd), cudaMemcpyDeviceToDevice, st));
    prof_begin(PH_ENV, st);
    VB_TRY(env_update(s, false, i, mL, mR, s->R[i + 1], s->A[i], s->R[i]));
    prof_end(PH_ENV, st, 0.0);
    HeffOp op0{-1, i - 1, mL, mL, s->L[i], s->R[i]};
    VB_TRY(evolve(op0, s->q_Rm, (long long)mL * mL, -tau));
    // C_{i-1} = A_{i-1} Rm
    const long long n0 = (long long)s->bond[i - 1] * s->dims[i - 1];
    GemmArgs g{};
    g.M = (int)n0; g.N = mL; g.K = mL; g.batch = 1; g.opA = OP_N; g.opB = OP_N;
    g.A = s->A[i - 1]; g.lda = mL; g.B = s->q_Rm; g.ldb = mL; g.C = s->theta; g.ldc = mL;
    g.alpha = mkc(1.0, 0.0); g.beta = mkc(0.0, 0.0);
    g.a_size = n0 * mL; g.b_size = (long long)mL * mL; g.c_size = s->theta_cap;
    VB_TRY(zgemm(g, st));
    VB_TRY_CUDA(cudaMemcpyAsync(s->A[i - 1], s->theta, n0 * mL * sizeof(cd), cudaMemcpyDeviceToDevice, st));
  }
  VB_TRY(zero_point_phase(s, dt_fs));
  VB_TRY_CUDA(cudaStreamSynchronize(st));
  VB_TRY(take_wait_flag(s, "tdvp1_sweep"));
  ss.max_bond = 1;
  for (int b = 1; b < n; ++b) ss.max_bond = std::max(ss.max_bond, s->bond[b]);
  if (stats) *stats = ss;
  return VB_OK;
}

vb_status mps_overlap(const vb_mps *a, const vb_mps *b, double *out_host) {
  if (!a || !b || !out_host) return fail(VB_EINVAL, "mps_overlap: null argument");
  if (a->n != b->n || a->dims != b->dims) return fail(VB_EINVAL, "mps_overlap: states on different chains");
  if (a->device != b->device) return fail(VB_EINVAL, "mps_overlap: states on different devices");
  VB_TRY(set_device_of(const_cast<vb_mps *>(a)));
  if (b->st != a->st) VB_TRY_CUDA(cudaStreamSynchronize(b->st));
  vb::Alloc al = a->alloc;
  cd *res = nullptr;
  cd h = mkc(0.0, 0.0);
  {
    Scratch sc(&al);
    VB_TRY(overlap_dev(a, b, sc, &res));
    VB_TRY_CUDA(cudaMemcpyAsync(&h, res, sizeof(cd), cudaMemcpyDeviceToHost, a->st));
    VB_TRY_CUDA(cudaStreamSynchronize(a->st));
  }
  out_host[0] = h.x;
  out_host[1] = h.y;
  return VB_OK;
}

vb_status mps_energy(const vb_mps *s, double *out_host) {
  if (!s || !out_host) return fail(VB_EINVAL, "mps_energy: null argument");
  VB_TRY(set_device_of(const_cast<vb_mps *>(s)));
  vb::Alloc al = s->alloc;
  cd e = mkc(0.0, 0.0), nn = mkc(0.0, 0.0);
  {
    Scratch sc(&al);
    cd *re = nullptr, *rn = nullptr;
    VB_TRY(energy_dev(s, sc, &re));
    VB_TRY(overlap_dev(s, s, sc, &rn));
    VB_TRY_CUDA(cudaMemcpyAsync(&e, re, sizeof(cd), cudaMemcpyDeviceToHost, s->st));
    VB_TRY_CUDA(cudaMemcpyAsync(&nn, rn, sizeof(cd), cudaMemcpyDeviceToHost, s->st));
    VB_TRY_CUDA(cudaStreamSynchronize(s->st));
  }
  if (!(nn.x > 0.0)) return fail(VB_ESTATE, "mps_energy: zero norm");
  out_host[0] = e.x / nn.x;
  return VB_OK;
}

vb_status tdvp2_sweep_batched(vb_mps *const *mps, const vb_mpo *const *mpo, int count, double dt_fs,
                              const vb_tdvp_opts *opts, vb_sweep_stats *stats) {
  if (count < 0 || (count > 0 && (!mps || !mpo || !opts))) return fail(VB_EINVAL, "tdvp2_sweep_batched: bad argument");
  for (int i = 0; i < count; ++i)
    if (!mps[i] || !mpo[i]) return fail(VB_EINVAL, "tdvp2_sweep_batched: null instance");
  for (int i = 0; i < count; ++i)
    for (int j = i + 1; j < count; ++j)
      if (mps[i] == mps[j]) return fail(VB_EINVAL, "tdvp2_sweep_batched: an instance appears twice");
  // one host thread per instance: each instance's Lanczos loop waits on its
  // own stream, so instances on different streams overlap on the GPU. With
  // the profiler on (not thread-safe) the instances run one after another.
  std::vector<vb_status> rc(count, VB_OK);
  std::vector<std::string> msg(count);
  auto run = [&](int i) {
    vb_sweep_stats st{};
    vb_tdvp_opts oi = *opts;  // the bond cap of each instance: min(m_max, its m_cap)
    oi.m_max = std::min(opts->m_max, mps[i]->m_cap);
    rc[i] = tdvp2_sweep(mps[i], mpo[i], dt_fs, &oi, &st);
    if (rc[i] != VB_OK) msg[i] = vb_last_error();
    if (stats) stats[i] = st;
  };
  if (prof_on() || count <= 1) {
    for (int i = 0; i < count; ++i) run(i);
  } else {
    std::vector<std::thread> th;
    th.reserve(count);
    for (int i = 0; i < count; ++i) th.emplace_back(run, i);
    for (auto &x : th) x.join();
  }
  for (int i = 0; i < count; ++i)
    if (rc[i] != VB_OK) {
      vb::set_error("tdvp2_sweep_batched: instance " + std::to_string(i) + ": " + msg[i]);
      return rc[i];
    }
  return VB_OK;
}

vb_status measure_populations(const vb_mps *s, double *pop_host) {
  if (!s || !pop_host) return fail(VB_EINVAL, "measure_populations: null argument");
  if (s->center != 0) return fail(VB_ESTATE, "measure_populations: center is not on site 0");
  const int e = s->mpo->el_pos;
  const int d = s->dims[e];
  if (d > 64) return fail(VB_EINVAL, "measure_populations: more than 64 electronic states");
  if (e == 0) {
    populations_kernel<<<1, 256, 0, s->st>>>(s->A[0], d, s->bond[1], s->d_pop);
    VB_CHECK_LAUNCH();
  } else {
    // sites right of e are right-orthonormal, so only the transfer matrix of
    // sites 0 .. e-1 enters: P_k = sum conj(A_e[x', k, y]) (E A_e)[x', k, y]
    VB_TRY(set_device_of(const_cast<vb_mps *>(s)));
    vb::Alloc al = s->alloc;
    Scratch sc(&al);
    cd *E = nullptr, *X = nullptr;
    VB_TRY(transfer_left(s, s, e, sc, &E));
    const int me = s->bond[e], mr = s->bond[e + 1];
    VB_TRY(sc.get((void **)&X, (size_t)me * d * mr * sizeof(cd)));
    GemmArgs g{};  // X[x', (k y)] = E[x', x] A_e[x, (k y)]
    g.M = me; g.N = d * mr; g.K = me; g.batch = 1;
    g.opA = OP_N; g.opB = OP_N;
    g.A = E; g.lda = me; g.B = s->A[e]; g.ldb = (long long)d * mr; g.C = X; g.ldc = (long long)d * mr;
    g.alpha = mkc(1.0, 0.0); g.beta = mkc(0.0, 0.0);
    g.a_size = (long long)me * me; g.b_size = (long long)me * d * mr; g.c_size = (long long)me * d * mr;
    VB_TRY(zgemm(g, s->st));
    populations_proj_kernel<<<1, 256, 0, s->st>>>(s->A[e], X, me, d, mr, s->d_pop);
    VB_CHECK_LAUNCH();
    VB_TRY_CUDA(cudaMemcpyAsync(pop_host, s->d_pop, d * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    VB_TRY_CUDA(cudaStreamSynchronize(s->st));  // before the scratch returns to the allocator
    return VB_OK;
  }
  VB_TRY_CUDA(cudaMemcpyAsync(pop_host, s->d_pop, d * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  VB_TRY_CUDA(cudaStreamSynchronize(s->st));
  return VB_OK;
}

// ---- single operations on caller buffers
size_t vb_heff_work_elems(const vb_mpo *mpo, int site, int mL, int mR, int two_site) {
  if (!mpo || site < 0 || site >= mpo->n || (two_site && site + 1 >= mpo->n)) return 0;
  const MpoSite &S = mpo->sites[site];
  if (two_site) {
    const MpoSite &S2 = mpo->sites[site + 1];
    size_t th = (size_t)mL * S.d * S2.d * mR;
    size_t w = std::max(S.wl, std::max(S.wr, S2.wr));
    size_t mixed = (heff_mixed_work_bytes(mpo, site, 1, mL, mR) + sizeof(cd) - 1) / sizeof(cd);
    return std::max(2 * th * w, mixed);
  }
  size_t one = (size_t)mL * S.d * mR * std::max(S.wl, S.wr);
  size_t mixed = (heff_mixed_work_bytes(mpo, site, 0, mL, mR) + sizeof(cd) - 1) / sizeof(cd);
  return std::max(2 * one, mixed);
}

vb_status vb_heff2_apply(const vb_mpo *mpo, int i, int mL, int mR, const double *L, const double *R,
                         const double *theta, double *y, double *work, int dtype, void *stream) {
  if (!mpo || i < 0 || i + 1 >= mpo->n || mL < 1 || mR < 1 || !L || !R || !theta || !y || !work)
    return fail(VB_EINVAL, "vb_heff2_apply: bad argument");
  VB_TRY(mpo_upload(mpo));
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == VB_MIXED) {
    int *err = heff_mixed_err_flag(mpo, i, 1, mL, mR, work);
    VB_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    VB_TRY(heff_mixed_apply(mpo, i, 1, mL, mR, (const cd *)L, (const cd *)R, (const cd *)theta, (cd *)y, work,
                            vb_heff_work_elems(mpo, i, mL, mR, 1) * sizeof(cd), err, st, nullptr));
    if (i == 0 && mpo->e_zpe != 0.0) {  // site 0's FP32 operator leaves out the zero-point constant
      const long long el = (long long)mL * mpo->dims[0] * mpo->dims[1] * mR;
      add_scaled_kernel<<<grid1(el), 256, 0, st>>>((cd *)y, (const cd *)theta, mpo->e_zpe, el);
      VB_CHECK_LAUNCH();
    }
    int h = 0;
    VB_TRY_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VB_TRY_CUDA(cudaStreamSynchronize(st));
    return h ? fail(VB_ETIMEOUT, "vb_heff2_apply: a tensor-core kernel's wait ran out") : VB_OK;
  }
  const MpoSite &S = mpo->sites[i], &S2 = mpo->sites[i + 1];
  size_t th = (size_t)mL * S.d * S2.d * mR;
  size_t w = std::max(S.wl, std::max(S.wr, S2.wr));
  cd *T1 = (cd *)work, *T2 = T1 + th * w;
  return heff2_fp64(mpo, i, mL, mR, (const cd *)L, (const cd *)R, (const cd *)theta, (cd *)y, T1, T2,
                    (long long)(th * w), st);
}

vb_status vb_heff1_apply(const vb_mpo *mpo, int j, int mL, int mR, const double *L, const double *R,
                         const double *C, double *y, double *work, int dtype, void *stream) {
  if (!mpo || j < 0 || j >= mpo->n || mL < 1 || mR < 1 || !L || !R || !C || !y || !work)
    return fail(VB_EINVAL, "vb_heff1_apply: bad argument");
  VB_TRY(mpo_upload(mpo));
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == VB_MIXED) {
    int *err = heff_mixed_err_flag(mpo, j, 0, mL, mR, work);
    VB_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    VB_TRY(heff_mixed_apply(mpo, j, 0, mL, mR, (const cd *)L, (const cd *)R, (const cd *)C, (cd *)y, work,
                            vb_heff_work_elems(mpo, j, mL, mR, 0) * sizeof(cd), err, st, nullptr));
    if (j == 0 && mpo->e_zpe != 0.0) {  // site 0's FP32 operator leaves out the zero-point constant
      const long long el = (long long)mL * mpo->dims[0] * mR;
      add_scaled_kernel<<<grid1(el), 256, 0, st>>>((cd *)y, (const cd *)C, mpo->e_zpe, el);
      VB_CHECK_LAUNCH();
    }
    int h = 0;
    VB_TRY_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VB_TRY_CUDA(cudaStreamSynchronize(st));
    return h ? fail(VB_ETIMEOUT, "vb_heff1_apply: a tensor-core kernel's wait ran out") : VB_OK;
  }
  const MpoSite &S = mpo->sites[j];
  size_t one = (size_t)mL * S.d * mR * std::max(S.wl, S.wr);
  cd *T1 = (cd *)work, *T2 = T1 + one;
  return heff1_fp64(mpo, j, mL, mR, (const cd *)L, (const cd *)R, (const cd *)C, (cd *)y, T1, T2,
                    (long long)one, st);
}

size_t vb_env_work_elems(const vb_mpo *mpo, int site, int mL, int mR) {
  if (!mpo || site < 0 || site >= mpo->n) return 0;
  const MpoSite &S = mpo->sites[site];
  return 2 * (size_t)mL * S.d * mR * std::max(S.wl, S.wr);
}

vb_status vb_env_left_update(const vb_mpo *mpo, int p, int mL, int mR, const double *L, const double *A,
                             double *Lnew, double *work, void *stream) {
  if (!mpo || p < 0 || p >= mpo->n || mL < 1 || mR < 1 || !L || !A || !Lnew || !work)
    return fail(VB_EINVAL, "vb_env_left_update: bad argument");
  VB_TRY(mpo_upload(mpo));
  size_t half = vb_env_work_elems(mpo, p, mL, mR) / 2;
  return env_left<double>(mpo, p, mL, mR, (const cd *)L, (const cd *)A, (cd *)Lnew, (cd *)work, (cd *)work + half,
                  (long long)half, (cudaStream_t)stream);
}

vb_status vb_env_right_update(const vb_mpo *mpo, int p, int mL, int mR, const double *R, const double *B,
                              double *Rnew, double *work, void *stream) {
  if (!mpo || p < 0 || p >= mpo->n || mL < 1 || mR < 1 || !R || !B || !Rnew || !work)
    return fail(VB_EINVAL, "vb_env_right_update: bad argument");
  VB_TRY(mpo_upload(mpo));
  size_t half = vb_env_work_elems(mpo, p, mL, mR) / 2;
  return env_right<double>(mpo, p, mL, mR, (const cd *)R, (const cd *)B, (cd *)Rnew, (cd *)work, (cd *)work + half,
                   (long long)half, (cudaStream_t)stream);
}

size_t vb_eig_work_bytes(int n, int k_want) {
  if (n < 1 || k_want < 1) return 0;
  return EigWork::bytes(n, k_want);
}

vb_status vb_herm_eig_top(int n, double *rho, int k_want, int k_vec, double *evals, double *evecs,
                          void *work, void *stream) {
  if (n < 1 || !rho || k_want < 1 || k_want > n || k_vec < 0 || k_vec > k_want || !evals || !work ||
      (k_vec > 0 && !evecs))
    return fail(VB_EINVAL, "vb_herm_eig_top: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  VB_TRY(eig_values(n, (cd *)rho, k_want, evals, work, st));
  if (k_vec > 0) VB_TRY(eig_vectors(n, (cd *)rho, k_want, k_vec, evals, (cd *)evecs, work, st));
  return EigWork::check(n, k_want, sizeof(double), work, st);
}

}  // extern "C"

// ===========================================================================
// Gradient of an electronic population with respect to linear vibronic
// couplings (the differentiable form of the 2TDVP path).
//
// For H(g) with dH/dg^I_ij = q_I (|i><j| + |j><i|) (Eq. Helvib_2; one term
// for i = j) and P_k(t) = <psi(t)| |k><k| |psi(t)>, the Duhamel formula gives
//   dP_k/dg = (2/hbar) Im int_0^t <lambda(s)| dH/dg |psi(s)> ds,
//   lambda(s) = U(s, t) |k><k| psi(t)        (the costate, propagated back),
// psi(s) the forward 2TDVP trajectory. The adjoint of the H_eff products and
// of the local exponentials of a unitary step is the same step run backwards
// (H_eff is Hermitian), so lambda comes from 2TDVP sweeps with -dt on a second
// state; the coupling derivative enters only through <lambda|q_I x |i><j||psi>,
// a transfer-matrix contraction with one operator inserted per parameter.
// The integral over the step grid s_k = k dt uses composite closed
// Newton-Cotes rules (Boole's 5-point rule on as many panels of four steps as
// fit, Simpson or the 3/8 rule for the rest, a trapezoid for a single step).
// Step checkpointing: the forward states are kept at every c-th step; the
// backward pass recomputes each segment of c steps from its checkpoint (the
// split's random-fill counter and the Krylov start hints are restored, so
// the recomputed states equal the first ones) and consumes it in reverse;
// the last segment is kept from the forward pass. About 3 - c/n_steps sweeps
// per step in all.
// ===========================================================================
namespace vb {
namespace {

// site tensors of a state in one device buffer, laid out at the handle's
// capacities, plus the host-side state needed to resume sweeps from it
struct Snap {
  std::vector<int> bond;
  unsigned long long split_calls = 0;
  std::vector<int> khint;
  char *buf = nullptr;
};

size_t snap_bytes(const vb_mps *s) {
  size_t b = 0;
  for (int p = 0; p < s->n; ++p) b += (size_t)s->bcap[p] * s->dims[p] * s->bcap[p + 1] * sizeof(cd);
  return b;
}

vb_status snap_save(const vb_mps *s, Snap &sn) {
  sn.bond = s->bond;
  sn.split_calls = s->split_calls;
  sn.khint = s->khint;
  char *o = sn.buf;
  for (int p = 0; p < s->n; ++p) {
    const size_t el = (size_t)s->bond[p] * s->dims[p] * s->bond[p + 1];
    VB_TRY_CUDA(cudaMemcpyAsync(o, s->A[p], el * sizeof(cd), cudaMemcpyDeviceToDevice, s->st));
    o += (size_t)s->bcap[p] * s->dims[p] * s->bcap[p + 1] * sizeof(cd);
  }
  return VB_OK;
}

// restore a state (center on site 0) and, when envs, its right environments
vb_status snap_load(vb_mps *s, const Snap &sn, bool envs = true) {
  s->bond = sn.bond;
  s->split_calls = sn.split_calls;
  s->khint = sn.khint;
  const char *o = sn.buf;
  for (int p = 0; p < s->n; ++p) {
    const size_t el = (size_t)s->bond[p] * s->dims[p] * s->bond[p + 1];
    VB_TRY_CUDA(cudaMemcpyAsync(s->A[p], o, el * sizeof(cd), cudaMemcpyDeviceToDevice, s->st));
    o += (size_t)s->bcap[p] * s->dims[p] * s->bcap[p + 1] * sizeof(cd);
  }
  s->center = 0;
  return envs ? build_right_envs(s) : VB_OK;
}

// A[x, s', y] <- sum_s O[s', s] A[x, s, y] for site p (O: d x d complex on the
// device), through the handle's theta buffer
__global__ void site_op_kernel(const cd *__restrict__ A, int ml, int d, int mr, const cd *__restrict__ O,
                               cd *__restrict__ out) {
  const long long tot = (long long)ml * d * mr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(e % mr);
    const long long t = e / mr;
    const int sp = (int)(t % d);
    const long long x = t / d;
    cd acc = mkc(0.0, 0.0);
    for (int s = 0; s < d; ++s) acc = cadd(acc, cmul(O[sp * d + s], A[(x * d + s) * mr + y]));
    out[e] = acc;
  }
}

vb_status apply_site_op(vb_mps *s, int p, const cd *O) {
  const long long el = (long long)s->bond[p] * s->dims[p] * s->bond[p + 1];
  if (el > s->theta_cap) return fail(VB_EINVAL, "site operator: tensor larger than the two-site buffer");
  const int blocks = (int)std::min<long long>((el + 255) / 256, 152LL * 16);
  site_op_kernel<<<std::max(1, blocks), 256, 0, s->st>>>(s->A[p], s->bond[p], s->dims[p], s->bond[p + 1], O,
                                                          s->theta);
  VB_CHECK_LAUNCH();
  VB_TRY_CUDA(cudaMemcpyAsync(s->A[p], s->theta, el * sizeof(cd), cudaMemcpyDeviceToDevice, s->st));
  return VB_OK;
}

// out[j * out_stride] = <bra| O_j at site sites[j] |ket> for n_ops
// single-site operators (ops: device, operator j at ops + j * dmax * dmax,
// row-major d x d), by left transfer matrices E_p of sites < p and right ones
// F_p of sites >= p (all kept, computed once for all operators), complex FP64
// GEMMs on bra's stream; out: device
// transfer matrices and temporaries of expect_site_ops, sized once for two
// states with the bond capacities of `s`
struct ExpectWork {
  std::vector<cd *> E, F;
  cd *X = nullptr, *Y = nullptr;
  long long x_cap = 1;
  vb_status init(const vb_mps *s, Scratch &sc) {
    const int n = s->n;
    E.assign(n + 1, nullptr);
    F.assign(n + 1, nullptr);
    for (int p = 0; p <= n; ++p) {
      const long long sz = (long long)s->bcap[p] * s->bcap[p];
      VB_TRY(sc.get((void **)&E[p], sz * sizeof(cd)));
      VB_TRY(sc.get((void **)&F[p], sz * sizeof(cd)));
    }
    for (int p = 0; p < n; ++p) x_cap = std::max<long long>(x_cap, (long long)s->bcap[p] * s->dims[p] * s->bcap[p + 1]);
    VB_TRY(sc.get((void **)&X, x_cap * sizeof(cd)));
    VB_TRY(sc.get((void **)&Y, x_cap * sizeof(cd)));
    return VB_OK;
  }
};

vb_status expect_site_ops(const vb_mps *bra, const vb_mps *ket, int n_ops, const int *sites, const cd *ops,
                          int dmax, cd *out, long long out_stride, ExpectWork &ew) {
  const int n = bra->n;
  cudaStream_t st = bra->st;
  const cd one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  std::vector<cd *> &E = ew.E, &F = ew.F;
  const long long x_cap = ew.x_cap;
  cd *X = ew.X, *Y = ew.Y;
  VB_TRY_CUDA(cudaMemcpyAsync(E[0], &one, sizeof(cd), cudaMemcpyHostToDevice, st));
  VB_TRY_CUDA(cudaMemcpyAsync(F[n], &one, sizeof(cd), cudaMemcpyHostToDevice, st));
  // E_{p+1}[y', y] = sum conj(bra[x', s, y']) E_p[x', x] ket[x, s, y]
  for (int p = 0; p < n; ++p) {
    const int xa = bra->bond[p], ya = bra->bond[p + 1], xb = ket->bond[p], yb = ket->bond[p + 1], d = bra->dims[p];
    GemmArgs g{};
    g.M = xa; g.N = d * yb; g.K = xb; g.batch = 1; g.opA = OP_N; g.opB = OP_N;
    g.A = E[p]; g.lda = xb; g.B = ket->A[p]; g.ldb = (long long)d * yb; g.C = X; g.ldc = (long long)d * yb;
    g.alpha = one; g.beta = zero;
    g.a_size = (long long)xa * xb; g.b_size = (long long)xb * d * yb; g.c_size = x_cap;
    VB_TRY(zgemm(g, st));
    GemmArgs h{};
    h.M = ya; h.N = yb; h.K = xa * d; h.batch = 1; h.opA = OP_C; h.opB = OP_N;
    h.A = bra->A[p]; h.lda = ya; h.B = X; h.ldb = yb; h.C = E[p + 1]; h.ldc = yb;
    h.alpha = one; h.beta = zero;
    h.a_size = (long long)xa * d * ya; h.b_size = x_cap; h.c_size = (long long)ya * yb;
    VB_TRY(zgemm(h, st));
  }
  // F_p[x', x] = sum conj(bra[x', s, y']) ket[x, s, y] F_{p+1}[y', y]
  for (int p = n - 1; p >= 0; --p) {
    const int xa = bra->bond[p], ya = bra->bond[p + 1], xb = ket->bond[p], yb = ket->bond[p + 1], d = bra->dims[p];
    GemmArgs g{};  // X[(x s), y'] = ket[(x s), y] F^T[y, y']
    g.M = xb * d; g.N = ya; g.K = yb; g.batch = 1; g.opA = OP_N; g.opB = OP_T;
    g.A = ket->A[p]; g.lda = yb; g.B = F[p + 1]; g.ldb = yb; g.C = X; g.ldc = ya;
    g.alpha = one; g.beta = zero;
    g.a_size = (long long)xb * d * yb; g.b_size = (long long)ya * yb; g.c_size = x_cap;
    VB_TRY(zgemm(g, st));
    GemmArgs h{};  // F[x', x] = conj(bra)[x', (s y')] X[x, (s y')]^T
    h.M = xa; h.N = xb; h.K = d * ya; h.batch = 1; h.opA = OP_R; h.opB = OP_T;
    h.A = bra->A[p]; h.lda = (long long)d * ya; h.B = X; h.ldb = (long long)d * ya; h.C = F[p]; h.ldc = xb;
    h.alpha = one; h.beta = zero;
    h.a_size = (long long)xa * d * ya; h.b_size = x_cap; h.c_size = (long long)xa * xb;
    VB_TRY(zgemm(h, st));
  }
  // value_j = sum E_p[x', x] conj(bra[x', s', y']) O[s', s] ket[x, s, y] F_{p+1}[y', y]
  for (int j = 0; j < n_ops; ++j) {
    const int p = sites[j];
    const int xa = bra->bond[p], ya = bra->bond[p + 1], xb = ket->bond[p], yb = ket->bond[p + 1], d = bra->dims[p];
    GemmArgs g{};  // X[x, s', y] = O[s', s] ket[x, s, y]  (batched over x)
    g.M = d; g.N = yb; g.K = d; g.batch = xb; g.opA = OP_N; g.opB = OP_N;
    g.A = ops + (size_t)j * dmax * dmax; g.lda = d; g.sA = 0;
    g.B = ket->A[p]; g.ldb = yb; g.sB = (long long)d * yb;
    g.C = X; g.ldc = yb; g.sC = (long long)d * yb;
    g.alpha = one; g.beta = zero;
    g.a_size = (long long)d * d; g.b_size = (long long)xb * d * yb; g.c_size = x_cap;
    VB_TRY(zgemm(g, st));
    GemmArgs h{};  // Y[x', (s' y)] = E_p[x', x] X[x, (s' y)]
    h.M = xa; h.N = d * yb; h.K = xb; h.batch = 1; h.opA = OP_N; h.opB = OP_N;
    h.A = E[p]; h.lda = xb; h.B = X; h.ldb = (long long)d * yb; h.C = Y; h.ldc = (long long)d * yb;
    h.alpha = one; h.beta = zero;
    h.a_size = (long long)xa * xb; h.b_size = x_cap; h.c_size = x_cap;
    VB_TRY(zgemm(h, st));
    GemmArgs k{};  // X[(x' s'), y'] = Y[(x' s'), y] F_{p+1}^T[y, y']
    k.M = xa * d; k.N = ya; k.K = yb; k.batch = 1; k.opA = OP_N; k.opB = OP_T;
    k.A = Y; k.lda = yb; k.B = F[p + 1]; k.ldb = yb; k.C = X; k.ldc = ya;
    k.alpha = one; k.beta = zero;
    k.a_size = x_cap; k.b_size = (long long)ya * yb; k.c_size = x_cap;
    VB_TRY(zgemm(k, st));
    // <bra_p, X> = sum conj(bra[x', s', y']) X[x', s', y']
    VB_TRY(vec_multi_dot(bra->A[p], 0, 1, X, (long long)xa * d * ya, out + j * out_stride, bra->d_partc,
                         reduce_parts((long long)xa * d * ya), st));
  }
  return VB_OK;
}

// weights of the composite closed Newton-Cotes rule on k_steps + 1 equally
// spaced samples (spacing h)
std::vector<double> quad_weights(int k_steps, double h) {
  std::vector<double> w(k_steps + 1, 0.0);
  int a = 0, rest = k_steps;
  auto panel = [&](int len, std::initializer_list<double> c, double scale) {
    int o = 0;
    for (double x : c) w[a + o++] += x * scale * h;
    a += len;
    rest -= len;
  };
  while (rest >= 4 && (rest % 4 == 0 || rest - 4 >= 2)) panel(4, {7, 32, 12, 32, 7}, 2.0 / 45.0);
  if (rest == 3) panel(3, {1, 3, 3, 1}, 3.0 / 8.0);
  if (rest == 2) panel(2, {1, 4, 1}, 1.0 / 3.0);
  if (rest == 1) panel(1, {1, 1}, 0.5);
  return w;
}

// q = (b + b^+)/sqrt(2) on d levels, row-major
std::vector<cd> position_operator(int d) {
  std::vector<cd> q((size_t)d * d, mkc(0.0, 0.0));
  for (int k = 0; k + 1 < d; ++k) {
    const double v = std::sqrt((double)(k + 1) / 2.0);
    q[(size_t)k * d + k + 1] = mkc(v, 0.0);
    q[(size_t)(k + 1) * d + k] = mkc(v, 0.0);
  }
  return q;
}

}  // namespace
}  // namespace vb

extern "C" vb_status tdvp2_population_gradient(vb_mps *psi, const vb_mpo *mpo, double dt_fs, int n_steps,
                                               const vb_tdvp_opts *opts, int el_state, int n_param,
                                               const int *param_mode, const int *param_i, const int *param_j,
                                               int checkpoint_every, double *pop_out, double *grad_out) {
  using namespace vb;
  if (!psi || !mpo || !opts || !pop_out || (n_param > 0 && (!param_mode || !param_i || !param_j || !grad_out)))
    return fail(VB_EINVAL, "tdvp2_population_gradient: null argument");
  if (mpo != psi->mpo) return fail(VB_EINVAL, "tdvp2_population_gradient: MPS was created for another MPO");
  if (n_steps < 1 || checkpoint_every < 1 || n_param < 0)
    return fail(VB_EINVAL, "tdvp2_population_gradient: n_steps, checkpoint_every must be >= 1");
  if (mpo->el_pos != 0) return fail(VB_EINVAL, "tdvp2_population_gradient: the electronic site must be site 0");
  const int n_el = mpo->n_el;
  if (el_state < 0 || el_state >= n_el) return fail(VB_EINVAL, "tdvp2_population_gradient: el_state out of range");
  const int n_modes = (int)mpo->pos_of_mode.size();
  for (int r = 0; r < n_param; ++r)
    if (param_mode[r] < 0 || param_mode[r] >= n_modes || param_i[r] < 0 || param_i[r] >= n_el || param_j[r] < 0 ||
        param_j[r] >= n_el)
      return fail(VB_EINVAL, "tdvp2_population_gradient: parameter out of range");
  if (psi->center != 0) return fail(VB_ESTATE, "tdvp2_population_gradient: center is not on site 0");
  VB_TRY(set_device_of(psi));
  cudaStream_t st = psi->st;
  vb::Alloc al = psi->alloc;
  Scratch sc(&al);
  // second handle for the costate and a scratch handle for the recomputed states
  vb_mps_opts o{};
  o.m_cap = psi->m_cap;
  o.dtype = psi->dtype;
  o.krylov_cap = psi->kcap;
  o.cuda_stream = st;
  o.alloc = psi->alloc.user;
  vb_mps *lam = nullptr, *work = nullptr;
  VB_TRY(mps_setup(mpo, &o, &lam));
  struct Own {
    vb_mps *a, **b;
    ~Own() {
      if (a) mps_destroy(a);
      if (*b) mps_destroy(*b);
    }
  } own{lam, &work};
  VB_TRY(mps_setup(mpo, &o, &work));
  // operators: the electronic ones |i><j| (+ |j><i|) of every parameter group,
  // and q of every parameter's mode (padded to dmax x dmax)
  int dmax = 1;
  for (int d : mpo->dims) dmax = std::max(dmax, d);
  std::vector<std::pair<int, int>> groups;
  std::vector<int> group_of(n_param);
  for (int r = 0; r < n_param; ++r) {
    const int a = std::min(param_i[r], param_j[r]), b = std::max(param_i[r], param_j[r]);
    auto it = std::find(groups.begin(), groups.end(), std::make_pair(a, b));
    group_of[r] = (int)(it - groups.begin());
    if (it == groups.end()) groups.emplace_back(a, b);
  }
  const int ng = (int)groups.size();
  std::vector<cd> h_el((size_t)(ng + 1) * n_el * n_el, mkc(0.0, 0.0));
  for (int g = 0; g < ng; ++g) {
    cd *E = h_el.data() + (size_t)g * n_el * n_el;
    E[groups[g].first * n_el + groups[g].second] = mkc(1.0, 0.0);
    E[groups[g].second * n_el + groups[g].first] = mkc(1.0, 0.0);
  }
  h_el[(size_t)ng * n_el * n_el + el_state * n_el + el_state] = mkc(1.0, 0.0);  // the projector |k><k|
  // q operators and sites in group order: the parameters of group g are
  // order[gstart[g] .. gstart[g + 1])
  std::vector<int> order, gstart(ng + 1, 0);
  for (int g = 0; g < ng; ++g) {
    gstart[g] = (int)order.size();
    for (int r = 0; r < n_param; ++r)
      if (group_of[r] == g) order.push_back(r);
  }
  gstart[ng] = (int)order.size();
  std::vector<cd> h_q((size_t)std::max(1, n_param) * dmax * dmax, mkc(0.0, 0.0));
  std::vector<int> sites(std::max(1, n_param));
  for (int u = 0; u < n_param; ++u) {
    const int p = mpo->pos_of_mode[param_mode[order[u]]];
    sites[u] = p;
    const std::vector<cd> q = position_operator(mpo->dims[p]);
    std::copy(q.begin(), q.end(), h_q.begin() + (size_t)u * dmax * dmax);
  }
  cd *d_el = nullptr, *d_q = nullptr, *d_f = nullptr;
  VB_TRY(sc.get((void **)&d_el, h_el.size() * sizeof(cd)));
  VB_TRY(sc.get((void **)&d_q, h_q.size() * sizeof(cd)));
  const int n_samples = n_steps + 1;
  VB_TRY(sc.get((void **)&d_f, (size_t)std::max(1, n_param) * n_samples * sizeof(cd)));
  VB_TRY_CUDA(cudaMemcpyAsync(d_el, h_el.data(), h_el.size() * sizeof(cd), cudaMemcpyHostToDevice, st));
  VB_TRY_CUDA(cudaMemcpyAsync(d_q, h_q.data(), h_q.size() * sizeof(cd), cudaMemcpyHostToDevice, st));
  // checkpoints every c steps (and the segment being replayed)
  const int c = std::min(checkpoint_every, n_steps);
  const int n_ckpt = (n_steps - 1) / c + 1;  // states 0, c, 2c, ... < n_steps
  const size_t sb = snap_bytes(psi);
  std::vector<Snap> ckpt(n_ckpt), seg(c + 1);
  for (Snap &x : ckpt) VB_TRY(sc.get((void **)&x.buf, sb));
  for (Snap &x : seg) VB_TRY(sc.get((void **)&x.buf, sb));
  // forward pass; the states of the last segment go straight into the
  // segment buffer, which the backward pass consumes first without a replay
  const int a_last = (n_ckpt - 1) * c;
  for (int k = 0; k < n_steps; ++k) {
    if (k % c == 0) VB_TRY(snap_save(psi, ckpt[k / c]));
    if (k >= a_last) VB_TRY(snap_save(psi, seg[k - a_last]));
    VB_TRY(tdvp2_sweep(psi, mpo, dt_fs, opts, nullptr));
  }
  VB_TRY(snap_save(psi, seg[n_steps - a_last]));
  VB_TRY(measure_populations(psi, pop_out));
  // costate at t: |k><k| psi(t), normalised (the sweeps keep unit norm); its
  // norm sqrt(P_k) scales the integrand back
  VB_TRY(snap_load(lam, seg[n_steps - a_last]));
  const double pk = pop_out[el_state];
  if (pk <= 0.0) {
    for (int r = 0; r < n_param; ++r) grad_out[r] = 0.0;
    return VB_OK;
  }
  VB_TRY(apply_site_op(lam, 0, d_el + (size_t)ng * n_el * n_el));
  {
    // rescale the center (site 0) to unit norm
    const long long el0 = (long long)lam->bond[0] * lam->dims[0] * lam->bond[1];
    const double sc0 = 1.0 / std::sqrt(pk);
    std::vector<cd> h0(el0);
    VB_TRY_CUDA(cudaMemcpyAsync(h0.data(), lam->A[0], el0 * sizeof(cd), cudaMemcpyDeviceToHost, st));
    VB_TRY_CUDA(cudaStreamSynchronize(st));
    for (cd &z : h0) z = mkc(z.x * sc0, z.y * sc0);
    VB_TRY_CUDA(cudaMemcpyAsync(lam->A[0], h0.data(), el0 * sizeof(cd), cudaMemcpyHostToDevice, st));
    VB_TRY(build_right_envs(lam));
  }
  // backward pass over the segments, last first; d_f row u = parameter order[u]
  ExpectWork ew;
  VB_TRY(ew.init(psi, sc));
  for (int sgm = n_ckpt - 1; sgm >= 0; --sgm) {
    const int a = sgm * c, b = std::min(n_steps, a + c);
    if (sgm != n_ckpt - 1) {  // replay the segment from its checkpoint
      VB_TRY(snap_load(work, ckpt[sgm]));
      for (int k = a; k <= b; ++k) {
        VB_TRY(snap_save(work, seg[k - a]));
        if (k < b) VB_TRY(tdvp2_sweep(work, mpo, dt_fs, opts, nullptr));
      }
    }
    for (int k = b; k >= a; --k) {
      if (k == b && sgm != n_ckpt - 1) continue;  // sample b was taken with the later segment
      // integrand at s_k: <lambda| q_I x |i><j| |psi(s_k)> for every parameter
      for (int g = 0; g < ng; ++g) {
        VB_TRY(snap_load(work, seg[k - a], false));
        VB_TRY(apply_site_op(work, 0, d_el + (size_t)g * n_el * n_el));
        const int u0 = gstart[g], nu = gstart[g + 1] - gstart[g];
        VB_TRY(expect_site_ops(lam, work, nu, sites.data() + u0, d_q + (size_t)u0 * dmax * dmax, dmax,
                               d_f + (size_t)u0 * n_samples + k, n_samples, ew));
      }
      if (k > 0) VB_TRY(tdvp2_sweep(lam, mpo, -dt_fs, opts, nullptr));
    }
  }
  std::vector<cd> f((size_t)std::max(1, n_param) * n_samples);
  VB_TRY_CUDA(cudaMemcpyAsync(f.data(), d_f, f.size() * sizeof(cd), cudaMemcpyDeviceToHost, st));
  VB_TRY_CUDA(cudaStreamSynchronize(st));
  const std::vector<double> w = quad_weights(n_steps, dt_fs);
  const double scale = 2.0 / HBAR_EV_FS * std::sqrt(pk);
  for (int u = 0; u < n_param; ++u) {
    double acc = 0.0;
    for (int k = 0; k < n_samples; ++k) acc += w[k] * f[(size_t)u * n_samples + k].y;
    grad_out[order[u]] = scale * acc;
  }
  return VB_OK;
}

// ===========================================================================
// Global Krylov step (Sec. 2.1.2, Eqs. Krylov subspace and global Krylov),
// with the direct MPO application (Sec. 2.1.1, Eqs. direct app 1/2), the
// compression and the MPS sums it needs, on the GPU. Used for a few
// pre-steps that grow the bonds of a product state before one-site TDVP.
//   k_0 = psi/|psi|, k_{j+1} = compress(H k_j)/|.|   (Krylov vectors as MPSs)
//   S_ij = <k_i|k_j>, H_ij = <k_i|H k_j>             (H k_j uncompressed)
//   S = L L^+, X = L^{-+}: Krylov-ordered orthonormal basis u = k X,
//   H_r = X^+ H X, b = X^+ S e_0, c = X exp(-i H_r dt/hbar) b
//   psi(t + dt) = compress(sum_j c_j k_j) scaled to |psi|.
// The Krylov vectors live in device tensors of their own (bond dimensions
// are not bounded by the handle's caps while the basis is built); only the
// result must fit the handle. Compression: Gram matrices of the left parts
// (G_{p+1} = sum_s A_p[s]^+ G_p A_p[s]), then right to left the site matrix
// M (the site times what was carried from the right) gives the reduced
// density matrix rho = M^+ G_p M of its left bond, whose leading eigenvectors
// (FP64 eigensolver, the 2TDVP split's truncation rule) become the new
// right-orthonormal site and M V_k is carried left. All contractions are
// complex FP64 GEMMs; the r x r algebra runs on the host in double.
// ===========================================================================
namespace vb {
namespace {

struct DevMps {
  std::vector<int> bond;  // [n + 1], bond[0] = bond[n] = 1
  std::vector<cd *> A;    // device [bond[p]][d_p][bond[p + 1]]
};

vb_status dm_alloc(DevMps &m, const std::vector<int> &bond, const std::vector<int> &dims, Scratch &sc) {
  const int n = (int)dims.size();
  m.bond = bond;
  m.A.assign(n, nullptr);
  for (int p = 0; p < n; ++p)
    VB_TRY(sc.get((void **)&m.A[p], (size_t)bond[p] * dims[p] * bond[p + 1] * sizeof(cd)));
  return VB_OK;
}

// out[(w a), s, (v b)] = sum_t W[w, s, t, v] A[a, t, b]  (W real)
__global__ void apply_mpo_site_kernel(const double *__restrict__ W, int wl, int d, int wr, const cd *__restrict__ A,
                                      int ml, int mr, cd *__restrict__ out) {
  const long long tot = (long long)wl * ml * d * wr * mr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long t = e;
    const int b = (int)(t % mr);
    t /= mr;
    const int v = (int)(t % wr);
    t /= wr;
    const int s = (int)(t % d);
    t /= d;
    const int a = (int)(t % ml);
    const int w = (int)(t / ml);
    const double *Wr = W + ((long long)(w * d + s) * d) * wr + v;
    cd acc = mkc(0.0, 0.0);
    for (int u = 0; u < d; ++u) {
      const double c = Wr[(long long)u * wr];
      if (c != 0.0) {
        const cd x = A[((long long)a * d + u) * mr + b];
        acc = mkc(acc.x + c * x.x, acc.y + c * x.y);
      }
    }
    out[e] = acc;
  }
}

int grid_of_elems(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16)); }

vb_status dm_apply_mpo(const vb_mpo *mpo, const std::vector<double *> &Wd, const DevMps &in, DevMps &out,
                       Scratch &sc, cudaStream_t st) {
  const int n = mpo->n;
  std::vector<int> bond(n + 1, 1);
  for (int p = 0; p <= n; ++p) {
    const int w = p == 0 ? 1 : (p == n ? 1 : mpo->sites[p].wl);
    bond[p] = in.bond[p] * w;
  }
  VB_TRY(dm_alloc(out, bond, mpo->dims, sc));
  for (int p = 0; p < n; ++p) {
    const MpoSite &S = mpo->sites[p];
    const long long tot = (long long)S.wl * in.bond[p] * S.d * S.wr * in.bond[p + 1];
    apply_mpo_site_kernel<<<grid_of_elems(tot), 256, 0, st>>>(Wd[p], S.wl, S.d, S.wr, in.A[p], in.bond[p],
                                                              in.bond[p + 1], out.A[p]);
    VB_CHECK_LAUNCH();
  }
  return VB_OK;
}

// <a|b> on the device (out: one complex)
vb_status dm_overlap(const DevMps &a, const DevMps &b, const std::vector<int> &dims, cd *out, Scratch &sc,
                     cudaStream_t st) {
  const int n = (int)dims.size();
  long long e_cap = 1, x_cap = 1;
  for (int p = 0; p <= n; ++p) e_cap = std::max<long long>(e_cap, (long long)a.bond[p] * b.bond[p]);
  for (int p = 0; p < n; ++p) x_cap = std::max<long long>(x_cap, (long long)a.bond[p] * dims[p] * b.bond[p + 1]);
  cd *E0 = nullptr, *E1 = nullptr, *X = nullptr;
  VB_TRY(sc.get((void **)&E0, e_cap * sizeof(cd)));
  VB_TRY(sc.get((void **)&E1, e_cap * sizeof(cd)));
  VB_TRY(sc.get((void **)&X, x_cap * sizeof(cd)));
  const cd one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  VB_TRY_CUDA(cudaMemcpyAsync(E0, &one, sizeof(cd), cudaMemcpyHostToDevice, st));
  for (int p = 0; p < n; ++p) {
    const int xa = a.bond[p], ya = a.bond[p + 1], xb = b.bond[p], yb = b.bond[p + 1], d = dims[p];
    GemmArgs g{};
    g.M = xa; g.N = d * yb; g.K = xb; g.batch = 1; g.opA = OP_N; g.opB = OP_N;
    g.A = E0; g.lda = xb; g.B = b.A[p]; g.ldb = (long long)d * yb; g.C = X; g.ldc = (long long)d * yb;
    g.alpha = one; g.beta = zero;
    g.a_size = (long long)xa * xb; g.b_size = (long long)xb * d * yb; g.c_size = x_cap;
    VB_TRY(zgemm(g, st));
    GemmArgs h{};
    h.M = ya; h.N = yb; h.K = xa * d; h.batch = 1; h.opA = OP_C; h.opB = OP_N;
    h.A = a.A[p]; h.lda = ya; h.B = X; h.ldb = yb; h.C = E1; h.ldc = yb;
    h.alpha = one; h.beta = zero;
    h.a_size = (long long)xa * d * ya; h.b_size = x_cap; h.c_size = e_cap;
    VB_TRY(zgemm(h, st));
    std::swap(E0, E1);
  }
  VB_TRY_CUDA(cudaMemcpyAsync(out, E0, sizeof(cd), cudaMemcpyDeviceToDevice, st));
  return VB_OK;
}

__global__ void scale_kernel(cd *x, long long n, cd c) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = cmul(x[i], c);
}

// compress `in` into a right-canonical `out` (norm on site 0) with the 2TDVP
// split's truncation rule; *disc = summed relative discarded weight
vb_status dm_compress(const DevMps &in, const std::vector<int> &dims, const TruncOpts &o, DevMps &out, double *disc,
                      Scratch &sc, cudaStream_t st) {
  const int n = (int)dims.size();
  const cd one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  *disc = 0.0;
  // Gram matrices of the left parts: G[p] (bond[p] x bond[p]), sites < p
  std::vector<cd *> G(n, nullptr);
  long long x_cap = 1;
  for (int p = 0; p < n; ++p) x_cap = std::max<long long>(x_cap, (long long)in.bond[p] * dims[p] * in.bond[p + 1]);
  cd *X = nullptr, *T = nullptr;
  VB_TRY(sc.get((void **)&X, x_cap * sizeof(cd)));
  for (int p = 0; p < n; ++p) VB_TRY(sc.get((void **)&G[p], (size_t)in.bond[p] * in.bond[p] * sizeof(cd)));
  VB_TRY_CUDA(cudaMemcpyAsync(G[0], &one, sizeof(cd), cudaMemcpyHostToDevice, st));
  for (int p = 0; p + 1 < n; ++p) {
    const int x = in.bond[p], y = in.bond[p + 1], d = dims[p];
    GemmArgs g{};  // X[x', (s y)] = G[x', x] A[x, (s y)]
    g.M = x; g.N = d * y; g.K = x; g.batch = 1; g.opA = OP_N; g.opB = OP_N;
    g.A = G[p]; g.lda = x; g.B = in.A[p]; g.ldb = (long long)d * y; g.C = X; g.ldc = (long long)d * y;
    g.alpha = one; g.beta = zero;
    g.a_size = (long long)x * x; g.b_size = (long long)x * d * y; g.c_size = x_cap;
    VB_TRY(zgemm(g, st));
    GemmArgs h{};  // G'[y', y] = sum conj(A[(x' s), y']) X[(x' s), y]
    h.M = y; h.N = y; h.K = x * d; h.batch = 1; h.opA = OP_C; h.opB = OP_N;
    h.A = in.A[p]; h.lda = y; h.B = X; h.ldb = y; h.C = G[p + 1]; h.ldc = y;
    h.alpha = one; h.beta = zero;
    h.a_size = (long long)x * d * y; h.b_size = x_cap; h.c_size = (long long)y * y;
    VB_TRY(zgemm(h, st));
  }
  // right to left: carried matrix C (bond[p + 1] x k), new sites into out
  std::vector<int> nb(n + 1, 1);
  std::vector<cd *> B(n, nullptr);
  cd *C = nullptr;
  VB_TRY(sc.get((void **)&C, sizeof(cd)));
  VB_TRY_CUDA(cudaMemcpyAsync(C, &one, sizeof(cd), cudaMemcpyHostToDevice, st));
  int kprev = 1;
  double *d_ev = nullptr, *d_tr = nullptr;
  VB_TRY(sc.get((void **)&d_tr, sizeof(double)));
  for (int p = n - 1; p >= 1; --p) {
    const int ml = in.bond[p], mr = in.bond[p + 1], d = dims[p];
    const int nr = d * kprev;  // columns of M
    cd *M = nullptr, *rho = nullptr, *evec = nullptr, *Cn = nullptr;
    VB_TRY(sc.get((void **)&M, (size_t)ml * nr * sizeof(cd)));
    VB_TRY(sc.get((void **)&T, (size_t)ml * nr * sizeof(cd)));
    VB_TRY(sc.get((void **)&rho, (size_t)nr * nr * sizeof(cd)));
    GemmArgs g{};  // M[(x s), j] = A[(x s), y] C[y, j]
    g.M = ml * d; g.N = kprev; g.K = mr; g.batch = 1; g.opA = OP_N; g.opB = OP_N;
    g.A = in.A[p]; g.lda = mr; g.B = C; g.ldb = kprev; g.C = M; g.ldc = kprev;
    g.alpha = one; g.beta = zero;
    g.a_size = (long long)ml * d * mr; g.b_size = (long long)mr * kprev; g.c_size = (long long)ml * nr;
    VB_TRY(zgemm(g, st));
    GemmArgs h{};  // T = G M  (ml x nr)
    h.M = ml; h.N = nr; h.K = ml; h.batch = 1; h.opA = OP_N; h.opB = OP_N;
    h.A = G[p]; h.lda = ml; h.B = M; h.ldb = nr; h.C = T; h.ldc = nr;
    h.alpha = one; h.beta = zero;
    h.a_size = (long long)ml * ml; h.b_size = (long long)ml * nr; h.c_size = (long long)ml * nr;
    VB_TRY(zgemm(h, st));
    GemmArgs r{};  // rho = M^+ T  (nr x nr)
    r.M = nr; r.N = nr; r.K = ml; r.batch = 1; r.opA = OP_C; r.opB = OP_N;
    r.A = M; r.lda = nr; r.B = T; r.ldb = nr; r.C = rho; r.ldc = nr;
    r.alpha = one; r.beta = zero;
    r.a_size = (long long)ml * nr; r.b_size = (long long)ml * nr; r.c_size = (long long)nr * nr;
    VB_TRY(zgemm(r, st));
    trace_kernel<<<1, 256, 0, st>>>(rho, nr, d_tr);
    VB_CHECK_LAUNCH();
    const int kw = std::min(nr, o.m_max + 1);
    void *work = nullptr;
    VB_TRY(sc.get(&work, EigWork::bytes(nr, kw)));
    VB_TRY(sc.get((void **)&d_ev, (size_t)kw * sizeof(double)));
    VB_TRY(eig_values(nr, rho, kw, d_ev, work, st));
    std::vector<double> lam(kw);
    double tot = 0.0;
    VB_TRY_CUDA(cudaMemcpyAsync(lam.data(), d_ev, kw * sizeof(double), cudaMemcpyDeviceToHost, st));
    VB_TRY_CUDA(cudaMemcpyAsync(&tot, d_tr, sizeof(double), cudaMemcpyDeviceToHost, st));
    VB_TRY_CUDA(cudaStreamSynchronize(st));
    VB_TRY(EigWork::check(nr, kw, sizeof(double), work, st));
    for (double &x : lam) x = std::max(x, 0.0);
    // the Schmidt rank is also bounded by the full dimension of the sites to
    // the left (the input's own bond may be far larger, e.g. w m after H)
    long long left_full = 1;
    for (int q = 0; q < p && left_full < (1LL << 30); ++q) left_full *= dims[q];
    const int rank_bound = (int)std::min<long long>(std::min(ml, nr), left_full);
    double dd = 0.0;
    const int k = choose_rank(lam, nr, tot, rank_bound, o, &dd);
    *disc += dd;
    VB_TRY(sc.get((void **)&evec, (size_t)k * nr * sizeof(cd)));
    VB_TRY(eig_vectors(nr, rho, kw, k, d_ev, evec, work, st));
    // new site: rows conj(v_j) (k x d x kprev), right-orthonormal
    VB_TRY(sc.get((void **)&B[p], (size_t)k * nr * sizeof(cd)));
    conj_copy_kernel<<<grid_of_elems((long long)k * nr), 256, 0, st>>>(evec, (long long)k * nr, B[p]);
    VB_CHECK_LAUNCH();
    // carried: C' = M V_k  (ml x k), V_k[(s j'), j] = evec[j][(s j')]
    VB_TRY(sc.get((void **)&Cn, (size_t)ml * k * sizeof(cd)));
    GemmArgs c{};
    c.M = ml; c.N = k; c.K = nr; c.batch = 1; c.opA = OP_N; c.opB = OP_T;
    c.A = M; c.lda = nr; c.B = evec; c.ldb = nr; c.C = Cn; c.ldc = k;
    c.alpha = one; c.beta = zero;
    c.a_size = (long long)ml * nr; c.b_size = (long long)k * nr; c.c_size = (long long)ml * k;
    VB_TRY(zgemm(c, st));
    C = Cn;
    kprev = k;
    nb[p] = k;
  }
  // site 0 absorbs the carried matrix
  {
    const int d = dims[0], mr = in.bond[1];
    VB_TRY(sc.get((void **)&B[0], (size_t)d * kprev * sizeof(cd)));
    GemmArgs g{};
    g.M = d; g.N = kprev; g.K = mr; g.batch = 1; g.opA = OP_N; g.opB = OP_N;
    g.A = in.A[0]; g.lda = mr; g.B = C; g.ldb = kprev; g.C = B[0]; g.ldc = kprev;
    g.alpha = one; g.beta = zero;
    g.a_size = (long long)d * mr; g.b_size = (long long)mr * kprev; g.c_size = (long long)d * kprev;
    VB_TRY(zgemm(g, st));
  }
  out.bond = nb;
  out.A = B;
  return VB_OK;
}

// sum_j c_j |k_j> (block tensors: site 0 side by side with the c_j, the
// last site stacked, the others block-diagonal)
__global__ void put_block_kernel(const cd *__restrict__ src, int sl, int d, int sr, cd *__restrict__ dst, int dl,
                                 int dr, int r0, int c0, cd scale) {
  const long long tot = (long long)sl * d * sr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(e % sr);
    const long long t = e / sr;
    const int s = (int)(t % d);
    const int x = (int)(t / d);
    dst[((long long)(r0 + x) * d + s) * dr + c0 + y] = cmul(src[e], scale);
  }
}

vb_status dm_sum(const std::vector<std::complex<double>> &c, const std::vector<DevMps> &K, const std::vector<int> &dims,
                 DevMps &out, Scratch &sc, cudaStream_t st) {
  const int n = (int)dims.size(), m = (int)c.size();
  std::vector<int> bond(n + 1, 1);
  for (int p = 1; p < n; ++p) {
    bond[p] = 0;
    for (int j = 0; j < m; ++j) bond[p] += K[j].bond[p];
  }
  VB_TRY(dm_alloc(out, bond, dims, sc));
  for (int p = 0; p < n; ++p)
    VB_TRY_CUDA(cudaMemsetAsync(out.A[p], 0, (size_t)bond[p] * dims[p] * bond[p + 1] * sizeof(cd), st));
  std::vector<int> r0(n + 1, 0);
  for (int j = 0; j < m; ++j) {
    for (int p = 0; p < n; ++p) {
      const int sl = K[j].bond[p], sr = K[j].bond[p + 1];
      const int ro = p == 0 ? 0 : r0[p], co = p == n - 1 ? 0 : r0[p + 1];
      const cd scale = p == 0 ? mkc(c[j].real(), c[j].imag()) : mkc(1.0, 0.0);
      put_block_kernel<<<grid_of_elems((long long)sl * dims[p] * sr), 256, 0, st>>>(
          K[j].A[p], sl, dims[p], sr, out.A[p], bond[p], bond[p + 1], ro, co, scale);
      VB_CHECK_LAUNCH();
    }
    for (int p = 1; p < n; ++p) r0[p] += K[j].bond[p];
  }
  return VB_OK;
}

// ---- small dense complex Hermitian algebra on the host (r <= 64)
typedef std::complex<double> zc;

// cyclic Jacobi: A (r x r Hermitian, row-major) -> eigenvalues lam, eigenvectors as columns of V
void herm_jacobi(std::vector<zc> A, int r, std::vector<double> &lam, std::vector<zc> &V) {
  V.assign((size_t)r * r, zc(0.0, 0.0));
  for (int i = 0; i < r; ++i) V[(size_t)i * r + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int p = 0; p < r; ++p)
      for (int q = 0; q < r; ++q) (p == q ? dia : off) += std::norm(A[(size_t)p * r + q]);
    if (off <= 1e-30 * std::max(dia, 1e-300)) break;
    for (int p = 0; p < r; ++p)
      for (int q = p + 1; q < r; ++q) {
        const zc apq = A[(size_t)p * r + q];
        const double g = std::abs(apq);
        if (g == 0.0) continue;
        const double app = A[(size_t)p * r + p].real(), aqq = A[(size_t)q * r + q].real();
        const double theta = 0.5 * std::atan2(2.0 * g, aqq - app);
        const double cs = std::cos(theta), sn = std::sin(theta);
        const zc ph = apq / g;  // e^{i phi}
        // rotation: columns p, q of A and V: a_p' = cs a_p - sn conj(ph) a_q ... (unitary J)
        for (int k = 0; k < r; ++k) {
          const zc akp = A[(size_t)k * r + p], akq = A[(size_t)k * r + q];
          A[(size_t)k * r + p] = cs * akp - sn * std::conj(ph) * akq;
          A[(size_t)k * r + q] = sn * ph * akp + cs * akq;
        }
        for (int k = 0; k < r; ++k) {
          const zc apk = A[(size_t)p * r + k], aqk = A[(size_t)q * r + k];
          A[(size_t)p * r + k] = cs * apk - sn * ph * aqk;
          A[(size_t)q * r + k] = sn * std::conj(ph) * apk + cs * aqk;
        }
        for (int k = 0; k < r; ++k) {
          const zc vkp = V[(size_t)k * r + p], vkq = V[(size_t)k * r + q];
          V[(size_t)k * r + p] = cs * vkp - sn * std::conj(ph) * vkq;
          V[(size_t)k * r + q] = sn * ph * vkp + cs * vkq;
        }
      }
  }
  lam.resize(r);
  for (int i = 0; i < r; ++i) lam[i] = A[(size_t)i * r + i].real();
}

// Cholesky S = L L^+ (lower); false when S is not positive definite
bool herm_cholesky(const std::vector<zc> &S, int r, std::vector<zc> &L) {
  L.assign((size_t)r * r, zc(0.0, 0.0));
  for (int j = 0; j < r; ++j) {
    double dgl = S[(size_t)j * r + j].real();
    for (int k = 0; k < j; ++k) dgl -= std::norm(L[(size_t)j * r + k]);
    if (!(dgl > 0.0)) return false;
    const double ljj = std::sqrt(dgl);
    L[(size_t)j * r + j] = ljj;
    for (int i = j + 1; i < r; ++i) {
      zc s = S[(size_t)i * r + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * r + k] * std::conj(L[(size_t)j * r + k]);
      L[(size_t)i * r + j] = s / ljj;
    }
  }
  return true;
}

}  // namespace
}  // namespace vb

extern "C" vb_status global_krylov_step(vb_mps *psi, const vb_mpo *mpo, double dt_fs, const vb_tdvp_opts *opts,
                                        int r_max, double tol, vb_krylov_info *info) {
  using namespace vb;
  if (!psi || !mpo || !opts) return fail(VB_EINVAL, "global_krylov_step: null argument");
  if (mpo != psi->mpo) return fail(VB_EINVAL, "global_krylov_step: MPS was created for another MPO");
  if (psi->center != 0) return fail(VB_ESTATE, "global_krylov_step: center is not on site 0");
  if (r_max < 1 || r_max > 40 || !(tol > 0.0) || opts->m_max < 1 || opts->m_max > psi->m_cap)
    return fail(VB_EINVAL, "global_krylov_step: r_max in 1..40, tol > 0, m_max in 1..m_cap");
  if (psi->n < 2) return fail(VB_EINVAL, "global_krylov_step: needs at least two sites");
  VB_TRY(set_device_of(psi));
  cudaStream_t st = psi->st;
  vb::Alloc al = psi->alloc;
  Scratch sc(&al);
  const int n = psi->n;
  const std::vector<int> &dims = psi->dims;
  const TruncOpts to{opts->m_max, opts->eps, opts->zero_floor};
  vb_krylov_info inf{};
  // dense MPO tensors on the device
  std::vector<double *> Wd(n, nullptr);
  for (int p = 0; p < n; ++p) {
    const MpoSite &S = mpo->sites[p];
    VB_TRY(sc.get((void **)&Wd[p], S.dense.size() * sizeof(double)));
    VB_TRY_CUDA(cudaMemcpyAsync(Wd[p], S.dense.data(), S.dense.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  cd *d_z = nullptr;
  VB_TRY(sc.get((void **)&d_z, sizeof(cd)));
  auto overlap = [&](const DevMps &a, const DevMps &b, zc *v) -> vb_status {
    VB_TRY(dm_overlap(a, b, dims, d_z, sc, st));
    cd h;
    VB_TRY_CUDA(cudaMemcpyAsync(&h, d_z, sizeof(cd), cudaMemcpyDeviceToHost, st));
    VB_TRY_CUDA(cudaStreamSynchronize(st));
    *v = zc(h.x, h.y);
    return VB_OK;
  };
  auto scale0 = [&](DevMps &a, zc c) {
    const long long el = (long long)a.bond[0] * dims[0] * a.bond[1];
    scale_kernel<<<grid_of_elems(el), 256, 0, st>>>(a.A[0], el, mkc(c.real(), c.imag()));
  };
  // k_0 = psi / |psi| (its own copy)
  DevMps k0;
  VB_TRY(dm_alloc(k0, psi->bond, dims, sc));
  for (int p = 0; p < n; ++p)
    VB_TRY_CUDA(cudaMemcpyAsync(k0.A[p], psi->A[p], (size_t)psi->bond[p] * dims[p] * psi->bond[p + 1] * sizeof(cd),
                                cudaMemcpyDeviceToDevice, st));
  zc nn0;
  VB_TRY(overlap(k0, k0, &nn0));
  const double nrm = std::sqrt(std::abs(nn0.real()));
  if (nrm == 0.0) return fail(VB_EINVAL, "global_krylov_step: zero state");
  scale0(k0, zc(1.0 / nrm, 0.0));
  VB_CHECK_LAUNCH();
  std::vector<DevMps> K{k0}, HK;
  std::vector<zc> S(1, zc(1.0, 0.0)), Hm;
  std::vector<zc> cvec;
  auto solve = [&](int m, std::vector<zc> &c, std::vector<zc> &ub) -> bool {
    std::vector<zc> L;
    if (!herm_cholesky(S, m, L)) return false;
    // X = L^{-+}: solve L^+ X = I (upper triangular)
    std::vector<zc> X((size_t)m * m, zc(0.0, 0.0));
    for (int col = 0; col < m; ++col)
      for (int i = m - 1; i >= 0; --i) {
        zc s = (i == col) ? zc(1.0, 0.0) : zc(0.0, 0.0);
        for (int k = i + 1; k < m; ++k) s -= std::conj(L[(size_t)k * m + i]) * X[(size_t)k * m + col];
        X[(size_t)i * m + col] = s / std::conj(L[(size_t)i * m + i]);
      }
    std::vector<zc> Hr((size_t)m * m, zc(0.0, 0.0)), T((size_t)m * m, zc(0.0, 0.0));
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        for (int k = 0; k < m; ++k) T[(size_t)i * m + j] += Hm[(size_t)i * m + k] * X[(size_t)k * m + j];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        for (int k = 0; k < m; ++k) Hr[(size_t)i * m + j] += std::conj(X[(size_t)k * m + i]) * T[(size_t)k * m + j];
    for (int i = 0; i < m; ++i)
      for (int j = i; j < m; ++j) {
        const zc a = 0.5 * (Hr[(size_t)i * m + j] + std::conj(Hr[(size_t)j * m + i]));
        Hr[(size_t)i * m + j] = a;
        Hr[(size_t)j * m + i] = std::conj(a);
      }
    std::vector<double> lam;
    std::vector<zc> V;
    herm_jacobi(Hr, m, lam, V);
    std::vector<zc> b(m, zc(0.0, 0.0));
    for (int i = 0; i < m; ++i)
      for (int k = 0; k < m; ++k) b[i] += std::conj(X[(size_t)k * m + i]) * S[(size_t)k * m + 0];
    std::vector<zc> y(m, zc(0.0, 0.0));
    for (int a = 0; a < m; ++a) {
      zc s(0.0, 0.0);
      for (int i = 0; i < m; ++i) s += std::conj(V[(size_t)i * m + a]) * b[i];
      y[a] = std::exp(zc(0.0, -lam[a] * dt_fs / HBAR_EV_FS)) * s;
    }
    ub.assign(m, zc(0.0, 0.0));
    for (int i = 0; i < m; ++i)
      for (int a = 0; a < m; ++a) ub[i] += V[(size_t)i * m + a] * y[a];
    c.assign(m, zc(0.0, 0.0));
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) c[i] += X[(size_t)i * m + j] * ub[j];
    return true;
  };
  // H_00 through H k_0 (the first uncompressed vector)
  {
    DevMps hk;
    VB_TRY(dm_apply_mpo(mpo, Wd, K[0], hk, sc, st));
    HK.push_back(hk);
    zc h;
    VB_TRY(overlap(K[0], HK[0], &h));
    Hm.assign(1, h);
  }
  std::vector<zc> ub;
  if (!solve(1, cvec, ub)) return fail(VB_ECUDA, "global_krylov_step: Gram matrix not positive");
  for (int r = 1; r <= r_max; ++r) {
    DevMps nxt;
    double dd = 0.0;
    VB_TRY(dm_compress(HK.back(), dims, to, nxt, &dd, sc, st));
    zc nn;
    VB_TRY(overlap(nxt, nxt, &nn));
    if (nn.real() <= 0.0) {
      inf.converged = 1;
      break;
    }
    scale0(nxt, zc(1.0 / std::sqrt(nn.real()), 0.0));
    VB_CHECK_LAUNCH();
    const int m = (int)K.size() + 1;
    std::vector<zc> S2((size_t)m * m);
    for (int i = 0; i < m - 1; ++i)
      for (int j = 0; j < m - 1; ++j) S2[(size_t)i * m + j] = S[(size_t)i * (m - 1) + j];
    for (int i = 0; i < m - 1; ++i) {
      zc v;
      VB_TRY(overlap(K[i], nxt, &v));
      S2[(size_t)i * m + m - 1] = v;
      S2[(size_t)(m - 1) * m + i] = std::conj(v);
    }
    S2[(size_t)(m - 1) * m + m - 1] = zc(1.0, 0.0);
    std::vector<double> ev;
    std::vector<zc> Vs;
    herm_jacobi(S2, m, ev, Vs);
    const double emin = *std::min_element(ev.begin(), ev.end()), emax = *std::max_element(ev.begin(), ev.end());
    if (emin <= 1e-13 * emax) {  // the new vector lies in the span: the space is invariant
      inf.converged = 1;
      break;
    }
    K.push_back(nxt);
    S = S2;
    inf.disc_basis += dd;
    int mb = 1;
    for (int p = 1; p < n; ++p) mb = std::max(mb, nxt.bond[p]);
    inf.max_bond_basis = std::max(inf.max_bond_basis, mb);
    // H k_{m-1} (uncompressed) and the new row / column of H
    DevMps hk;
    VB_TRY(dm_apply_mpo(mpo, Wd, K.back(), hk, sc, st));
    HK.push_back(hk);
    std::vector<zc> H2((size_t)m * m);
    for (int i = 0; i < m - 1; ++i)
      for (int j = 0; j < m - 1; ++j) H2[(size_t)i * m + j] = Hm[(size_t)i * (m - 1) + j];
    for (int i = 0; i < m; ++i) {
      zc v;
      VB_TRY(overlap(K[i], HK[m - 1], &v));
      H2[(size_t)i * m + m - 1] = v;
      if (i < m - 1) {
        zc w;
        VB_TRY(overlap(K[m - 1], HK[i], &w));
        H2[(size_t)(m - 1) * m + i] = w;
      }
    }
    Hm = H2;
    if (!solve(m, cvec, ub)) return fail(VB_ECUDA, "global_krylov_step: Gram matrix not positive");
    inf.r = r;
    if (std::abs(ub.back()) < tol) {
      inf.converged = 1;
      break;
    }
  }
  // the new state: sum_j c_j k_j, compressed, scaled to |psi|
  DevMps sum, out;
  VB_TRY(dm_sum(cvec, std::vector<DevMps>(K.begin(), K.begin() + cvec.size()), dims, sum, sc, st));
  double dd = 0.0;
  VB_TRY(dm_compress(sum, dims, to, out, &dd, sc, st));
  inf.disc_final = dd;
  zc on;
  VB_TRY(overlap(out, out, &on));
  for (int p = 1; p < n; ++p)
    if (out.bond[p] > psi->bcap[p])
      return fail(VB_EINVAL, "global_krylov_step: result bond exceeds the handle's capacity");
  scale0(out, zc(nrm / std::sqrt(on.real()), 0.0));
  VB_CHECK_LAUNCH();
  for (int p = 0; p < n; ++p)
    VB_TRY_CUDA(cudaMemcpyAsync(psi->A[p], out.A[p], (size_t)out.bond[p] * dims[p] * out.bond[p + 1] * sizeof(cd),
                                cudaMemcpyDeviceToDevice, st));
  psi->bond = out.bond;
  psi->center = 0;
  VB_TRY(build_right_envs(psi));
  VB_TRY_CUDA(cudaStreamSynchronize(st));
  if (info) *info = inf;
  return VB_OK;
}
