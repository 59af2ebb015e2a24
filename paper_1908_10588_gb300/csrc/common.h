// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/vibtdvp.h"

namespace vb {

// ------------------------------------------------------------ errors
void set_error(const std::string &msg);
const char *get_error();

#define VB_TRY_CUDA(call)                                                        \
  do {                                                                           \
    cudaError_t _e = (call);                                                     \
    if (_e != cudaSuccess) {                                                     \
      ::vb::set_error(std::string(#call) + ": " + cudaGetErrorString(_e) + " (" + \
                      __FILE__ + ":" + std::to_string(__LINE__) + ")");          \
      return VB_ECUDA;                                                           \
    }                                                                            \
  } while (0)

#define VB_TRY(call)               \
  do {                             \
    vb_status _s = (call);         \
    if (_s != VB_OK) return _s;    \
  } while (0)

void count_launch();
#define VB_CHECK_LAUNCH()  \
  do {                     \
    ::vb::count_launch();  \
    VB_TRY_CUDA(cudaGetLastError()); \
  } while (0)

// ---- per-phase event profiler (host side, single-threaded use)
enum { PH_HEFF2 = 0, PH_HEFF1 = 1, PH_KRYLOV = 2, PH_SPLIT = 3, PH_ENV = 4, PH_MERGE = 5, PH_RHO = 6, PH_EIGVAL = 7,
       PH_EIGVEC = 8, PH_SPLITOUT = 9, PH_SUBPROD = 10, PH_SUBORTH = 11, PH_INVIT = 12,
       PH_CGS = 13, PH_BACKT = 14, PH_RR = 15, PH_RR32 = 16, PH_RR64 = 17, PH_CHOL = 18,
       PH_ORTHGEMM = 19, PH_TC = 20, PH_WLEG = 21, PH_PREP = 22, PH_JACOBI = 23, PH_COUNT = 24 };
bool prof_on();
void prof_begin(int phase, cudaStream_t st);
// flops / bytes: algorithmic work of the call, summed per phase
void prof_end(int phase, cudaStream_t st, double flops, double bytes = 0.0);
void prof_collect();  // after a stream synchronisation: fold finished events into the totals
// add a count to a phase's flops slot (PH_JACOBI: Jacobi sweeps, not flops)
void prof_note(int phase, double v);

inline vb_status fail(vb_status s, const std::string &msg) {
  set_error(msg);
  return s;
}

// ------------------------------------------------------------ complex
// interleaved complex of real type R (double on the FP64 path, float on the
// mixed path); same memory layout as C99 complex
template <class R>
struct alignas(2 * sizeof(R)) cplx {
  R x, y;
};
typedef cplx<double> cd;
typedef cplx<float> cf;

template <class R>
__host__ __device__ inline cplx<R> mkc(R a, R b) {
  cplx<R> r;
  r.x = a;
  r.y = b;
  return r;
}
template <class R>
__host__ __device__ inline cplx<R> cadd(cplx<R> a, cplx<R> b) { return mkc<R>(a.x + b.x, a.y + b.y); }
template <class R>
__host__ __device__ inline cplx<R> csub(cplx<R> a, cplx<R> b) { return mkc<R>(a.x - b.x, a.y - b.y); }
template <class R>
__host__ __device__ inline cplx<R> cmul(cplx<R> a, cplx<R> b) {
  return mkc<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class R>
__host__ __device__ inline cplx<R> cconj(cplx<R> a) { return mkc<R>(a.x, -a.y); }
template <class R>
__host__ __device__ inline cplx<R> cscale(cplx<R> a, R s) { return mkc<R>(a.x * s, a.y * s); }
// conj(a) * b
template <class R>
__host__ __device__ inline cplx<R> cdotc(cplx<R> a, cplx<R> b) {
  return mkc<R>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <class R>
__host__ __device__ inline R cabs2(cplx<R> a) { return a.x * a.x + a.y * a.y; }

// ------------------------------------------------------------ memory
struct Alloc {
  const vb_allocator *user = nullptr;
  cudaStream_t stream = nullptr;
  vb_status get(void **p, size_t bytes);
  void put(void *p);
};

// Device buffer owned by a handle.
struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
  template <class T>
  T *as() const {
    return reinterpret_cast<T *>(p);
  }
};

// ------------------------------------------------------------ GEMM
// op codes for the strided batched complex GEMM
enum Op { OP_N = 0, OP_T = 1, OP_C = 2 /* conj transpose */, OP_R = 3 /* conj, no transpose */ };

template <class R>
struct GemmArgsT {
  int M, N, K, batch;
  int opA, opB;
  const cplx<R> *A;
  long long lda, sA;
  const cplx<R> *B;
  long long ldb, sB;
  cplx<R> *C;
  long long ldc, sC;
  cplx<R> alpha, beta;
  // element counts of the three buffers (required); every address the
  // kernel forms is checked against them on the host before the launch
  long long a_size, b_size, c_size;
  // optional split-K (batch must be 1): the K range is cut into chunks of kc
  // that run as separate CTAs into ws (ws_elems >= chunks * M * N), then an
  // ordered reduction writes C; used when M x N alone gives too few CTAs
  cplx<R> *ws;
  long long ws_elems;
  // internal: set by gemm() for the chunk launch
  long long kc, kfull;
};
typedef GemmArgsT<double> GemmArgs;
typedef GemmArgsT<float> GemmArgsF;
// C[b] = alpha op(A[b]) op(B[b]) + beta C[b]; op(A) is M x K, op(B) is K x N.
template <class R>
vb_status gemm(const GemmArgsT<R> &g, cudaStream_t st);
inline vb_status zgemm(const GemmArgs &g, cudaStream_t st) { return gemm<double>(g, st); }

// ------------------------------------------------------------ MPO
// Terms of the vibronic Hamiltonian (Eqs. Hel_2, Hvib_2, Helvib_2) as
// products of local operators. A factor's `pos` is a chain position in the
// builder; model_terms() returns factors on entities instead: ENT_EL the
// electronic site, k >= 0 mode k, ENT_POS0 chain position 0 whatever sits
// there (the zero-point constant).
enum { OPC_ID = 0, OPC_Q = 1, OPC_Q2 = 2, OPC_N = 3, OPC_E = 16 /* + i*n_el + j */ };
constexpr int ENT_EL = -1, ENT_POS0 = -2;
struct Factor {
  int pos, code;
};
struct Term {
  double coef;
  std::vector<Factor> f;
};
// every nonzero term of the model, factors on entities (unsorted); checks the
// coupling indices; `who` prefixes error messages
vb_status model_terms(const vb_model *m, const char *who, std::vector<Term> &terms);

// algorithmic floating-point operations of one H_eff,2 application at the
// pair (i, i + 1): the left environment contraction, the two W-site
// applications (a non-identity d x d block costs 4 d^2 per stacked vector,
// an identity block 2 d) and the right environment contraction
inline double heff2_flops_of(double mL, double mR, int d1, int d2, int wl1, int wr2, long long nop1,
                             long long nid1, long long nop2, long long nid2) {
  const double th = mL * d1 * d2 * mR;
  const double w1 = (double)nid1 * 2.0 * d1 + (double)nop1 * 4.0 * d1 * d1;
  const double w2 = (double)nid2 * 2.0 * d2 + (double)nop2 * 4.0 * d2 * d2;
  return 8.0 * th * mL * wl1 + w1 * (mL * d2 * mR) + w2 * (mL * d1 * mR) + 8.0 * th * wr2 * mR;
}

struct MpoBlock {
  int win, wout;
  int ident;   // operator is the identity
  int op_off;  // row-pointer base of the operator in csr_ptr (non-identity blocks)
};

struct MpoSite {
  int wl = 0, d = 0, wr = 0;
  std::vector<double> dense;  // [wl][d][d][wr]
  std::vector<MpoBlock> blocks;
  std::vector<double> ops;  // concatenated non-identity operators
  // the same operators row-compressed: for a block whose entry carries
  // off = b, rows so have nonzeros csr_col/val[csr_ptr[b + so] .. csr_ptr[b + so + 1])
  std::vector<int> csr_ptr, csr_col;
  std::vector<double> csr_val;
  // device copies: operators, and for each direction a CSR over the produced
  // bond index: entries (consumed index, ident, operator row-pointer base)
  double *d_ops = nullptr;
  float *d_ops32 = nullptr;
  int *d_csr_ptr = nullptr, *d_csr_col = nullptr;
  double *d_csr_val = nullptr;
  float *d_csr_val32 = nullptr;
  int *d_fwd_ptr = nullptr, *d_fwd_ent = nullptr;  // produce w_out from w_in
  int *d_bwd_ptr = nullptr, *d_bwd_ent = nullptr;  // produce w_in from w_out
  long long nnz_ops = 0;                           // non-identity blocks
  long long n_ident = 0;
};

}  // namespace vb

struct vb_mpo {
  int n = 0;
  int n_el = 0;
  int el_pos = 0;
  std::vector<int> dims;
  std::vector<int> pos_of_mode;  // chain position of every vibrational mode
  // channels of bond b - 1 (b = 0 .. n; the left block L[b] and the right
  // block R[b] carry them): the one with no operator placed yet (START, the
  // right block's complete Hamiltonian) and the finished one (DONE, the left
  // block's complete Hamiltonian); -1 where absent
  std::vector<int> ch_start, ch_done;
  // zero-point energy sum_I hbar omega_I / 2 (Eq. Hvib_2), a constant the MPO
  // carries as an identity term on site 0. The FP32 operators of the mixed
  // form leave it out (their rounding errors then scale with the spread of
  // H, not with this offset, which for a 300-mode bath is ~30 eV); a mixed
  // sweep restores it as the exact global phase exp(-i e_zpe dt / hbar).
  double e_zpe = 0.0;
  std::vector<vb::MpoSite> sites;
  int max_w = 0;
  int max_d = 0;
  bool uploaded = false;
  int device = -1;
  std::vector<void *> dev_allocs;
};

namespace vb {
vb_status mpo_upload(const vb_mpo *mpo);

// Sparse MPO application, one site:
//  dir 0: Y[p, s', wo, q] = sum_{blocks wi->wo} sum_s O[s', s] X[p, wi, s, q]
//  dir 1: Y[p, s', wi, q] = sum_{blocks wi->wo} sum_s O[s', s] X[p, wo, s, q]
struct WStrides {
  long long p, w, s, q;
};
// strides named explicitly: WS(p=..., w=..., s=..., q=...)
inline WStrides WS(long long p, long long w, long long s, long long q) { return WStrides{p, w, s, q}; }
// x_size / y_size: element counts of X and Y; the largest offset the kernel
// forms is checked against them before the launch
template <class R>
vb_status wapply(const MpoSite &site, int dir, const cplx<R> *X, WStrides xs, long long x_size,
                 cplx<R> *Y, WStrides ys, long long y_size, int P, int Q, cudaStream_t st);

// ------------------------------------------------------------ vectors
vb_status vec_multi_dot(const cd *V, long long ldv, int nv, const cd *w, long long n, cd *out,
                        cd *partial, int n_part, cudaStream_t st, unsigned int *cnt = nullptr);
// w -= sum_j c[j] V[j] (sign = -1) or w += ... (sign = +1); c on device; cscale applied
// w32 (nullable): also write the FP32 copy of the result
vb_status vec_multi_axpy(const cd *V, long long ldv, int nv, const cd *c, double sign, cd *w,
                         long long n, cudaStream_t st, cf *w32 = nullptr);
// Gram-Schmidt of the mixed form on FP32 copies of the Krylov vectors (FP32
// products, FP64 sums; cnt: zeroed counters, required). vs (nullable): the
// copies are stored unnormalised and vs[j] is the factor that normalises
// copy j; the inner products returned are those with the normalised vectors
// and the coefficients given are applied to them.
struct LanczosRecord {  // written by the last block of the full-pass update (all nullable)
  double *vs_next;      // 1/|w| (0 for w = 0): factor of the new vector's stored copies
  double *beta_k;       // |w|
  double *alpha_k;      // Re(ck + c2k)
  const cd *ck, *c2k;
};
vb_status vec_multi_dot32(const cf *V, long long ldv, int nv, const cf *w, long long n, cd *out, cd *partial,
                          int n_part, cudaStream_t st, unsigned int *cnt, const double *vs = nullptr);
// the update of the FP64 w followed by |w| (into out); w32 (nullable) gets
// the FP32 copy of the new w
vb_status vec_multi_axpy32_norm(const cf *V, long long ldv, int nv, const cd *c, double sign, cd *w, long long n,
                                double *out, double *partial, cudaStream_t st, unsigned int *cnt,
                                const double *vs = nullptr, cf *w32 = nullptr,
                                const LanczosRecord &rec = LanczosRecord{});
// the same update without the norm, writing the FP32 copy of the new w into w32
vb_status vec_multi_axpy32(const cf *V, long long ldv, int nv, const cd *c, double sign, cd *w, long long n,
                           cf *w32, cudaStream_t st, const double *vs = nullptr);
// inner products of FP32 copies with the FP64 w rounded to FP32 on load
vb_status vec_multi_dot32(const cf *V, long long ldv, int nv, const cd *w, long long n, cd *out, cd *partial,
                          int n_part, cudaStream_t st, unsigned int *cnt, const double *vs = nullptr);
// w += sign * sum_{j<n1} c1_j V1_j (n1 <= 2, FP32 correction; vs1: factors of
// the V1 copies) fused with out_j = <V_j, w32> for j < nv on the updated w
// (vs: factors of the V copies); partial holds partial_elems complex entries,
// cnt one zeroed counter. axpy_dot32_blocks gives the block count it would
// use, 0 where the sizes do not fit (then use the two passes).
constexpr long long AXPY_DOT_CHUNK = 4096;       // elements per block aimed at
constexpr long long AXPY_DOT_MAX_CHUNK = 12288;  // shared-memory bound (96 KB)
constexpr long long AXPY_DOT_MAX_BLOCKS = 2048;
constexpr long long PARTC_ELEMS = 2048LL * 64;   // complex partial sums per handle
int axpy_dot32_blocks(long long n, int nv, long long partial_elems);
vb_status vec_axpy_dot32(const cf *V1, int n1, const cd *c1, double sign, cd *w, long long n, const cf *V,
                         long long ldv, int nv, cd *out, cd *partial, long long partial_elems, cudaStream_t st,
                         unsigned int *cnt, const double *vs1 = nullptr, const double *vs = nullptr);
// ------------------------------------------------------------ subspace iteration
struct SubspaceWork {
  cf *G, *W, *T;  // r x r Gram matrix, r x r transform, r x n scratch rows
  int *flag;      // r + 1: rows refilled at random, then their count
  cf *ws;         // split-K workspace of the Gram product
  long long ws_elems;
};
// largest subspace of the mixed split (m_max + 9 rows for bond caps up to 135)
constexpr int SUBSPACE_MAX_R = 144;
size_t subspace_chol_smem(int r);
// Q (r x n, FP32 rows): rows j < m_warm copied from the old bond tensor (left:
// n x m_old, row j = column j; right: m_old x n, row j = row j), the others
// drawn from a counter-based generator keyed by seed
vb_status subspace_init(cf *Q, int r, int n, const cd *warm, int m_old, int m_warm, bool left,
                        unsigned long long seed, cudaStream_t st);
// orthonormalise the rows of Q (r <= SUBSPACE_MAX_R) in place: row-scaled Cholesky QR,
// twice; rows found dependent are refilled at random before the second pass
vb_status subspace_orth(cf *Q, int r, int n, const SubspaceWork &w, unsigned long long seed, cudaStream_t st);
// k largest eigenpairs of a small Hermitian S (2 <= n <= 112) by a one-CTA
// Jacobi solver: evals descending, eigenvectors as rows W[k][n]; info[0] =
// sweeps used. VB_EINVAL for larger n (use eig_values / eig_vectors)
vb_status ritz_eig_small(const cf *S, int n, int k, float *evals, cf *W, int *info, cudaStream_t st);
// FP64 Cholesky factor W (r x r, r <= 112) with W G W^+ = I on the accepted
// rows of the Gram matrix G; rejected rows (scaled pivot <= 1e-28: zero rows
// and exact dependencies) are zero in W with flag[i] = 1, flag[r] = their count
vb_status chol_w64(const cd *G, int r, cd *W, int *flag, cudaStream_t st);
// *out = sum |x_i|^2 accumulated in FP64
vb_status norm2_sq_f32(const cf *x, long long n, double *out, double *partial, int n_part, cudaStream_t st);
// out[0] = *capt, out[1] = *cnt
vb_status subspace_status(const double *capt, const int *cnt, double *out, cudaStream_t st);
// vec_multi_axpy, then *out = |w| (partial: at least 512 doubles)
// cnt (nullable, zeroed device counters: one per group of 8 vectors for the
// inner products, one for the norm): the last block reduces, no extra launch
vb_status vec_multi_axpy_norm(const cd *V, long long ldv, int nv, const cd *c, double sign, cd *w, long long n,
                              double *out, double *partial, cudaStream_t st, unsigned int *cnt = nullptr);
vb_status vec_norm2(const cd *x, long long n, double *out, double *partial, int n_part,
                    cudaStream_t st);
// x *= 1/ (*nrm) (device scalar; a zero norm gives zero); keep (nullable):
// *keep = *nrm; alpha_k (nullable): *alpha_k = Re *c + Re *c2
// shadow (nullable): also write the FP32 copy of the scaled vector
vb_status vec_scale_inv(cd *x, long long n, const double *nrm, cudaStream_t st, double *keep = nullptr,
                        const cd *c = nullptr, const cd *c2 = nullptr, double *alpha_k = nullptr,
                        cf *shadow = nullptr);
// y = s * x with s = *num / *den (device scalars; den may be null -> 1)
vb_status vec_copy_scaled(const cd *x, cd *y, long long n, cudaStream_t st);
// combine: y = (*nrm) * sum_j u[j] vs[j] V[j] (vs nullable: 1)
vb_status vec_combine(const cd *V, long long ldv, int nv, const cd *u, const double *nrm, cd *y,
                      long long n, cudaStream_t st, const double *vs = nullptr);
int reduce_parts(long long n);

// ------------------------------------------------------------ eigen
struct EigWork {
  // layout inside one device buffer (real type of size real_bytes)
  static size_t bytes(int n, int k_want, int real_bytes = 8);
  // synchronises st and returns VB_ETIMEOUT if a bounded wait of the last
  // eig_values on this workspace ran out
  static vb_status check(int n, int k_want, int real_bytes, const void *work, cudaStream_t st);
};
// phase 1: reduce rho (n x n, destroyed) to real tridiagonal form and compute
// the k_want largest eigenvalues (descending) into evals (device)
template <class R>
vb_status eig_values(int n, cplx<R> *rho, int k_want, R *evals, void *work, cudaStream_t st);
// phase 2: eigenvectors for the first k_vec of those eigenvalues, written as
// rows of evecs [k_vec][n] (device). Needs the same rho/work after phase 1.
// rounds: inverse-iteration rounds (0: 3 in FP64, 2 in FP32)
template <class R>
vb_status eig_vectors(int n, const cplx<R> *rho, int k_want, int k_vec, const R *evals,
                      cplx<R> *evecs, void *work, cudaStream_t st, int rounds = 0);

// Krylov tridiagonal exponential: from alpha[0..k], beta[0..k-1] (device),
// u = exp(-i T tau) e_1 (k+1 complex); out[0] = bnext * |u_k|, out[1] =
// bnext (device or mapped host). With c, c2 given, alpha[k] is first set to
// Re c[k] + Re c2[k] (the two Gram-Schmidt passes' <v_k, H v_k>).
vb_status tridiag_expm(const cd *c, const cd *c2, double *alpha, const double *beta, int kdim, double tau,
                       const double *bnext, cd *u, double *out, cudaStream_t st);

}  // namespace vb
