/*
 * vibtdvp — C ABI of the GB300 two-site TDVP (2TDVP) library for vibronic
 * Hamiltonians (Xie et al., arXiv:1908.10588).
 *
 * The method: an MPS (Sec. 2.1.1, Eq. MPS tensor) is propagated in time by
 * the two-site time-dependent variational principle (Sec. 2.1.2): at every
 * bond the two-site tensor is evolved with the two-site effective Hamiltonian
 * (Eq. two-site Hamiltonian) through a Krylov exponential (Eq. Krylov
 * subspace), split and truncated (DBSS / fixed M, Sec. 2.1.1), and the new
 * center site is evolved backward with the one-site effective Hamiltonian
 * (Eq. one-site Hamiltonian 1). The Hamiltonian is the vibronic model of
 * Sec. 2.2 (Eqs. Hel_2, Hvib_2, Helvib_2), given to mpo_build as its sum of
 * terms and turned into an MPO (Eq. MPO).
 *
 * Conventions for every entry point:
 *  - Units: energies in eV, times in fs, hbar = 0.6582119569 eV fs.
 *  - Complex numbers are interleaved (re, im) pairs of double (or float
 *    where stated); every tensor is dense and row-major in the index order
 *    written next to it.
 *  - Host pointers are borrowed for the duration of the call only. Device
 *    pointers are owned by the caller unless a handle owns them.
 *  - No C++ exception crosses this boundary. Every call returns a vb_status;
 *    on an error outputs are left unspecified and vb_last_error() returns a
 *    thread-local message. Handles are not thread-safe.
 *  - All device work of a handle runs on the stream given at creation
 *    (NULL = the legacy default stream); calls that return host data
 *    synchronise that stream.
 */
#ifndef VIBTDVP_H
#define VIBTDVP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VB_OK = 0,
  VB_EINVAL = -1,    /* bad argument, size or layout */
  VB_ENOMEM = -2,    /* device allocation failed */
  VB_ECUDA = -3,     /* a CUDA call failed; message in vb_last_error() */
  VB_ENOCONV = -4,   /* Krylov exponential not converged and policy = fail */
  VB_ETIMEOUT = -5,  /* a device-side wait ran out of its iteration budget */
  VB_ESTATE = -6     /* handle in the wrong state (e.g. center not at site 0) */
} vb_status;

enum { VB_FP64 = 0, VB_MIXED = 1 };

/* Vibronic model, Sec. 2.2. Host memory, borrowed by mpo_build.
 * H = sum_ij h_ij |i><j|  with h_ii = e0[i], h_ij = v0[i*n_el+j] (i != j)  (Eq. Hel_2)
 *   + sum_I omega[I] (b_I^+ b_I + include_zpe/2)                          (Eq. Hvib_2)
 *   + sum_{I,i,j} g1[(I*n_el+i)*n_el+j] q_I |i><j|
 *   + sum_k g2_val[k] q_I q_J |i><j|, (I,J,i,j) = g2_idx[4k..4k+3], I <= J,
 *     I == J meaning q_I^2                                                (Eq. Helvib_2)
 * with q = (b + b^+)/sqrt(2) on the basis |0..levels[I]-1>.
 * site_order[n_modes+1] gives the chain: -1 = electronic site, k = mode k;
 * NULL = electronic site first, then the modes in index order. */
typedef struct {
  int n_el;
  const double *e0;
  const double *v0;
  int n_modes;
  const double *omega;
  const int *levels;
  const double *g1;
  int n_g2;
  const int *g2_idx;
  const double *g2_val;
  const int *site_order;
  int include_zpe;
} vb_model;

/* Optional device allocator (e.g. a framework's caching allocator). */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *ctx);
  void (*free)(void *ptr, void *stream, void *ctx);
  void *ctx;
} vb_allocator;

typedef struct {
  int m_cap;          /* largest bond dimension the handle reserves memory for */
  int dtype;          /* VB_FP64, or VB_MIXED: H_eff products on the tensor cores in split TF32
                         with FP32 accumulation, FP32 environments and merge, FP32 directions of
                         the split with FP64 weights, Lanczos Gram-Schmidt on FP32 copies of the
                         FP64 vectors; the Lanczos vectors, coefficients, small exponential and
                         the stored tensors stay FP64 */
  int pad_full;       /* mps_create: pad the product state to full bonds (<= m_cap) */
  int krylov_cap;     /* largest Krylov dimension reserved (default 40) */
  void *cuda_stream;  /* cudaStream_t */
  const vb_allocator *alloc; /* NULL = cudaMalloc / cudaFree */
} vb_mps_opts;

/* Truncation (Sec. 2.1.1) and Krylov (Eq. Krylov subspace) parameters. */
typedef struct {
  int m_max;          /* fixed-M cap, <= m_cap */
  double eps;         /* DBSS: discarded weight <= eps * trace (0 = off) */
  double zero_floor;  /* always drop weights <= zero_floor * trace (0 = keep) */
  int krylov_max;     /* <= krylov_cap */
  double krylov_tol;  /* a-posteriori error bound of each local exponential */
  int on_noconv;      /* 0 = continue with the last iterate, 1 = return VB_ENOCONV */
} vb_tdvp_opts;

typedef struct {
  int max_bond;
  double discarded_weight;  /* sum over the step's splits of the relative discarded weight */
  int krylov_iters_max;
  int krylov_iters_total;
  int noconv;               /* number of local exponentials that hit krylov_max */
} vb_sweep_stats;

typedef struct vb_mpo vb_mpo;
typedef struct vb_mps vb_mps;

const char *vb_last_error(void);
int vb_version(void);

/* ---- MPO (Eq. MPO): finite-state-automaton construction from the terms.
 * Host only until first use by an MPS (device upload is lazy), so these
 * calls work without a GPU. */
vb_status mpo_build(const vb_model *model, vb_mpo **out);
vb_status mpo_destroy(vb_mpo *mpo);
int mpo_n_sites(const vb_mpo *mpo);
/* w_in, d, w_out of site p */
vb_status mpo_site_dims(const vb_mpo *mpo, int site, int *w_in, int *d, int *w_out);
/* dense real W[w_in][s_out][s_in][w_out] copied to host_out */
vb_status mpo_site_tensor(const vb_mpo *mpo, int site, double *host_out);

/* ---- MPS (Eq. MPS tensor), mixed-canonical with the center on site 0. */
/* Product state |init_index[p]> on every site p (Sec. 3.1 initial state). */
vb_status mps_create(const vb_mpo *mpo, const int *init_index, const vb_mps_opts *opts,
                     vb_mps **out);
/* Arbitrary right-canonical MPS: bond_dims[n-1]; host_tensors[p] is complex
 * double [m_{p-1}][d_p][m_p] (m_{-1} = m_{n-1} = 1); sites 1..n-1 must be
 * right-orthonormal (Eq. r orthonormal), site 0 carries the norm. */
vb_status mps_create_from_tensors(const vb_mpo *mpo, const int *bond_dims,
                                  const double *const *host_tensors,
                                  const vb_mps_opts *opts, vb_mps **out);
vb_status mps_destroy(vb_mps *mps);
int mps_n_sites(const vb_mps *mps);
vb_status mps_bond_dims(const vb_mps *mps, int *host_out /* [n-1] */);
/* complex double [m_{p-1}][d_p][m_p] of site p copied to host_out */
vb_status mps_get_site(const vb_mps *mps, int site, double *host_out);
/* The same tensor copied device to device into dev_out (caller-owned device
 * memory of at least m_{p-1} d_p m_p complex doubles), the bridge to tensors
 * of a host framework (e.g. torch) without a host round trip. The copy runs
 * on the handle's stream; when `stream` (cudaStream_t) is another stream the
 * handle's stream is synchronised before returning, so dev_out is ready for
 * work queued on `stream` afterwards. */
vb_status mps_get_tensor(const vb_mps *mps, int site, double *dev_out, void *stream);

/* ---- one 2TDVP time step (Sec. 2.1.2): left-to-right half sweep with
 * dt/2 then right-to-left half sweep with dt/2; the center returns to site 0.
 * Mixed form: a tensor-core kernel whose bounded wait ran out raises a flag
 * on the device; the sweep (and tdvp1_sweep) reads it at its end, returns
 * VB_ETIMEOUT (the state is then invalid) and clears the flag. */
vb_status tdvp2_sweep(vb_mps *mps, const vb_mpo *mpo, double dt_fs, const vb_tdvp_opts *opts,
                      vb_sweep_stats *stats /* nullable */);

/* ---- one one-site TDVP time step (Sec. 2.1.2, the one-site variant) at
 * the state's current bond dimensions (no truncation, no growth): left to
 * right with dt/2, each site evolved by H_eff,1, split by a QR into an
 * orthonormal site tensor and a bond matrix that is evolved backwards by the
 * zero-site H_eff,0 and absorbed into the next site; then right to left with
 * dt/2, mirrored (LQ). The QR/LQ are Cholesky QR done twice in FP64 (bond
 * dimensions up to 112; columns that depend on earlier ones get orthonormal
 * completions). Norm and energy are conserved up to the Krylov tolerance.
 * m_max, eps and zero_floor of opts are not used. Works in both forms (H_eff,1
 * as in tdvp2_sweep; H_eff,0, QR and LQ in FP64). */
vb_status tdvp1_sweep(vb_mps *mps, const vb_mpo *mpo, double dt_fs, const vb_tdvp_opts *opts,
                      vb_sweep_stats *stats /* nullable */);

/* ---- differentiation: dP_k(t)/dg for linear vibronic couplings g^I_ij
 * (Eq. Helvib_2; the parameters of the model, Sec. 2.2), t = n_steps * dt.
 * psi is propagated by n_steps tdvp2_sweep calls (opts, dt_fs) and left at t;
 * pop_out [n_el] (host) receives the populations at t, grad_out [n_param]
 * (host) dP_{el_state}/dg for every parameter r = (mode param_mode[r],
 * states param_i[r], param_j[r]); for i != j the parameter moves g_ij and
 * g_ji together (H stays Hermitian), dH/dg = q_I (|i><j| + |j><i|).
 * Method (Duhamel): dP_k/dg = (2/hbar) Im int_0^t <lambda(s)| dH/dg |psi(s)> ds,
 * lambda(s) = exp(-iH(s - t)) |k><k| psi(t): the costate is propagated back
 * with tdvp2_sweep(-dt) on a second state (the adjoint of a unitary local
 * step is the step backwards; H_eff is Hermitian), the integrand at every step
 * is a transfer-matrix contraction with q_I inserted, and the time integral
 * uses composite closed Newton-Cotes rules on the step grid (Boole's rule on
 * panels of four steps, Simpson / 3/8 / trapezoid for the remainder). With
 * full bonds the propagation is exact and the gradient is exact up to the
 * quadrature; with truncated bonds it is the gradient of the exact dynamics
 * evaluated on the 2TDVP states. Step checkpointing: the state is stored
 * every c = checkpoint_every steps and each segment but the last is recomputed
 * once in the backward pass (two extra handles and about n_steps/c + c + 1
 * state copies from psi's allocator; c = n_steps keeps every state and
 * recomputes nothing). Needs the electronic site at position 0 and the center
 * on site 0. Cost: 3 - c/n_steps sweeps per step. */
vb_status tdvp2_population_gradient(vb_mps *psi, const vb_mpo *mpo, double dt_fs, int n_steps,
                                    const vb_tdvp_opts *opts, int el_state, int n_param, const int *param_mode,
                                    const int *param_i, const int *param_j, int checkpoint_every,
                                    double *pop_out, double *grad_out);

/* ---- global Krylov step (Sec. 2.1.2, Eqs. Krylov subspace and global
 * Krylov): psi <- exp(-iH dt/hbar) psi in the Krylov space spanned by the
 * MPSs k_0 = psi/|psi|, k_{j+1} = compress(H k_j)/|.|, H applied as the MPO
 * directly (Sec. 2.1.1, Eqs. direct app 1/2: bond dimensions multiply) and
 * compressed with the 2TDVP split's truncation rule (opts: m_max, eps,
 * zero_floor; Sec. 2.1.1). The basis is orthonormalised through its Gram
 * matrix S_ij = <k_i|k_j> in Krylov order (Cholesky), H is projected as
 * <k_i|H k_j> with the uncompressed H k_j, the propagator is exact in the
 * span, and the state becomes sum_j c_j k_j, compressed and scaled back to
 * |psi|. Stops when the newest orthonormal direction's coefficient is below
 * tol, when a new vector lies in the span (smallest eigenvalue of S <= 1e-13
 * of its largest), or at r_max vectors (<= 40). The result must fit the
 * handle's bond capacities (VB_EINVAL otherwise; psi unchanged then). Used
 * for pre-steps that grow the bonds of a product state before tdvp1_sweep
 * (Sec. 2.1.2, one-site TDVP paragraph). All contractions are complex FP64
 * GEMMs on the device; the Krylov vectors (bonds up to w x m_max) are held in
 * temporaries from psi's allocator for the duration of the call. */
typedef struct {
  int r;                /* Krylov vectors beyond k_0 that were kept */
  int converged;        /* 1: stopped on tol or an invariant space */
  double disc_basis;    /* summed discarded weight of the basis compressions */
  double disc_final;    /* discarded weight of the final compression */
  int max_bond_basis;   /* largest bond of a compressed basis vector */
} vb_krylov_info;
vb_status global_krylov_step(vb_mps *psi, const vb_mpo *mpo, double dt_fs, const vb_tdvp_opts *opts, int r_max,
                             double tol, vb_krylov_info *info /* nullable */);

/* Electronic populations P_k = <psi| |k><k| |psi> / <psi|psi> (Sec. 3.1).
 * Needs the center on site 0 (where every sweep leaves it). The electronic
 * site may sit anywhere on the chain: at position e > 0 the transfer matrix
 * of sites 0 .. e-1 is contracted first (complex FP64, temporaries of
 * m_e^2 + m_e d m_{e+1} elements and the transfer blocks from the state's
 * allocator); the sites right of e are right-orthonormal and drop out. */
vb_status measure_populations(const vb_mps *mps, double *pop_host /* [n_el] */);

/* Overlap <a|b> of two states on the same chain (same site dimensions), in
 * any gauge: the transfer matrices are contracted site by site in complex
 * FP64 on a's stream (b's stream is synchronised first). out_host[0], [1]
 * receive the real and imaginary parts. With a = the initial state and b
 * = the propagated one this is the autocorrelation function
 * C(t) = <psi(0)|psi(t)> whose Fourier transform gives the spectra of
 * Sec. 3.1 (Eq. autocorrelation). Temporaries (two m x m blocks and one
 * m x d x m block) come from a's allocator. */
vb_status mps_overlap(const vb_mps *a, const vb_mps *b, double *out_host /* [2] */);

/* Spectrum from the autocorrelation function (Sec. 3.1: the pyrazine
 * spectra are the Fourier transform of C(t) damped by exp(-|t|/tau)):
 *   I(E) = 1/(pi hbar) Re sum_k w_k C(k dt) exp(+i E k dt/hbar) exp(-k dt/tau)
 * with trapezoidal weights w_k = dt (dt/2 for k = 0 and k = n_t - 1): the
 * half-axis integral, whose real part is half the transform over the whole
 * time axis since C(-t) = conj C(t); a stationary state exp(-i E0 t/hbar)
 * gives a unit-area Lorentzian of half-width hbar/tau at E0 (long records).
 * c_t: device, n_t complex doubles C(0), C(dt), ... (e.g. from mps_overlap
 * after every step); energies: device [n_e] eV; out: device [n_e]. dt_fs,
 * tau_fs > 0. Complex FP64, one kernel on `stream` (cudaStream_t); no host
 * synchronisation, no allocation. */
vb_status vb_spectrum(const double *c_t, int n_t, double dt_fs, double tau_fs, const double *energies,
                      int n_e, double *out, void *stream);

/* Energy <psi|H|psi> / <psi|psi> in eV, H the MPO the state was created for
 * (Eq. vibronic Hamiltonian): left environments contracted over the whole
 * chain in FP64. Two-site TDVP conserves it up to truncation (Sec. 2.1.2).
 * Temporaries from the state's allocator. */
vb_status mps_energy(const vb_mps *mps, double *out_host /* [1] */);

/* One tdvp2_sweep for each of `count` independent instances (Sec. 2.1.2 per
 * instance; a batch of models or parameters): one host thread per instance,
 * so instances created on different CUDA streams run concurrently on the
 * GPU; with the profiler on they run one after another. stats (nullable)
 * receives one entry per instance. On failure the error of the first failing
 * instance (in index order) is returned and its message is available from
 * vb_last_error(); the other instances have completed their sweep. An
 * instance may not appear twice. Instances of uneven size share opts except
 * for the bond cap, which is min(opts->m_max, the instance's m_cap). */
vb_status tdvp2_sweep_batched(vb_mps *const *mps, const vb_mpo *const *mpo, int count, double dt_fs,
                              const vb_tdvp_opts *opts, vb_sweep_stats *stats /* [count], nullable */);

/* ---- ordering of the chain sites (Sec. 3.1, ordering of local sites;
 * Sec. 4: strongly coupled sites next to each other, the small-basis
 * entangled sites in the middle, bath modes at one end). Host only: these
 * calls need no GPU and ignore model->site_order unless stated.
 *
 * Cost model of an order (n = n_modes + 1 sites, the MPO of that order as
 * mpo_build would build it, MPS bonds at their saturated size
 * m_b = min(m_max, product of the site dimensions on either side of bond b)):
 *   heff_flops    F = sum over pairs i of the floating-point operations of
 *                 one H_eff,2 application (Eq. two-site Hamiltonian; counted as
 *                 vb_profile counts them);
 *   tensor_elems  T = sum over pairs of m_{i-1} d_i d_{i+1} m_{i+1} (the
 *                 Krylov vectors and the split scale with it);
 *   max_tensor    the largest two-site tensor;
 *   coupling_dist D = sum over site pairs (a, b) of K_ab |pos_a - pos_b|,
 *                 K_ab = sum of |c| / omega-bar over the terms c * (...) of
 *                 Eqs. Helvib_2 acting on both a and b, omega-bar the geometric
 *                 mean frequency of the term's modes;
 *   objective     J = (w_F F/F0 + w_T T/T0 + w_D D/D0) / (w_F + w_T + w_D),
 *                 F0, T0, D0 those of the default order (electronic site
 *                 first, modes by index), which therefore has J = 1;
 *   max_w         the largest MPO bond dimension. */
typedef struct {
  int m_max;                /* MPS bond cap of the saturated-bond estimate */
  double w_flops;           /* weights of F, T and D in J (>= 0, not all 0) */
  double w_size;
  double w_coupling;
  int iters;                /* search: 0 = every order for n <= 8 sites, else
                               max(2000, 20000 * min(n, 32) / n) annealing
                               moves; > 0 = that many moves; < 0 = every
                               order (n <= 10) */
  unsigned long long seed;  /* annealing random stream */
  int n_strong;             /* modes the rule of thumb places around the
                               electronic site (0 = 4) */
} vb_order_opts;

typedef struct {
  double heff_flops;
  double tensor_elems;
  double max_tensor;
  double coupling_dist;
  double objective;
  int max_w;
} vb_order_cost;

/* Cost of `order` ([n] chain positions -> -1 electronic site / k mode k; NULL
 * = model->site_order, or the default order if that is NULL too). opts NULL =
 * m_max 64, all weights 1. mpo_bonds [n-1] (nullable) receives the MPO bond
 * dimensions; site_blocks [2n] (nullable) the number of nonzero operator
 * blocks (non-identity, identity) of every site's MPO tensor. */
vb_status vb_site_order_cost(const vb_model *model, const int *order, const vb_order_opts *opts,
                             vb_order_cost *out, int *mpo_bonds, int *site_blocks);
/* The order minimising J over all orders (n <= 8 by default) or the best
 * one met by simulated annealing (swaps, segment reversals, single-site
 * moves), started from the better of the default order and
 * vb_site_order_rule's. Deterministic for a given seed. order_out: [n]. */
vb_status vb_site_order_search(const vb_model *model, const vb_order_opts *opts, int *order_out,
                               vb_order_cost *cost_out /* nullable */);
/* The paper's rule of thumb (Sec. 3.1): the n_strong modes with the largest
 * total coupling strength sum_b K_ab, in decreasing strength, alternately
 * to the right and to the left of the electronic site; the remaining (bath)
 * modes after them by increasing frequency. order_out: [n]. */
vb_status vb_site_order_rule(const vb_model *model, int n_strong, int *order_out);

/* ---- single operations on caller-owned device buffers (complex double).
 * These run the same kernels as tdvp2_sweep; `stream` is a cudaStream_t. */

/* y[a',s',t',b'] = sum L[a',w0,a] W_i[w0,s',s,w1] W_{i+1}[w1,t',t,w2] R[b',w2,b] theta[a,s,t,b]
 * (Eq. two-site Hamiltonian). L: [mL][w_in(i)][mL], R: [mR][w_out(i+1)][mR],
 * theta, y: [mL][d_i][d_{i+1}][mR]. work: >= vb_heff_work_elems(...) complex. */
vb_status vb_heff2_apply(const vb_mpo *mpo, int site_i, int mL, int mR, const double *L,
                         const double *R, const double *theta, double *y, double *work,
                         int dtype, void *stream);
/* y[a',t',b'] = sum L[a',w0,a] W[w0,t',t,w1] R[b',w1,b] C[a,t,b] (Eq. one-site Hamiltonian 1) */
vb_status vb_heff1_apply(const vb_mpo *mpo, int site, int mL, int mR, const double *L,
                         const double *R, const double *C, double *y, double *work,
                         int dtype, void *stream);
/* complex elements of work needed by vb_heff2_apply (two_site=1) / vb_heff1_apply */
size_t vb_heff_work_elems(const vb_mpo *mpo, int site, int mL, int mR, int two_site);
/* L_new[y',v,y] = sum conj(A[x,s',y']) L[x,w,z] W[w,s',s,v] A[z,s,y] (left block of
 * Eq. one-site Hamiltonian 1). A: [mL][d][mR], L: [mL][w_in][mL], L_new: [mR][w_out][mR]. */
vb_status vb_env_left_update(const vb_mpo *mpo, int site, int mL, int mR, const double *L,
                             const double *A, double *L_new, double *work, void *stream);
/* R_new[a',w,a] = sum conj(B[a',t',y]) R[y,v,z] W[w,t',t,v] B[a,t,z].
 * B: [mL][d][mR], R: [mR][w_out][mR], R_new: [mL][w_in][mL]. */
vb_status vb_env_right_update(const vb_mpo *mpo, int site, int mL, int mR, const double *R,
                              const double *B, double *R_new, double *work, void *stream);
size_t vb_env_work_elems(const vb_mpo *mpo, int site, int mL, int mR);

/* Leading eigenpairs of a Hermitian n x n matrix rho (complex double,
 * row-major; destroyed). Householder reduction to tridiagonal form,
 * bisection for the k_want largest eigenvalues, inverse iteration and back
 * transformation. evals: [k_want] descending (device); evecs: [k_vec][n]
 * (device, row j = eigenvector j); k_vec <= k_want. work: >= vb_eig_work_bytes(n, k_want).
 * Synchronises `stream` before returning: the cooperative reduction used for
 * 64 < n <= 256 has a bounded grid barrier whose error word is read back, and
 * a barrier that ran out returns VB_ETIMEOUT (evals / evecs then invalid). */
vb_status vb_herm_eig_top(int n, double *rho, int k_want, int k_vec, double *evals,
                          double *evecs, void *work, void *stream);
size_t vb_eig_work_bytes(int n, int k_want);

/* vb_herm_eig_top without a workspace argument and without any device
 * allocation (the paper has no counterpart: this is for callers that cannot
 * allocate, e.g. code whose device memory is owned by a host framework's
 * pool, or a latency-critical loop that must avoid cudaMalloc's implicit
 * synchronisation). The workspace is a fixed 3 MiB array in the library's
 * device image, held on every GPU that loads the library until the process
 * exits. Limits: n <= 256, k_want <= 128; larger sizes return VB_EINVAL.
 * The caller still owns rho (destroyed), evals and evecs. The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * The address lookup itself is safe from several host threads at once.
 * All calls share the one array: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * The array keeps the previous call's contents; the solver writes every
 * entry it reads, so nothing needs clearing. Like vb_herm_eig_top the call
 * synchronises `stream` and returns VB_ETIMEOUT when a grid barrier of the
 * reduction ran out. */
vb_status vb_herm_eig_top_noalloc(int n, double *rho, int k_want, int k_vec, double *evals,
                                  double *evecs, void *stream);

/* Test hook of the failure path (the paper has no counterpart): sets the
 * device flag of a mixed-form handle that a tensor-core kernel raises when a
 * bounded wait runs out, exactly as that kernel would, without any fault. The
 * next tdvp2_sweep / tdvp1_sweep must then return VB_ETIMEOUT and clear it.
 * VB_EINVAL for an FP64-form handle. */
vb_status vb_test_raise_wait_flag(vb_mps *mps);

/* ---- autotuner of the tensor-core tiles (the paper has no counterpart).
 * The L leg of the mixed H_eff products (a resident-B tcgen05 GEMM) groups
 * up to G M tiles per resident B block; on the first call for a GEMM shape
 * (device, M, N, K) the candidates G in {2, 4, 8, 12, 24} (<= the M tiles)
 * are each timed once with CUDA events (every candidate writes the same
 * result, so the output is unaffected) and the fastest is kept for that
 * shape. enable: 1 on (default), 0 off (G = 8 for new shapes), -1 unchanged;
 * reset != 0 clears the table. n_entries (nullable) receives the table size,
 * text (nullable, text_len bytes) one line per shape "M= N= K= group= ms=". */
vb_status vb_autotune(int enable, int reset, int *n_entries, char *text, int text_len);

/* ---- measurement (not part of the method; the paper has no counterpart).
 * Number of CUDA kernels this library has launched since it was loaded. */
unsigned long long vb_kernel_launches(void);

/* Per-phase device time of tdvp2_sweep measured with CUDA events recorded on
 * the handle's stream around every phase (0 = H_eff,2 products, 1 = H_eff,1
 * products, 2 = Krylov vector work and the small exponential, 3 = split:
 * reduced density matrix, eigensolver and the new tensors, 4 = environment
 * updates, 5 = merge of two sites; sub-phases of 3: 6 = reduced density
 * matrix, 7 = tridiagonal reduction and eigenvalues, 8 = eigenvectors,
 * 9 = new tensors and normalisation; in the mixed form 10 and 11 are the
 * products and the orthonormalisations of the subspace iteration inside 7,
 * 15 its Rayleigh-Ritz step, split into 16 (FP32 Ritz vectors) and 17 (FP64
 * basis, projection and weights), and 18 / 19 the Cholesky kernels and the
 * Gram and transform products of the orthonormalisations; 12, 13, 14 are the
 * inverse iteration, Gram-Schmidt and back-transformation parts of every
 * eigenvector stage; inside the mixed-form H_eff products 20 = the tcgen05
 * legs (L and R contractions, incl. their split-K reductions), 21 = the
 * sparse MPO legs, 22 = the operand preparation; 23 = the one-CTA Jacobi
 * eigensolver of the Rayleigh-Ritz step, inside 16). flops[p] / bytes[p] are
 * the algorithmic work of every call of phase p (2, mixed form: bytes of
 * the Gram-Schmidt kernels; 20: the useful complex flops of the two dense
 * legs; 21: one read of each leg's input and one write of its output, FP32;
 * 23: flops[23] counts Jacobi sweeps instead; 0 where not counted). heff_flops[c] counts the algorithmic
 * floating-point operations of the H_eff products of class c (a complex
 * multiply-add is 8, real-times-complex 4, an identity-block add 2);
 * krylov_flops counts the FP64 operations of the Krylov vector work (phase
 * 2: inner products, updates, norms, scaling, the final combination) the same
 * way. Each event pair costs a few microseconds of host time on the
 * launching thread, about 10^4 pairs per time step of a 25-site chain, so
 * the profiler can sample: vb_profile_enable(k) records events for the calls
 * of each phase numbered 0, k, 2k, ... (every run of k consecutive calls
 * gives one) and ms[p] = sampled time x calls[p] / sampled calls; calls and
 * flops count every call. k = 1 times every call, 0 switches the profiler
 * off. Host-side state, not thread-safe. */
typedef struct {
  double ms[24];
  long long calls[24];
  double heff_flops[2];
  double krylov_flops;
  double flops[24];
  double bytes[24];
} vb_profile;
vb_status vb_profile_enable(int every);
vb_status vb_profile_read(vb_profile *out, int reset);

#ifdef __cplusplus
}
#endif
#endif
