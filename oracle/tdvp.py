"""Two-site TDVP (Sec. 2.1.2) for an MPS under an MPO - oracle side.

Test infrastructure only (see the package docstring).

Index conventions (all complex128):
  MPS site tensor       A[p][a_left, s, a_right]                 (Eq. MPS tensor)
  MPO site tensor       W[p][w_in, s_out, s_in, w_out]             (Eq. MPO)
  left environment      L[i][a', w, a]  block of sites 0..i-1, a' the bra index
  right environment     R[i][b', w, b]  block of sites i..n-1, b' the bra index
  two-site tensor       theta[a, s, t, b]
H_eff,2 (Eq. two-site Hamiltonian) acts as
  y[a',s',t',b'] = sum L[a',w0,a] W_i[w0,s',s,w1] W_{i+1}[w1,t',t,w2] R[b',w2,b] theta[a,s,t,b]
and H_eff,1 (Eq. one-site Hamiltonian 1) is the same with one W.

One time step (readings of the paper's sweep description, Sec. 2.1.2):
  left-to-right half sweep with tau = dt/2 over pairs (0,1) ... (n-2,n-1):
    merge theta = C_i B_{i+1}; theta <- exp(-i H_eff,2 tau/hbar) theta;
    split theta = A_i C_{i+1} (truncated, DBSS); grow L;
    backward C_{i+1} <- exp(+i H_eff,1 tau/hbar) C_{i+1}, except at the last pair
  right-to-left half sweep with tau = dt/2, mirrored; the center ends on site 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import eigh_tridiagonal

from vibmodels import HBAR_EV_FS

ZERO_FLOOR = 1e-14       # relative weight below which a Schmidt direction is dropped
MULTIPLET_RTOL = 1e-10   # relative gap under which two weights count as degenerate


@dataclass
class TdvpOptions:
    m_max: int = 1 << 30          # bond cap M (fixed-M truncation, Sec. 2.1.1)
    eps: float = 0.0              # DBSS threshold on the discarded weight
    zero_floor: float = ZERO_FLOOR  # drop weights <= zero_floor * trace (0: keep all)
    krylov_max: int = 30
    krylov_tol: float = 1e-13


@dataclass
class StepStats:
    max_bond: int = 0
    discarded: float = 0.0
    krylov_max_iters: int = 0
    noconv: int = 0
    krylov_iters: list = field(default_factory=list)


class MPS:
    def __init__(self, tensors, center=0):
        self.A = [np.array(t, dtype=np.complex128) for t in tensors]
        self.center = center

    @property
    def n(self):
        return len(self.A)

    def bond_dims(self):
        return [t.shape[2] for t in self.A[:-1]]

    def copy(self):
        return MPS([t.copy() for t in self.A], self.center)


# ----------------------------------------------------------- initial states
def product_mps(dims, indices) -> MPS:
    """Bond-dimension-1 product state; trivially right-canonical."""
    ts = []
    for d, k in zip(dims, indices):
        t = np.zeros((1, d, 1), dtype=np.complex128)
        t[0, k, 0] = 1.0
        ts.append(t)
    return MPS(ts, 0)


def padded_product_mps(dims, indices, m_pad=None) -> MPS:
    """The product state written with larger bond dimensions
    D_b = min(prod_{p<=b} d_p, prod_{p>b} d_p, m_pad). Every B_p (p >= 1) is
    right-orthonormal: its first row carries the product state and the other
    rows are distinct unit vectors (a deterministic orthonormal completion)."""
    n = len(dims)
    D = []
    for b in range(n - 1):
        left = 1
        for d in dims[: b + 1]:
            left *= int(d)
        right = 1
        for d in dims[b + 1:]:
            right *= int(d)
        v = min(left, right)
        if m_pad is not None:
            v = min(v, m_pad)
        D.append(v)
    Dfull = [1] + D + [1]
    ts = []
    for p in range(n):
        dl, d, dr = Dfull[p], dims[p], Dfull[p + 1]
        t = np.zeros((dl, d, dr), dtype=np.complex128)
        if p == 0:
            t[0, indices[0], 0] = 1.0
        else:
            cols = d * dr
            first = indices[p] * dr + 0
            others = [c for c in range(cols) if c != first]
            mat = np.zeros((dl, cols), dtype=np.complex128)
            mat[0, first] = 1.0
            for r in range(1, dl):
                mat[r, others[r - 1]] = 1.0
            t = mat.reshape(dl, d, dr)
        ts.append(t)
    return MPS(ts, 0)


# -------------------------------------------------------------- contractions
def env_left_update(L, A, W):
    """L_new[y', v, y] = sum conj(A[x,s',y']) L[x,w,z] W[w,s',s,v] A[z,s,y]."""
    T1 = np.einsum("xwz,zsy->xwsy", L, A, optimize=True)
    T2 = np.einsum("wpsv,xwsy->xpvy", W, T1, optimize=True)
    return np.einsum("xpq,xpvy->qvy", np.conj(A), T2, optimize=True)


def env_right_update(R, B, W):
    """R_new[a', w, a] = sum conj(B[a',t',y]) R[y,v,z] W[w,t',t,v] B[a,t,z]."""
    T1 = np.einsum("atz,yvz->atyv", B, R, optimize=True)
    T2 = np.einsum("wqtv,atyv->awqy", W, T1, optimize=True)
    return np.einsum("xqy,awqy->xwa", np.conj(B), T2, optimize=True)


def heff2_apply(L, Wi, Wj, R, theta):
    """y = H_eff,2 theta in the order L, W_i, W_{i+1}, R."""
    T1 = np.einsum("xwa,astb->xwstb", L, theta, optimize=True)
    T2 = np.einsum("wpsv,xwstb->xpvtb", Wi, T1, optimize=True)
    T3 = np.einsum("vqtu,xpvtb->xpqub", Wj, T2, optimize=True)
    return np.einsum("yub,xpqub->xpqy", R, T3, optimize=True)


def heff1_apply(L, W, R, C):
    """y = H_eff,1 C in the order L, W, R."""
    T1 = np.einsum("xwa,atb->xwtb", L, C, optimize=True)
    T2 = np.einsum("wqtv,xwtb->xqvb", W, T1, optimize=True)
    return np.einsum("yvb,xqvb->xqy", R, T2, optimize=True)


def heff0_apply(L, R, X):
    """y = H_eff,0 X for the bond matrix between two sites (zero-site
    Hamiltonian of the one-site TDVP, Sec. 2.1.2):
    y[a', b'] = sum L[a', w, a] R[b', w, b] X[a, b]."""
    T = np.einsum("xwa,ab->xwb", L, X, optimize=True)
    return np.einsum("ywb,xwb->xy", R, T, optimize=True)


# ------------------------------------------------------ Krylov exponential
def krylov_expm(apply, theta, dt_fs, kmax=30, tol=1e-13):
    """exp(-i H dt/hbar) theta from the Krylov space of Eq. Krylov subspace.

    Lanczos with full re-orthogonalisation (two classical Gram-Schmidt passes
    against all previous vectors); the exponential of the small tridiagonal T
    comes from its eigendecomposition (library routine). Stops when the
    a-posteriori estimate beta_{k+1} |[exp(-i T dt/hbar) e_1]_k| < tol, when
    the space is exhausted, or at kmax. Returns (result, iterations,
    converged)."""
    nrm = np.linalg.norm(theta)
    if nrm == 0.0:
        return theta.copy(), 0, True
    shape = theta.shape
    dim = theta.size
    V = [theta.reshape(-1) / nrm]
    alpha, beta = [], []
    u = None
    k = 0
    converged = False
    for k in range(min(kmax, dim)):
        w = apply(V[k].reshape(shape)).reshape(-1)
        Vm = np.array(V)
        c = np.conj(Vm) @ w
        w = w - Vm.T @ c
        c2 = np.conj(Vm) @ w
        w = w - Vm.T @ c2
        alpha.append(float(np.real(c[k] + c2[k])))
        b = float(np.linalg.norm(w))
        lam, S = eigh_tridiagonal(np.array(alpha), np.array(beta)) if k > 0 else \
            (np.array(alpha), np.ones((1, 1)))
        u = S @ (np.exp(-1j * lam * dt_fs / HBAR_EV_FS) * S[0, :])
        err = b * abs(u[k])
        if err < tol or b <= 1e-300 or k + 1 == dim:
            converged = True
            break
        beta.append(b)
        V.append(w / b)
    out = nrm * (np.array(V[: len(u)]).T @ u)
    return out.reshape(shape), k + 1, converged


# ----------------------------------------------------------- truncation
def choose_rank(lam_desc, opts: TdvpOptions, rank_bound: int | None = None) -> int:
    """Number of kept Schmidt directions from the descending eigenvalues of
    the reduced density matrix (DBSS, Sec. 2.1.1): the smallest k whose
    discarded weight is <= eps * trace, capped at m_max; weights at or below
    zero_floor * trace are always dropped (none when zero_floor is 0); a
    degenerate multiplet is never split; k >= 1 and k <= rank_bound (the
    smaller side of the matrix, which bounds the Schmidt rank)."""
    n = len(lam_desc)
    tot = float(np.sum(lam_desc))
    k = n if rank_bound is None else min(n, rank_bound)
    if opts.zero_floor > 0.0:
        k = min(k, int(np.sum(lam_desc > opts.zero_floor * tot)))
    if opts.eps > 0.0:
        tail = 0.0
        kk = n
        # walk from the smallest weight upward while the tail stays within eps
        for j in range(n - 1, -1, -1):
            if tail + lam_desc[j] <= opts.eps * tot:
                tail += lam_desc[j]
                kk = j
            else:
                break
        k = min(k, kk)
    k = min(k, opts.m_max)
    k = max(k, 1)
    while 1 < k < n and (lam_desc[k - 1] - lam_desc[k]) < MULTIPLET_RTOL * lam_desc[k - 1]:
        k -= 1
    return k


def split_left(theta, opts: TdvpOptions):
    """theta[a,s,t,b] = A[a,s,k] C[k,t,b] with A left-orthonormal (Eq. l
    orthonormal). A = leading eigenvectors of rho = M M^+, M = theta as an
    (a s) x (t b) matrix; C = A^+ M renormalised to unit norm."""
    mL, d1, d2, mR = theta.shape
    M = theta.reshape(mL * d1, d2 * mR)
    rho = M @ np.conj(M.T)
    lam, U = np.linalg.eigh(rho)
    lam, U = lam[::-1], U[:, ::-1]
    k = choose_rank(lam, opts, min(mL * d1, d2 * mR))
    tot = float(np.sum(lam))
    disc = float(np.sum(lam[k:])) / tot if tot > 0 else 0.0
    Uk = U[:, :k]
    C = np.conj(Uk.T) @ M
    C = C / np.linalg.norm(C)
    return Uk.reshape(mL, d1, k), C.reshape(k, d2, mR), disc


def split_right(theta, opts: TdvpOptions):
    """theta[a,s,t,b] = C[a,s,k] B[k,t,b] with B right-orthonormal (Eq. r
    orthonormal). B = V_k^+ from the leading eigenvectors V of
    rho = M^+ M; C = M V_k renormalised to unit norm."""
    mL, d1, d2, mR = theta.shape
    M = theta.reshape(mL * d1, d2 * mR)
    rho = np.conj(M.T) @ M
    lam, V = np.linalg.eigh(rho)
    lam, V = lam[::-1], V[:, ::-1]
    k = choose_rank(lam, opts, min(mL * d1, d2 * mR))
    tot = float(np.sum(lam))
    disc = float(np.sum(lam[k:])) / tot if tot > 0 else 0.0
    Vk = V[:, :k]
    C = M @ Vk
    C = C / np.linalg.norm(C)
    B = np.conj(Vk.T)
    return C.reshape(mL, d1, k), B.reshape(k, d2, mR), disc


# ------------------------------------------------------------- the sweep
class Tdvp2:
    """State of a 2TDVP propagation: MPS, MPO and cached environments."""

    def __init__(self, mps: MPS, W, opts: TdvpOptions | None = None):
        assert mps.center == 0
        self.mps = mps
        self.W = [np.asarray(w, dtype=np.complex128) for w in W]
        self.opts = opts or TdvpOptions()
        n = mps.n
        one = np.ones((1, 1, 1), dtype=np.complex128)
        self.L = [None] * (n + 1)
        self.R = [None] * (n + 1)
        self.L[0] = one
        self.R[n] = one
        for p in range(n - 1, 0, -1):
            self.R[p] = env_right_update(self.R[p + 1], self.mps.A[p], self.W[p])
        self.time = 0.0

    def _evolve(self, apply, x, dt, st: StepStats):
        y, it, conv = krylov_expm(apply, x, dt, self.opts.krylov_max, self.opts.krylov_tol)
        st.krylov_iters.append(it)
        st.krylov_max_iters = max(st.krylov_max_iters, it)
        if not conv:
            st.noconv += 1
        return y

    def step(self, dt_fs: float, max_pairs: int | None = None) -> StepStats:
        """One time step = left-to-right half sweep with dt/2 followed by the
        right-to-left half sweep with dt/2. `max_pairs` stops after that many
        two-site updates (a bounded timing sample; the state is then left
        mid-sweep and the step is not complete)."""
        st = StepStats()
        for done, _ in enumerate(self.step_updates(dt_fs, st)):
            if max_pairs is not None and done + 1 >= max_pairs:
                break
        return st

    def step_updates(self, dt_fs: float, st: StepStats):
        """The time step of `step` as a generator that yields after every
        two-site update (2 (n - 1) of them), so that a caller can time the
        sweep in consecutive slices; the step is complete once it is exhausted."""
        n = self.mps.n
        tau = 0.5 * dt_fs
        for i in range(n - 1):  # left to right
            self.update_left_to_right(i, tau, st)
            yield i
        for i in range(n - 2, -1, -1):  # right to left
            self.update_right_to_left(i, tau, st)
            if i == 0:
                self.mps.center = 0
                st.max_bond = max(self.mps.bond_dims())
                self.time += dt_fs
            yield i
        if n < 2:
            st.max_bond = 1
            self.time += dt_fs

    def update_left_to_right(self, i: int, tau: float, st: StepStats):
        """The two-site update at pair (i, i+1) of the left-to-right half
        sweep (center on site i, L[i] and R[i+2] current): merge, forward
        exponential, split with A_i left-orthonormal, grow L, and the backward
        one-site step of the new center unless i + 1 is the last site."""
        A, W, L, R = self.mps.A, self.W, self.L, self.R
        n = self.mps.n
        theta = np.einsum("asx,xtb->astb", A[i], A[i + 1], optimize=True)
        Li, Wi, Wj, Rj = L[i], W[i], W[i + 1], R[i + 2]
        theta = self._evolve(lambda x: heff2_apply(Li, Wi, Wj, Rj, x), theta, tau, st)
        A[i], C, disc = split_left(theta, self.opts)
        st.discarded += disc
        L[i + 1] = env_left_update(L[i], A[i], W[i])
        if i < n - 2:
            L1, W1, R1 = L[i + 1], W[i + 1], R[i + 2]
            C = self._evolve(lambda x: heff1_apply(L1, W1, R1, x), C, -tau, st)
        A[i + 1] = C

    def update_right_to_left(self, i: int, tau: float, st: StepStats):
        """The mirror of update_left_to_right at pair (i, i+1) of the
        right-to-left half sweep (center on site i+1)."""
        A, W, L, R = self.mps.A, self.W, self.L, self.R
        theta = np.einsum("asx,xtb->astb", A[i], A[i + 1], optimize=True)
        Li, Wi, Wj, Rj = L[i], W[i], W[i + 1], R[i + 2]
        theta = self._evolve(lambda x: heff2_apply(Li, Wi, Wj, Rj, x), theta, tau, st)
        C, A[i + 1], disc = split_right(theta, self.opts)
        st.discarded += disc
        R[i + 1] = env_right_update(R[i + 2], A[i + 1], W[i + 1])
        if i > 0:
            L0, W0, R0 = L[i], W[i], R[i + 1]
            C = self._evolve(lambda x: heff1_apply(L0, W0, R0, x), C, -tau, st)
        A[i] = C


class Tdvp1:
    """One-site TDVP (Sec. 2.1.2, the one-site variant) at the fixed bond
    dimensions of the initial state. One time step = left-to-right half sweep
    with tau = dt/2, then right-to-left with tau = dt/2 (as for 2TDVP):
      left to right, site i: C_i <- exp(-i H_eff,1 tau) C_i; unless i is the
      last site: C_i = A_i R (QR), grow L, R <- exp(+i H_eff,0 tau) R,
      C_{i+1} = R B_{i+1};
      right to left, mirrored with C_i = R Q (QR of C_i^+), grow R,
      R <- exp(+i H_eff,0 tau) R, C_{i-1} = A_{i-1} R.
    The last site is evolved twice in a row at the turn (once per half)."""

    def __init__(self, mps: MPS, W, opts: TdvpOptions | None = None):
        assert mps.center == 0
        self.mps = mps
        self.W = [np.asarray(w, dtype=np.complex128) for w in W]
        self.opts = opts or TdvpOptions()
        n = mps.n
        one = np.ones((1, 1, 1), dtype=np.complex128)
        self.L = [None] * (n + 1)
        self.R = [None] * (n + 1)
        self.L[0] = one
        self.R[n] = one
        for p in range(n - 1, 0, -1):
            self.R[p] = env_right_update(self.R[p + 1], self.mps.A[p], self.W[p])
        self.time = 0.0

    def _evolve(self, apply, x, dt, st: StepStats):
        y, it, conv = krylov_expm(apply, x, dt, self.opts.krylov_max, self.opts.krylov_tol)
        st.krylov_iters.append(it)
        st.krylov_max_iters = max(st.krylov_max_iters, it)
        if not conv:
            st.noconv += 1
        return y

    def step(self, dt_fs: float) -> StepStats:
        st = StepStats()
        A, W, L, R = self.mps.A, self.W, self.L, self.R
        n = self.mps.n
        tau = 0.5 * dt_fs
        # left to right
        for i in range(n):
            Li, Wi, Ri = L[i], W[i], R[i + 1]
            C = self._evolve(lambda x: heff1_apply(Li, Wi, Ri, x), A[i], tau, st)
            if i == n - 1:
                A[i] = C
                break
            mL, d, mR = C.shape
            Q, Rm = np.linalg.qr(C.reshape(mL * d, mR))
            A[i] = Q.reshape(mL, d, mR)
            L[i + 1] = env_left_update(L[i], A[i], W[i])
            L1, R1 = L[i + 1], R[i + 1]
            Rm = self._evolve(lambda x: heff0_apply(L1, R1, x), Rm, -tau, st)
            A[i + 1] = np.einsum("ab,bsc->asc", Rm, A[i + 1])
        # right to left
        for i in range(n - 1, -1, -1):
            Li, Wi, Ri = L[i], W[i], R[i + 1]
            C = self._evolve(lambda x: heff1_apply(Li, Wi, Ri, x), A[i], tau, st)
            if i == 0:
                A[0] = C
                break
            mL, d, mR = C.shape
            Qh, Rh = np.linalg.qr(C.reshape(mL, d * mR).conj().T)  # C = Rh^+ Qh^+
            A[i] = Qh.conj().T.reshape(mL, d, mR)
            R[i] = env_right_update(R[i + 1], A[i], W[i])
            L0, R0 = L[i], R[i]
            Rm = self._evolve(lambda x: heff0_apply(L0, R0, x), Rh.conj().T, -tau, st)
            A[i - 1] = np.einsum("asb,bc->asc", A[i - 1], Rm)
        self.mps.center = 0
        st.max_bond = max(self.mps.bond_dims()) if n > 1 else 1
        self.time += dt_fs
        return st


# ------------------------------------------------------------ observables
def expect_local(mps: MPS, pos: int, op: np.ndarray) -> complex:
    """<psi|op_pos|psi> / <psi|psi> by a transfer-matrix contraction."""
    num = np.ones((1, 1), dtype=np.complex128)
    den = np.ones((1, 1), dtype=np.complex128)
    for p, A in enumerate(mps.A):
        Aop = np.einsum("st,atb->asb", op, A) if p == pos else A
        num = np.einsum("xy,xsa,ysb->ab", num, np.conj(A), Aop)
        den = np.einsum("xy,xsa,ysb->ab", den, np.conj(A), A)
    return num[0, 0] / den[0, 0]


def populations(mps: MPS, el_pos: int = 0) -> np.ndarray:
    """Electronic populations P_k = <psi| |k><k| |psi> (Sec. 3.1)."""
    d = mps.A[el_pos].shape[1]
    out = np.zeros(d)
    for k in range(d):
        P = np.zeros((d, d))
        P[k, k] = 1.0
        out[k] = float(np.real(expect_local(mps, el_pos, P)))
    return out


def overlap(phi: MPS, psi: MPS) -> complex:
    """<phi|psi> by the transfer-matrix contraction of Eq. overlap 2."""
    E = np.ones((1, 1), dtype=np.complex128)
    for Ap, Aq in zip(phi.A, psi.A):
        E = np.einsum("xy,xsa,ysb->ab", E, np.conj(Ap), Aq)
    return E[0, 0]


def energy(mps: MPS, W) -> float:
    """<psi|H|psi> / <psi|psi> from the full MPO sandwich."""
    E = np.ones((1, 1, 1), dtype=np.complex128)
    for A, Wp in zip(mps.A, W):
        E = env_left_update(E, A, np.asarray(Wp, dtype=np.complex128))
    return float(np.real(E[0, 0, 0] / overlap(mps, mps)))


def to_vector(mps: MPS) -> np.ndarray:
    """Contract the MPS into the full state vector (tiny systems)."""
    v = mps.A[0][0]  # [s, b]
    for A in mps.A[1:]:
        v = np.einsum("Sx,xtb->Stb", v, A).reshape(-1, A.shape[2])
    return v[:, 0]
