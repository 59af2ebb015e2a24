"""Global Krylov time step of an MPS (Sec. 2.1.2, Eqs. Krylov subspace and
global Krylov), with the MPO application (Sec. 2.1.1, Eqs. direct app 1/2)
and the MPS compression and sums it needs - oracle side.

Test infrastructure only (see the package docstring).

The step follows the paper's description: the order-r Krylov space of H and
|psi> is spanned by |psi>, H|psi>, ..., H^r|psi>; every vector is an MPS, made
by applying the MPO directly to the previous one and compressing the result
(truncation rule of the 2TDVP split, Sec. 2.1.1); the space is
orthonormalised, the propagator is exact inside it, and the new state is the
projection back: |psi(t + dt)> = P_r^+ U' P_r |psi(t)>. Orthonormalisation
goes through the Gram matrix S_ij = <k_i|k_j> of the (normalised, compressed)
basis MPSs (Gram-Schmidt in Krylov order written as the Cholesky factor of
S), so no MPS differences are formed; H is projected as H_ij = <k_i|H|k_j>
through the MPO. The result, a linear combination of the
basis MPSs, is summed (block tensors) and compressed once.

Pre-steps (Sec. 2.1.2, one-site TDVP paragraph): a few global Krylov steps
grow the bonds of a product state before one-site TDVP, whose bonds are
fixed.
"""
from __future__ import annotations

import numpy as np

from vibmodels import HBAR_EV_FS

from .tdvp import MPS, TdvpOptions, Tdvp1, choose_rank, overlap


# ------------------------------------------------------------ MPO x MPS
def apply_mpo(W, mps: MPS) -> MPS:
    """Direct application (Eqs. direct app 1/2): the new site tensor is
    A'[(w a), s, (v b)] = sum_s' W[w, s, s', v] A[a, s', b], bond dimensions
    multiply (w-major combined index)."""
    out = []
    for Wp, A in zip(W, mps.A):
        wl, d, _, wr = Wp.shape
        ml, _, mr = A.shape
        T = np.einsum("wstv,atb->wasvb", np.asarray(Wp, dtype=np.complex128), A)
        out.append(T.reshape(wl * ml, d, wr * mr))
    return MPS(out, 0)


# ------------------------------------------------------------ compression
def compress(mps: MPS, opts: TdvpOptions):
    """MPS -> right-canonical MPS (norm on site 0, center 0) of the same
    vector up to truncation. Left-to-right QR sweep (exact), then
    right-to-left: at each bond the Schmidt weights are the eigenvalues of
    rho = M^+ M of the site matrix M (m_left x d m_right; the left part is
    left-orthonormal and the right part right-orthonormal, so these are the
    squared singular values of the whole vector at that bond); the kept
    directions are chosen by the 2TDVP split's rule (choose_rank: m_max,
    DBSS eps, zero floor, multiplets). Returns (mps, summed relative
    discarded weight). The norm is not restored."""
    A = [t.copy() for t in mps.A]
    n = len(A)
    for p in range(n - 1):
        ml, d, mr = A[p].shape
        Q, R = np.linalg.qr(A[p].reshape(ml * d, mr))
        A[p] = Q.reshape(ml, d, Q.shape[1])
        A[p + 1] = np.einsum("ab,bsc->asc", R, A[p + 1])
    disc = 0.0
    for p in range(n - 1, 0, -1):
        ml, d, mr = A[p].shape
        M = A[p].reshape(ml, d * mr)
        rho = np.conj(M.T) @ M
        lam, V = np.linalg.eigh(rho)
        lam, V = lam[::-1], V[:, ::-1]
        lam = np.clip(lam, 0.0, None)
        k = choose_rank(lam, opts, min(ml, d * mr))
        tot = float(np.sum(lam))
        if tot > 0:
            disc += float(np.sum(lam[k:])) / tot
        Vk = V[:, :k]
        A[p] = np.conj(Vk.T).reshape(k, d, mr)
        A[p - 1] = np.einsum("asb,bk->ask", A[p - 1], M @ Vk)
    return MPS(A, 0), disc


def mps_sum(coefs, states) -> MPS:
    """sum_j c_j |states_j> as one MPS: block-diagonal middle tensors, the
    first site's blocks side by side (scaled by c_j), the last site's stacked
    (bond dimensions add)."""
    n = states[0].n
    out = []
    for p in range(n):
        blocks = [s.A[p] for s in states]
        d = blocks[0].shape[1]
        if n == 1:
            out.append(sum(c * b for c, b in zip(coefs, blocks)))
            continue
        if p == 0:
            out.append(np.concatenate([c * b for c, b in zip(coefs, blocks)], axis=2))
        elif p == n - 1:
            out.append(np.concatenate(blocks, axis=0))
        else:
            ml = sum(b.shape[0] for b in blocks)
            mr = sum(b.shape[2] for b in blocks)
            T = np.zeros((ml, d, mr), dtype=np.complex128)
            r0 = c0 = 0
            for b in blocks:
                T[r0:r0 + b.shape[0], :, c0:c0 + b.shape[2]] = b
                r0 += b.shape[0]
                c0 += b.shape[2]
            out.append(T)
    return MPS(out, 0)


def expect_between(phi: MPS, W, psi: MPS) -> complex:
    """<phi|H|psi> through left environments E[a', w, a] built with the bra
    phi and the ket psi."""
    E = np.ones((1, 1, 1), dtype=np.complex128)
    for B, Wp, A in zip(phi.A, W, psi.A):
        E = np.einsum("xwz,xsy,wstv,ztb->yvb", E, np.conj(B), np.asarray(Wp, dtype=np.complex128), A,
                      optimize=True)
    return complex(E[0, 0, 0])


def _scaled(mps: MPS, c) -> MPS:
    out = mps.copy()
    out.A[0] = out.A[0] * c
    return out


# ------------------------------------------------------------ the step
def _solve(S, Hm, dt_fs):
    """Exact propagator in span{k_0..k_{m-1}}: Krylov-ordered orthonormal
    basis u = k X from the Cholesky factor S = L L^+ (X = L^{-+}, upper
    triangular, so u_j lies in span{k_0..k_j}); H_r = X^+ H X; start vector
    b = X^+ S e_0; returns (c = X exp(-i H_r dt/hbar) b, exp(...) b)."""
    L = np.linalg.cholesky(S)
    X = np.conj(np.linalg.inv(L).T)
    Hr = np.conj(X.T) @ Hm @ X
    Hr = 0.5 * (Hr + np.conj(Hr.T))
    lam, V = np.linalg.eigh(Hr)
    b = np.conj(X.T) @ S[:, 0]
    ub = V @ (np.exp(-1j * lam * dt_fs / HBAR_EV_FS) * (np.conj(V.T) @ b))
    return X @ ub, ub


def global_krylov_step(psi: MPS, W, dt_fs: float, opts: TdvpOptions, r_max: int = 20, tol: float = 1e-12,
                       s_floor: float = 1e-13):
    """One global Krylov step (Eqs. Krylov subspace, global Krylov).

    k_0 = psi/|psi|; k_{j+1} = compress(H k_j) / |.|. After each new vector
    the space is orthonormalised in Krylov order through the Gram matrix
    S_ij = <k_i|k_j> and H is projected (H_ij = <k_i|H|k_j>, from the
    uncompressed H k_j where it exists), see _solve. The step stops once the
    newest orthonormal direction's coefficient of the propagated start vector
    is below tol, when the newest vector is (to s_floor) in the span of the
    others (the space is invariant; the vector is dropped), or at r_max. The
    state is sum_j c_j k_j, compressed and scaled back to |psi| (the
    propagator is unitary). Returns (new MPS, info dict)."""
    nrm = np.sqrt(abs(overlap(psi, psi)))
    K = [_scaled(psi, 1.0 / nrm)]
    HK = []          # H k_j, uncompressed
    info = {"r": 0, "converged": False, "disc_basis": 0.0, "disc_final": 0.0, "basis_bonds": []}
    S = np.ones((1, 1), dtype=np.complex128)
    Hm = np.array([[expect_between(K[0], W, K[0])]])
    c, _ = _solve(S, Hm, dt_fs)
    for r in range(1, r_max + 1):
        HK.append(apply_mpo(W, K[-1]))
        nxt, dd = compress(HK[-1], opts)
        nn = np.sqrt(abs(overlap(nxt, nxt)))
        if nn == 0.0:
            info["converged"] = True
            break
        K.append(_scaled(nxt, 1.0 / nn))
        m = len(K)
        S = np.array([[overlap(K[i], K[j]) for j in range(m)] for i in range(m)])
        S = 0.5 * (S + np.conj(S.T))
        ev = np.linalg.eigvalsh(S)
        if ev[0] <= s_floor * ev[-1]:
            K.pop()
            info["converged"] = True
            break
        info["disc_basis"] += dd
        info["basis_bonds"].append(max(K[-1].bond_dims()) if K[-1].n > 1 else 1)
        Hm = np.zeros((m, m), dtype=np.complex128)
        for i in range(m):
            for j in range(m):
                Hm[i, j] = overlap(K[i], HK[j]) if j < len(HK) else expect_between(K[i], W, K[j])
        c, ub = _solve(S, Hm, dt_fs)
        info["r"] = r
        if abs(ub[-1]) < tol:
            info["converged"] = True
            break
    out, dd = compress(mps_sum(list(c), K[: len(c)]), opts)
    info["disc_final"] = dd
    on = np.sqrt(abs(overlap(out, out)))
    out.A[0] = out.A[0] * (nrm / on)
    return out, info


def prestep_then_tdvp1(psi: MPS, W, dt_fs: float, n_pre: int, n_tdvp1: int, opts: TdvpOptions,
                       r_max: int = 20, tol: float = 1e-12):
    """n_pre global Krylov steps (bond growth), then n_tdvp1 one-site TDVP
    steps at the bonds the pre-steps reached (Sec. 2.1.2, one-site TDVP
    paragraph). Returns the list of states after every step."""
    states = []
    cur = psi
    for _ in range(n_pre):
        cur, _ = global_krylov_step(cur, W, dt_fs, opts, r_max, tol)
        states.append(cur.copy())
    sim = Tdvp1(cur.copy(), W, opts)
    for _ in range(n_tdvp1):
        sim.step(dt_fs)
        states.append(sim.mps.copy())
    return states
