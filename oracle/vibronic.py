"""Vibronic Hamiltonian in second quantisation (Sec. 2.2) - oracle side.

Test infrastructure only (see the package docstring).

H = sum_ij h_ij a_i^+ a_j                               (Eq. Hel_2)
  + sum_I omega_I (b_I^+ b_I + 1/2)                      (Eq. Hvib_2)
  + sum_{I,ij} g^I_ij q_I a_i^+ a_j
  + sum_{(I,J,i,j)} g^{IJ}_ij q_I q_J a_i^+ a_j          (Eq. Helvib_2)
with q = (b + b^+)/sqrt(2). The electronic states form one chain site of
dimension n_el whose operators are |i><j|; each g2 entry is one operator term
(I == J gives q_I^2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import expm_multiply

from vibmodels import HBAR_EV_FS, chain_order, local_dims


# ------------------------------------------------------------ local operators
def boson_b(d: int) -> np.ndarray:
    """Annihilator on the truncated basis |0..d-1>: b|n> = sqrt(n)|n-1>."""
    b = np.zeros((d, d))
    for n in range(1, d):
        b[n - 1, n] = np.sqrt(n)
    return b


def boson_q(d: int) -> np.ndarray:
    b = boson_b(d)
    return (b + b.T) / np.sqrt(2.0)


def boson_n(d: int) -> np.ndarray:
    return np.diag(np.arange(d, dtype=float))


def el_proj(n_el: int, i: int, j: int) -> np.ndarray:
    e = np.zeros((n_el, n_el))
    e[i, j] = 1.0
    return e


def local_matrix(model: dict, pos: int, op) -> np.ndarray:
    """Dense matrix of a local operator `op` at chain position `pos`.
    op: ('E', i, j) | ('q',) | ('q2',) | ('n',) | ('id',)"""
    site = chain_order(model)[pos]
    d = local_dims(model)[pos]
    kind = op[0]
    if kind == "id":
        return np.eye(d)
    if kind == "E":
        assert site < 0
        return el_proj(d, op[1], op[2])
    assert site >= 0
    if kind == "q":
        return boson_q(d)
    if kind == "q2":
        q = boson_q(d)
        return q @ q
    if kind == "n":
        return boson_n(d)
    raise ValueError(op)


# ------------------------------------------------------------------ term list
def term_list(model: dict):
    """The Hamiltonian as a list of (coefficient, {chain position: op}).

    Constants (zero-point energies) are attached as identity on position 0."""
    order = chain_order(model)
    pos_of = {s: p for p, s in enumerate(order)}
    e = pos_of[-1]
    n_el = int(model["n_el"])
    terms = []
    # Eq. Hel_2
    for i in range(n_el):
        for j in range(n_el):
            h = model["e0"][i] if i == j else model["v0"][i][j]
            if h != 0.0:
                terms.append((float(h), {e: ("E", i, j)}))
    # Eq. Hvib_2
    zpe = 0.0
    for I, w in enumerate(model["omega"]):
        terms.append((float(w), {pos_of[I]: ("n",)}))
        zpe += 0.5 * float(w)
    if model.get("include_zpe", 1) and zpe != 0.0:
        terms.append((zpe, {0: ("id",)}))
    # Eq. Helvib_2, linear part
    g1 = np.asarray(model["g1"])
    for I in range(g1.shape[0]):
        for i in range(n_el):
            for j in range(n_el):
                g = float(g1[I, i, j])
                if g != 0.0:
                    terms.append((g, {e: ("E", i, j), pos_of[I]: ("q",)}))
    # Eq. Helvib_2, second-order part
    for (I, J, i, j, v) in model["g2"]:
        if v == 0.0:
            continue
        if I == J:
            terms.append((float(v), {e: ("E", i, j), pos_of[I]: ("q2",)}))
        else:
            terms.append((float(v), {e: ("E", i, j), pos_of[I]: ("q",), pos_of[J]: ("q",)}))
    return terms


# ------------------------------------------------- full-space (tiny systems)
def hamiltonian_sparse(model: dict) -> sp.csr_matrix:
    """H on the full product basis (chain position 0 most significant)."""
    dims = local_dims(model)
    n = len(dims)
    H = None
    for coef, ops in term_list(model):
        mat = None
        for p in range(n):
            loc = local_matrix(model, p, ops[p]) if p in ops else np.eye(dims[p])
            locs = sp.csr_matrix(loc)
            mat = locs if mat is None else sp.kron(mat, locs, format="csr")
        H = coef * mat if H is None else H + coef * mat
    return H.tocsr()


def product_vector(model: dict, indices) -> np.ndarray:
    dims = local_dims(model)
    v = np.ones(1, dtype=complex)
    for p, d in enumerate(dims):
        e = np.zeros(d, dtype=complex)
        e[indices[p]] = 1.0
        v = np.kron(v, e)
    return v


def exact_propagate(model: dict, psi0: np.ndarray, dt_fs: float, n_steps: int):
    """psi(k dt) = exp(-i H k dt / hbar) psi0 for k = 0..n_steps (scipy
    expm_multiply on the sparse H)."""
    H = hamiltonian_sparse(model)
    A = (-1j / HBAR_EV_FS) * H
    return expm_multiply(A, psi0, start=0.0, stop=dt_fs * n_steps,
                         num=n_steps + 1, endpoint=True)


def populations_from_vector(model: dict, psi: np.ndarray) -> np.ndarray:
    dims = local_dims(model)
    order = chain_order(model)
    e = order.index(-1)
    t = psi.reshape(dims)
    t = np.moveaxis(t, e, 0).reshape(dims[e], -1)
    return np.sum(np.abs(t) ** 2, axis=1)


# ------------------------------------------------------------- closed forms
def independent_boson_autocorrelation(model: dict, el_state: int, t_fs) -> np.ndarray:
    """C(t) = <psi(0)|psi(t)> for |el_state> (x) |0...0> when V = 0 and the
    couplings are diagonal (displaced harmonic oscillators):
    C(t) = exp(-i eps t) prod_I exp(-i w t / 2) exp(S (e^{-i w t} - 1) + i S w t)
    with S = g^2/(2 w^2), times in units of hbar."""
    t = np.asarray(t_fs, dtype=float) / HBAR_EV_FS
    c = np.exp(-1j * model["e0"][el_state] * t)
    for I, w in enumerate(model["omega"]):
        g = model["g1"][I][el_state][el_state]
        S = g * g / (2.0 * w * w)
        ph = np.exp(-1j * 0.5 * w * t) if model.get("include_zpe", 1) else 1.0
        c = c * ph * np.exp(S * (np.exp(-1j * w * t) - 1.0) + 1j * S * w * t)
    return c
