"""Gradient of the electronic populations with respect to the linear
vibronic couplings g^I_ij (Eq. Helvib_2) - oracle side.

Test infrastructure only (see the package docstring).

This is the quantity a differentiable propagation returns: dP_k(t)/dg for
the populations of Sec. 3.1 after propagation under the model of Sec. 2.2.
For a time-independent H(g), psi(t) = exp(-iHt/hbar) psi0 and (Duhamel)
  dpsi/dg = -(i/hbar) int_0^t exp(-iH(t-s)/hbar) (dH/dg) exp(-iHs/hbar) psi0 ds.
In the eigenbasis H = V diag(E) V^T this is
  dpsi/dg = V [ (V^T (dH/dg) V) o Phi(t) ] V^T psi0,
  Phi_ab = (exp(-iE_a t/hbar) - exp(-iE_b t/hbar)) / (E_a - E_b)   (E_a != E_b)
  Phi_aa = -(i t/hbar) exp(-iE_a t/hbar)
and dP_k/dg = 2 Re <psi(t)| (|k><k| x 1) |dpsi/dg>. Tiny systems only (dense
eigendecomposition of H on the full product basis).

A parameter (I, i, j) is the coupling g^I_ij of mode I between electronic
states i and j; for i != j it moves g^I_ij and g^I_ji together, so H stays
Hermitian.
"""
from __future__ import annotations

import copy

import numpy as np

from vibmodels import HBAR_EV_FS, chain_order, local_dims

from .vibronic import exact_propagate, hamiltonian_sparse, populations_from_vector


def _with_g1(model: dict, I: int, i: int, j: int, value: float) -> dict:
    m = copy.deepcopy(model)
    g1 = np.array(m["g1"], dtype=float)
    g1[I, i, j] = value
    g1[I, j, i] = value
    m["g1"] = g1
    return m


def coupling_derivative(model: dict, I: int, i: int, j: int) -> np.ndarray:
    """dH/dg^I_ij on the full basis: the Hamiltonian of the model with every
    coefficient zero except g^I_ij (and g^I_ji) = 1."""
    n_el = int(model["n_el"])
    m = copy.deepcopy(model)
    m["e0"] = np.zeros(n_el)
    m["v0"] = np.zeros((n_el, n_el))
    m["omega"] = np.zeros(len(model["omega"]))
    m["g1"] = np.zeros_like(np.asarray(model["g1"], dtype=float))
    m["g2"] = []
    m["include_zpe"] = 0
    m = _with_g1(m, I, i, j, 1.0)
    return hamiltonian_sparse(m).toarray()


def _el_projectors(model: dict):
    dims = local_dims(model)
    e = chain_order(model).index(-1)
    n_el = dims[e]
    idx = np.indices(dims).reshape(len(dims), -1)[e]
    return [idx == k for k in range(n_el)]


def population_gradient(model: dict, psi0: np.ndarray, t_fs: float, params) -> np.ndarray:
    """[len(params), n_el] array of dP_k(t)/dg for the parameters (I, i, j),
    by the Duhamel formula in the eigenbasis of H."""
    H = hamiltonian_sparse(model).toarray()
    E, V = np.linalg.eigh(H)
    x = t_fs / HBAR_EV_FS
    ph = np.exp(-1j * E * x)
    dE = E[:, None] - E[None, :]
    near = np.abs(dE) * max(x, 1.0) < 1e-9
    Phi = np.where(near, -1j * x * 0.5 * (ph[:, None] + ph[None, :]),
                   (ph[:, None] - ph[None, :]) / np.where(near, 1.0, dE))
    c0 = V.T @ psi0
    psi_t = V @ (ph * c0)
    projs = _el_projectors(model)
    out = np.zeros((len(params), len(projs)))
    for r, (I, i, j) in enumerate(params):
        G = V.T @ coupling_derivative(model, I, i, j) @ V
        dpsi = V @ ((G * Phi) @ c0)
        for k, P in enumerate(projs):
            out[r, k] = 2.0 * np.real(np.vdot(psi_t[P], dpsi[P]))
    return out


def population_gradient_fd(model: dict, psi0: np.ndarray, t_fs: float, params, h: float = 1e-5,
                           propagate=None) -> np.ndarray:
    """Central finite differences (P(g + h) - P(g - h)) / 2h of the
    populations at t. propagate(model) -> populations; default exact
    propagation of psi0."""
    if propagate is None:
        def propagate(m):
            return populations_from_vector(m, exact_propagate(m, psi0, t_fs, 1)[-1])
    g1 = np.asarray(model["g1"], dtype=float)
    out = []
    for (I, i, j) in params:
        g = float(g1[I, i, j])
        up = propagate(_with_g1(model, I, i, j, g + h))
        dn = propagate(_with_g1(model, I, i, j, g - h))
        out.append((np.asarray(up) - np.asarray(dn)) / (2.0 * h))
    return np.array(out)
