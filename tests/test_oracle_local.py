"""Pins of the oracle's local operations: environments, H_eff,1 / H_eff,2
(Eqs. one-site Hamiltonian 1, two-site Hamiltonian), the Krylov exponential
(Eq. Krylov subspace) and the truncated split (Sec. 2.1.1)."""
import numpy as np
import pytest
import scipy.linalg as sla

import vibmodels as vm
from oracle import mpo, tdvp, vibronic


def _block_bases(rng, dims, D, i):
    """Random isometries for the left block (sites < i) and the right block
    (sites > i+1) together with their MPS tensors."""
    n = len(dims)
    Db = [1] + D + [1]
    tens = [None] * n
    for p in range(i):
        dl, d, dr = Db[p], dims[p], Db[p + 1]
        rows = vm.random_isometry_rows(rng, dr, dl * d)  # dr x (dl d), orthonormal rows
        tens[p] = np.conj(rows.T).reshape(dl, d, dr)     # left-orthonormal
    for p in range(i + 2, n):
        dl, d, dr = Db[p], dims[p], Db[p + 1]
        tens[p] = vm.random_isometry_rows(rng, dl, d * dr).reshape(dl, d, dr)
    # block bases as explicit matrices
    PL = np.ones((1, 1), dtype=complex)
    for p in range(i):
        PL = np.einsum("Xa,asb->Xsb", PL, tens[p]).reshape(-1, Db[p + 1])
    PR = np.ones((1, 1), dtype=complex)
    for p in range(n - 1, i + 1, -1):
        PR = np.einsum("asb,bY->asY", tens[p], PR).reshape(Db[p], -1)
    return tens, PL, PR, Db


@pytest.mark.parametrize("i", [0, 1, 2])
def test_heff2_equals_dense_projection(i):
    rng = np.random.Generator(np.random.PCG64(5 + i))
    m = vm.model_internal_conversion(n_modes=4, level_range=(2, 3), n_offdiag=2, n_bilinear=3)
    dims = vm.local_dims(m)
    n = len(dims)
    D = [2, 3, 3, 2][: n - 1]
    tens, PL, PR, Db = _block_bases(rng, dims, D, i)
    W = [w.astype(complex) for w in mpo.build_mpo(m)]
    L = np.ones((1, 1, 1), dtype=complex)
    for p in range(i):
        L = tdvp.env_left_update(L, tens[p], W[p])
    R = np.ones((1, 1, 1), dtype=complex)
    for p in range(n - 1, i + 1, -1):
        R = tdvp.env_right_update(R, tens[p], W[p])
    theta = vm.random_complex(rng, (Db[i], dims[i], dims[i + 1], Db[i + 2]))
    y = tdvp.heff2_apply(L, W[i], W[i + 1], R, theta)
    # dense: P = PL (x) 1 (x) 1 (x) PR^T maps theta into the full space
    H = vibronic.hamiltonian_sparse(m).toarray()
    full = np.einsum("Xa,astb,bY->XstY", PL, theta, PR).reshape(-1)
    Hf = (H @ full).reshape(PL.shape[0], dims[i], dims[i + 1], PR.shape[1])
    yd = np.einsum("Xa,XstY,bY->astb", np.conj(PL), Hf, np.conj(PR))
    assert np.max(np.abs(y - yd)) < 1e-12 * max(1.0, np.max(np.abs(yd)))


@pytest.mark.parametrize("i", [0, 1, 3])
def test_heff1_equals_dense_projection(i):
    rng = np.random.Generator(np.random.PCG64(17 + i))
    m = vm.model_small_2state(n_modes=3, levels=3)
    dims = vm.local_dims(m)
    n = len(dims)
    D = [2, 3, 3]
    Db = [1] + D + [1]
    # left block = sites < i, right block = sites > i
    tens = [None] * n
    for p in range(i):
        rows = vm.random_isometry_rows(rng, Db[p + 1], Db[p] * dims[p])
        tens[p] = np.conj(rows.T).reshape(Db[p], dims[p], Db[p + 1])
    for p in range(i + 1, n):
        tens[p] = vm.random_isometry_rows(rng, Db[p], dims[p] * Db[p + 1]).reshape(Db[p], dims[p], Db[p + 1])
    PL = np.ones((1, 1), dtype=complex)
    for p in range(i):
        PL = np.einsum("Xa,asb->Xsb", PL, tens[p]).reshape(-1, Db[p + 1])
    PR = np.ones((1, 1), dtype=complex)
    for p in range(n - 1, i, -1):
        PR = np.einsum("asb,bY->asY", tens[p], PR).reshape(Db[p], -1)
    W = [w.astype(complex) for w in mpo.build_mpo(m)]
    L = np.ones((1, 1, 1), dtype=complex)
    for p in range(i):
        L = tdvp.env_left_update(L, tens[p], W[p])
    R = np.ones((1, 1, 1), dtype=complex)
    for p in range(n - 1, i, -1):
        R = tdvp.env_right_update(R, tens[p], W[p])
    C = vm.random_complex(rng, (Db[i], dims[i], Db[i + 1]))
    y = tdvp.heff1_apply(L, W[i], R, C)
    H = vibronic.hamiltonian_sparse(m).toarray()
    full = np.einsum("Xa,atb,bY->XtY", PL, C, PR).reshape(-1)
    Hf = (H @ full).reshape(PL.shape[0], dims[i], PR.shape[1])
    yd = np.einsum("Xa,XtY,bY->atb", np.conj(PL), Hf, np.conj(PR))
    assert np.max(np.abs(y - yd)) < 1e-12 * max(1.0, np.max(np.abs(yd)))


@pytest.mark.parametrize("dt", [0.25, -0.25, 1.0])
def test_krylov_matches_library_expm(dt):
    rng = np.random.Generator(np.random.PCG64(3))
    n = 60
    X = vm.random_complex(rng, (n, n), 0.3)
    H = 0.5 * (X + X.conj().T)
    v = vm.random_complex(rng, (n,))
    y, it, conv = tdvp.krylov_expm(lambda x: H @ x, v, dt, kmax=40, tol=1e-13)
    ref = sla.expm(-1j * H * dt / vm.HBAR_EV_FS) @ v
    assert conv
    assert np.linalg.norm(y - ref) < 1e-11 * np.linalg.norm(v)


def test_krylov_exhausts_small_space_exactly():
    rng = np.random.Generator(np.random.PCG64(4))
    X = vm.random_complex(rng, (5, 5))
    H = X + X.conj().T
    v = vm.random_complex(rng, (5,))
    y, it, conv = tdvp.krylov_expm(lambda x: H @ x, v, 2.0, kmax=30, tol=1e-30)
    assert it == 5 and conv
    ref = sla.expm(-1j * H * 2.0 / vm.HBAR_EV_FS) @ v
    assert np.linalg.norm(y - ref) < 1e-11 * np.linalg.norm(v)


def test_krylov_eigenvector_breakdown():
    H = np.diag([1.0, 2.0, 3.0]).astype(complex)
    v = np.array([0, 1.0, 0], dtype=complex)
    y, it, conv = tdvp.krylov_expm(lambda x: H @ x, v, 0.7)
    assert it == 1 and conv
    assert np.allclose(y, np.exp(-1j * 2.0 * 0.7 / vm.HBAR_EV_FS) * v, atol=1e-14)


def test_split_left_reconstructs_and_matches_svd():
    rng = np.random.Generator(np.random.PCG64(8))
    theta = vm.random_complex(rng, (3, 4, 5, 2))
    theta /= np.linalg.norm(theta)
    A, C, disc = tdvp.split_left(theta, tdvp.TdvpOptions())
    M = theta.reshape(12, 10)
    s = np.linalg.svd(M, compute_uv=False)
    assert A.shape[2] == 10 and disc < 1e-15
    k = A.shape[2]
    Am = A.reshape(12, k)
    assert np.allclose(Am.conj().T @ Am, np.eye(k), atol=1e-13)
    assert np.allclose(np.einsum("ask,ktb->astb", A, C), theta, atol=1e-13)
    sc = np.linalg.svd(C.reshape(k, -1), compute_uv=False)
    assert np.allclose(sc, s, atol=1e-13)


def test_split_right_truncates_to_cap_like_svd():
    rng = np.random.Generator(np.random.PCG64(9))
    theta = vm.random_complex(rng, (4, 3, 3, 4))
    theta /= np.linalg.norm(theta)
    C, B, disc = tdvp.split_right(theta, tdvp.TdvpOptions(m_max=5))
    M = theta.reshape(12, 12)
    s = np.linalg.svd(M, compute_uv=False)
    assert B.shape[0] == 5
    Bm = B.reshape(5, -1)
    assert np.allclose(Bm @ Bm.conj().T, np.eye(5), atol=1e-13)
    assert abs(disc - np.sum(s[5:] ** 2) / np.sum(s ** 2)) < 1e-13
    # best rank-5 approximation (Eckart-Young), renormalised
    U, S, Vh = np.linalg.svd(M)
    best = (U[:, :5] * S[:5]) @ Vh[:5]
    best /= np.linalg.norm(best)
    assert np.allclose(np.einsum("ask,ktb->astb", C, B).reshape(12, 12), best, atol=1e-12)


def test_choose_rank_rules():
    o = tdvp.TdvpOptions(eps=1e-3)
    lam = np.array([0.6, 0.3, 0.0995, 0.0004, 0.0001])
    # tail 0.0005 > 1e-3*1.0? no: 0.0005 <= 0.001 -> drop two
    assert tdvp.choose_rank(lam, o) == 3
    assert tdvp.choose_rank(lam, tdvp.TdvpOptions(m_max=2)) == 2
    # never split a degenerate multiplet
    lam2 = np.array([0.5, 0.2, 0.2, 0.1])
    assert tdvp.choose_rank(lam2, tdvp.TdvpOptions(m_max=2)) == 1
    # zero floor
    lam3 = np.array([1.0, 1e-15, 1e-16])
    assert tdvp.choose_rank(lam3, tdvp.TdvpOptions()) == 1
    assert tdvp.choose_rank(lam3, tdvp.TdvpOptions(zero_floor=0.0)) == 3
    # rank bound
    assert tdvp.choose_rank(np.array([0.5, 0.5, 0.0]), tdvp.TdvpOptions(zero_floor=0.0), 2) == 2
