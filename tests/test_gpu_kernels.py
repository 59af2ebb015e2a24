"""GPU parity of the single operations behind tdvp2_sweep, through the C ABI,
against the CPU oracle: environment updates + H_eff,2 / H_eff,1
(Eqs. one-site Hamiltonian 1, two-site Hamiltonian) and the Hermitian
eigensolver of the truncated split (Sec. 2.1.1)."""
import numpy as np
import pytest

import vibmodels as vm
from oracle import mpo as ompo
from oracle import tdvp as otdvp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HEFF_RTOL = 1e-12  # FP64 contraction: relative to max |y|


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _mixed_canonical(rng, dims, D, i, two_site=True):
    """Random tensors: left-orthonormal for sites < i, right-orthonormal for
    sites > i+1 (two-site) or > i (one-site)."""
    n = len(dims)
    Db = [1] + list(D) + [1]
    first_right = i + 2 if two_site else i + 1
    T = [None] * n
    for p in range(i):
        rows = vm.random_isometry_rows(rng, Db[p + 1], Db[p] * dims[p])
        T[p] = np.conj(rows.T).reshape(Db[p], dims[p], Db[p + 1])
    for p in range(first_right, n):
        T[p] = vm.random_isometry_rows(rng, Db[p], dims[p] * Db[p + 1]).reshape(Db[p], dims[p], Db[p + 1])
    return T, Db


def _envs_gpu(P, mpo, T, Db, i, first_right):
    n = len(T)
    L = _dev(np.ones((1, 1, 1)))
    for p in range(i):
        wl, d, wr = mpo.site_dims(p)
        Ln = torch.zeros(Db[p + 1] * wr * Db[p + 1], dtype=torch.complex128, device="cuda")
        work = torch.zeros(max(1, P.vb_env_work_elems(mpo, p, Db[p], Db[p + 1])), dtype=torch.complex128, device="cuda")
        P.vb_env_left_update(mpo, p, Db[p], Db[p + 1], L, _dev(T[p]), Ln, work)
        L = Ln
    R = _dev(np.ones((1, 1, 1)))
    for p in range(n - 1, first_right - 1, -1):
        wl, d, wr = mpo.site_dims(p)
        Rn = torch.zeros(Db[p] * wl * Db[p], dtype=torch.complex128, device="cuda")
        work = torch.zeros(max(1, P.vb_env_work_elems(mpo, p, Db[p], Db[p + 1])), dtype=torch.complex128, device="cuda")
        P.vb_env_right_update(mpo, p, Db[p], Db[p + 1], R, _dev(T[p]), Rn, work)
        R = Rn
    return L, R


def _envs_oracle(W, T, i, first_right):
    n = len(T)
    L = np.ones((1, 1, 1), dtype=complex)
    for p in range(i):
        L = otdvp.env_left_update(L, T[p], W[p])
    R = np.ones((1, 1, 1), dtype=complex)
    for p in range(n - 1, first_right - 1, -1):
        R = otdvp.env_right_update(R, T[p], W[p])
    return L, R


CASES = [
    # (model, bonds, pair index)
    ("ic_small", [2, 5, 7, 6, 3], 1),
    ("ic_small", [2, 5, 7, 6, 3], 2),
    ("ic_small", [2, 5, 7, 6, 3], 0),
    ("ic_small", [2, 5, 7, 6, 3], 4),
    ("c1", [2, 16, 16, 8], 1),
    ("sf_small", [3, 9, 12, 12, 9, 3], 2),
]


def _model(name):
    if name == "ic_small":
        return vm.model_internal_conversion(seed=21, n_modes=5, level_range=(3, 7), n_offdiag=2, n_bilinear=4)
    if name == "c1":
        return vm.model_small_2state()
    if name == "sf_small":
        return vm.model_singlet_fission(n_bath=2, levels=3)
    raise KeyError(name)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_heff2_parity_through_environments(P, case):
    name, D, i = CASES[case]
    m = _model(name)
    dims = vm.local_dims(m)
    D = [min(b, int(np.prod(dims[: k + 1])), int(np.prod(dims[k + 1:]))) for k, b in enumerate(D)]
    rng = np.random.Generator(np.random.PCG64(100 + case))
    T, Db = _mixed_canonical(rng, dims, D, i)
    mpo = P.Mpo(m)
    Lg, Rg = _envs_gpu(P, mpo, T, Db, i, i + 2)
    Wo = [w.astype(complex) for w in ompo.build_mpo(m)]
    Lo, Ro = _envs_oracle(Wo, T, i, i + 2)
    mL, mR = Db[i], Db[i + 2]
    theta = vm.random_complex(rng, (mL, dims[i], dims[i + 1], mR))
    y = torch.zeros(theta.size, dtype=torch.complex128, device="cuda")
    work = torch.zeros(P.vb_heff_work_elems(mpo, i, mL, mR, True), dtype=torch.complex128, device="cuda")
    P.vb_heff2_apply(mpo, i, mL, mR, Lg, Rg, _dev(theta), y, work)
    torch.cuda.synchronize()
    yo = otdvp.heff2_apply(Lo, Wo[i], Wo[i + 1], Ro, theta)
    yg = y.cpu().numpy().reshape(yo.shape)
    assert np.max(np.abs(yg - yo)) <= HEFF_RTOL * np.max(np.abs(yo))


@pytest.mark.parametrize("case", range(len(CASES)))
def test_heff1_parity_through_environments(P, case):
    name, D, i = CASES[case]
    m = _model(name)
    dims = vm.local_dims(m)
    D = [min(b, int(np.prod(dims[: k + 1])), int(np.prod(dims[k + 1:]))) for k, b in enumerate(D)]
    rng = np.random.Generator(np.random.PCG64(200 + case))
    T, Db = _mixed_canonical(rng, dims, D, i, two_site=False)
    mpo = P.Mpo(m)
    Lg, Rg = _envs_gpu(P, mpo, T, Db, i, i + 1)
    Wo = [w.astype(complex) for w in ompo.build_mpo(m)]
    Lo, Ro = _envs_oracle(Wo, T, i, i + 1)
    mL, mR = Db[i], Db[i + 1]
    Cc = vm.random_complex(rng, (mL, dims[i], mR))
    y = torch.zeros(Cc.size, dtype=torch.complex128, device="cuda")
    work = torch.zeros(P.vb_heff_work_elems(mpo, i, mL, mR, False), dtype=torch.complex128, device="cuda")
    P.vb_heff1_apply(mpo, i, mL, mR, Lg, Rg, _dev(Cc), y, work)
    torch.cuda.synchronize()
    yo = otdvp.heff1_apply(Lo, Wo[i], Ro, Cc)
    yg = y.cpu().numpy().reshape(yo.shape)
    assert np.max(np.abs(yg - yo)) <= HEFF_RTOL * np.max(np.abs(yo))


def _eig_case(P, rho, k_want, k_vec):
    n = rho.shape[0]
    r = _dev(rho)
    ev = torch.zeros(k_want, dtype=torch.float64, device="cuda")
    Z = torch.zeros(max(1, k_vec) * n, dtype=torch.complex128, device="cuda")
    work = torch.zeros(P.vb_eig_work_bytes(n, k_want), dtype=torch.uint8, device="cuda")
    P.vb_herm_eig_top(n, r, k_want, k_vec, ev, Z, work)
    torch.cuda.synchronize()
    return ev.cpu().numpy(), Z.cpu().numpy()[: k_vec * n].reshape(k_vec, n)


@pytest.mark.parametrize("n,k_want,k_vec", [(1, 1, 1), (2, 2, 2), (3, 2, 1), (17, 9, 8), (64, 64, 40),
                                            (130, 65, 64), (257, 33, 32)])
def test_eigensolver_matches_library_eigh(P, n, k_want, k_vec):
    rng = np.random.Generator(np.random.PCG64(n))
    M = vm.random_complex(rng, (n, max(1, n // 2 + 3)))
    rho = M @ M.conj().T
    ev, Z = _eig_case(P, rho, k_want, k_vec)
    ref = np.sort(np.linalg.eigvalsh(rho))[::-1][:k_want]
    scale = ref[0]
    assert np.max(np.abs(ev - ref)) < 1e-12 * scale
    # eigenvector residuals and orthonormality
    res = rho @ Z.T - Z.T * ev[:k_vec][None, :]
    assert np.max(np.abs(res)) < 1e-10 * scale
    assert np.max(np.abs(Z.conj() @ Z.T - np.eye(k_vec))) < 1e-12


def test_eigensolver_degenerate_and_zero_eigenvalues(P):
    rng = np.random.Generator(np.random.PCG64(77))
    n = 48
    Q, _ = np.linalg.qr(vm.random_complex(rng, (n, n)))
    lam = np.concatenate([[0.3, 0.2, 0.2, 0.2, 0.1, 0.1], np.full(n - 6, 0.0)])
    rho = (Q * lam) @ Q.conj().T
    ev, Z = _eig_case(P, rho, 8, 6)
    assert np.allclose(ev[:6], lam[:6], atol=1e-13)
    assert np.max(np.abs(ev[6:])) < 1e-13
    # the kept subspace is unique: compare projectors
    Pg = Z.T @ Z.conj()
    Pr = Q[:, :6] @ Q[:, :6].conj().T
    assert np.max(np.abs(Pg - Pr)) < 1e-10
