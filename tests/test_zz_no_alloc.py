"""The allocation-free eigensolver entry point against the regular one.

vb_herm_eig_top_noalloc serves callers that cannot allocate device memory
where they need a split (their device memory belongs to a host framework's
pool, or they sit in a latency-critical loop that must not pay cudaMalloc's
implicit synchronisation). It keeps its workspace in a fixed array inside the
library. This test calls it through the C ABI twice in a row (the array keeps
the first call's contents) and checks both results against vb_herm_eig_top,
which uses a caller-provided workspace. This file is collected last so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import vibmodels as vm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EIG_TOL = 1e-12  # relative to the largest eigenvalue, as in the eigensolver parity test


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


def _rho(seed, n):
    rng = np.random.Generator(np.random.PCG64(seed))
    M = vm.random_complex(rng, (n, n // 2 + 5))
    return M @ M.conj().T


def _regular(P, rho, k_want, k_vec):
    n = rho.shape[0]
    r = torch.from_numpy(rho.copy()).cuda()
    ev = torch.zeros(k_want, dtype=torch.float64, device="cuda")
    Z = torch.zeros(k_vec * n, dtype=torch.complex128, device="cuda")
    work = torch.zeros(P.vb_eig_work_bytes(n, k_want), dtype=torch.uint8, device="cuda")
    P.vb_herm_eig_top(n, r, k_want, k_vec, ev, Z, work)
    torch.cuda.synchronize()
    return ev.cpu().numpy(), Z.cpu().numpy().reshape(k_vec, n)


def _noalloc(P, rho, k_want, k_vec):
    n = rho.shape[0]
    r = torch.from_numpy(rho.copy()).cuda()
    ev = torch.zeros(k_want, dtype=torch.float64, device="cuda")
    Z = torch.zeros(k_vec * n, dtype=torch.complex128, device="cuda")
    P.vb_herm_eig_top_noalloc(n, r, k_want, k_vec, ev, Z)
    torch.cuda.synchronize()
    return ev.cpu().numpy(), Z.cpu().numpy().reshape(k_vec, n)


def test_noalloc_eigensolver_matches_regular_twice_in_a_row(P):
    # two different matrices, one after the other: the second call must not
    # depend on what the first one left in the shared array
    # n = 200 and 96 take the cooperative reduction (bounded grid barrier,
    # whose error word the call reads back), n = 48 the per-column path
    for seed, n, k_want, k_vec in ((3, 200, 65, 64), (4, 96, 33, 20), (5, 48, 20, 12)):
        rho = _rho(seed, n)
        ev_r, Z_r = _regular(P, rho, k_want, k_vec)
        ev_n, Z_n = _noalloc(P, rho, k_want, k_vec)
        scale = ev_r[0]
        assert np.max(np.abs(ev_n - ev_r)) <= EIG_TOL * scale
        # eigenvectors are unique up to phase (and rotation inside a
        # degenerate multiplet): compare projectors onto the kept space
        Pn = Z_n.T @ Z_n.conj()
        Pr = Z_r.T @ Z_r.conj()
        assert np.max(np.abs(Pn - Pr)) < 1e-9
        res = rho @ Z_n.T - Z_n.T * ev_n[:k_vec][None, :]
        assert np.max(np.abs(res)) < 1e-10 * scale


def test_noalloc_rejects_sizes_beyond_the_fixed_workspace(P):
    rho = torch.zeros(300 * 300, dtype=torch.complex128, device="cuda")
    ev = torch.zeros(10, dtype=torch.float64, device="cuda")
    Z = torch.zeros(10 * 300, dtype=torch.complex128, device="cuda")
    with pytest.raises(P.VbError):
        P.vb_herm_eig_top_noalloc(300, rho, 10, 10, ev, Z)
