"""Checks at the full size of the benchmark workload (2 states + 24 modes,
d = 10..30, bonds 64), in the configuration bench.py times: the H_eff,2
product at the largest pair against the oracle (both forms), and one whole
time step of the mixed form against the FP64 form from the same
bond-saturated state (properties that hold at any size: unit norm, bonds
within the cap, populations of the two forms agreeing)."""
import numpy as np
import pytest

import vibmodels as vm
from oracle import mpo as ompo
from oracle import tdvp as otdvp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M = 64


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


@pytest.fixture(scope="module")
def model():
    return vm.model_internal_conversion()


def _envs(P, mpo, W, T, Db, i):
    """Environments of the pair (i, i+1) built on the GPU and by the oracle
    from the same random mixed-canonical tensors."""
    n = len(T)
    Lg = torch.ones(1, dtype=torch.complex128, device="cuda")
    Lo = np.ones((1, 1, 1), dtype=complex)
    for p in range(i):
        wl, d, wr = mpo.site_dims(p)
        Ln = torch.zeros(Db[p + 1] * wr * Db[p + 1], dtype=torch.complex128, device="cuda")
        work = torch.zeros(P.vb_env_work_elems(mpo, p, Db[p], Db[p + 1]), dtype=torch.complex128, device="cuda")
        P.vb_env_left_update(mpo, p, Db[p], Db[p + 1], Lg, torch.from_numpy(T[p]).cuda(), Ln, work)
        Lg = Ln
        Lo = otdvp.env_left_update(Lo, T[p], W[p])
    Rg = torch.ones(1, dtype=torch.complex128, device="cuda")
    Ro = np.ones((1, 1, 1), dtype=complex)
    for p in range(n - 1, i + 1, -1):
        wl, d, wr = mpo.site_dims(p)
        Rn = torch.zeros(Db[p] * wl * Db[p], dtype=torch.complex128, device="cuda")
        work = torch.zeros(P.vb_env_work_elems(mpo, p, Db[p], Db[p + 1]), dtype=torch.complex128, device="cuda")
        P.vb_env_right_update(mpo, p, Db[p], Db[p + 1], Rg, torch.from_numpy(T[p]).cuda(), Rn, work)
        Rg = Rn
        Ro = otdvp.env_right_update(Ro, T[p], W[p])
    return Lg, Rg, Lo, Ro


@pytest.mark.parametrize("form,tol", [("fp64", 1e-11), ("mixed", 2e-5)])
def test_heff2_largest_pair_full_size(P, model, form, tol):
    dims = vm.local_dims(model)
    i = max(range(1, len(dims) - 2), key=lambda k: dims[k] * dims[k + 1])
    Db = [1] + vm.bond_caps(dims, M) + [1]
    rng = np.random.Generator(np.random.PCG64(2024))
    n = len(dims)
    T = [None] * n
    for p in range(i):
        rows = vm.random_isometry_rows(rng, Db[p + 1], Db[p] * dims[p])
        T[p] = np.ascontiguousarray(np.conj(rows.T).reshape(Db[p], dims[p], Db[p + 1]))
    for p in range(i + 2, n):
        T[p] = np.ascontiguousarray(vm.random_isometry_rows(rng, Db[p], dims[p] * Db[p + 1]).reshape(Db[p], dims[p], Db[p + 1]))
    mpo = P.Mpo(model)
    Wo = [w.astype(complex) for w in ompo.build_mpo(model)]
    Lg, Rg, Lo, Ro = _envs(P, mpo, Wo, T, Db, i)
    mL, mR = Db[i], Db[i + 2]
    x = vm.random_complex(rng, (mL, dims[i], dims[i + 1], mR))
    y = torch.zeros(x.size, dtype=torch.complex128, device="cuda")
    work = torch.zeros(P.vb_heff_work_elems(mpo, i, mL, mR, True), dtype=torch.complex128, device="cuda")
    dt = P.VB_MIXED if form == "mixed" else P.VB_FP64
    P.vb_heff2_apply(mpo, i, mL, mR, Lg, Rg, torch.from_numpy(x).cuda(), y, work, dt)
    torch.cuda.synchronize()
    yo = otdvp.heff2_apply(Lo, Wo[i], Wo[i + 1], Ro, x)
    yg = y.cpu().numpy().reshape(yo.shape)
    assert np.max(np.abs(yg - yo)) <= tol * np.max(np.abs(yo))


def test_full_size_step_mixed_vs_fp64(P, model):
    dims = vm.local_dims(model)
    ts = vm.random_right_canonical_mps(424242, dims, M)
    mpo = P.Mpo(model)
    kw = dict(m_max=M, eps=1e-8, zero_floor=1e-14, krylov_max=30, krylov_tol=1e-13)
    out = {}
    for name, dt in (("fp64", P.VB_FP64), ("mixed", P.VB_MIXED)):
        mps = P.Mps(mpo, m_cap=M, dtype=dt, tensors=ts)
        st = mps.sweep(0.5, **kw)
        pops = mps.populations()
        bonds = mps.bond_dims()
        assert abs(pops.sum() - 1.0) < 1e-12 and np.all(pops >= 0)
        assert max(bonds) <= M and st.noconv == 0
        out[name] = (pops, bonds, st)
        mps.close()
    assert np.max(np.abs(out["fp64"][0] - out["mixed"][0])) < 1e-4
    assert abs(out["fp64"][2].discarded_weight - out["mixed"][2].discarded_weight) < 1e-6
