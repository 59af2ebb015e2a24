"""Mixed-precision form (H_eff products and environments in complex FP32,
kept directions of the split found in FP32; Lanczos, exponential, split
tensors and weights in FP64) against the FP64 oracle: single products within
FP32 accuracy and whole 2TDVP runs with populations within 1e-4."""
import numpy as np
import pytest

import vibmodels as vm
from oracle import mpo as ompo
from oracle import tdvp as otdvp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_kernels import CASES, _dev, _envs_gpu, _envs_oracle, _mixed_canonical, _model  # noqa: E402

HEFF_MIXED_RTOL = 2e-5   # FP32 products with FP32 accumulation, relative to max |y|
POP_TOL_MIXED = 1e-4     # populations vs the FP64 oracle


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("two_site", [True, False])
def test_mixed_heff_parity(P, case, two_site):
    name, D, i = CASES[case]
    m = _model(name)
    dims = vm.local_dims(m)
    D = [min(b, int(np.prod(dims[: k + 1])), int(np.prod(dims[k + 1:]))) for k, b in enumerate(D)]
    rng = np.random.Generator(np.random.PCG64(300 + case))
    T, Db = _mixed_canonical(rng, dims, D, i, two_site)
    mpo = P.Mpo(m)
    fr = i + 2 if two_site else i + 1
    Lg, Rg = _envs_gpu(P, mpo, T, Db, i, fr)
    Wo = [w.astype(complex) for w in ompo.build_mpo(m)]
    Lo, Ro = _envs_oracle(Wo, T, i, fr)
    mL, mR = Db[i], Db[fr]
    if two_site:
        x = vm.random_complex(rng, (mL, dims[i], dims[i + 1], mR))
        yo = otdvp.heff2_apply(Lo, Wo[i], Wo[i + 1], Ro, x)
    else:
        x = vm.random_complex(rng, (mL, dims[i], mR))
        yo = otdvp.heff1_apply(Lo, Wo[i], Ro, x)
    y = torch.zeros(x.size, dtype=torch.complex128, device="cuda")
    work = torch.zeros(P.vb_heff_work_elems(mpo, i, mL, mR, two_site), dtype=torch.complex128, device="cuda")
    if two_site:
        P.vb_heff2_apply(mpo, i, mL, mR, Lg, Rg, _dev(x), y, work, P.VB_MIXED)
    else:
        P.vb_heff1_apply(mpo, i, mL, mR, Lg, Rg, _dev(x), y, work, P.VB_MIXED)
    torch.cuda.synchronize()
    yg = y.cpu().numpy().reshape(yo.shape)
    assert np.max(np.abs(yg - yo)) <= HEFF_MIXED_RTOL * np.max(np.abs(yo))


def _run(P, m, steps, dt, m_max, eps=0.0):
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, idx, m_cap=m_max, dtype=P.VB_MIXED)
    ref = otdvp.Tdvp2(otdvp.product_mps(dims, idx), ompo.build_mpo(m), otdvp.TdvpOptions(m_max=m_max, eps=eps))
    errs = []
    for _ in range(steps):
        st = mps.sweep(dt, m_max=m_max, eps=eps, krylov_tol=1e-10)
        ref.step(dt)
        errs.append(np.max(np.abs(mps.populations() - otdvp.populations(ref.mps))))
        assert st.noconv == 0
    return errs


def test_mixed_sweeps_two_state_four_mode_m16(P):
    errs = _run(P, vm.model_small_2state(), 16, 0.5, 16)
    assert max(errs) < POP_TOL_MIXED


def test_mixed_sweeps_dbss(P):
    m = vm.model_internal_conversion(seed=31, n_modes=5, level_range=(3, 6), n_offdiag=2, n_bilinear=4)
    errs = _run(P, m, 10, 0.5, 24, eps=1e-6)
    assert max(errs) < POP_TOL_MIXED


def test_mixed_sweeps_large_split_rayleigh_ritz(P):
    # bonds up to 32 with d = 12..16: reduced density matrices of dimension
    # > 192 go through the subspace-iteration split (FP32 directions, FP64
    # basis, projection and weights)
    m = vm.model_internal_conversion(seed=41, n_modes=5, level_range=(12, 16), n_offdiag=2, n_bilinear=4)
    dims = vm.local_dims(m)
    ts = vm.random_right_canonical_mps(77, dims, 32)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, m_cap=32, dtype=P.VB_MIXED, tensors=ts)
    ref = otdvp.Tdvp2(otdvp.MPS(ts), ompo.build_mpo(m), otdvp.TdvpOptions(m_max=32, eps=1e-8))
    assert max(32 * d for d in dims) > 192
    for _ in range(4):
        st = mps.sweep(0.5, m_max=32, eps=1e-8, krylov_tol=1e-10)
        ref.step(0.5)
        assert st.noconv == 0
        assert np.max(np.abs(mps.populations() - otdvp.populations(ref.mps))) < POP_TOL_MIXED


def test_mixed_sweeps_product_state_rank_deficient_splits(P):
    # d = 20..24 from a product state with no discarded-weight threshold:
    # splits of dimension up to ~480 (> 192, subspace iteration) while the
    # Schmidt rank (<= 20) is below the subspace size, so the orthonormalisation
    # meets dependent rows and refills them
    m = vm.model_internal_conversion(seed=43, n_modes=4, level_range=(20, 24), n_offdiag=2, n_bilinear=3)
    dims = vm.local_dims(m)
    assert max(24 * d for d in dims) > 192
    errs = _run(P, m, 8, 0.5, 24, eps=0.0)
    assert max(errs) < POP_TOL_MIXED


def test_wait_flag_reported_and_cleared_by_both_sweeps(P):
    # the failure path of a bounded tensor-core wait, made on the host: the
    # flag such a wait raises is set through the test hook (no kernel times
    # out, nothing faults); each sweep form must report VB_ETIMEOUT once and
    # clear the flag, so the following sweep succeeds
    m = vm.model_small_2state(n_modes=3, levels=6)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, vm.product_state_indices(m), m_cap=16, dtype=P.VB_MIXED)
    mps.sweep(0.5, m_max=16)
    for run in (lambda: mps.sweep1(0.5), lambda: mps.sweep(0.5, m_max=16)):
        mps.raise_wait_flag()
        with pytest.raises(P.VbError) as e:
            run()
        assert e.value.code == P.binding.VB_ETIMEOUT
        mps2 = P.Mps(mpo, vm.product_state_indices(m), m_cap=16, dtype=P.VB_MIXED)
        mps2.sweep(0.5, m_max=16)  # a fresh handle is unaffected
        run()  # the flag was cleared when it was reported


def test_autotuner_picks_a_group_and_keeps_the_result(P):
    # the L leg's resident-B GEMM at the largest pair of the internal-conversion
    # workload (24 M tiles): the tuned group size changes only the schedule,
    # never the arithmetic of a tile (bit-equal products)
    m = vm.model_internal_conversion()
    mpo = P.Mpo(m)
    i, mL, mR = 15, 64, 64
    wl, d1, _ = mpo.site_dims(i)
    _, d2, wr = mpo.site_dims(i + 1)
    rng = np.random.Generator(np.random.PCG64(901))
    L = _dev(vm.random_hermitian_env(rng, mL, wl))
    R = _dev(vm.random_hermitian_env(rng, mR, wr))
    x = _dev(vm.random_complex(rng, (mL, d1, d2, mR)))
    work = torch.zeros(P.vb_heff_work_elems(mpo, i, mL, mR, True), dtype=torch.complex128, device="cuda")
    ys, tables = [], []
    for enable in (1, 0):
        P.vb_autotune(enable, reset=True)
        y = torch.zeros_like(x)
        for _ in range(2):  # the first call tunes, the second uses the table
            P.vb_heff2_apply(mpo, i, mL, mR, L, R, x, y, work, P.VB_MIXED)
        torch.cuda.synchronize()
        ys.append(y.cpu().numpy())
        tables.append(P.vb_autotune())
    P.vb_autotune(1, reset=True)
    print("autotuner table:", tables[0])
    assert len(tables[0]) >= 1 and any("ms=-1" not in t for t in tables[0])
    assert all("group=8" in t for t in tables[1])
    assert np.array_equal(ys[0], ys[1])
