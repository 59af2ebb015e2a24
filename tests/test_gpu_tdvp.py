"""GPU parity of whole 2TDVP time steps (Sec. 2.1.2) through the C ABI
(mps_create, tdvp2_sweep, measure_populations) against the CPU oracle, plus
the exactness and closed-form pins on the GPU results."""
import numpy as np
import pytest

import vibmodels as vm
from oracle import mpo as ompo
from oracle import tdvp as otdvp
from oracle import vibronic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

POP_TOL = 1e-8  # FP64 path: populations vs the FP64 oracle


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


def _run_pair(P, m, steps, dt, m_max, eps=0.0, floor=1e-14, pad=False, init=None):
    dims = vm.local_dims(m)
    idx = init if init is not None else vm.product_state_indices(m)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, idx, m_cap=m_max, pad_full=pad)
    o0 = otdvp.padded_product_mps(dims, idx, m_max) if pad else otdvp.product_mps(dims, idx)
    ref = otdvp.Tdvp2(o0, ompo.build_mpo(m), otdvp.TdvpOptions(m_max=m_max, eps=eps, zero_floor=floor))
    assert mps.bond_dims() == ref.mps.bond_dims()
    out = []
    for k in range(steps):
        sg = mps.sweep(dt, m_max=m_max, eps=eps, zero_floor=floor)
        so = ref.step(dt)
        out.append((mps.populations(), otdvp.populations(ref.mps), mps.bond_dims(),
                    ref.mps.bond_dims(), sg, so))
    return mps, ref, out


def test_small_model_populations_match_oracle_every_step(P):
    m = vm.model_small_2state(n_modes=3, levels=4)
    _, _, out = _run_pair(P, m, 12, 0.5, 8)
    for pg, po, bg, bo, sg, so in out:
        assert bg == bo
        assert np.max(np.abs(pg - po)) < POP_TOL
        assert sg.noconv == 0


def test_two_state_four_mode_model_m16_parity(P):
    # 2 states + 4 modes x 8 levels (8192-dim), max bond 16, dt = 0.5 fs
    m = vm.model_small_2state()
    mps, ref, out = _run_pair(P, m, 16, 0.5, 16)
    for pg, po, bg, bo, sg, so in out:
        assert bg == bo
        assert np.max(np.abs(pg - po)) < POP_TOL
        assert sg.max_bond <= 16
        assert abs(sg.discarded_weight - so.discarded) < 1e-10
    # the gauge-invariant state itself agrees
    vg = otdvp.to_vector(otdvp.MPS(mps.tensors()))
    vo = otdvp.to_vector(ref.mps)
    assert abs(abs(np.vdot(vg, vo)) - 1.0) < 1e-9


def test_dbss_truncation_parity(P):
    m = vm.model_internal_conversion(seed=31, n_modes=5, level_range=(3, 6), n_offdiag=2, n_bilinear=4)
    _, _, out = _run_pair(P, m, 10, 0.5, 24, eps=1e-6)
    for pg, po, bg, bo, sg, so in out:
        assert bg == bo
        assert np.max(np.abs(pg - po)) < POP_TOL


def test_full_bond_gpu_2tdvp_is_exact(P):
    m = vm.model_small_2state(n_modes=3, levels=4)
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, idx, m_cap=64, pad_full=True)
    ex = vibronic.exact_propagate(m, vibronic.product_vector(m, idx), 0.5, 10)
    for k in range(10):
        mps.sweep(0.5, m_max=64, zero_floor=0.0)
        pe = vibronic.populations_from_vector(m, ex[k + 1])
        assert np.max(np.abs(mps.populations() - pe)) < 1e-9
    v = otdvp.to_vector(otdvp.MPS(mps.tensors()))
    assert np.linalg.norm(v - ex[-1]) < 1e-8


def test_independent_boson_closed_form_on_gpu(P):
    m = vm.model_independent_boson()
    dims = vm.local_dims(m)
    idx = vm.product_state_indices(m, 1)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, idx, m_cap=4)
    p0 = otdvp.product_mps(dims, idx)
    for k in range(20):
        mps.sweep(1.0, m_max=4)
        c = otdvp.overlap(p0, otdvp.MPS(mps.tensors()))
        ref = vibronic.independent_boson_autocorrelation(m, 1, (k + 1) * 1.0)
        assert abs(c - ref) < 1e-10
    assert mps.bond_dims() == [1] * (len(dims) - 1)


def test_sf_like_three_state_chain_parity(P):
    m = vm.model_singlet_fission(n_bath=3, levels=4)
    _, _, out = _run_pair(P, m, 6, 1.0, 12)
    for pg, po, bg, bo, sg, so in out:
        assert bg == bo
        assert np.max(np.abs(pg - po)) < POP_TOL


def test_sweep_rejects_bad_options(P):
    m = vm.model_small_2state(n_modes=2, levels=3)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, vm.product_state_indices(m), m_cap=4)
    with pytest.raises(P.VbError):
        mps.sweep(0.5, m_max=5)
    with pytest.raises(P.VbError):
        mps.sweep(0.5, m_max=4, krylov_max=100)
    with pytest.raises(P.VbError):
        P.Mps(mpo, [5, 0, 0], m_cap=4)
