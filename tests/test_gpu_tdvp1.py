"""One-site TDVP (tdvp1_sweep, Sec. 2.1.2 one-site variant) through the C ABI
against the oracle's Tdvp1: populations at fixed reduced bonds, exactness at
full bonds (also from a zero-padded product state, where the QR meets
dependent columns), norm and energy conservation, and the mixed form."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import vibmodels as vm
from oracle import mpo as ompo
from oracle import tdvp as otdvp
from oracle import vibronic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

POP_TOL = 1e-8
POP_TOL_MIXED = 1e-4


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


def _pair(P, m, ts, dtype, steps, dt=0.5):
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, m_cap=max(t.shape[2] for t in ts), dtype=dtype, tensors=ts)
    ref = otdvp.Tdvp1(otdvp.MPS(ts), ompo.build_mpo(m))
    out = []
    for _ in range(steps):
        st = mps.sweep1(dt)
        ref.step(dt)
        assert st.noconv == 0
        out.append((mps.populations(), otdvp.populations(ref.mps), mps.bond_dims(), ref.mps.bond_dims()))
    return mps, ref, out


def test_tdvp1_parity_reduced_bonds_fp64(P):
    m = vm.model_small_2state(n_modes=4, levels=6)
    ts = vm.random_right_canonical_mps(6, vm.local_dims(m), 5)
    mps, ref, out = _pair(P, m, ts, P.VB_FP64, 6)
    for pg, po, bg, bo in out:
        assert bg == bo == [2, 5, 5, 5]
        assert np.max(np.abs(pg - po)) < POP_TOL
    assert abs(mps.energy() - otdvp.energy(ref.mps, ompo.build_mpo(m))) < 1e-9


def test_tdvp1_conserves_energy_and_norm_on_gpu(P):
    m = vm.model_internal_conversion(seed=61, n_modes=5, level_range=(4, 8), n_offdiag=2, n_bilinear=4)
    ts = vm.random_right_canonical_mps(7, vm.local_dims(m), 12)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, m_cap=12, tensors=ts)
    e0, n0 = mps.energy(), mps.overlap(mps).real
    for _ in range(6):
        mps.sweep1(0.5)
        assert abs(mps.energy() - e0) < 1e-9 * max(1.0, abs(e0))
        assert abs(mps.overlap(mps).real - n0) < 1e-11


def test_tdvp1_full_bonds_exact(P):
    m = vm.model_small_2state(n_modes=3, levels=4)
    ts = vm.random_right_canonical_mps(5, vm.local_dims(m), 64)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, m_cap=64, tensors=ts)
    v = otdvp.to_vector(otdvp.MPS(ts))
    H = vibronic.hamiltonian_sparse(m)
    for _ in range(4):
        mps.sweep1(0.5)
        v = sla.expm_multiply(-1j * H * (0.5 / vm.HBAR_EV_FS), v)
        assert np.max(np.abs(otdvp.to_vector(otdvp.MPS(mps.tensors())) - v)) < 1e-9


def test_tdvp1_padded_product_state_full_bonds_exact(P):
    # zero-padded product state: the QR of every site meets dependent columns
    # and completes them; at full bonds the propagation is exact regardless
    m = vm.model_small_2state(n_modes=3, levels=4)
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, idx, m_cap=64, pad_full=True)
    v = otdvp.to_vector(otdvp.product_mps(dims, idx))
    H = vibronic.hamiltonian_sparse(m)
    for _ in range(4):
        mps.sweep1(0.5)
        v = sla.expm_multiply(-1j * H * (0.5 / vm.HBAR_EV_FS), v)
        assert np.max(np.abs(otdvp.to_vector(otdvp.MPS(mps.tensors())) - v)) < 1e-9


def test_tdvp1_mixed_form(P):
    m = vm.model_small_2state(n_modes=4, levels=6)
    ts = vm.random_right_canonical_mps(6, vm.local_dims(m), 5)
    _, _, out = _pair(P, m, ts, P.VB_MIXED, 6)
    for pg, po, bg, bo in out:
        assert bg == bo
        assert np.max(np.abs(pg - po)) < POP_TOL_MIXED
