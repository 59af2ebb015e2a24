"""Whole-state observables and the batched sweep through the C ABI:
mps_overlap (the autocorrelation C(t) of Sec. 3.1) and mps_energy against the
oracle and the independent-boson closed form, energy conservation of full-bond
2TDVP, tdvp2_sweep_batched against one-by-one sweeps, and the checkpoint
round trip."""
import numpy as np
import pytest

import vibmodels as vm
from oracle import mpo as ompo
from oracle import tdvp as otdvp
from oracle import vibronic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


def test_overlap_matches_oracle(P):
    m = vm.model_internal_conversion(seed=51, n_modes=4, level_range=(3, 6), n_offdiag=2, n_bilinear=3)
    dims = vm.local_dims(m)
    ta = vm.random_right_canonical_mps(11, dims, 12)
    tb = vm.random_right_canonical_mps(12, dims, 9)
    mpo = P.Mpo(m)
    a, b = P.Mps(mpo, m_cap=12, tensors=ta), P.Mps(mpo, m_cap=12, tensors=tb)
    ref_ab = otdvp.overlap(otdvp.MPS(ta), otdvp.MPS(tb))
    ref_aa = otdvp.overlap(otdvp.MPS(ta), otdvp.MPS(ta))
    assert abs(a.overlap(b) - ref_ab) < 1e-12 * max(1.0, abs(ref_ab))
    assert abs(b.overlap(a) - np.conj(ref_ab)) < 1e-12 * max(1.0, abs(ref_ab))
    assert abs(a.overlap(a) - ref_aa) < 1e-12 * abs(ref_aa)


def test_autocorrelation_independent_boson_closed_form(P):
    m = vm.model_independent_boson()
    idx = vm.product_state_indices(m, 1)
    mpo = P.Mpo(m)
    psi0 = P.Mps(mpo, idx, m_cap=4)
    psi = P.Mps(mpo, idx, m_cap=4)
    for k in range(12):
        psi.sweep(1.0, m_max=4)
        ref = vibronic.independent_boson_autocorrelation(m, 1, (k + 1) * 1.0)
        assert abs(psi0.overlap(psi) - ref) < 1e-10


def test_energy_matches_oracle_and_is_conserved_at_full_bonds(P):
    m = vm.model_small_2state(n_modes=3, levels=4)
    dims = vm.local_dims(m)
    ts = vm.random_right_canonical_mps(21, dims, 64)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, m_cap=64, tensors=ts)
    e_ref = otdvp.energy(otdvp.MPS(ts), ompo.build_mpo(m))
    e0 = mps.energy()
    assert abs(e0 - e_ref) < 1e-11 * max(1.0, abs(e_ref))
    for _ in range(5):
        mps.sweep(0.5, m_max=64, zero_floor=0.0)
        assert abs(mps.energy() - e0) < 1e-9 * max(1.0, abs(e0))


def test_batched_sweep_equals_one_by_one(P):
    models = [vm.model_small_2state(seed=1001 + i, n_modes=3, levels=5) for i in range(3)]
    streams = [torch.cuda.Stream() for _ in models]
    runs = []
    for batched in (False, True):
        states = []
        for m, s in zip(models, streams):
            states.append(P.Mps(P.Mpo(m), vm.product_state_indices(m), m_cap=16, stream=s))
        for _ in range(4):
            if batched:
                stats = P.sweep_batched(states, 0.5, m_max=16)
                assert len(stats) == len(states) and all(st.noconv == 0 for st in stats)
            else:
                for st in states:
                    st.sweep(0.5, m_max=16)
        torch.cuda.synchronize()
        runs.append([(st.populations(), st.bond_dims()) for st in states])
    for (p1, b1), (p2, b2) in zip(*runs):
        assert b1 == b2
        assert np.max(np.abs(p1 - p2)) < 1e-13


def test_batched_sweep_rejects_duplicates(P):
    m = vm.model_small_2state(n_modes=2, levels=3)
    mps = P.Mps(P.Mpo(m), vm.product_state_indices(m), m_cap=4)
    with pytest.raises(P.VbError):
        P.sweep_batched([mps, mps], 0.5, m_max=4)


def test_checkpoint_round_trip(P, tmp_path):
    m = vm.model_small_2state(n_modes=3, levels=5)
    mpo = P.Mpo(m)
    a = P.Mps(mpo, vm.product_state_indices(m), m_cap=16)
    for _ in range(3):
        a.sweep(0.5, m_max=16)
    path = str(tmp_path / "state.npz")
    a.save(path)
    b = P.Mps.load(mpo, path, m_cap=16)
    assert b.bond_dims() == a.bond_dims()
    assert abs(a.overlap(b) - 1.0) < 1e-12
    for _ in range(3):
        a.sweep(0.5, m_max=16)
        b.sweep(0.5, m_max=16)
    assert np.max(np.abs(a.populations() - b.populations())) < 1e-13
