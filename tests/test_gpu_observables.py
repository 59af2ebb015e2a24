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


def test_spectrum_of_gpu_autocorrelation(P):
    # Sec. 3.1 spectra: C(t) from GPU 2TDVP (mps_overlap after every step)
    # Fourier transformed with damping on the GPU (vb_spectrum), against the
    # oracle's transform of the same samples and the Poisson closed form of
    # the independent-boson model (tests/test_oracle_spectrum.py)
    from oracle import spectrum as ospec
    from test_oracle_spectrum import _poisson_lines, _trapezoid_closed_form
    m = vm.model_independent_boson(n_modes=2, levels=12, s_max=0.3)
    idx = vm.product_state_indices(m, 0)
    mpo = P.Mpo(m)
    psi0 = P.Mps(mpo, idx, m_cap=4)
    psi = P.Mps(mpo, idx, m_cap=4)
    dt, n_t, tau = 1.0, 120, 30.0
    c = [psi0.overlap(psi)]
    for _ in range(n_t - 1):
        psi.sweep(dt, m_max=4)
        c.append(psi0.overlap(psi))
    c = np.array(c)
    ws, es = _poisson_lines(m, 0)
    E = np.linspace(es.min() - 0.1, es.max() + 0.1, 151)
    c_d = torch.from_numpy(c).cuda()
    E_d = torch.from_numpy(E).cuda()
    out = torch.zeros(E.size, dtype=torch.float64, device="cuda")
    P.vb_spectrum(c_d, n_t, dt, tau, E_d, E.size, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    same = ospec.spectrum(c, dt, tau, E)
    assert np.max(np.abs(got - same)) < 1e-12 * np.max(np.abs(same))
    ref = _trapezoid_closed_form(ws, es, n_t, dt, tau, E)
    assert np.max(np.abs(got - ref)) < 1e-8 * np.max(np.abs(ref))


def test_batch_configuration_instances_match_the_oracle(P):
    # the batched coupling scan (64 uneven two-state models, couplings scaled
    # 0.5..2x, per-instance bond caps): the four 8-mode instances run together
    # through tdvp2_sweep_batched (one stream each, one shared call with the
    # largest cap, each instance capped at its own m_cap) and match the oracle
    # with each instance's own cap
    batch = vm.batch_models(seed=1004, n=64)
    pick = [i for i, (m, _) in enumerate(batch) if len(m["omega"]) == 8][:4]
    assert len(pick) == 4
    streams = [torch.cuda.Stream() for _ in pick]
    states, refs = [], []
    for i, s in zip(pick, streams):
        m, mm = batch[i]
        idx = vm.product_state_indices(m)
        states.append(P.Mps(P.Mpo(m), idx, m_cap=mm, stream=s))
        refs.append(otdvp.Tdvp2(otdvp.product_mps(vm.local_dims(m), idx), ompo.build_mpo(m),
                                otdvp.TdvpOptions(m_max=mm)))
    for _ in range(6):
        stats = P.sweep_batched(states, 0.5, m_max=max(batch[i][1] for i in pick))
        assert all(st.noconv == 0 for st in stats)
        for r in refs:
            r.step(0.5)
    for q, r in zip(states, refs):
        assert np.max(np.abs(q.populations() - otdvp.populations(r.mps))) < 1e-8
        assert q.bond_dims() == r.mps.bond_dims()
