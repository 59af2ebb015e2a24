"""Pins of the oracle's 2TDVP time stepping (Sec. 2.1.2) against exact
state-vector propagation, closed forms and conservation laws."""
import numpy as np
import pytest

import vibmodels as vm
from oracle import mpo, tdvp, vibronic


def test_full_bond_2tdvp_is_exact_small_chain():
    # with complete bond bases the tangent-space projector is the identity
    m = vm.model_small_2state(n_modes=3, levels=4)
    W = mpo.build_mpo(m)
    dims, ix = vm.local_dims(m), vm.product_state_indices(m)
    sim = tdvp.Tdvp2(tdvp.padded_product_mps(dims, ix), W, tdvp.TdvpOptions(zero_floor=0.0))
    psi0 = vibronic.product_vector(m, ix)
    ex = vibronic.exact_propagate(m, psi0, 0.5, 12)
    for k in range(12):
        sim.step(0.5)
    v = tdvp.to_vector(sim.mps)
    assert np.linalg.norm(v - ex[-1]) < 1e-9
    assert np.allclose(tdvp.populations(sim.mps), vibronic.populations_from_vector(m, ex[-1]), atol=1e-11)


@pytest.mark.slow
def test_full_bond_2tdvp_is_exact_8192_dim_model():
    # 2 states + 4 modes x 8 levels (8192-dim), padded to full bonds [2,16,64,8]
    m = vm.model_small_2state()
    W = mpo.build_mpo(m)
    dims, ix = vm.local_dims(m), vm.product_state_indices(m)
    sim = tdvp.Tdvp2(tdvp.padded_product_mps(dims, ix), W, tdvp.TdvpOptions(zero_floor=0.0))
    assert sim.mps.bond_dims() == [2, 16, 64, 8]
    psi0 = vibronic.product_vector(m, ix)
    ex = vibronic.exact_propagate(m, psi0, 0.5, 8)
    for k in range(8):
        sim.step(0.5)
        pe = vibronic.populations_from_vector(m, ex[k + 1])
        assert np.allclose(tdvp.populations(sim.mps), pe, atol=1e-9)
    assert np.linalg.norm(tdvp.to_vector(sim.mps) - ex[-1]) < 1e-7


@pytest.mark.parametrize("el_state", [0, 1])
def test_independent_boson_autocorrelation_closed_form(el_state):
    m = vm.model_independent_boson()
    W = mpo.build_mpo(m)
    dims, ix = vm.local_dims(m), vm.product_state_indices(m, el_state)
    p0 = tdvp.product_mps(dims, ix)
    sim = tdvp.Tdvp2(p0.copy(), W)
    for k in range(30):
        sim.step(1.0)
        c = tdvp.overlap(p0, sim.mps)
        ref = vibronic.independent_boson_autocorrelation(m, el_state, sim.time)
        assert abs(c - ref) < 1e-10
        pops = tdvp.populations(sim.mps)
        assert abs(pops[el_state] - 1.0) < 1e-12
    assert sim.mps.bond_dims() == [1] * (len(dims) - 1)


def _nn_error(m, dt, T, floor):
    W = mpo.build_mpo(m)
    d, ix = vm.local_dims(m), vm.product_state_indices(m)
    n = int(round(T / dt))
    sim = tdvp.Tdvp2(tdvp.product_mps(d, ix), W, tdvp.TdvpOptions(zero_floor=floor))
    for k in range(n):
        sim.step(dt)
    ex = vibronic.exact_propagate(m, vibronic.product_vector(m, ix), dt, n)[-1]
    full = [2, 6, 18, 9, 3]
    return np.linalg.norm(tdvp.to_vector(sim.mps) - ex), sim.mps.bond_dims(), full


def test_nearest_neighbour_chain_has_no_projection_error():
    # Sec. 2.1.2: 2TDVP evolves nearest-neighbour Hamiltonians without a
    # projection error, even with bonds below their full size
    nn = vm.model_nn_chain(n_modes=5, levels=3)
    lr = vm.model_nn_chain(n_modes=5, levels=3)
    lr["g1"][4, 0, 0], lr["g1"][4, 1, 1] = 0.06, -0.06  # electron - last mode: long range
    for dt in (1.0, 0.5):
        e_nn, bonds, full = _nn_error(nn, dt, 8.0, 1e-18)
        e_lr, _, _ = _nn_error(lr, dt, 8.0, 1e-18)
        assert e_nn < 5e-8
        assert any(b < f for b, f in zip(bonds, full))
        assert e_lr > 1e-3


def test_norm_and_energy_conserved_without_truncation():
    m = vm.model_small_2state(n_modes=3, levels=4)
    W = mpo.build_mpo(m)
    dims, ix = vm.local_dims(m), vm.product_state_indices(m)
    sim = tdvp.Tdvp2(tdvp.padded_product_mps(dims, ix), W, tdvp.TdvpOptions(zero_floor=0.0))
    e0 = tdvp.energy(sim.mps, W)
    for k in range(20):
        sim.step(1.0)
    assert abs(np.linalg.norm(tdvp.to_vector(sim.mps)) - 1.0) < 1e-12
    assert abs(tdvp.energy(sim.mps, W) - e0) < 1e-10


def test_capped_run_populations_physical_and_bonds_bounded():
    m = vm.model_small_2state()
    W = mpo.build_mpo(m)
    dims, ix = vm.local_dims(m), vm.product_state_indices(m)
    sim = tdvp.Tdvp2(tdvp.product_mps(dims, ix), W, tdvp.TdvpOptions(m_max=8))
    for k in range(10):
        st = sim.step(0.5)
        p = tdvp.populations(sim.mps)
        assert abs(p.sum() - 1.0) < 1e-12 and np.all(p >= -1e-15)
        assert st.max_bond <= 8 and st.noconv == 0
    assert max(sim.mps.bond_dims()) >= 4
