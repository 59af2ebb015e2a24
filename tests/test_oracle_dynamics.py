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


# ---- one-site TDVP (Sec. 2.1.2, the one-site variant)
def test_full_bond_1tdvp_is_exact():
    # at full bond dimensions the tangent-space projector is the identity and
    # the one-site projector-splitting step reproduces exact propagation
    import scipy.sparse.linalg as sla
    m = vm.model_small_2state(n_modes=3, levels=4)
    dims = vm.local_dims(m)
    ts = vm.random_right_canonical_mps(5, dims, 64)
    W = mpo.build_mpo(m)
    st = tdvp.Tdvp1(tdvp.MPS(ts), W)
    v = tdvp.to_vector(tdvp.MPS(ts))
    H = vibronic.hamiltonian_sparse(m)
    for _ in range(6):
        st.step(0.5)
        v = sla.expm_multiply(-1j * H * (0.5 / vm.HBAR_EV_FS), v)
        assert np.max(np.abs(tdvp.to_vector(st.mps) - v)) < 1e-9
    assert st.mps.bond_dims() == [2, 8, 4]


def test_1tdvp_conserves_norm_and_energy_at_reduced_bonds():
    # fixed bond dimensions below full: the state leaves the exact
    # trajectory, but 1TDVP conserves norm and energy (no truncation)
    m = vm.model_small_2state(n_modes=4, levels=6)
    dims = vm.local_dims(m)
    ts = vm.random_right_canonical_mps(6, dims, 5)
    W = mpo.build_mpo(m)
    st = tdvp.Tdvp1(tdvp.MPS(ts), W)
    e0, n0 = tdvp.energy(st.mps, W), tdvp.overlap(st.mps, st.mps)
    v = tdvp.to_vector(tdvp.MPS(ts))
    H = vibronic.hamiltonian_sparse(m)
    import scipy.sparse.linalg as sla
    for _ in range(6):
        st.step(0.5)
        v = sla.expm_multiply(-1j * H * (0.5 / vm.HBAR_EV_FS), v)
        assert abs(tdvp.energy(st.mps, W) - e0) < 1e-10 * max(1.0, abs(e0))
        assert abs(tdvp.overlap(st.mps, st.mps) - n0) < 1e-12
    assert st.mps.bond_dims() == [2, 5, 5, 5]
    # and the projection error is real at these bonds
    assert np.max(np.abs(tdvp.to_vector(st.mps) - v)) > 1e-6


def test_heff0_is_the_bond_projection_of_h():
    # <X'|H_eff,0|X> equals <psi(X')|H|psi(X)> for states that share the
    # orthonormal tensors left and right of the bond
    m = vm.model_small_2state(n_modes=3, levels=3)
    dims = vm.local_dims(m)
    ts = vm.random_right_canonical_mps(9, dims, 64)
    W = mpo.build_mpo(m)
    H = vibronic.hamiltonian_sparse(m).toarray()
    rng = np.random.default_rng(3)
    # left-orthonormal A_0, A_1 from QR, right-orthonormal B_2, B_3 as given
    A = [np.array(t) for t in ts]
    for i in range(2):
        mL, d, mR = A[i].shape
        Q, Rm = np.linalg.qr(A[i].reshape(mL * d, mR))
        A[i] = Q.reshape(mL, d, mR)
        A[i + 1] = np.einsum("ab,bsc->asc", Rm, A[i + 1])
    mb = A[1].shape[2]
    Lb = np.ones((1, 1, 1), dtype=np.complex128)
    for i in range(2):
        Lb = tdvp.env_left_update(Lb, A[i], W[i])
    Rb = np.ones((1, 1, 1), dtype=np.complex128)
    for i in range(3, 1, -1):
        Rb = tdvp.env_right_update(Rb, A[i], W[i])
    X = rng.standard_normal((mb, mb)) + 1j * rng.standard_normal((mb, mb))
    Y = rng.standard_normal((mb, mb)) + 1j * rng.standard_normal((mb, mb))

    def vec(Z):
        B = [A[0], np.einsum("asb,bc->asc", A[1], Z), A[2], A[3]]
        return tdvp.to_vector(tdvp.MPS(B))
    lhs = np.vdot(Y, tdvp.heff0_apply(Lb, Rb, X))
    rhs = np.vdot(vec(Y), H @ vec(X))
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)
