"""Pins of the oracle's population gradient dP_k(t)/dg^I_ij (the target of a
differentiable propagation; model of Sec. 2.2, populations of Sec. 3.1):
the eigenbasis Duhamel formula against central finite differences of exact
propagation; invariants (the gradients of the populations sum to zero, vanish
at t = 0 and in the independent-boson model, whose populations no diagonal
coupling can move); and finite differences of the oracle's full-bond 2TDVP,
which must reach the same exact gradient."""
import numpy as np

import vibmodels as vm
from oracle import gradient as og
from oracle import mpo as ompo
from oracle import tdvp as otdvp
from oracle import vibronic


def _setup():
    m = vm.model_small_2state(n_modes=3, levels=4)
    psi0 = vibronic.product_vector(m, vm.product_state_indices(m))
    # every diagonal linear coupling, and one off-diagonal (vibronic) one
    params = [(I, s, s) for I in range(3) for s in (0, 1)] + [(1, 0, 1)]
    return m, psi0, params


def test_duhamel_gradient_matches_finite_differences_of_exact_propagation():
    m, psi0, params = _setup()
    for t in (3.0, 10.0):
        g = og.population_gradient(m, psi0, t, params)
        fd = og.population_gradient_fd(m, psi0, t, params, h=1e-5)
        assert np.max(np.abs(g - fd)) < 1e-7
        assert np.max(np.abs(g)) > 1e-2  # a nontrivial gradient


def test_gradient_invariants():
    m, psi0, params = _setup()
    g = og.population_gradient(m, psi0, 10.0, params)
    assert np.max(np.abs(g.sum(axis=1))) < 1e-12  # sum_k P_k = 1 for every g
    assert np.max(np.abs(og.population_gradient(m, psi0, 0.0, params))) == 0.0
    # V = 0 and diagonal couplings: every population is conserved for any g
    mb = vm.model_independent_boson(n_modes=2, levels=6)
    pb = vibronic.product_vector(mb, vm.product_state_indices(mb, 1))
    gb = og.population_gradient(mb, pb, 7.0, [(I, s, s) for I in range(2) for s in range(2)])
    assert np.max(np.abs(gb)) < 1e-12


def test_finite_differences_of_full_bond_2tdvp_reach_the_exact_gradient():
    m, psi0, params = _setup()
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)

    def propagate(mm):
        sim = otdvp.Tdvp2(otdvp.padded_product_mps(dims, idx, 64), ompo.build_mpo(mm),
                          otdvp.TdvpOptions(m_max=64, zero_floor=0.0))
        for _ in range(10):
            sim.step(0.5)
        return otdvp.populations(sim.mps)

    g = og.population_gradient(m, psi0, 5.0, params[:6])
    fd = og.population_gradient_fd(m, psi0, 5.0, params[:6], h=1e-5, propagate=propagate)
    assert np.max(np.abs(g - fd)) < 1e-8
