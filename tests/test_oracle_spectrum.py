"""Pins of the oracle's spectrum (Sec. 3.1: Fourier transform of the damped
autocorrelation function) and of its energy functional.

Spectrum: in the independent-boson (displaced-oscillator) model the
autocorrelation is a Poisson-weighted sum of stationary phases,
C(t) = sum_n p_n exp(-i E_n t/hbar) with p_n = prod_I exp(-S_I) S_I^n_I / n_I!
and E_n = eps + sum_I w_I (1/2 - S_I + n_I). The trapezoidal sum of each phase
is a geometric series, so the discrete spectrum has a closed form that the
oracle's time-domain sum must reproduce to rounding; its continuous limit is
a sum of unit-area Lorentzians."""
import itertools
import math

import numpy as np

import vibmodels as vm
from oracle import mpo, spectrum, tdvp, vibronic

HBAR = vm.HBAR_EV_FS


def _poisson_lines(m, el_state, n_max=40):
    """(weights, energies) of the stationary states in C(t) of |el_state, 0>."""
    modes = []
    for I, w in enumerate(m["omega"]):
        g = m["g1"][I][el_state][el_state]
        S = g * g / (2.0 * w * w)
        ks = np.arange(n_max)
        p = np.array([math.exp(-S) * S ** k / math.factorial(k) for k in ks])
        e = w * (0.5 - S + ks)
        modes.append((p, e))
    ws, es = [], []
    for combo in itertools.product(*[range(n_max) for _ in modes]):
        p = 1.0
        e = m["e0"][el_state]
        for (pk, ek), k in zip(modes, combo):
            p *= pk[k]
            e += ek[k]
        if p > 1e-18:
            ws.append(p)
            es.append(e)
    return np.array(ws), np.array(es)


def _trapezoid_closed_form(ws, es, n_t, dt, tau, energies):
    out = np.zeros(len(energies))
    for j, E in enumerate(energies):
        z = np.exp((1j * (E - es) / HBAR - 1.0 / tau) * dt)
        geo = (1.0 - z ** n_t) / (1.0 - z)
        s = dt * (geo - 0.5 - 0.5 * z ** (n_t - 1))
        out[j] = float(np.real(np.sum(ws * s))) / (np.pi * HBAR)
    return out


def test_spectrum_equals_poisson_geometric_series_closed_form():
    m = vm.model_independent_boson(n_modes=2, s_max=0.3)
    ws, es = _poisson_lines(m, 1)
    assert abs(ws.sum() - 1.0) < 1e-12
    dt, n_t, tau = 0.5, 400, 40.0
    t = dt * np.arange(n_t)
    c = vibronic.independent_boson_autocorrelation(m, 1, t)
    E = np.linspace(es.min() - 0.2, es.max() + 0.2, 301)
    ref = _trapezoid_closed_form(ws, es, n_t, dt, tau, E)
    got = spectrum.spectrum(c, dt, tau, E)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))


def test_stationary_state_gives_unit_area_lorentzian():
    # continuous limit: fine steps, a record much longer than tau
    E0, tau, dt = 0.3, 20.0, 0.05
    t = dt * np.arange(int(400 / dt) + 1)
    c = np.exp(-1j * E0 * t / HBAR)
    gam = HBAR / tau
    E = np.linspace(E0 - 60 * gam, E0 + 60 * gam, 4001)
    got = spectrum.spectrum(c, dt, tau, E)
    lor = (gam / np.pi) / ((E - E0) ** 2 + gam ** 2)
    assert np.max(np.abs(got - lor)) < 2e-3 * lor.max()
    assert abs(E[np.argmax(got)] - E0) <= (E[1] - E[0])
    # the Lorentzian tails beyond +-60 half-widths hold 2 atan(1/60)/pi of the area
    area = np.trapezoid(got, E)
    assert abs(area - (1.0 - 2.0 * np.arctan(1.0 / 60.0) / np.pi)) < 2e-3


def test_spectrum_of_2tdvp_autocorrelation_matches_closed_form():
    # end to end on the oracle: C(t) from 2TDVP (mps overlap) -> spectrum
    m = vm.model_independent_boson(n_modes=2, levels=12, s_max=0.3)
    W = mpo.build_mpo(m)
    dims, ix = vm.local_dims(m), vm.product_state_indices(m, 0)
    p0 = tdvp.product_mps(dims, ix)
    sim = tdvp.Tdvp2(p0.copy(), W)
    dt, n_t, tau = 1.0, 120, 30.0
    c = [tdvp.overlap(p0, sim.mps)]
    for _ in range(n_t - 1):
        sim.step(dt)
        c.append(tdvp.overlap(p0, sim.mps))
    ws, es = _poisson_lines(m, 0)
    E = np.linspace(es.min() - 0.1, es.max() + 0.1, 151)
    ref = _trapezoid_closed_form(ws, es, n_t, dt, tau, E)
    got = spectrum.spectrum(np.array(c), dt, tau, E)
    # C(t) itself is exact to the Poisson tail of d = 12 levels and the Krylov tolerance
    assert np.max(np.abs(got - ref)) < 1e-8 * np.max(np.abs(ref))


def test_energy_equals_dense_expectation_value():
    # <psi|H|psi>/<psi|psi> from the MPO sandwich against the term-list
    # Hamiltonian; with and without zero-point energy, unnormalised states,
    # electronic site first and inside the chain
    for seed, zpe, order in ((5, 1, None), (6, 0, None), (7, 1, [1, -1, 0, 2])):
        m = vm.model_internal_conversion(seed=seed, n_modes=3, level_range=(3, 5), n_offdiag=2, n_bilinear=2)
        m["include_zpe"] = zpe
        m["site_order"] = order
        dims = vm.local_dims(m)
        ts = vm.random_right_canonical_mps(seed, dims, 6)
        ts[0] = ts[0] * 1.7
        psi = tdvp.MPS(ts)
        v = tdvp.to_vector(psi)
        H = vibronic.hamiltonian_sparse(m)
        ref = float(np.real(np.vdot(v, H @ v) / np.vdot(v, v)))
        got = tdvp.energy(psi, mpo.build_mpo(m))
        assert abs(got - ref) < 1e-12 * max(1.0, abs(ref))
