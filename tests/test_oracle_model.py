"""Pins of the oracle's Hamiltonian and MPO (Sec. 2.2, Eq. MPO)."""
import json
import os

import numpy as np
import pytest

import vibmodels as vm
from oracle import mpo, vibronic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_models():
    ic = vm.model_internal_conversion(n_modes=4, level_range=(3, 4), n_offdiag=2, n_bilinear=3)
    sf = vm.model_singlet_fission(n_bath=2, levels=3)
    c1 = vm.model_small_2state(n_modes=3, levels=4)
    moved = vm.model_small_2state(n_modes=3, levels=3)
    moved["site_order"] = [0, -1, 2, 1]
    return [c1, ic, sf, vm.model_nn_chain(), moved]


@pytest.mark.parametrize("k", range(5))
def test_mpo_contracts_to_term_list_hamiltonian(k):
    m = _small_models()[k]
    W = mpo.build_mpo(m)
    Hd = mpo.mpo_to_dense(W)
    Hs = vibronic.hamiltonian_sparse(m).toarray()
    assert Hd.shape == Hs.shape
    assert np.max(np.abs(Hd - Hs)) < 1e-13
    assert np.max(np.abs(Hs - Hs.T)) == 0.0


def test_uncoupled_spectrum_is_harmonic_ladder():
    # V = 0 and g = 0: eigenvalues are eps_i + sum_I omega_I (n_I + 1/2)
    m = vm.model_small_2state(n_modes=2, levels=3)
    m["v0"][:] = 0.0
    m["g1"][:] = 0.0
    H = vibronic.hamiltonian_sparse(m).toarray()
    ev = np.sort(np.linalg.eigvalsh(H))
    ref = []
    for e in m["e0"]:
        for n1 in range(3):
            for n2 in range(3):
                ref.append(e + m["omega"][0] * (n1 + 0.5) + m["omega"][1] * (n2 + 0.5))
    assert np.allclose(ev, np.sort(ref), atol=1e-13)


def test_boson_operators_textbook():
    d = 6
    b = vibronic.boson_b(d)
    n = vibronic.boson_n(d)
    # [b, b^+] = 1 except at the truncation edge
    comm = b @ b.T - b.T @ b
    assert np.allclose(np.diag(comm)[:-1], 1.0)
    assert np.allclose(b.T @ b, n)
    q = vibronic.boson_q(d)
    # <n|q^2|n> = n + 1/2 below the edge
    assert np.allclose(np.diag(q @ q)[:-1], np.arange(d - 1) + 0.5)


def test_mpo_bond_dimension_small():
    # electronic-first ordering: channels start/done/E_ij, no bilinear terms
    W = mpo.build_mpo(vm.model_small_2state())
    assert mpo.mpo_bond_dims(W) == [4, 4, 4, 4]


def test_debye_reorganisation_energy_riemann_limit():
    # sum_I g_I^2 / (2 omega_I) -> lam (2/pi) atan(omega_max / omega_c)
    lam, wc, wmax = 0.05, 0.1, 0.4
    ref = lam * (2.0 / np.pi) * np.arctan(wmax / wc)
    errs = []
    for n in (100, 400, 1600):
        w, g = vm.debye_couplings(n, lam, wc, wmax)
        errs.append(abs(np.sum(g * g / (2.0 * w)) - ref))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-3 * ref


def test_paper_constants():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        g = json.load(f)
    t = g["time_step_au_to_fs"]
    assert abs(t["dt_au"] * vm.AU_TIME_FS - t["dt_fs_approx"]) < t["rel_tol"] * t["dt_fs_approx"]
    sf = vm.model_singlet_fission(n_bath=1)
    assert np.allclose(sf["e0"], np.diag(g["sf_electronic_hamiltonian_eV"]["matrix"]))
    assert sf["v0"][0, 1] == 0.0 and sf["v0"][0, 2] < 0 and sf["v0"][1, 2] < 0
