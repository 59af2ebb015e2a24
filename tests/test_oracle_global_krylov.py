"""Pins of the oracle's global Krylov step (Sec. 2.1.2, Eqs. Krylov subspace
and global Krylov) and its parts (Sec. 2.1.1: direct MPO application,
compression, sums) against dense-vector mathematics: the dense Hamiltonian,
the SVD's optimal truncation (Eckart-Young), exact propagation, the
independent-boson closed form; and the pre-steps' purpose (Sec. 2.1.2, one-
site TDVP paragraph): bonds grown by global steps let one-site TDVP follow
the exact dynamics that it misses from a product state."""
import numpy as np
import pytest

import vibmodels as vm
from oracle import global_krylov as gk
from oracle import mpo as ompo
from oracle import tdvp as otdvp
from oracle import vibronic

FULL = otdvp.TdvpOptions(zero_floor=0.0)


def _model():
    return vm.model_small_2state(n_modes=3, levels=4)


def _random_mps(seed, dims, m):
    return otdvp.MPS(vm.random_right_canonical_mps(seed, dims, m))


def test_direct_mpo_application_is_h_times_psi():
    m = vm.model_internal_conversion(seed=71, n_modes=3, level_range=(3, 4), n_offdiag=2, n_bilinear=2)
    dims = vm.local_dims(m)
    psi = _random_mps(72, dims, 6)
    H = vibronic.hamiltonian_sparse(m)
    out = gk.apply_mpo(ompo.build_mpo(m), psi)
    v, hv = otdvp.to_vector(out), H @ otdvp.to_vector(psi)
    assert np.linalg.norm(v - hv) <= 1e-12 * np.linalg.norm(hv)
    w = [ompo.build_mpo(m)[p].shape[3] for p in range(len(dims) - 1)]
    assert out.bond_dims() == [a * b for a, b in zip(w, psi.bond_dims())]


def test_compression_without_truncation_is_exact_and_right_canonical():
    m = _model()
    dims = vm.local_dims(m)
    x = gk.apply_mpo(ompo.build_mpo(m), _random_mps(73, dims, 8))
    y, disc = gk.compress(x, FULL)
    assert disc < 1e-14
    assert np.linalg.norm(otdvp.to_vector(y) - otdvp.to_vector(x)) <= 1e-12 * np.linalg.norm(otdvp.to_vector(x))
    for B in y.A[1:]:
        Bm = B.reshape(B.shape[0], -1)
        assert np.max(np.abs(Bm @ np.conj(Bm.T) - np.eye(B.shape[0]))) < 1e-12


@pytest.mark.parametrize("k", [1, 3, 6])
def test_compression_is_the_optimal_truncation_on_two_sites(k):
    # two sites: the kept state must be the best rank-k approximation
    rng = np.random.Generator(np.random.PCG64(74 + k))
    V = vm.random_complex(rng, (7, 9))
    U, s, Vh = np.linalg.svd(V, full_matrices=False)
    x = otdvp.MPS([(U * s).reshape(1, 7, 7), Vh.reshape(7, 9, 1)])
    y, disc = gk.compress(x, otdvp.TdvpOptions(m_max=k, zero_floor=0.0))
    best = (U[:, :k] * s[:k]) @ Vh[:k]
    assert np.linalg.norm(otdvp.to_vector(y) - best.reshape(-1)) < 1e-12 * np.linalg.norm(best)
    assert disc == pytest.approx(float(np.sum(s[k:] ** 2) / np.sum(s ** 2)), rel=1e-10)


def test_mps_sum_and_matrix_element():
    m = _model()
    dims = vm.local_dims(m)
    a, b, c = (_random_mps(s, dims, mm) for s, mm in ((75, 4), (76, 8), (77, 2)))
    coefs = [0.3 - 0.2j, -1.1, 0.5j]
    ssum = gk.mps_sum(coefs, [a, b, c])
    ref = sum(cc * otdvp.to_vector(x) for cc, x in zip(coefs, [a, b, c]))
    assert np.linalg.norm(otdvp.to_vector(ssum) - ref) < 1e-12 * np.linalg.norm(ref)
    H = vibronic.hamiltonian_sparse(m)
    val = gk.expect_between(a, ompo.build_mpo(m), b)
    dense = np.vdot(otdvp.to_vector(a), H @ otdvp.to_vector(b))
    assert abs(val - dense) < 1e-12 * max(1.0, abs(dense))


def test_global_krylov_at_full_bonds_is_exact_propagation():
    m = _model()
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)
    W = ompo.build_mpo(m)
    ex = vibronic.exact_propagate(m, vibronic.product_vector(m, idx), 0.5, 4)
    cur = otdvp.product_mps(dims, idx)
    for k in range(4):
        cur, info = gk.global_krylov_step(cur, W, 0.5, FULL)
        assert info["converged"]
        v = otdvp.to_vector(cur)
        assert np.linalg.norm(v - ex[k + 1]) < 1e-9
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12


def test_global_krylov_independent_boson_closed_form():
    m = vm.model_independent_boson()
    dims, idx = vm.local_dims(m), vm.product_state_indices(m, 1)
    W = ompo.build_mpo(m)
    psi0 = otdvp.product_mps(dims, idx)
    cur = psi0
    for k in range(4):
        cur, _ = gk.global_krylov_step(cur, W, 1.0, otdvp.TdvpOptions())
        ref = vibronic.independent_boson_autocorrelation(m, 1, (k + 1) * 1.0)
        assert abs(otdvp.overlap(psi0, cur) - ref) < 1e-9


def test_truncated_global_krylov_converges_with_the_bond_cap():
    m = _model()
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)
    W = ompo.build_mpo(m)
    ex = vibronic.exact_propagate(m, vibronic.product_vector(m, idx), 0.5, 3)
    errs = []
    for cap in (2, 4, 8):
        cur = otdvp.product_mps(dims, idx)
        for _ in range(3):
            cur, _ = gk.global_krylov_step(cur, W, 0.5, otdvp.TdvpOptions(m_max=cap, zero_floor=0.0))
            assert max(cur.bond_dims()) <= cap
            assert abs(np.linalg.norm(otdvp.to_vector(cur)) - 1.0) < 1e-12
        errs.append(np.linalg.norm(otdvp.to_vector(cur) - ex[-1]))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9


def test_presteps_let_one_site_tdvp_follow_the_exact_dynamics():
    m = _model()
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)
    W = ompo.build_mpo(m)
    ex = vibronic.exact_propagate(m, vibronic.product_vector(m, idx), 0.5, 6)
    pe = [vibronic.populations_from_vector(m, v) for v in ex]
    # one-site TDVP alone keeps the product state's bond 1 (mean-field motion)
    alone = otdvp.Tdvp1(otdvp.product_mps(dims, idx), W, FULL)
    for _ in range(6):
        alone.step(0.5)
    err_alone = np.max(np.abs(otdvp.populations(alone.mps) - pe[6]))
    states = gk.prestep_then_tdvp1(otdvp.product_mps(dims, idx), W, 0.5, 2, 4, FULL)
    assert states[1].bond_dims() == [2, 8, 4]  # full bonds after the pre-steps
    err = max(np.max(np.abs(otdvp.populations(s) - pe[k + 1])) for k, s in enumerate(states))
    assert err_alone > 1e-4  # about 9e-4 after 3 fs
    assert err < 1e-9
