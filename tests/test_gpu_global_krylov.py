"""Global Krylov steps on the GPU (global_krylov_step: direct MPO application,
compression, MPS sums, Krylov-ordered Gram orthonormalisation, Sec. 2.1.1 /
2.1.2) against the oracle (oracle/global_krylov.py, pinned to dense vectors
and exact propagation) and against exact propagation; pre-steps followed by
GPU one-site TDVP."""
import numpy as np
import pytest

import vibmodels as vm
from oracle import global_krylov as gk
from oracle import mpo as ompo
from oracle import tdvp as otdvp
from oracle import vibronic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FULL = dict(zero_floor=0.0)


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


def _model():
    return vm.model_small_2state(n_modes=3, levels=4)


def _vector(mps):
    return otdvp.to_vector(otdvp.MPS(mps.tensors()))


def test_full_bond_global_krylov_is_exact_propagation(P):
    m = _model()
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)
    ex = vibronic.exact_propagate(m, vibronic.product_vector(m, idx), 0.5, 4)
    mps = P.Mps(P.Mpo(m), idx, m_cap=64)
    for k in range(4):
        inf = mps.global_krylov(0.5, 64, **FULL)
        assert inf.converged == 1
        v = _vector(mps)
        assert np.linalg.norm(v - ex[k + 1]) < 1e-9
    # at most the full bonds; Schmidt weights below ~1e-16 of the total are not
    # resolved by the Gram-matrix compression (rho = M^+ G M squares them), so
    # a bond may stop short of full where the exact state's weights are that small
    assert all(b <= f for b, f in zip(mps.bond_dims(), [2, 8, 4]))


def test_truncated_global_krylov_matches_the_oracle(P):
    # bond cap 4 < full: every compression truncates with the 2TDVP rule
    m = vm.model_internal_conversion(seed=71, n_modes=3, level_range=(3, 4), n_offdiag=2, n_bilinear=2)
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)
    W = ompo.build_mpo(m)
    cur = otdvp.product_mps(dims, idx)
    mps = P.Mps(P.Mpo(m), idx, m_cap=8)
    for _ in range(3):
        cur, info = gk.global_krylov_step(cur, W, 0.5, otdvp.TdvpOptions(m_max=4, zero_floor=0.0))
        inf = mps.global_krylov(0.5, 4, zero_floor=0.0)
        assert inf.r == info["r"]
        assert mps.bond_dims() == cur.bond_dims()
        a, b = _vector(mps), otdvp.to_vector(cur)
        assert abs(abs(np.vdot(a, b)) - 1.0) < 1e-10  # same state up to a phase
        assert np.max(np.abs(mps.populations() - otdvp.populations(cur))) < 1e-10
        # the discarded weight (~1e-9 here) through rho = M^+ G M: absolute
        # accuracy ~1e-16 times the conditioning of the basis' Gram matrices
        assert abs(inf.disc_final - info["disc_final"]) < 1e-12


def test_independent_boson_closed_form(P):
    m = vm.model_independent_boson()
    idx = vm.product_state_indices(m, 1)
    mpo = P.Mpo(m)
    psi0 = P.Mps(mpo, idx, m_cap=8)
    mps = P.Mps(mpo, idx, m_cap=8)
    for k in range(4):
        mps.global_krylov(1.0, 8)
        ref = vibronic.independent_boson_autocorrelation(m, 1, (k + 1) * 1.0)
        assert abs(psi0.overlap(mps) - ref) < 1e-9


def test_presteps_then_one_site_tdvp_follow_exact_dynamics(P):
    m = _model()
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)
    ex = vibronic.exact_propagate(m, vibronic.product_vector(m, idx), 0.5, 6)
    pe = [vibronic.populations_from_vector(m, v) for v in ex]
    mps = P.Mps(P.Mpo(m), idx, m_cap=64)
    errs = []
    for k in range(2):
        mps.global_krylov(0.5, 64, **FULL)
        errs.append(np.max(np.abs(mps.populations() - pe[k + 1])))
    assert mps.bond_dims() == [2, 8, 4]  # full bonds after the pre-steps
    for k in range(2, 6):
        mps.sweep1(0.5)
        errs.append(np.max(np.abs(mps.populations() - pe[k + 1])))
    assert max(errs) < 1e-9
