"""2TDVP on reordered chains (Sec. 3.1, ordering of local sites): the
electronic site inside the chain, orders from the search and the rule of
thumb. Populations through measure_populations (the transfer matrix of the
sites left of the electronic one) against the oracle, and exactness at full
bonds against the dense propagation, which no site order can change."""
import numpy as np
import pytest

import vibmodels as vm
from oracle import mpo as ompo
from oracle import tdvp as otdvp
from oracle import vibronic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

POP_TOL = 1e-8         # FP64 path vs the FP64 oracle
POP_TOL_MIXED = 1e-4   # mixed form vs the FP64 oracle


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


def test_populations_of_a_random_state_with_the_electronic_site_inside(P):
    base = vm.model_internal_conversion(seed=61, n_modes=4, level_range=(3, 6), n_offdiag=2, n_bilinear=3)
    for order in ([1, 0, -1, 3, 2], [2, 3, 1, 0, -1], [0, -1, 1, 2, 3]):
        m = dict(base, site_order=order)
        dims = vm.local_dims(m)
        ts = vm.random_right_canonical_mps(62, dims, 10)
        mps = P.Mps(P.Mpo(m), m_cap=10, tensors=ts)
        ref = otdvp.populations(otdvp.MPS(ts), order.index(-1))
        ref = ref / ref.sum()
        assert np.max(np.abs(mps.populations() - ref)) < 1e-13


@pytest.mark.parametrize("dtype,tol", [("fp64", POP_TOL), ("mixed", POP_TOL_MIXED)])
def test_sweeps_with_the_electronic_site_inside_match_oracle(P, dtype, tol):
    base = vm.model_internal_conversion(seed=63, n_modes=5, level_range=(3, 6), n_offdiag=2, n_bilinear=4)
    order, _ = P.site_order_search(base, m_max=16)
    assert order[0] != -1  # the search moves the electronic site into the chain
    m = dict(base, site_order=order)
    dims, idx = vm.local_dims(m), vm.product_state_indices(m)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, idx, m_cap=16, dtype=P.VB_MIXED if dtype == "mixed" else P.VB_FP64)
    ref = otdvp.Tdvp2(otdvp.product_mps(dims, idx), ompo.build_mpo(m), otdvp.TdvpOptions(m_max=16, eps=1e-9))
    e = order.index(-1)
    for _ in range(8):
        st = mps.sweep(0.5, m_max=16, eps=1e-9, krylov_tol=1e-10 if dtype == "mixed" else 1e-13)
        ref.step(0.5)
        assert st.noconv == 0
        assert np.max(np.abs(mps.populations() - otdvp.populations(ref.mps, e))) < tol
    if dtype == "fp64":
        assert mps.bond_dims() == ref.mps.bond_dims()


def test_full_bond_dynamics_do_not_depend_on_the_site_order(P):
    base = vm.model_small_2state(n_modes=3, levels=4)
    searched, _ = P.site_order_search(base, m_max=64)
    orders = [None, searched, P.site_order_rule(base, 2), [2, 1, 0, -1]]
    for order in orders:
        m = base if order is None else dict(base, site_order=order)
        idx = vm.product_state_indices(m)
        ex = vibronic.exact_propagate(m, vibronic.product_vector(m, idx), 0.5, 6)
        mps = P.Mps(P.Mpo(m), idx, m_cap=64, pad_full=True)
        for k in range(6):
            mps.sweep(0.5, m_max=64, zero_floor=0.0)
            pe = vibronic.populations_from_vector(m, ex[k + 1])
            assert np.max(np.abs(mps.populations() - pe)) < 1e-9


def test_mixed_split_from_the_small_side(P):
    # the electronic site (d = 2) between modes with d = 12..16 at bonds 32:
    # at its pairs one side of theta is 32 * 2 = 64 wide, the other up to
    # 32 * 16 = 512, so the mixed form splits from the small side's Gram
    # matrix and maps the vectors across (Cholesky QR twice)
    base = vm.model_internal_conversion(seed=41, n_modes=5, level_range=(12, 16), n_offdiag=2, n_bilinear=4)
    order = [0, 1, -1, 2, 3, 4]
    m = dict(base, site_order=order)
    dims = vm.local_dims(m)
    e = order.index(-1)
    assert max(32 * dims[e - 1], 32 * dims[e + 1]) > 192 and 32 * dims[e] <= 192
    ts = vm.random_right_canonical_mps(78, dims, 32)
    mps = P.Mps(P.Mpo(m), m_cap=32, dtype=P.VB_MIXED, tensors=ts)
    ref = otdvp.Tdvp2(otdvp.MPS(ts), ompo.build_mpo(m), otdvp.TdvpOptions(m_max=32, eps=1e-8))
    for _ in range(4):
        st = mps.sweep(0.5, m_max=32, eps=1e-8, krylov_tol=1e-10)
        ref.step(0.5)
        assert st.noconv == 0
        assert np.max(np.abs(mps.populations() - otdvp.populations(ref.mps, e))) < POP_TOL_MIXED
    # every site right of the center stays right-orthonormal
    for B in mps.tensors()[1:]:
        Bm = B.reshape(B.shape[0], -1)
        assert np.max(np.abs(Bm @ Bm.conj().T - np.eye(B.shape[0]))) < 1e-11
