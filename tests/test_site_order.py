"""Ordering of the chain sites (Sec. 3.1, ordering of local sites; Sec. 4):
the host-side cost model and search of the C ABI (vb_site_order_cost,
vb_site_order_search, vb_site_order_rule). No GPU needed.

Pins: the MPO structure the cost model counts without building tensors
equals the builder's (bond dimensions and nonzero / identity blocks of every
site, read from the dense tensors of mpo_build, itself pinned to the dense
Hamiltonian); saturated bonds and tensor sizes against hand-computed values;
the coupling distance against closed forms (a star of equal couplings, whose
optimum puts the electronic site in the middle; a hand-summed three-site
model); annealing against the exhaustive optimum; the rule of thumb's
layout."""
import itertools

import numpy as np
import pytest

import vibmodels as vm


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    return p


def _builder_structure(P, model, order):
    mpo = P.Mpo(dict(model, site_order=order))
    n = mpo.n_sites
    bonds = [mpo.site_dims(p)[2] for p in range(n - 1)]
    blocks = []
    for p in range(n):
        W = mpo.site_tensor(p)
        d = W.shape[1]
        nop = nid = 0
        for a in range(W.shape[0]):
            for b in range(W.shape[3]):
                B = W[a, :, :, b]
                if not B.any():
                    continue
                if np.array_equal(B, np.eye(d)):
                    nid += 1
                else:
                    nop += 1
        blocks.append([nop, nid])
    return mpo, bonds, blocks


def _hand_model(n_el, omega, levels, g1=None, g2=(), e0=None, v=0.02):
    nm = len(omega)
    m = dict(n_el=n_el, e0=np.linspace(0.0, 0.1, n_el) if e0 is None else np.asarray(e0, float),
             v0=np.full((n_el, n_el), v) - np.diag(np.full(n_el, v)), omega=np.asarray(omega, float),
             levels=np.asarray(levels, dtype=np.int64),
             g1=np.zeros((nm, n_el, n_el)) if g1 is None else np.asarray(g1, float),
             g2=list(g2), site_order=None, include_zpe=1)
    return m


STRUCT_MODELS = [
    lambda: vm.model_internal_conversion(seed=31, n_modes=5, level_range=(3, 6), n_offdiag=2, n_bilinear=4),
    lambda: vm.model_small_2state(n_modes=4, levels=3),
    # levels down to 1 (q, q^2 and n vanish there: zero blocks the builder drops)
    lambda: vm.model_internal_conversion(seed=32, n_modes=6, level_range=(1, 4), n_offdiag=3, n_bilinear=6),
    lambda: vm.model_singlet_fission(seed=5, n_bath=4, levels=3),
]


@pytest.mark.parametrize("which", range(len(STRUCT_MODELS)))
def test_cost_model_counts_the_builders_mpo_structure(P, which):
    m = STRUCT_MODELS[which]()
    nm = len(m["omega"])
    rng = np.random.default_rng(100 + which)
    for _ in range(10):
        order = [int(x) for x in rng.permutation([-1] + list(range(nm)))]
        _, bonds, blocks = P.site_order_cost(m, order)
        _, b2, bl2 = _builder_structure(P, m, order)
        assert bonds == b2
        assert blocks == bl2


def test_heff_flops_follow_the_profilers_convention(P):
    # F = sum over pairs of one H_eff,2 application's flops, as vb_profile
    # counts them (8 per complex multiply-add of the environment legs, 4 d^2
    # per vector for a non-identity W block, 2 d for an identity block)
    m = vm.model_internal_conversion(seed=33, n_modes=4, level_range=(3, 5), n_offdiag=2, n_bilinear=3)
    order = [2, -1, 0, 3, 1]
    mmax = 7
    c, _, _ = P.site_order_cost(m, order, m_max=mmax)
    mpo, _, blocks = _builder_structure(P, m, order)
    dims = [mpo.site_dims(p)[1] for p in range(mpo.n_sites)]
    n = len(dims)
    mb = [1] + [min(mmax, int(np.prod(dims[:b])), int(np.prod(dims[b:]))) for b in range(1, n)] + [1]
    F = 0.0
    for i in range(n - 1):
        mL, mR, d1, d2 = mb[i], mb[i + 2], dims[i], dims[i + 1]
        th = mL * d1 * d2 * mR
        w1 = blocks[i][1] * 2 * d1 + blocks[i][0] * 4 * d1 * d1
        w2 = blocks[i + 1][1] * 2 * d2 + blocks[i + 1][0] * 4 * d2 * d2
        F += 8 * th * mL * mpo.site_dims(i)[0] + w1 * mL * d2 * mR + w2 * mL * d1 * mR + 8 * th * mpo.site_dims(i + 1)[2] * mR
    assert c["heff_flops"] == pytest.approx(F, rel=1e-14)


def test_saturated_bonds_and_tensor_sizes_hand_computed(P):
    m = _hand_model(2, [0.1, 0.2], [3, 4], g1=[[[0.05, 0], [0, -0.05]], [[0.02, 0], [0, 0.0]]])
    c, _, _ = P.site_order_cost(m, None, m_max=64)
    # dims [2, 3, 4]: bonds min(2, 12) = 2 and min(6, 4) = 4; pairs 1*2*3*4 + 2*3*4*1
    assert c["tensor_elems"] == 48 and c["max_tensor"] == 24
    c3, _, _ = P.site_order_cost(m, None, m_max=3)
    # second bond capped at 3: 1*2*3*3 + 2*3*4*1
    assert c3["tensor_elems"] == 42 and c3["max_tensor"] == 24
    cr, _, _ = P.site_order_cost(m, [1, 0, -1], m_max=64)
    # dims [4, 3, 2]: bonds 4 and 2: 1*4*3*2 + 4*3*2*1
    assert cr["tensor_elems"] == 48


def test_coupling_distance_of_a_star_and_its_optimum(P):
    # six modes with equal dimensionless couplings |g|/omega = 1 to the
    # electronic site: D = sum of distances to it; default order (electronic
    # site first) 1 + ... + 6 = 21, optimum 1+1+2+2+3+3 = 12 with the
    # electronic site in the middle
    g = [[[0.05, 0.0], [0.0, -0.05]]] * 6
    m = _hand_model(2, [0.1] * 6, [3] * 6, g1=g)
    c0, _, _ = P.site_order_cost(m)
    assert c0["coupling_dist"] == pytest.approx(21.0, rel=1e-14)
    assert c0["objective"] == pytest.approx(1.0, rel=1e-14)
    order, c = P.site_order_search(m, w_flops=0, w_size=0, w_coupling=1)
    assert c["coupling_dist"] == pytest.approx(12.0, rel=1e-14)
    assert order.index(-1) == 3
    assert c["objective"] == pytest.approx(12.0 / 21.0, rel=1e-14)


def test_coupling_distance_hand_summed_with_bilinear_and_quadratic_terms(P):
    # one bilinear term g q0 q1 |0><0| couples (el, 0), (el, 1), (0, 1) with
    # |g| / sqrt(w0 w1) = 0.03 / 0.2 = 0.15 each; a linear coupling on mode 1
    # adds (0.2 + 0) / 0.4 = 0.5 to (el, 1); a quadratic term 0.04 q1^2 |1><1|
    # adds 0.04 / 0.4 = 0.1 to (el, 1)
    g1 = np.zeros((2, 2, 2))
    g1[1, 0, 0] = 0.2
    m = _hand_model(2, [0.1, 0.4], [3, 3], g1=g1, g2=[(0, 1, 0, 0, 0.03), (1, 1, 1, 1, 0.04)])
    for order, dist in (([-1, 0, 1], 0.15 * 4 + 0.6 * 2), ([0, -1, 1], 0.15 * 4 + 0.6 * 1),
                        ([1, 0, -1], 0.15 * 4 + 0.6 * 2), ([0, 1, -1], 0.15 * 4 + 0.6 * 1)):
        c, _, _ = P.site_order_cost(m, order)
        assert c["coupling_dist"] == pytest.approx(dist, rel=1e-13)


def test_default_search_is_the_exhaustive_minimum(P):
    m = vm.model_internal_conversion(seed=34, n_modes=5, level_range=(2, 7), n_offdiag=2, n_bilinear=4)
    nm = len(m["omega"])
    best = min(P.site_order_cost(m, list(o), m_max=16)[0]["objective"]
               for o in itertools.permutations([-1] + list(range(nm))))
    order, c = P.site_order_search(m, m_max=16)
    assert c["objective"] == pytest.approx(best, rel=1e-14)
    assert P.site_order_cost(m, order, m_max=16)[0]["objective"] == pytest.approx(best, rel=1e-14)


@pytest.mark.parametrize("seed,weights", [(35, (1, 1, 1)), (36, (1, 0, 1))])
def test_annealing_reaches_the_exhaustive_optimum(P, seed, weights):
    m = vm.model_internal_conversion(seed=seed, n_modes=8, level_range=(2, 9), n_offdiag=2, n_bilinear=5)
    wf, ws, wc = weights
    _, ex = P.site_order_search(m, m_max=24, w_flops=wf, w_size=ws, w_coupling=wc, iters=-1)
    order, an = P.site_order_search(m, m_max=24, w_flops=wf, w_size=ws, w_coupling=wc, iters=20000, seed=7)
    assert an["objective"] == pytest.approx(ex["objective"], rel=1e-12)
    assert sorted(order) == [-1] + list(range(8))


def test_rule_of_thumb_layout(P):
    # total strengths sum |g1| / omega: mode 3 > 0 > 5 > 1 > 2 > 4
    s = [0.8, 0.4, 0.3, 1.0, 0.2, 0.6]
    w = [0.1, 0.2, 0.05, 0.15, 0.3, 0.25]
    g1 = np.zeros((6, 2, 2))
    for I in range(6):
        g1[I, 0, 0], g1[I, 1, 1] = s[I] * w[I] / 2, -s[I] * w[I] / 2
    m = _hand_model(2, w, [4] * 6, g1=g1)
    # strongest right of the electronic site, next left, alternating; bath by
    # increasing frequency at the end
    assert P.site_order_rule(m, 2) == [0, -1, 3, 2, 1, 5, 4]
    assert P.site_order_rule(m, 4) == [1, 0, -1, 3, 5, 2, 4]
    assert P.site_order_rule(m, 0) == [-1, 2, 0, 3, 1, 5, 4]


def test_search_on_the_24_mode_workload_model(P):
    # predicted effect on the benchmark's model (m_max 64): the searched order
    # needs well under half the H_eff,2 work of the default order
    m = vm.model_internal_conversion()
    c0, b0, _ = P.site_order_cost(m)
    order, c = P.site_order_search(m)
    assert sorted(order) == [-1] + list(range(24))
    assert c["objective"] < 0.6
    assert c["heff_flops"] < 0.5 * c0["heff_flops"]
    assert c["tensor_elems"] < 0.8 * c0["tensor_elems"]
    again, c2 = P.site_order_search(m)
    assert again == order and c2 == c  # deterministic for a given seed


def test_order_calls_reject_bad_arguments(P):
    m = vm.model_small_2state(n_modes=3, levels=3)
    with pytest.raises(P.VbError):
        P.site_order_cost(m, [0, 0, -1, 2])
    with pytest.raises(P.VbError):
        P.site_order_cost(m, [0, 1, 5, -1])
    with pytest.raises(P.VbError):
        P.site_order_cost(m, None, w_flops=0, w_size=0, w_coupling=0)
    with pytest.raises(P.VbError):
        P.site_order_cost(m, None, w_flops=-1)
    with pytest.raises(P.VbError):
        P.site_order_search(vm.model_internal_conversion(n_modes=12), iters=-1)


def test_chains_of_one_and_two_sites(P):
    m0 = _hand_model(2, [], [])
    assert P.site_order_rule(m0, 4) == [-1]
    order, c = P.site_order_search(m0)
    assert order == [-1] and c["objective"] == 1.0 and c["tensor_elems"] == 0
    m1 = _hand_model(2, [0.1], [5], g1=[[[0.03, 0.01], [0.01, -0.03]]])
    for order in ([-1, 0], [0, -1]):
        _, bonds, blocks = P.site_order_cost(m1, order)
        _, b2, bl2 = _builder_structure(P, m1, order)
        assert bonds == b2 and blocks == bl2
    order, c = P.site_order_search(m1)
    assert sorted(order) == [-1, 0]
    assert c["tensor_elems"] == 10  # one pair: 1 * 2 * 5 * 1
