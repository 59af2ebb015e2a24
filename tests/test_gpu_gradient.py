"""The differentiable form: dP_upper(t)/d(linear couplings) through the C ABI
(tdvp2_population_gradient) and the torch.autograd bridge.

  - full bonds (2 states + 4 modes x 8 levels, bonds padded to full size):
    2TDVP is exact, so the adjoint gradient must equal the exact Duhamel
    gradient of the oracle (oracle/gradient.py, pinned to finite differences
    of exact propagation) up to the step-grid quadrature: 1e-6;
  - truncated bonds: the adjoint gradient against central finite
    differences (h = 1e-5 eV) of the GPU's own FP64 propagation, 1e-4
    relative (the adjoint is the gradient of the exact dynamics evaluated
    on the 2TDVP states, the differences that of the truncated map);
  - step checkpointing does not change the result (bit-equal for several
    checkpoint intervals: the recomputed segments equal the first pass).
"""
import numpy as np
import pytest

import vibmodels as vm
from oracle import gradient as ograd
from oracle import vibronic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL_EXACT = 1e-6
GRAD_RTOL_FD = 1e-4


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


def test_full_bond_gradient_equals_exact_duhamel(P):
    m = vm.model_small_2state()
    up = vm.upper_state_index(m)
    idx = vm.product_state_indices(m)
    params = [(I, up, up) for I in range(4)] + [(1, 0, 1)]
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, idx, m_cap=64, pad_full=True)
    t, dt = 50.0, 0.25
    pops, grad = mps.population_gradient(dt, int(round(t / dt)), params, up, 64, zero_floor=0.0,
                                         checkpoint_every=200)
    psi0 = vibronic.product_vector(m, idx)
    ref = ograd.population_gradient(m, psi0, t, params)[:, up]
    pe = vibronic.populations_from_vector(m, vibronic.exact_propagate(m, psi0, t, 1)[-1])
    assert np.max(np.abs(pops - pe)) < 1e-9
    print("full-bond gradient", grad, "exact", ref, "max |diff|", np.max(np.abs(grad - ref)))
    assert np.max(np.abs(grad - ref)) < GRAD_TOL_EXACT


def test_checkpoint_interval_does_not_change_the_gradient(P):
    m = vm.model_small_2state(n_modes=3, levels=6)
    up = vm.upper_state_index(m)
    idx = vm.product_state_indices(m)
    params = [(I, up, up) for I in range(3)]
    mpo = P.Mpo(m)
    out = []
    for c in (1, 3, 7, 40):
        mps = P.Mps(mpo, idx, m_cap=12)
        out.append(mps.population_gradient(0.5, 24, params, up, 12, checkpoint_every=c))
    for pops, grad in out[1:]:
        assert np.array_equal(pops, out[0][0])
        assert np.array_equal(grad, out[0][1])


def _fd(P, m, idx, params, up, dt, steps, m_max, h=1e-5):
    mpo0 = P.Mpo(m)
    res = []
    g1 = np.asarray(m["g1"], dtype=float)
    for (I, i, j) in params:
        vals = []
        for sgn in (1.0, -1.0):
            mm = dict(m)
            g = g1.copy()
            g[I, i, j] += sgn * h
            if i != j:
                g[I, j, i] += sgn * h
            mm["g1"] = g
            mps = P.Mps(P.Mpo(mm), idx, m_cap=m_max)
            for _ in range(steps):
                mps.sweep(dt, m_max=m_max)
            vals.append(mps.populations()[up])
        res.append((vals[0] - vals[1]) / (2 * h))
    del mpo0
    return np.array(res)


def test_truncated_bond_gradient_vs_finite_differences(P):
    # 12 modes x 8 levels (the two-state model family of the gradient
    # configuration), bond cap 24, 40 steps of 0.5 fs
    m = vm.model_small_2state(seed=1005, n_modes=12, levels=8)
    up = vm.upper_state_index(m)
    idx = vm.product_state_indices(m)
    params = [(0, up, up), (5, up, up), (11, up, up)]
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, idx, m_cap=24)
    steps, dt, m_max = 40, 0.5, 24
    pops, grad = mps.population_gradient(dt, steps, params, up, m_max, checkpoint_every=8)
    fd = _fd(P, m, idx, params, up, dt, steps, m_max)
    rel = np.abs(grad - fd) / np.max(np.abs(fd))
    print("truncated gradient", grad, "fd", fd, "rel", rel)
    assert np.max(rel) < GRAD_RTOL_FD


def test_autograd_bridge(P):
    from paper_1908_10588_gb300 import autograd as pag
    m = vm.model_small_2state(n_modes=3, levels=6)
    up = vm.upper_state_index(m)
    idx = vm.product_state_indices(m)
    params = [(I, up, up) for I in range(3)]
    g = torch.tensor([m["g1"][I][up][up] for I in range(3)], dtype=torch.float64, requires_grad=True)
    p = pag.population(g, m, params, up, 0.5, 24, 12, init_index=idx)
    (3.0 * p).backward()
    mps = P.Mps(P.Mpo(m), idx, m_cap=12)
    pops, grad = mps.population_gradient(0.5, 24, params, up, 12)
    assert abs(p.item() - pops[up]) == 0.0
    assert np.allclose(g.grad.numpy(), 3.0 * grad, rtol=0, atol=0)
