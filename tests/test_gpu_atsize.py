"""Parity of whole trajectories at the stated sizes against stored oracle runs.

The expected values come from `tests/golden/make_golden.py`, which runs only
the CPU oracle (complex128 2TDVP, Sec. 2.1.2) and exact propagation; each
file carries a fingerprint of its inputs, checked first. Tolerances: FP64
form 1e-8 on populations, mixed form 1e-4 (split-TF32 H_eff products, FP32
directions of the split, FP64 everything else).

  - two states + four modes x 8 levels, bond cap 16, the full 200 steps of
    100 fs: every step, both forms; the error of the bond-16 run against the
    exact 8192-dimensional propagation is the oracle's (stored beside it);
  - the internal-conversion workload at full size (24 modes, d 10..30, bond
    64, DBSS 1e-8) from the bond-saturated state: whole steps of both forms;
  - a reduced internal-conversion model (8 modes, d 10..30, bond 64, DBSS
    1e-8) from the product state over the whole stored trajectory: the mixed
    form must not drift away from the oracle as the bonds grow and saturate;
  - the singlet-fission-like model at its stated size (301 sites, bond 128):
    mixed form against the FP64 form (the oracle is far too slow there).
"""
import json
import os

import numpy as np
import pytest

import vibmodels as vm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
POP_TOL_FP64 = 1e-8
POP_TOL_MIXED = 1e-4


@pytest.fixture(scope="module")
def P():
    import paper_1908_10588_gb300 as p
    from paper_1908_10588_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return p


def _golden(name, model, tensors=None):
    import sys
    sys.path.insert(0, GOLDEN)
    from make_golden import fingerprint
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    with open(path) as f:
        g = json.load(f)
    fp = fingerprint(model, tensors)
    for k, v in g["fingerprint"].items():
        assert np.allclose(np.asarray(fp[k], dtype=float), np.asarray(v, dtype=float), rtol=1e-12, atol=0), k
    return g


def _sweep_kw(g):
    return dict(m_max=g["m_max"], eps=g["eps"], zero_floor=g["zero_floor"], krylov_max=30,
                krylov_tol=g["krylov_tol"])


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_c1_200_steps_every_step(P, form):
    m = vm.model_small_2state()
    g = _golden("c1_m16_200steps.json", m)
    mpo = P.Mpo(m)
    dtype = P.VB_FP64 if form == "fp64" else P.VB_MIXED
    tol = POP_TOL_FP64 if form == "fp64" else POP_TOL_MIXED
    mps = P.Mps(mpo, vm.product_state_indices(m), m_cap=16, dtype=dtype)
    kw = _sweep_kw(g)
    if form == "mixed":
        kw["krylov_tol"] = 1e-10
    worst = 0.0
    worst_exact = 0.0
    for k, (pops, bonds) in enumerate(zip(g["populations"], g["bonds"])):
        st = mps.sweep(g["dt_fs"], **kw)
        assert st.noconv == 0
        pg = mps.populations()
        err = float(np.max(np.abs(pg - np.array(pops))))
        worst = max(worst, err)
        assert err < tol, (k, err)
        if form == "fp64":
            assert mps.bond_dims() == bonds, k
        worst_exact = max(worst_exact, float(np.max(np.abs(pg - np.array(g["exact_populations"][k])))))
    assert len(g["populations"]) == 200
    # the bond-16 truncation error against the exact 8192-dim propagation is
    # the oracle's own (a few 1e-6 at 100 fs), not a GPU effect
    oracle_exact = max(float(np.max(np.abs(np.array(a) - np.array(b))))
                       for a, b in zip(g["populations"], g["exact_populations"]))
    assert abs(worst_exact - oracle_exact) <= tol
    print(f"c1 {form}: max |dP| vs oracle {worst:.2e}, vs exact {worst_exact:.2e} (oracle vs exact {oracle_exact:.2e})")


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_ic24_full_size_steps(P, form):
    m = vm.model_internal_conversion()
    dims = vm.local_dims(m)
    ts = vm.random_right_canonical_mps(424242, dims, 64)
    g = _golden("ic24_step.json", m, ts)
    mpo = P.Mpo(m)
    dtype = P.VB_FP64 if form == "fp64" else P.VB_MIXED
    tol = POP_TOL_FP64 if form == "fp64" else POP_TOL_MIXED
    mps = P.Mps(mpo, m_cap=64, dtype=dtype, tensors=ts)
    kw = _sweep_kw(g)
    for k, (pops, bonds, disc) in enumerate(zip(g["populations"], g["bonds"], g["discarded"])):
        st = mps.sweep(g["dt_fs"], **kw)
        assert st.noconv == 0
        err = float(np.max(np.abs(mps.populations() - np.array(pops))))
        print(f"ic24 {form} step {k + 1}: max |dP| vs oracle {err:.2e}, discarded {st.discarded_weight:.3e} "
              f"(oracle {disc:.3e}), bonds equal: {mps.bond_dims() == bonds}")
        assert err < tol
        assert mps.bond_dims() == bonds
        # the discarded weights of 48 splits summed; the mixed form resolves
        # the weights to ~1e-7 of the largest
        assert abs(st.discarded_weight - disc) <= (1e-8 if form == "fp64" else 1e-3) * disc + 1e-12


def test_ic8_trajectory_mixed_does_not_drift(P):
    import sys
    sys.path.insert(0, GOLDEN)
    from make_golden import ic8_model
    m = ic8_model()
    g = _golden("ic8_trajectory.json", m)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, vm.product_state_indices(m), m_cap=64, dtype=P.VB_MIXED)
    kw = _sweep_kw(g)
    errs = []
    for k, pops in enumerate(g["populations"]):
        st = mps.sweep(g["dt_fs"], **kw)
        assert st.noconv == 0
        errs.append(float(np.max(np.abs(mps.populations() - np.array(pops)))))
        assert errs[-1] < POP_TOL_MIXED, (k, errs[-1])
    assert len(errs) >= 60
    print(f"ic8 mixed over {len(errs)} steps: max |dP| vs oracle {max(errs):.2e}, last {errs[-1]:.2e}, "
          f"bonds {mps.bond_dims()} (oracle {g['bonds'][-1]})")


def test_ic8_trajectory_fp64_first_steps(P):
    import sys
    sys.path.insert(0, GOLDEN)
    from make_golden import ic8_model
    m = ic8_model()
    g = _golden("ic8_trajectory.json", m)
    mpo = P.Mpo(m)
    mps = P.Mps(mpo, vm.product_state_indices(m), m_cap=64, dtype=P.VB_FP64)
    kw = _sweep_kw(g)
    n = min(30, len(g["populations"]))
    for k in range(n):
        mps.sweep(g["dt_fs"], **kw)
        assert float(np.max(np.abs(mps.populations() - np.array(g["populations"][k])))) < POP_TOL_FP64, k
        assert mps.bond_dims() == g["bonds"][k], k


def test_singlet_fission_full_size_mixed_vs_fp64(P):
    # 3 states x 100-mode Debye baths, 10 levels, 301 sites, bond cap 128:
    # the mixed form (subspace split of m_max + 9 = 137 rows) follows the
    # FP64 form from the product state
    m = vm.model_singlet_fission()
    mpo = P.Mpo(m)
    idx = vm.product_state_indices(m)
    kw = dict(m_max=128, eps=1e-8, zero_floor=1e-14, krylov_max=30, krylov_tol=1e-13)
    a = P.Mps(mpo, idx, m_cap=128, dtype=P.VB_FP64)
    b = P.Mps(mpo, idx, m_cap=128, dtype=P.VB_MIXED)
    worst = 0.0
    for _ in range(6):
        a.sweep(1.0, **kw)
        b.sweep(1.0, **kw)
        worst = max(worst, float(np.max(np.abs(a.populations() - b.populations()))))
    print(f"SF 301 sites: mixed vs FP64 over 6 steps {worst:.2e}, bonds {max(a.bond_dims())}/{max(b.bond_dims())}")
    assert worst < POP_TOL_MIXED
