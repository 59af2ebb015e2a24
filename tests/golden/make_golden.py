"""Writes the stored oracle trajectories the at-size parity tests compare with.

Calls only `oracle/` and the seeded input generators of `vibmodels/`: every
expected value in the files it writes is the CPU oracle's (complex128 2TDVP,
Sec. 2.1.2) or exact state-vector propagation. The runs are too long to
repeat inside a GPU test, so they are computed once here:

  c1_m16_200steps.json   2 states + 4 modes x 8 levels (seed 1001), bond cap 16,
                         no threshold, dt 0.5 fs, 200 steps from |upper, 0>:
                         oracle populations, bonds, discarded weights per step,
                         and exact 8192-dim populations
  ic24_step.json         the internal-conversion workload at full size (2 states
                         + 24 modes, d 10..30, seed 1002), bond cap 64, DBSS 1e-8,
                         from the bond-saturated random state (seed 424242):
                         one (or more) oracle steps
  ic8_trajectory.json    a reduced internal-conversion model (8 modes, d 10..30,
                         seed 1002), bond cap 64, DBSS 1e-8, dt 0.5 fs, from
                         |upper, 0>: populations per step over a long trajectory

Each file also records a fingerprint of its inputs (model parameters and the
initial tensors' norms) that the tests check before comparing.

    python tests/golden/make_golden.py c1|ic24|ic8 [steps]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import vibmodels as vm  # noqa: E402
from oracle import mpo as ompo  # noqa: E402
from oracle import tdvp as otdvp  # noqa: E402
from oracle import vibronic  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def fingerprint(model: dict, tensors=None) -> dict:
    """Numbers that identify the inputs a golden file was computed from."""
    fp = {
        "omega_sum": float(np.sum(model["omega"])),
        "levels": [int(x) for x in model["levels"]],
        "g1_abs_sum": float(np.sum(np.abs(model["g1"]))),
        "g2_count": len(model["g2"]),
        "g2_abs_sum": float(sum(abs(v) for (*_, v) in model["g2"])),
    }
    if tensors is not None:
        fp["tensor_abs_sums"] = [float(np.sum(np.abs(t))) for t in tensors]
    return fp


def _run(sim: otdvp.Tdvp2, steps: int, dt: float, path: str, meta: dict, exact=None, model=None):
    rec = dict(meta)
    rec.update({"populations": [], "bonds": [], "discarded": [], "seconds": []})
    if exact is not None:
        rec["exact_populations"] = []
    for k in range(steps):
        t0 = time.perf_counter()
        st = sim.step(dt)
        rec["seconds"].append(time.perf_counter() - t0)
        rec["populations"].append([float(x) for x in otdvp.populations(sim.mps)])
        rec["bonds"].append([int(b) for b in sim.mps.bond_dims()])
        rec["discarded"].append(float(st.discarded))
        if exact is not None:
            rec["exact_populations"].append([float(x) for x in vibronic.populations_from_vector(model, exact[k + 1])])
        with open(path, "w") as f:  # written after every step: a partial run is still usable
            json.dump(rec, f)
        print(f"{os.path.basename(path)}: step {k + 1}/{steps} {rec['seconds'][-1]:.1f} s "
              f"pops {rec['populations'][-1]} bonds max {max(rec['bonds'][-1])}", flush=True)


def make_c1(steps: int = 200):
    m = vm.model_small_2state()
    dims, ix = vm.local_dims(m), vm.product_state_indices(m)
    opts = otdvp.TdvpOptions(m_max=16, eps=0.0)
    sim = otdvp.Tdvp2(otdvp.product_mps(dims, ix), ompo.build_mpo(m), opts)
    exact = vibronic.exact_propagate(m, vibronic.product_vector(m, ix), 0.5, steps)
    meta = {"model": "model_small_2state(seed=1001, n_modes=4, levels=8)", "m_max": 16, "eps": 0.0,
            "zero_floor": opts.zero_floor, "krylov_tol": opts.krylov_tol, "dt_fs": 0.5, "init": "product",
            "fingerprint": fingerprint(m)}
    _run(sim, steps, 0.5, os.path.join(HERE, "c1_m16_200steps.json"), meta, exact=exact, model=m)


def make_ic24(steps: int = 1):
    m = vm.model_internal_conversion()
    dims = vm.local_dims(m)
    ts = vm.random_right_canonical_mps(424242, dims, 64)
    opts = otdvp.TdvpOptions(m_max=64, eps=1e-8)
    sim = otdvp.Tdvp2(otdvp.MPS([t.copy() for t in ts]), ompo.build_mpo(m), opts)
    meta = {"model": "model_internal_conversion(seed=1002)", "m_max": 64, "eps": 1e-8,
            "zero_floor": opts.zero_floor, "krylov_tol": opts.krylov_tol, "dt_fs": 0.5,
            "init": "random_right_canonical_mps(424242, dims, 64)", "fingerprint": fingerprint(m, ts)}
    _run(sim, steps, 0.5, os.path.join(HERE, "ic24_step.json"), meta)


def ic8_model():
    return vm.model_internal_conversion(seed=1002, n_modes=8, level_range=(10, 30), n_offdiag=2, n_bilinear=8)


def make_ic8(steps: int = 60):
    m = ic8_model()
    dims, ix = vm.local_dims(m), vm.product_state_indices(m)
    opts = otdvp.TdvpOptions(m_max=64, eps=1e-8)
    sim = otdvp.Tdvp2(otdvp.product_mps(dims, ix), ompo.build_mpo(m), opts)
    meta = {"model": "model_internal_conversion(seed=1002, n_modes=8, level_range=(10, 30), n_offdiag=2, "
                     "n_bilinear=8)", "m_max": 64, "eps": 1e-8, "zero_floor": opts.zero_floor,
            "krylov_tol": opts.krylov_tol, "dt_fs": 0.5, "init": "product", "fingerprint": fingerprint(m)}
    _run(sim, steps, 0.5, os.path.join(HERE, "ic8_trajectory.json"), meta)


if __name__ == "__main__":
    which = sys.argv[1]
    n = int(sys.argv[2]) if len(sys.argv) > 2 else None
    f = {"c1": make_c1, "ic24": make_ic24, "ic8": make_ic8}[which]
    f(n) if n else f()
