"""Benchmark: 2TDVP time steps (sweeps) of the internal-conversion-like model.

Workload: 2 electronic states + 24 harmonic modes (d_I in 10..30), linear,
quadratic intra-mode and 24 bilinear inter-mode couplings (seed 1002), max
bond dimension 64, DBSS threshold 1e-8, dt = 0.5 fs. One step = one 2TDVP
time step (left-to-right + right-to-left half sweeps). The timed state is a
random right-canonical MPS with every bond at min(64, full dimension), i.e.
the steady state at the bond cap that a long propagation reaches.

Prints ONE JSON line (rank 0). `value` is device-timed sweeps/s summed over
ranks (each rank propagates its own replica: a single trajectory does not
shard); `e2e` is the same metric through the C ABI with host buffers;
`roofline` describes the H_eff products (the operation the metric names)
measured live with CUDA events, `roofline_krylov` the Krylov vector
work; `site_order_search` times the
same workload on the chain order the cost-model search picks (Sec. 3.1,
ordering of local sites); `cpu_baseline` times the CPU oracle on a
bounded sample of the same sweep. `--impl reference` times that oracle as
the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import vibmodels as vm  # noqa: E402

METRIC = "2TDVP sweeps/s & H_eff·ψ TFLOP/s (% peak), mixed vs FP64 at stated population error"
UNIT = "sweeps/s"
M_MAX = 64
EPS = 1e-8
DT_FS = 0.5
STATE_SEED = 424242
PROF_EVERY = 4  # per-phase events on one call in four (systematic sampling; each event pair costs host time)
WORKLOAD = ("internal-conversion-like: 2 states + 24 modes (d 10-30, seed 1002), linear + quadratic "
            "+ 24 bilinear couplings, max bond 64, DBSS 1e-8, dt 0.5 fs, bond-saturated state")
# GB300 FP64 FMA peak: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense tf32 / bf16 tensor-core ratio
# DRAM bytes (read + write) per launch from one ncu capture of the kernels as
# they are now, at the workload's largest pair (profiles/heff2_mixed_ic24_launches.md);
# a kernel changed since its capture has no entry (null)
TRAFFIC: dict = {
    "tc_gemm_tf32_kernel": 0.5 * (616.6e6 + 717.3e6),  # mean of the L and R leg launches
    "sparse_legs": 1300.5e6,
}
TRAFFIC_CASE = ("DRAM bytes per launch at the largest pair (15, 16), mL = mR = 64, from ncu; "
                "equal to the algorithmic bytes there (no re-reads)")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _aggregate_replicas(ms: float, steps: int, ws: int, device="cuda"):
    """Whole-job timing of N independent replicas (a trajectory does not
    shard: each rank propagates its own): the timed region's duration is the
    maximum over ranks, and the rate counts every rank's steps.
    Returns (max ms, sweeps/s summed over ranks)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, ws * steps / (ms / 1e3)


def _clock_sampler_start():
    fd, path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
    os.close(fd)
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200", "-f", path], stdout=subprocess.DEVNULL,
                                stderr=subprocess.DEVNULL)
    except OSError:
        proc = None
    return proc, path


def _clock_sampler_stop(proc, path, gpu_index):
    out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    if proc is None:
        return out
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        with open(path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9 or not c[0].isdigit() or int(c[0]) != gpu_index:
                    continue
                try:
                    sm.append(float(c[1]))
                    smax.append(float(c[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, c[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(path)
    except OSError:
        pass
    if sm:
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
               "samples": len(sm)}
    return out


def _oracle_sweep(model, tensors):
    """One whole 2TDVP time step (sweep) of the CPU oracle on the workload from
    the same bond-saturated state, timed whole (about 9 minutes on 16 Arm
    cores at the internal-conversion size). Returns (seconds, updates)."""
    from oracle import mpo as ompo
    from oracle import tdvp as otdvp
    sim = otdvp.Tdvp2(otdvp.MPS([t.copy() for t in tensors]), ompo.build_mpo(model),
                      otdvp.TdvpOptions(m_max=M_MAX, eps=EPS, krylov_max=30, krylov_tol=1e-13))
    t0 = time.perf_counter()
    sim.step(DT_FS)
    return time.perf_counter() - t0, 2 * (len(tensors) - 1)


def _oracle_positions(model, tensors, k: int, warmup: int = 0):
    """Stratified sample of the oracle's sweep: the left-to-right two-site
    update (merge, forward Krylov exponential, split, environment update,
    backward one-site step) at k chain pairs spread evenly over the chain
    (pair j = floor((j + 1/2) (n - 1) / k)), each timed from the bench state
    brought into mixed-canonical form with the center on that pair (the sites
    to its left made left-orthonormal by QR and their environments built,
    untimed). The sweep time is estimated as 2 (n - 1) times the mean update
    time (the right-to-left half mirrors the left-to-right one). Returns
    (per-pair seconds, pairs, estimated sweep seconds)."""
    from oracle import mpo as ompo
    from oracle import tdvp as otdvp
    W = ompo.build_mpo(model)
    n = len(tensors)
    npairs = n - 1
    k = max(1, min(k, npairs))
    pairs = [int((j + 0.5) * npairs / k) for j in range(k)]
    sim = otdvp.Tdvp2(otdvp.MPS([t.copy() for t in tensors]), W,
                      otdvp.TdvpOptions(m_max=M_MAX, eps=EPS, krylov_max=30, krylov_tol=1e-13))
    A, L = sim.mps.A, sim.L
    snaps = {}
    for p in range(max(pairs) + 1):
        if p in pairs or p == 0:
            snaps[p] = (A[p].copy(), A[p + 1].copy(), L[p])
        mL, d, mR = A[p].shape
        Q, Rm = np.linalg.qr(A[p].reshape(mL * d, mR))
        A[p] = Q.reshape(mL, d, Q.shape[1])
        A[p + 1] = np.einsum("ab,bsc->asc", Rm, A[p + 1])
        L[p + 1] = otdvp.env_left_update(L[p], A[p], W[p])
    tau = 0.5 * DT_FS

    def one(p):
        a0, a1, l0 = snaps[p]
        A[p], A[p + 1], L[p] = a0.copy(), a1.copy(), l0
        t0 = time.perf_counter()
        sim.update_left_to_right(p, tau, otdvp.StepStats())
        return time.perf_counter() - t0

    for _ in range(warmup):
        one(0)
    secs = [one(p) for p in pairs]
    return secs, pairs, 2 * npairs * float(np.mean(secs))


def _cpu_info():
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    import platform
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu": model}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    model = vm.model_internal_conversion()
    tensors = vm.random_right_canonical_mps(STATE_SEED, vm.local_dims(model), M_MAX)
    secs, pairs, est = _oracle_positions(model, tensors, args.steps, warmup=args.warmup)
    value = 1.0 / est
    steps = len(secs)
    info = _cpu_info()
    sample = (f"stratified sample: the left-to-right two-site update at {steps} of the {len(tensors) - 1} chain "
              f"pairs {pairs}, one per step, {sum(secs):.1f} s in all; sweep = 2 x {len(tensors) - 1} x mean "
              f"update = {est:.1f} s")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "one two-site update of the oracle at one chain pair", "host": info},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["nproc"], "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _trajectory_error(P, stream, dtype):
    """Mixed (or FP64) form over the stored oracle trajectory of the reduced
    internal-conversion model (8 modes, d 10..30, bond 64, DBSS 1e-8, from the
    product state; tests/golden/ic8_trajectory.json, written by the oracle):
    the largest population difference over all its steps."""
    path = os.path.join(ROOT, "tests", "golden", "ic8_trajectory.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        g = json.load(f)
    m = vm.model_internal_conversion(seed=1002, n_modes=8, level_range=(10, 30), n_offdiag=2, n_bilinear=8)
    if [int(x) for x in m["levels"]] != g["fingerprint"]["levels"]:
        return None
    mps = P.Mps(P.Mpo(m), vm.product_state_indices(m), m_cap=64, dtype=dtype, krylov_cap=40, stream=stream)
    errs = []
    t0 = time.perf_counter()
    for pops in g["populations"]:
        mps.sweep(g["dt_fs"], m_max=g["m_max"], eps=g["eps"], zero_floor=g["zero_floor"], krylov_max=30,
                  krylov_tol=g["krylov_tol"])
        errs.append(float(np.max(np.abs(mps.populations() - np.array(pops)))))
    wall = time.perf_counter() - t0
    mps.close()
    return {"model": g["model"], "steps": len(errs), "fs": len(errs) * g["dt_fs"],
            "max_pop_err_vs_oracle": max(errs), "pop_err_vs_oracle_last_step": errs[-1],
            "oracle_bond_max": max(g["bonds"][-1]), "wall_s": round(wall, 2)}


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1908_10588_gb300 import build as pbuild
    pbuild.build()
    import paper_1908_10588_gb300 as P

    dtype = P.VB_MIXED if args.dtype == "mixed" else P.VB_FP64
    model = vm.model_internal_conversion()
    dims = vm.local_dims(model)
    tensors = vm.random_right_canonical_mps(STATE_SEED + rank, dims, M_MAX)
    mpo = P.Mpo(model)
    stream = torch.cuda.current_stream()
    mps = P.Mps(mpo, m_cap=M_MAX, dtype=dtype, krylov_cap=40, stream=stream, tensors=tensors)
    sweep_kw = dict(m_max=M_MAX, eps=EPS, zero_floor=1e-14, krylov_max=30, krylov_tol=1e-13)
    for _ in range(args.warmup):
        mps.sweep(DT_FS, **sweep_kw)
    torch.cuda.synchronize()

    # ---- timed region (device time, CUDA events on the library's stream)
    P.vb_profile_read(reset=True)
    P.vb_profile_enable(True, every=PROF_EVERY)
    launches0 = P.vb_kernel_launches()
    proc, cpath = _clock_sampler_start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(mps.sweep(DT_FS, **sweep_kw))
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = _clock_sampler_stop(proc, cpath, local)
    launches = P.vb_kernel_launches() - launches0
    P.vb_profile_enable(False)
    prof = P.vb_profile_read(reset=True)
    ms, value = _aggregate_replicas(ev0.elapsed_time(ev1), args.steps, ws, "cuda")
    pops = mps.populations()
    bonds = mps.bond_dims()

    # ---- end to end through the C ABI with host buffers
    e2e_steps = 0 if args.no_e2e else 1
    h2d = sum(t.nbytes for t in tensors)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        m2 = P.Mps(mpo, m_cap=M_MAX, dtype=dtype, krylov_cap=40, stream=stream, tensors=tensors)
        m2.sweep(DT_FS, **sweep_kw)
        out = m2.tensors()
        pe = m2.populations()
        d2h = sum(o.nbytes for o in out) + pe.nbytes
        m2.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = ws * e2e_steps / e2e_s if e2e_steps else None

    # ---- FP64 form beside the mixed one: one step from the same state, and the
    # population difference between the two forms after that step
    compare = None
    if dtype == P.VB_MIXED and not args.no_fp64_compare:
        m64 = P.Mps(mpo, m_cap=M_MAX, dtype=P.VB_FP64, krylov_cap=40, stream=stream, tensors=tensors)
        m32 = P.Mps(mpo, m_cap=M_MAX, dtype=P.VB_MIXED, krylov_cap=40, stream=stream, tensors=tensors)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        m64.sweep(DT_FS, **sweep_kw)
        c1.record(stream)
        m32.sweep(DT_FS, **sweep_kw)
        torch.cuda.synchronize()
        fp64_ms = c0.elapsed_time(c1)
        perr = float(np.max(np.abs(m64.populations() - m32.populations())))
        compare = {"fp64_sweeps_per_s": 1e3 / fp64_ms, "fp64_ms_per_step": fp64_ms,
                   "speedup_mixed_over_fp64": (1e3 / fp64_ms) and value / (ws * 1e3 / fp64_ms),
                   "pop_err_mixed_vs_fp64_after_1_step": perr}
        m64.close()
        m32.close()

    # ---- one-site TDVP (the next row of the scope) on the same state at the
    # same fixed bonds: one warm-up and two timed steps, energy drift
    tdvp1 = None
    if not args.no_tdvp1:
        m1 = P.Mps(mpo, m_cap=M_MAX, dtype=dtype, krylov_cap=40, stream=stream, tensors=tensors)
        e0 = m1.energy()
        m1.sweep1(DT_FS)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(2):
            m1.sweep1(DT_FS)
        c1.record(stream)
        torch.cuda.synchronize()
        t1_ms = c0.elapsed_time(c1) / 2
        tdvp1 = {"sweeps_per_s": 1e3 / t1_ms, "ms_per_step": t1_ms, "steps_timed": 2,
                 "energy_drift_ev_after_3_steps": abs(m1.energy() - e0), "bond_dims": "fixed at the state's (<= 64)"}
        m1.close()

    # ---- site ordering (Sec. 3.1): the order the cost-model search picks for
    # this model, timed from a random state at that order's saturated bonds
    # (one warm-up and two timed steps), beside the default order above
    order_line = None
    if not args.no_order_search:
        t0 = time.perf_counter()
        order, cost = P.site_order_search(model, m_max=M_MAX)
        search_s = time.perf_counter() - t0
        cdef = P.site_order_cost(model, None, m_max=M_MAX)[0]
        mo = dict(model, site_order=order)
        mpo_o = P.Mpo(mo)
        to = vm.random_right_canonical_mps(STATE_SEED + rank, vm.local_dims(mo), M_MAX)
        mso = P.Mps(mpo_o, m_cap=M_MAX, dtype=dtype, krylov_cap=40, stream=stream, tensors=to)
        mso.sweep(DT_FS, **sweep_kw)
        torch.cuda.synchronize()
        P.vb_profile_read(reset=True)
        P.vb_profile_enable(True, every=PROF_EVERY)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        st_o = [mso.sweep(DT_FS, **sweep_kw) for _ in range(2)]
        c1.record(stream)
        torch.cuda.synchronize()
        P.vb_profile_enable(False)
        prof_o = P.vb_profile_read(reset=True)
        o_ms = c0.elapsed_time(c1) / 2
        po = mso.populations()
        order_line = {
            "order": order, "search_s": round(search_s, 3),
            "predicted_vs_default": {"heff_flops": cost["heff_flops"] / cdef["heff_flops"],
                                     "tensor_elems": cost["tensor_elems"] / cdef["tensor_elems"],
                                     "coupling_dist": cost["coupling_dist"] / cdef["coupling_dist"],
                                     "max_mpo_bond": [cdef["max_w"], cost["max_w"]]},
            "ms_per_step": o_ms, "steps_timed": 2, "speedup_vs_default_order": (ms / args.steps) / o_ms,
            "krylov_iters_max": max(x.krylov_iters_max for x in st_o), "max_bond": max(mso.bond_dims()),
            "krylov_iters_per_step": sum(x.krylov_iters_total for x in st_o) / 2,
            "phases_ms_per_step": {k: round(prof_o[k]["ms"] / 2, 3)
                                   for k in ("heff2", "heff1", "krylov", "split", "env", "merge")},
            "heff_flops_per_step": (prof_o["heff2"]["flops"] + prof_o["heff1"]["flops"]) / 2,
            "populations": [float(x) for x in po],
        }
        mso.close()

    # ---- rooflines. The metric's H_eff TFLOP/s is the whole product (all its
    # kernels); `roofline` is its dominant kernel alone: in the mixed form the
    # tcgen05 GEMM of the two dense legs (tensor pipe), in the FP64 form the
    # FP64 complex GEMM of the same legs (FP64 FMA pipe)
    peaks, src = _peaks()
    h2 = prof["heff2"]
    heff_ms = h2["ms"] + prof["heff1"]["ms"]
    heff_flops = h2["flops"] + prof["heff1"]["flops"]
    achieved = heff_flops / (heff_ms / 1e3) / 1e12 if heff_ms > 0 else 0.0
    events = f"CUDA events on 1 of every {PROF_EVERY} calls of each phase in the timed region, times scaled"
    if dtype == P.VB_FP64:
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "FP64 FMA: 152 SMs x 2 FMA/clk x 2 x 2.07 GHz (nominal)",
                "kernel": "H_eff products (two- and one-site), algorithmic flops / event time"}
        roof_legs = None
    else:
        pk = peaks["bf16_tflops_sustained"] * TF32_PER_BF16
        tc = prof["heff_tc_legs"]
        tc_ach = tc["flops"] / (tc["ms"] / 1e3) / 1e12 if tc["ms"] > 0 else 0.0
        roof = {"bound": "tensor", "achieved": tc_ach, "peak": pk, "unit": "TFLOP/s", "frac": tc_ach / pk,
                "traffic": TRAFFIC.get("tc_gemm_tf32_kernel"), "traffic_case": TRAFFIC_CASE,
                "peak_source": f"{src} bf16 sustained x nominal tf32/bf16 ratio (tf32 pipe), of measured",
                "useful_ceiling_split_tf32": pk / 3.0, "frac_of_useful_ceiling": tc_ach / (pk / 3.0),
                "kernel": "tc_gemm_tf32_kernel (tcgen05 kind::tf32, split-TF32 x3): the dense L and R legs of "
                          "every H_eff product; useful complex flops 8|theta|(mL wL + mR wR) / event time",
                "launches_per_step": tc["calls"] / args.steps, "ms_per_step": tc["ms"] / args.steps,
                "ms_per_launch": tc["ms"] / max(1, tc["calls"])}
        wl = prof["heff_sparse_legs"]
        w_gbs = wl["bytes"] / (wl["ms"] / 1e3) / 1e9 if wl["ms"] > 0 else 0.0
        roof_legs = {
            "sparse_mpo_legs": {"bound": "hbm", "achieved": w_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                "frac": w_gbs / peaks["hbm_gbs"], "traffic": TRAFFIC.get("sparse_legs"),
                                "traffic_case": TRAFFIC_CASE,
                                "kernel": "sparse MPO legs (FP32, CUDA cores); algorithmic bytes = one read of "
                                          "each leg's input and one write of its output",
                                "ms_per_step": wl["ms"] / args.steps, "launches_per_step": wl["calls"] / args.steps},
            "operand_prep_ms_per_step": prof["heff_prep"]["ms"] / args.steps,
            "heff_products": {"achieved": achieved, "unit": "TFLOP/s", "frac_of_tf32_peak": achieved / pk,
                              "frac_of_useful_ceiling": achieved / (pk / 3.0),
                              "kernel": "whole H_eff products (all legs, prep and reductions)"},
        }
    roof["events"] = events
    roof["heff_calls"] = h2["calls"] + prof["heff1"]["calls"]
    roof["heff_ms_per_call"] = heff_ms / max(1, roof["heff_calls"])
    # the Krylov vector work: in the FP64 form FP64 ALU-bound; in the mixed form
    # the Gram-Schmidt passes read FP32 copies of the vectors and are bound by
    # HBM bandwidth (algorithmic bytes recorded by the library per iteration)
    kr = prof["krylov"]
    kr_ms = kr["ms"]
    if dtype == P.VB_MIXED and kr["bytes"] > 0 and kr_ms > 0:
        kr_gbs = kr["bytes"] / (kr_ms / 1e3) / 1e9
        roof_krylov = {"bound": "hbm", "achieved": kr_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": kr_gbs / peaks["hbm_gbs"], "traffic": None,
                       "peak_source": "measured copy bandwidth, of measured",
                       "kernel": "Krylov vector kernels of the mixed form (Gram-Schmidt on FP32 copies: inner "
                                 "products, updates, norms); algorithmic bytes of the two passes / event time of "
                                 "the whole phase, which also holds the small exponential, scaling, the final "
                                 "combination and the host convergence checks",
                       "ms_per_step": kr_ms / args.steps}
    else:
        kr_ach = kr["flops"] / (kr_ms / 1e3) / 1e12 if kr_ms > 0 else 0.0
        roof_krylov = {"bound": "alu", "achieved": kr_ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": kr_ach / FP64_PEAK_TFLOPS, "traffic": None,
                       "peak_source": "FP64 FMA: 152 SMs x 2 FMA/clk x 2 x 2.07 GHz (nominal)",
                       "kernel": "Krylov vector kernels (Gram-Schmidt inner products and updates, norms, "
                                 "scaling, combination); algorithmic FP64 flops / event time of the whole phase, "
                                 "which also holds the small exponential and the per-iteration host check",
                       "ms_per_step": kr_ms / args.steps}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if dtype == P.VB_FP64 else "tf32x3-f32acc/f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_sites": len(dims), "m_max": M_MAX, "eps": EPS, "dt_fs": DT_FS,
                   "site_order": "electronic site first, modes by index",
                   "parallelism": f"replicas x{ws}",
                   "l2": "per-step working set (Krylov basis ~0.8 GB) exceeds L2"},
        "roofline": roof,
        "roofline_legs": roof_legs,
        "roofline_krylov": roof_krylov,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "phases_ms_per_step": {k: round(v["ms"] / args.steps, 3) for k, v in prof.items()},
        "phase_share": {k: round(prof[k]["ms"] / max(1e-9, sum(prof[q]["ms"] for q in
                                                                ("heff2", "heff1", "krylov", "split", "env", "merge"))), 4)
                        for k in ("heff2", "heff1", "krylov", "split", "env", "merge")},
        "heff_tflops": achieved,
        "ritz_jacobi_sweeps_per_call": (prof["ritz_jacobi"]["flops"] / prof["ritz_jacobi"]["calls"]
                                        if prof.get("ritz_jacobi", {}).get("calls") else None),
        "krylov_iters_max": max(s.krylov_iters_max for s in stats),
        "krylov_iters_per_step": sum(s.krylov_iters_total for s in stats) / len(stats),
        "heff_flops_per_step": heff_flops / args.steps,
        "max_bond": max(bonds),
        "populations": [float(x) for x in pops],
    }
    if compare is not None:
        line["fp64_form"] = compare
    if not args.no_trajectory:
        tr = _trajectory_error(P, stream, dtype)
        if tr is not None:
            line["trajectory_error"] = tr
    if tdvp1 is not None:
        line["tdvp1"] = tdvp1
    if order_line is not None:
        line["site_order_search"] = order_line
    if rank == 0 and not args.no_cpu_baseline:
        secs, pairs, est = _oracle_positions(model, tensors, args.cpu_pairs, warmup=1)
        info = _cpu_info()
        line["cpu_baseline"] = {
            "value": 1.0 / est, "unit": UNIT, "cores": info["nproc"], "kind": "oracle",
            "sample": f"stratified: left-to-right two-site updates at chain pairs {pairs} of {len(dims) - 1} "
                      f"({sum(secs):.1f} s), sweep = 2 x {len(dims) - 1} x mean update = {est:.1f} s",
            "host": info}
        if args.cpu_full:
            full_s, upd = _oracle_sweep(model, tensors)
            line["cpu_baseline"]["whole_sweep"] = {"value": 1.0 / full_s, "seconds": full_s, "updates": upd}
    if rank == 0:
        print(json.dumps(line), flush=True)
    mps.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_kernel_case(args):
    """One H_eff,2 product at the largest two-site shape of the workload
    (mL = mR = 64, the two largest adjacent d), repeated --steps times; a
    small, self-contained case for profiler captures (about 1.5 GB)."""
    import torch
    from paper_1908_10588_gb300 import build as pbuild
    pbuild.build()
    import paper_1908_10588_gb300 as P
    dtype = P.VB_MIXED if args.dtype == "mixed" else P.VB_FP64
    model = vm.model_internal_conversion()
    dims = vm.local_dims(model)
    i = max(range(1, len(dims) - 2), key=lambda k: dims[k] * dims[k + 1])
    mpo = P.Mpo(model)
    wl, d1, _ = mpo.site_dims(i)
    _, d2, wr = mpo.site_dims(i + 1)
    rng = np.random.Generator(np.random.PCG64(5))
    L = torch.from_numpy(vm.random_hermitian_env(rng, M_MAX, wl)).cuda()
    R = torch.from_numpy(vm.random_hermitian_env(rng, M_MAX, wr)).cuda()
    x = torch.from_numpy(vm.random_complex(rng, (M_MAX, d1, d2, M_MAX))).cuda()
    y = torch.empty_like(x)
    work = torch.empty(P.vb_heff_work_elems(mpo, i, M_MAX, M_MAX, True), dtype=torch.complex128, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        P.vb_heff2_apply(mpo, i, M_MAX, M_MAX, L, R, x, y, work, dtype, st)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        P.vb_heff2_apply(mpo, i, M_MAX, M_MAX, L, R, x, y, work, dtype, st)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"case": "heff2", "site": i, "d1": d1, "d2": d2, "w_in": wl, "w_out": wr,
                      "ms_per_apply": ms}), flush=True)
    return 0


def run_order_case(args):
    """Site ordering (Sec. 3.1): the workload on the default order, the
    orders the cost-model search picks under three weightings and the rule of
    thumb, each from a random state at its saturated bonds (one warm-up step,
    --steps timed, per-phase events on one call in PROF_EVERY). One JSON line."""
    import torch
    from paper_1908_10588_gb300 import build as pbuild
    pbuild.build()
    import paper_1908_10588_gb300 as P
    dtype = P.VB_MIXED if args.dtype == "mixed" else P.VB_FP64
    model = vm.model_internal_conversion()
    sweep_kw = dict(m_max=M_MAX, eps=EPS, zero_floor=1e-14, krylov_max=30, krylov_tol=1e-13)
    st = torch.cuda.current_stream()
    cands = [("default", None), ("search w=(1,1,1)", P.site_order_search(model, m_max=M_MAX)[0]),
             ("search w=(1,1,0)", P.site_order_search(model, m_max=M_MAX, w_coupling=0)[0]),
             ("search w=(0,1,0)", P.site_order_search(model, m_max=M_MAX, w_flops=0, w_coupling=0)[0]),
             ("rule of thumb, 4 strong modes", P.site_order_rule(model, 4))]
    c0 = P.site_order_cost(model, None, m_max=M_MAX)[0]
    if args.order_growth > 0:
        return _order_growth(args, P, model, cands[:2] + cands[-1:], sweep_kw, st, dtype)
    rows = []
    for name, order in cands:
        m = model if order is None else dict(model, site_order=order)
        ts = vm.random_right_canonical_mps(STATE_SEED, vm.local_dims(m), M_MAX)
        mps = P.Mps(P.Mpo(m), m_cap=M_MAX, dtype=dtype, krylov_cap=40, stream=st, tensors=ts)
        mps.sweep(DT_FS, **sweep_kw)
        torch.cuda.synchronize()
        P.vb_profile_read(reset=True)
        P.vb_profile_enable(True, every=PROF_EVERY)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            mps.sweep(DT_FS, **sweep_kw)
        e1.record(st)
        torch.cuda.synchronize()
        P.vb_profile_enable(False)
        pr = P.vb_profile_read(reset=True)
        c = P.site_order_cost(model, order, m_max=M_MAX)[0]
        rows.append({"order_name": name, "order": order if order is not None else "electronic site first",
                     "ms_per_step": e0.elapsed_time(e1) / args.steps,
                     "predicted_vs_default": {"heff_flops": c["heff_flops"] / c0["heff_flops"],
                                              "tensor_elems": c["tensor_elems"] / c0["tensor_elems"],
                                              "coupling_dist": c["coupling_dist"] / c0["coupling_dist"],
                                              "max_mpo_bond": c["max_w"]},
                     "phases_ms_per_step": {k: round(pr[k]["ms"] / args.steps, 2) for k in
                                            ("heff2", "heff1", "krylov", "split", "env", "merge",
                                             "split_subspace_products", "split_subspace_orth",
                                             "split_rayleigh_ritz", "split_rho", "split_out")},
                     "subspace_iterations_per_step": pr["split_subspace_products"]["calls"] / args.steps,
                     "populations": [float(x) for x in mps.populations()]})
        mps.close()
    print(json.dumps({"case": "site_order", "workload": WORKLOAD, "steps": args.steps, "orders": rows}), flush=True)
    return 0


def _order_growth(args, P, model, cands, sweep_kw, st, dtype):
    """Bond growth under DBSS from the product state |upper state> x |0..0>
    (Sec. 3.1): --order-growth steps on each chain order, every step timed
    with CUDA events; bonds and populations along the way."""
    import torch
    rows = []
    for name, order in cands:
        m = model if order is None else dict(model, site_order=order)
        mps = P.Mps(P.Mpo(m), vm.product_state_indices(m), m_cap=M_MAX, dtype=dtype, krylov_cap=40, stream=st)
        ms, bonds, pops, disc = [], [], [], 0.0
        for _ in range(args.order_growth):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            sg = mps.sweep(DT_FS, **sweep_kw)
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            bonds.append(max(mps.bond_dims()))
            pops.append(float(mps.populations()[0]))
            disc += sg.discarded_weight
        rows.append({"order_name": name, "total_ms": sum(ms), "ms_per_step": [round(x, 1) for x in ms],
                     "max_bond_per_step": bonds, "population_0_per_step": pops, "discarded_weight_sum": disc})
        mps.close()
    print(json.dumps({"case": "site_order_growth", "workload": WORKLOAD, "start": "product state",
                      "steps": args.order_growth, "orders": rows}), flush=True)
    return 0


def run_sf_case(args):
    """The singlet-fission-like configuration at its stated size: 3 electronic
    states (LE, TT, CT), each linearly coupled to its own 100-mode Debye bath
    (lambda 0.05 eV, omega_c 0.1 eV), 10 levels per mode, 301 sites, bond cap
    128, DBSS 1e-8, dt 1 fs. (a) steady state at the cap (random
    right-canonical state, every bond at min(128, full)): --steps timed steps
    of the mixed form after one warm-up, one FP64-form step; (b) from the
    product state |LE> x |0...0>: --sf-steps steps of both forms, the largest
    population difference between them along the way. --sf-mixed-only: (a)
    for the mixed form alone."""
    import torch
    from paper_1908_10588_gb300 import build as pbuild
    pbuild.build()
    import paper_1908_10588_gb300 as P
    m = vm.model_singlet_fission()
    dims = vm.local_dims(m)
    mmax = 128
    kw = dict(m_max=mmax, eps=1e-8, zero_floor=1e-14, krylov_max=30, krylov_tol=1e-13)
    st = torch.cuda.current_stream()
    mpo = P.Mpo(m)
    ts = vm.random_right_canonical_mps(STATE_SEED, dims, mmax)
    out = {"case": "singlet_fission", "model": "model_singlet_fission(seed=1003, n_bath=100, levels=10)",
           "n_sites": len(dims), "m_max": mmax, "eps": 1e-8, "dt_fs": 1.0}
    forms = (("mixed", P.VB_MIXED, args.steps),) + (() if args.sf_mixed_only else (("fp64", P.VB_FP64, 1),))
    for name, dtype, nsteps in forms:
        mps = P.Mps(mpo, m_cap=mmax, dtype=dtype, stream=st, tensors=ts)
        if name == "mixed":
            mps.sweep(1.0, **kw)
        torch.cuda.synchronize()
        P.vb_profile_read(reset=True)
        P.vb_profile_enable(True, every=PROF_EVERY)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(nsteps):
            mps.sweep(1.0, **kw)
        e1.record(st)
        torch.cuda.synchronize()
        P.vb_profile_enable(False)
        pr = P.vb_profile_read(reset=True)
        ms = e0.elapsed_time(e1) / nsteps
        hms = pr["heff2"]["ms"] + pr["heff1"]["ms"]
        hfl = pr["heff2"]["flops"] + pr["heff1"]["flops"]
        out[f"steady_{name}"] = {"ms_per_step": ms, "sweeps_per_s": 1e3 / ms, "steps_timed": nsteps,
                                 "heff_tflops": hfl / (hms / 1e3) / 1e12 if hms > 0 else None,
                                 "phases_ms_per_step": {k: round(pr[k]["ms"] / nsteps, 2) for k in
                                                        ("heff2", "heff1", "krylov", "split", "env", "merge")},
                                 "max_bond": max(mps.bond_dims())}
        if name == "mixed":
            tc = pr["heff_tc_legs"]
            out[f"steady_{name}"]["tc_legs_tflops"] = tc["flops"] / (tc["ms"] / 1e3) / 1e12 if tc["ms"] > 0 else None
        mps.close()
    if args.sf_mixed_only:
        print(json.dumps(out), flush=True)
        return 0
    idx = vm.product_state_indices(m)
    runs = {}
    for name, dtype in (("mixed", P.VB_MIXED), ("fp64", P.VB_FP64)):
        mps = P.Mps(mpo, idx, m_cap=mmax, dtype=dtype, stream=st)
        pops, t0 = [], time.perf_counter()
        for _ in range(args.sf_steps):
            mps.sweep(1.0, **kw)
            pops.append(mps.populations())
        runs[name] = (np.array(pops), time.perf_counter() - t0, max(mps.bond_dims()))
        mps.close()
    err = np.max(np.abs(runs["mixed"][0] - runs["fp64"][0]), axis=1)
    out["from_product_state"] = {"steps": args.sf_steps, "max_pop_err_mixed_vs_fp64": float(err.max()),
                                 "pop_err_last_step": float(err[-1]),
                                 "wall_s": {k: round(v[1], 2) for k, v in runs.items()},
                                 "max_bond": {k: v[2] for k, v in runs.items()},
                                 "populations_last_step_fp64": [float(x) for x in runs["fp64"][0][-1]]}
    print(json.dumps(out), flush=True)
    return 0


def run_batch_case(args):
    """The batched configuration: 64 independent two-state models (mode counts
    8..40, bond caps 16..96 drawn per instance, all couplings scaled 0.5..2x
    across the batch; vibmodels.batch_models, seed 1004), --batch-steps steps
    of dt = 0.5 fs from the product state. Timed two ways with the same
    states: one instance after another on one stream, and all instances at
    once with tdvp2_sweep_batched (one host thread and one stream per
    instance). Reports instance-steps per second and checks that both give
    the same populations."""
    import torch
    from paper_1908_10588_gb300 import build as pbuild
    pbuild.build()
    import paper_1908_10588_gb300 as P
    dtype = P.VB_MIXED if args.dtype == "mixed" else P.VB_FP64
    batch = vm.batch_models(seed=1004, n=64)
    mpos = [P.Mpo(m) for m, _ in batch]
    out = {"case": "batch", "instances": len(batch), "steps": args.batch_steps, "dtype": args.dtype,
           "mode_counts": [len(m["omega"]) for m, _ in batch], "m_max": [mm for _, mm in batch]}
    res = {}
    for how in ("one_stream", "batched"):
        streams = [torch.cuda.Stream() for _ in batch] if how == "batched" else [torch.cuda.current_stream()] * len(batch)
        states = [P.Mps(mpo, vm.product_state_indices(m), m_cap=mm, dtype=dtype, stream=st)
                  for (m, mm), mpo, st in zip(batch, mpos, streams)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.batch_steps):
            if how == "batched":
                P.sweep_batched(states, 0.5, m_max=max(mm for _, mm in batch), eps=0.0)
            else:
                for q, (_, mm) in zip(states, batch):
                    q.sweep(0.5, m_max=mm, eps=0.0)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        res[how] = ([q.populations() for q in states], wall, [max(q.bond_dims()) for q in states])
        for q in states:
            q.close()
    diff = max(float(np.max(np.abs(a - b))) for a, b in zip(res["one_stream"][0], res["batched"][0]))
    n_is = len(batch) * args.batch_steps
    out.update({"one_stream": {"wall_s": res["one_stream"][1], "instance_steps_per_s": n_is / res["one_stream"][1]},
                "batched": {"wall_s": res["batched"][1], "instance_steps_per_s": n_is / res["batched"][1]},
                "speedup_batched": res["one_stream"][1] / res["batched"][1],
                "max_pop_diff_batched_vs_one_stream": diff,
                "max_bond_at_end": res["batched"][2]})
    print(json.dumps(out), flush=True)
    return 0


def run_gradient_case(args):
    """The differentiation configuration: dP_upper(50 fs)/d kappa_I for the 24
    diagonal linear couplings of the upper state in the two-state model
    family of the plain configuration extended to 24 modes (d = 8, seed
    1005), bond cap 64, 100 steps of 0.5 fs, from the product state
    (tdvp2_population_gradient: forward sweeps, costate sweeps backwards,
    step checkpointing every 10 steps). --grad-m, --grad-params and
    --grad-floor change the bond cap, the number of couplings and the
    zero-weight floor of the truncation (0: every bond grows to its cap, so
    the bond dimensions no longer depend on the couplings). With
    --fd-params k, central finite differences (step --fd-h, default 1e-5 eV)
    of the same-form propagation for couplings --fd-start .. --fd-start+k-1,
    their relative difference to the adjoint gradient, and whether the +h and
    -h propagations took the same bond dimensions at every step (a differing
    truncation choice makes the difference quotient meaningless)."""
    import torch
    from paper_1908_10588_gb300 import build as pbuild
    pbuild.build()
    import paper_1908_10588_gb300 as P
    dtype = P.VB_MIXED if args.dtype == "mixed" else P.VB_FP64
    m = vm.model_small_2state(seed=1005, n_modes=24, levels=8)
    up = vm.upper_state_index(m)
    idx = vm.product_state_indices(m)
    n_par = max(1, min(24, args.grad_params))
    params = [(I, up, up) for I in range(24)]
    steps, dt, m_max = 100, 0.5, args.grad_m
    st = torch.cuda.current_stream()
    out = {"case": "gradient", "model": "model_small_2state(seed=1005, n_modes=24, levels=8)", "m_max": m_max,
           "dt_fs": dt, "steps": steps, "t_fs": steps * dt, "dtype": args.dtype, "params": "kappa_I = g^I_upper,upper",
           "zero_floor": args.grad_floor}
    grad = None
    if not args.fd_only:
        mps = P.Mps(P.Mpo(m), idx, m_cap=m_max, dtype=dtype, stream=st)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pops, grad = mps.population_gradient(dt, steps, params[:n_par], up, m_max, zero_floor=args.grad_floor,
                                             checkpoint_every=10)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        bonds = mps.bond_dims()
        mps.close()
        out.update({"n_params": n_par, "wall_s": wall, "population_upper": float(pops[up]),
                    "max_bond_at_t": max(bonds), "gradient": [float(x) for x in grad]})
    if args.fd_params > 0:
        h = args.fd_h
        fd, same, disc = [], [], []
        t0 = time.perf_counter()
        sel = params[args.fd_start: args.fd_start + args.fd_params]
        for (I, i, j) in sel:
            vals, seqs, dws = [], [], []
            for sgn in (1.0, -1.0):
                mm = dict(m)
                g = np.array(m["g1"], dtype=float)
                g[I, i, j] += sgn * h
                mm["g1"] = g
                q = P.Mps(P.Mpo(mm), idx, m_cap=m_max, dtype=dtype, stream=st)
                seq, dw = [], 0.0
                for _ in range(steps):
                    s_ = q.sweep(dt, m_max=m_max, zero_floor=args.grad_floor)
                    seq.append(tuple(q.bond_dims()))
                    dw += s_.discarded_weight
                vals.append(q.populations()[up])
                seqs.append(seq)
                dws.append(dw)
                q.close()
            fd.append((vals[0] - vals[1]) / (2 * h))
            same.append(seqs[0] == seqs[1])
            disc.append(dws)
        fd = np.array(fd)
        out.update({"fd_h_ev": h, "fd_params": [p[0] for p in sel], "fd": [float(x) for x in fd],
                    "fd_wall_s": time.perf_counter() - t0, "fd_bonds_equal_plus_minus": same,
                    "fd_discarded_weight_sum_plus_minus": disc})
        if grad is not None and args.fd_start + len(fd) <= len(grad):
            ga = np.asarray(grad[args.fd_start: args.fd_start + len(fd)])
            out["max_rel_diff_adjoint_vs_fd"] = float(np.max(np.abs(ga - fd)) / np.max(np.abs(fd)))
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-trajectory", action="store_true")
    ap.add_argument("--cpu-pairs", type=int, default=3)
    ap.add_argument("--cpu-full", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tdvp1", action="store_true")
    ap.add_argument("--no-order-search", action="store_true")
    ap.add_argument("--kernel-case", default=None, choices=[None, "heff2"])
    ap.add_argument("--order-case", action="store_true")
    ap.add_argument("--order-growth", type=int, default=0)
    ap.add_argument("--gradient-case", action="store_true")
    ap.add_argument("--sf-case", action="store_true")
    ap.add_argument("--batch-case", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--sf-steps", type=int, default=20)
    ap.add_argument("--sf-mixed-only", action="store_true")
    ap.add_argument("--fd-params", type=int, default=0)
    ap.add_argument("--fd-start", type=int, default=0)
    ap.add_argument("--fd-h", type=float, default=1e-5)
    ap.add_argument("--fd-only", action="store_true")
    ap.add_argument("--grad-m", type=int, default=64)
    ap.add_argument("--grad-params", type=int, default=24)
    ap.add_argument("--grad-floor", type=float, default=1e-14)
    args = ap.parse_args()
    if args.kernel_case:
        return run_kernel_case(args)
    if args.gradient_case:
        return run_gradient_case(args)
    if args.sf_case:
        return run_sf_case(args)
    if args.batch_case:
        return run_batch_case(args)
    if args.order_case:
        return run_order_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
