"""Benchmark: cell-timesteps/s of the Picard / backward-Euler / PCG Richards
solve on the 512x512x64 synthetic watershed (10 x 10 x 0.5 m cells,
diamond-square terrain masking the cells above the surface, four sampled van
Genuchten layers, hourly Poisson storms, seepage bottom), Picard tolerance
1e-6 m.

One "step" is one accepted backward-Euler time step: every Picard iteration
(closures, chord capacity, assembly, PCG solve, global max|dh| test), EBATS
reruns and the water balance.  ``value`` is the plain FP64 path (FP64
closures, FP64 Jacobi-PCG) over exactly K steps that start at the first hour
of the seed's first storm, when EBATS has grown dt to dt_max; the state at
that time is spun up from t = 0 by the solver, untimed, and every path starts
from it.  The working set (several GB) is far larger than L2, so no flush is
needed between steps.  Beside it: the FP64 path with double-float closures,
the mixed path (FP32 inner PCG in FP64 defect correction) with Jacobi,
multigrid and DIC preconditioners, the time to solution of the whole 30
simulated days, the other synthetic configurations over their whole periods,
per-kernel device times against their binding roofs, and the CPU oracle on
the host cores over the same window.  ``e2e`` drives the headline steps
through the C ABI from pinned host buffers (state uploaded and read back
every step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

With N > 1 (torchrun, one rank per GPU) every rank runs an independent replica
(different seed): the solve of one domain does not shard without a halo
exchange, so this is replicas-only weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "watershed_512x512x64"
METRIC = "cell-timesteps/s at Picard tol 1e-6 m"
UNIT = "cell-timesteps/s"


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-full-period", action="store_true", help="skip the 30-day time-to-solution legs")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble leg")
    ap.add_argument("--ensemble-window", type=float, default=600.0,
                    help="simulated seconds of the ensemble leg (172800: its whole 2 days)")
    ap.add_argument("--ensemble-precond", default="zline", choices=["zline", "jacobi"],
                    help="inner PCG preconditioner of the ensemble leg (vertical-line solve or Jacobi)")
    ap.add_argument("--no-warmstart", action="store_true", help="skip the learned warm-start leg")
    ap.add_argument("--no-configs", action="store_true", help="skip the column and box legs")
    ap.add_argument("--no-stiff", action="store_true", help="skip the stiff-solve preconditioner comparison")
    ap.add_argument("--slope", action="store_true",
                    help="add the tilted slope's 10 days (36 M cells, the paper's strong-scaling case; about 2 min)")
    ap.add_argument("--ws-train-size", type=int, default=128, help="nx = ny of the training box (nz = 64)")
    ap.add_argument("--ws-eval-size", type=int, default=256, help="nx = ny of the held-out boxes (nz = 64)")
    ap.add_argument("--ws-eval-seeds", type=int, default=1, help="held-out seeds evaluated")
    ap.add_argument("--ws-snapshots", type=int, default=64, help="training snapshots (accepted plain steps)")
    ap.add_argument("--ws-train-steps", type=int, default=600, help="Adam steps (one full box per step)")
    ap.add_argument("--ws-eval-hours", type=float, default=1.0, help="simulated hours of each held-out run")
    ap.add_argument("--ws-eval-start", type=float, default=3.0,
                    help="simulated hour at which the held-out runs start (inside the 6 h of rain; spun up untimed)")
    return ap.parse_args()


def config_dict(extra=None):
    d = {"workload": WORKLOAD, "cells": 512 * 512 * 64, "cell_size_m": [10.0, 10.0, 0.5],
         "terrain": "diamond-square 513^2, roughness 0.8, surface 16-32 m", "layers": 4,
         "rain": "hourly Poisson storms, mean gap 48 h, Exp(6 h) durations, Exp(3 mm/h) intensities, 720 h",
         "bottom": "seepage face", "picard_tol_m": 1e-6, "cg_tol_rel": 1e-10,
         "ebats": "dt0 1 s, x1.3 after 10 easy steps, max 600 s",
         "l2": "working set (several GB) larger than the 129 MB L2; not flushed"}
    if extra:
        d.update(extra)
    return d


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if "Active" in r[3 + i]
                          and "Not" not in r[3 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------ CPU baseline
def oracle_from_state(case, h, meta, openmp=False):
    """The CPU oracle on a workload, resumed at a saved state (time and EBATS
    counters included)."""
    from tests.helpers import oracle_from_case
    o = oracle_from_case(case, openmp=openmp)
    o.set_state(h, meta["t"])
    o.set_clock(meta["t"], meta["dt_nom"], meta["easy"])
    return o


def oracle_steps(o, n_steps=None, budget_s=20.0):
    """Time accepted oracle steps: n_steps, or as many as fit in budget_s."""
    t0 = time.perf_counter()
    k = picard = 0
    while (n_steps is None or k < n_steps) and time.perf_counter() - t0 < budget_s:
        picard += o.step().picard
        k += 1
    return k, time.perf_counter() - t0, picard


def oracle_threads():
    """Threads of the OpenMP build of the oracle (0 when it cannot be built)."""
    from oracle import oracle as O
    return O.num_threads(openmp=True)


def cpu_baseline(case, h, meta, budget_s=20.0):
    """The oracle as it stands on the host cores (its OpenMP build on all of
    them) over the first steps of the GPU's timed window, from the same state;
    the one-thread build over its first step beside it."""
    threads = oracle_threads()
    o = oracle_from_state(case, h, meta, openmp=threads > 0)
    k, t, pic = oracle_steps(o, None, budget_s)
    out = {"value": k * case.n_active() / t, "unit": UNIT, "cores": max(threads, 1), "kind": "oracle",
           "sample": f"the first {k} accepted steps of the timed window of {WORKLOAD} (from t = {meta['t'] / 3600:.0f} h, "
                     f"{pic} Picard iterations, {t:.1f} s; C oracle"
                     + (f", OpenMP, {threads} threads)" if threads else ", one thread)")}
    del o
    if threads > 0:
        o = oracle_from_state(case, h, meta)
        k1, t1, _ = oracle_steps(o, 1, budget_s)
        out["single_thread"] = {"value": k1 * case.n_active() / t1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"the first accepted step of the same window ({t1:.1f} s, one-thread C oracle)"}
    return out


def oracle_configs(args, W):
    """The oracle on the other workloads, bounded samples of each: the 1-D
    column over the GPU leg's whole window (one thread), the first accepted
    steps of the box from t = 0 (OpenMP build), and a stratified sample of the
    ensemble's instances from t = 0 (one thread)."""
    from tests.helpers import oracle_from_case

    def steps_within(o, budget_s, t_stop=None):
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < budget_s:
            info = o.step() if t_stop is None else o.run(t_stop, log_cap=1)
            if t_stop is not None:
                k += len(info) if isinstance(info, list) else 1
                break
            k += 1
        return k, time.perf_counter() - t0

    out = {}
    col = W.infiltration_column(t_end=2 * 3600.0)
    o = oracle_from_case(col)
    t0 = time.perf_counter()
    steps = o.run(col.t_end)
    dt = time.perf_counter() - t0
    out["infiltration_column_1x1x200"] = {
        "value": len(steps) * col.N / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": f"the GPU leg's whole window: {len(steps)} accepted steps over the first 2 simulated hours, "
                  f"one-thread C oracle ({dt:.2f} s)"}
    del o
    threads = oracle_threads()
    box = W.heterogeneous_box(128, 128, 64, seed=args.seed)
    o = oracle_from_case(box, openmp=threads > 0)
    k, dt, _ = oracle_steps(o, None, 10.0)
    out["heterogeneous_box_128x128x64"] = {
        "value": k * box.n_active() / dt, "unit": UNIT, "cores": max(threads, 1), "kind": "oracle",
        "sample": f"first {k} accepted steps from t=0 ({dt:.1f} s, C oracle"
                  + (f", OpenMP, {threads} threads)" if threads else ", one thread)")}
    del o
    cases = W.ensemble(256, seed=args.seed)
    by_size = sorted(range(len(cases)), key=lambda i: cases[i].N)
    sample = by_size[8::32]
    cell_steps, total = 0, 0.0
    for i in sample:
        o = oracle_from_case(cases[i])
        k, dt, _ = oracle_steps(o, None, 1.5)
        cell_steps += k * cases[i].n_active()
        total += dt
        del o
    out["ensemble_256_uneven"] = {
        "value": cell_steps / total, "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": f"{len(sample)} of the 256 instances (every 32nd by size), each from t=0 for at most 1.5 s, "
                  f"one-thread C oracle"}
    return out


# ------------------------------------------------------------ native arm
def max_over_ranks(x, world, device):
    """The largest x over all ranks: the job's time is its slowest rank's."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, t_max):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / t_max


PROFILE_JSON = os.path.join(ROOT, "profiles", "ncu_watershed_kernels.json")


def sources_sha(files):
    """SHA-256 (16 hex digits) of the concatenated kernel sources."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1809_10895_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_entry(kernel):
    """The committed ncu summary of a kernel (DRAM bytes and FP64 arithmetic
    per launch on the watershed); None when absent or taken on different
    kernel sources (the .cu file and the headers holding its arithmetic)
    than the ones built now."""
    try:
        d = json.load(open(PROFILE_JSON))
        e = d["kernels"][kernel]
        if sources_sha(e["sources"]) != e["sources_sha"]:
            return None
        return e
    except Exception:
        return None


def traffic_for(kernel, active_cells):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    workload's active cells (the captured grid is a smaller slice of the
    same watershed)."""
    e = profile_entry(kernel)
    return None if e is None else e["dram_bytes_per_launch"] * active_cells / e["active_cells"]


def storm_start(case, min_hours=7.0):
    """Start of the timed window: the first hour of rain of the workload's
    series at or after min_hours (EBATS has grown dt from 1 s to dt_max by
    then), else min_hours."""
    import numpy as np
    top = next(b for b in case.bcs if b.face == "zmax")
    t, v = np.asarray(top.t), np.asarray(top.v)
    i = np.nonzero((v > 0) & (t >= min_hours * 3600.0))[0]
    return float(t[i[0]]) if len(i) else min_hours * 3600.0


def fp64_counts(kernel):
    """FP64 arithmetic instructions per active cell of a kernel from the
    committed ncu summary (None when absent or stale)."""
    e = profile_entry(kernel)
    return e if e and e.get("fp64_inst_per_cell") else None


def native(args):
    import numpy as np
    import torch

    from __graft_entry__ import build
    build()
    from paper_1809_10895_gb300 import rf
    from paper_1809_10895_gb300 import workloads as W

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    case = W.watershed(512, 512, 64, seed=args.seed + rank, hours=720)
    n_act = case.n_active()
    t0_win = storm_start(case)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- the window's start state: the mixed path (fastest) runs from t = 0
    # to the storm's first hour, untimed; every leg starts from this state
    sp = rf.Solver.from_case(case, precision="mixed")
    sp.run(t0_win)
    h_start = torch.empty(case.N, dtype=torch.float64, device="cuda")
    sp.get_state_device(h_start)
    _, meta0 = sp.get_state()
    mb0 = sp.mass_balance()
    mass7 = [mb0["storage0"], 0.0, mb0["inflow_cum"], mb0["outflow_cum"], 0.0, 0.0, mb0["nonlinear_defect_cum"]]
    sp.close()
    del sp

    def start(s):
        s.set_state_device(h_start, meta0["t"])
        s.set_meta(meta0, mass7)

    def timed_window(precision, **kw):
        """W warm-up steps (graph capture included), back to the start state,
        then exactly K steps timed by CUDA events on the solver's stream."""
        s = rf.Solver.from_case(case, precision=precision, **kw)
        start(s)
        for _ in range(args.warmup):
            s.step()
        start(s)
        c0 = s.launch_counts()
        picard = cg = rej = 0
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        w0 = time.perf_counter()
        ev0.record(s.stream)
        for _ in range(args.steps):
            info = s.step()
            picard += info.picard
            cg += info.cg
            rej += info.rejected
        ev1.record(s.stream)
        barrier()
        wall = time.perf_counter() - w0
        ms = ev0.elapsed_time(ev1)
        c1 = s.launch_counts()
        counts = {k: (c1[k][0] - c0[k][0], c1[k][1] - c0[k][1]) for k in c1}
        t_end = s.get_state()[1]["t"]
        return s, ms, wall, counts, dict(picard=picard, cg=cg, rejected=rej, t_end=t_end)

    # ---- headline: the plain FP64 path (FP64 closures, FP64 Jacobi-PCG)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)        # let the sampler start before the timed region
    s64, ms64, wall64, counts64, st64 = timed_window("fp64")
    clk = clocks.stop()
    t64 = max_over_ranks(ms64 / 1e3, world, "cuda")
    value = job_value(args.steps * n_act, world, t64)
    launches = sum(v[0] for v in counts64.values())

    def leg(precision, **kw):
        try:
            s, ms, wall, counts, st = timed_window(precision, **kw)
            t = max_over_ranks(ms / 1e3, world, "cuda")
            out = {"value": job_value(args.steps * n_act, world, t), "unit": UNIT, "ms_per_step": t * 1e3 / args.steps,
                   "picard_per_step": st["picard"] / args.steps, "cg_iters": st["cg"], "rejected": st["rejected"],
                   "wall_s": wall, "gpu_launches": sum(v[0] for v in counts.values())}
            return s, out, counts
        except Exception as ex:                           # recorded, not fatal to the other legs
            return None, {"error": f"{type(ex).__name__}: {ex}"[:300]}, None

    s_df, leg_df, _ = leg("fp64", closure_arith="double_float")
    if s_df is not None:
        s_df.close()
    s_mix, leg_mix, counts_mix = leg("mixed")
    others = {"fp64_double_float_closures": leg_df, "mixed_jacobi": leg_mix}
    for pc in ("mg", "dic"):
        s_, out, _ = leg("mixed", precond=pc)
        others[f"mixed_{pc}"] = out
        if s_ is not None:
            s_.close()

    # ---- per-kernel device times on the window's end state; shares of the
    # headline leg from the device launch counters (launches that did work)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp64_peak = 2.0 * sms * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9    # G FP64 instructions / s

    def kernel_table(s, kinds):
        out = {}
        for kind in kinds:
            avg_ms, by = s.profile_kernel(kind, reps=20)
            out[kind] = {"avg_ms": avg_ms, "bytes": by, "gbs": by / (avg_ms * 1e-3) / 1e9}
        return out

    names = {"closure": "k_closure_picard", "assemble": "k_assemble", "cg64_spmv": "k_cg64_spmv",
             "cg64_update": "k_cg64_update", "resid64": "k_resid64", "cg32_spmv": "k_cg32_spmv_tma",
             "cg32_update": "k_cg32_update"}
    kern64 = kernel_table(s64, ("closure", "assemble", "cg64_spmv", "cg64_update"))
    work64 = {"closure": counts64["closure_picard"][1] + counts64["closure"][1],
              "assemble": counts64["assemble"][1], "cg64_spmv": counts64["cg64_spmv"][1],
              "cg64_update": counts64["cg64_update"][1]}
    est = {k: work64[k] * kern64[k]["avg_ms"] for k in work64}
    dom = max(est, key=lambda k: est[k])

    def roof_of(kind, kd):
        """The kernel against its binding roof: the FP64 pipe when its FP64
        arithmetic per cell (ncu counts) takes longer at 2 instructions per
        clock per SM than its algorithmic bytes at the HBM peak, else HBM."""
        ent = fp64_counts(names[kind])
        tr = traffic_for(names[kind], n_act)
        hbm = {"achieved": kd["gbs"], "peak": hbm_peak, "unit": "GB/s", "frac": kd["gbs"] / hbm_peak}
        if ent and ent.get("fp64_inst_per_cell"):
            inst = ent["fp64_inst_per_cell"] * n_act
            if inst / (fp64_peak * 1e9) > kd["bytes"] / (hbm_peak * 1e9):
                ach = inst / (kd["avg_ms"] * 1e-3) / 1e9
                return {"kernel": names[kind], "bound": "alu", "achieved": ach, "peak": fp64_peak,
                        "unit": "G FP64 inst/s", "frac": ach / fp64_peak,
                        "peak_source": f"derived: 2 FP64 instructions/clk/SM x {sms} SMs x "
                                       f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz (MEASURED_PEAKS.json sm_max_mhz)",
                        "traffic": tr, "fp64_inst_per_cell": ent["fp64_inst_per_cell"],
                        "algorithmic_fp64_inst_per_launch": inst, "avg_launch_ms": kd["avg_ms"],
                        "algorithmic_bytes_per_launch": kd["bytes"], "hbm": hbm}
        return {"kernel": names[kind], "bound": "hbm", "achieved": kd["gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": kd["gbs"] / hbm_peak, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": tr, "algorithmic_bytes_per_launch": kd["bytes"], "avg_launch_ms": kd["avg_ms"]}

    roof = roof_of(dom, kern64[dom])
    kernels64 = {names[k]: dict(roof_of(k, v), launches_worked=work64[k], est_ms=est[k],
                                share_of_window=est[k] / ms64) for k, v in kern64.items()}
    kernels_mix = None
    if s_mix is not None:
        names["closure"] = "k_closure_picard_df"      # the mixed path's double-float closures
        km = kernel_table(s_mix, ("closure", "assemble", "resid64", "cg32_spmv", "cg32_update"))
        wm = {"closure": counts_mix["closure_picard"][1] + counts_mix["closure"][1],
              "assemble": counts_mix["assemble"][1], "resid64": counts_mix["resid64"][1],
              "cg32_spmv": counts_mix["cg32_spmv"][1], "cg32_update": counts_mix["cg32_update"][1]}
        kernels_mix = {names[k]: dict(roof_of(k, v), launches_worked=wm[k], est_ms=wm[k] * v["avg_ms"])
                       for k, v in km.items()}
        s_mix.close()

    # ---- end to end through the C ABI with host buffers: every step uploads
    # the state from pinned memory and reads it back
    e2e = None
    if not args.no_e2e:
        h_pin = torch.empty(case.N, dtype=torch.float64, pin_memory=True)
        h_pin.copy_(h_start)
        h_np = h_pin.numpy()
        meta = dict(meta0)
        start(s64)
        barrier()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            s64.set_state(h_np, meta["t"])
            s64.set_meta(meta, mass7)
            s64.step()
            _, meta = s64.get_state(out=h_np)
        barrier()
        te = max_over_ranks(time.perf_counter() - w0, world, "cuda")
        e2e = {"value": job_value(args.steps * n_act, world, te), "unit": UNIT, "h2d_bytes_per_step": 8 * case.N,
               "d2h_bytes_per_step": 8 * case.N, "precision": "fp64"}
    s64.close()

    # ---- time to solution of the whole 30 simulated days, from t = 0
    full = None
    if not args.no_full_period:
        full = {}
        for name, prec, kw in (("fp64", "fp64", {}), ("mixed", "mixed", {})):
            s = rf.Solver.from_case(case, precision=prec, **kw)
            s.step()                                   # graph capture outside the timing
            s.set_state(case.h0, 0.0)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            ev0.record(s.stream)
            steps = s.run(case.t_end)
            ev1.record(s.stream)
            barrier()
            ms = ev0.elapsed_time(ev1)
            mb = s.mass_balance()
            full[name] = {"simulated_s": case.t_end, "time_to_solution_s": ms / 1e3, "steps": len(steps),
                          "picard": sum(x.picard for x in steps), "cg_iters": sum(x.cg for x in steps),
                          "rejected": sum(x.rejected for x in steps),
                          "value": len(steps) * n_act / (ms / 1e3), "unit": UNIT,
                          "closure_rel": mb["closure_rel"]}
            s.close()

    # ---- batched ensemble: 256 uneven instances over their whole 2 days
    ens = None
    if not args.no_ensemble:
        try:
            ens = ensemble_leg(args, rank, rf, W, barrier)
        except Exception as ex:
            ens = {"error": f"{type(ex).__name__}: {ex}"[:300]}

    # ---- learned warm start
    wsl = None
    if not args.no_warmstart:
        try:
            wsl = warmstart_leg(args, rank, rf, W, peaks)
        except Exception as ex:
            wsl = {"error": f"{type(ex).__name__}: {ex}"[:300]}

    # ---- the other synthetic configurations
    cfg = None
    if not args.no_configs:
        cfg = configs_leg(args, rank, rf, W)
    stiff = None
    if not args.no_stiff:
        stiff = stiff_leg(rf, W)
    slope = None
    if args.slope:
        slope = slope_leg(rf, W)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t64 * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (closures, operator, PCG, Picard test, balance)",
            "data": "synthetic (seeded diamond-square terrain, sampled soil layers, Poisson storms; no dataset)",
            "config": config_dict({"window": f"{args.steps} accepted steps from t = {t0_win / 3600:.0f} h "
                                             f"(the first hour of the seed's first storm, dt grown to dt_max), "
                                             f"state spun up from t = 0 untimed",
                                   "window_end_s": st64["t_end"], "precision": "fp64", "precond": "jacobi",
                                   "parallelism": "replicas" if world > 1 else "single GPU",
                                   "active_cells": n_act, "picard_iters": st64["picard"], "cg_iters": st64["cg"],
                                   "rejected": st64["rejected"], "wall_s": wall64}),
            "gpu_launches": launches,
            "launch_counts": {k: {"launched": v[0], "worked": v[1]} for k, v in counts64.items() if v[0]},
            "roofline": roof,
            "kernels": kernels64,
            "kernels_mixed": kernels_mix,
            "clocks": clk,
            "e2e": e2e,
            "other_paths": others,
            "speedup_mixed_vs_fp64": (leg_mix["value"] / value) if "value" in leg_mix else None,
            "time_to_solution": full,
            "ensemble": ens,
            "warmstart": wsl,
            "other_configs": cfg,
            "stiff_solve": stiff,
            "tilted_slope": slope,
        }
        if not args.no_baseline:
            # host-side legs: an error is recorded in the line, never lost with it
            try:
                line["cpu_baseline"] = cpu_baseline(case, h_start.cpu().numpy(), meta0, budget_s=20.0)
            except Exception as ex:
                line["cpu_baseline"] = {"error": f"{type(ex).__name__}: {ex}"[:300]}
            if not args.no_configs:
                try:
                    line["cpu_baseline_other_configs"] = oracle_configs(args, W)
                except Exception as ex:
                    line["cpu_baseline_other_configs"] = {"error": f"{type(ex).__name__}: {ex}"[:300]}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def ensemble_leg(args, rank, rf, W, barrier):
    import torch
    cases = W.ensemble(256, seed=args.seed + rank)
    e = rf.Ensemble.from_cases(cases, precision="mixed", precond=args.ensemble_precond)
    cluster, cta_threads, n_wide, probe_ms = e.tune(min(20.0, args.ensemble_window))
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(e.stream)
    e.run(args.ensemble_window)
    ev1.record(e.stream)
    torch.cuda.synchronize()
    ens_ms = ev0.elapsed_time(ev1)
    stats = [e.get(i, want_h=False)[1] for i in range(len(cases))]
    cell_steps = sum(st["steps"] * st["cells"] for st in stats)
    out = {"workload": "ensemble_256_uneven", "instances": len(cases), "cells": sum(c.N for c in cases),
           "simulated_window_s": args.ensemble_window, "cluster_ctas": cluster, "cta_threads": cta_threads,
           "wide_instances": n_wide, "tuner_probe_ms": probe_ms, "kernel_ms": ens_ms, "time_to_solution_s": ens_ms / 1e3,
           "cell_timesteps": cell_steps, "value": cell_steps / (ens_ms * 1e-3), "unit": UNIT,
           "steps_total": sum(st["steps"] for st in stats), "picard_total": sum(st["picard_iters"] for st in stats),
           "inner_pcg_total": sum(st["cg_iters"] for st in stats),
           "failed_instances": sum(1 for st in stats if st["status"] != 0), "precision": "mixed",
           "precond": args.ensemble_precond,
           "max_closure_rel": max(st["closure_abs"] / max(st["storage0"] + st["inflow_cum"] + st["outflow_cum"], 1e-300)
                                  for st in stats)}
    e.close()
    return out


def slope_leg(rf, W):
    """Time to solution of the tilted slope (850 x 850 x 50 cells of 2 x 2 x
    0.2 m, 10 days, Picard 1 mm, dt 0.1 s .. 30 min), FP64 and mixed paths,
    event-timed from t = 0 (after one untimed warm-up step and a reset)."""
    import torch
    case = W.tilted_slope()
    out = {"workload": case.name, "cells": case.N, "simulated_s": case.t_end}
    for prec in ("fp64", "mixed"):
        try:
            s = rf.Solver.from_case(case, precision=prec)
            s.step()
            s.set_state(case.h0, 0.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s.stream)
            steps = s.run(case.t_end)
            b.record(s.stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            mb = s.mass_balance()
            out[prec] = {"time_to_solution_s": ms / 1e3, "steps": len(steps),
                         "picard": sum(x.picard for x in steps), "cg_iters": sum(x.cg for x in steps),
                         "rejected": sum(x.rejected for x in steps), "closure_rel": mb["closure_rel"],
                         "value": len(steps) * case.N / (ms / 1e3), "unit": UNIT}
            s.close()
        except Exception as ex:
            out[prec] = {"error": f"{type(ex).__name__}: {ex}"[:300]}
    return out


def stiff_leg(rf, W):
    """One linear solve from x = 0 on a stiff system (saturated, 10:1
    anisotropic, storage-poor 256x256x64 block) per preconditioner of the
    mixed path, at two time steps: inner iterations and event-timed ms."""
    import torch
    case = W.stiff_block(256, 256, 64)
    dev = dict(dtype=torch.float64, device="cuda")
    hk = torch.as_tensor(case.h0, **dev)
    out = {"workload": case.name, "cells": case.N, "tol_cg_rel": case.params["tol_cg"], "precision": "mixed"}
    for dt in (60.0, 3600.0):
        for pc in ("jacobi", "mg", "dic"):
            try:
                s = rf.Solver.from_case(case, precision="mixed", precond=pc)
                s.assemble(hk, hk, dt, 0.0)
                x = torch.zeros(case.N, **dev)
                s.solve(x)                      # first solve builds the graphs
                x.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s.stream)
                its = s.solve(x)
                b.record(s.stream)
                torch.cuda.synchronize()
                out[f"{pc}_dt{int(dt)}"] = {"inner_iters": its, "ms": a.elapsed_time(b)}
                s.close()
            except Exception as ex:
                out[f"{pc}_dt{int(dt)}"] = {"error": str(ex)[:200]}
    return out


def configs_leg(args, rank, rf, W):
    import torch

    def timed_run(s, t_end):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        steps = s.run(t_end)
        b.record(s.stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), steps

    out = {}
    # 1-D column: its feasible window, the first 2 simulated hours (R-stall), plain FP64
    col = W.infiltration_column(t_end=2 * 3600.0)
    s = rf.Solver.from_case(col, precision="fp64")
    s.step()
    s.set_state(col.h0, 0.0)
    ms, steps = timed_run(s, col.t_end)
    out["infiltration_column_1x1x200"] = {"precision": "fp64", "simulated_s": col.t_end, "steps": len(steps),
                                          "time_to_solution_s": ms / 1e3, "ms_per_step": ms / len(steps),
                                          "picard_per_step": sum(x.picard for x in steps) / len(steps),
                                          "value": len(steps) * col.N / (ms / 1e3), "unit": UNIT}
    s.close()
    # the same column on the device-resident integrator (the ensemble kernel
    # with one instance on one CTA: EBATS, Picard and PCG all on the device)
    e = rf.Ensemble.from_cases([col], precision="fp64")
    e.set_tiling(1, 128)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(e.stream)
    e.run(col.t_end)
    b.record(e.stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    st = e.get(0, want_h=False)[1]
    out["infiltration_column_1x1x200"]["device_resident"] = {
        "steps": st["steps"], "picard_iters": st["picard_iters"], "cg_iters": st["cg_iters"],
        "time_to_solution_s": ms / 1e3, "ms_per_step": ms / max(1, st["steps"]),
        "value": st["steps"] * col.N / (ms / 1e3), "unit": UNIT}
    e.close()
    # the heterogeneous box over its whole 48 h, both paths
    box = W.heterogeneous_box(128, 128, 64, seed=args.seed + rank)
    for prec in ("fp64", "mixed"):
        try:
            s = rf.Solver.from_case(box, precision=prec)
            s.step()
            s.set_state(box.h0, 0.0)
            ms, steps = timed_run(s, box.t_end)
            mb = s.mass_balance()
            out[f"heterogeneous_box_128x128x64_{prec}"] = {
                "precision": prec, "simulated_s": box.t_end, "steps": len(steps), "time_to_solution_s": ms / 1e3,
                "picard_per_step": sum(x.picard for x in steps) / len(steps),
                "cg_iters": sum(x.cg for x in steps), "closure_rel": mb["closure_rel"],
                "value": len(steps) * box.n_active() / (ms / 1e3), "unit": UNIT}
            s.close()
        except Exception as ex:
            out[f"heterogeneous_box_128x128x64_{prec}"] = {"error": str(ex)[:200]}
    return out


def warmstart_leg(args, rank, rf, W, peaks):
    import numpy as np
    import torch
    from paper_1809_10895_gb300 import warmstart as WS

    def ev():
        return torch.cuda.Event(enable_timing=True)

    n_tr, n_ev = args.ws_train_size, args.ws_eval_size
    tc = W.heterogeneous_box(n_tr, n_tr, 64, seed=1000 + rank)
    sc = WS.scales_for(tc)
    s = rf.Solver.from_case(tc, precision="mixed")
    pilot = WS.collect(s, tc, sc, 16)
    sc.out_scale = WS.target_rms(pilot)
    del pilot
    s.close()
    # snapshots spread over the first day (rain, then redistribution)
    s = rf.Solver.from_case(tc, precision="mixed")
    a, b = ev(), ev()
    a.record(s.stream)
    snaps = WS.collect(s, tc, sc, args.ws_snapshots, t_end=86400.0, stride=4)
    b.record(s.stream)
    torch.cuda.synchronize()
    collect_ms = a.elapsed_time(b)
    s.close()
    net = rf.Network()
    net.set_params(W.nn_init_params(7 + rank))
    l0 = net.launch_count()
    a, b = ev(), ev()
    a.record(net.stream)
    losses = WS.train(net, snaps, steps=args.ws_train_steps, batch=1, lr=2e-3, log_every=max(1, args.ws_train_steps // 6))
    b.record(net.stream)
    torch.cuda.synchronize()
    train_ms = a.elapsed_time(b)
    train_launches = net.launch_count() - l0
    vox = tc.N
    flop_fwd = 2.0 * 27 * (8 * 32 + 8 * 32 * 32 + 32 * 8) * vox   # padded channels, per forward
    # forward (inference) kernel throughput on a held-out box
    ec = W.heterogeneous_box(n_ev, n_ev, 64, seed=2000 + rank)
    xf = torch.empty((1, 64, n_ev, n_ev, 4), dtype=torch.float32, device="cuda")
    yf = torch.empty((1, 64, n_ev, n_ev), dtype=torch.float32, device="cuda")
    se = rf.Solver.from_case(ec)
    se.ws_features(sc, 0.0, 600.0, xf.view(-1, 4))
    se.close()
    for _ in range(2):
        net.forward(xf, yf)
    a, b = ev(), ev()
    a.record(net.stream)
    reps = 5
    for _ in range(reps):
        net.forward(xf, yf)
    b.record(net.stream)
    torch.cuda.synchronize()
    fwd_ms = a.elapsed_time(b) / reps
    fwd_flop = 2.0 * 27 * (8 * 32 + 8 * 32 * 32 + 32 * 8) * ec.N
    bf16_peak = peaks.get("bf16_tflops")
    runs = {}
    t0_ev = args.ws_eval_start * 3600.0
    t_eval = t0_ev + args.ws_eval_hours * 3600.0
    max_diff = 0.0
    for seed in range(args.ws_eval_seeds):
        ec = W.heterogeneous_box(n_ev, n_ev, 64, seed=2000 + 97 * seed + rank)
        # the window's start state (inside the rain, dt grown), spun up by the plain mixed path
        sp = rf.Solver.from_case(ec, precision="mixed")
        sp.run(t0_ev)
        h_s = torch.empty(ec.N, dtype=torch.float64, device="cuda")
        sp.get_state_device(h_s)
        meta_s = sp.get_state()[1]
        sp.close()
        states = {}
        for prec in ("fp64", "mixed"):
            for warm in (False, True):
                key = f"{'warm' if warm else 'plain'}_{prec}"
                s = rf.Solver.from_case(ec, precision=prec)
                if warm:
                    s.ws_attach(net, sc)
                s.step()                            # graph capture, workspaces: outside the timing
                s.set_state_device(h_s, t0_ev)
                s.set_meta(meta_s)
                if warm:
                    s.ws_attach(net, sc)            # counters from zero
                a, b = ev(), ev()
                a.record(s.stream)
                steps = picard = rej = 0
                t = t0_ev
                while t < t_eval * (1 - 1e-12):
                    info = s.step()
                    t = info.t
                    steps += 1
                    picard += info.picard
                    rej += info.rejected
                b.record(s.stream)
                torch.cuda.synchronize()
                r = runs.setdefault(key, {"steps": 0, "picard": 0, "rejected": 0, "ms": 0.0, "fallbacks": 0,
                                          "guesses": 0})
                r["steps"] += steps
                r["picard"] += picard
                r["rejected"] += rej
                r["ms"] += a.elapsed_time(b)
                if warm:
                    st = s.ws_stats()
                    r["fallbacks"] += st["fallbacks"]
                    r["guesses"] += st["guesses"]
                states[key] = s.get_state()[0]
                s.close()
        for prec in ("fp64", "mixed"):
            max_diff = max(max_diff, float(np.max(np.abs(states[f"warm_{prec}"] - states[f"plain_{prec}"]))))
    # equal-accuracy check at an identical step sequence (fixed dt = 300 s):
    # the warm-started and plain solutions differ only within the Picard tolerance
    ec = W.heterogeneous_box(n_ev, n_ev, 64, seed=2000 + rank)
    fixed = {}
    for warm in (False, True):
        s = rf.Solver.from_case(ec, precision="mixed", dt0=300.0, f_grow=1.0)
        if warm:
            s.ws_attach(net, sc)
        its = [s.step().picard for _ in range(12)]
        fixed["warm" if warm else "plain"] = (s.get_state()[0], sum(its))
        s.close()
    fixed_diff = float(np.max(np.abs(fixed["warm"][0] - fixed["plain"][0])))
    for r in runs.values():
        r["picard_per_step"] = r["picard"] / max(r["steps"], 1)
        r["time_to_solution_s"] = r["ms"] / 1e3
        r["ms_per_picard"] = r["ms"] / max(r["picard"], 1)
        if r["guesses"]:
            r["fallback_rate"] = r["fallbacks"] / r["guesses"]
    # break-even: the guess (one forward pass per step) pays when it saves
    # more Picard iterations per step than forward_ms / (ms per Picard iteration)
    pm, wm = runs["plain_mixed"], runs["warm_mixed"]
    break_even = {"forward_ms_per_guess": fwd_ms, "plain_mixed_ms_per_picard": pm["ms_per_picard"],
                  "picard_saved_needed_per_step": fwd_ms / pm["ms_per_picard"],
                  "picard_saved_per_step": pm["picard_per_step"] - wm["picard_per_step"],
                  "plain_fp64_ms_per_picard": runs["plain_fp64"]["ms_per_picard"]}
    return {
        "train_workload": f"heterogeneous_box_{n_tr}x{n_tr}x64", "eval_workload": f"heterogeneous_box_{n_ev}x{n_ev}x64",
        "eval_seeds": args.ws_eval_seeds, "eval_window_s": [t0_ev, t_eval], "snapshots": len(snaps),
        "break_even": break_even,
        "snapshot_collect_ms": collect_ms, "train_steps": args.ws_train_steps, "train_ms": train_ms,
        "train_voxels_per_s": args.ws_train_steps * vox / (train_ms / 1e3),
        "train_tflops": 3 * flop_fwd * args.ws_train_steps / (train_ms / 1e3) / 1e12,
        "train_kernel_launches": train_launches, "loss_log": losses,
        "forward_ms": fwd_ms, "forward_tflops": fwd_flop / (fwd_ms / 1e3) / 1e12,
        "forward_frac_of_bf16_peak": (fwd_flop / (fwd_ms / 1e3) / 1e12 / bf16_peak) if bf16_peak else None,
        "runs": runs, "max_abs_h_diff_warm_vs_plain_ebats_m": max_diff,
        "fixed_dt_check": {"dt_s": 300.0, "steps": 12, "max_abs_h_diff_m": fixed_diff,
                           "picard_plain": fixed["plain"][1], "picard_warm": fixed["warm"][1]},
        "speedup_warm_mixed_vs_plain_fp64": runs["plain_fp64"]["ms"] / runs["warm_mixed"]["ms"],
    }


# ---------------------------------------------------------- reference arm
def reference(args):
    """The CPU oracle, as it stands, on the same workload, window and metric:
    its OpenMP build on all host cores (the one-thread build where gcc cannot
    build that).  The oracle spins the watershed up from t = 0 to the window's
    start itself (untimed), then times the window's first steps, at most K and
    at most about a minute of them."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1809_10895_gb300 import workloads as W
    from tests.helpers import oracle_from_case
    O.build()
    O.build(openmp=True)
    case = W.watershed(512, 512, 64, seed=args.seed, hours=720)
    t0_win = storm_start(case)
    threads = O.num_threads(openmp=True)          # all host cores; 0: one-thread build only
    o = oracle_from_case(case, openmp=threads > 0)
    cores = max(threads, 1)
    w0 = time.perf_counter()
    o.run(t0_win)
    spin = time.perf_counter() - w0
    k, dt, pic = oracle_steps(o, max(1, args.steps), 60.0)
    v = k * case.n_active() / dt
    sample = (f"accepted steps 1..{k} of the timed window of {WORKLOAD} (from t = {t0_win / 3600:.0f} h, "
              f"{pic} Picard iterations, {dt:.1f} s) after an untimed spin-up from t = 0 ({spin:.0f} s); C oracle, "
              + (f"OpenMP, {threads} threads" if threads else "one thread"))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": k, "warmup": 0,
        "ms_per_step": dt * 1e3 / k, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded diamond-square terrain, sampled soil layers, Poisson storms; no dataset)",
        "config": config_dict({"window": f"steps from t = {t0_win / 3600:.0f} h (the first hour of the seed's first "
                                         f"storm), state spun up from t = 0 untimed", "precision": "fp64"}),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference(a)
    else:
        native(a)
