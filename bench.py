"""Benchmark: cell-timesteps/s of the Picard / backward-Euler / PCG Richards
solve on the 128x128x64 heterogeneous box (0.25 m cubes, log-normal Ks with
exponential covariance, hydrostatic start, 6 h of rain), Picard tolerance
1e-6 m.

One "step" is one accepted backward-Euler time step: every Picard iteration
(closures, assembly, PCG solve, global max|dh| test), EBATS reruns and the
water balance.  ``value`` is the FP32-inner / FP64-defect-correction path
(closures, Picard test and mass balance in FP64); the plain FP64 path is
reported beside it.  Inputs are resident in HBM; L2 is flushed between timed
steps.  ``e2e`` drives the same steps through the C ABI from pinned host
buffers (state uploaded and downloaded every step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

With N > 1 (torchrun, one rank per GPU) every rank runs an independent replica
(different seed): the solve of one box does not shard without a halo
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

WORKLOAD = "heterogeneous_box_128x128x64"
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
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-pcg-hbm", action="store_true", help="skip the large-grid PCG kernel bandwidth leg")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble leg")
    ap.add_argument("--ensemble-window", type=float, default=600.0, help="simulated seconds of the ensemble leg")
    ap.add_argument("--no-warmstart", action="store_true", help="skip the learned warm-start leg")
    ap.add_argument("--no-configs", action="store_true", help="skip the column and watershed step legs")
    ap.add_argument("--config-steps", type=int, default=20, help="timed steps of the watershed step leg")
    ap.add_argument("--ws-train-size", type=int, default=128, help="nx = ny of the training box (nz = 64)")
    ap.add_argument("--ws-eval-size", type=int, default=256, help="nx = ny of the held-out boxes (nz = 64)")
    ap.add_argument("--ws-eval-seeds", type=int, default=1, help="held-out seeds evaluated")
    ap.add_argument("--ws-snapshots", type=int, default=64, help="training snapshots (accepted plain steps)")
    ap.add_argument("--ws-train-steps", type=int, default=600, help="Adam steps (one full box per step)")
    ap.add_argument("--ws-eval-hours", type=float, default=1.0, help="simulated hours of each held-out run")
    return ap.parse_args()


def config_dict(extra=None):
    d = {"workload": WORKLOAD, "cells": 128 * 128 * 64, "cell_size_m": 0.25, "lnKs_sigma": 1.0,
         "corr_len_cells": 8, "picard_tol_m": 1e-6, "cg_tol_rel": 1e-10, "ebats": "dt0 1 s, x1.3, max 600 s",
         "step": "one accepted backward-Euler step from t=0 after warm-up", "l2": "flushed between timed steps"}
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
def oracle_steps(case, n_steps=None, budget_s=20.0, openmp=False):
    """Time the CPU oracle (as it stands: one thread, or the same source built
    with OpenMP on all cores) on the first accepted steps of the same
    workload; stops at n_steps or after budget_s."""
    from tests.helpers import oracle_from_case
    o = oracle_from_case(case, openmp=openmp)
    t0 = time.perf_counter()
    k = 0
    while (n_steps is None or k < n_steps) and time.perf_counter() - t0 < budget_s:
        o.step()
        k += 1
    dt = time.perf_counter() - t0
    return k, dt


def oracle_threads():
    """Threads of the OpenMP build of the oracle (0 when it cannot be built)."""
    from oracle import oracle as O
    return O.num_threads(openmp=True)


def cpu_baseline(case, budget_s=20.0):
    """The oracle on the host cores: the OpenMP build on all of them, with the
    one-thread build beside it, both over the same first steps (as many as the
    one-thread build takes in half the budget)."""
    k1, t1 = oracle_steps(case, None, budget_s / 2)
    single = {"value": k1 * case.n_active() / t1, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"first {k1} accepted steps of {WORKLOAD} from t=0 ({t1:.1f} s, one-thread C oracle)"}
    threads = oracle_threads()
    if threads < 1:
        return dict(single, note="OpenMP build of the oracle unavailable (gcc -fopenmp failed)")
    k, t = oracle_steps(case, k1, budget_s / 2, openmp=True)
    return {"value": k * case.n_active() / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {k} accepted steps of {WORKLOAD} from t=0 ({t:.1f} s, C oracle built with "
                      f"OpenMP, {threads} threads)",
            "single_thread": single}


def oracle_configs(args, W):
    """The oracle on the other workloads, bounded samples of each: the 1-D
    column over the GPU leg's timed steps (one thread), the first accepted
    steps of the watershed from t = 0 (OpenMP build), and a stratified sample
    of the ensemble's instances from t = 0 within its window (one thread)."""
    from tests.helpers import oracle_from_case

    def steps_within(o, budget_s, max_steps=None, t_stop=None):
        t0 = time.perf_counter()
        k = 0
        while (max_steps is None or k < max_steps) and time.perf_counter() - t0 < budget_s:
            info = o.step()
            k += 1
            if t_stop is not None and info.t >= t_stop - 1e-9:
                break
        return k, time.perf_counter() - t0

    out = {}
    col = W.infiltration_column()
    o = oracle_from_case(col)
    for _ in range(5):
        o.step()
    k, dt = steps_within(o, 10.0, max_steps=400)
    out["infiltration_column_1x1x200"] = {
        "value": k * col.N / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": f"accepted steps 6..{5 + k} from t=0 (the GPU leg's timed steps), one-thread C oracle"}
    del o
    threads = oracle_threads()
    ws = W.watershed(512, 512, 64, seed=args.seed, hours=24)
    o = oracle_from_case(ws, openmp=threads > 0)
    k, dt = steps_within(o, 10.0)
    out["watershed_512x512x64"] = {
        "value": k * ws.n_active() / dt, "unit": UNIT, "cores": max(threads, 1), "kind": "oracle",
        "sample": f"first {k} accepted steps from t=0 ({dt:.1f} s, C oracle"
                  + (f", OpenMP, {threads} threads)" if threads else ", one thread)")}
    del o
    cases = W.ensemble(256, seed=args.seed)
    by_size = sorted(range(len(cases)), key=lambda i: cases[i].N)
    sample = by_size[8::32]
    cell_steps, total = 0, 0.0
    for i in sample:
        o = oracle_from_case(cases[i])
        k, dt = steps_within(o, 1.5, t_stop=args.ensemble_window)
        cell_steps += k * cases[i].n_active()
        total += dt
        del o
    out["ensemble_256_uneven"] = {
        "value": cell_steps / total, "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": f"{len(sample)} of the 256 instances (every 32nd by size), each from t=0 for at most 1.5 s "
                  f"or {args.ensemble_window:g} s simulated, one-thread C oracle"}
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


def profile_entry(kernel):
    """The committed ncu summary of a kernel; None when absent or taken on a
    different kernel source."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
        e = d["kernels"][kernel]
        src = open(os.path.join(ROOT, "paper_1809_10895_gb300", "csrc", e["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != e["source_sha"]:
            return None
        return e
    except Exception:
        return None


def traffic_for(kernel, cells):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    workload's cells."""
    e = profile_entry(kernel)
    return None if e is None else e["dram_bytes_per_launch"] * cells / e["cells"]


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
    case = W.heterogeneous_box(seed=args.seed + rank)
    n_act = case.n_active()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed_run(precision):
        s = rf.Solver.from_case(case, precision=precision)
        stream = s.stream
        for _ in range(args.warmup):
            s.step()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        c0 = s.launch_counts()
        picard = cg = rej = 0
        barrier()
        w0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            info = s.step()
            ends[i].record(stream)
            picard += info.picard
            cg += info.cg
            rej += info.rejected
        barrier()
        wall = time.perf_counter() - w0
        ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
        c1 = s.launch_counts()
        counts = {k: (c1[k][0] - c0[k][0], c1[k][1] - c0[k][1]) for k in c1}
        return s, ms, wall, counts, dict(picard=picard, cg=cg, rejected=rej)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)        # let the sampler start before the timed region
    s_mix, ms_mix, wall_mix, counts_mix, st_mix = timed_run("mixed")
    clk = clocks.stop()
    s64, ms64, wall64, counts64, st64 = timed_run("fp64")
    launches_mix = sum(v[0] for v in counts_mix.values())

    t_mix, t64 = max_over_ranks(ms_mix / 1e3, world, "cuda"), max_over_ranks(ms64 / 1e3, world, "cuda")
    value = job_value(args.steps * n_act, world, t_mix)
    value64 = job_value(args.steps * n_act, world, t64)

    # ---- per-kernel device times on the state reached (roofline)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    kern = {}
    for kind in ("closure", "assemble", "resid64", "cg32_spmv", "cg32_update", "cg64_spmv", "cg64_update"):
        avg_ms, by = s_mix.profile_kernel(kind, reps=30)
        kern[kind] = {"avg_ms": avg_ms, "bytes": by, "gbs": by / (avg_ms * 1e-3) / 1e9}
    # device time of each kernel in the timed region: launches that did work
    # (device counters) x mean launch time (events); the closure kernel that
    # ends a Picard iteration does the work of the timed closure kernel
    work = {"closure": counts_mix["closure_picard"][1] + counts_mix["closure"][1],
            "assemble": counts_mix["assemble"][1], "resid64": counts_mix["resid64"][1],
            "cg32_spmv": counts_mix["cg32_spmv"][1], "cg32_update": counts_mix["cg32_update"][1]}
    est = {k: work[k] * kern[k]["avg_ms"] for k in work}
    tot_est = sum(est.values())
    dom = max(est, key=lambda k: est[k])
    kd = kern[dom]
    names = {"closure": "k_closure_picard", "assemble": "k_assemble", "resid64": "k_resid64",
             "cg32_spmv": "k_cg32_spmv", "cg32_update": "k_cg32_update"}
    roof = {"kernel": names[dom], "bound": "hbm", "achieved": kd["gbs"], "peak": hbm_peak, "unit": "GB/s",
            "frac": kd["gbs"] / hbm_peak, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": traffic_for(names[dom], n_act), "algorithmic_bytes_per_launch": kd["bytes"],
            "avg_launch_ms": kd["avg_ms"]}
    # FP64-pipe roof: GB300 issues 2 FP64 thread instructions per clock per
    # SM; a kernel whose FP64 arithmetic takes longer at that rate than its
    # bytes at the HBM peak is bound by the FP64 pipe (reported as "alu")
    ent = profile_entry(names[dom])
    if ent and ent.get("fp64_arith_inst_per_cell"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        fp64_peak = 2.0 * sms * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e9   # G FP64 instructions / s
        fp64_inst = ent["fp64_arith_inst_per_cell"] * n_act
        if fp64_inst / (fp64_peak * 1e9) > kd["bytes"] / (hbm_peak * 1e9):
            achieved = fp64_inst / (kd["avg_ms"] * 1e-3) / 1e9
            roof = {"kernel": names[dom], "bound": "alu", "achieved": achieved, "peak": fp64_peak,
                    "unit": "G FP64 inst/s", "frac": achieved / fp64_peak,
                    "peak_source": f"derived: 2 FP64 instructions/clk/SM x {sms} SMs x "
                                   f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz (MEASURED_PEAKS.json sm_max_mhz)",
                    "traffic": traffic_for(names[dom], n_act), "algorithmic_fp64_inst_per_launch": fp64_inst,
                    "fp64_arith_inst_per_cell": ent["fp64_arith_inst_per_cell"],
                    "fp64_pipe_active_pct_ncu": ent.get("fp64_pipe_active_pct"),
                    "algorithmic_bytes_per_launch": kd["bytes"], "avg_launch_ms": kd["avg_ms"],
                    "hbm": {"achieved": kd["gbs"], "peak": hbm_peak, "unit": "GB/s", "frac": kd["gbs"] / hbm_peak}}

    # ---- PCG stencil kernels on a grid far larger than L2 (HBM regime):
    # the 512x512x64 watershed (16.8 M cells), kernels timed by events
    pcg_hbm = None
    if not args.no_pcg_hbm:
        ws = W.watershed(512, 512, 64, seed=args.seed + rank, hours=24)
        sw = rf.Solver.from_case(ws, precision="mixed")
        pcg_hbm = {"workload": "watershed_512x512x64", "cells": ws.N, "active_cells": ws.n_active(),
                   "peak_gbs": hbm_peak, "kernels": {}}
        for kind in ("cg32_spmv", "cg32_update", "cg64_spmv", "cg64_update", "resid64"):
            avg_ms, by = sw.profile_kernel(kind, reps=20)
            gbs = by / (avg_ms * 1e-3) / 1e9
            pcg_hbm["kernels"][kind] = {"avg_us": avg_ms * 1e3, "algorithmic_MB": by / 1e6, "GBps": gbs,
                                        "frac_of_hbm_peak": gbs / hbm_peak}
        sw.close()
        del sw
        # one stiff solve on that grid (x0 = 0, dt = 600 s): inner FP32 PCG
        # preconditioned by Jacobi vs by the multigrid V-cycle
        hk = torch.as_tensor(ws.h0, dtype=torch.float64, device="cuda")
        pcg_hbm["solve_x0_zero"] = {}
        for pc in ("jacobi", "mg", "dic"):
            try:
                sv = rf.Solver.from_case(ws, precision="mixed", precond=pc)
                sv.assemble(hk, hk, 600.0, 0.0)
                res = None
                for rep in range(2):                      # the first call captures the graph
                    x = torch.zeros(ws.N, dtype=torch.float64, device="cuda")
                    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(sv.stream)
                    its = sv.solve(x)
                    b_.record(sv.stream)
                    torch.cuda.synchronize()
                    res = {"inner_iterations": its, "ms": a.elapsed_time(b_)}
                pcg_hbm["solve_x0_zero"][pc] = res
                sv.close()
                del sv
            except Exception as ex:                       # recorded, not fatal to the other legs
                pcg_hbm["solve_x0_zero"][pc] = {"error": str(ex)[:200]}

    # ---- batched ensemble: 256 uneven instances (1 cm cells, footprints
    # 1..16 x 1..16, depths 50..400) in one persistent graph-launched kernel
    ens = None
    if not args.no_ensemble:
        cases = W.ensemble(256, seed=args.seed + rank)
        e = rf.Ensemble.from_cases(cases, precision="mixed")
        cluster, cta_threads, n_wide, probe_ms = e.tune(min(20.0, args.ensemble_window))
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(e.stream)
        e.run(args.ensemble_window)
        ev1.record(e.stream)
        torch.cuda.synchronize()
        ens_ms = ev0.elapsed_time(ev1)
        cell_steps = 0
        stats = [e.get(i, want_h=False)[1] for i in range(len(cases))]
        cell_steps = sum(st["steps"] * st["cells"] for st in stats)
        ens = {"workload": "ensemble_256_uneven", "instances": len(cases), "cells": sum(c.N for c in cases),
               "simulated_window_s": args.ensemble_window, "cluster_ctas": cluster, "cta_threads": cta_threads, "wide_instances": n_wide,
               "tuner_probe_ms": probe_ms,
               "kernel_ms": ens_ms, "cell_timesteps": cell_steps, "value": cell_steps / (ens_ms * 1e-3),
               "unit": UNIT, "steps_total": sum(st["steps"] for st in stats),
               "picard_total": sum(st["picard_iters"] for st in stats),
               "failed_instances": sum(1 for st in stats if st["status"] != 0), "precision": "mixed"}
        e.close()
        del e

    # ---- learned warm start: snapshots from the plain solver on one box,
    # Adam training by the library's kernels, then held-out boxes run with and
    # without the network's first Picard iterate (same tolerance, same EBATS)
    wsl = None
    if not args.no_warmstart:
        wsl = warmstart_leg(args, rank, rf, W, peaks)

    # ---- the other synthetic configurations, whole steps: the 1-D column
    # (plain FP64 path) and the 512x512x64 watershed (mixed, Jacobi and MG)
    cfg = None
    if not args.no_configs:
        cfg = configs_leg(args, rank, rf, W)

    # ---- end to end through host buffers
    e2e = None
    if not args.no_e2e:
        s = rf.Solver.from_case(case, precision="mixed")
        for _ in range(args.warmup):
            s.step()
        h_pin = torch.empty(case.N, dtype=torch.float64, pin_memory=True)
        h_np = h_pin.numpy()
        h_np[:], meta = s.get_state()
        mb = s.mass_balance()
        mass7 = [mb["storage0"], 0, mb["inflow_cum"], mb["outflow_cum"], 0, 0, mb["nonlinear_defect_cum"]]
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s.set_state(h_np, meta["t"])
            s.set_meta(meta, mass7)
            s.step()
            h_np[:], meta = s.get_state()
        barrier()
        te = time.perf_counter() - t0
        te = max_over_ranks(te, world, "cuda")
        e2e = {"value": job_value(args.steps * n_act, world, te), "unit": UNIT, "h2d_bytes_per_step": 8 * case.N,
               "d2h_bytes_per_step": 8 * case.N}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_mix * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner PCG / f64 closures, residual, Picard test",
            "data": "synthetic (seeded Gaussian random field, no dataset)",
            "config": config_dict({"precision": "mixed", "parallelism": "replicas" if world > 1 else "single GPU",
                                   "picard_iters": st_mix["picard"], "cg_inner_iters": st_mix["cg"],
                                   "rejected": st_mix["rejected"], "wall_s": wall_mix}),
            "plain_fp64": {"value": value64, "unit": UNIT, "ms_per_step": t64 * 1e3 / args.steps,
                           "picard_iters": st64["picard"], "cg_iters": st64["cg"], "wall_s": wall64},
            "speedup_mixed_vs_fp64": value / value64,
            "gpu_launches": launches_mix,
            "launch_counts": {k: {"launched": v[0], "worked": v[1]} for k, v in counts_mix.items() if v[0]},
            "kernel_time_shares": {k: {"launches": work[k], "est_ms": est[k], "share_of_step_time":
                                       est[k] / (t_mix * 1e3)} for k in est},
            "roofline": roof,
            "kernels": {k: {"avg_us": v["avg_ms"] * 1e3, "GBps": v["gbs"]} for k, v in kern.items()},
            "clocks": clk,
            "e2e": e2e,
            "pcg_hbm": pcg_hbm,
            "ensemble": ens,
            "warmstart": wsl,
            "other_configs": cfg,
        }
        if not args.no_baseline:
            # host-side legs: an error is recorded in the line, never lost with it
            try:
                line["cpu_baseline"] = cpu_baseline(case)
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


def configs_leg(args, rank, rf, W):
    import torch

    def timed_steps(s, n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        picard = 0
        for _ in range(n):
            picard += s.step().picard
        b.record(s.stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), picard

    out = {}
    col = W.infiltration_column()
    s = rf.Solver.from_case(col, precision="fp64")
    for _ in range(5):
        s.step()
    n = 400
    ms, pic = timed_steps(s, n)
    out["infiltration_column_1x1x200"] = {"precision": "fp64", "steps": n, "ms_per_step": ms / n,
                                          "picard_per_step": pic / n, "value": n * col.N / (ms / 1e3), "unit": UNIT,
                                          "note": "200 cells: launch- and synchronisation-bound"}
    s.close()
    ws = W.watershed(512, 512, 64, seed=args.seed + rank, hours=24)
    for pc in ("jacobi", "mg", "dic"):
        try:
            s = rf.Solver.from_case(ws, precision="mixed", precond=pc)
            for _ in range(3):
                s.step()
            n = args.config_steps
            ms, pic = timed_steps(s, n)
            out[f"watershed_512x512x64_{pc}"] = {"precision": "mixed", "precond": pc, "steps": n,
                                                  "ms_per_step": ms / n, "picard_per_step": pic / n,
                                                  "active_cells": ws.n_active(),
                                                  "value": n * ws.n_active() / (ms / 1e3), "unit": UNIT}
            s.close()
        except Exception as ex:                           # recorded, not fatal to the other legs
            out[f"watershed_512x512x64_{pc}"] = {"error": str(ex)[:200]}
    # the benchmark box with the classical (chord) and the modified Picard
    # linearisation (Sec. 2.2), mixed precision, same steps from t = 0
    box = W.heterogeneous_box(128, 128, 64, seed=args.seed + rank)
    for form in ("chord", "modified"):
        s = rf.Solver.from_case(box, precision="mixed", picard_form=form)
        for _ in range(args.warmup):
            s.step()
        n = args.steps
        ms, pic = timed_steps(s, n)
        mb = s.mass_balance()
        scale = mb["storage0"] + mb["inflow_cum"] + mb["outflow_cum"]
        out[f"heterogeneous_box_128x128x64_{form}_picard"] = {
            "precision": "mixed", "picard_form": form, "steps": n, "ms_per_step": ms / n,
            "picard_per_step": pic / n, "simulated_s": s.get_state()[1]["t"],
            "closure_rel": mb["closure_rel"], "nonlinear_defect_rel": abs(mb["nonlinear_defect_cum"]) / scale,
            "value": n * box.n_active() / (ms / 1e3), "unit": UNIT}
        s.close()
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
    t_eval = args.ws_eval_hours * 3600.0
    max_diff = 0.0
    for seed in range(args.ws_eval_seeds):
        ec = W.heterogeneous_box(n_ev, n_ev, 64, seed=2000 + 97 * seed + rank)
        states = {}
        for prec in ("fp64", "mixed"):
            for warm in (False, True):
                key = f"{'warm' if warm else 'plain'}_{prec}"
                s = rf.Solver.from_case(ec, precision=prec)
                if warm:
                    s.ws_attach(net, sc)
                s.step()                            # graph capture, workspaces: outside the timing
                h0 = torch.as_tensor(ec.h0, dtype=torch.float64, device="cuda")
                s.set_state_device(h0, 0.0)
                if warm:
                    s.ws_attach(net, sc)            # counters from zero
                a, b = ev(), ev()
                a.record(s.stream)
                steps = picard = rej = 0
                t = 0.0
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
        if r["guesses"]:
            r["fallback_rate"] = r["fallbacks"] / r["guesses"]
    return {
        "train_workload": f"heterogeneous_box_{n_tr}x{n_tr}x64", "eval_workload": f"heterogeneous_box_{n_ev}x{n_ev}x64",
        "eval_seeds": args.ws_eval_seeds, "eval_window_s": t_eval, "snapshots": len(snaps),
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
    """The CPU oracle, as it stands, on the same workload and metric: its
    OpenMP build on all host cores, or the one-thread build where gcc cannot
    build that."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1809_10895_gb300 import workloads as W
    O.build()
    case = W.heterogeneous_box(seed=args.seed)
    # each step is one accepted oracle step; warm-up and timed steps are
    # bounded so the whole run stays within a few minutes
    w = min(args.warmup, 3)
    k = max(1, min(args.steps, 40))
    from tests.helpers import oracle_from_case
    threads = O.num_threads(openmp=True)          # all host cores; 0: one-thread build only
    o = oracle_from_case(case, openmp=threads > 0)
    cores = max(threads, 1)
    for _ in range(w):
        o.step()
    t0 = time.perf_counter()
    for _ in range(k):
        o.step()
    dt = time.perf_counter() - t0
    v = k * case.n_active() / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": k, "warmup": w,
        "ms_per_step": dt * 1e3 / k, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded Gaussian random field, no dataset)", "config": config_dict(),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"accepted steps {w + 1}..{w + k} of {WORKLOAD} (C oracle, "
                                   + (f"OpenMP, {threads} threads)" if threads else "one thread)")},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference(a)
    else:
        native(a)
