"""Event-timed launches of single solver / network kernels on a workload
(``rf_profile_kernel`` for the solver kernels, ``rf_nn_forward`` for the
network), for profiling one kernel at a time.

    python -m paper_1809_10895_gb300.kernel_timing box --kinds assemble,resid64
    python -m paper_1809_10895_gb300.kernel_timing watershed --nx 512 --ny 256 --kinds cg32_spmv
    python -m paper_1809_10895_gb300.kernel_timing watershed --nx 512 --ny 256 --precision fp64 --t-start 11 \
        --kinds closure,assemble,cg64_spmv,cg64_update
    python -m paper_1809_10895_gb300.kernel_timing network --nx 128 --ny 128 --nz 64
    python -m paper_1809_10895_gb300.kernel_timing training --nx 128 --ny 128 --nz 64
    python -m paper_1809_10895_gb300.kernel_timing ensemble --instances 64 --window 10 --cluster 4

Prints one JSON line: per kind the mean launch time and the algorithmic bytes
per launch (solver kernels), or the forward / training-step time and TFLOP/s
(network), or the persistent ensemble launch time with per-instance busy
times (ensemble).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["box", "watershed", "network", "training", "ensemble"])
    ap.add_argument("--nx", type=int, default=None)
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--nz", type=int, default=64)
    ap.add_argument("--kinds", default="assemble,closure,resid64,cg32_spmv,cg32_update")
    ap.add_argument("--steps", type=int, default=5, help="accepted steps before timing (box)")
    ap.add_argument("--t-start", type=float, default=0.0,
                    help="watershed: simulated hours run before timing (11: the first storm of seed 0)")
    ap.add_argument("--reps", type=int, default=24)
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--instances", type=int, default=64, help="ensemble instances")
    ap.add_argument("--window", type=float, default=10.0, help="simulated seconds (ensemble)")
    ap.add_argument("--cluster", type=int, default=4, help="CTAs per cluster (ensemble)")
    ap.add_argument("--threads", type=int, default=512, help="threads per CTA (ensemble)")
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "zline"],
                    help="inner PCG preconditioner (ensemble, mixed precision)")
    a = ap.parse_args(argv)

    import torch
    from paper_1809_10895_gb300 import build, rf
    from paper_1809_10895_gb300 import workloads as W
    build.build()
    rf.load()
    torch.cuda.set_device(0)
    out = {"workload": a.workload}
    if a.workload == "ensemble":
        cases = W.ensemble(a.instances, seed=0)
        e = rf.Ensemble.from_cases(cases, precision=a.precision,
                                   **({"precond": a.precond} if a.precond != "jacobi" else {}))
        e.set_tiling(a.cluster, a.threads)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(e.stream)
        e.run(a.window)
        e1.record(e.stream)
        torch.cuda.synchronize()
        st = [e.get(i, want_h=False)[1] for i in range(len(cases))]
        out.update(instances=a.instances, window_s=a.window, cluster=a.cluster, threads=a.threads,
                   ms=e0.elapsed_time(e1), cell_timesteps=sum(x["steps"] * x["cells"] for x in st),
                   cg_iters=sum(x["cg_iters"] for x in st), max_busy_s=max(x["busy_s"] for x in st),
                   failed=sum(1 for x in st if x["status"] != 0))
        print(json.dumps(out))
        return
    if a.workload == "training":
        nx, ny = a.nx or 128, a.ny or 128
        shape = (1, a.nz, ny, nx)
        gen = torch.Generator(device="cuda").manual_seed(0)
        x = torch.randn(shape + (4,), device="cuda", generator=gen)
        t = torch.randn(shape, device="cuda", generator=gen)
        net = rf.Network()
        net.set_params(W.nn_init_params(1))
        for _ in range(2):
            net.train_step(x, t, want_loss=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(net.stream)
        for _ in range(a.reps):
            net.train_step(x, t, want_loss=False)
        e1.record(net.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        flop = 3 * 2.0 * 27 * (8 * 32 + 8 * 32 * 32 + 32 * 8) * x[..., 0].numel()
        out.update(shape=list(shape), train_step_ms=ms, tflops_3x_forward=flop / ms / 1e9)
    elif a.workload == "network":
        nx, ny = a.nx or 128, a.ny or 128
        shape = (1, a.nz, ny, nx)
        x = torch.randn(shape + (4,), device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
        y = torch.empty(shape, device="cuda")
        net = rf.Network()
        net.set_params(W.nn_init_params(1))
        for _ in range(2):
            net.forward(x, y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(net.stream)
        for _ in range(a.reps):
            net.forward(x, y)
        e1.record(net.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        flop = 2.0 * 27 * (8 * 32 + 8 * 32 * 32 + 32 * 8) * x[..., 0].numel()
        out.update(shape=list(shape), forward_ms=ms, tflops=flop / ms / 1e9)
    else:
        if a.workload == "box":
            case = W.heterogeneous_box(a.nx or 128, a.ny or 128, a.nz, seed=0)
        else:
            case = W.watershed(a.nx or 512, a.ny or 512, a.nz, seed=0, hours=24)
        s = rf.Solver.from_case(case, precision=a.precision)
        if a.workload == "box":
            for _ in range(a.steps):
                s.step()
        elif a.t_start > 0:
            s.run(a.t_start * 3600.0)
        out.update(cells=case.N, active=case.n_active(), kernels={})
        for k in a.kinds.split(","):
            ms, by = s.profile_kernel(k, reps=a.reps)
            out["kernels"][k] = {"us": ms * 1e3, "MB": by / 1e6, "GBps": by / ms / 1e6}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
