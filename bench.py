"""Benchmark of the multiresolution step on one GB300 (or N replicas/shards).

Metric: adaptive grid points x RK stages per second, where the points of a step
are sum over the blocks of the adapted grid G (before the safety refinement) of
Bs^d, times 4 stages; the time is the whole mr_step (refine-all, 4 x (ghost
sync + RK stage), coarsening rounds, tree rebuild).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload adv3d|swirl|adv2d]
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)

Prints one JSON line on rank 0.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Synthetic workloads shaped like the paper's runs: analytic initial fields, seeded parameters.
WORKLOADS = {
    # 3D linear advection, Gaussian sigma 0.04, u = (1,1,1), 17^3 blocks, Jmax 6,
    # eps 1e-4, FP32 stencils + FP64 details, Hilbert-ordered pool.
    "adv3d": dict(dim=3, Bs=17, precision="fp32", detail_fp64=True, rhs="adv",
                  tree=dict(Jmin=2, Jmax=6, eps=1e-4, ic="gauss",
                            ic_params=(0.5, 0.5, 0.5, 0.04), rhs_params=(1.0, 1.0, 1.0)),
                  umax=math.sqrt(3.0), capacity=20_000,
                  name="3D advection, Gaussian sigma 0.04, u=(1,1,1), 17^3 blocks, ng 4, "
                       "Jmin 2, Jmax 6, eps 1e-4, FP32 RHS + FP64 details, CFL 0.5"),
    # 2D swirl (Sec. 3, Eq. 1), t_a = 5, 17^2 blocks, Jmax 8, eps 1e-4, FP32 + FP64 details
    "swirl": dict(dim=2, Bs=17, precision="fp32", detail_fp64=True, rhs="swirl",
                  tree=dict(Jmin=1, Jmax=8, eps=1e-4, ic="gauss",
                            ic_params=(0.5, 0.75, 0.0, math.sqrt(0.005)), rhs_params=(5.0,)),
                  umax=1.0, capacity=60_000, full_time=5.0,
                  name="2D swirl t_a=5, blob (0.5,0.75) beta 0.01, 17^2 blocks, Jmax 8, eps 1e-4, "
                       "FP32 RHS + FP64 details, CFL 0.5"),
    # 2D constant advection, plain FP64
    "adv2d": dict(dim=2, Bs=17, precision="fp64", detail_fp64=False, rhs="adv",
                  tree=dict(Jmin=2, Jmax=5, eps=1e-3, ic="gauss",
                            ic_params=(0.5, 0.5, 0.0, 0.05), rhs_params=(1.0, 0.5, 0.0)),
                  umax=math.hypot(1.0, 0.5), capacity=20_000,
                  name="2D advection u=(1,0.5), sigma 0.05, 17^2 blocks, Jmin 2, Jmax 5, eps 1e-3, FP64"),
}


def dt_of(w):
    t = w["tree"]
    dx = 1.0 / ((w["Bs"] - 1) * (1 << t["Jmax"]))
    return 0.5 * dx / w["umax"]


def bytes_per_stage_block(w):
    """Algorithmic bytes of one RK stage over one block, averaged over the 4
    stages: 16 array passes per step over Bs^d nodes (3 + 5 + 5 + 3)."""
    n = w["Bs"] ** w["dim"]
    if w["precision"] == "fp64":
        return 16 * n * 8 / 4
    if w["precision"] == "fp32":
        return 16 * n * 4 / 4
    return (10 * n * 8 + 6 * n * 4) / 4  # FP64 y_n / acc, FP32 stage fields


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(w, seconds_target=15.0):
    """Times the FP64 CPU oracle (single thread) on a bounded sample of the
    workload: same physics, Jmax reduced so a step takes seconds; returns
    (points x stages / s, description)."""
    import oracle
    t = dict(w["tree"])
    jmax = {3: 3, 2: 5}[w["dim"]]
    jmin = min(t["Jmin"], jmax - 1)
    cfg = dict(dim=w["dim"], Bs=w["Bs"], Jmin=jmin, Jmax=jmax, eps=t["eps"], rhs=w["rhs"],
               rhs_params=t["rhs_params"], ic="gauss", ic_params=t["ic_params"])
    o = oracle.Oracle(cfg)
    o.init_tree()
    dx = 1.0 / ((w["Bs"] - 1) * (1 << jmax))
    dt = 0.5 * dx / w["umax"]
    pts, steps, t0 = 0, 0, time.perf_counter()
    while True:
        pts += o.n * w["Bs"] ** w["dim"] * 4
        o.step(steps * dt, dt)
        steps += 1
        if time.perf_counter() - t0 > seconds_target or steps >= 200:
            break
    el = time.perf_counter() - t0
    desc = ("FP64 oracle, 1 thread, %d step(s) of the same workload with Jmin %d, Jmax %d "
            "(%d..%d blocks)" % (steps, jmin, jmax, o.n, o.n))
    return pts / el, desc, steps, el


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build_oracle()
    per_step = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    vals = []
    for s in range(args.warmup + args.steps):
        v, desc, _, _ = oracle_sample(w, seconds_target=per_step)
        if s >= args.warmup:
            vals.append(v)
    value = sum(vals) / len(vals)
    line = {"metric": "adaptive grid-points x RK-stages/sec", "value": value,
            "unit": "points*stages/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w["name"] + " (oracle sample)", "l2_flush": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "points*stages/s", "cores": 1,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "points*stages/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="swirl", choices=sorted(WORKLOADS))
    ap.add_argument("--capacity", type=int, default=0)
    ap.add_argument("--eps", type=float, default=0.0)
    ap.add_argument("--no-full", action="store_true",
                    help="swirl: do not run on to t = t_a for the error (timed window only)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--spinup", type=int, default=-1,
                    help="untimed steps after init before warm-up (default per workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    w = dict(WORKLOADS[args.workload])
    w["tree"] = dict(w["tree"])
    if args.eps > 0:
        w["tree"]["eps"] = args.eps
        w["name"] = w["name"].replace("eps %g" % WORKLOADS[args.workload]["tree"]["eps"], "eps %g" % args.eps)
    if args.capacity > 0:
        w["capacity"] = args.capacity
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import torch
    import numpy as np
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00088_gb300 as mr

    stream = torch.cuda.Stream()
    # Independent replicas per rank (the path has no exchange between trees);
    # each rank advances its own instance: weak scaling.
    g = mr.Forest(dim=w["dim"], Bs=w["Bs"], precision=w["precision"], detail_fp64=w["detail_fp64"],
                  rhs=w["rhs"], trees=[w["tree"]], capacity=w["capacity"],
                  stream=stream.cuda_stream)
    B, d = w["Bs"], w["dim"]
    npts = B ** d
    dt = dt_of(w)
    g.init_tree()
    t = 0.0
    full = "full_time" in w and not args.no_full
    nfull = int(math.ceil(w["full_time"] / dt)) if "full_time" in w else 0
    if full:
        dt = w["full_time"] / nfull  # land exactly on t = t_a
    if args.spinup >= 0:
        spin = args.spinup
    elif "full_time" in w:
        # time the window around t_a / 2, where the deformation and the grid peak
        spin = max(0, nfull // 2 - args.warmup - args.steps // 2)
    else:
        spin = 0
    for _ in range(spin + args.warmup):
        g.step(t, dt)
        t += dt
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    # ---- timed region: K full steps, device timing with CUDA events ----
    g.reset_stats()
    g.enable_timing(True)
    launches0 = g.launch_count()
    nb = g.num_blocks()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    points = 0
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            points += nb * npts * 4
            g.step(t, dt)
            t += dt
            nb = g.num_blocks()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = g.launch_count() - launches0
    st = g.stats()
    g.enable_timing(False)
    ms_t = torch.tensor([ms], device="cuda")
    if world > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = points * world / (ms_max / 1e3)

    # roofline of the dominant kernel (RK stage): algorithmic bytes / stage time
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    stage_ms = st["ms"]["stage"]
    stage_bytes = st["stage_blocks"] * bytes_per_stage_block(w)
    achieved = stage_bytes / (stage_ms / 1e3) / 1e9 if stage_ms > 0 else 0.0
    per_launch_us = stage_ms * 1e3 / max(1, st["stage_launches"])
    err = g.error(0, t) if w["rhs"] == "adv" else None
    nsteps_done = spin + args.warmup + args.steps
    if full:
        # continue untimed to t = t_a, where the swirl returns to the initial state
        for s_ in range(nsteps_done, nfull):
            g.step(s_ * dt, dt)
        t = nfull * dt
        err = g.error(0, 0.0)

    # ---- end-to-end through the C ABI with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        info, f = g.get_blocks()
        k2 = max(1, min(args.steps, 5))
        ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pts2, bi, bo = 0, 0, 0
        torch.cuda.synchronize()
        ev2.record(stream)
        for _ in range(k2):
            n = len(info)
            lvl = torch.from_numpy(np.ascontiguousarray(info["level"])).pin_memory().numpy()
            crd = torch.from_numpy(np.ascontiguousarray(info["coords"])).pin_memory().numpy()
            fld = torch.from_numpy(f).pin_memory().numpy()
            g.set_blocks(lvl, crd, fld)
            bi += lvl.nbytes + crd.nbytes + fld.nbytes
            pts2 += n * npts * 4
            g.step(t, dt)
            t += dt
            info, f = g.get_blocks()
            bo += info.nbytes + f.nbytes
        ev3.record(stream)
        torch.cuda.synchronize()
        e2e_ms = ev2.elapsed_time(ev3)
        e2e = {"value": pts2 / (e2e_ms / 1e3), "unit": "points*stages/s",
               "h2d_bytes_per_step": bi // k2, "d2h_bytes_per_step": bo // k2,
               "steps": k2, "api": "mr_set_blocks (host) + mr_step + mr_get_blocks (host)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, desc, steps, el = oracle_sample(w)
        cpu = {"value": v, "unit": "points*stages/s", "cores": 1, "kind": "oracle",
               "sample": desc + ", %.1f s" % el}

    if rank == 0:
        line = {
            "metric": "adaptive grid-points x RK-stages/sec",
            "value": value, "unit": "points*stages/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32 (f64 details)", "fp64": "f64", "fp32_acc64": "f32/f64"}[w["precision"]],
            "data": "synthetic",
            "config": {"workload": w["name"], "blocks_at_end": nb, "Bs": B, "dim": d,
                       "dt": dt, "parallelism": "replicas" if world > 1 else "single",
                       "l2_flush": "no flush; working set per step (stage fields over the "
                                   "refined grid) exceeds the 129 MB L2" if args.workload == "adv3d"
                                   else "no flush; small working set (L2-resident)",
                       "l2_rel_error": None if err is None else err["l2"],
                       "linf_rel_error": None if err is None else err["linf"],
                       "error_at_t": t if err is not None else None,
                       "timed_window_t": [(spin + args.warmup) * dt, (spin + args.warmup + args.steps) * dt],
                       "phase_ms": st["ms"]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "k_stage_adv (RK stage incl. fused ghost gather)",
                         "stage_launch_us": per_launch_us, "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
            "gpu_launches": launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        if clk.summary():
            line["clocks"] = clk.summary()
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
