"""Benchmark of the multiresolution step on one GB300 (or N replicas/shards).

Metric: adaptive grid points x RK stages per second, where the points of a step
are sum over the blocks of the adapted grid G (before the safety refinement) of
Bs^d, times 4 stages; the time is the whole mr_step (refine-all, 4 x (ghost
sync + RK stage), coarsening rounds, tree rebuild).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload adv3d|swirl|adv2d|forest|ns|ns_thin|dsl|...]
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
    # 64 independent 2D advection instances (seeded), one context, graph replays
    "forest": dict(dim=2, Bs=17, precision="fp32", detail_fp64=True, rhs="adv",
                   trees=None, capacity=600_000,
                   name="64 independent 2D advection trees (seeded: sigma 0.02-0.1, |u_i|<=1, "
                        "Jmax 4-8, eps 1e-5..1e-3), 17^2 blocks, FP32 RHS + FP64 details"),
    # 2D compressible Navier-Stokes temporal mixing layer (Sec. 4 setup, reduced):
    # u = 0.5 tanh(2y/delta), delta 0.1, Mach 0.3, Re 1000, seeded perturbation
    # 1e-3; 4 conserved variables, FP32 stages and details (eps 1e-3 of the
    # normalised variables is far above FP32 resolution) with FP64
    # state/accumulator; 33^2 blocks, Jmax 7, eps 1e-3; learned refinement proposal
    # trained on the run's own adapt decisions.
    "ns": dict(dim=2, Bs=33, nvar=4, norm_kind=1, precision="fp32_acc64", detail_fp64=False, rhs="ns",
               tree=None, capacity=20_000, oracle_jmax=4, learned=dict(collect_steps=60, epochs=6),
               name="2D NS temporal mixing layer (delta 0.1, Ma 0.3, Re 1000, seeded perturbation 1e-3), "
                    "33^2 blocks, Jmin 2, Jmax 7, eps 1e-3, FP32 stages and details + FP64 state/acc, "
                    "learned proposal, CFL 0.5"),
    # The same flow with the layer thickness of the paper's Sec. 4 run relative
    # to its domain (1/240 of the box): the grid adapts to the layer and to the
    # roll-up, which a delta of 0.1 resolved at the coarsest level never needs.
    "ns_thin": dict(dim=2, Bs=33, nvar=4, norm_kind=1, precision="fp32_acc64", detail_fp64=False, rhs="ns",
                    tree=None, capacity=60_000, oracle_jmax=4, spinup=1500,
                    learned=dict(collect_steps=100, epochs=6),
                    name="2D NS temporal mixing layer, delta 1/240 (Ma 0.3, Re 1000, seeded perturbation "
                         "1e-3), 33^2 blocks, Jmin 2, Jmax 7, eps 1e-3, FP32 stages and details + FP64 state/acc, "
                         "learned proposal, CFL 0.5"),
    # The double shear layer of Sec. 4 as the paper runs it: L = 8, layers at
    # x = L/2 -+ 0.25 (rho 2/1, v 1/-1, width L/240), p = 2.5, u = 0.1 sin(2 pi
    # (y - L/2)), mu 1e-6, gamma 1.4, Pr 0.71, skew-symmetric form, shock filter
    # r_th 1e-5 after every step, eps 1e-3; 17^2 blocks, Jmax 7; FP32 stages and
    # details with FP64 state/accumulator.  Timed at t = 3, when the acoustic
    # waves have filled about three quarters of the finest level.
    "dsl": dict(dim=2, Bs=17, nvar=4, norm_kind=1, precision="fp32_acc64", detail_fp64=False,
                rhs="ns_skew", L=8.0, capacity=60_000, oracle_jmax=4, spinup=4410,
                tree=dict(Jmin=2, Jmax=7, eps=1e-3, ic="shear_layer",
                          ic_params=(2.0, 1.0, 1.0, -1.0, 8.0 / 240.0, 2.5, 0.1, 0.25, 4.0, 4.0),
                          rhs_params=(1.4, 1e-6, 0.71, 1e-5)),
                umax=1.0 + math.sqrt(1.4 * 2.5 / 1.0),  # |v| + c in the light layer
                name="2D NS double shear layer of Sec. 4 (L 8, rho 2/1, v +-1, lw L/240, p 2.5, mu 1e-6), "
                     "skew-symmetric form + shock filter r_th 1e-5, 17^2 blocks, Jmin 2, Jmax 7, eps 1e-3, "
                     "FP32 stages and details + FP64 state/acc, CFL 0.5, timed from t = 3"),
    # Uniform grids at the finest level (no adaptation happens): the stage
    # kernel at a size where HBM bandwidth matters.
    "uniform2d": dict(dim=2, Bs=17, precision="fp32", detail_fp64=True, rhs="adv",
                      tree=dict(Jmin=9, Jmax=9, eps=1e-3, ic="gauss", ic_params=(0.5, 0.5, 0.0, 0.05),
                                rhs_params=(1.0, 0.5, 0.0)),
                      umax=math.hypot(1.0, 0.5), capacity=(1 << 18) + 64,
                      name="2D advection on a uniform grid of 512^2 blocks of 17^2 (Jmin = Jmax = 9), FP32"),
    "uniform3d": dict(dim=3, Bs=17, precision="fp32", detail_fp64=True, rhs="adv",
                      tree=dict(Jmin=5, Jmax=5, eps=1e-4, ic="gauss", ic_params=(0.5, 0.5, 0.5, 0.04),
                                rhs_params=(1.0, 1.0, 1.0)),
                      umax=math.sqrt(3.0), capacity=(1 << 15) + 64,
                      name="3D advection on a uniform grid of 32^3 blocks of 17^3 (Jmin = Jmax = 5), FP32"),
    "adv2d": dict(dim=2, Bs=17, precision="fp64", detail_fp64=False, rhs="adv",
                  tree=dict(Jmin=2, Jmax=5, eps=1e-3, ic="gauss",
                            ic_params=(0.5, 0.5, 0.0, 0.05), rhs_params=(1.0, 0.5, 0.0)),
                  umax=math.hypot(1.0, 0.5), capacity=20_000,
                  name="2D advection u=(1,0.5), sigma 0.05, 17^2 blocks, Jmin 2, Jmax 5, eps 1e-3, FP64"),
}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum), averaged
# over the launches of one step (the four RK stages; the details of the
# coarsening rounds; the filter), from an ncu capture per workload (profiles/),
# valid only for the device sources it was taken on (the digest in each entry);
# otherwise reported as null.
TRAFFIC = {
    # workload: {kernel: DRAM bytes per launch}, plus the digest of the device sources it was taken on
    "adv3d": {"digest": ("DEVICE", "1001c46c9ab0dc4b"), "stage": (36.01e6 + 99.01e6 + 98.98e6 + 60.53e6) / 4,
              "details": (32.93e6 + 6.51e6 + 7.59e6 + 2.80e6) / 4},
    "dsl": {"digest": ("NS", "2a19634679daf7a6"), "stage": (279.74e6 + 336.89e6 + 336.16e6 + 289.24e6) / 4,
            "details": (113.75e6 + 11.25e6 + 4.95e6 + 2.66e6) / 4,
            "filter": 71.71e6},
}


DEVICE_SOURCES = ("mr_device.cuh", "mr_internal.h", "mr_kernels.cuh", "mr_launch.cuh")
NS_SOURCES = DEVICE_SOURCES + ("mr_ns.cuh",)  # the skew-symmetric stage and the shock filter


def source_digest(names=DEVICE_SOURCES):
    """Digest of device code (kernels, device helpers, launch configuration), without its
    comments and blank lines (an edited comment does not change a kernel)."""
    import hashlib
    import re
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1902_00088_gb300", "csrc")
    for f in [os.path.join(csrc, n) for n in names]:
        h.update(os.path.basename(f).encode())
        with open(f) as fh:
            code = [re.sub(r"//.*", "", l).rstrip() for l in fh]
        h.update("\n".join(l for l in code if l).encode())
    return h.hexdigest()[:16]


def _forest_trees():
    import synthetic as inputs
    return inputs.forest_trees(64)


WORKLOADS["forest"]["trees"] = _forest_trees()


def _mixing_layer_tree(seed=20190201, delta=0.1):
    import synthetic as inputs
    a, phi = inputs.mixing_layer_perturbation(seed)
    U0, Ma, gam, amp = 0.5, 0.3, 1.4, 1e-3
    return dict(Jmin=2, Jmax=7, eps=1e-3, ic="mixing",
                ic_params=(delta, U0, Ma, gam, amp) + tuple(a) + tuple(phi),
                rhs_params=(gam, U0 * delta / 1000.0, 0.71), x0=(0.0, -0.5, 0.0))


WORKLOADS["ns"]["tree"] = _mixing_layer_tree()
WORKLOADS["ns_thin"]["tree"] = _mixing_layer_tree(delta=1.0 / 240.0)
WORKLOADS["ns"]["umax"] = WORKLOADS["ns_thin"]["umax"] = 0.5 + 0.5 / 0.3  # |u| + c0


def dt_of(w):
    t = w["tree"]
    dx = w.get("L", 1.0) / ((w["Bs"] - 1) * (1 << t["Jmax"]))
    return 0.5 * dx / w["umax"]


def bytes_per_stage_block(w):
    """Algorithmic bytes of one RK stage over one block, averaged over the 4
    stages: 16 array passes per step over Bs^d nodes (3 + 5 + 5 + 3)."""
    n = w["Bs"] ** w["dim"] * w.get("nvar", 1)
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
        # Sampling starts before the timed region; the first sample is awaited
        # so that the sampler is running when the region begins.
        import threading
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self
        first = threading.Event()

        def reader():
            for l in self.proc.stdout:
                if l.strip():
                    self.lines.append((time.perf_counter(), l))
                    first.set()
            first.set()

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        first.wait(10.0)
        self.t0 = time.perf_counter()
        return self

    def __exit__(self, *a):
        if self.proc:
            self.t1 = time.perf_counter()
            time.sleep(0.05)  # one more sample after the region
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)
        # samples taken inside the region, else the ones bracketing it
        inside = [l for (t, l) in self.lines if self.t0 <= t <= self.t1] if self.proc else []
        if not inside and self.proc:
            before = [l for (t, l) in self.lines if t < self.t0][-1:]
            after = [l for (t, l) in self.lines if t > self.t1][:1]
            inside = before + after
            self.bracketed = True
        self.lines = inside

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
        out = {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
               "samples": len(sm)}
        if getattr(self, "bracketed", False):
            out["note"] = "region shorter than the sampling interval: samples just before and after it"
        return out


def oracle_sample(w, seconds_target=15.0):
    """Times the FP64 CPU oracle (single thread) on a bounded sample of the
    workload: same physics, Jmax reduced so a step takes seconds; returns
    (points x stages / s, description, steps, elapsed seconds)."""
    import oracle
    t = dict(w["tree"] if "tree" in w else w["trees"][0])
    umax = w.get("umax") or math.hypot(*t["rhs_params"][:2]) or 1.0
    jmax = w.get("oracle_jmax") or {3: 3, 2: 5}[w["dim"]]
    jmin = min(t["Jmin"], jmax - 1)
    cfg = dict(dim=w["dim"], Bs=w["Bs"], nvar=w.get("nvar", 1), Jmin=jmin, Jmax=jmax, eps=t["eps"],
               rhs=w["rhs"], rhs_params=t["rhs_params"], ic=t.get("ic", "gauss"), ic_params=t["ic_params"],
               norm_kind=w.get("norm_kind", 0), L=w.get("L", 1.0))
    if "x0" in t:
        cfg["x0"] = t["x0"]
    o = oracle.Oracle(cfg)
    o.init_tree()
    dx = w.get("L", 1.0) / ((w["Bs"] - 1) * (1 << jmax))
    dt = 0.5 * dx / umax
    pts, steps, t0 = 0, 0, time.perf_counter()
    while True:
        pts += o.n * w["Bs"] ** w["dim"] * 4
        o.step(steps * dt, dt)
        steps += 1
        if time.perf_counter() - t0 > seconds_target or steps >= 200:
            break
    el = time.perf_counter() - t0
    desc = ("FP64 oracle, 1 thread, %d step(s) of the same workload with Jmin %d, Jmax %d "
            "(%d blocks at the end) instead of the timed Jmin %d, Jmax %d; rate per adapted point and stage"
            % (steps, jmin, jmax, o.n, t["Jmin"], t["Jmax"]))
    return pts / el, desc, steps, el


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build_oracle()
    per_step = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    vals, ms = [], []
    for s in range(args.warmup + args.steps):
        v, desc, nst, el = oracle_sample(w, seconds_target=per_step)
        if s >= args.warmup:
            vals.append(v)
            ms.append(1e3 * el / max(1, nst))
    value = sum(vals) / len(vals)
    # ms_per_step: wall time of one oracle step of the sample (a reduced grid, stated in cpu_baseline)
    line = {"metric": "adaptive grid-points x RK-stages/sec", "value": value,
            "unit": "points*stages/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w["name"] + " (oracle sample)", "l2_flush": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "points*stages/s", "cores": 1,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "points*stages/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def swirl_study(jmaxs=(4, 5), epss=(1e-3, 1e-4, 1e-5, 1e-6), betas=(1e-2,), bs=33, uniform=False):
    """The swirl study of Sec. 3 (Fig. 4A-D as data): 33^2 blocks, blob beta 1e-2 at (0.5, 0.75), t_a 5,
    Jmin 1, CFL 0.5, plain FP64, steps replayed as CUDA graphs up to t_a; per run the error against the
    initial field, the adapted grid's size against the uniform one and the time per step.  uniform: the
    equidistant grid at each Jmax instead (Jmin = Jmax, one run per Jmax; Fig. 4D's comparison)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00088_gb300 as mr
    stream = torch.cuda.Stream()
    t_a = 5.0
    for beta, jmax, eps in ((b, j, e) for b in betas for j in jmaxs for e in (epss[:1] if uniform else epss)):
        # Sec. 3: phi_0 = exp(-r^2 / beta) = exp(-r^2 / (2 sigma^2)), sigma = sqrt(beta / 2)
        tree = dict(Jmin=jmax if uniform else 1, Jmax=jmax, eps=eps, ic="gauss",
                    ic_params=(0.5, 0.75, 0.0, math.sqrt(beta / 2)), rhs_params=(t_a,))
        g = mr.Forest(dim=2, Bs=bs, precision="fp64", rhs="swirl", trees=[tree], capacity=400_000,
                      stream=stream.cuda_stream)
        g.init_tree()
        n = int(math.ceil(t_a / (0.5 / ((bs - 1) * (1 << jmax)))))
        g.set_time(0.0, t_a / n)
        g.step_graph(1)  # captures the step graph (untimed)
        g.step_history(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        g.step_graph(n - 1)
        e1.record(stream)
        torch.cuda.synchronize()
        el = e0.elapsed_time(e1) / 1e3
        hist = g.step_history(reset=True)
        err = g.error(0, 0.0)
        print(json.dumps(dict(study="swirl33", grid="uniform" if uniform else "adaptive", Bs=bs, beta=beta, Jmax=jmax,
                              eps=None if uniform else eps, steps=n, l2=err["l2"], linf=err["linf"],
                              blocks_mean=float(np.mean(hist)), blocks_max=int(np.max(hist)),
                              uniform_blocks=4 ** jmax, ms_per_step=1e3 * el / (n - 1),
                              timing="CUDA events around graph replays 2..n on the context's stream")),
              flush=True)
        del g


def swirl_half_study(jmaxs=(5, 6), epss=(1e-3, 1e-4, 1e-5, 1e-6), betas=(1e-2, 1e-4), bs=33, jref=7,
                     uniform_jmaxs=(4, 5, 6)):
    """Fig. 4D of Sec. 3 as data: error at t_a / 2 (the swirl's largest deformation) against a reference, for
    adaptive grids (Jmin 1, Jmax, eps) and equidistant ones (Jmin = Jmax), with the GPU time to get there.
    The paper's reference is pseudo-spectral; here it is the equidistant grid at level jref (4th order in
    space and time, far finer than the runs compared).  Errors over the unique nodes of each run, relative,
    L2 weighted by dx^2 and Linf; plain FP64, CFL 0.5 at each run's finest level, steps as graph replays."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00088_gb300 as mr
    stream = torch.cuda.Stream()
    t_a = 5.0

    def run(beta, jmin, jmax, eps):
        tree = dict(Jmin=jmin, Jmax=jmax, eps=eps, ic="gauss", ic_params=(0.5, 0.75, 0.0, math.sqrt(beta / 2)),
                    rhs_params=(t_a,))
        g = mr.Forest(dim=2, Bs=bs, precision="fp64", rhs="swirl", trees=[tree], capacity=400_000,
                      stream=stream.cuda_stream)
        g.init_tree()
        n = int(math.ceil(t_a / (0.5 / ((bs - 1) * (1 << jmax)))))
        n += n % 2  # t_a / 2 after n / 2 steps
        g.set_time(0.0, t_a / n)
        g.step_graph(1)  # captures the step graph (untimed)
        g.step_history(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        g.step_graph(n // 2 - 1)
        e1.record(stream)
        torch.cuda.synchronize()
        hist = g.step_history(reset=True)
        info, f = g.get_blocks()
        del g
        return n // 2, e0.elapsed_time(e1) / (n // 2 - 1), float(np.mean(hist)), info, f

    for beta in betas:
        _, ref_ms, _, info, f = run(beta, jref, jref, 1e-3)
        ref = uniform_field(info, f, bs, jref)[0]
        cases = [("uniform", j, j, None) for j in uniform_jmaxs] + [("adaptive", 1, j, e) for j in jmaxs for e in epss]
        for kind, jmin, jmax, eps in cases:
            steps, ms, bmean, info, f = run(beta, jmin, jmax, eps if eps else 1e-3)
            l2, linf = error_vs_reference(info, f[:, 0], ref, bs, jref)
            print(json.dumps(dict(study="swirl33_half", grid=kind, Bs=bs, beta=beta, Jmax=jmax, eps=eps,
                                  steps=steps, l2=l2, linf=linf, blocks_mean=bmean,
                                  ms_per_step=ms, gpu_s=ms * steps / 1e3, reference="equidistant level %d" % jref,
                                  timing="CUDA events around graph replays 2..n/2 on the context's stream")),
                  flush=True)


def error_vs_reference(info, f, ref, Bs, jref):
    """Relative errors (L2 weighted by dx^2, Linf) of the blocks' field f (n x Bs x Bs, 2D) against a
    periodic reference on the uniform node grid of level jref; each block's unique nodes (its last node per
    axis dropped) are nodes of the reference lattice."""
    import numpy as np
    Nr = ref.shape[0]
    e2 = r2 = ei = ri = 0.0
    ii = np.arange(Bs - 1)
    for lv in np.unique(info["level"]):
        sel = info["level"] == lv
        sc = 1 << (jref - int(lv))
        cx = info["coords"][sel, 0].astype(np.int64)
        cy = info["coords"][sel, 1].astype(np.int64)
        X = ((cx[:, None] * (Bs - 1) + ii[None, :]) * sc) % Nr
        Y = ((cy[:, None] * (Bs - 1) + ii[None, :]) * sc) % Nr
        rv = ref[Y[:, :, None], X[:, None, :]]
        d = f[sel, : Bs - 1, : Bs - 1] - rv
        w = (1.0 / ((Bs - 1) << int(lv))) ** 2
        e2 += w * float((d * d).sum())
        r2 += w * float((rv * rv).sum())
        ei = max(ei, float(np.abs(d).max()))
        ri = max(ri, float(np.abs(rv).max()))
    return math.sqrt(e2 / r2), ei / ri


def uniform_field(info, f, Bs, J):
    """Blocks all at level J -> the periodic node grid (n_var, N, N), N = (Bs-1) 2^J
    (each block's last node per axis is its neighbour's first and is dropped)."""
    import numpy as np
    N = (Bs - 1) << J
    out = np.zeros((f.shape[1], N, N))
    for q in range(len(info)):
        cx, cy = int(info["coords"][q][0]), int(info["coords"][q][1])
        out[:, cy * (Bs - 1):(cy + 1) * (Bs - 1), cx * (Bs - 1):(cx + 1) * (Bs - 1)] = f[q, :, :Bs - 1, :Bs - 1]
    return out


def kinetic_energy_spectrum(psi_x, psi_y, L):
    """Shell-summed spectrum of the kinetic energy density |psi|^2 / 2 (psi = sqrt(rho) u):
    E(k) = sum over |k'| in [k - 1/2, k + 1/2) of |psi_hat(k')|^2 / 2, wavenumbers in units of
    2 pi / L, normalised so that sum_k E(k) is the mean kinetic energy density (Parseval)."""
    import numpy as np
    N = psi_x.shape[0]
    ex = np.fft.fft2(psi_x) / (N * N)
    ey = np.fft.fft2(psi_y) / (N * N)
    e = 0.5 * (np.abs(ex) ** 2 + np.abs(ey) ** 2)
    k1 = np.fft.fftfreq(N, 1.0 / N)
    kk = np.sqrt(k1[None, :] ** 2 + k1[:, None] ** 2)
    shell = np.rint(kk).astype(np.int64)
    return np.bincount(shell.ravel(), weights=e.ravel())[: N // 2 + 1]


def dsl_study(jmaxs=(7, 8), fixed=(7,), eps=1e-3, bs=17, t_end=4.0, form="fp32_acc64"):
    """The double shear layer of Sec. 4 (Fig. 6 as data): adaptive runs (Jmin 2, eps) at each Jmax and
    fixed grids at each level of `fixed`, advanced by graph replays to t_end; per run the compression
    rate (blocks / 4^J) over time and the kinetic energy spectrum at t_end after refining the grid to
    its finest level."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00088_gb300 as mr
    w = WORKLOADS["dsl"]
    stream = torch.cuda.Stream()
    runs = [("adaptive", j) for j in jmaxs] + [("fixed", j) for j in fixed]
    for kind, J in runs:
        tree = dict(w["tree"])
        tree.update(Jmin=2 if kind == "adaptive" else J, Jmax=J, eps=eps)
        cap = int(1.3 * 4 ** J) + 20_000
        g = mr.Forest(dim=2, Bs=bs, nvar=4, precision=form, detail_fp64=False, rhs="ns_skew", trees=[tree],
                      capacity=cap, norm_kind=1, L=w["L"], stream=stream.cuda_stream)
        g.init_tree()
        dx = w["L"] / ((bs - 1) << J)
        n = int(math.ceil(t_end / (0.5 * dx / w["umax"])))
        dt = t_end / n
        g.set_time(0.0, dt)
        chunk = max(1, n // 40)
        comp, done, ms = [], 0, 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        status = "ok"
        try:
            while done < n:
                k = min(chunk, n - done)
                e0.record(stream)
                g.step_graph(k)
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                done += k
                comp.append((round(done * dt, 4), g.num_blocks() / 4 ** J))
            for _ in range(J):  # refine to the finest level for the spectrum
                info, _ = g.get_blocks(fields=False)
                lv = info["level"]
                if (lv == J).all():
                    break
                g.set_refine_mask((lv < J).astype(np.int8))
                g.adapt("refine_flagged")
            info, f = g.get_blocks()
            u = uniform_field(info, f, bs, J)
            spec = kinetic_energy_spectrum(u[1], u[2], w["L"])
            ks = [k for k in (1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048) if k < len(spec)]
            extra = dict(spectrum={str(k): float(spec[k]) for k in ks},
                         spectrum_sum=float(spec.sum()), rho_min=float((u[0] ** 2).min()),
                         rho_max=float((u[0] ** 2).max()))
        except mr.MRError as ex:
            status, extra = "failed: %s" % ex, {}
        print(json.dumps(dict(study="dsl", kind=kind, J=J, Jmin=tree["Jmin"], eps=eps, Bs=bs, form=form,
                              steps=done, t=done * dt, status=status, ms_per_step=ms / max(1, done),
                              compression=comp[:: max(1, len(comp) // 20)] + comp[-1:], **extra)), flush=True)
        del g


def reduce_over_ranks(ms, points, world):
    """Whole-job figures over the ranks: the slowest rank's time (the job ends
    with it) and the points all ranks advanced (each rank runs its own
    replica; nothing is exchanged during the steps)."""
    if world <= 1:
        return float(ms), float(points)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    p = torch.tensor([float(points)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def trees_of(w):
    return w["trees"] if "trees" in w else [w["tree"]]


def dts_of(w):
    if "trees" in w:
        import synthetic as inputs
        return [inputs.cfl_dt(t, w["Bs"]) for t in w["trees"]]
    return [dt_of(w)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="adv3d", choices=sorted(WORKLOADS))
    ap.add_argument("--capacity", type=int, default=0)
    ap.add_argument("--eps", type=float, default=0.0)
    ap.add_argument("--precision", default="", choices=["", "fp64", "fp32", "fp32_acc64"],
                    help="override the workload's arithmetic form (fp64 = plain FP64 method)")
    ap.add_argument("--no-full", action="store_true",
                    help="swirl: do not run on to t = t_a for the error (timed window only)")
    ap.add_argument("--eager", action="store_true", help="host-driven steps instead of CUDA graph replays")
    ap.add_argument("--autotune", type=int, default=-1, help="steps per autotuner candidate (0 = off)")
    ap.add_argument("--overlap", action="store_true", help="programmatic dependent launch of the step's kernels")
    ap.add_argument("--study", default="", choices=["", "swirl33", "swirl33_half", "dsl"],
                    help="instead of the benchmark: the paper's swirl study (33^2 blocks, eps x Jmax) or its double "
                         "shear layer (compression over time, energy spectra at t = 4), one JSON line per run")
    ap.add_argument("--study-t", type=float, default=4.0, help="dsl: end time")
    ap.add_argument("--study-fixed", default="7", help="dsl: comma-separated levels of the fixed-grid runs")
    ap.add_argument("--study-jmax", default="4,5", help="swirl33: comma-separated Jmax values")
    ap.add_argument("--study-eps", default="1e-3,1e-4,1e-5,1e-6", help="swirl33: comma-separated eps values")
    ap.add_argument("--study-beta", default="1e-2", help="swirl33: comma-separated pulse widths beta")
    ap.add_argument("--study-bs", type=int, default=33, help="swirl33: block size (the paper's study uses 33)")
    ap.add_argument("--study-uniform", action="store_true",
                    help="swirl33: equidistant grids at each Jmax instead of adaptive ones (Fig. 4D comparison)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--spinup", type=int, default=-1,
                    help="untimed steps after init before warm-up (default per workload)")
    ap.add_argument("--save-state", default="", help="write the state reached after spin-up + warm-up (npz)")
    ap.add_argument("--load-state", default="", help="start from a saved state instead of init + spin-up")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="refine all instead of the learned proposal")
    ap.add_argument("--learned", type=int, default=0,
                    help="train the proposal on this many refine-all steps after the spin-up, then time the "
                         "learned form (workloads without a proposal by default)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    w = dict(WORKLOADS[args.workload])
    if "tree" in w:
        w["tree"] = dict(w["tree"])
        if args.eps > 0:
            w["tree"]["eps"] = args.eps
            w["name"] = w["name"].replace("eps %g" % WORKLOADS[args.workload]["tree"]["eps"], "eps %g" % args.eps)
    if args.capacity > 0:
        w["capacity"] = args.capacity
    if args.learned > 0:
        w["learned"] = dict(collect_steps=args.learned, epochs=6)
        w["name"] += " [learned proposal]"
    if args.precision:
        w["precision"] = args.precision
        w["detail_fp64"] = args.precision != "fp32" or w["detail_fp64"]
        w["name"] += " [form: %s]" % args.precision
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return
    if args.study == "dsl":
        if rank == 0:
            jm = [int(x) for x in args.study_jmax.split(",")] if args.study_jmax != "4,5" else [7, 8]
            dsl_study(jmaxs=jm, fixed=[int(x) for x in args.study_fixed.split(",") if x],
                      eps=float(args.study_eps.split(",")[0]) if args.study_eps != "1e-3,1e-4,1e-5,1e-6" else 1e-3,
                      bs=args.study_bs if args.study_bs != 33 else 17, t_end=args.study_t)
        return
    if args.study == "swirl33_half":
        if rank == 0:
            swirl_half_study(jmaxs=[int(x) for x in args.study_jmax.split(",")],
                             epss=[float(x) for x in args.study_eps.split(",")],
                             betas=[float(x) for x in args.study_beta.split(",")], bs=args.study_bs)
        return
    if args.study:
        if rank == 0:
            swirl_study(jmaxs=[int(x) for x in args.study_jmax.split(",")],
                        epss=[float(x) for x in args.study_eps.split(",")],
                        betas=[float(x) for x in args.study_beta.split(",")], bs=args.study_bs,
                        uniform=args.study_uniform)
        return

    import numpy as np
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00088_gb300 as mr

    stream = torch.cuda.Stream()
    trees = trees_of(w)
    nt = len(trees)
    # Independent replicas per rank (trees never exchange data): weak scaling.
    g = mr.Forest(dim=w["dim"], Bs=w["Bs"], nvar=w.get("nvar", 1), precision=w["precision"],
                  detail_fp64=w["detail_fp64"], rhs=w["rhs"], trees=trees, capacity=w["capacity"],
                  norm_kind=w.get("norm_kind", 0), L=w.get("L", 1.0), stream=stream.cuda_stream)
    if args.overlap:
        g.set_launch_overlap(True)
    B, d = w["Bs"], w["dim"]
    npts = B ** d
    dts = np.array(dts_of(w))
    graph = not args.eager
    g.init_tree()
    full = "full_time" in w and not args.no_full
    nfull = int(math.ceil(w["full_time"] / dts[0])) if "full_time" in w else 0
    if full:
        dts[:] = w["full_time"] / nfull  # land exactly on t = t_a
    if args.spinup >= 0:
        spin = args.spinup
    elif "full_time" in w:
        # time the window around t_a / 2, where the deformation and the grid peak
        spin = max(0, nfull // 2 - args.warmup - args.steps // 2)
    else:
        spin = w.get("spinup", 0)
    t = np.zeros(nt)
    tuned = None
    steps_done = 0
    if args.load_state:
        z = np.load(args.load_state)
        g.set_blocks(z["level"], z["coords"], z["fields"], tree=z["tree"])
        t = z["t"].copy()
        steps_done = int(z["steps_done"])
        spin = 0
    if spin > 0:  # untimed evolution before the proposal is trained and the warm-up
        if graph:
            g.set_time(t, dts)
            g.step_graph(spin)
            t = g.get_time()
        else:
            for _ in range(spin):
                g.step(t, dts)
                t = t + dts
        steps_done += spin
    learned = None
    if w.get("learned") and not args.no_learned:
        # Train the proposal network on this run's own decisions: refine-all
        # steps record (tile features, was the refinement needed) pairs, then
        # the network is trained by the library's forward/backward/Adam kernels.
        import synthetic as inputs
        L = w["learned"]
        t0 = time.perf_counter()
        g.proposal_collect(True, 200_000)
        for _ in range(L["collect_steps"]):
            g.step(t, dts)
            t = t + dts
        steps_done += L["collect_steps"]
        nsamp, npos = g.proposal_dataset()
        init = inputs.cnn_init_params(mr.Forest.CNN_SHAPES, seed=20190201)
        g.proposal_collect(False)
        try:
            tau, loss = g.proposal_train(init, epochs=L["epochs"], batch=256, lr=1e-3, w_pos=0.0,
                                         recall=0.999, holdout=0.2)
        except mr.MRError as e:  # e.g. no positive sample: the step stays refine-all
            learned = {"collect_steps": L["collect_steps"], "samples": nsamp, "positives": npos,
                       "not_trained": str(e)}
        else:
            g.set_refine_mode("learned")
            g.proposal_stats(reset=True)
            learned = {"collect_steps": L["collect_steps"], "samples": nsamp, "positives": npos,
                       "epochs": L["epochs"], "tau": tau, "final_loss": loss,
                       "setup_s": time.perf_counter() - t0}
    if graph:
        g.set_time(t, dts)
        autotune = args.autotune if args.autotune >= 0 else (3 if "trees" in w else 0)
        if autotune > 0:
            t_ = g.autotune(autotune)
            form = (t_ // 100) % 10
            tuned = {"ctas_per_sm": t_ % 100 or "occupancy", "stage_form": ["cta per block", "warp per block"][form]}
            if form == 1:
                tuned.update(blocks_per_cta=(t_ // 1000) % 10, staging="bulk copies" if t_ // 10000 else "loads")
            steps_done += 7 * (autotune + 1) + 0
        g.step_graph(args.warmup)
        steps_done += args.warmup
    else:
        for _ in range(args.warmup):
            g.step(t, dts)
            t = t + dts
        steps_done += args.warmup
    if args.save_state:
        info, fl = g.get_blocks()
        tt = g.get_time() if graph else t
        np.savez(args.save_state, level=info["level"], tree=info["tree"], coords=info["coords"],
                 fields=fl, t=tt, steps_done=steps_done)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    # ---- timed region: K full steps, device timing with CUDA events ----
    g.reset_stats()
    g.enable_timing(not graph)
    g.step_history(reset=True)
    launches0 = g.launch_count()
    nb0 = g.num_blocks()
    # Between timed steps a buffer twice the L2 size is written (untimed), so
    # every step starts with its working set evicted from L2.
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    points = 0
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        nb = nb0
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0[k].record(stream)
            if graph:
                g.step_graph(1)
            else:
                points += nb * npts * 4
                g.step(t, dts)
                t = t + dts
            ev1[k].record(stream)
            if not graph:
                nb = g.num_blocks()
        torch.cuda.synchronize()
    per_step = [ev0[k].elapsed_time(ev1[k]) for k in range(args.steps)]
    ms = sum(per_step)
    per_step.sort()
    del flush
    launches = g.launch_count() - launches0
    if graph:
        hist = g.step_history(reset=True)
        points = int(hist.astype(np.int64).sum()) * npts * 4
    steps_done += args.steps
    nb = g.num_blocks()
    g.enable_timing(False)
    st = g.stats()
    ms_max, points_all = reduce_over_ranks(ms, points, world)
    value = points_all / (ms_max / 1e3)

    if learned is not None and "tau" in learned:
        learned["timed_region"] = g.proposal_stats(reset=True)
        learned["stage_blocks_per_step"] = st["stage_blocks"] / args.steps
        if graph:
            # The same state advanced by refine-all steps: the work and time the
            # proposal saves (untimed for the metric).
            k3 = 5
            g.set_refine_mode("all")
            g.step_graph(1)
            g.reset_stats()
            g.step_history(reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            g.step_graph(k3)
            e1.record(stream)
            torch.cuda.synchronize()
            ms3 = e0.elapsed_time(e1)
            h3 = g.step_history(reset=True)
            st3 = g.stats()
            learned["refine_all_same_state"] = {
                "steps": k3, "ms_per_step": ms3 / k3, "stage_blocks_per_step": st3["stage_blocks"] / k3,
                "value": int(h3.astype(np.int64).sum()) * npts * 4 / (ms3 / 1e3)}
            g.set_refine_mode("learned")
            steps_done += k3 + 1

    # Roofline of the dominant kernel (RK stage): algorithmic bytes / stage time.
    # The stage time comes from CUDA events around the RK phase in a separate
    # eager pass over the same grid (graph replays carry no per-phase events).
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    peak_source = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else \
        "6.8 TB/s copy bandwidth of an earlier GB300 measurement (of fallback)"
    if graph:
        g.reset_stats()
        g.enable_timing(True)
        tt = g.get_time()
        for k in range(3):
            g.step(tt, dts)
            tt = tt + dts
        g.enable_timing(False)
        st = g.stats()
        g.set_time(tt, dts)
        steps_done += 3
    # Algorithmic bytes: RK stage = 4 array passes over Bs^d nodes per block
    # (16 per step); details = one read of the synchronised block per block
    # evaluated.  Achieved = bytes / event time of the kernel's phase.
    kern = {}
    stage_ms = st["ms"]["stage"]
    kern["stage"] = dict(
        kernel="%s (RK stage incl. fused ghost gather)" % {"ns": "k_stage_ns", "ns_skew": "k_stage_nss"}.get(
            w["rhs"], "k_stage_adv"),
        ms=stage_ms, launches=st["stage_launches"], blocks=st["stage_blocks"],
        bytes=st["stage_blocks"] * bytes_per_stage_block(w))
    det_s = 4 if w["precision"] == "fp32" else 8
    kern["details"] = dict(
        kernel="k_details (ghost gather + wavelet details + block norms)", ms=st["ms"]["details"],
        launches=st["det_launches"], blocks=st["det_blocks"],
        bytes=st["det_blocks"] * (w["Bs"] ** w["dim"]) * w.get("nvar", 1) * det_s)
    if st["ms"].get("filter", 0.0) > 0:
        # shock filter: one read of the state's copy in the stage type and one
        # write of the state per block; it runs once per step on the list the four
        # stages saw
        fst = {"fp32": 4 + 4, "fp64": 8 + 8}.get(w["precision"], 4 + 8)
        fblocks = st["stage_blocks"] // 4
        kern["filter"] = dict(
            kernel="k_filter (shock filter incl. fused ghost gather, in place)", ms=st["ms"]["filter"],
            launches=st["calls"]["filter"], blocks=fblocks,
            bytes=fblocks * (w["Bs"] ** w["dim"]) * w.get("nvar", 1) * fst)
    for v in kern.values():
        v["achieved_gbs"] = v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else 0.0
        v["launch_us"] = v["ms"] * 1e3 / max(1, v["launches"])
    dom = max(kern, key=lambda n: kern[n]["ms"])
    achieved = kern[dom]["achieved_gbs"]
    # DRAM bytes per launch of the dominant kernel from an ncu capture of the
    # same device code, averaged over one step's launches of it, else null
    traffic, traffic_note = None, None
    twl = TRAFFIC.get(args.workload, {})
    tr = twl.get(dom)
    dig_ok = bool(twl) and source_digest(NS_SOURCES if twl["digest"][0] == "NS" else DEVICE_SOURCES) == twl["digest"][1]
    if tr and dig_ok and not args.precision and not args.learned:
        traffic = tr
        traffic_note = {"kernel": kern[dom]["kernel"],
                        "algorithmic_bytes_per_launch": kern[dom]["bytes"] / max(1, kern[dom]["launches"]),
                        "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the same device code, "
                                  "mean over one step's launches of the kernel"}

    err = None
    tnow = g.get_time() if graph else t
    if w["rhs"] == "adv" and nt == 1:
        err = g.error(0, float(tnow[0]))
    if full:
        # continue untimed to t = t_a, where the swirl returns to the initial state
        remaining = nfull - steps_done
        if remaining > 0:
            if graph:
                g.step_graph(remaining)
            else:
                for s_ in range(remaining):
                    g.step(tnow, dts)
                    tnow = tnow + dts
        err = g.error(0, 0.0)

    # ---- end-to-end through the C ABI with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        # pinned host buffers, allocated before the timed region: every step copies its
        # inputs from them and its result into them
        info, f = g.get_blocks()
        room = 4 * len(info) + 64
        pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()
        lvl_p, trs_p = pin((room,), torch.int32), pin((room,), torch.int32)
        crd_p = pin((room, 3), torch.int32)
        ib_p = pin((room * mr.BLOCK_INFO_DTYPE.itemsize,), torch.uint8).view(mr.BLOCK_INFO_DTYPE)
        fb_p = pin((room,) + f.shape[1:], torch.float64)
        fb_p[:len(info)] = f
        fld = fb_p[:len(info)]
        k2 = max(1, min(args.steps, 5))
        ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pts2, bi, bo = 0, 0, 0
        tt = g.get_time() if graph else tnow
        torch.cuda.synchronize()
        ev2.record(stream)
        for _ in range(k2):
            n = len(info)
            lvl_p[:n] = info["level"]
            trs_p[:n] = info["tree"]
            crd_p[:n] = info["coords"]
            g.set_blocks(lvl_p[:n], crd_p[:n], fld, tree=trs_p[:n])
            bi += lvl_p[:n].nbytes + trs_p[:n].nbytes + crd_p[:n].nbytes + fld.nbytes
            pts2 += n * npts * 4
            if graph:
                g.step_graph(1)
            else:
                g.step(tt, dts)
                tt = tt + dts
            info, fld = g.get_blocks(out=(ib_p, fb_p))
            bo += info.nbytes + fld.nbytes
        ev3.record(stream)
        torch.cuda.synchronize()
        e2e_ms = ev2.elapsed_time(ev3)
        e2e = {"value": pts2 / (e2e_ms / 1e3), "unit": "points*stages/s",
               "h2d_bytes_per_step": bi // k2, "d2h_bytes_per_step": bo // k2,
               "steps": k2, "api": "mr_set_blocks (pinned host) + mr_step + mr_get_blocks (pinned host)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, desc, steps, el = oracle_sample(w)
        cpu = {"value": v, "unit": "points*stages/s", "cores": 1, "kind": "oracle",
               "sample": desc + ", %.1f s" % el}

    if rank == 0:
        pct = lambda q: per_step[min(len(per_step) - 1, int(round(q * (len(per_step) - 1))))]
        line = {
            "metric": "adaptive grid-points x RK-stages/sec",
            "value": value, "unit": "points*stages/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32 (f64 details)", "fp64": "f64", "fp32_acc64": "f32/f64"}[w["precision"]],
            "data": "synthetic",
            "config": {"workload": w["name"], "trees": nt, "blocks_at_start": nb0, "blocks_at_end": nb,
                       "Bs": B, "dim": d, "dt": float(dts[0]) if nt == 1 else "per tree",
                       "mode": "eager" if not graph else "cuda-graph step replay (%s rounds)" % g.graph_mode(),
                       "autotuned": tuned,
                       "launch_overlap": g.launch_overlap(),
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2_flush": "256 MiB written between timed steps (untimed)",
                       "step_ms_p50": pct(0.5), "step_ms_p99": pct(0.99),
                       "l2_rel_error": None if err is None else err["l2"],
                       "linf_rel_error": None if err is None else err["linf"],
                       "error_at_t": None if err is None else (w.get("full_time") if full else float(tnow[0])),
                       "phase_ms_eager_probe": st["ms"],
                       "learned_proposal": learned},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
                         "kernel": kern[dom]["kernel"], "launch_us": kern[dom]["launch_us"],
                         "kernels_eager_probe": kern,
                         "peak_source": peak_source},
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
