"""Benchmark: refined-wall solves per second at a certified relative residual
of 1e-10, mixed precision against FP64, on the constricted channel.

Default workload (one GPU): the 2048-panel channel wall (32768 points,
65536 unknowns, HBS leaf 64, ID tolerance 1e-12, operator tolerance 1e-14).
One step = one time step of the moving-window schedule: an 8-panel window
advancing one panel per step, refined 2-5 levels (seeded), 64 right-hand
sides from seeded pairs of exterior Stokeslets.  Each step runs the whole hot
path: refinement factorisation (added nodes, A_pp and its inverse, row IDs,
X, W^{-1}), boundary data at the refined nodes, the solve of all 64
right-hand sides to a relative residual <= 1e-10 of the extended system
against the operator at 1e-14, and the interior velocity at 16 targets.  The
reference wall's HBS (built once) is static and excluded, as the paper's
T_static.

Two arms run the same steps:
  * the headline, RW_MODE_DIRECT_IR_DF: Algorithm 1 plus iterative
    refinement against the operator at 1e-14, every product in double-FP32
    (each FP64 factor held as a pair of FP32 numbers, products and sums
    compensated: FP64-level accuracy from the FP32 units), X = A~^{-1} L of
    the refinement by double-FP32 sweeps;
  * "fp64_arm", RW_MODE_DIRECT_IR: the same algorithm in FP64 (the plain
    FP64 path to the same certified residual).
(--mode mixed: FP64 FGMRES preconditioned by Algorithm 1 with FP32 sweeps,
operator products in double-FP32.)
After the timed steps, sampled steps of each arm are re-run and their
density checked against the exact refined operator A_nn (every entry
evaluated on the fly): the true relative residual is printed per arm.

`value`: solves per second (steps x right-hand sides / time) with the
Stokeslet inputs resident on the device.  `e2e`: the same through host
buffers (inputs copied in and density and velocity copied out inside the
timed region).
--impl reference: the CPU oracle (dense Nystrom assembly + LAPACK LU) timed on
the host cores on a bounded sample of the same workload family (see
cpu_baseline.sample).
Multi-GPU: replicas only (independent walls and windows per rank).
"""
import argparse
import datetime
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TARGETS = 16
N_SRC = 5
OP_TOL = 1e-14

# workload -> panels, right-hand sides per step, data kind
WORKLOADS = {
    "mixed2048": dict(P=2048, nrhs=64, pairs=True),
    "channel1024": dict(P=1024, nrhs=1, pairs=False),
}
P_PANELS = 2048
NRHS = 64
PAIRS = True


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="df_ir",
                    choices=["df_ir", "mixed", "fp64_ir", "direct", "gmres", "gmres_bf16", "refined"])
    ap.add_argument("--compare", default="fp64_ir", choices=["fp64_ir", "mixed", "direct", "gmres", "none"],
                    help="second arm timed on the same steps (none: skip)")
    ap.add_argument("--verify-steps", type=int, default=3, help="steps of each arm re-run and checked against A_nn")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=48, help="serving workload: number of requests per phase")
    ap.add_argument("--walls", type=int, default=32, help="batched workload: number of walls")
    ap.add_argument("--workload", default="mixed2048",
                    choices=["mixed2048", "channel1024", "serving", "batched", "holes", "exterior"],
                    help="mixed2048: 2048-panel channel, 64 RHS per step from Stokeslet pairs (default); "
                         "channel1024: 1024-panel channel, 1 RHS per step")
    ap.add_argument("--solve-probe", action="store_true",
                    help="profiling driver: the headline wall, the second step's refinement, one 64-RHS solve")
    ap.add_argument("--refine-probe", type=int, default=0,
                    help="profiling driver: build the wall, run this many refinement steps, print their times")
    return ap.parse_args()


MODE_NAMES = {"df_ir": "MODE_DIRECT_IR_DF", "mixed": "MODE_GMRES_MIXED", "fp64_ir": "MODE_DIRECT_IR",
              "direct": "MODE_DIRECT", "gmres": "MODE_GMRES_FP32", "gmres_bf16": "MODE_GMRES_BF16",
              "refined": "MODE_DIRECT_REFINED"}
MODE_DTYPE = {"df_ir": "f32x2+f64", "mixed": "f64+f32", "fp64_ir": "f64", "direct": "f64",
              "gmres": "f64+f32", "gmres_bf16": "f64+bf16", "refined": "f64"}
# how each arm's refinements compute X = A~^{-1} L (rw_opts.mixed_factor):
# FP64 sweeps for the FP64 arms, double-FP32 sweeps for the double-FP32
# iterative refinement, FP32 sweeps for the FP32-preconditioned FGMRES
MODE_FACTOR = {"df_ir": 2, "mixed": 1, "gmres": 1, "gmres_bf16": 1}


def mode_id(name):
    from paper_2108_07205_gb300 import rwsolve
    return getattr(rwsolve, MODE_NAMES[name])


def dist_env():
    from paper_2108_07205_gb300 import replicas
    return replicas.rank_info()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (background).

    The sampler starts before the warm-up, so that nvidia-smi's own start-up
    (slow on a fresh machine) stays out of the timed region, and stop() keeps
    only the samples stamped inside [t0, t1] (host wall clock of the timed
    region)."""

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--id={self.index}",
               "--query-gpu=timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
               "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
               "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self, t0=None, t1=None):
        if self.proc is None:
            return None
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            if t0 is not None:
                try:
                    ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    continue
                if ts < t0 or ts > t1:
                    continue
            f = f[1:]
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def stokeslet_inputs(step, rank):
    from paper_2108_07205_gb300 import inputs
    if not PAIRS:
        sx, sy, f = inputs.stokeslets_channel(1000 * rank + step, nrhs=NRHS, n=N_SRC)
    else:
        sx, sy, f = inputs.stokeslet_pairs_channel(1000 * rank + step, NRHS)
    src = np.ascontiguousarray(np.stack([sx, sy], 1))
    fd = np.ascontiguousarray(np.transpose(f, (2, 0, 1)))
    tx, ty = inputs.targets_channel(7 + step, TARGETS)
    tg = np.ascontiguousarray(np.stack([tx, ty], 1))
    return src, fd, tg


def run_arm(args, wall, mode_name, sched, dev_in, host_in, flush, local, profile=False, verify=0):
    """Time one solve mode on the step schedule: W warm-up steps, then K timed
    steps with device inputs and K with host inputs; optionally a profiled
    repeat and a re-run of sampled steps checked against the exact operator."""
    import torch
    from paper_2108_07205_gb300 import rwsolve, replicas
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    mode = mode_id(mode_name)
    total = args.warmup + args.steps

    def step(s, host, keep=False):
        panels, levels = sched[s]
        ref = wall.refine(panels, levels, stream=stream)
        n_n = ref.stats()["n_n"]
        if host:
            src, fd, tg = host_in[s]
            g = torch.empty((NRHS, 2 * n_n), dtype=torch.float64, device=dev)
            ref.stokeslet_data(src.numpy(), fd.numpy(), g, nrhs=NRHS, stream=stream)
            tau = np.empty((NRHS, 2 * n_n))
            u = np.empty((NRHS, 2 * TARGETS))
            info = ref.solve(g, tau, nrhs=NRHS, targets=tg.numpy(), u=u, mode=mode, stream=stream)
        else:
            src, fd, tg = dev_in[s]
            g = torch.empty((NRHS, 2 * n_n), dtype=torch.float64, device=dev)
            ref.stokeslet_data(src, fd, g, nrhs=NRHS, stream=stream)
            tau = torch.empty_like(g)
            u = torch.empty((NRHS, 2 * TARGETS), dtype=torch.float64, device=dev)
            info = ref.solve(g, tau, nrhs=NRHS, targets=tg, u=u, mode=mode, stream=stream)
        st = ref.stats()
        if keep:
            return ref, g, tau, st, info
        ref.close()
        return st, info

    def timed(offset, host):
        clk = Clocks(local)
        clk.start()
        try:
            for w in range(args.warmup):
                flush.zero_()
                step(offset + w, host)
            replicas.barrier()
            torch.cuda.synchronize()
            lat = []
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            stats = []
            t_start = time.time()
            n_launch0 = rwsolve.kernel_launches()
            ev0.record(stream)
            for i in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st, info = step(offset + args.warmup + i, host)
                e1.record(stream)
                stats.append((st, info))
                lat.append((e0, e1))
            ev1.record(stream)
            torch.cuda.synchronize()
            t_end = time.time()
        except BaseException:
            clk.stop()   # never leave the sampler running
            raise
        launches = rwsolve.kernel_launches() - n_launch0
        clocks = clk.stop(t_start, t_end)
        replicas.barrier()
        ms = ev0.elapsed_time(ev1)
        lats = [a.elapsed_time(b) for a, b in lat]
        return ms, lats, stats, clocks, launches

    ms, lats, stats, clocks, launches = timed(0, host=False)
    ms_e2e, lats_e2e, _, _, _ = timed(total, host=True)
    out = {"mode": mode_name, "ms": ms, "ms_e2e": ms_e2e, "lat": lats, "lat_e2e": lats_e2e, "clocks": clocks,
           "launches": launches, "k_mean": float(np.mean([s[0]["k"] for s in stats])),
           "np_range": [min(s[0]["n_p"] for s in stats), max(s[0]["n_p"] for s in stats)],
           "iters": [s[1]["iters"] for s in stats], "relres": max(s[1]["rel_residual"] for s in stats),
           "nn_mean": float(np.mean([s[0]["n_n"] for s in stats]))}
    if profile:
        # profiled repeat of the device-input steps: per-kernel-class CUDA-event
        # durations (on each launch's stream) and algorithmic flops
        rwsolve.profile(True)
        for i in range(args.steps):
            step(args.warmup + i, False)
        out["prof"] = rwsolve.profile_read()
        rwsolve.profile(False)
    # solve-only rate on one refinement (same shapes)
    ref, g, tau, _, _ = step(0, False, keep=True)
    for _ in range(2):
        ref.solve(g, tau, nrhs=NRHS, mode=mode, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nsolve = 10 if NRHS > 8 else 50
    e0.record(stream)
    for _ in range(nsolve):
        ref.solve(g, tau, nrhs=NRHS, mode=mode, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    out["solve_ms"] = e0.elapsed_time(e1) / nsolve
    ref.close()
    # accuracy: re-run sampled timed steps (same inputs, same kernels) and
    # apply the exact refined operator A_nn to the density
    checks, taus = [], {}
    for i in np.linspace(0, args.steps - 1, max(verify, 0)).astype(int) if verify else []:
        s = args.warmup + int(i)
        ref, g, tau, _, info = step(s, False, keep=True)
        y = torch.empty_like(g)
        ref.apply_refined(tau, y, nrhs=NRHS, stream=stream)
        res = ((y - g).norm(dim=1) / g.norm(dim=1)).max().item()
        checks.append({"step": s, "true_rel_residual_max": res, "solver_rel_residual": info["rel_residual"],
                       "iters": info["iters"]})
        taus[s] = tau.cpu()
        ref.close()
    out["verify"] = checks
    out["taus"] = taus
    return out


def cpu_baseline(budget_s=25.0, single_thread=True):
    """Oracle (dense assembly + LAPACK LU) on the host cores on a bounded
    sample of the workload: moving-window steps on the same channel family at
    256 panels, one right-hand side each (the dense solve of a full-size step,
    2N_n ~ 70000, needs about 40 GB for the matrix and several times that for
    the assembly's temporaries); each measured time is scaled to the full-size
    step by the LU flop ratio (2N_n / 2N_full)^3 and the step's right-hand
    sides share the factorisation, so solves/s = nrhs / scaled time.  The
    single-thread figure repeats one sample step in a child process with every
    BLAS pool held to one thread."""
    from oracle import discretize as D, stokes as S, dense as DN
    from paper_2108_07205_gb300 import inputs
    cores = os.cpu_count()
    P = 256
    sched = inputs.time_schedule(17, P, 50)
    times, ns = [], []
    t_start = time.time()
    for s, (panels, levels) in enumerate(sched):
        o = D.refine("channel", {}, P, panels, levels)
        sx, sy, f = inputs.stokeslets_channel(s)
        t0 = time.time()
        g = S.boundary_data(o["n"], sx, sy, f)[:, 0]
        DN.solve_refined(o, g)
        times.append(time.time() - t0)
        ns.append(2 * o["n"]["x"].size)
        if time.time() - t_start > budget_s:
            break
    full = inputs.time_schedule(17, P_PANELS, 1)[0]
    n_full = 2 * (16 * P_PANELS - 16 * len(full[0]) + 16 * sum(2 ** L for L in full[1]))
    # the measured steps have varying sizes: scale each to the full step
    scaled = [t * (n_full / n) ** 3 for t, n in zip(times, ns)]
    v = NRHS / float(np.mean(scaled))
    out = {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
           "blas_threads": _blas_threads(),
           "sample": f"{len(times)} steps of the 256-panel channel window schedule "
                     f"(2N_n {min(ns)}-{max(ns)}), dense assembly + LAPACK LU, 1 RHS; time scaled by "
                     f"(2N_n / {n_full})^3 to the full-size step, {NRHS} RHS sharing it; "
                     f"raw mean {np.mean(times):.3f} s per sample step",
           "sample_s_per_step": float(np.mean(times))}
    if single_thread:
        out["single_thread"] = _single_thread_sample(n_full)
    return out


def _blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return f"{k}={os.environ[k]}"
    return f"default (BLAS pool sized to the {os.cpu_count()} host cores)"


def _single_thread_sample(n_full):
    """One 256-panel sample step of the oracle with one BLAS thread, scaled as
    cpu_baseline scales its steps; run in a child process (the thread count of
    a BLAS pool is fixed when it starts)."""
    code = ("import sys, time, json; sys.path.insert(0, %r)\n"
            "from oracle import discretize as D, stokes as S, dense as DN\n"
            "from paper_2108_07205_gb300 import inputs\n"
            "panels, levels = inputs.time_schedule(17, 256, 1)[0]\n"
            "o = D.refine('channel', {}, 256, panels, levels)\n"
            "sx, sy, f = inputs.stokeslets_channel(0)\n"
            "t0 = time.time(); g = S.boundary_data(o['n'], sx, sy, f)[:, 0]; DN.solve_refined(o, g)\n"
            "print(json.dumps({'s': time.time() - t0, 'n': 2 * o['n']['x'].size}))\n" % ROOT)
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None
    return {"value": NRHS / (d["s"] * (n_full / d["n"]) ** 3), "unit": "solves/s", "cores": 1,
            "sample_s": d["s"], "sample_2n": d["n"]}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is one bounded sample
    (cpu_baseline's scaling to the full-size step); ms_per_step is the time
    the samples actually took, value the scaled solves/s."""
    if rank != 0:
        return
    rates, took = [], []
    budget = 150.0 / max(1, args.steps + args.warmup)
    cb = None
    for i in range(args.warmup + args.steps):
        t0 = time.time()
        cb = cpu_baseline(budget_s=budget, single_thread=False)
        if i >= args.warmup:
            rates.append(cb["value"])
            took.append(time.time() - t0)
    v = 1.0 / float(np.mean([1.0 / r for r in rates]))
    line = {"impl": "reference", "metric": "refined-wall solves/s at rel. residual 1e-10", "value": v,
            "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(took)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": v,
                             "unit": "solves/s", "blas_threads": cb["blas_threads"]},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(args):
    w = {"mixed2048": "channel 2048 panels x 16 nodes (65536 unknowns), moving 8-panel window refined 2-5 levels, "
                      "64 RHS from Stokeslet pairs per step; refine + data + solve to relative residual <= 1e-10 + "
                      "velocity at 16 targets",
         "channel1024": "channel 1024 panels x 16 nodes (32768 unknowns), moving 8-panel window refined 2-5 levels, "
                        "1 RHS from 5 Stokeslets per step; refine + data + solve + velocity at 16 targets"}
    return {"workload": w.get(args.workload, args.workload), "mode": MODE_NAMES[args.mode],
            "compare": None if args.compare == "none" else MODE_NAMES[args.compare],
            "hbs_leaf": 64, "id_tol": 1e-12, "op_tol": OP_TOL, "residual_tol": 1e-10,
            "x_factor": {m: ["FP64", "FP32", "double-FP32"][MODE_FACTOR.get(m, 0)] + " sweeps"
                         for m in ([args.mode] + ([] if args.compare == "none" else [args.compare]))},
            "l2": "flushed (256 MB write) before each step"}


def refine_probe(k):
    import torch
    from paper_2108_07205_gb300 import rwsolve, inputs
    rwsolve.load(build_if_missing=True)
    # the wall of the headline arm: operator tolerance 1e-14, double-FP32 sweeps for X
    wall = rwsolve.Wall("channel", P_PANELS, opts=rwsolve.default_opts(op_tol=OP_TOL, mixed_factor=2))
    torch.cuda.synchronize()
    for panels, levels in inputs.time_schedule(17, P_PANELS, k):
        t0 = time.time()
        ref = wall.refine(panels, levels)
        torch.cuda.synchronize()
        print(json.dumps({"level": levels[0], "refine_ms": 1e3 * (time.time() - t0), **ref.stats()}))
        ref.close()
    wall.close()


def solve_probe():
    """One step of the headline arm for profiling: the wall (operator
    tolerance 1e-14, double-FP32 X), the second step of the window schedule,
    Stokeslet-pair data for 64 right-hand sides, one RW_MODE_DIRECT_IR_DF
    solve."""
    import torch
    from paper_2108_07205_gb300 import rwsolve, inputs
    rwsolve.load(build_if_missing=True)
    dev = torch.device("cuda")
    wall = rwsolve.Wall("channel", P_PANELS, opts=rwsolve.default_opts(op_tol=OP_TOL, mixed_factor=2))
    panels, levels = inputs.time_schedule(17, P_PANELS, 2)[1]
    ref = wall.refine(panels, levels)
    sx, sy, f = inputs.stokeslet_pairs_channel(0, NRHS)
    src = torch.from_numpy(np.ascontiguousarray(np.stack([sx, sy], 1))).to(dev)
    fd = torch.from_numpy(np.ascontiguousarray(np.transpose(f, (2, 0, 1)))).to(dev)
    g = torch.empty(NRHS, 2 * ref.stats()["n_n"], dtype=torch.float64, device=dev)
    ref.stokeslet_data(src, fd, g, nrhs=NRHS)
    tau = torch.empty_like(g)
    info = ref.solve(g, tau, nrhs=NRHS, mode=rwsolve.MODE_DIRECT_IR_DF)
    torch.cuda.synchronize()
    print(json.dumps({"level": levels[0], "k": ref.stats()["k"], "iters": info["iters"],
                      "rel_residual": info["rel_residual"]}))
    ref.close()
    wall.close()


def run_serving(args):
    """Serving workload: resident walls (channel 512/1024/2048 panels, star 1024
    panels, operator tolerance 1e-14); each request refines 1-64 contiguous
    panels by 2-6 levels and carries 1-32 right-hand sides from exterior point
    forces, solved in --mode (default the double-FP32 iterative refinement to
    a certified 1e-10).
    Closed loop (all requests at once) gives the saturation rate; an open loop
    with Poisson arrivals at 0.8 x that rate gives p50/p99 latency.  Sampled
    open-loop requests are refactored afterwards and their densities checked
    against the exact refined operator."""
    import torch
    from paper_2108_07205_gb300 import rwsolve, inputs
    rwsolve.load(build_if_missing=True)
    mode = mode_id(args.mode)
    op = rwsolve.default_opts(op_tol=OP_TOL, mixed_factor=MODE_FACTOR.get(args.mode, 0))
    walls = [rwsolve.Wall("channel", 512, opts=op), rwsolve.Wall("channel", 1024, opts=op),
             rwsolve.Wall("channel", 2048, opts=op), rwsolve.Wall("star", 1024, (0.3, 5, 1.0), opts=op)]
    torch.cuda.synchronize()

    def make(seed):
        g = inputs.rng(seed)
        w = walls[int(g.integers(0, len(walls)))]
        m = int(g.integers(1, 65))
        L = int(g.integers(2, 7))
        nrhs = int(g.integers(1, 33))
        panels, _ = inputs.refinement_window(seed, w.n_panels, m, L, L)
        if w is walls[3]:
            sx, sy, f = inputs.stokeslets_star(seed, nrhs=nrhs)
            tx, ty = inputs.targets_star(seed, 16)
        else:
            sx, sy, f = inputs.stokeslets_channel(seed, nrhs=nrhs)
            tx, ty = inputs.targets_channel(seed, 16)
        return (w, panels, [L] * m, np.stack([sx, sy], 1), np.transpose(f, (2, 0, 1)).copy(), nrhs,
                np.stack([tx, ty], 1))

    sv = rwsolve.Server(n_workers=4, max_device_bytes=200 << 30)
    warm = [sv.submit(*make(10 ** 6 + i)[:5], nrhs=1, mode=mode)[0] for i in range(2)]
    for t in warm:
        sv.wait(t)
    reqs = [make(i) for i in range(args.requests)]
    t0 = time.time()
    tk = [sv.submit(w, p, l, s, f, nrhs=n, targets=tg, mode=mode)[0] for (w, p, l, s, f, n, tg) in reqs]
    lat_closed = [sv.wait(t) for t in tk]
    t_closed = time.time() - t0
    nsolves = sum(r[5] for r in reqs)
    sat = args.requests / t_closed
    lam = 0.8 * sat
    g = inputs.rng(4242)
    gaps = g.exponential(1.0 / lam, size=args.requests)
    reqs2 = [make(10 ** 5 + i) for i in range(args.requests)]
    t0 = time.time()
    tk2, outs = [], []
    for gap, (w, p, l, s, f, n, tg) in zip(gaps, reqs2):
        time.sleep(gap)
        t, tau, _ = sv.submit(w, p, l, s, f, nrhs=n, targets=tg, mode=mode)
        tk2.append(t)
        outs.append(tau)
    lat_open = [sv.wait(t) for t in tk2]
    t_open = time.time() - t0
    nsolves2 = sum(r[5] for r in reqs2)
    sv.close()
    # accuracy of sampled served results against the exact refined operator
    worst = 0.0
    sample = inputs.rng(99).choice(args.requests, min(16, args.requests), replace=False)
    for i in sample:
        w, p, l, s_, f, n, _ = reqs2[i]
        ref = w.refine(p, l)
        g = np.empty((n, 2 * ref.stats()["n_n"]))
        ref.stokeslet_data(np.ascontiguousarray(s_), f, g, nrhs=n)
        y = np.empty_like(g)
        ref.apply_refined(np.ascontiguousarray(outs[i]), y, nrhs=n)
        worst = max(worst, float((np.linalg.norm(y - g, axis=1) / np.linalg.norm(g, axis=1)).max()))
        ref.close()
    line = {"metric": "refined-wall solves/s (serving, open loop at 0.8 x saturation)",
            "value": nsolves2 / t_open, "unit": "solves/s", "n_gpus": 1, "steps": args.requests, "warmup": 2,
            "ms_per_step": 1e3 * t_open / args.requests, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": MODE_DTYPE[args.mode], "data": "synthetic",
            "config": {"workload": "serving: walls channel 512/1024/2048 + star 1024 panels (op_tol 1e-14); "
                                   "requests refine 1-64 panels by 2-6 levels with 1-32 RHS; 4 workers, "
                                   "200 GB budget", "mode": MODE_NAMES[args.mode]},
            "true_rel_residual_max_sampled": worst, "sampled_requests": len(sample),
            "p50_ms": float(np.percentile(lat_open, 50)), "p99_ms": float(np.percentile(lat_open, 99)),
            "saturation": {"requests_per_s": sat, "solves_per_s": nsolves / t_closed,
                           "p50_ms": float(np.percentile(lat_closed, 50)),
                           "p99_ms": float(np.percentile(lat_closed, 99))},
            "arrival_rate_per_s": lam}
    print(json.dumps(line))


def run_batched(args):
    """Batched uneven instances: star walls r = 1 + a cos(k t), a ~ U[0.1, 0.4],
    k ~ U{3..8}, 128-1024 panels, each refined at a seeded window (2-16
    panels, 2-4 levels), 8 RHS each.  Walls and refinements are built first
    (static); the timed region is the batched solve of all instances (one
    persistent launch per 8 RHS, replayed from a CUDA graph, tile height
    autotuned), against the same solves issued one instance at a time; then
    the batched iterative refinement to a certified relative residual of
    1e-10 (Algorithm 1 and the operators of all instances in batched launches,
    FP64 corrections), with sampled instances checked against their exact
    refined operators."""
    import torch
    from paper_2108_07205_gb300 import rwsolve, inputs
    rwsolve.load(build_if_missing=True)
    nrhs = 8
    g0 = inputs.rng(555)
    walls, refs, gs = [], [], []
    t0 = time.time()
    for i in range(args.walls):
        a = float(g0.uniform(0.1, 0.4))
        k = int(g0.integers(3, 9))
        P = int(g0.integers(128, 1025))
        m = int(g0.integers(2, 17))
        L = int(g0.integers(2, 5))
        w = rwsolve.Wall("star", P, (a, k, 1.0), opts=rwsolve.default_opts(op_tol=OP_TOL))
        panels, levels = inputs.refinement_window(1000 + i, P, m, L, L)
        r = w.refine(panels, levels)
        sx, sy, f = inputs.stokeslets_star(2000 + i, nrhs=nrhs, radius=2.5)
        g = np.empty((nrhs, 2 * r.stats()["n_n"]))
        r.stokeslet_data(np.stack([sx, sy], 1), np.transpose(f, (2, 0, 1)).copy(), g, nrhs=nrhs)
        walls.append(w)
        refs.append(r)
        gs.append(g)
    setup_s = time.time() - t0
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    b = rwsolve.Batch(refs)
    gall = torch.from_numpy(np.ascontiguousarray(np.concatenate(gs, axis=1))).to(dev)
    tau = torch.empty_like(gall)
    tr, tune_ms = b.autotune(nrhs=nrhs)
    for _ in range(args.warmup):
        b.solve(gall, tau, nrhs=nrhs, use_graph=True, stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.solve(gall, tau, nrhs=nrhs, use_graph=True, stream=stream)
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(c) for a, c in times]))
    # the same solves, one instance at a time
    dg = [torch.from_numpy(g).to(dev) for g in gs]
    dt = [torch.empty_like(x) for x in dg]
    for r, x, y in zip(refs, dg, dt):
        r.solve(x, y, nrhs=nrhs, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for r, x, y in zip(refs, dg, dt):
        r.solve(x, y, nrhs=nrhs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    maxdiff = max(float((tau[:, b.offsets[i]:b.offsets[i + 1]] - dt[i]).abs().max() /
                        dt[i].abs().max()) for i in range(len(refs)))
    # the batch to a certified 1e-10
    tau_ir = torch.empty_like(gall)
    info = b.solve_ir(gall, tau_ir, nrhs=nrhs, tol=1e-10, stream=stream)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = b.solve_ir(gall, tau_ir, nrhs=nrhs, tol=1e-10, stream=stream)
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    ms_ir = float(np.mean([a.elapsed_time(c) for a, c in times]))
    worst_true = 0.0
    for i in inputs.rng(7).choice(len(refs), min(8, len(refs)), replace=False):
        x = tau_ir[:, b.offsets[i]:b.offsets[i + 1]].contiguous()
        y = torch.empty_like(x)
        refs[i].apply_refined(x, y, nrhs=nrhs, stream=stream)
        gi = dg[i]
        worst_true = max(worst_true, float(((y - gi).norm(dim=1) / gi.norm(dim=1)).max()))
    line = {"metric": "refined-wall solves/s (batched uneven walls, one persistent launch per 8 RHS)",
            "value": args.walls * nrhs / (ms / 1e3), "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.walls} star walls, 128-1024 panels, refined 2-16 panels by 2-4 levels, "
                                   "8 RHS each; solve only (walls and refinements static)",
                       "l2": "flushed before each solve"},
            "sequential_per_instance_solves_per_s": args.walls * nrhs / (ms_seq / 1e3),
            "autotuned_tile_rows": tr, "autotune_ms": tune_ms, "setup_s": setup_s,
            "rows": b.offsets[-1], "max_rel_diff_vs_individual": maxdiff,
            "certified": {"what": "rw_batch_solve_ir to relative residual <= 1e-10 (op_tol 1e-14 operators)",
                          "solves_per_s": args.walls * nrhs / (ms_ir / 1e3), "ms": ms_ir,
                          "corrections": info["iters"], "certified_rel_residual_max": info["rel_residual"],
                          "true_rel_residual_max_sampled": worst_true, "sampled_instances": min(8, len(refs))}}
    print(json.dumps(line))
    b.close()


def run_holes(args):
    """Channel with three added holes (App. B; Sec. 5.2, Tab. holes): the
    channel at the paper's three sizes (2N = 30720, 61440, 122880: 960, 1920
    and 3840 panels) with three circular holes of 10 panels (960 hole
    unknowns), data from 5 exterior Stokeslets and 2 + 2 + 1 inside the holes.
    Per size: the wall's HBS build (static), the holes factorisation
    (T_ELS,comp + T_ELS,inv of the paper; median of --steps runs after the
    warm-up), and the direct and refined solves of one right-hand side (CUDA
    events, L2 flushed before each), with the velocity error at fluid targets
    against the closed-form Stokeslet field.  One JSON line per size."""
    import torch
    from paper_2108_07205_gb300 import rwsolve, inputs
    rwsolve.load(build_if_missing=True)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for P in (960, 1920, 3840):
        t0 = time.time()
        w = rwsolve.Wall("channel", P)
        build_s = time.time() - t0
        hl = inputs.holes_channel(3, n_panels=10)
        sx, sy, f = inputs.stokeslets_channel(0, nrhs=1)
        hx, hy, hf = inputs.stokeslets_in_holes(1, hl, [2, 2, 1], nrhs=1)
        src = np.ascontiguousarray(np.stack([np.concatenate([sx, hx]), np.concatenate([sy, hy])], 1))
        fd = np.ascontiguousarray(np.transpose(np.concatenate([f, hf]), (2, 0, 1)))
        for _ in range(max(1, args.warmup)):
            w.add_holes(hl).close()
        torch.cuda.synchronize()
        fac = []
        for _ in range(max(1, args.steps)):
            t0 = time.time()
            r = w.add_holes(hl)
            torch.cuda.synchronize()
            fac.append(time.time() - t0)
            if _ < args.steps - 1:
                r.close()
        st = r.stats()
        n = 2 * st["n_n"]
        g = torch.empty(n, dtype=torch.float64, device=dev)
        r.stokeslet_data(torch.from_numpy(src).to(dev), torch.from_numpy(fd).to(dev), g)
        tau = torch.empty_like(g)
        out = {}
        for name, mode in (("direct", rwsolve.MODE_DIRECT), ("refined", rwsolve.MODE_DIRECT_REFINED)):
            for _ in range(3):
                r.solve(g, tau, mode=mode, stream=stream)
            ts = []
            for _ in range(max(3, args.steps)):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r.solve(g, tau, mode=mode, stream=stream)
                e1.record(stream)
                ts.append((e0, e1))
            torch.cuda.synchronize()
            out[name] = float(np.median([a.elapsed_time(b) for a, b in ts]))
        tx, ty = inputs.targets_fluid(4, hl, "channel", 32)
        tg = torch.from_numpy(np.ascontiguousarray(np.stack([tx, ty], 1))).to(dev)
        u = torch.empty(2 * tx.size, dtype=torch.float64, device=dev)
        r.solve(g, tau, targets=tg, u=u, mode=rwsolve.MODE_DIRECT_REFINED, stream=stream)
        ue = _stokeslet_field(tx, ty, src, fd[0])
        err = float(np.abs(u.cpu().numpy().reshape(-1, 2) - ue).max() / np.abs(ue).max())
        line = {"metric": "holed-wall solves/s (direct, 1 RHS)", "value": 1e3 / out["direct"], "unit": "solves/s",
                "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["direct"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": f"channel {P} panels (2N = {32 * P}) + 3 circular holes x 10 panels "
                                       "(960 hole unknowns), App. B", "l2": "flushed before each solve"},
                "factor_ms": 1e3 * float(np.median(fac)), "hbs_build_s": build_s,
                "refined_solve_ms": out["refined"], "k_woodbury": st["k"], "k_far": st["k_far"],
                "k_near": st["k_near"], "k_pk": st["k_pk"], "ref_bytes": st["bytes"],
                "velocity_rel_error_closed_form": err}
        print(json.dumps(line))
        r.close()
        w.close()


def run_exterior(args):
    """Exterior Stokes problem (Sec. 2.2, Eq. exterior_BIE): the fluid outside
    the star wall r = 1 + 0.3 cos 5t with 2048 panels (65536 unknowns), the
    combined field 1/2 I + D + S.  The wall is built with operator tolerance
    1e-14 and double-FP32 X.  Each step moves an 8-panel window refined 2-5
    levels, factors it, makes the data of 64 right-hand sides (3 Stokeslets
    inside the wall, strengths N(0, I2) per right-hand side), solves to a
    relative residual <= 1e-10 (RW_MODE_DIRECT_IR_DF) and evaluates the
    velocity at 16 fluid targets.  The step is timed on the host around a
    synchronised step (median).  The solve alone is timed by CUDA events (L2
    flushed before it).  On the last step the true relative residual of every
    right-hand side comes from the exact refined operator (every entry on the
    fly, with the singular rule).  The velocity error against the
    closed-form Stokeslet field is taken at the targets.  One JSON line."""
    import torch
    from paper_2108_07205_gb300 import rwsolve, inputs
    rwsolve.load(build_if_missing=True)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    P, nrhs = 2048, 64
    t0 = time.time()
    w = rwsolve.Wall("star", P, (0.3, 5, 1.0), exterior=True,
                     opts=rwsolve.default_opts(op_tol=OP_TOL, mixed_factor=2))
    torch.cuda.synchronize()
    build_s = time.time() - t0
    sx, sy, f = inputs.stokeslets_inside_star(23, nrhs=nrhs)
    src = torch.from_numpy(np.ascontiguousarray(np.stack([sx, sy], 1))).to(dev)
    fd = torch.from_numpy(np.ascontiguousarray(np.transpose(f, (2, 0, 1)))).to(dev)
    tx, ty = inputs.targets_outside_star(24, n=TARGETS)
    tg = torch.from_numpy(np.ascontiguousarray(np.stack([tx, ty], 1))).to(dev)
    sched = inputs.time_schedule(29, P, args.warmup + args.steps)
    steps, solve_ms, iters, relres, ks = [], [], [], [], []
    for s_, (panels, levels) in enumerate(sched):
        torch.cuda.synchronize()
        t0 = time.time()
        r = w.refine(panels, levels, stream=stream)
        n = 2 * r.stats()["n_n"]
        g = torch.empty((nrhs, n), dtype=torch.float64, device=dev)
        r.stokeslet_data(src, fd, g, nrhs=nrhs, stream=stream)
        tau = torch.empty_like(g)
        u = torch.empty((nrhs, 2 * TARGETS), dtype=torch.float64, device=dev)
        info = r.solve(g, tau, nrhs=nrhs, targets=tg, u=u, mode=rwsolve.MODE_DIRECT_IR_DF, stream=stream)
        torch.cuda.synchronize()
        dt = time.time() - t0
        if s_ < args.warmup:
            r.close()
            continue
        steps.append(dt)
        iters.append(info["iters"])
        relres.append(info["rel_residual"])
        ks.append(r.stats()["k"])
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.solve(g, tau, nrhs=nrhs, mode=rwsolve.MODE_DIRECT_IR_DF, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        solve_ms.append(e0.elapsed_time(e1))
        if s_ == len(sched) - 1:
            y = torch.empty_like(tau)
            r.apply_refined(tau, y, nrhs=nrhs, stream=stream)
            torch.cuda.synchronize()
            true_res = float(((g - y).norm(dim=1) / g.norm(dim=1)).max())
            ue = np.transpose(_stokeslet_field_multi(tx, ty, sx, sy, f), (2, 0, 1)).reshape(nrhs, -1)
            vel_err = float(np.abs(u.cpu().numpy() - ue).max() / np.abs(ue).max())
        r.close()
    w.close()
    ms = 1e3 * float(np.median(steps))
    line = {"metric": "exterior refined-wall solves/s at rel. residual 1e-10", "value": nrhs * 1e3 / ms,
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": MODE_DTYPE["df_ir"],
            "data": "synthetic",
            "config": {"workload": "exterior star r = 1 + 0.3 cos 5t, 2048 panels x 16 nodes (65536 unknowns), "
                                   "combined field (Sec. 2.2); moving 8-panel window refined 2-5 levels; 64 RHS "
                                   "from 3 Stokeslets inside the wall; refine + data + solve to 1e-10 + velocity "
                                   "at 16 fluid targets",
                       "mode": MODE_NAMES["df_ir"], "op_tol": OP_TOL, "id_tol": 1e-12,
                       "step_timing": "host clock around a synchronised step (median)",
                       "solve_timing": "CUDA events, L2 flushed (256 MB write) before the solve"},
            "solve_only_per_s": nrhs * 1e3 / float(np.median(solve_ms)), "solve_only_ms": float(np.median(solve_ms)),
            "iters": [int(i) for i in iters], "solver_rel_residual_max": float(max(relres)),
            "true_rel_residual_max": true_res, "velocity_rel_error_closed_form": vel_err,
            "k_mean": float(np.mean(ks)), "hbs_build_s": build_s}
    print(json.dumps(line))


def _stokeslet_field_multi(tx, ty, sx, sy, f):
    """Closed-form velocity (nt, 2, nrhs) of point forces f (ns, 2, nrhs)."""
    rx = tx[:, None] - sx[None, :]
    ry = ty[:, None] - sy[None, :]
    r2 = rx * rx + ry * ry
    lg = -0.5 * np.log(r2)
    rf = (rx[:, :, None] * f[None, :, 0, :] + ry[:, :, None] * f[None, :, 1, :]) / r2[:, :, None]
    ux = (lg[:, :, None] * f[None, :, 0, :] + rx[:, :, None] * rf).sum(1) / (4.0 * np.pi)
    uy = (lg[:, :, None] * f[None, :, 1, :] + ry[:, :, None] * rf).sum(1) / (4.0 * np.pi)
    return np.stack([ux, uy], 1)


def _stokeslet_field(tx, ty, src, f):
    """Closed-form velocity of point forces f (ns x 2) at src (ns x 2), mu = 1
    (Eq. stokeslet), for the error column of the holes workload."""
    rx = tx[:, None] - src[None, :, 0]
    ry = ty[:, None] - src[None, :, 1]
    r2 = rx * rx + ry * ry
    rf = (rx * f[None, :, 0] + ry * f[None, :, 1]) / r2
    lg = -0.5 * np.log(r2)
    ux = ((lg * f[None, :, 0] + rx * rf).sum(1)) / (4.0 * np.pi)
    uy = ((lg * f[None, :, 1] + ry * rf).sum(1)) / (4.0 * np.pi)
    return np.stack([ux, uy], 1)


def run_ours(args, rank, world, local):
    """Build the wall, the schedule and the inputs, then time each arm."""
    import torch
    from paper_2108_07205_gb300 import rwsolve, inputs, replicas
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    rwsolve.load(build_if_missing=True)
    arms = [args.mode] + ([args.compare] if args.compare not in ("none", args.mode) else [])
    # one wall per factorisation kind the arms need (the HBS of A_oo is the
    # same; only how refinements compute X differs)
    walls = {}
    build_s = None
    for m in arms:
        mf = MODE_FACTOR.get(m, 0)
        if mf in walls:
            continue
        t0 = time.time()
        walls[mf] = rwsolve.Wall("channel", P_PANELS, opts=rwsolve.default_opts(op_tol=OP_TOL, mixed_factor=mf))
        torch.cuda.synchronize()
        if build_s is None:
            build_s = time.time() - t0
    wall = walls[MODE_FACTOR.get(arms[0], 0)]
    hst = wall.stats()
    total = args.warmup + args.steps
    sched = inputs.time_schedule(replicas.schedule_seed(rank), P_PANELS, 2 * total + 1)
    dev_in, host_in = [], []
    for s in range(2 * total + 1):
        src, fd, tg = stokeslet_inputs(s, rank)
        host_in.append((torch.from_numpy(src).pin_memory(), torch.from_numpy(fd).pin_memory(),
                        torch.from_numpy(tg).pin_memory()))
        dev_in.append(tuple(x.to(dev) for x in (torch.from_numpy(src), torch.from_numpy(fd), torch.from_numpy(tg))))
    # L2 flush buffer (> 129 MB L2)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    for i, m in enumerate(arms):
        try:
            res[m] = run_arm(args, walls[MODE_FACTOR.get(m, 0)], m, sched, dev_in, host_in, flush, local,
                             profile=(i == 0),
                             verify=args.verify_steps)
        except rwsolve.RWError as e:
            res[m] = {"error": str(e)}
    # HBS inverse sweep alone (s1 on the reference wall, 1 RHS): algorithmic
    # bytes = matrix entries read (FP64) + vectors
    b = torch.randn(2 * hst["n_points"], dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    for _ in range(5):
        wall.apply_inverse(b, x, stream=stream)
    torch.cuda.synchronize()
    times = []
    for _ in range(50):
        flush.zero_()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        wall.apply_inverse(b, x, stream=stream)
        a1.record(stream)
        times.append((a0, a1))
    torch.cuda.synchronize()
    sweep = {"ms": float(np.mean([a.elapsed_time(c) for a, c in times])),
             "bytes": 8 * hst["inv_elems"] + 8 * 4 * 2 * hst["n_points"]}
    for w in walls.values():
        w.close()
    for m in res:
        if "ms" in res[m]:
            res[m]["ms"], res[m]["ms_e2e"] = replicas.max_over_ranks([res[m]["ms"], res[m]["ms_e2e"]])
    h2d = int(sum(x.numel() * x.element_size() for x in host_in[0]))
    return {"arms": res, "order": arms, "build_s": build_s, "hbs": hst, "sweep": sweep, "h2d": h2d}


# Peaks of the ALU-bound kernel classes, from the unit counts and the SM clock
# sampled under load: 152 SMs; FP64 4 flop/clk/SM; FP32 128 lanes x 2
# flop/clk/SM; double-FP32 products take 12 FP32 lane operations per
# multiply-add (2 FP64-equivalent flops).
def alu_peak_tflops(cls, sm_mhz):
    clk = sm_mhz * 1e6
    probe = " (an FMA-chain probe on this part measured FP64 1.258 and FP32 76.87 TFLOP/s at 2070 MHz)"
    if cls == "gemm_f32":
        return 152 * 256 * clk / 1e12, "FP32: 152 SMs x 128 lanes x 2 flop/clk x median SM clock" + probe
    if cls == "gemm_df":
        return 152 * 128 * 2 / 12 * clk / 1e12, ("double-FP32: 152 SMs x 128 FP32 lanes / 12 lane-ops per "
                                                  "multiply-add x 2 flop x median SM clock" + probe)
    return 152 * 4 * clk / 1e12, "FP64: 152 SMs x 4 flop/clk x median SM clock" + probe


KCLASS_NAMES = {"id": "column-pivoted QR (cluster and grid-wide kernels, FP64)", "gemm": "batched tiled GEMM (FP64)",
                "gemv": "batched GEMV / HBS sweeps", "inverse": "batched Gauss-Jordan inverse (FP64)",
                "eval": "kernel-entry evaluation (FP64)", "other": "bookkeeping kernels",
                "gemm_f32": "batched GEMM, FP32 accumulation (preconditioner sweeps)",
                "gemm_df": "batched double-FP32 GEMM (FP64-accurate operator products)"}


def roofline_of(prof, steps, sm_mhz, hbm, hbm_src):
    dom = max(prof, key=lambda c: prof[c]["ms"])
    dp = prof[dom]
    if dom == "gemv" or dom == "other":
        ach = dp["bytes"] / (dp["ms"] / 1e3) / 1e9
        return {"kernel": KCLASS_NAMES[dom], "class": dom, "bound": "hbm", "achieved": ach, "peak": hbm,
                "unit": "GB/s", "frac": ach / hbm, "traffic": None, "launches_per_step": dp["launches"] / steps,
                "avg_launch_ms": dp["ms"] / max(dp["launches"], 1), "peak_source": hbm_src}
    peak, src = alu_peak_tflops(dom, sm_mhz)
    ach = dp["flops"] / (dp["ms"] / 1e3) / 1e12
    return {"kernel": KCLASS_NAMES[dom], "class": dom, "bound": "alu", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "traffic": None, "launches_per_step": dp["launches"] / steps,
            "avg_launch_ms": dp["ms"] / max(dp["launches"], 1), "peak_source": "derived " + src}


def arm_summary(a, args, world):
    if "error" in a:
        return {"mode": a.get("mode"), "error": a["error"]}
    v = world * args.steps * NRHS / (a["ms"] / 1e3)
    checks = a["verify"]
    return {"mode": MODE_NAMES[a["mode"]], "value": v, "unit": "solves/s", "ms_per_step": a["ms"] / args.steps,
            "e2e": world * args.steps * NRHS / (a["ms_e2e"] / 1e3),
            "p50_ms": float(np.percentile(a["lat"], 50)), "p99_ms": float(np.percentile(a["lat"], 99)),
            "solve_only_per_s": NRHS * 1e3 / a["solve_ms"], "solve_only_ms": a["solve_ms"],
            "iters": a["iters"], "solver_rel_residual_max": a["relres"], "k_mean": a["k_mean"],
            "true_rel_residual_max": max((c["true_rel_residual_max"] for c in checks), default=None),
            "verified_steps": [c["step"] for c in checks], "dtype": MODE_DTYPE[a["mode"]],
            "gpu_launches": a["launches"]}


def main():
    global P_PANELS, NRHS, PAIRS
    args = parse()
    if args.workload in WORKLOADS:
        wl = WORKLOADS[args.workload]
        P_PANELS, NRHS, PAIRS = wl["P"], wl["nrhs"], wl["pairs"]
    if args.solve_probe:
        solve_probe()
        return
    if args.refine_probe:
        refine_probe(args.refine_probe)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "holes":
        run_holes(args)
        return
    if args.workload == "exterior":
        run_exterior(args)
        return
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as td
        td.init_process_group("gloo" if args.impl == "reference" else "nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    out = run_ours(args, rank, world, local)
    if rank != 0 or out is None:
        return
    peaks, hbm_src = {}, "profiling recipe fallback 6800 GB/s (MEASURED_PEAKS.json absent)"
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_src = "MEASURED_PEAKS.json hbm_gbs"
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    head = out["arms"][out["order"][0]]
    if "error" in head:
        print(json.dumps({"metric": "refined-wall solves/s at rel. residual 1e-10", "value": None,
                          "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": MODE_DTYPE[args.mode], "data": "synthetic", "config": workload_config(args),
                          "error": head["error"]}))
        return
    hs = arm_summary(head, args, world)
    sm_mhz = (head["clocks"] or {}).get("sm_mhz") or 2070.0
    prof = head["prof"]
    share = {c: round(prof[c]["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-9), 4) for c in prof}
    roof = roofline_of(prof, args.steps, sm_mhz, hbm, hbm_src)
    by_class = {}
    for c in ("gemm_df", "gemm_f32", "gemm", "id"):
        if prof.get(c, {}).get("launches"):
            pk, src = alu_peak_tflops(c, sm_mhz)
            ach = prof[c]["flops"] / (prof[c]["ms"] / 1e3) / 1e12
            by_class[c] = {"achieved_tflops": ach, "peak_tflops": pk, "frac": ach / pk,
                           "launches_per_step": prof[c]["launches"] / args.steps}
    fp64_peak = alu_peak_tflops("gemm", sm_mhz)[0]
    sw = out["sweep"]
    sweep_gbs = sw["bytes"] / (sw["ms"] / 1e3) / 1e9
    sweep_flops = 2.0 * out["hbs"]["inv_elems"]
    h2d = out["h2d"]   # point forces, their positions and the velocity targets of one step
    line = {
        "metric": "refined-wall solves/s at rel. residual 1e-10", "value": hs["value"], "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": hs["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": MODE_DTYPE[args.mode],
        "data": "synthetic", "config": workload_config(args),
        "p50_ms": hs["p50_ms"], "p99_ms": hs["p99_ms"],
        "solve_only_per_s": hs["solve_only_per_s"], "iters": hs["iters"],
        "solver_rel_residual_max": hs["solver_rel_residual_max"],
        "true_rel_residual_max": hs["true_rel_residual_max"], "verified_steps": hs["verified_steps"],
        "k_mean": hs["k_mean"], "n_p_range": head["np_range"], "hbs_build_s": out["build_s"],
        "e2e": {"value": hs["e2e"], "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(8 * NRHS * (2 * TARGETS + 2 * head["nn_mean"]))},
        "roofline": roof,
        "roofline_by_class": by_class,
        "kernel_time_share": share,
        "roofline_sweep": {"kernel": "HBS inverse sweep (s1, FP64, 1 RHS, L2 flushed)", "ms": sw["ms"],
                           "hbm_achieved_gbs": sweep_gbs, "hbm_frac": sweep_gbs / hbm,
                           "fp64_achieved_tflops": sweep_flops / (sw["ms"] / 1e3) / 1e12,
                           "fp64_frac": sweep_flops / (sw["ms"] / 1e3) / 1e12 / fp64_peak},
        "clocks": head["clocks"],
        "gpu_launches": hs["gpu_launches"],
    }
    if len(out["order"]) > 1:
        other = out["arms"][out["order"][1]]
        line["fp64_arm" if out["order"][1] == "fp64_ir" else "compare_arm"] = arm_summary(other, args, world)
        if "error" not in other:
            line["speedup_vs_compare"] = hs["value"] / (world * args.steps * NRHS / (other["ms"] / 1e3))
            diffs = []
            for s_, t in head["taus"].items():
                if s_ in other["taus"]:
                    o = other["taus"][s_]
                    diffs.append(float(((t - o).norm(dim=1) / o.norm(dim=1)).max()))
            line["density_rel_diff_vs_compare"] = max(diffs) if diffs else None
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
