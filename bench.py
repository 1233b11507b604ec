"""Benchmark: refined-wall solves per second on the constricted channel.

Workload (one GPU): the 1024-panel channel wall (16384 points, 32768
unknowns, HBS leaf 64, ID tolerance 1e-12).  One step = one time step of the
moving-window schedule: an 8-panel window advancing one panel per step,
refined 2-5 levels (seeded), so each step runs the whole hot path:
refinement factorisation (added nodes, A_pp^{-1}, row IDs, X, W^{-1}),
boundary data from 5 exterior Stokeslets at the refined nodes, the Woodbury
solve for the density, and the interior velocity at 16 targets.  The
reference wall's HBS (built once) is static and excluded, as the paper's
T_static.

`value`: steps per second with the Stokeslet inputs resident on the device.
`e2e`: the same through host buffers (inputs copied in and density and
velocity copied out inside the timed region).
--impl reference: the CPU oracle (dense Nystrom assembly + LAPACK LU) timed on
the host cores on the same workload family (see cpu_baseline.sample).
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

P_PANELS = 1024
TARGETS = 16
N_SRC = 5
NRHS = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="direct", choices=["direct", "gmres", "gmres_bf16", "refined"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=48, help="serving workload: number of requests per phase")
    ap.add_argument("--walls", type=int, default=32, help="batched workload: number of walls")
    ap.add_argument("--workload", default="channel1024",
                    choices=["channel1024", "mixed2048", "serving", "batched", "holes"],
                    help="channel1024: 1 RHS per step (default); mixed2048: 2048-panel channel, 64 RHS per "
                         "step from Stokeslet pairs")
    ap.add_argument("--refine-probe", type=int, default=0,
                    help="profiling driver: build the wall, run this many refinement steps, print their times")
    return ap.parse_args()


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
    if NRHS == 1:
        sx, sy, f = inputs.stokeslets_channel(1000 * rank + step, nrhs=1, n=N_SRC)
    else:
        sx, sy, f = inputs.stokeslet_pairs_channel(1000 * rank + step, NRHS)
    src = np.ascontiguousarray(np.stack([sx, sy], 1))
    fd = np.ascontiguousarray(np.transpose(f, (2, 0, 1)))
    tx, ty = inputs.targets_channel(7 + step, TARGETS)
    tg = np.ascontiguousarray(np.stack([tx, ty], 1))
    return src, fd, tg


def run_ours(args, rank, world, local):
    import torch
    from paper_2108_07205_gb300 import rwsolve, inputs, replicas
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    rwsolve.load(build_if_missing=True)
    mode = {"direct": rwsolve.MODE_DIRECT, "gmres": rwsolve.MODE_GMRES_FP32,
            "refined": rwsolve.MODE_DIRECT_REFINED, "gmres_bf16": rwsolve.MODE_GMRES_BF16}[args.mode]
    t0 = time.time()
    wall = rwsolve.Wall("channel", P_PANELS)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    hst = wall.stats()
    total = args.warmup + args.steps
    sched = inputs.time_schedule(replicas.schedule_seed(rank), P_PANELS, 2 * total + 1)
    # device-resident inputs for every step
    dev_in = []
    host_in = []
    for s in range(2 * total + 1):
        src, fd, tg = stokeslet_inputs(s, rank)
        host_in.append((torch.from_numpy(src).pin_memory(), torch.from_numpy(fd).pin_memory(),
                        torch.from_numpy(tg).pin_memory()))
        dev_in.append(tuple(x.to(dev) for x in (torch.from_numpy(src), torch.from_numpy(fd), torch.from_numpy(tg))))
    # L2 flush buffer (> 129 MB L2)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(s, host):
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

    try:
        ms, lats, stats, clocks, launches = timed(0, host=False)
    except rwsolve.RWError as e:
        if args.mode != "gmres_bf16" or e.code != -4:
            raise
        # BF16 sweeps as the preconditioner do not converge on this wall: the
        # BF16 rounding of the inverse times the wall's conditioning exceeds one
        if rank == 0:
            print(json.dumps({"metric": "refined-wall solves/s", "value": None, "unit": "solves/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                              "scaling": "weak", "vs_baseline": None, "dtype": "f64+bf16", "data": "synthetic",
                              "config": workload_config(args), "not_converged": str(e)}))
        return
    ms_e2e, lats_e2e, _, _, _ = timed(total, host=True)
    # profiled repeat of the device-input steps: per-kernel-class CUDA-event
    # durations (on each launch's stream) and algorithmic flops
    rwsolve.profile(True)
    for i in range(args.steps):
        step(args.warmup + i, False)
    prof = rwsolve.profile_read()
    rwsolve.profile(False)
    ms, ms_e2e = replicas.max_over_ranks([ms, ms_e2e])
    ks = [s[0]["k"] for s in stats]
    nps = [s[0]["n_p"] for s in stats]
    out = {
        "ms": ms, "ms_e2e": ms_e2e, "lat": lats, "lat_e2e": lats_e2e, "clocks": clocks,
        "build_s": build_s, "hbs": hst, "k_mean": float(np.mean(ks)), "np_range": [min(nps), max(nps)],
        "iters": [s[1]["iters"] for s in stats], "launches": launches, "prof": prof,
    }
    # solve-only rate on one refinement (same shapes), and the sweep kernel roofline
    panels, levels = sched[0]
    ref = wall.refine(panels, levels, stream=stream)
    n_n = ref.stats()["n_n"]
    src, fd, tg = dev_in[0]
    g = torch.empty((NRHS, 2 * n_n), dtype=torch.float64, device=dev)
    ref.stokeslet_data(src, fd, g, nrhs=NRHS, stream=stream)
    tau = torch.empty_like(g)
    for _ in range(5):
        ref.solve(g, tau, nrhs=NRHS, mode=mode, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nsolve = 50
    e0.record(stream)
    for _ in range(nsolve):
        ref.solve(g, tau, nrhs=NRHS, mode=mode, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    out["solve_ms"] = e0.elapsed_time(e1) / nsolve
    ref.close()
    # HBS inverse sweep alone (s1 on the reference wall): algorithmic bytes =
    # matrix entries read (FP64) + vectors
    b = torch.randn(2 * hst["n_points"], dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    for _ in range(5):
        wall.apply_inverse(b, x, stream=stream)
    torch.cuda.synchronize()
    nsw = 50
    times = []
    for _ in range(nsw):
        flush.zero_()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        wall.apply_inverse(b, x, stream=stream)
        a1.record(stream)
        times.append((a0, a1))
    torch.cuda.synchronize()
    sweep_ms = float(np.mean([a.elapsed_time(c) for a, c in times]))
    out["sweep_ms"] = sweep_ms
    out["sweep_bytes"] = 8 * hst["inv_elems"] + 8 * 4 * 2 * hst["n_points"]
    wall.close()
    return out


def cpu_baseline(budget_s=25.0):
    """Oracle (dense assembly + LAPACK LU) on the host cores on a bounded
    sample of the workload: one moving-window step on the same channel family
    at 256 panels (the dense solve of the 1024-panel step does not fit the
    time budget); the rate is scaled to the full-size step by the LU flop
    ratio (n_sample / n_full)^3."""
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
    v = 1.0 / float(np.mean(scaled))
    return {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} steps of the 256-panel channel window schedule "
                      f"(2N_n {min(ns)}-{max(ns)}), dense assembly + LAPACK LU, time scaled by "
                      f"(2N_n / {n_full})^3 to the 1024-panel step; raw mean {np.mean(times):.3f} s/solve"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    t_all = []
    budget = 150.0 / max(1, args.steps + args.warmup)
    cb = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(budget_s=budget)
        if i >= args.warmup:
            t_all.append(1.0 / cb["value"])
    v = 1.0 / float(np.mean(t_all))
    line = {"impl": "reference", "metric": "refined-wall solves/s", "value": v, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": v,
                             "unit": "solves/s"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(args):
    if args.workload == "mixed2048":
        return {"workload": "channel 2048 panels x 16 nodes (65536 unknowns), moving 8-panel window refined "
                            "2-5 levels, refine + data + solve + velocity per step, 64 RHS from Stokeslet pairs",
                "mode": args.mode, "hbs_leaf": 64, "id_tol": 1e-12, "l2": "flushed (256 MB write) before each step"}
    return {"workload": "channel 1024 panels x 16 nodes (32768 unknowns), moving 8-panel window refined "
                        "2-5 levels, refine + data + solve + velocity per step, 1 RHS",
            "mode": args.mode, "hbs_leaf": 64, "id_tol": 1e-12, "l2": "flushed (256 MB write) before each step"}


def refine_probe(k):
    import torch
    from paper_2108_07205_gb300 import rwsolve, inputs
    rwsolve.load(build_if_missing=True)
    wall = rwsolve.Wall("channel", P_PANELS)
    torch.cuda.synchronize()
    for panels, levels in inputs.time_schedule(17, P_PANELS, k):
        t0 = time.time()
        ref = wall.refine(panels, levels)
        torch.cuda.synchronize()
        print(json.dumps({"level": levels[0], "refine_ms": 1e3 * (time.time() - t0), **ref.stats()}))
        ref.close()
    wall.close()


def run_serving(args):
    """Serving workload: resident walls (channel 512/1024/2048 panels, star 1024
    panels); each request refines 1-64 contiguous panels by 2-6 levels and
    carries 1-32 right-hand sides from exterior point forces.  Closed loop
    (all requests at once) gives the saturation rate; an open loop with
    Poisson arrivals at 0.8 x that rate gives p50/p99 latency."""
    import torch
    from paper_2108_07205_gb300 import rwsolve, inputs
    rwsolve.load(build_if_missing=True)
    walls = [rwsolve.Wall("channel", 512), rwsolve.Wall("channel", 1024), rwsolve.Wall("channel", 2048),
             rwsolve.Wall("star", 1024, (0.3, 5, 1.0))]
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
    warm = [sv.submit(*make(10 ** 6 + i)[:5], nrhs=1)[0] for i in range(2)]
    for t in warm:
        sv.wait(t)
    reqs = [make(i) for i in range(args.requests)]
    t0 = time.time()
    tk = [sv.submit(w, p, l, s, f, nrhs=n, targets=tg)[0] for (w, p, l, s, f, n, tg) in reqs]
    lat_closed = [sv.wait(t) for t in tk]
    t_closed = time.time() - t0
    nsolves = sum(r[5] for r in reqs)
    sat = args.requests / t_closed
    lam = 0.8 * sat
    g = inputs.rng(4242)
    gaps = g.exponential(1.0 / lam, size=args.requests)
    reqs2 = [make(10 ** 5 + i) for i in range(args.requests)]
    t0 = time.time()
    tk2 = []
    for gap, (w, p, l, s, f, n, tg) in zip(gaps, reqs2):
        time.sleep(gap)
        tk2.append(sv.submit(w, p, l, s, f, nrhs=n, targets=tg)[0])
    lat_open = [sv.wait(t) for t in tk2]
    t_open = time.time() - t0
    nsolves2 = sum(r[5] for r in reqs2)
    sv.close()
    line = {"metric": "refined-wall solves/s (serving, open loop at 0.8 x saturation)",
            "value": nsolves2 / t_open, "unit": "solves/s", "n_gpus": 1, "steps": args.requests, "warmup": 2,
            "ms_per_step": 1e3 * t_open / args.requests, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "serving: walls channel 512/1024/2048 + star 1024 panels; requests refine "
                                   "1-64 panels by 2-6 levels with 1-32 RHS; 4 workers, 200 GB budget"},
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
    autotuned), against the same solves issued one instance at a time."""
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
        w = rwsolve.Wall("star", P, (a, k, 1.0))
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
    line = {"metric": "refined-wall solves/s (batched uneven walls, one persistent launch per 8 RHS)",
            "value": args.walls * nrhs / (ms / 1e3), "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.walls} star walls, 128-1024 panels, refined 2-16 panels by 2-4 levels, "
                                   "8 RHS each; solve only (walls and refinements static)",
                       "l2": "flushed before each solve"},
            "sequential_per_instance_solves_per_s": args.walls * nrhs / (ms_seq / 1e3),
            "autotuned_tile_rows": tr, "autotune_ms": tune_ms, "setup_s": setup_s,
            "rows": b.offsets[-1], "max_rel_diff_vs_individual": maxdiff}
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


def main():
    global P_PANELS, NRHS
    args = parse()
    if args.workload == "mixed2048":
        P_PANELS, NRHS = 2048, 64
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
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    value = world * args.steps * NRHS / (out["ms"] / 1e3)
    e2e = world * args.steps * NRHS / (out["ms_e2e"] / 1e3)
    # FP64 ALU peak: 152 SMs x 4 FP64 flop/clk (nominal 1.25 TFLOP/s at the
    # 2070 MHz maximum clock), evaluated at the median SM clock under load
    sm_mhz = (out["clocks"] or {}).get("sm_mhz") or 2070.0
    fp64_peak = 152 * 4 * sm_mhz * 1e6 / 1e12
    prof = out["prof"]
    dom = max(prof, key=lambda c: prof[c]["ms"])
    dp = prof[dom]
    dom_names = {"id": "column-pivoted QR (cluster and grid-wide kernels, FP64)", "gemm": "batched tiled GEMM (FP64)",
                 "gemv": "batched GEMV / HBS sweeps (FP64)", "inverse": "batched Gauss-Jordan inverse (FP64)",
                 "eval": "kernel-entry evaluation (FP64)", "other": "bookkeeping kernels"}
    if dom in ("id", "gemm", "inverse", "eval"):
        ach = dp["flops"] / (dp["ms"] / 1e3) / 1e12
        roof = {"kernel": dom_names[dom], "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": ach / fp64_peak, "traffic": None, "launches_per_step": dp["launches"] / args.steps,
                "avg_launch_ms": dp["ms"] / max(dp["launches"], 1),
                "peak_source": "derived FP64 peak (152 SMs x 4 flop/clk x median SM clock)"}
    else:
        ach = dp["bytes"] / (dp["ms"] / 1e3) / 1e9
        roof = {"kernel": dom_names[dom], "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": None, "launches_per_step": dp["launches"] / args.steps,
                "avg_launch_ms": dp["ms"] / max(dp["launches"], 1), "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    achieved = out["sweep_bytes"] / (out["sweep_ms"] / 1e3) / 1e9
    sweep_flops = 2.0 * out["hbs"]["inv_elems"]
    share = {c: round(prof[c]["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-9), 4) for c in prof}
    line = {
        "metric": "refined-wall solves/s", "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"gmres": "f64+f32", "gmres_bf16": "f64+bf16"}.get(args.mode, "f64"), "data": "synthetic",
        "config": workload_config(args),
        "p50_ms": float(np.percentile(out["lat"], 50)), "p99_ms": float(np.percentile(out["lat"], 99)),
        "solve_only_per_s": NRHS * 1e3 / out["solve_ms"], "k_mean": out["k_mean"], "n_p_range": out["np_range"],
        "hbs_build_s": out["build_s"], "gmres_iters": out["iters"] if args.mode in ("gmres", "gmres_bf16") else None,
        "e2e": {"value": e2e, "unit": "solves/s",
                "h2d_bytes_per_step": 8 * (2 * N_SRC + 2 * N_SRC * NRHS + 2 * TARGETS) if NRHS == 1 else
                8 * (4 * NRHS + 4 * NRHS * NRHS + 2 * TARGETS),
                "d2h_bytes_per_step": 8 * NRHS * (2 * TARGETS + 2 * 16 * P_PANELS)},
        "roofline": roof,
        "kernel_time_share": share,
        "roofline_sweep": {"kernel": "HBS inverse sweep (s1, FP64, 1 RHS, L2 flushed)", "ms": out["sweep_ms"],
                           "hbm_achieved_gbs": achieved, "hbm_frac": achieved / hbm,
                           "fp64_achieved_tflops": sweep_flops / (out["sweep_ms"] / 1e3) / 1e12,
                           "fp64_frac": sweep_flops / (out["sweep_ms"] / 1e3) / 1e12 / fp64_peak},
        "clocks": out["clocks"],
        "gpu_launches": out["launches"],
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
