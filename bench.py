"""Benchmark of the differentiable MLS-MPM hot path (forward + reverse rollouts) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

One timed step = one whole rollout of the workload (every simulation step: controller, bin/sort,
P2G, grid, G2P) plus its full reverse pass (segment recompute from checkpoints, adjoint scatter,
grid adjoint, adjoint gather, controller adjoint), with the inputs resident in HBM.  The default
workload is the largest one that fits one GPU, the 3D box cluster: 128^3 grid, 1,000,000
particles, 200 steps, sinusoid actuation of 64 groups, the checkpoint store limited to 4 GiB (every
15th state kept, segments recomputed in the reverse pass), loss = mean final x_0.  The 2D walker
(~31k particles, 1000 steps, checkpoint every 64) and the other workloads are reported beside it.
Prints one JSON line (rank 0).

--impl reference times the FP64 CPU oracle (the reference arm of this method) on a bounded
sample of the same workload.  With N > 1 (torchrun), every rank runs an independent replica
(scenes are independent; no collective on the data path) and the value is the sum over ranks.
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

import numpy as np  # noqa: E402

METRIC = "particle-steps/s fwd and fwd+bwd at oracle tolerance; rollout p50/p99 latency"
UNIT = "particle-steps/s"

# Algorithmic bytes per particle of each timed kernel kind (FP32 state records: 2D x2 F4 v2 C4 =
# 48 B, 3D 96 B; group id 4 B).  Grid-node bytes are not counted (they are a few bytes per particle
# at these densities), so `achieved` is a lower bound.
ALGO_BYTES = {
    # kind: (2D, 3D)
    "adj_gather": (48 + 48 + 48 + 4, 96 + 96 + 96 + 4),  # state n + adjoint n+1 in, adjoint n out, group
    "p2g_adj": (48 + 48 + 4, 96 + 96 + 4),               # state n + adjoint n+1 in, group
    "p2g": (48 + 4, 96 + 4),                             # state in, group
    "g2p": (24 + 48, 48 + 96),                           # x, F in; state out
}
# with per-particle material: E_p and m_p read by the P2G kernels and the adjoint gather, and the
# (dL/dE_p, dL/dm_p) accumulator read and written by the adjoint gather
MATERIAL_EXTRA = {"adj_gather": 8 + 16, "p2g_adj": 8, "p2g": 8, "g2p": 0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="box_cluster_3d")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-material", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-replicas", action="store_true")
    ap.add_argument("--no-soft", action="store_true")
    ap.add_argument("--no-walker", action="store_true")
    ap.add_argument("--no-permuted", action="store_true")
    ap.add_argument("--no-paper-cube", action="store_true")
    ap.add_argument("--no-cpu-aggregate", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--no-budget-sweep", action="store_true")
    ap.add_argument("--ncu-fp64", action="store_true",
                    help="short run for profilers: the FP64 form on a 200k-particle 3D cluster (64^3 grid), "
                         "2 steps and their reverse pass")
    ap.add_argument("--ncu", type=int, default=0, metavar="SIM_STEPS",
                    help="profiling mode: one short rollout of SIM_STEPS steps + reverse pass, no timing")
    return ap.parse_args()


def material_variant(spec):
    from paper_1810_01054_gb300 import scenes as S
    return S.with_material(spec, 21)


def workload(name, rank=0):
    from paper_1810_01054_gb300 import scenes as S
    seeds = {"walker_square_2d": 0, "walker_2d": 1, "soft_body_3d": 2, "box_cluster_3d": 3}
    spec = S.WORKLOADS[name](seeds[name] + 1000 * rank)
    return spec


def ckpt_of(spec):
    return spec.ckpt_interval if spec.ckpt_interval else 0


# Device-memory budget of the checkpoint store per workload (0 = no limit): the 1M-particle cluster
# keeps its checkpoints within 4 GiB, where the library takes a checkpoint every 7 steps (the
# smallest interval whose store, with the overlapped recompute's, fits).
BUDGET = {"box_cluster_3d": 4 << 30}


def budget_of(spec):
    return BUDGET.get(spec.name, 0)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def kernel_source_hash():
    h = hashlib.sha1()
    for f in ("mpm_kernels.cu", "mpm_device.cuh"):
        with open(os.path.join(ROOT, "paper_1810_01054_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_traffic(kernel, workload_name, n_particles):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled to this workload's
    particle count; None if no capture matches the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
        e = rec.get(workload_name, {}).get(kernel)
        if not e or e.get("kernel_hash") != kernel_source_hash():
            return None
        return e["dram_bytes_per_particle"] * n_particles
    except (ValueError, KeyError, OSError):
        return None


PLANES_BYTES = {2: 48, 3: 96}  # particle state bytes (x, F, v, C as float4 planes)
L2_BYTES = 129 * 10 ** 6


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            p = json.load(open(path))
            return float(p["hbm_gbs"]), "measured"
        except (ValueError, KeyError):
            pass
    return 6800.0, "fallback"


def host_record():
    """CPU model name and logical core count of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


def _oracle_sample(name, seed, n_steps, barrier, out):
    """One oracle process: builds its scene, waits for the others, then runs forward + reverse of
    the first n_steps of workload `name` with `seed`; puts (particle-steps, start, end) on `out`."""
    from oracle import oracle as O
    from paper_1810_01054_gb300 import scenes as S
    spec = S.WORKLOADS[name](seed)
    sc = O.Scene(spec)
    seed_g = np.zeros((sc.N, sc.dim))
    seed_g[:, 0] = 1.0 / sc.N
    barrier.wait()
    t0 = time.time()
    tr = sc.rollout(n_steps)
    sc.backward(tr, (seed_g, None, None, None))
    out.put((sc.N * n_steps, t0, time.time()))


def cpu_baseline(spec, budget_s=20.0, aggregate=True):
    """The FP64 oracle, as it stands: forward + reverse over the first steps of the workload, as
    many as fit in about `budget_s` seconds, on one host core; then one oracle process per core,
    each on an independent seeded scene of the same workload (scenes are independent), for the
    host's aggregate rate.  The rate is per particle-step, so a sample of the first steps stands
    for the whole rollout without extrapolation of anything but the step mix."""
    from oracle import oracle as O
    sc = O.Scene(spec)
    seed = np.zeros((sc.N, sc.dim))
    seed[:, 0] = 1.0 / sc.N
    t0 = time.time()
    tr = sc.rollout(1)
    sc.backward(tr, (seed, None, None, None))
    per = max(time.time() - t0, 1e-3)
    n = int(max(1, min(spec.n_steps, budget_s / per)))
    t0 = time.time()
    tr = sc.rollout(n)
    sc.backward(tr, (seed, None, None, None))
    dt = time.time() - t0
    del tr, sc
    rec = {"value": spec.n_particles * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"FP64 oracle forward+reverse of the first {n} of {spec.n_steps} steps of {spec.name} "
                     f"({spec.n_particles} particles), single thread, {dt:.1f} s", **host_record()}
    if aggregate:
        import multiprocessing as mp
        mpc = mp.get_context("spawn")  # never fork a process that holds a CUDA context
        cores = os.cpu_count() or 1
        barrier, out = mpc.Barrier(cores), mpc.Queue()
        procs = [mpc.Process(target=_oracle_sample, args=(spec.name, 77 + 1000 * i, n, barrier, out))
                 for i in range(cores)]
        for pr in procs:
            pr.start()
        res = [out.get() for _ in procs]
        for pr in procs:
            pr.join()
        units = sum(u for u, _, _ in res)
        wall = max(e for _, _, e in res) - min(b for _, b, _ in res)
        rec["aggregate"] = {"value": units / wall, "unit": UNIT, "cores": cores, "processes": cores,
                            "sample": f"{cores} oracle processes at once, each forward+reverse of the first {n} "
                                      f"steps of its own seeded {spec.name}; {wall:.1f} s from the first start "
                                      f"to the last finish (scene set-up untimed)"}
    return rec


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    spec = workload(args.workload)
    sc = O.Scene(spec)
    seed = np.zeros((sc.N, sc.dim))
    seed[:, 0] = 1.0 / sc.N
    # bounded sample per step: enough simulation steps for ~2 s of CPU work (one step of the
    # 1M-particle cluster takes longer than that on its own)
    t0 = time.time()
    tr = sc.rollout(1)
    sc.backward(tr, (seed, None, None, None))
    per = max(time.time() - t0, 1e-3)
    n = int(max(1, min(spec.n_steps, 2.0 / per)))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.time()
        tr = sc.rollout(n)
        sc.backward(tr, (seed, None, None, None))
        if i >= args.warmup:
            times.append(time.time() - t0)
    tot = sum(times)
    value = sc.N * n * len(times) / tot
    sample = (f"FP64 oracle forward+reverse of the first {n} of {spec.n_steps} steps of {spec.name} "
              f"({sc.N} particles) per step, single thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": spec.name, "particles": sc.N, "sim_steps_per_step": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             **host_record()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- multi-rank
def whole_job_rate(local_ms, units_per_rank, world, device=None):
    """Whole-job throughput over N independent replicas: the timed span is the maximum over
    ranks, the units are those of every rank (weak scaling; no collective on the data path)."""
    import torch
    t = torch.tensor([float(local_ms)], device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    span_ms = float(t.item())
    return world * units_per_rank / (span_ms / 1e3), span_ms


# ----------------------------------------------------------------------------- our arm
def measure(args, spec, rank, world, dev, stream, ctx, *, e2e=True, plain=True):
    """Times K whole forward+reverse rollouts of `spec` (graph replays, inputs resident in HBM, L2
    flushed before every step), then per-kernel durations in a directly-launched repeat, forward-only
    rollouts, optionally the end-to-end host-buffer path and the plain atomic form."""
    import torch
    from paper_1810_01054_gb300 import mpm

    T, k, budget = spec.n_steps, ckpt_of(spec), budget_of(spec)
    N, d = spec.n_particles, spec.dim
    scene = mpm.Scene(ctx, spec)
    k_eff = scene.plan_rollout(T, k, budget)[0]  # the interval the library takes (0: multi-level)
    x0 = torch.tensor(spec.x0, dtype=torch.float32, device=dev)
    v0 = torch.tensor(spec.v0, dtype=torch.float32, device=dev)
    C0 = torch.tensor(spec.C0, dtype=torch.float32, device=dev)
    F0 = torch.tensor(spec.F0, dtype=torch.float32, device=dev)
    seed = torch.zeros((N, d), dtype=torch.float32, device=dev)
    seed[:, 0] = 1.0 / N
    outs = [torch.empty((N, d), device=dev), torch.empty((N, d), device=dev), torch.empty((N, d, d), device=dev),
            torch.empty((N, d, d), device=dev), torch.empty((max(scene.n_params, 1),), device=dev)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_step(backward=True, sc=scene):
        sc.set_state(x0, v0, C0, F0, step=0)
        sc.rollout(T, k, budget)
        if backward:
            sc.backward(seed, out=outs)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        one_step()
    barrier()

    # -- timed region: K whole fwd+bwd rollouts (graph replays), L2 flushed before each (untimed)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    n_launch0 = mpm.launch_count()
    with ClockSampler(dev.index) as clk:
        barrier()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            one_step()
            ev[i][1].record(stream)
        barrier()
    n_launch = mpm.launch_count() - n_launch0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, tot_ms = whole_job_rate(sum(step_ms), N * T * args.steps, world, dev)

    # -- per-kernel durations: CUDA events around every launch of the hot kernels, in a repeat of
    #    the timed steps launched directly (event pairs cannot bracket kernels inside a graph)
    kinds = (("adj_gather", mpm.K_ADJ_GATHER), ("p2g_adj", mpm.K_P2G_ADJ), ("p2g", mpm.K_P2G), ("g2p", mpm.K_G2P),
             ("sort", mpm.K_SORT), ("ctrl", mpm.K_CTRL))
    ctx.profile_start([kk for _, kk in kinds], max_launches=args.steps * 12 * T + 64)
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    pa.record(stream)
    for i in range(args.steps):
        one_step()
    pb.record(stream)
    barrier()
    prof_total_ms = pa.elapsed_time(pb)
    prof = {nm: ctx.profile_read(kk) for nm, kk in kinds}
    ctx.profile_start([], max_launches=0)

    # -- forward-only throughput (same rollouts without the reverse pass)
    fwd_ms = []
    for i in range(max(2, args.steps // 2)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        one_step(backward=False)
        b.record(stream)
        torch.cuda.synchronize(dev)
        fwd_ms.append(a.elapsed_time(b))
    value_fwd = world * N * T / (statistics.median(fwd_ms) / 1e3)

    # -- e2e through the public API with pinned host buffers (H2D inputs, D2H gradients)
    e2e_rec = None
    if e2e:
        hx = torch.tensor(spec.x0, dtype=torch.float32).pin_memory()
        hv = torch.tensor(spec.v0, dtype=torch.float32).pin_memory()
        hC = torch.tensor(spec.C0, dtype=torch.float32).pin_memory()
        hF = torch.tensor(spec.F0, dtype=torch.float32).pin_memory()
        hseed = seed.cpu().pin_memory()
        houts = [torch.empty(o.shape).pin_memory() for o in outs]
        h2d = sum(t.numel() * 4 for t in (hx, hv, hC, hF, hseed))
        d2h = sum(t.numel() * 4 for t in houts[:4]) + 4 * scene.n_params
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            scene.set_state(hx, hv, hC, hF, step=0)
            scene.rollout(T, k, budget)
            scene.backward(hseed, out=houts)
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_rec = {"value": world * N * T * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h}

    # -- the plain single-scene form (global float atomics, dense grid) on the same workload
    plain_rec = None
    if plain and rank == 0:
        ps = mpm.Scene(ctx, spec, impl=mpm.IMPL_PLAIN)
        for _ in range(2):
            one_step(sc=ps)
        torch.cuda.synchronize(dev)
        pm = []
        for _ in range(2):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            one_step(sc=ps)
            b.record(stream)
            torch.cuda.synchronize(dev)
            pm.append(a.elapsed_time(b))
        plain_rec = {"value": N * T / (min(pm) / 1e3), "unit": UNIT, "form": "plain single-scene (float atomics)"}
        ps.close()
    launch = {mpm.TILE_KERNELS[kk]: list(scene.launch(kk)) for kk in range(4)}  # [ctas/SM, threads, tuned]
    scene.close()

    # roofline of the dominant hot kernel (largest summed time in the profiled repeat)
    dom = max(ALGO_BYTES, key=lambda kk: prof[kk][1])
    cnt, ms = prof[dom]
    hbm, src = peaks()
    material = spec.E_arr is not None or spec.mass_arr is not None
    bpp = ALGO_BYTES[dom][0 if d == 2 else 1] + (MATERIAL_EXTRA[dom] if material else 0)
    launch_ms = ms / max(cnt, 1)
    achieved = bpp * N / (launch_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": measured_traffic(dom, spec.name, N), "peak_source": src, "algo_bytes_per_particle": bpp,
            "launches": cnt, "avg_launch_us": 1e3 * launch_ms,
            "timing": "CUDA events around every launch of the kernel in a directly-launched repeat of the timed steps"}
    work_mb = 3 * N * PLANES_BYTES[d] / 1e6  # a reverse step's state, adjoint in and adjoint out
    if work_mb * 1e6 < L2_BYTES:  # the step's working set stays in L2: HBM is not the limit
        roof["regime"] = (f"latency: a step's {work_mb:.1f} MB working set (state, adjoint in and out) stays in "
                          f"the 129 MB L2 across steps and each launch is one chain of per-tile dependent loads; "
                          f"the HBM-scale case is large_scene")
    share = {kk: round(v[1] / prof_total_ms, 4) for kk, v in prof.items()}
    return {"value": value, "tot_ms": tot_ms, "step_ms": step_ms, "value_fwd": value_fwd, "roofline": roof,
            "share": share, "e2e": e2e_rec, "plain": plain_rec, "gpu_launches": n_launch, "clocks": clk.summary(),
            "N": N, "T": T, "k": k_eff, "budget": budget, "launch": launch}


def measure_replicas(args, dev, stream, sizes=(1, 64, 1024, 4096), edges=(8, 4)):
    """The smallest workload (walker_square_2d: 1,024 particles, 100 steps, forward + reverse) as B
    independent replicas advanced together by one batch, B in `sizes`, for each tile edge in
    `edges` (8 x 8-cell tiles are what the library chooses for this sparse scene; 4 x 4 beside
    it): one such scene leaves the GPU idle (launch and latency bound); a batch fills it.  Each
    request is a rollout with its reverse pass (loss = mean final x_0); the timed span is
    admission to the last result (the replicas' states are reset before it, untimed), L2 flushed
    before it."""
    import torch
    from paper_1810_01054_gb300 import mpm
    from paper_1810_01054_gb300 import scenes as S
    base = S.walker_square_2d(0)
    T, N = base.n_steps, base.n_particles
    ctx = mpm.Context(dev.index, stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    by_edge = {}
    for edge in edges:
        spec = base.copy(tile_edge=edge)
        out = {}
        for B in sizes:
            scenes = [mpm.Scene(ctx, spec) for _ in range(B)]
            batch = mpm.Batch(ctx, 2)

            def reset():
                for sc in scenes:
                    sc.set_state(spec.x0, spec.v0, spec.C0, spec.F0, step=0)

            def run():
                slots = [batch.admit(sc, T, True) for sc in scenes]
                while not all(batch.poll(sl) for sl in slots):
                    batch.tick(16)
                bad = [batch.status(sl) for sl in slots if batch.status(sl) != mpm.MPM_OK]
                for sl in slots:
                    batch.release(sl)
                if bad:
                    raise RuntimeError(f"replica requests failed: {bad[:4]}")

            for _ in range(max(1, args.warmup)):
                reset()
                run()
            ms = []
            for _ in range(max(1, min(args.steps, 3))):
                reset()
                flush.zero_()
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms.append(e0.elapsed_time(e1))
            batch.close()
            for sc in scenes:
                sc.close()
            best = float(np.median(ms))
            out[str(B)] = {"value": B * N * T / (best / 1e3), "ms": best}
        by_edge[str(edge)] = out
    # the tile-edge autotuner on one such scene and on the 2D walker: each edge's pass of 64
    # forward steps and their reverse pass, after two untimed ones
    tuned = {}
    for tspec in (base, workload("walker_2d")):
        e, ms4, ms8 = mpm.tune_tile_edge(ctx, tspec, steps=64)
        tuned[tspec.name] = {"edge": e, "ms_per_step_4x4": ms4, "ms_per_step_8x8": ms8}
    ctx.close()
    return {"workload": spec.name, "particles_per_replica": N, "sim_steps": T, "unit": UNIT,
            "pass": "forward+reverse per replica, one batch", "tile_edge_chosen": edges[0],
            "by_replicas": by_edge[str(edges[0])], "by_tile_edge": by_edge, "tile_edge_tuning": tuned}


def measure_budget_sweep(args, dev, stream, budgets_gib=(32, 4, 1)):
    """Full-horizon gradient of the 1M-particle cluster (200 steps) under device-memory budgets for
    the checkpoint store: every state when they fit (k = 1); else every k-th state with the segments
    recomputed beside the reverse steps (k the smallest interval whose store fits);
    below that the multi-level store (a recursive schedule planned for the fewest recomputed steps).
    Each budget's final state and gradients are compared bit for bit with the first budget's."""
    import torch
    from paper_1810_01054_gb300 import mpm
    spec = workload("box_cluster_3d")
    T, N, d = spec.n_steps, spec.n_particles, spec.dim
    ctx = mpm.Context(dev.index, stream=stream)
    sc = mpm.Scene(ctx, spec)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    x0, v0, C0, F0 = t(spec.x0), t(spec.v0), t(spec.C0), t(spec.F0)
    seed = torch.zeros((N, d), dtype=torch.float32, device=dev)
    seed[:, 0] = 1.0 / N
    outs = [torch.empty((N, d), device=dev), torch.empty((N, d), device=dev), torch.empty((N, d, d), device=dev),
            torch.empty((N, d, d), device=dev), torch.empty((max(sc.n_params, 1),), device=dev)]
    final = [torch.empty((N, d), device=dev), torch.empty((N, d), device=dev), torch.empty((N, d, d), device=dev),
             torch.empty((N, d, d), device=dev)]
    S = sc.info()["state_bytes"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res, ref = {}, None
    for gib in budgets_gib:
        budget = gib << 30
        try:
            kk, fwd_steps, multi = sc.plan_rollout(T, 0, budget)
        except mpm.MPMError as e:
            res[f"{gib}GiB"] = {"status": e.status}
            continue
        # states stored at most: the multi-level plan's; the checkpoints and the two sets of recompute
        # buffers of the overlapped reverse pass
        stored = mpm.plan_checkpoints(T, budget // S)[1] if multi else (T + kk - 1) // kk + 2 * (kk - 1)
        rec = {"store": "multi-level" if multi else "single-level", "stored_states": stored,
               "store_gb": stored * S / 1e9, "forward_steps": fwd_steps}
        if not multi:
            rec["ckpt_interval"] = kk

        def one():
            sc.set_state(x0, v0, C0, F0, step=0)
            sc.rollout(T, 0, budget)
            sc.backward(seed, out=outs)

        try:
            one()
        except mpm.MPMError as e:
            rec["status"] = e.status
            res[f"{gib}GiB"] = rec
            continue
        sc.get_state(out=final)
        got = [o.clone() for o in outs + final]
        if ref is None:
            ref = got
        else:
            rec["bitwise_equal_to_" + f"{budgets_gib[0]}GiB"] = all(torch.equal(a, b) for a, b in zip(got, ref))
        ms = []
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        rec["value"] = N * T / (min(ms) / 1e3)
        rec["ms"] = min(ms)
        res[f"{gib}GiB"] = rec
    sc.close()
    ctx.close()
    return {"workload": spec.name, "particles": N, "sim_steps": T, "unit": UNIT, "state_bytes": S,
            "by_budget": res}


def measure_serving(dev, stream, n_requests=1000, seed=4, loads=(0.25, 0.5, 0.75, 0.9), per_load=250):
    """Serving mix (Poisson stream of rollout/gradient requests, 2D and 3D box clusters): first the
    saturation rate (all `n_requests` queued at once), then, for each load in `loads`, Poisson
    arrivals at that fraction of the saturation rate over `per_load` requests of the same mix;
    latency = arrival -> result on the host."""
    from paper_1810_01054_gb300 import scenes as S
    from paper_1810_01054_gb300.serve import Server
    reqs = [S.serving_request(i, seed) for i in range(n_requests)]

    def run(sub, arrivals):
        srv = Server(device=dev.index, mem_fraction=0.3, tick_steps=8, stream=stream, keep_results=False)
        for (sp, g), t in zip(sub, arrivals):
            srv.submit(sp, g, arrival=t)
        t0 = time.perf_counter()
        srv.run()
        span = time.perf_counter() - t0
        p50, p99 = srv.latency_percentiles()
        failed = sum(1 for r in srv.results.values() if r["status"] != 0)
        srv.close()
        return span, p50, p99, failed

    run(reqs[:8], [0.0] * 8)  # warm-up of the first requests' code paths
    work = sum(sp.n_particles * sp.n_steps for sp, _ in reqs)
    span, _, _, failed = run(reqs, [0.0] * n_requests)
    rate = n_requests / span
    rng = np.random.default_rng(seed)
    by_load = {}
    for i, load in enumerate(loads):
        sub = reqs[(i * per_load) % n_requests:][:per_load]
        arrivals = np.cumsum(rng.exponential(1.0 / (load * rate), size=len(sub)))
        span2, p50, p99, f2 = run(sub, list(arrivals))
        sub_work = sum(sp.n_particles * sp.n_steps for sp, _ in sub)
        by_load[str(load)] = {"requests": len(sub), "arrival_req_per_s": load * rate, "p50_ms": 1e3 * p50,
                              "p99_ms": 1e3 * p99, "aggregate_particle_steps_per_s": sub_work / span2,
                              "span_s": span2, "failed": f2}
    return {"requests": n_requests, "saturation_req_per_s": rate,
            "saturation_particle_steps_per_s": work / span, "saturation_failed": failed, "by_load": by_load,
            "mix": "seeded serving requests: dim 2/3 50/50, n in {32..128}, N log-uniform 1e3-2e5, T 50-500, "
                   "60% with gradient (loss = mean final x_0)",
            "percentiles": "numpy linear interpolation over each load's requests"}


# The paper's speed table (Table II): time per frame of its CUDA implementation on an NVIDIA GTX
# 1080 Ti for a falling elastic cube, forward (F) and backward (B); the steps per frame are not
# stated, so these are particle-frames/s, context rather than a like-for-like rate.
PAPER_TABLE2 = {
    "falling_cube_3d_8000": {"F_ms_per_frame": 0.392, "B_ms_per_frame": 0.406},
    "falling_cube_3d_64000": {"F_ms_per_frame": 1.594, "B_ms_per_frame": 1.774},
    "falling_cube_3d_512000": {"F_ms_per_frame": 10.501, "B_ms_per_frame": 11.594},
    "falling_cube_2d_6400": {"F_ms_per_frame": 0.10, "B_ms_per_frame": 0.14},
}


def measure_paper_cube(args, dev, stream, sizes=((3, 20), (3, 40), (3, 80), (2, 80)), T=100):
    """The paper's speed-comparison workload, a falling elastic cube at its particle counts:
    forward (T-step rollout keeping every state) and backward (the reverse pass alone) timed
    separately with device events, beside the paper's per-frame times on its GPU."""
    import torch
    from paper_1810_01054_gb300 import mpm
    from paper_1810_01054_gb300 import scenes as S
    ctx = mpm.Context(dev.index, stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {}
    for dim, side in sizes:
        spec = S.falling_cube(dim, side, n_steps=T)
        N = spec.n_particles
        sc = mpm.Scene(ctx, spec)
        seed = torch.zeros((N, dim), dtype=torch.float32, device=dev)
        seed[:, 0] = 1.0 / N
        outs = [torch.empty((N, dim), device=dev), torch.empty((N, dim), device=dev),
                torch.empty((N, dim, dim), device=dev), torch.empty((N, dim, dim), device=dev),
                torch.empty((1,), device=dev)]
        fwd, bwd = [], []
        for i in range(max(1, args.warmup) + 3):
            sc.set_state(spec.x0, spec.v0, spec.C0, spec.F0, step=0)
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            sc.rollout(T, 1)
            ev[1].record(stream)
            sc.backward(seed, out=outs)
            ev[2].record(stream)
            torch.cuda.synchronize(dev)
            if i >= max(1, args.warmup):
                fwd.append(ev[0].elapsed_time(ev[1]))
                bwd.append(ev[1].elapsed_time(ev[2]))
        sc.close()
        f_ms, b_ms = float(np.median(fwd)) / T, float(np.median(bwd)) / T
        paper = PAPER_TABLE2.get(spec.name, {})
        out[spec.name] = {"particles": N, "grid": "x".join(map(str, spec.n_grid)), "sim_steps": T,
                          "F_us_per_step": 1e3 * f_ms, "B_us_per_step": 1e3 * b_ms,
                          "F_particle_steps_per_s": N / (f_ms / 1e3), "B_particle_steps_per_s": N / (b_ms / 1e3),
                          "paper_gtx1080ti": {**paper,
                                              "F_particle_frames_per_s": N / (paper["F_ms_per_frame"] / 1e3),
                                              "B_particle_frames_per_s": N / (paper["B_ms_per_frame"] / 1e3)}}
    ctx.close()
    return {"workload": "falling elastic cube (Table II's scene; grid and material are this build's choice)",
            "unit": UNIT, "by_size": out,
            "paper_note": "the paper times frames of unstated step count on a GTX 1080 Ti: context only"}


# FP64 roofline: GB300 SMs issue 2 FP64 thread-ops per clock (the nominal 1.25 TFLOP/s FP64 rate:
# 152 SMs x 2 DFMA x 2 flops x 2.07 GHz); no measured FP64 peak exists for this machine.
F64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64 arithmetic of the per-particle adjoint kernel (S4 (F)-(K), (J)), DADD + DMUL + 2 DFMA thread
# instructions per particle from the ncu counters of the 3D capture (profiles/k64_fp64_box_cluster_3d.md)
F64_ADJ_FLOPS_3D = 3700.0


def table_of(spec, T):
    """The sinusoid actuation a_g(t_n) = A_g sin(2 pi f t_n) of a CTRL_SIN workload as a per-step
    table (the FP64 form's actuation input)."""
    t = np.arange(T) * spec.dt
    return np.asarray(spec.ctrl_params)[None, :] * np.sin(2 * np.pi * spec.ctrl_freq * t)[:, None]


def measure_fp64(args, dev, stream):
    """Double-precision plain form (the float64 accuracy case of Section VI): throughput of a
    1000-step forward+reverse rollout of the colliding-discs scene with the oracle timed beside it,
    the accuracy study (GPU adjoint vs GPU central differences), and the FP64-pipe roofline of the
    per-particle adjoint kernel on the 1M-particle 3D cluster (8 steps, sinusoid as a table)."""
    import torch
    from oracle import oracle as O
    from paper_1810_01054_gb300 import mpm
    from paper_1810_01054_gb300 import scenes as S

    ctx = mpm.Context(dev.index, stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    spec = S.billiards_2d()
    T, N = spec.n_steps, spec.n_particles
    a = S.billiards_ball_a(spec)
    w = np.zeros_like(spec.x0)
    w[~a, 0] = 1.0 / (~a).sum()  # loss: x centroid of ball B at step T
    sc = mpm.Scene64(ctx, spec)
    for _ in range(args.warmup):
        sc.rollout(T)
        sc.backward(w)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    for e in ev:
        flush.zero_()
        e[0].record(stream)
        sc.rollout(T)
        e[1].record(stream)
        sc.backward(w)
        e[2].record(stream)
    torch.cuda.synchronize(dev)
    fwd = [e[0].elapsed_time(e[1]) for e in ev]
    tot = [e[0].elapsed_time(e[2]) for e in ev]
    # accuracy: dL/d(vx of ball A) by the adjoint and by FP64 central differences (h = 1e-6)
    acc = {}
    for TT in (1, 10, 100, 1000):
        sc.set_state(spec.x0, spec.v0, spec.C0, spec.F0)
        sc.rollout(TT)
        g = float(sc.backward(w)[1][a, 0].sum())
        L = []
        for sgn in (1, -1):
            v0 = spec.v0.copy()
            v0[a, 0] += sgn * 1e-6
            sc.set_state(spec.x0, v0, spec.C0, spec.F0)
            sc.rollout(TT)
            L.append(float(np.sum(w * sc.get_state()[0])))
        fd = (L[0] - L[1]) / 2e-6
        acc[str(TT)] = {"adjoint": g, "fd": fd, "rel_err": abs(g - fd) / abs(fd) if g != 0.0 else None}
    sc.close()
    # the oracle on the same scene (bounded sample: 100 steps forward + reverse, one thread)
    osc = O.Scene(spec)
    t0 = time.time()
    tr = osc.rollout(100)
    osc.backward(tr, (w, None, None, None))
    odt = time.time() - t0
    # FP64-pipe roofline of the per-particle adjoint on the 1M-particle 3D cluster
    lspec = S.box_cluster_3d()
    LT, LN = 8, lspec.n_particles
    lsc = mpm.Scene64(ctx, lspec, act=table_of(lspec, LT))
    lw = np.zeros_like(lspec.x0)
    lw[:, 0] = 1.0 / LN
    lsc.rollout(LT)
    lsc.backward(lw)
    kinds = (("adjoint", mpm.K_F64_ADJ), ("p2g_adj", mpm.K_F64_P2G_ADJ), ("p2g", mpm.K_F64_P2G),
             ("g2p", mpm.K_F64_G2P), ("grid", mpm.K_F64_GRID))
    ctx.profile_start([k for _, k in kinds], max_launches=8 * LT + 16)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    e0.record(stream)
    lsc.rollout(LT)
    lsc.backward(lw)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    lms = e0.elapsed_time(e1)
    per = {nm: ctx.profile_read(k) for nm, k in kinds}
    lsc.close()
    ctx.close()
    n_adj, t_adj = per["adjoint"]
    adj_s = t_adj / max(n_adj, 1) / 1e3
    achieved = F64_ADJ_FLOPS_3D * LN / adj_s / 1e12
    return {
        "workload": spec.name, "particles": N, "sim_steps": T, "dtype": "f64",
        "pass": "forward+reverse rollout, every state kept; device events around the rollout and reverse calls",
        "value": N * T / (np.median(tot) / 1e3), "value_fwd": N * T / (np.median(fwd) / 1e3), "unit": UNIT,
        "ms_per_rollout_and_reverse": float(np.median(tot)),
        "accuracy": {"loss": "x centroid of ball B at step T", "wrt": "x velocity of every ball-A particle",
                     "fd": "central, h = 1e-6, GPU FP64", "by_steps": acc,
                     "paper_rel_err": {"100": 2.39e-8, "1000": 2.83e-8}},
        "oracle": {"value": N * 100 / odt, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"FP64 oracle forward+reverse of 100 steps of {spec.name}, single thread, {odt:.2f} s"},
        "large": {"workload": lspec.name, "particles": LN, "sim_steps": LT, "value": LN * LT / (lms / 1e3),
                  "unit": UNIT, "ms": lms,
                  "kernel_avg_us": {nm: 1e3 * t / max(n, 1) for nm, (n, t) in per.items()},
                  "roofline": {"bound": "alu", "kernel": "k64_adjoint<3>", "achieved": achieved,
                               "peak": F64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / F64_PEAK_TFLOPS,
                               "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz",
                               "flops_per_particle": F64_ADJ_FLOPS_3D}},
    }


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1810_01054_gb300 import mpm

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # a dedicated stream: the library enqueues on it and every event below is recorded on it
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = mpm.Context(local_rank, stream=stream)
    spec = workload(args.workload, rank)

    if args.ncu_fp64:
        from paper_1810_01054_gb300 import scenes as S
        fspec = S.box_cluster_3d(n_particles=200_000, n=64)
        sc = mpm.Scene64(ctx, fspec, act=table_of(fspec, 2))
        sc.rollout(2)
        seed = np.zeros_like(fspec.x0)
        seed[:, 0] = 1.0 / fspec.n_particles
        sc.backward(seed)
        sc.close()
        print(json.dumps({"ncu_run": "fp64 " + fspec.name, "particles": fspec.n_particles, "sim_steps": 2}), flush=True)
        return

    if args.ncu:
        # short run for profilers: one rollout of --ncu steps (checkpoint interval kept) + reverse pass
        T = min(spec.n_steps, args.ncu)
        sc = mpm.Scene(ctx, spec)
        sc.rollout(T, min(ckpt_of(spec), T) if ckpt_of(spec) else 0)
        seed = np.zeros((spec.n_particles, spec.dim), np.float32)
        seed[:, 0] = 1.0 / spec.n_particles
        sc.backward(seed)
        print(json.dumps({"ncu_run": spec.name, "sim_steps": T, "launches": mpm.launch_count()}), flush=True)
        return

    r = measure(args, spec, rank, world, dev, stream, ctx, e2e=not args.no_e2e, plain=not args.no_plain)

    def extra(xspec, rec):
        return {"workload": xspec.name, "particles": rec["N"], "grid": "x".join(map(str, xspec.n_grid)),
                "sim_steps": rec["T"], "ckpt_interval": rec["k"], "value": rec["value"],
                "value_fwd": rec["value_fwd"], "unit": UNIT, "ms_per_step": rec["tot_ms"] / args.steps,
                "roofline": rec["roofline"], "kernel_share_of_profiled_step": rec["share"],
                "launch": rec["launch"]}

    large = None
    if args.workload != "box_cluster_3d" and not args.no_large:
        lspec = workload("box_cluster_3d", rank)
        large = extra(lspec, measure(args, lspec, rank, world, dev, stream, ctx, e2e=False, plain=False))
    walker = None
    if args.workload != "walker_2d" and not args.no_walker:
        # the 2D soft walker: 31k particles, 1000 steps with a checkpoint every 64, basis controller
        wspec = workload("walker_2d", rank)
        walker = extra(wspec, measure(args, wspec, rank, world, dev, stream, ctx, e2e=False, plain=False))
    soft = None
    if args.workload != "soft_body_3d" and not args.no_soft:
        # the 3D soft body with its MLP controller on group centroids, 500 steps, checkpoint every
        # ceil(sqrt(500)) = 23 steps (forward+backward with recomputation)
        sspec = workload("soft_body_3d", rank)
        sspec = sspec.copy(ckpt_interval=int(np.ceil(np.sqrt(sspec.n_steps))))
        soft = extra(sspec, measure(args, sspec, rank, world, dev, stream, ctx, e2e=False, plain=False))
    permuted = None
    if not args.no_permuted:
        # the same workload with its particles handed over in a random order: the library's
        # storage order (by tile, cell and position) makes the kernels read neighbouring memory
        # anyway, so time and result bits match the ordered input
        pr = np.random.default_rng(17).permutation(spec.n_particles)
        pspec = spec.copy(x0=spec.x0[pr], v0=spec.v0[pr], C0=spec.C0[pr], F0=spec.F0[pr], group=spec.group[pr])
        pr_rec = measure(args, pspec, rank, world, dev, stream, ctx, e2e=False, plain=False)
        permuted = {"workload": spec.name + " (particles in a random order)", "value": pr_rec["value"],
                    "value_fwd": pr_rec["value_fwd"], "unit": UNIT, "ms_per_step": pr_rec["tot_ms"] / args.steps,
                    "ratio_to_ordered": pr_rec["value"] / r["value"], "roofline": pr_rec["roofline"]}
    sweep = None
    if rank == 0 and not args.no_budget_sweep:
        sweep = measure_budget_sweep(args, dev, stream)
    replicas = None
    if rank == 0 and not args.no_replicas:
        replicas = measure_replicas(args, dev, stream)
    material = None
    if not args.no_material:
        # the walker with per-particle Young's modulus and mass and their gradients
        mspec = material_variant(workload("walker_2d", rank))
        mr = measure(args, mspec, rank, world, dev, stream, ctx, e2e=False, plain=False)
        material = {"workload": mspec.name, "value": mr["value"], "value_fwd": mr["value_fwd"], "unit": UNIT,
                    "ms_per_step": mr["tot_ms"] / args.steps, "roofline": mr["roofline"],
                    "kernel_share_of_profiled_step": mr["share"],
                    "gradients": "dL/dx0, v0, C0, F0, controller parameters, E_p, m_p"}
    paper_cube = None
    if rank == 0 and not args.no_paper_cube:
        paper_cube = measure_paper_cube(args, dev, stream)
    serving = None
    if rank == 0 and not args.no_serve:
        serving = measure_serving(dev, stream, n_requests=args.serve_requests)
    fp64 = None
    if rank == 0 and not args.no_fp64:
        fp64 = measure_fp64(args, dev, stream)
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline(spec, aggregate=not args.no_cpu_aggregate)
    lat = sorted(r["step_ms"])
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["tot_ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": spec.name, "particles": r["N"], "grid": "x".join(map(str, spec.n_grid)),
                   "sim_steps": r["T"], "ckpt_interval": r["k"],
                   "ckpt_budget_bytes": r["budget"] or None,
                   "pass": "forward+reverse rollout (full-horizon gradient)",
                   "loss": "mean final x_0", "l2": "flushed before every timed step (256 MB write, untimed)",
                   "parallelism": f"replicas x{world}", "launch": r["launch"]},
        "value_fwd": r["value_fwd"],
        "rollout_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "roofline": r["roofline"], "kernel_share_of_profiled_step": r["share"],
        "cpu_baseline": cpu, "e2e": r["e2e"], "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
        "plain_form": r["plain"], "walker": walker, "large_scene": large, "material": material,
        "serving": serving, "fp64": fp64, "large_scene_budgets": sweep, "small_scene_replicas": replicas,
        "soft_body": soft, "permuted_order": permuted, "paper_workload": paper_cube,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
