"""Benchmark of the fused D3Q19 MRT-LES + STG channel step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                [--config c4] [--precision fp32|fp16|bf16|fp16row]

One bench step is one time step of the method over the whole lattice: the STG
inlet ring refill (every 64 steps, beside the steps), the interior and wall-row
step kernels (stream, inlet, wall model, collide), and the FP64 statistics
every 10 steps.  Default workload: the Re_tau = 5200 channel, 1536 x 192 x 384
lattice (113 M cells), N = 400 STG modes, FP32 storage; the two lattices
(17.2 GB) exceed the 129 MB L2, so no L2 flush is needed between steps.  The
headline is the median of repeated regions of exactly K steps; the step
kernels' roofline comes from a separate pass; the line also carries the 16-bit
storages and the FP16 / FP32 ratios at three lattice sizes, the adjoint cost,
an end-to-end loop through the C ABI with host buffers, and the FP64 oracle on
the host cores.

Prints one JSON line (rank 0).  With N > 1 (torchrun) the channel is cut into
N x-slabs, one per GPU, with the halo moved over NCCL before every step:
strong scaling, the whole channel's cells per second.
"""
import argparse
import ctypes as ct
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS of fused D3Q19 MRT-LES+STG step & % HBM roofline; adjoint/forward time"

CONFIGS = {
    "c1": dict(shape=(64, 32, 32), re_tau=1000.0, n_modes=100, seed=1,
               name="small channel 64x32x32 (4d x 2d x 2d), Re_tau=1000, N=100 STG modes"),
    "c2": dict(shape=(384, 96, 96), re_tau=1000.0, n_modes=200, seed=2,
               name="Re_tau=1000 channel 384x96x96, N=200 STG modes"),
    "c3": dict(shape=(768, 128, 192), re_tau=2000.0, n_modes=300, seed=3,
               name="Re_tau=2000 channel 768x128x192, N=300 STG modes"),
    "c4": dict(shape=(1536, 192, 384), re_tau=5200.0, n_modes=400, seed=4,
               name="Re_tau=5200 channel 1536x192x384, N=400 STG modes"),
}
BYTES_PER_CELL = {"fp32": 152, "fp16": 76, "bf16": 76, "fp16row": 76}   # 19 loads + 19 stores
STATS_EVERY = 10


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """The largest x over the ranks (a job's time is its slowest rank's);
    x itself on one rank."""
    if ws == 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash():
    """Hash of the source of the kernels the traffic record holds (the pair,
    quad and wall-row step kernels, all in lbm_device.cuh)."""
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2304_04214_gb300", "csrc", "lbm_device.cuh"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


KERNEL_NAMES = {"cell": "lbmk::step_kernel", "pair": "lbmk::step2_kernel + lbmk::wall_kernel",
                "quad": "lbmk::step4_kernel + lbmk::wall_kernel",
                "staged": "lbmk::staged_kernel + lbmk::wall_kernel"}


def recorded_traffic(cfg_key, precision, kernel, ncell):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None when the summary is for another build of the kernel."""
    try:
        with open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    ent = rec.get("entries", {}).get(f"{cfg_key}_{precision}_{kernel}")
    if not ent:
        return None
    return ent["bytes_per_cell"] * ncell


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 6:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        s = sorted(sm)
        return {"sm_mhz": s[len(s) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def smi_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [p for p in vis.split(",") if p.strip()]
    if parts and parts[min(local_rank, len(parts) - 1)].strip().isdigit():
        return int(parts[min(local_rank, len(parts) - 1)])
    return local_rank


# --------------------------------------------------------------------------
def cpu_oracle_mlups(cfg, budget_s=10.0, steps=None, nz_sample=None, warmup=0):
    """Time the FP64 oracle on this host's cores on the workload's lattice (or a
    spanwise slice of it), returning (MLUPS, threads, sample description)."""
    from oracle.oracle import Oracle, default_config, oracle_threads
    from paper_2304_04214_gb300.inputs import stg_uniforms
    nx, ny, nz = cfg["shape"]
    nzs = nz if nz_sample is None else nz_sample
    un = stg_uniforms(cfg["n_modes"], cfg["seed"])
    o = Oracle(default_config(nx, ny, nzs, re_tau=cfg["re_tau"], n_modes=cfg["n_modes"], stats=0),
               uniforms=un)
    if warmup:
        o.step(warmup)
    if steps is None:
        t0 = time.perf_counter()
        o.step(1)
        t1 = time.perf_counter() - t0
        n = max(1, int(budget_s / max(t1, 1e-6)) - 1)
        t0 = time.perf_counter()
        o.step(n)
        dt = time.perf_counter() - t0 + t1
        n += 1
    else:
        n = steps
        t0 = time.perf_counter()
        o.step(n)
        dt = time.perf_counter() - t0
    mlups = nx * ny * nzs * n / dt / 1e6
    return mlups, oracle_threads(), f"{nx}x{ny}x{nzs} lattice, {n} steps, {dt:.1f} s", dt, n


def run_reference(args, cfg, ws, rank):
    if rank != 0:
        return
    from oracle import build as ob
    ob.build()
    # calibrate a spanwise slice so that W + K steps take about two minutes
    nx, ny, nz = cfg["shape"]
    m1, _, _, dt1, n1 = cpu_oracle_mlups(cfg, steps=1, nz_sample=max(1, nz // 8))
    per_cell = 1.0 / (m1 * 1e6)
    budget = 120.0 / max(1, args.steps + args.warmup)
    nzs = int(max(1, min(nz, budget / (per_cell * nx * ny))))
    mlups, thr, sample, dt, n = cpu_oracle_mlups(cfg, steps=args.steps, nz_sample=nzs, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * dt / n, 3), "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg["name"] + " (oracle on a spanwise slice)", "storage": "fp64",
                   "lattice": list(cfg["shape"]), "sample_lattice": [nx, ny, nzs]},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": thr, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
def timed_region(ch, steps, barrier, stream):
    """Device time in ms of exactly `steps` steps (of a channel, or of this
    rank's slab with its halo exchanges): barrier and synchronize on both
    sides, CUDA events on the library's stream."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    ch.step(steps)
    e1.record(stream)
    barrier()
    return e0.elapsed_time(e1)


def repeat_count(first_ms, min_total_ms=1000.0, lo=3, hi=50):
    """Repeats of the timed region: at least `lo`, and enough that all of them
    together last about `min_total_ms`."""
    return int(max(lo, min(hi, -(-min_total_ms // max(first_ms, 1e-3)))))


def median(xs):
    s = sorted(xs)
    n = len(s)
    return s[n // 2] if n % 2 else 0.5 * (s[n // 2 - 1] + s[n // 2])


def kernel_pass(ch, steps, stepper=None):
    """Mean CUDA-event time in ms of one step's step kernels (interior and wall
    rows, the side stream joined inside), every step bracketed, graphs off:
    a pass of its own, after the headline region, so that its events do not
    cost the timed steps anything.  `stepper` (a slab) steps with its halo
    exchanges, which stay outside the brackets."""
    import ctypes as ct
    from paper_2304_04214_gb300 import _abi
    lib, h = ch.lib, ch.h
    ms_k, nk, nall = ct.c_double(), ct.c_long(), ct.c_long()
    ch.set_graphs(False)
    _abi.check(lib.lbm_profile_enable(h, 1), "lbm_profile_enable")
    lib.lbm_profile_read(h, ct.byref(ms_k), ct.byref(nk), ct.byref(nall))    # reset
    (stepper or ch).step(steps)
    _abi.check(lib.lbm_profile_read(h, ct.byref(ms_k), ct.byref(nk), ct.byref(nall)), "lbm_profile_read")
    lib.lbm_profile_enable(h, 0)
    ch.set_graphs(True)
    return ms_k.value / max(nk.value, 1), nk.value


def storage_sweep(dev, args, barrier, stream, fp32_c4_mlups):
    """Whole-step MLUPS of the other storages and lattices, each the median of
    three timed regions of about 0.3 s: the 16-bit storages at 1536x192x384
    and FP32 / FP16 / FP16 row base at 768x128x192 and 384x96x96, with the
    16-bit / FP32 ratios the 1.6x target refers to."""
    import torch
    from paper_2304_04214_gb300.channel import LBMChannel
    peaks, _ = measured_peaks()
    out = {}
    for key, prec in (("c4", "fp16"), ("c4", "bf16"), ("c4", "fp16row"), ("c3", "fp32"), ("c3", "fp16"),
                      ("c3", "fp16row"), ("c2", "fp32"), ("c2", "fp16"), ("c2", "fp16row")):
        if key == args.config and prec == args.precision:
            continue
        cfg = CONFIGS[key]
        nx, ny, nz = cfg["shape"]
        ncell = nx * ny * nz
        ch = LBMChannel(nx, ny, nz, re_tau=cfg["re_tau"], n_modes=cfg["n_modes"], seed=cfg["seed"],
                        precision=prec, stats_every=STATS_EVERY, device=dev)
        ch.step(20)
        first = timed_region(ch, 64, barrier, stream)
        steps = max(64, int(300.0 / max(first / 64, 1e-4)))
        ms = median([timed_region(ch, steps, barrier, stream) for _ in range(3)])
        kern_ms, _ = kernel_pass(ch, 64)
        ch.close()
        del ch
        torch.cuda.empty_cache()
        mlups = ncell * steps / (ms * 1e-3) / 1e6
        b = BYTES_PER_CELL[prec] * ncell
        out[f"{key}_{prec}"] = {"lattice": [nx, ny, nz], "mlups": round(mlups, 1), "steps": steps,
                                "ms_per_step": round(ms / steps, 5), "kernel_ms": round(kern_ms, 5),
                                "frac_whole_step": round(b / (ms / steps * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                                "frac": round(b / (kern_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
    m = {k: v["mlups"] for k, v in out.items()}
    if args.config == "c4" and args.precision == "fp32":
        m["c4_fp32"] = fp32_c4_mlups
    ratios = {}
    for prec in ("fp16", "fp16row"):
        ratios[prec] = {c: round(m[f"{c}_{prec}"] / m[f"{c}_fp32"], 3) for c in ("c2", "c3", "c4")
                        if f"{c}_{prec}" in m and f"{c}_fp32" in m}
    return out, ratios


def run_native(args, cfg, ws, rank, local):
    import numpy as np
    import torch
    from paper_2304_04214_gb300 import _abi
    from paper_2304_04214_gb300.channel import LBMChannel

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    nx, ny, nz = cfg["shape"]
    ncell = nx * ny * nz
    kw = dict(re_tau=cfg["re_tau"], n_modes=cfg["n_modes"], seed=cfg["seed"], precision=args.precision,
              stats_every=STATS_EVERY, step_kernel=args.kernel, device=dev)
    if ws > 1:
        # one channel cut into x-slabs, one per rank, halos over NCCL: strong scaling
        from paper_2304_04214_gb300.slab import P2PTransport, SlabChannel
        run = SlabChannel(nx, ny, nz, rank, ws, P2PTransport(device_buffers=True), **kw)
        ch = run.ch
    else:
        run = ch = LBMChannel(nx, ny, nz, **kw)
    ch.set_graphs(args.graphs == "on")
    local_cells = ch.ncell
    lib, h = ch.lib, ch.h
    kernel = ch.step_kernel
    stream = torch.cuda.current_stream(dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()

    # ---- warm-up ----
    barrier()                                    # (under NCCL: a first collective of all ranks)
    run.step(args.warmup)
    ch.sync()
    barrier()

    # ---- timed region: exactly K steps, repeated (median), nothing else on
    # the stream; clocks sampled throughout ----
    ms_k, nk, nall = ct.c_double(), ct.c_long(), ct.c_long()
    regions = []
    with ClockSampler(smi_index(local)) as clk:
        lib.lbm_profile_read(h, ct.byref(ms_k), ct.byref(nk), ct.byref(nall))   # reset the launch count
        regions.append(timed_region(run, args.steps, barrier, stream))
        lib.lbm_profile_read(h, ct.byref(ms_k), ct.byref(nk), ct.byref(nall))
        launches = int(nall.value)
        reps = repeat_count(regions[0]) if args.repeats <= 0 else args.repeats
        if ws > 1:                                   # every rank times the same number of regions
            reps = int(max_over_ranks(reps, ws, dev))
        for _ in range(reps - 1):
            regions.append(timed_region(run, args.steps, barrier, stream))
    ch.sync()
    ms = median(regions)
    ms = max_over_ranks(ms, ws, dev)
    value = ncell * args.steps / (ms * 1e-3) / 1e6      # the whole channel, over all ranks
    ms_step = ms / args.steps

    # ---- roofline of the step kernels, from a pass of its own ----
    peaks, peak_kind = measured_peaks()
    kern_steps = max(64, min(args.steps, 256))
    kern_ms, kern_n = kernel_pass(ch, kern_steps, run if ws > 1 else None)
    alg_bytes = BYTES_PER_CELL[args.precision] * local_cells          # this GPU's lattice
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    traffic = recorded_traffic(args.config, args.precision, kernel, ncell)
    if kern_ms > ms_step:
        print(f"bench: step kernels {kern_ms:.5f} ms > whole step {ms_step:.5f} ms", file=sys.stderr)
    traffic = traffic if ws == 1 else None

    # ---- end to end through the C ABI with host buffers ----
    # each step: the RANS-side inlet profile (U, R) from pinned host memory,
    # one time step, and that step's z-averaged wall shear copied back into
    # one of two pinned buffers; the host takes step n's wall shear while
    # step n + 1 runs (the one-step lag of a RANS/LES coupling loop)
    U = torch.empty(ny, dtype=torch.float64).pin_memory()
    R = torch.empty(6 * ny, dtype=torch.float64).pin_memory()
    tws = [torch.empty(2 * nx, dtype=torch.float64).pin_memory() for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    dp = lambda x: ct.cast(x.data_ptr(), ct.POINTER(ct.c_double))   # noqa: E731
    _abi.check(lib.lbm_get_inlet_profile(h, dp(U), dp(R)), "lbm_get_inlet_profile")
    n_e2e = int(max(args.steps, min(2000, 500.0 / max(ms_step, 1e-4))))
    taken = []

    def coupled_step(n):
        _abi.check(lib.lbm_set_inlet_profile(h, dp(U), dp(R)), "lbm_set_inlet_profile")
        if ws > 1:
            run.step(1)
        else:
            _abi.check(lib.lbm_step(h, 1), "lbm_step")
        _abi.check(lib.lbm_wall_shear_async(h, dp(tws[n % 2])), "lbm_wall_shear_async")
        evs[n % 2].record(stream)
        if n >= 1:                                 # step n - 1's wall shear is on the host
            evs[(n - 1) % 2].synchronize()
            taken.append(float(tws[(n - 1) % 2][0]))

    for n in range(3):
        coupled_step(n)
    barrier()
    taken.clear()
    t0 = time.perf_counter()
    for n in range(n_e2e):
        coupled_step(n)
    evs[(n_e2e - 1) % 2].synchronize()
    taken.append(float(tws[(n_e2e - 1) % 2][0]))
    barrier()
    dt_e2e = time.perf_counter() - t0
    dt_e2e = max_over_ranks(dt_e2e, ws, dev)
    e2e = ncell * n_e2e / dt_e2e / 1e6
    assert len(taken) == n_e2e and np.all(np.isfinite(taken)) and np.all(np.isfinite(tws[0].numpy()))
    ch.sync()
    run.close()
    del ch, run
    torch.cuda.empty_cache()

    sweep, ratios = None, None
    if rank == 0 and ws == 1 and not args.no_sweep:
        sweep, ratios = storage_sweep(dev, args, barrier, stream, value)

    adjoint = None
    if rank == 0 and not args.no_adjoint:
        adjoint = adjoint_timing(dev)

    line = None
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            # a spanwise slice of the lattice keeps the oracle's memory (360 B
            # per cell) and the sample's duration bounded
            nzs = max(1, min(nz, int(2.0e6 // (nx * ny))))
            m, thr, sample, _, _ = cpu_oracle_mlups(cfg, budget_s=10.0, nz_sample=nzs)
            cpu = {"value": round(m, 3), "unit": "MLUPS", "cores": thr, "kind": "oracle",
                   "sample": sample}
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "repeats": len(regions), "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg["name"] + f", {args.precision.upper()} storage",
                       "lattice": list(cfg["shape"]), "re_tau": cfg["re_tau"],
                       "n_modes": cfg["n_modes"], "storage": args.precision,
                       "stats_every": STATS_EVERY,
                       "l2": "no flush: the two lattices (%.0f MB) exceed the 129 MB L2"
                             % (BYTES_PER_CELL[args.precision] * local_cells / 1e6),
                       "timing": "median of %d regions of exactly %d steps, each bracketed by a barrier and a "
                                 "device synchronize, CUDA events on the library's stream"
                                 % (len(regions), args.steps),
                       "parallelism": f"x-slabs over {ws} GPUs, halo over NCCL" if ws > 1 else "single",
                       "cuda_graphs": args.graphs == "on"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                         "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": round(achieved / peaks["hbm_gbs"], 4),
                         "traffic": traffic, "peak_source": peak_kind,
                         "kernel": KERNEL_NAMES[kernel],
                         "kernel_ms": round(kern_ms, 5), "kernel_timed_steps": kern_n,
                         "kernel_timing": "separate pass after the timed region, graphs off, every step's "
                                          "step kernels bracketed by CUDA events",
                         "kernel_ms_le_step_ms": bool(kern_ms <= ms_step),
                         "frac_whole_step": round(alg_bytes / (ms_step * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                         "algorithmic_bytes": alg_bytes},
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e, 1), "unit": "MLUPS", "steps": n_e2e,
                    "h2d_bytes_per_step": 7 * ny * 4, "d2h_bytes_per_step": 2 * nx * 8},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "storages": sweep,
            "fp16_over_fp32": ratios["fp16"] if ratios else None,
            "fp16row_over_fp32": ratios["fp16row"] if ratios else None,
            "adjoint": adjoint,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()               # rank 0's extra work (adjoint, line) is done
        torch.distributed.destroy_process_group()
    return line


def adjoint_timing(dev, reps=3):
    """Adjoint cost on the adjoint workload: Re_tau = 1000, 256x64x64, N = 100,
    a 64-step window with a checkpoint every 8 steps, J_tau over 24 <= i < 48
    and J_R at i = 40.  forward = 64 plain steps; the adjoint call runs the same
    64 steps (storing checkpoints) plus the recomputation and the reverse
    sweep; ratio = (adjoint call - forward) / forward."""
    import torch
    from paper_2304_04214_gb300.channel import LBMChannel
    nx, ny, nz, N, T, K = 256, 64, 64, 100, 64, 8
    ch = LBMChannel(nx, ny, nz, re_tau=1000.0, n_modes=N, seed=5, device=dev)
    stream = torch.cuda.current_stream(dev)
    obj = (24, 48, 40)
    ch.adjoint_step(T, K, obj)            # warm-up (binds the workspace)
    ch.step(T)
    torch.cuda.synchronize(dev)
    fw, ad = [], []
    for _ in range(reps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ch.step(T)
        e1.record(stream)
        e1.synchronize()
        t0 = time.perf_counter()
        J, dJ = ch.adjoint_step(T, K, obj)
        ad.append((time.perf_counter() - t0) * 1e3)
        fw.append(e0.elapsed_time(e1))
    ch.close()
    f, a = min(fw), min(ad)
    return {"workload": "Re_tau=1000 channel 256x64x64, N=100, window 64, checkpoint every 8",
            "forward_ms": round(f, 3), "adjoint_call_ms": round(a, 3),
            "ratio": round((a - f) / f, 3), "J": J,
            "dJ_dtheta": [float(x) for x in dJ]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--config", default="c4", choices=sorted(CONFIGS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16", "fp16row"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--kernel", default="auto", choices=["auto", "cell", "pair", "quad", "staged"])
    ap.add_argument("--graphs", default="on", choices=["on", "off"],
                    help="launch STG ring periods of steps as CUDA graphs")
    ap.add_argument("--repeats", type=int, default=0,
                    help="timed regions of K steps (median reported); 0: enough for about 1 s, at least 3")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the other storages and lattices (16-bit / FP32 ratios)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        run_reference(args, cfg, ws, rank)
    else:
        run_native(args, cfg, ws, rank, local)


if __name__ == "__main__":
    main()
