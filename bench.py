"""Throughput of the forward propagator in Gpoint-updates/s on one or more GPUs.

One bench step = one mmod_forward: the whole hot path (interior and damping
updates, source injection, receiver gather, the nt-step time loop) over the
workload.  Default workload: 240^3 grid, 1000 steps, four-layer velocity model
with a smoothed +-5% perturbation, 20-cell damping layers, Ricker 10 Hz source
at depth 40 m, 240 x 240 surface receivers (synthetic, seeded).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mmod|reference]

With N > 1 the script runs under torch.distributed.run; each rank advances its
own replica of the workload on its own GPU (independent shots: weak scaling,
no collective on the data path), and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpoint-updates/s and % HBM roofline (fwd, adjoint, batched shots) at stated error"
UNIT = "Gpoint-updates/s"
BYTES_PER_POINT = 16      # read u^n, u^{n-1}, c; write u^{n+1} (FP32)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def make_workload(name: str, nt: int | None):
    import workloads as W
    if name == "layered240":
        return W.layered_240(nt or 1000)
    if name == "homogeneous64":
        return W.small_homogeneous(nt or 100)
    if name == "gradient200":
        return W.smooth_gradient_200(nt or 1000)
    raise SystemExit(f"unknown workload {name}")


def describe(p, extra=None):
    nz, ny, nx = p.vel.shape
    cfg = {"workload": p.name, "grid": [nx, ny, nz], "h_m": list(p.h), "nt": p.nt, "dt_s": p.dt,
           "nbl": p.nbl, "order": p.order, "nsrc": int(len(p.src_ijk)), "nrec": int(len(p.rec_ijk)),
           "cache": "inputs larger than L2: each time step streams three %.1f MB FP32 volumes (> 129 MB L2)"
                    % (nx * ny * nz * 4 / 1e6)}
    if extra:
        cfg.update(extra)
    return cfg


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        sm = [r[0] for r in rows]
        loaded = [r[0] for r in rows if r[2] > 200.0] or sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "power_w_max": max(r[2] for r in rows), "reasons": reasons}


PAPER_CONTEXT = {"value": 240 ** 3 * 300 / 30.47 / 1e9, "unit": UNIT,
                 "what": "the paper's sequential example run (acoustic_iso_cd, 240^3, 20 m, 300 steps, "
                         "Time Kernel 30.47 s, one thread, hardware not stated, FP32; Sec. 5.3): context, "
                         "a different configuration, not a baseline"}


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


_ALL_THREADS = None


def oracle_sample(p, seconds_target=20.0, max_steps=None, nthreads=0):
    """Time the FP64 oracle on the host cores on the first steps of the workload
    (nthreads 0: every core)."""
    import oracle
    global _ALL_THREADS
    oracle.build()
    if _ALL_THREADS is None:   # before any single-thread run changes the OpenMP default
        _ALL_THREADS = oracle.max_threads()
    threads = nthreads or _ALL_THREADS
    npts = p.npoints
    def run(n):
        t0 = time.perf_counter()
        oracle.forward(p.vel, p.h, p.dt, n, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet[:, :n],
                       rec_ijk=p.rec_ijk, nthreads=threads)
        return time.perf_counter() - t0

    # per-step time from the difference of two short runs (set-up cancels)
    t_a, t_b = run(1), run(5)
    per_step = max((t_b - t_a) / 4.0, 1e-6)
    steps = int(max(2, min(p.nt, seconds_target / max(per_step, 1e-6))))
    if max_steps:
        steps = min(steps, max_steps)
    t0 = time.perf_counter()
    oracle.forward(p.vel, p.h, p.dt, steps, nbl=p.nbl, src_ijk=p.src_ijk, wavelet=p.wavelet[:, :steps],
                   rec_ijk=p.rec_ijk, nthreads=threads)
    dt = time.perf_counter() - t0
    return {"value": npts * steps / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"{p.name}: first {steps} of {p.nt} steps, FP64, OpenMP {threads} threads, "
                      f"{dt:.1f} s"}, dt, steps


def weak_throughput(world: int, npts: int, nt: int, steps: int, ms: float) -> float:
    """Whole-job Gpoint-updates/s: every rank advanced its own replica."""
    return world * npts * nt * steps / (ms * 1e-3) / 1e9


def reduce_max(value: float, dist, device) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    p = make_workload(args.workload, args.nt)
    vals, secs = [], 0.0
    for _ in range(args.warmup):
        oracle_sample(p, seconds_target=2.0)
    for _ in range(args.steps):
        cb, dt, steps = oracle_sample(p, seconds_target=args.ref_seconds)
        vals.append(cb["value"])
        secs += dt
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": describe(p),
            "cpu_baseline": {**cb, "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def traffic_from_profiles(kernel_tag: str):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    valid only while the kernel's source hash matches."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    try:
        blob = b"".join(open(os.path.join(ROOT, "paper_2007_06048_gb300", "csrc", f), "rb").read()
                        for f in rec.get("source", []))
    except OSError:
        return None
    digest = hashlib.sha256(blob).hexdigest()[:16]
    if digest != rec.get("source_sha256_16") or rec.get("kernel") != kernel_tag:
        return None
    return rec


def run_mmod(args):
    import torch
    import torch.distributed as dist

    import paper_2007_06048_gb300 as M

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = make_workload(args.workload, args.nt)
    nz, ny, nx = p.vel.shape
    npts = p.npoints
    prop = M.Propagator.from_problem(p, device=local)
    if args.kernel != "auto":
        prop.set_kernel({"simple": M.KERNEL_SIMPLE, "tma": M.KERNEL_TMA}[args.kernel])
    if args.variant >= 0:
        prop.set_variant(args.variant)
    if args.pdl is not None:
        prop.set_option(M.OPT_PDL, args.pdl)
    if args.claim is not None:
        prop.set_option(M.OPT_CLAIM, args.claim)
    if args.persistent is not None:
        prop.set_option(M.OPT_PERSISTENT, args.persistent)
    if args.zlen is not None:
        prop.set_option(M.OPT_ZLEN, args.zlen)
    stream = torch.cuda.current_stream(dev)
    vel_d = torch.from_numpy(p.vel).to(dev)
    wav_d = torch.from_numpy(np.ascontiguousarray(p.wavelet)).to(dev)
    tr_d = torch.empty((p.nt, len(p.rec_ijk)), device=dev)
    prop.set_model(vel_d, stream)
    kernel_tag = "tma" if (args.kernel in ("auto", "tma") and prop_uses_tma(prop)) else "simple"
    plan = prop.plan() if kernel_tag == "tma" else None

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        prop.forward(wav_d, tr_d, None, stream)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    loop_ms = []
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            prop.forward(wav_d, tr_d, None, stream)
            loop_ms.append(prop.loop_ms())     # CUDA events around the step loop, same stream
        e1.record(stream)
        barrier()
    launches = prop.launches * args.steps
    ms = e0.elapsed_time(e1)
    ms_max = reduce_max(ms, dist, dev)
    value = weak_throughput(ws, npts, p.nt, args.steps, ms_max)

    # roofline of the dominant kernel: the step kernel, one launch per time step
    peak, peak_kind = load_peaks()
    step_ms = float(np.mean(loop_ms)) / p.nt
    achieved = BYTES_PER_POINT * npts / (step_ms * 1e-3) / 1e9
    tr_rec = traffic_from_profiles(kernel_tag)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "kernel": f"step_{kernel_tag}", "bytes_per_point": BYTES_PER_POINT,
                "launch_ms": step_ms,
                "traffic": None if tr_rec is None else tr_rec["dram_bytes_per_launch"] * npts / tr_rec["npoints"]}

    # end-to-end through the C ABI with host buffers (pinned), copies inside the timed region
    vel_h = torch.from_numpy(p.vel).pin_memory()
    wav_h = torch.from_numpy(np.ascontiguousarray(p.wavelet)).pin_memory()
    tr_h = torch.empty((p.nt, len(p.rec_ijk)), pin_memory=True)
    e2e_steps = max(1, min(args.steps, 5))
    prop.set_model(vel_h, stream)
    prop.forward(wav_h, tr_h, None, stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        prop.set_model(vel_h, stream)
        prop.forward(wav_h, tr_h, None, stream)
    barrier()
    e2e_s = reduce_max(time.perf_counter() - t0, dist, dev)
    e2e = {"value": weak_throughput(ws, npts, p.nt, e2e_steps, e2e_s * 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(vel_h.numel() * 4 + wav_h.numel() * 4),
           "d2h_bytes_per_step": int(tr_h.numel() * 4),
           "api": "mmod_set_model + mmod_forward with pinned host buffers, wall clock"}

    extra = {}
    fwd_gpts = value / ws
    measures = {"adjoint": lambda: measure_adjoint(M, prop, p, dev, stream, fwd_gpts),
                "gradient": lambda: measure_gradient(M, dev, stream, fwd_gpts, args.nt or 1000),
                "batched": lambda: measure_batched(M, dev, stream, fwd_gpts),
                "large": lambda: measure_large(M, dev, stream, peak),
                "free_surface": lambda: measure_free_surface(M, dev, stream, fwd_gpts),
                "cpml": lambda: measure_cpml(M, dev, stream, fwd_gpts, args.nt or 1000),
                "variable_density": lambda: measure_vd(M, dev, stream, fwd_gpts, peak, args.nt or 1000)}
    for name in extras_of(args):
        extra[name] = measures[name]()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, _, _ = oracle_sample(p, seconds_target=args.ref_seconds)
        one, _, _ = oracle_sample(p, seconds_target=min(args.ref_seconds, 8.0), nthreads=1)
        cpu["single_thread"] = {"value": one["value"], "sample": one["sample"]}
        cpu["paper_context"] = PAPER_CONTEXT
    clocks = clk.summary()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": describe(p),
                "launch": {"parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                           "kernel": kernel_tag, "plan": plan,
                           "variant": None if plan is None else M.mmod_tma_variant_name(plan["variant"])},
                "hbm_roofline_pct": 100.0 * BYTES_PER_POINT * value / ws / peak,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks, **extra}
        if extra:   # last, so that a reader of the line's tail sees every headline figure
            line["summary"] = summarize(value, roofline, extra)
        print(json.dumps(line), flush=True)
    prop.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def _r(x, nd=3):
    return None if x is None else round(float(x), nd)


def summarize(value, roofline, extra):
    """Headline figures of the main line and of every extra measurement."""
    out = {"forward_gpts": _r(value, 1), "forward_frac": _r(roofline["frac"])}
    if "adjoint" in extra:
        a = extra["adjoint"]
        out["adjoint"] = {"gpts": _r(a["value"], 1), "vs_fwd": _r(a["vs_forward"]), "frac": _r(a["roofline"]["frac"])}
    if "gradient" in extra:
        g = extra["gradient"]
        out["gradient"] = {k: {"ms": _r(g[k]["ms"], 1), "vs_fwd": _r(g[k]["vs_forward"]),
                               "frac": _r(g[k]["roofline"]["frac"])}
                           for k in ("fp32", "bf16", "bfp16", "fp32_every_state") if k in g}
    if "batched" in extra:
        b = extra["batched"]
        out["batched"] = {"gpts": _r(b["value"], 1), "vs_fwd": _r(b["vs_forward"]), "fused": _r(b["fused"], 1),
                          "persistent": _r(b["persistent"], 1), "one_by_one": _r(b["one_by_one"], 1)}
    if "large" in extra:
        lg = extra["large"]
        out["large"] = {"gpts": _r(lg["forward"]["value"], 1), "frac": _r(lg["forward"]["roofline"]["frac"]),
                        "grad_fp16_ms": _r(lg["gradient_fp16"]["ms"], 1),
                        "grad_gb": _r(lg["gradient_fp16"]["device_gb"], 1)}
    if "free_surface" in extra:
        out["free_surface"] = {"gpts": _r(extra["free_surface"]["value"], 1)}
    if "cpml" in extra:
        c = extra["cpml"]
        out["cpml"] = {"gpts": _r(c["value"], 1), "vs_fwd": _r(c["vs_forward"]), "frac": _r(c["roofline"]["frac"]),
                       "passes_frac": c["layer_passes"]["frac"]}
    if "variable_density" in extra:
        v = extra["variable_density"]
        out["variable_density"] = {"gpts": _r(v["value"], 1), "frac": _r(v["roofline"]["frac"]),
                                   "frac_512": _r(v["large"]["roofline"]["frac"])}
    return out


def roofline_of(bytes_per_call, ms, peak, what):
    achieved = bytes_per_call / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "bytes_per_call": bytes_per_call, "what": what}


def cpml_layer_bytes(nx, ny, nz, L, free_surface=False):
    """Algorithmic bytes of the CPML layer terms per step: a layer cell with k
    axes in their layers reads u^n and c and updates u^{n+1} once (16 B), and
    updates psi_a and zeta_a of each of its k axes (16k B)."""
    def inside(n, lo_layer=True):
        m = np.zeros(n, bool)
        if lo_layer:
            m[:L] = True
        m[n - L:] = True
        return m
    ax = inside(nx)
    ay = inside(ny)
    az = inside(nz, not free_surface)
    cells = int(np.logical_or.outer(np.logical_or.outer(az, ay), ax).sum())
    axes = int(ax.sum()) * ny * nz + int(ay.sum()) * nx * nz + int(az.sum()) * nx * ny
    return 16 * cells + 16 * axes, cells, axes


def time_calls(fn, reps, stream):
    """Median device time (ms) of fn() over reps calls, CUDA events on stream."""
    import torch
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return float(np.median(out))


def measure_adjoint(M, prop, p, dev, stream, fwd_gpts, reps=3):
    """mmod_adjoint on the bench workload: the residual has the traces' shape."""
    import torch
    rng = np.random.default_rng(7)
    r = torch.from_numpy(rng.standard_normal((p.nt, len(p.rec_ijk))).astype(np.float32)).to(dev)
    a = torch.empty((len(p.src_ijk), p.nt), device=dev)
    prop.adjoint(r, a, stream)
    ms = time_calls(lambda: prop.adjoint(r, a, stream), reps, stream)
    v = p.npoints * p.nt / (ms * 1e-3) / 1e9
    roof = roofline_of(BYTES_PER_POINT * p.npoints * p.nt, ms, load_peaks()[0],
                       "16 B per point and adjoint step (the forward step kernel on psi), whole call")
    return {"value": v, "unit": UNIT, "ms": ms, "vs_forward": v / fwd_gpts, "workload": p.name, "roofline": roof,
            "what": "mmod_adjoint: nt adjoint steps, receivers injected, sources gathered"}


def measure_gradient(M, dev, stream, fwd_gpts, nt=1000, reps=2):
    """mmod_gradient on the 200^3 smooth-gradient workload: 20 FP32 or BF16
    checkpoints, and FP32 with every state kept (no replay)."""
    import torch
    import workloads as W
    p = W.smooth_gradient_200(nt)
    prop = M.Propagator.from_problem(p, device=dev.index or 0)
    prop.set_model(torch.from_numpy(p.vel).to(dev), stream)
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet)).to(dev)
    rng = np.random.default_rng(8)
    r = torch.from_numpy(rng.standard_normal((p.nt, len(p.rec_ijk))).astype(np.float32)).to(dev)
    g = torch.empty(p.vel.shape, device=dev)
    out = {"workload": p.name, "unit": UNIT,
           "what": "mmod_gradient: forward sweep with checkpoints, segment replay, adjoint, imaging; "
                   "value counts nt forward-equivalent steps per call"}
    peak = load_peaks()[0]
    for name, dtype, ck in (("fp32", M.CKPT_FP32, 20), ("bf16", M.CKPT_BF16, 20), ("bfp16", M.CKPT_BFP16, 20),
                            ("fp32_every_state", M.CKPT_FP32, p.nt)):
        prop.gradient(wav, r, g, ck, dtype, stream)
        ms = time_calls(lambda: prop.gradient(wav, r, g, ck, dtype, stream), reps, stream)
        v = p.npoints * p.nt / (ms * 1e-3) / 1e9
        bpp, what = gradient_bytes_per_point_step(ck >= p.nt and dtype == M.CKPT_FP32,
                                                  ck if dtype == M.CKPT_FP32 else 0)
        out[name] = {"value": v, "ms": ms, "vs_forward": v / fwd_gpts, "checkpoints": ck,
                     "memory_gb": prop.gradient_memory(ck, dtype) / 1e9,
                     "roofline": roofline_of(bpp * p.npoints * p.nt, ms, peak, what)}
    prop.close()
    return out


def gradient_bytes_per_point_step(every_state, fp32_segments=0):
    """Algorithmic bytes per grid point and time step of mmod_gradient
    (checkpoint saves and restores, once per segment, left out).  With S FP32
    segments the first sweep writes g^n of the last segment (+4 B on 1/S of
    the steps) and that segment is not replayed (-20 B on 1/S of the steps)."""
    if every_state:
        return 48, ("forward sweep 20 B (u^{n-1}, u^n, c read, u^{n+1} and g^n = L u^n + s^n written), adjoint "
                    "step 16 B, paired imaging 12 B (psi^{n+1}, psi^n, g^n, g^{n-1} read, accumulator "
                    "read and written per two steps)")
    what = ("forward sweep 16 B, segment replay 20 B (g^n written as well), adjoint step 16 B, paired "
            "imaging 12 B per point and step")
    if fp32_segments > 0:
        return 64 - 16.0 / fp32_segments, what + (f"; the last of {fp32_segments} FP32 segments keeps g^n from the "
                                                 f"first sweep (+4 B) and is not replayed (-20 B)")
    return 64, what


def measure_batched(M, dev, stream, fwd_gpts, reps=3):
    """mmod_batch_forward on 32 uneven shots x 800 steps (one launch per step for
    all shots, variant chosen by mmod_batch_autotune), against the same shots
    run one after another through mmod_forward."""
    import torch
    import workloads as W
    shots = W.batched_shots()
    props = [M.Propagator.from_problem(p, device=dev.index or 0) for p in shots]
    for pr, p in zip(props, shots):
        pr.set_model(torch.from_numpy(p.vel).to(dev), stream)
    wav = [torch.from_numpy(np.ascontiguousarray(p.wavelet)).to(dev) for p in shots]
    trs = [torch.empty((p.nt, len(p.rec_ijk)), device=dev) for p in shots]
    work = sum(p.npoints * p.nt for p in shots)
    b = M.Batch(props)
    b.set_mode(M.BATCH_FUSED)                 # the fused launch, for the record
    fused_variant = b.autotune(10, stream)
    b.forward(wav, trs, stream)
    ms_fused = time_calls(lambda: b.forward(wav, trs, stream), reps, stream)
    b.set_mode(M.BATCH_PERSISTENT)            # one cooperative launch for every shot's loop
    b.set_variant(2)
    b.forward(wav, trs, stream)
    ms_persist = time_calls(lambda: b.forward(wav, trs, stream), reps, stream)
    b.set_mode(M.BATCH_STREAMS)               # the default mode
    variant = b.autotune(10, stream)
    b.forward(wav, trs, stream)
    ms = time_calls(lambda: b.forward(wav, trs, stream), reps, stream)
    loop_ms = b.loop_ms()

    def one_by_one():
        for pr, w, t in zip(props, wav, trs):
            pr.forward(w, t, None, stream)
    one_by_one()
    ms_single = time_calls(one_by_one, reps, stream)
    b.close()
    for pr in props:
        pr.close()
    v = work / (ms * 1e-3) / 1e9
    return {"value": v, "unit": UNIT, "ms": ms, "loop_ms": loop_ms, "vs_forward": v / fwd_gpts,
            "hbm_frac": BYTES_PER_POINT * v / load_peaks()[0],
            "one_by_one": work / (ms_single * 1e-3) / 1e9, "fused": work / (ms_fused * 1e-3) / 1e9,
            "persistent": work / (ms_persist * 1e-3) / 1e9,
            "fused_variant": M.mmod_tma_variant_name(fused_variant),
            "shots": len(shots), "nt": shots[0].nt,
            "points": int(sum(p.npoints for p in shots)), "variant": M.mmod_tma_variant_name(variant),
            "what": "mmod_batch_forward, streams mode: the shots' graphs overlap on four streams; "
                    "fused: one launch per step for all shots; persistent: one cooperative launch for every "
                    "shot's whole loop"}


def measure_free_surface(M, dev, stream, fwd_gpts, reps=3):
    """The bench workload with the free surface on (receivers one plane under
    it): the cost of the odd image and the surface projection."""
    import torch
    import workloads as W
    p = W.layered_240(1000)
    p.free_surface = True
    p.rec_ijk[:, 2] = 1
    prop = M.Propagator.from_problem(p, device=dev.index or 0)
    prop.set_model(torch.from_numpy(p.vel).to(dev), stream)
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet)).to(dev)
    tr = torch.empty((p.nt, len(p.rec_ijk)), device=dev)
    prop.forward(wav, tr, None, stream)
    ms = time_calls(lambda: prop.forward(wav, tr, None, stream), reps, stream)
    prop.close()
    v = p.npoints * p.nt / (ms * 1e-3) / 1e9
    return {"value": v, "unit": UNIT, "ms": ms, "vs_forward": v / fwd_gpts, "workload": p.name + " + free surface"}


def measure_cpml(M, dev, stream, fwd_gpts, nt=1000, reps=3):
    """The bench workload with CPML layers (20 cells, 10 Hz shift) instead of
    damping layers: the memory variables' cost."""
    import torch
    import workloads as W
    p = W.layered_240(nt)
    p.cpml, p.cpml_f0 = True, 10.0
    prop = M.Propagator.from_problem(p, device=dev.index or 0)
    prop.set_model(torch.from_numpy(p.vel).to(dev), stream)
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet)).to(dev)
    tr = torch.empty((p.nt, len(p.rec_ijk)), device=dev)
    prop.forward(wav, tr, None, stream)
    ms = time_calls(lambda: prop.forward(wav, tr, None, stream), reps, stream)
    prop.close()
    v = p.npoints * p.nt / (ms * 1e-3) / 1e9
    nz, ny, nx = p.vel.shape
    lb, cells, axes = cpml_layer_bytes(nx, ny, nz, p.nbl)
    roof = roofline_of((BYTES_PER_POINT * p.npoints + lb) * p.nt, ms, load_peaks()[0],
                       f"per step 16 B per point (step kernel) + 16 + 16k B per layer cell with k axes in their "
                       f"layers (u^n, c, u^{{n+1}} once; psi_a, zeta_a per axis): {cells} layer cells, {axes} cell-axes")
    # the layer passes alone: the step's time less the forward run's time per
    # step (the same step kernel), against their own algorithmic bytes
    step_us = 1e3 * ms / p.nt
    fwd_us = 1e6 * p.npoints / (fwd_gpts * 1e9)
    pass_us = step_us - fwd_us
    peak = load_peaks()[0]
    passes = {"bytes_per_step": lb, "us_per_step": _r(pass_us, 2),
              "gbs": _r(lb / (pass_us * 1e-6) / 1e9, 1) if pass_us > 0 else None,
              "frac": _r(lb / (pass_us * 1e-6) / 1e9 / peak) if pass_us > 0 and peak else None,
              "note": "us per step less the forward run's us per step"}
    return {"value": v, "unit": UNIT, "ms": ms, "vs_forward": v / fwd_gpts, "workload": p.name + " + CPML (L=20)",
            "roofline": roof, "layer_bytes_per_step": lb, "layer_passes": passes,
            "what": "per step: the undamped step kernel, then one tiled pass per axis (units of 64 lines of a "
                    "layer range loaded whole into shared memory by bulk-tensor copies, two stages per block; "
                    "psi_a^n, zeta_a^n and the u^{n+1} correction), the four kernels chained by programmatic "
                    "dependent launch"}


VD_BYTES_PER_POINT = 56   # velocity kernel 32 B + pressure kernel 24 B (FP32)


def measure_vd(M, dev, stream, fwd_gpts, peak, nt, reps=3):
    """The variable-density staggered system (velocity and pressure kernels
    per step) on the 240^3 layered model with Gardner densities."""
    import torch
    import workloads as W
    p = W.layered_240_vd(nt)
    prop = M.StaggeredPropagator.from_problem(p, device=dev.index or 0)
    prop.set_model(torch.from_numpy(p.vel).to(dev), torch.from_numpy(p.rho).to(dev), stream)
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet)).to(dev)
    tr = torch.empty((p.nt, len(p.rec_ijk)), device=dev)
    prop.forward(wav, tr, None, stream)
    loops = []

    def fwd():
        prop.forward(wav, tr, None, stream)
        loops.append(prop.loop_ms())
    ms = time_calls(fwd, reps, stream)
    step_ms = float(np.median(loops)) / p.nt
    plan = prop.plan()
    launches = prop.launches
    prop.close()
    v = p.npoints * p.nt / (ms * 1e-3) / 1e9
    achieved = VD_BYTES_PER_POINT * p.npoints / (step_ms * 1e-3) / 1e9
    large = measure_vd_large(M, dev, stream, peak)
    return {"value": v, "unit": UNIT, "ms": ms, "step_ms": step_ms, "vs_forward": v / fwd_gpts, "large": large,
            "workload": p.name, "plan": plan, "launches_per_run": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "bytes_per_point": VD_BYTES_PER_POINT,
                         "what": "per step: velocity kernel reads p, vx, vy, vz, dt/rho and writes vx, vy, vz "
                                 "(32 B); pressure kernel reads vx, vy, vz, p, dt K and writes p (24 B)"},
            "what": "mmod_vd_forward: TMA velocity + pressure kernels and the source add per step"}


def measure_vd_large(M, dev, stream, peak, n=512, nt=100, reps=2):
    """The staggered system on 512^3 (layers and Gardner densities without
    perturbation): the kernels' steady state, where per-launch ramp and tail
    weigh less than on 240^3."""
    import torch
    import workloads as W
    p = W.layered_vd_plain(nt, n)
    prop = M.StaggeredPropagator.from_problem(p, device=dev.index or 0)
    prop.set_model(torch.from_numpy(p.vel).to(dev), torch.from_numpy(p.rho).to(dev), stream)
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet)).to(dev)
    tr = torch.empty((p.nt, len(p.rec_ijk)), device=dev)
    prop.forward(wav, tr, None, stream)
    loops = []

    def fwd():
        prop.forward(wav, tr, None, stream)
        loops.append(prop.loop_ms())
    ms = time_calls(fwd, reps, stream)
    step_ms = float(np.median(loops)) / p.nt
    plan = prop.plan()
    prop.close()
    del tr
    torch.cuda.empty_cache()
    achieved = VD_BYTES_PER_POINT * p.npoints / (step_ms * 1e-3) / 1e9
    return {"workload": p.name, "nt": p.nt, "value": p.npoints * p.nt / (ms * 1e-3) / 1e9, "ms": ms,
            "step_ms": step_ms, "plan": plan,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "bytes_per_point": VD_BYTES_PER_POINT}}


def extras_of(args):
    names = ["adjoint", "gradient", "batched", "large", "free_surface", "cpml", "variable_density"]
    if args.no_extra or args.extra == "none":
        return []
    if args.extra == "all":
        return names
    want = [x.strip() for x in args.extra.split(",") if x.strip()]
    bad = [x for x in want if x not in names]
    if bad:
        raise SystemExit(f"unknown --extra {bad}; choose from {names}")
    return want


def measure_large(M, dev, stream, peak, reps=2):
    """The 1024 x 1024 x 512 shot (h = 12.5 m, L = 32, 500 steps, 1024^2
    receivers): forward throughput and the step kernel's roofline fraction,
    then the velocity gradient with 25 FP16 checkpoints (segments scheme) and
    the device memory the whole run holds."""
    import torch
    import workloads as W
    p = W.fractal_large(500)
    npts = p.npoints
    torch.cuda.synchronize(dev)
    free0 = torch.cuda.mem_get_info(dev)[0]
    prop = M.Propagator.from_problem(p, device=dev.index or 0)
    prop.set_model(torch.from_numpy(p.vel).to(dev), stream)
    wav = torch.from_numpy(np.ascontiguousarray(p.wavelet)).to(dev)
    tr = torch.empty((p.nt, len(p.rec_ijk)), device=dev)
    prop.forward(wav, tr, None, stream)
    loops = []

    def fwd():
        prop.forward(wav, tr, None, stream)
        loops.append(prop.loop_ms())
    fwd_ms = time_calls(fwd, reps, stream)
    fwd_v = npts * p.nt / (fwd_ms * 1e-3) / 1e9
    step_ms = float(np.median(loops)) / p.nt
    achieved = BYTES_PER_POINT * npts / (step_ms * 1e-3) / 1e9
    gen = torch.Generator(device=dev).manual_seed(11)
    r = torch.randn((p.nt, len(p.rec_ijk)), device=dev, generator=gen)
    g = torch.empty(p.vel.shape, device=dev)
    prop.gradient(wav, r, g, 25, M.CKPT_FP16, stream)
    torch.cuda.synchronize(dev)
    used = free0 - torch.cuda.mem_get_info(dev)[0]
    grad_ms = time_calls(lambda: prop.gradient(wav, r, g, 25, M.CKPT_FP16, stream), 1, stream)
    grad_v = npts * p.nt / (grad_ms * 1e-3) / 1e9
    plan = prop.plan()
    prop.close()
    del tr, r, g
    torch.cuda.empty_cache()
    return {"workload": p.name, "grid": [p.vel.shape[2], p.vel.shape[1], p.vel.shape[0]], "nt": p.nt,
            "nrec": int(len(p.rec_ijk)), "unit": UNIT,
            "forward": {"value": fwd_v, "ms": fwd_ms, "step_ms": step_ms,
                        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                     "frac": achieved / peak}, "variant": M.mmod_tma_variant_name(plan["variant"])},
            "gradient_fp16": {"value": grad_v, "ms": grad_ms, "checkpoints": 25, "scheme": "segments",
                              "device_gb": used / 1e9, "budget_gb": 180,
                              "what": "forward-equivalent Gpoint-updates/s (nt steps per call)"}}


def prop_uses_tma(prop) -> bool:
    """True when the handle's automatic kernel choice is the TMA kernel."""
    import paper_2007_06048_gb300 as M
    try:
        prop.set_kernel(M.KERNEL_TMA)
    except M.MmodError:
        return False
    prop.set_kernel(M.KERNEL_AUTO)
    return True


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mmod", "reference"], default="mmod")
    ap.add_argument("--workload", default="layered240")
    ap.add_argument("--nt", type=int, default=None, help="override the workload's step count")
    ap.add_argument("--kernel", choices=["auto", "simple", "tma"], default="auto")
    ap.add_argument("--variant", type=int, default=-1, help="TMA kernel variant (-1 = automatic)")
    ap.add_argument("--pdl", type=int, choices=[0, 1], default=None, help="override MMOD_OPT_PDL")
    ap.add_argument("--persistent", type=int, choices=[0, 1], default=None, help="override MMOD_OPT_PERSISTENT")
    ap.add_argument("--zlen", type=int, default=None, help="override MMOD_OPT_ZLEN (planes per z range)")
    ap.add_argument("--claim", type=int, default=None,
                    help="override MMOD_OPT_CLAIM (planes per claimed work unit; 0 = the static plan)")
    ap.add_argument("--ref-seconds", type=float, default=20.0,
                    help="CPU seconds per oracle sample (cpu_baseline / reference arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip every extra measurement (same as --extra none)")
    ap.add_argument("--extra", default="all",
                    help="extra measurements after the main line: all, none, or a comma list of adjoint, gradient, "
                         "batched, large, free_surface, cpml, variable_density")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "mmod":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_mmod(args)


if __name__ == "__main__":
    sys.exit(main())
