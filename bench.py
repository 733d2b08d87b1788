"""Benchmark of the per-iteration hot path: recovery iterations per second.

One step = one recovery iteration of the plain method with the pixel-grid SOS
on the 512x512 / 512-element / 144 patches of 80x80 / 32-channel / 128x128 SOS
workload: sos_to_delays -> fused mc_deconv_loss + adjoint -> sos_to_delays_adj
-> TV -> Adam (8 libpact kernel launches).  Inputs are resident in HBM; L2 is
flushed (256 MB write) before every timed step; every step is timed with CUDA
events on the launching stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

--impl reference times the FP64 CPU oracle (as it stands) on a bounded sample
of the same workload (a subset of the patches per step, scaled to the full
iteration).  Under torchrun with N > 1 every rank runs its own independent
recovery problem (weak scaling; no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import tempfile
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "recovery iters/s (fwd+adjoint+Adam), pixel-grid SOS"
WORKLOAD = "pg512_ring512_p80_m32: 512x512 @0.1mm, 512-el ring R=40mm, 144 patches 80x80, M=32, SOS 128x128"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


VARIANTS = ("neural_field", "siren_field", "das_stack", "channels", "tv_sweep", "channel_data")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true")
    ap.add_argument("--ws-samples", type=int, default=20000, help="training stacks for the warm-start CNN")
    ap.add_argument("--ws-epochs", type=int, default=8)
    ap.add_argument("--variants", default="all",
                    help="comma-separated subset of " + ",".join(VARIANTS) + " (default: all)")
    ap.add_argument("--ws-stages", default="all", choices=["all", "train"],
                    help="'train': the warm start stops after generating the stacks and training the CNN")
    args = ap.parse_args()
    args.variants = list(VARIANTS) if args.variants == "all" else args.variants.split(",")
    bad = [v for v in args.variants if v not in VARIANTS]
    if bad:
        ap.error(f"unknown variants {bad}")
    return args


def dist_env():
    from paper_2409_10876_gb300 import ranks
    return ranks.dist_env()


# ---------------------------------------------------------------- CPU oracle legs

def cpu_model() -> str:
    """The host CPU's model name (Linux), else the platform's processor string."""
    import platform
    part = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":", 1)[0].strip().lower()
            if key == "model name":
                return line.split(":", 1)[1].strip()
            if key == "cpu part" and part is None:
                part = line.split(":", 1)[1].strip()
    except OSError:
        pass
    return f"{platform.machine()} (CPU part {part})" if part else (platform.processor() or platform.machine())


class OracleIteration:
    """One FP64 oracle recovery iteration (Eq. 3-7 with the autograd adjoint,
    TV, Adam) on the patches `idx` of the workload, on the host cores; the
    measurement Y is the oracle's own (Eq. 5 + the seeded noise)."""

    def __init__(self, cfg, case, idx=None):
        from oracle import pact_oracle as O
        self.O, self.cfg, self.case = O, cfg, case
        self.g = O.geom(cfg)
        Y, _, _ = O.make_measurement(self.g, case)
        self.idx = np.arange(cfg.n_patches) if idx is None else np.asarray(idx)
        self.Y = Y[self.idx]
        self.cen = case["centres"][self.idx]
        self.sos = case["sos_init"].astype(np.float64)
        self.m = np.zeros_like(self.sos)
        self.v = np.zeros_like(self.sos)
        self.t = 0

    def step(self):
        O, cfg = self.O, self.cfg
        self.t += 1
        L, _, _, gs = O.objective(self.g, self.sos, self.Y, self.cen, self.case["d"], cfg.eps, cfg.tv_lambda)
        self.sos, self.m, self.v = (x.numpy() for x in O.adam_step(self.sos, gs, self.m, self.v, self.t, cfg.lr,
                                                                   mask=self.case["mask"]))
        return float(L)


def oracle_whole_iterations(cfg, case, iters: int):
    """Seconds per whole-workload FP64 oracle iteration (all patches, no
    sampling): the median of `iters` iterations after one untimed one."""
    it = OracleIteration(cfg, case)
    it.step()
    times = []
    for _ in range(iters):
        t0 = time.perf_counter()
        it.step()
        times.append(time.perf_counter() - t0)
    return statistics.median(times), times


def run_reference(args, cfg, case, rank, world):
    """Reference arm: the FP64 oracle on the host cores.  A step is one whole
    iteration of the workload (all patches) when the run fits the time budget;
    with many steps it becomes an evenly spaced sample of the patches, chosen
    after the first warm-up step (a whole iteration) so that the run stays
    within about two minutes, and the line says which."""
    if rank != 0:
        return
    import torch
    budget_s = 120.0
    full = OracleIteration(cfg, case)
    t0 = time.perf_counter()
    full.step()
    t_full = time.perf_counter() - t0
    n_patch = int(min(cfg.n_patches, max(1, cfg.n_patches * budget_s / max(args.steps + args.warmup, 1) / t_full)))
    if n_patch == cfg.n_patches:
        it = full
        warm_left = max(args.warmup - 1, 0)
    else:
        it = OracleIteration(cfg, case, np.linspace(0, cfg.n_patches - 1, n_patch).round().astype(int))
        warm_left = args.warmup
    for _ in range(warm_left):
        it.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        it.step()
    el = time.perf_counter() - t0
    per_full = el / args.steps * cfg.n_patches / n_patch
    val = 1.0 / per_full
    sample = ("whole iterations (all %d patches), no scaling" % cfg.n_patches if n_patch == cfg.n_patches else
              f"{n_patch} of {cfg.n_patches} patches per step (evenly spaced), time scaled by "
              f"{cfg.n_patches / n_patch:.2f}; a whole iteration took {t_full:.2f} s")
    cores = torch.get_num_threads()
    line = {"metric": METRIC, "value": val, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "oracle_sample": sample},
            "cpu_baseline": {"value": val, "unit": "iters/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu": cpu_model()},
            "e2e": {"value": val, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"pact_clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, fl in rows for k, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- GPU arm

class _GraphEvents:
    """CUDA events recorded inside a captured graph (external event-record nodes,
    cudaEventRecordWithFlags with cudaEventRecordExternal), through the CUDA
    runtime that the process already uses: the breakdown of one graph replay."""

    def __init__(self, n: int):
        import ctypes
        lib = None
        for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if lib is None:
            raise RuntimeError("libcudart not found")
        self.ct, self.lib = ctypes, lib
        self.ev = []
        for _ in range(n):
            e = ctypes.c_void_p()
            if lib.cudaEventCreate(ctypes.byref(e)) != 0:
                raise RuntimeError("cudaEventCreate failed")
            self.ev.append(e)

    def record(self, k: int, stream_handle: int):
        if self.lib.cudaEventRecordWithFlags(self.ev[k], self.ct.c_void_p(stream_handle), 1) != 0:
            raise RuntimeError("cudaEventRecordWithFlags failed")

    def elapsed_ms(self, a: int, b: int) -> float:
        ms = self.ct.c_float()
        if self.lib.cudaEventElapsedTime(self.ct.byref(ms), self.ev[a], self.ev[b]) != 0:
            raise RuntimeError("cudaEventElapsedTime failed")
        return float(ms.value)


def run_gpu(args, cfg, case, rank, world, local):
    import torch
    from paper_2409_10876_gb300 import pact, ranks
    from paper_2409_10876_gb300.recovery import PGRecovery, measurement_spectra, recover, synthesize_stack

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    pact.load()
    pb = pact.Problem(cfg, dev)
    Y = measurement_spectra(pb, case, dev)
    rec = PGRecovery(pb, Y, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, torch.as_tensor(case["sos_init"]),
                     torch.as_tensor(case["mask"]))
    # one graph per iteration (as recovery uses it), with event-record nodes between
    # its three parts: rays | fused deconvolution + adjoint | ray adjoint + TV + Adam
    st0 = rec.state()
    rec.step()
    torch.cuda.synchronize()
    rec.set_state(st0)
    try:
        gev = _GraphEvents(5)
    except Exception:
        gev = None
    def capture(events):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            mark = (lambda k: events.record(k, torch.cuda.current_stream().cuda_stream)) if events else None
            rec.step(mark)
        return g

    g_step = capture(None)                        # the timed iteration
    g_step_ev = capture(gev) if gev else None     # the same with event nodes, for the breakdown
    torch.cuda.synchronize()
    launches_per_step = 4                         # rays (+ TV terms), fused pass, ray adjoint, partial sums + Adam
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def one(ev=None, g=None):
        flush.zero_()
        if ev is not None:
            ev[0].record(stream)
        (g or g_step).replay()
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    loss_start = rec.loss()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    gpu_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if world > 1 else \
        os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clk = ClockSampler(gpu_id) if rank == 0 else None
    time.sleep(0.3 if clk else 0)
    ranks.barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        one(evs[k])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = clk.stop() if clk else None
    step_ms = [e[0].elapsed_time(e[1]) for e in evs]
    tot_ms = sum(step_ms)
    loss_end = rec.loss()
    # breakdown: the in-graph events of single replays (each read back before the next)
    rays_ms, mcd_ms, rest_ms, adj_ms = [], [], [], []
    if gev:
        for _ in range(min(200, args.steps)):
            one(g=g_step_ev)
            torch.cuda.synchronize()
            rays_ms.append(gev.elapsed_ms(0, 1))
            mcd_ms.append(gev.elapsed_ms(1, 2))
            rest_ms.append(gev.elapsed_ms(2, 3))
            adj_ms.append(gev.elapsed_ms(2, 4))
    else:
        rays_ms = mcd_ms = rest_ms = adj_ms = [float("nan")]
    tot_ms = ranks.job_time_ms(tot_ms, world, dev)
    value = ranks.job_value(world, args.steps, tot_ms)

    # roofline of the fused deconvolution + adjoint call (dominant kernel): its
    # launch duration as the difference of two graphs on the bench's stream,
    # K x (L2 flush, fused pass) and K x (L2 flush), so that neither event nodes
    # nor the graph launch are counted; the in-iteration event interval is kept
    # beside it
    N, M, F, n_t = pb.n, rec.m, pb.f, pb.n_t
    alg_bytes = 8 * N * M * F + 2 * 4 * N * n_t
    mcd_avg_s = kernel_duration_s(lambda: pact.mc_deconv_loss(pb, rec.w, rec.Y, rec.d, rec.eps, want_grad=True,
                                                              out=rec.out, ws=rec.ws_mcd, tables=rec.tables,
                                                              accumulate=True), flush, stream)
    peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else None
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = alg_bytes / mcd_avg_s / 1e9
    adj_call_s = kernel_duration_s(lambda: pact.sos_to_delays_adj(pb, rec.sos, rec.out["dL_dw"], rec.grad,
                                                                  accumulate=False, ws=rec.ws_adj), flush, stream)
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "mc_deconv_loss_traffic.json")
    if os.path.exists(tr_path):
        tr = json.load(open(tr_path))
        if tr.get("kernel_rev") == kernel_revision():
            traffic = tr.get("bytes_per_launch")

    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "flushed (256 MB write) before every timed step",
                       "seed": args.seed, "eps": cfg.eps, "tv_lambda": cfg.tv_lambda},
            "breakdown_ms": {"sos_to_delays": statistics.mean(rays_ms), "mc_deconv_loss": statistics.mean(mcd_ms),
                             "adj_tv_adam": statistics.mean(rest_ms)},
            "roofline": {"bound": "hbm", "kernel": "mc_deconv_loss (fused Eq. 4-7 + adjoint, one kernel)",
                         "timing": f"launch duration {mcd_avg_s * 1e3:.4f} ms = (graph of {KDUR} x (256 MB L2 flush, "
                                   f"fused pass) - graph of {KDUR} x (flush)) / {KDUR}, the kernel in the accumulating "
                                   f"form the iteration launches (dL/dw cleared by the ray kernel before it); "
                                   f"between event nodes inside the iteration graph the call spans "
                                   f"{statistics.mean(mcd_ms):.4f} ms",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": "measured" if peaks else "fallback",
                         "algorithmic_bytes_per_launch": alg_bytes, "traffic": traffic},
            "roofline_rays": rays_roofline(cfg, adj_call_s * 1e3, clocks,
                                           torch.cuda.get_device_properties(dev).multi_processor_count),
            "gpu_launches": launches_per_step * args.steps,
            "context": "paper: full NF recovery 40.3 s vs 23 min for APACT ('35x faster'), PG 113.3 s, SOS-oracle "
                       "deconvolution 2.6 s, on an RTX A6000 in PyTorch (Table 1); no per-iteration figures",
            "wall_s_timed_region": wall,
            "loss": {"start": loss_start, "end": loss_end}}
    if clocks:
        line["clocks"] = clocks

    if rank == 0 and not args.no_cpu_baseline:
        per, times = oracle_whole_iterations(cfg, case, 3)
        cores = torch.get_num_threads()
        torch.set_num_threads(1)
        try:
            per1, times1 = oracle_whole_iterations(cfg, case, 1)
        finally:
            torch.set_num_threads(cores)
        line["cpu_baseline"] = {"value": 1.0 / per, "unit": "iters/s", "cores": cores, "kind": "oracle",
                                "sample": f"median of {len(times)} whole FP64 oracle iterations (all "
                                          f"{cfg.n_patches} patches, no scaling) after one untimed",
                                "one_thread": {"value": 1.0 / per1, "unit": "iters/s", "cores": 1,
                                               "sample": "one whole iteration after one untimed"},
                                "nproc": os.cpu_count(), "cpu": cpu_model()}
    if rank == 0 and not args.no_cpu_baseline:
        line["error_vs_fp64_oracle"] = oracle_errors(cfg, case, pb, dev)
    if not args.no_e2e:
        stack = synthesize_stack(pb, case, dev).cpu().pin_memory()
        iters = cfg.steps                                # one whole recovery of the configuration
        recover(pb, stack, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, torch.as_tensor(case["sos_init"]),
                torch.as_tensor(case["mask"]), 5)               # warm-up (graph capture paths, allocator)
        torch.cuda.synchronize()
        ranks.barrier(world)
        t0 = time.perf_counter()
        r = recover(pb, stack, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, torch.as_tensor(case["sos_init"]),
                    torch.as_tensor(case["mask"]), iters)
        torch.cuda.synchronize()
        el_ms = ranks.job_time_ms((time.perf_counter() - t0) * 1e3, world, dev)
        e2e = ranks.job_value(world, iters, el_ms)
        d2h = 4 * iters + r.sos.numel() * 4 + r.image.numel() * 4
        line["e2e"] = {"value": e2e, "unit": "iters/s", "h2d_bytes_per_step": stack.numel() * 4 / iters,
                       "d2h_bytes_per_step": d2h / iters,
                       "what": f"recover(): pinned host stack upload, patch spectra, graph capture, {iters} "
                               f"iterations with every loss read back and checked, then the recovered SOS and "
                               f"the stitched image copied to pinned host memory",
                       "restarts": len(r.restarts)}
    if not args.no_variants:
        run = {"neural_field": lambda: nf_variant(args, cfg, case, pb, Y, flush, stream),
               "siren_field": lambda: siren_variant(args, cfg, case, pb, Y, flush, stream),
               "das_stack": lambda: das_variant(dev, flush, stream),
               "channels": lambda: channels_variant(args, cfg, dev, flush, stream),
               "tv_sweep": lambda: tv_sweep_variant(args, cfg, case, pb, Y),
               "channel_data": lambda: channel_data_variant(args, dev, flush, stream)}
        line["variants"] = {name: run[name]() for name in VARIANTS if name in args.variants}
    if "channel_data" in line.get("variants", {}):
        cd = line["variants"]["channel_data"]["mc_deconv_loss"]
        line["roofline_channel_data"] = {
            "bound": "hbm", "kernel": "mc_deconv_loss on 3721 patches x 32 channels x 64x64 (2.0 GB of spectra, 16x L2)",
            "achieved": cd["achieved_gbs"], "peak": cd["peak_gbs"], "unit": "GB/s", "frac": cd["frac"],
            "peak_source": cd["peak_source"], "algorithmic_bytes_per_launch": cd["algorithmic_bytes"], "traffic": None}
    if rank == 0 and not args.no_warm_start:
        line["warm_start"] = warm_start_run(args, cfg, pb, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)


def oracle_errors(cfg, case, pb, dev):
    """Relative L2 errors of the GPU forward model and adjoint against the FP64
    oracle on the benchmark workload (all 144 patches, the oracle's own
    measurement spectra), at the uniform start and at the true SOS: w (Eq. 3),
    the data loss (Eq. 7), dL/dw (fused adjoint) and dL/dv (ray adjoint)."""
    import torch
    from oracle import pact_oracle as O
    from paper_2409_10876_gb300 import pact
    g = O.geom(cfg)
    Y64, _, _ = O.make_measurement(g, case)
    Y = torch.as_tensor(Y64.numpy().astype(np.complex64), device=dev)
    rel = lambda a, b: float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) /
                             max(np.linalg.norm(np.asarray(b, np.float64)), 1e-300))
    out = {"tolerances": {"w_loss": 1e-4, "gradients": 2e-3}}
    for name in ("sos_init", "sos_true"):
        sos = torch.as_tensor(case[name], device=dev)
        w = pact.sos_to_delays(pb, sos)
        r = pact.mc_deconv_loss(pb, w, Y, case["d"], cfg.eps, want_grad=True)
        gs = pact.sos_to_delays_adj(pb, sos, r["dL_dw"])
        torch.cuda.synchronize()
        L64, _, w64, gs64 = O.objective(g, case[name].astype(np.float64), Y64, case["centres"], case["d"], cfg.eps, 0.0)
        _, _, _, gw64 = O.mc_deconv_loss(g, w64, Y64, case["centres"], case["d"], cfg.eps)
        out["at_" + name.split("_")[1]] = {"w": rel(w.cpu().numpy(), w64.numpy()),
                                          "loss": abs(float(r["loss"].item()) - float(L64)) / abs(float(L64)),
                                          "dL_dw": rel(r["dL_dw"].cpu().numpy(), gw64.numpy()),
                                          "dL_dsos": rel(gs.cpu().numpy(), gs64.numpy())}
    return out


RAY_ADJ_OPS = 24   # FP32 lane operations of one adjoint sample (see the design notes)


def ray_samples(cfg) -> int:
    """Midpoint samples of all rays r'_i -> r_n inside the mask disk (from the
    geometry: ceil(chord / h) per ray)."""
    import numpy as np
    c = cfg.centres()
    x = (c[:, 1] - (cfg.img_w - 1) / 2) * cfg.dx
    y = (c[:, 0] - (cfg.img_h - 1) / 2) * cfg.dx
    th = 2 * np.pi * np.arange(cfg.n_t) / cfg.n_t + cfg.ring_phase
    dx = cfg.ring_radius * np.cos(th)[None] - x[:, None]
    dy = cfg.ring_radius * np.sin(th)[None] - y[:, None]
    L = np.hypot(dx, dy)
    ce = (x[:, None] * dx + y[:, None] * dy) / L
    disc = ce ** 2 - (x[:, None] ** 2 + y[:, None] ** 2 - cfg.mask_radius ** 2)
    sq = np.sqrt(np.maximum(disc, 0.0))
    s0, s1 = np.clip(-ce - sq, 0, L), np.clip(-ce + sq, 0, L)
    chord = np.where(disc > 0, np.maximum(s1 - s0, 0.0), 0.0)
    return int(np.ceil(chord / cfg.ray_step).sum())


def rays_roofline(cfg, adj_ms: float, clocks, sms: int):
    """The ray adjoint (the longest kernel of the iteration) against the FP32
    issue rate: RAY_ADJ_OPS algorithmic lane operations per sample over the
    duration of the call (kernel + partial-grid sum, timed as the fused pass
    is), peak = the device's SMs x 128 FP32 lanes x the SM clock sampled
    during the run."""
    samples = ray_samples(cfg)
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = sms * 128 * mhz * 1e6 / 1e12
    ach = samples * RAY_ADJ_OPS / (adj_ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "rays_adj_kernel + reduce_parts_kernel (Eq. 3 adjoint)",
            "achieved": ach, "peak": peak, "unit": "T lane-ops/s (FP32)", "frac": ach / peak,
            "samples_per_launch": samples, "ops_per_sample": RAY_ADJ_OPS, "ms": adj_ms,
            "peak_source": f"{sms} SMs x 128 FP32 lanes x sampled SM clock"}


KDUR = 20


def kernel_duration_s(call, flush, stream, reps: int = 9) -> float:
    """Duration of `call` (its kernels) after an L2 flush: the median
    over `reps` replays of (graph of KDUR x (flush, call) - graph of KDUR x
    (flush)) / KDUR, timed with events on `stream`."""
    import torch

    def graph(with_call):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(KDUR):
                flush.zero_()
                if with_call:
                    call()
        return g

    ga, gb = graph(True), graph(False)
    diffs = []
    for _ in range(reps):
        t = []
        for g in (ga, gb):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        diffs.append((t[0] - t[1]) / KDUR)
    del ga, gb
    return statistics.median(diffs) / 1e3


def _time_graph(g, flush, stream, steps: int):
    import torch
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
    for e in evs:
        flush.zero_()
        e[0].record(stream)
        g.replay()
        e[1].record(stream)
    torch.cuda.synchronize()
    return [e[0].elapsed_time(e[1]) for e in evs]


def nf_variant(args, cfg, case, pb, Y, flush, stream):
    """Neural-field SOS (BF16 tensor cores) on the same problem: one iteration =
    nf_forward + rays + fused pass + ray adjoint + nf_backward + Adam."""
    import torch
    from paper_2409_10876_gb300 import inputs
    from paper_2409_10876_gb300.recovery import NFRecovery
    rec = NFRecovery(pb, Y, case["d"], cfg.eps, inputs.NF_LR, inputs.nf_init(args.seed), case["mask"])
    g = rec.capture()
    for _ in range(3):
        g.replay()
    steps = max(20, min(args.steps, 500))
    ms = _time_graph(g, flush, stream, steps)
    out = {"iters_per_s": 1e3 / statistics.mean(ms), "ms_per_step": statistics.mean(ms), "steps": steps,
           "dtype": "bf16 (field) + f32 (forward model)", "params": int(rec.params.numel()),
           "gpu_launches_per_step": 9, "lr": inputs.NF_LR}
    del rec, g
    # what the field recovers: a fresh run of the configuration's iterations
    rec = NFRecovery(pb, Y, case["d"], cfg.eps, inputs.NF_LR, inputs.nf_init(args.seed), case["mask"])
    rec.capture()
    hist = rec.run(cfg.steps, record_every=cfg.steps // 4)
    m = case["mask"].astype(bool)
    sos = rec.sos.cpu().numpy().astype(np.float64)
    t = (sos[m] - 1525.0) / 125.0
    out["recovery"] = {"iters": cfg.steps, "loss": hist,
                       "sos_rms_mps": float(np.sqrt(np.mean((sos[m] - case["sos_true"][m]) ** 2))),
                       "saturated_nodes": int((np.abs(t) > 0.99).sum())}
    return out


def channels_variant(args, cfg, dev, flush, stream):
    """Iterations/s against the number of delay channels M at the same delay
    range, and the SOS error after the configuration's iterations (the
    trade-off behind the paper's channel-count ablation, Sec. S3.1)."""
    import torch
    from paper_2409_10876_gb300 import inputs, pact
    from paper_2409_10876_gb300.recovery import PGRecovery, measurement_spectra
    out = {}
    for m in (4, 8, 16, 32):
        c = cfg.replace(m=m)
        case = inputs.make_case(c, args.seed)
        pb = pact.Problem(c, dev)
        Y = measurement_spectra(pb, case, dev)
        rec = PGRecovery(pb, Y, case["d"], c.eps, c.tv_lambda, c.lr, torch.as_tensor(case["sos_init"]),
                         torch.as_tensor(case["mask"]))
        g = rec.capture()
        for _ in range(3):
            g.replay()
        ms = _time_graph(g, flush, stream, 200)
        out[str(m)] = {"iters_per_s": 1e3 / statistics.mean(ms), "ms_per_iter": statistics.mean(ms)}
        del rec, g
        # what M channels recover: the configuration's iterations from uniform
        rec = PGRecovery(pb, Y, case["d"], c.eps, c.tv_lambda, c.lr, torch.as_tensor(case["sos_init"]),
                         torch.as_tensor(case["mask"]))
        rec.capture()
        rec.run(c.steps)
        mk = case["mask"].astype(bool)
        sos = rec.sos.cpu().numpy().astype(np.float64)
        out[str(m)]["sos_rms_mps_after"] = float(np.sqrt(np.mean((sos[mk] - case["sos_true"][mk]) ** 2)))
        out[str(m)]["iters"] = c.steps
        del rec
    return out


def tv_sweep_variant(args, cfg, case, pb, Y, iters: int = 1000):
    """TV weight sweep (the paper's regulariser ablation) on the benchmark
    problem: `iters` pixel-grid iterations from uniform 1500 m/s for each
    lambda, with the final loss and the SOS error against the ground truth
    (RMS over the mask), and the loss at the ground truth for reference."""
    import numpy as np
    import torch
    from paper_2409_10876_gb300.recovery import PGRecovery
    mask = case["mask"].astype(bool)
    truth = case["sos_true"].astype(np.float64)
    rms = lambda s: float(np.sqrt(np.mean((s.astype(np.float64)[mask] - truth[mask]) ** 2)))
    out = {"iters": iters, "uniform_rms_mps": rms(case["sos_init"])}
    r = PGRecovery(pb, Y, case["d"], cfg.eps, 0.0, 0.0, torch.as_tensor(case["sos_true"]), torch.as_tensor(case["mask"]))
    r.step()
    out["data_loss_at_truth"] = r.loss()
    for lam in (1e-4, 1e-2, 1e-1, 1.0, 10.0):
        rec = PGRecovery(pb, Y, case["d"], cfg.eps, lam, cfg.lr, torch.as_tensor(case["sos_init"]),
                         torch.as_tensor(case["mask"]))
        g = rec.capture()
        for _ in range(iters):
            g.replay()
        out[f"lambda_{lam:g}"] = {"loss": rec.loss(), "rms_mps": rms(rec.sos.cpu().numpy())}
        del rec, g
    return out


def siren_variant(args, cfg, case, pb, Y, flush, stream):
    """The paper's neural field (SIREN, 1027 parameters, FP32) on the same
    problem: siren_forward + rays + fused pass + ray adjoint + siren_backward + Adam."""
    from paper_2409_10876_gb300 import inputs
    from paper_2409_10876_gb300.recovery import SirenRecovery
    rec = SirenRecovery(pb, Y, case["d"], cfg.eps, inputs.SIREN_LR, inputs.siren_init(args.seed), case["mask"])
    g = rec.capture()
    for _ in range(3):
        g.replay()
    steps = max(20, min(args.steps, 500))
    ms = _time_graph(g, flush, stream, steps)
    return {"iters_per_s": 1e3 / statistics.mean(ms), "ms_per_step": statistics.mean(ms), "steps": steps,
            "dtype": "f32", "params": int(rec.params.numel()), "gpu_launches_per_step": 8}


def channel_data_variant(args, dev, flush, stream):
    """End to end from channel data on the 1024 x 1024 / 1024-element workload:
    synthetic ring RF (4096 samples at 40 MHz, straight-ray times of flight
    through a 256 x 256 SOS map, vessel-tree sources) -> DAS stack (32 x
    1024 x 1024) -> patch spectra (3721 patches of 64 x 64: 2.0 GB) ->
    recovery iterations with the pixel-grid and the neural-field SOS.  The
    fused pass is also timed alone: its spectra are 16x the L2, so it is the
    HBM-bound figure."""
    import torch
    from paper_2409_10876_gb300 import inputs, pact
    from paper_2409_10876_gb300.recovery import NFRecovery, PGRecovery
    cfg = inputs.config_rf()
    case = inputs.make_case(cfg, args.seed)
    pb = pact.Problem(cfg, dev)
    ip = torch.as_tensor(case["ip"], device=dev)
    sos_t = torch.as_tensor(case["sos_true"], device=dev)
    rf = torch.empty((cfg.n_t, cfg.rf_ns), dtype=torch.float32, device=dev)
    ws = pact._ws(pact.rf_synth_workspace_size(pb, 65536), dev)
    stack = torch.empty((cfg.m, cfg.img_h, cfg.img_w), dtype=torch.float32, device=dev)
    Y = torch.empty(pb.spectra_shape(cfg.m), dtype=torch.complex64, device=dev)

    def timed(fn, reps):
        ms = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    def synth():
        pact.rf_synth(pb, ip, sos_t, cfg.rf_fs, cfg.rf_t0, cfg.rf_ns, cfg.rf_sigma, rf=rf, ws=ws)

    synth()
    t_rf = timed(synth, 2)
    t_das = timed(lambda: pact.das_stack(pb, rf, cfg.rf_fs, cfg.rf_t0, case["d"], stack), 2)
    t_fft = timed(lambda: pact.patch_fft(pb, stack, Y), 3)
    emitting = int((ip != 0).sum().item())
    out = {"workload": "rf1024_ring1024_p64_m32: 1024x1024 @0.05mm, 1024-el ring R=40mm, 4096 samples @40 MHz, "
                       "3721 patches 64x64, M=32, SOS 256x256",
           "rf_synth_ms": t_rf, "emitting_pixels": emitting,
           "das_stack_ms": t_das, "patch_fft_ms": t_fft}
    rec = PGRecovery(pb, Y, case["d"], cfg.eps, 1e-4, cfg.lr, torch.as_tensor(case["sos_init"]),
                     torch.as_tensor(case["mask"]))
    g = rec.capture()
    for _ in range(3):
        g.replay()
    ms = _time_graph(g, flush, stream, 20)
    out["pixel_grid"] = {"iters_per_s": 1e3 / statistics.mean(ms), "ms_per_iter": statistics.mean(ms),
                         "loss_after_23": rec.loss()}
    gm = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gm):
        pact.mc_deconv_loss(pb, rec.w, rec.Y, rec.d, rec.eps, want_grad=True, out=rec.out, ws=rec.ws_mcd,
                            tables=rec.tables, accumulate=True)
    for _ in range(3):
        gm.replay()
    ms = _time_graph(gm, flush, stream, 20)
    alg = 8 * pb.n * cfg.m * pb.f + 8 * pb.n * pb.n_t
    peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else None
    peak, src = (peaks["hbm_gbs"], "measured") if peaks else (6800.0, "fallback")
    ach = alg / (statistics.mean(ms) * 1e-3) / 1e9
    out["mc_deconv_loss"] = {"ms": statistics.mean(ms), "algorithmic_bytes": alg, "achieved_gbs": ach,
                             "peak_gbs": peak, "peak_source": src, "frac": ach / peak}
    del rec, g, gm
    nf = NFRecovery(pb, Y, case["d"], cfg.eps, inputs.NF_LR, inputs.nf_init(args.seed), case["mask"])
    g = nf.capture()
    for _ in range(3):
        g.replay()
    ms = _time_graph(g, flush, stream, 20)
    out["neural_field"] = {"iters_per_s": 1e3 / statistics.mean(ms), "ms_per_iter": statistics.mean(ms)}
    del nf, g
    out["mismatch"] = mismatch_study(pb, cfg, case, dev)
    return out


def mismatch_study(pb, cfg, case, dev, iters: int = 200):
    """Model mismatch in the channel data (geometric spreading, a ring-radius
    offset, a transducer band-limit): channel data -> DAS -> patch spectra, then the data loss at the
    true SOS against uniform 1500 m/s, and how far the pixel-grid recovery
    started at the true SOS drifts from it in `iters` iterations (RMS over
    the mask; lambda = 0)."""
    import numpy as np
    import torch
    from paper_2409_10876_gb300 import pact
    from paper_2409_10876_gb300.recovery import PGRecovery, channel_data_stack
    mask = case["mask"].astype(bool)
    truth = case["sos_true"].astype(np.float64)
    rms = lambda s: float(np.sqrt(np.mean((s.astype(np.float64)[mask] - truth[mask]) ** 2)))
    res = {}
    for name, spread, dr, bp in (("model", 0.0, 0.0, None), ("spreading_r^-1/2", 0.5, 0.0, None),
                                 ("ring_+0.1mm", 0.0, 0.1e-3, None), ("ring_+0.3mm", 0.0, 0.3e-3, None),
                                 ("bandlimit_5MHz_60%", 0.0, 0.0, (5e6, 0.6))):
        Y = pact.patch_fft(pb, channel_data_stack(pb, case, dev, spread, dr, bandpass=bp))
        losses = {}
        for start in ("sos_init", "sos_true"):
            r = PGRecovery(pb, Y, case["d"], cfg.eps, 0.0, 0.0, torch.as_tensor(case[start]),
                           torch.as_tensor(case["mask"]))
            r.step()
            losses[start] = r.loss()
        rec = PGRecovery(pb, Y, case["d"], cfg.eps, 0.0, 0.3, torch.as_tensor(case["sos_true"]),
                         torch.as_tensor(case["mask"]))
        g = rec.capture()
        for _ in range(iters):
            g.replay()
        res[name] = {"loss_true_over_uniform": losses["sos_true"] / losses["sos_init"],
                     "drift_rms_mps": rms(rec.sos.cpu().numpy()), "iters": iters,
                     "uniform_rms_mps": rms(case["sos_init"])}
        del rec, g, Y
    return res


def das_variant(dev, flush, stream):
    """Eq. 1 DAS stack at the channel-data scale (once per recovery): 1024-element
    ring, 4096 samples at 40 MHz -> 32 delay channels x 1024 x 1024 pixels."""
    import torch
    from paper_2409_10876_gb300 import inputs, pact
    cfg = inputs.config_rf()
    pb = pact.Problem(cfg, dev)
    rng = np.random.default_rng(7)
    rf = torch.as_tensor(rng.standard_normal((cfg.n_t, 4096)).astype(np.float32), device=dev)
    d = cfg.delays()
    stack = torch.empty((cfg.m, cfg.img_h, cfg.img_w), dtype=torch.float32, device=dev)
    pact.das_stack(pb, rf, 40e6, 0.0, d, stack)
    torch.cuda.synchronize()
    ms = []
    for _ in range(3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pact.das_stack(pb, rf, 40e6, 0.0, d, stack)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    taps = cfg.img_h * cfg.img_w * cfg.n_t * cfg.m
    t = statistics.median(ms) / 1e3
    return {"ms": statistics.median(ms), "taps": taps, "gtaps_per_s": taps / t / 1e9,
            "workload": "1024 el x 4096 samples -> 32 x 1024 x 1024"}


def cold_optimum_golden(cfg, seed: int, steps: int):
    """The FP64 oracle's cold optimum L*_cold of this problem
    (tests/golden/make_cold_optimum.py), if one was computed for exactly this
    configuration, seed and iteration count; else None."""
    import hashlib
    path = os.path.join(ROOT, "tests", "golden", f"cold_optimum_{cfg.name}_seed{seed}.json")
    if not os.path.exists(path):
        return None
    g = json.load(open(path))
    want = hashlib.sha1(repr((cfg, int(seed), int(steps))).encode()).hexdigest()[:16]
    return g if g.get("config_hash") == want else None


def warm_start_run(args, cfg, pb, dev):
    """Learned warm start on the full-size problem: the CNN is trained on the GPU
    (library kernels) on stacks the forward model generates from random SOS
    fields.  On a held-out problem the time to a loss within 1 % of L*_cold --
    the FP64 oracle's best loss over a 1000-iteration cold recovery (stored
    by tests/golden/make_cold_optimum.py), else the GPU cold run's -- is
    measured for the cold recovery and for the warm-started one
    (warmstart.recover_warm: warm branch with the cold branch as judge and
    fallback), including the network's inference.  The FP64 oracle
    re-evaluates the data loss at both end points."""
    import torch
    from paper_2409_10876_gb300 import inputs, pact, quality, warmstart
    from paper_2409_10876_gb300.recovery import measurement_spectra, synthesize_stack
    mask = inputs.sos_mask(cfg)
    t0 = time.perf_counter()
    gen = warmstart.StackGenerator(pb, cfg, n_ip=16, n_noise=8, seed=args.seed + 7)
    S = args.ws_samples
    X = torch.empty((S, cfg.sos_g, cfg.sos_g, pact.cnn_input_channels(cfg.m)), dtype=torch.bfloat16, device=dev)
    V = torch.empty((S, cfg.sos_g, cfg.sos_g), dtype=torch.float32, device=dev)
    gen.fill(X, V)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    B = 32
    net = pact.WarmStartCNN(pb, cfg.m, B, inputs.cnn_init(args.seed, cfg.m), mask)
    t0 = time.perf_counter()
    hist = warmstart.train(net, X, V, args.ws_epochs, lr=1e-3, seed=args.seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    steps = args.ws_epochs * (S // B)
    # algorithmic FLOPs of one training sample: forward of every conv, dgrad of layers 2-5, wgrad of all
    fl, res = 0.0, cfg.sos_g
    cin = pact.cnn_input_channels(cfg.m)
    for l, (_, cout, pool) in enumerate(inputs.CNN_CONVS):
        f = 2.0 * res * res * cin * cout * 9
        fl += f * (3 if l > 0 else 2)
        cin = cout
        res = res // 2 if pool else res
    train_tflops = fl * B * steps / t_train / 1e12
    del X, V
    train = {"train_samples": S, "epochs": args.ws_epochs, "batch": B, "generate_s": t_gen, "train_s": t_train,
             "train_step_ms": 1e3 * t_train / steps, "train_tflops_bf16": train_tflops,
             "train_loss": {"first_epoch": hist[0], "last_epoch": hist[-1]}}
    if args.ws_stages == "train":
        return train
    net1 = pact.WarmStartCNN(pb, cfg.m, 1, net.params.cpu().numpy(), mask)
    mask_d = torch.as_tensor(mask.astype(np.uint8), device=dev)
    held = inputs.config_held_out()
    seed = args.seed + 1000
    case = inputs.make_case(held, seed)
    Y = measurement_spectra(pb, case, dev)
    stack = synthesize_stack(pb, case, dev)
    v_true = torch.as_tensor(case["sos_true"], device=dev)
    v_cold = torch.full_like(v_true, cfg.v_bg)
    _, s_cold_all, h_cold, rec_cold = warmstart.time_to_target(pb, Y, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr,
                                                               v_cold, mask_d, -1.0, held.steps)
    gold = cold_optimum_golden(held, seed, held.steps)
    L_gpu = min(h_cold)
    L_star, src = (gold["L_star_cold"], "oracle_fp64") if gold else (L_gpu, "gpu_cold_run")
    target = 1.01 * L_star
    it_c, s_c, _, _ = warmstart.time_to_target(pb, Y, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, v_cold, mask_d,
                                               target, held.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    warmstart.predict(net1, pb, stack)
    torch.cuda.synchronize()
    e0.record()
    v_warm = warmstart.predict(net1, pb, stack)
    e1.record()
    torch.cuda.synchronize()
    s_pred = e0.elapsed_time(e1) * 1e-3
    r = warmstart.recover_warm(pb, Y, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, v_warm.clone(), mask_d,
                               2 * held.steps, target=target)
    it_w, s_w, h_w, rec_w = warmstart.time_to_target(pb, Y, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr,
                                                     v_warm.clone(), mask_d, target, held.steps)
    m = mask_d > 0
    truth = case["sos_true"].astype(np.float64)
    rms = lambda v: float(np.sqrt(np.mean((v.cpu().numpy().astype(np.float64)[mask] - truth[mask]) ** 2)))
    ip = case["ip"]
    pm = quality.image_mask(cfg)
    iq = {}
    for name, v in (("uniform_1500", v_cold), ("cold_end", rec_cold.sos), ("warm_end", rec_w.sos),
                    ("true_sos", v_true)):
        img = quality.recovered_image(pb, Y, case["d"], cfg.eps, v)
        iq[name] = {"psnr_db": quality.psnr(img, ip, 1.0, pm), "ssim": quality.ssim(img, ip, 1.0, pm),
                    "sos_rms_mps": rms(v)}
    warm_s = (r["reached_s"] + s_pred) if r["reached_s"] is not None else None
    cold_s = s_c if it_c else None
    out = {"image_quality": iq, **train,
           "sos_mae_mps": {"cnn": float((v_warm - v_true)[m].abs().mean()),
                           "uniform_1500": float((v_cold - v_true)[m].abs().mean())},
           "held_out": {"workload": held.name, "seed": seed},
           "L_star_cold": L_star, "L_star_source": src, "target": target, "L_gpu_cold_1000": L_gpu,
           "gpu_cold_over_oracle": (L_gpu / gold["L_star_cold"]) if gold else None,
           "cold": {"iters": it_c, "s": cold_s, "s_1000_iters": s_cold_all},
           "warm": {"what": "recover_warm (warm branch judged by the cold one, fallback to it) + CNN inference",
                    "reached": r["reached_s"] is not None, "s": warm_s, "cnn_s": s_pred, "iters": r["iters"],
                    "branch": r["branch"], "fallback": r["fallback"]},
           "warm_only": {"iters": it_w, "s": (s_w + s_pred) if it_w else None},
           "speedup": (cold_s / warm_s) if (cold_s and warm_s) else None}
    if gold:
        out["oracle_cold_run"] = {k: gold[k] for k in ("L_star_cold", "iteration_of_L_star", "loss_last",
                                                        "sos_rms_mps", "host")}
    if not args.no_cpu_baseline:
        from oracle import pact_oracle as O
        g = O.geom(held)
        Y64, _, _ = O.make_measurement(g, case)           # the oracle's own measurement of the seeded case
        for name, rec in (("cold_end", rec_cold), ("warm_end", rec_w)):
            w64 = O.wavefront_errors(g, rec.sos.cpu().numpy().astype(np.float64), case["centres"])
            L64 = O.mc_deconv_loss(g, w64, Y64, case["centres"], case["d"], cfg.eps, want_grad=False)[0]
            out[f"oracle_data_loss_{name}"] = float(L64)
            out[f"gpu_data_loss_{name}"] = float(pact.mc_deconv_loss(pb, pact.sos_to_delays(pb, rec.sos), Y,
                                                                     case["d"], cfg.eps, want_grad=False)["loss"])
    out["table1"] = table1_run(args, cfg, pb, dev, net1)
    return out


def table1_run(args, cfg, pb, dev, net1, seeds=(0, 1, 2, 3, 4)):
    """A synthetic counterpart of the paper's Table 1 (Sec. 4.1: averages over
    five phantoms): on seeds 0-4 of the benchmark workload, the stitched IP
    image (PSNR / SSIM inside the mask, range 1) and the SOS (PSNR / SSIM over
    the mask nodes, range sos_hi - sos_lo; RMS error) for deconvolution at the
    uniform SOS, the pixel-grid recovery from uniform (1000 iterations), the
    warm-started one (recover_warm, run until it settles), the paper's SIREN
    field and the Fourier-feature MLP field (1000 iterations each) and the true
    SOS ("SOS oracle"), with GPU wall times (synchronised host clock)."""
    import torch
    from paper_2409_10876_gb300 import inputs, quality, warmstart
    from paper_2409_10876_gb300.recovery import (NFRecovery, PGRecovery, SirenRecovery, measurement_spectra,
                                                 synthesize_stack)
    pm = quality.image_mask(cfg)
    nm = inputs.sos_mask(cfg).astype(bool)
    mask_d = torch.as_tensor(nm.astype(np.uint8), device=dev)
    rng_sos = cfg.sos_hi - cfg.sos_lo
    rows = {k: [] for k in ("uniform_sos", "pg_cold", "pg_warm", "siren", "nf_mlp", "sos_oracle")}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v = fn()
        torch.cuda.synchronize()
        return v, time.perf_counter() - t0

    for seed in seeds:
        case = inputs.make_case(cfg, seed)
        Y = measurement_spectra(pb, case, dev)
        stack = synthesize_stack(pb, case, dev)
        truth = case["sos_true"].astype(np.float64)
        v_u = torch.full((cfg.sos_g, cfg.sos_g), cfg.v_bg, device=dev)

        def pg_cold():
            rec = PGRecovery(pb, Y, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, v_u, mask_d)
            rec.capture()
            for _ in range(cfg.steps):
                rec.iterate()
            return rec.sos

        def pg_warm():
            vw = warmstart.predict(net1, pb, stack)
            return warmstart.recover_warm(pb, Y, case["d"], cfg.eps, cfg.tv_lambda, cfg.lr, vw, mask_d,
                                          2 * cfg.steps)["sos"]

        def siren():
            rec = SirenRecovery(pb, Y, case["d"], cfg.eps, inputs.SIREN_LR, inputs.siren_init(seed), case["mask"])
            rec.capture()
            for _ in range(cfg.steps):
                rec.iterate()
            return rec.sos

        def nf_mlp():
            rec = NFRecovery(pb, Y, case["d"], cfg.eps, inputs.NF_LR, inputs.nf_init(seed), case["mask"])
            rec.capture()
            for _ in range(cfg.steps):
                rec.iterate()
            return rec.sos

        for name, fn in (("uniform_sos", lambda: v_u), ("pg_cold", pg_cold), ("pg_warm", pg_warm),
                         ("siren", siren), ("nf_mlp", nf_mlp),
                         ("sos_oracle", lambda: torch.as_tensor(case["sos_true"], device=dev))):
            v, secs = timed(fn)
            img, s_img = timed(lambda: quality.recovered_image(pb, Y, case["d"], cfg.eps, v))
            vs = v.cpu().numpy().astype(np.float64)
            rows[name].append({"seed": seed, "s": secs + s_img,
                               "ip_psnr": quality.psnr(img, case["ip"], 1.0, pm),
                               "ip_ssim": quality.ssim(img, case["ip"], 1.0, pm),
                               "sos_psnr": quality.psnr(vs, truth, rng_sos, nm),
                               "sos_ssim": quality.ssim(vs, truth, rng_sos, nm),
                               "sos_rms_mps": float(np.sqrt(np.mean((vs[nm] - truth[nm]) ** 2)))})
    out = {"seeds": list(seeds), "sos_range_mps": rng_sos, "iters": cfg.steps}
    for name, rs in rows.items():
        out[name] = {k: float(np.mean([r[k] for r in rs])) for k in rs[0] if k != "seed"}
        out[name]["per_seed"] = rs
    return out


def kernel_revision() -> str:
    """Hash of the fused kernel source: stored traffic counters apply only to it."""
    import hashlib
    src = os.path.join(ROOT, "paper_2409_10876_gb300", "csrc", "deconv.cu")
    return hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]


def main():
    args = parse()
    rank, world, local = dist_env()
    from paper_2409_10876_gb300 import inputs
    cfg = inputs.config_full()
    from paper_2409_10876_gb300 import ranks
    case = inputs.make_case(cfg, ranks.rank_seed(args.seed, rank))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            if rank == 0:
                run_reference(args, cfg, case, rank, world)
            return
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, cfg, case, rank, world)
        return
    run_gpu(args, cfg, case, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
