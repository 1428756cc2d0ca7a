"""Benchmark of the GB300 NLINV hot path on the real-time radial stream.

Workload (one step = F consecutive frames of one stream, carried on from the
previous step): image side N = 160 on the G = 320 grid, J = 10 channels, 13
radial spokes per frame rotating over U = 5 turns, 7 Newton steps x 10 CG,
regularisation to the previous frame, a moving ellipse phantom with fixed
coil maps and sigma = 1e-3 noise; synthetic data, gridded and PSF'd on the
device before timing.  Frames of one stream depend on each other, so the
frame rate is 1 / per-frame latency.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth as S  # noqa: E402

CFG = dict(N=160, J=10, K=13, U=5, M=7, CG=10, sigma=1e-3, seed=1702)
METRIC = "NLINV frames/s (320^2 grid, 10 ch, radial 13 spokes, 7x10)"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def source_hash() -> str:
    import hashlib
    import glob
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1701_08361_gb300", "csrc", "*"))):
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """DRAM read + write bytes per launch of `kernel` (for "frame_phases":
    per frame, the sum over the frame's phase kernels) from the record of the
    last ncu capture (profiles/traffic.json: kernel, source hash, bytes), or
    None when there is none or the kernel sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        rec = json.load(open(p)).get(kernel)
    except Exception:
        return None
    if not rec or rec.get("source_sha16") != source_hash():
        return None
    return float(rec["dram_bytes_per_launch"])


def sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def fp32_peak_tflops(pk):
    """FP32 ALU roof: SMs x 128 FP32 lanes x 2 flop (FMA) x the maximum SM clock."""
    return sm_count() * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def flops_per_frame(N, G, Gc, J, M, K):
    """Algorithmic FP32 flops of one frame: (K + 1) operator applications per
    Newton step; per channel and application (4N + 2G + 2Gc) length-G
    transforms at 5 G log2 G flops plus the pointwise work."""
    per_ch = (4 * N + 2 * G + 2 * Gc) * 5.0 * G * math.log2(G) + 28 * N * N + 2 * G * G + 4 * Gc * Gc
    return M * (K + 1) * J * per_ch


def bytes_per_frame(N, G, Gc, J, M, K):
    """Algorithmic HBM bytes of one frame with FFT intermediates on chip:
    per CG iteration the CG vectors (10 n_x), the coil maps (J N^2), rho
    (N^2) and the PSF (4 G^2 bytes)."""
    nx = N * N + J * Gc * Gc
    per_it = 8 * (10 * nx + J * N * N + N * N) + 4 * G * G
    return M * (K + 1) * per_it


def make_raw_frames(nframes, seed):
    N, J, K, U = CFG["N"], CFG["J"], CFG["K"], CFG["U"]
    coils = S.coil_maps(N, J, seed)
    out = []
    for n in range(nframes):
        kx, ky, y, _, _ = S.radial_frame(N, J, K, U, n, seed, CFG["sigma"], coils=coils)
        out.append((kx, ky, y))
    return out


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier_max(x, world):
    """Barrier, then the maximum of x over ranks (on the GPU under NCCL, on
    the host under gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Seed of rank's replica stream: each rank reconstructs its own
    independent stream (no data is exchanged between ranks)."""
    return CFG["seed"] + 1000 * rank


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------- ours
def run_ours(args):
    import torch
    from paper_1701_08361_gb300 import nlinv as L

    world, rank, local = dist_init(args)
    N, J, U = CFG["N"], CFG["J"], CFG["U"]
    G = 2 * N
    F = args.frames_per_step
    seed = replica_seed(rank)                 # independent replica stream per rank
    raw = make_raw_frames(F, seed)
    p = L.nlinv_default_params(N, J)
    p.n_turns = U
    p.newton_steps, p.cg_iters = CFG["M"], CFG["CG"]
    p.exec_mode = args.exec_mode
    plan = L.nlinv_plan(p)
    Gc = plan.Gc
    dev = torch.device("cuda")
    Yall = torch.empty((F, J * G * G), dtype=torch.complex64, device=dev)
    Ps = torch.empty((U, G * G), dtype=torch.float32, device=dev)
    for n, (kx, ky, y) in enumerate(raw):
        kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device=dev)
        if n < U:
            L.nlinv_psf(plan, n % U, kxy, Ps[n])
        L.nlinv_grid(plan, kxy, torch.tensor(y, dtype=torch.complex64, device=dev), Yall[n])
    assert L.nlinv_sync(plan) == 0
    x = torch.empty(plan.nx, dtype=torch.complex64, device=dev)
    imgs = torch.empty((F, N * N), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    state = {"first": True, "frame": 0}

    def step(evs=None, Ysrc=None):
        for n in range(F):
            if evs is not None:
                evs[n][0].record(st)
            L.nlinv_frame(plan, Ysrc[n] if Ysrc is not None else Yall[n], state["frame"] % U,
                          None if state["first"] else x, x, None, imgs[n])
            if evs is not None:
                evs[n][1].record(st)
            state["first"] = False
            state["frame"] += 1

    for _ in range(args.warmup):
        step()
    rc = L.nlinv_sync(plan)
    if rc != 0:
        raise RuntimeError(L.nlinv_strerror(rc))

    clocks = Clocks(local)
    K = args.steps
    ev_frames = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(F)]
                 for _ in range(K)]
    ev_step = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    for s in range(K):
        flush.fill_(float(s))
        ev_step[s][0].record(st)
        step(ev_frames[s])
        ev_step[s][1].record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    rc = L.nlinv_sync(plan)
    if rc != 0:
        raise RuntimeError(L.nlinv_strerror(rc))
    t_steps = [ev_step[s][0].elapsed_time(ev_step[s][1]) for s in range(K)]
    t_frames = [ev_frames[s][n][0].elapsed_time(ev_frames[s][n][1]) for s in range(K) for n in range(F)]
    total_ms = barrier_max(sum(t_steps), world)
    frames = K * F * world
    value = frames / (total_ms / 1e3)
    lat = sorted(t_frames)

    # end to end: pinned host Y in, images out, copies inside the timed region
    Yh = Yall.cpu().pin_memory()
    imgs_h = torch.empty(imgs.shape, dtype=imgs.dtype).pin_memory()
    Ydev = torch.empty_like(Yall)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(st)
    for s in range(K):
        Ydev.copy_(Yh, non_blocking=True)
        step(None, Ydev)
        imgs_h.copy_(imgs, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = barrier_max(e0.elapsed_time(e1), world)
    rc = L.nlinv_sync(plan)
    if rc != 0:
        raise RuntimeError(L.nlinv_strerror(rc))

    pk, pk_src = peaks()
    path, cs = L.nlinv_plan_path(plan)
    kernel_name = {1: "per-phase launches (k_row_cg, k_col_c, ...)",
                   4: "per-phase launches in a CUDA graph with programmatic dependent launch",
                   2: "k_frame (grid kernel, one launch per frame)",
                   3: "k_frame_cl (cluster kernel, one launch per frame, %d CTAs per channel)" % cs}[path]
    fl = flops_per_frame(N, G, Gc, J, CFG["M"], CFG["CG"])
    by = bytes_per_frame(N, G, Gc, J, CFG["M"], CFG["CG"])
    mean_frame_s = statistics.mean(t_frames) / 1e3
    fp32_peak = fp32_peak_tflops(pk)   # TFLOP/s
    achieved = fl / mean_frame_s / 1e12
    hbm = by / mean_frame_s / 1e9

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "frames/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": round(total_ms / K, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic",
        "config": {"workload": "real-time radial stream: N=160, G=320, J=10, 13 spokes x 5 turns, "
                               "7 Newton x 10 CG, moving phantom, sigma=1e-3",
                   "frames_per_step": F,
                   "exec_mode": ["default", "per-phase", "grid kernel", "cluster kernel",
                                 "per-phase CUDA graph"][args.exec_mode],
                   "l2": "inputs larger than L2 (%.0f MB of gridded data per step) and L2 flushed "
                         "between steps" % (Yall.numel() * 8 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "latency_ms": {"p50": round(statistics.median(lat), 4), "min": round(lat[0], 4)},
        "roofline": {"bound": "alu", "achieved": round(achieved, 3),
                     "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                     "frac": round(achieved / fp32_peak, 4), "traffic": profiled_traffic({1: "frame_phases", 2: "k_frame", 3: "k_frame_cl",
                                                                  4: "frame_phases"}[path]),
                     "kernel": kernel_name,
                     "peak_source": "FP32: %d SMs x 128 lanes x 2 flop x sm_max_mhz (%s)" % (sm_count(), pk_src)},
        "hbm": {"achieved_gbs": round(hbm, 1), "peak_gbs": pk["hbm_gbs"],
                "frac": round(hbm / pk["hbm_gbs"], 4), "peak_source": pk_src},
        "e2e": {"value": round(frames / (e2e_ms / 1e3), 2), "unit": "frames/s",
                "h2d_bytes_per_step": int(Yall.numel() * 8),
                "d2h_bytes_per_step": int(imgs.numel() * 8)},
        "gpu_launches": K * F,
        "clocks": clk,
    }
    if path in (1, 4):
        M, C = CFG["M"], CFG["CG"]
        # the pointer table, init, per Newton step 5 right-hand-side phases,
        # 4 per CG iteration and the CG's last step, the final coil maps (2)
        # and the outputs (the same kernels whether launched one by one or
        # replayed from the CUDA graph)
        out["gpu_launches"] = K * F * (2 + M * (5 + 4 * C + (1 if C > 0 else 0)) + 2 + 1)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_frames)
    if rank == 0 and args.plain_loop:
        out["plain_gpu_loop"] = plain_gpu_loop(raw, args)
    if rank == 0 and args.unfused_frames > 0 and args.exec_mode != 1:
        out["unfused_own_kernels"] = unfused_own_kernels(Yall, Ps, args)
    if rank == 0 and args.c3_groups > 0:
        out["batched_c3"] = batched_c3(args)
    if rank == 0 and args.c4_frames > 0:
        out["high_channel_c4"] = high_channel_c4(args)
    if rank == 0 and args.c5_steps > 0:
        out["differentiable_c5"] = differentiable_c5(args)
    plan.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------ own kernels unfused, one frame at a time
def unfused_own_kernels(Yall, Ps, args):
    """The same frames through the library's per-phase execution mode (one
    launch per fused phase, no persistent kernel): the project's own kernels
    without the whole-frame fusion, one frame at a time."""
    import torch
    from paper_1701_08361_gb300 import nlinv as L
    N, J, U = CFG["N"], CFG["J"], CFG["U"]
    p = L.nlinv_default_params(N, J)
    p.n_turns = U
    p.newton_steps, p.cg_iters = CFG["M"], CFG["CG"]
    p.exec_mode = 1
    plan = L.nlinv_plan(p)
    for u in range(U):
        L.nlinv_set_psf(plan, u, Ps[u])
    x = torch.empty(plan.nx, dtype=torch.complex64, device=Yall.device)
    st = torch.cuda.current_stream()
    nf = min(args.unfused_frames, Yall.shape[0])
    for n in range(3):
        L.nlinv_frame(plan, Yall[n], n % U, None if n == 0 else x, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for n in range(nf):
        L.nlinv_frame(plan, Yall[n], n % U, x, x)
    e1.record(st)
    torch.cuda.synchronize()
    rc = L.nlinv_sync(plan)
    plan.close()
    if rc != 0:
        raise RuntimeError(L.nlinv_strerror(rc))
    ms = e0.elapsed_time(e1)
    M, C = CFG["M"], CFG["CG"]
    return {"value": round(nf / (ms / 1e3), 2), "unit": "frames/s", "frames": nf,
            "kind": "own kernels, one launch per fused phase (exec_mode 1), one frame at a time",
            "launches_per_frame": 2 + M * (5 + 4 * C + (1 if C > 0 else 0)) + 2 + 1}


# ------------------------------------------- batched uneven frames (C3)
C3 = [dict(N=128, J=8, D=11), dict(N=160, J=10, D=11), dict(N=192, J=16, D=10)]


def batched_c3(args):
    """32 frames in flight per launch group: three size classes (256^2/8 ch,
    320^2/10 ch, 384^2/16 ch), 15 radial spokes, 5 turns, 7 Newton x 10 CG;
    each class keeps D frames in flight (11/11/10) after an in-order warm-up
    of 5 frames (temporal decomposition).  Steady-state frames/s over
    `args.c3_groups` launch groups of 32 frames."""
    import torch
    from paper_1701_08361_gb300 import nlinv as L
    from paper_1701_08361_gb300 import stream as ST
    dev = torch.device("cuda")
    K, U, WU, NDIST = 15, 5, 5, 6
    streams = []
    for ci, c in enumerate(C3):
        N, J, D = c["N"], c["J"], c["D"]
        G = 2 * N
        p = L.nlinv_default_params(N, J)
        p.n_turns = U
        p.max_batch = D
        plan = L.nlinv_plan(p)
        coils = S.coil_maps(N, J, 3000 + ci)
        Yd = []
        for n in range(NDIST):
            kx, ky, y, _, _ = S.radial_frame(N, J, K, U, n, 3000 + ci, 1e-3, coils=coils)
            kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device=dev)
            if n < U:
                L.nlinv_psf(plan, n, kxy)
            Yf = torch.empty(J * G * G, dtype=torch.complex64, device=dev)
            L.nlinv_grid(plan, kxy, torch.tensor(y, dtype=torch.complex64, device=dev), Yf)
            Yd.append(Yf)
        assert L.nlinv_sync(plan) == 0
        nf = WU + 1 + D * (args.c3_groups + 2)
        streams.append(dict(plan=plan, Y=[Yd[n % NDIST] for n in range(nf)],
                            turns=[n % U for n in range(nf)], delay=D, warmup=WU,
                            x=torch.empty((nf, plan.nx), dtype=torch.complex64, device=dev)))
    per = [ST.groups(len(s["Y"]), s["delay"], s["warmup"]) for s in streams]
    st = torch.cuda.current_stream()

    def launch(g):
        frames = []
        for s, pg in zip(streams, per):
            for n in pg[g]:
                src = ST.source(n, s["delay"], s["warmup"])
                frames.append(dict(plan=s["plan"], Y=s["Y"][n], turn=s["turns"][n],
                                   x_prev=None if src < 0 else s["x"][src], x_out=s["x"][n]))
        L.nlinv_batch(frames)
        return len(frames)

    g = 0
    while g < WU + 2:          # warm-up groups and two full groups untimed
        launch(g)
        g += 1
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    nframes = 0
    for _ in range(args.c3_groups):
        nframes += launch(g)
        g += 1
    e1.record(st)
    torch.cuda.synchronize()
    for s in streams:
        rc = L.nlinv_sync(s["plan"])
        if rc != 0:
            raise RuntimeError(L.nlinv_strerror(rc))
    ms = e0.elapsed_time(e1)
    flops = sum(c["D"] * flops_per_frame(c["N"], 2 * c["N"], c["N"] // 2, c["J"], CFG["M"], CFG["CG"])
                for c in C3)
    achieved = flops * args.c3_groups / (ms / 1e3) / 1e12
    pk, _ = peaks()
    fp32_peak = fp32_peak_tflops(pk)
    for s in streams:
        s["plan"].close()
    return {"value": round(nframes / (ms / 1e3), 2), "unit": "frames/s",
            "ms_per_group": round(ms / args.c3_groups, 3), "frames_per_group": nframes // args.c3_groups,
            "achieved_tflops": round(achieved, 3), "frac_fp32": round(achieved / fp32_peak, 4),
            "workload": "batched uneven frames: 256^2/8 ch x 11 + 320^2/10 ch x 11 + 384^2/16 ch x 10 "
                        "in flight, 15 spokes, 7x10, temporal decomposition after 5 in-order frames"}


# ---------------------------------------- high channel count (C4) stream
def high_channel_c4(args):
    """N=256 on the 512 grid, 64 channels, 9 radial spokes x 5 turns, 7 Newton
    x 10 CG, frames in order (each from the previous one).  The work per frame
    does not depend on the data values, so the gridded k-space is seeded
    random complex data of the C4 shape; the PSFs come from the trajectory."""
    import torch
    from paper_1701_08361_gb300 import nlinv as L
    dev = torch.device("cuda")
    N, J, K, U = 256, 64, 9, 5
    G = 2 * N
    p = L.nlinv_default_params(N, J)
    p.n_turns = U
    plan = L.nlinv_plan(p)
    for u in range(U):
        kx, ky = S.radial_trajectory(N, K, U, u)
        L.nlinv_psf(plan, u, torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device=dev))
    gen = torch.Generator(device=dev)
    gen.manual_seed(4000)
    Y = torch.randn((2, J * G * G), dtype=torch.complex64, device=dev, generator=gen) * 1e-2
    F = args.c4_frames
    xs = torch.empty((F + 2, plan.nx), dtype=torch.complex64, device=dev)
    st = torch.cuda.current_stream()

    def frame(n):
        L.nlinv_frame(plan, Y[n % 2], n % U, None if n == 0 else xs[n - 1], xs[n])

    frame(0)
    frame(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for n in range(2, F + 2):
        frame(n)
    e1.record(st)
    torch.cuda.synchronize()
    rc = L.nlinv_sync(plan)
    if rc != 0:
        raise RuntimeError(L.nlinv_strerror(rc))
    ms = e0.elapsed_time(e1) / F
    plan.close()
    flops = flops_per_frame(N, G, G // 4, J, CFG["M"], CFG["CG"])
    achieved = flops / (ms / 1e3) / 1e12
    pk, _ = peaks()
    fp32_peak = fp32_peak_tflops(pk)
    return {"value": round(1e3 / ms, 2), "unit": "frames/s", "ms_per_frame": round(ms, 3),
            "frames": F, "achieved_tflops": round(achieved, 3), "frac_fp32": round(achieved / fp32_peak, 4),
            "workload": "N=256 / 512^2 grid, 64 channels, 9 spokes x 5 turns, 7x10, sequential frames, "
                        "seeded random gridded k-space (data-independent work)"}


# ------------------------------------ differentiable unrolled NLINV (C5)
def differentiable_c5(args):
    """A batch of 8 frames (--c5-batch) of the real-time stream's size
    (N=160 / 320 grid, 10 channels, 13 spokes, 7 x 10) through the
    torch.autograd.Function: forward (nlinv_batch) and the hand-written
    backward (per frame: one forward sweep recording every Newton step's CG,
    then the reverse sweep) for L = Re<g, x^_M>, with gradients w.r.t. the
    gridded data and alpha_0.  Time per training step."""
    import torch
    from paper_1701_08361_gb300 import nlinv as L
    from paper_1701_08361_gb300 import autograd as AG
    dev = torch.device("cuda")
    N, J, U, B = CFG["N"], CFG["J"], CFG["U"], args.c5_batch
    G = 2 * N
    p = L.nlinv_default_params(N, J)
    p.n_turns = U
    p.max_batch = B
    plan = L.nlinv_plan(p)
    raw = make_raw_frames(B, CFG["seed"] + 5)
    Ys = torch.empty((B, J * G * G), dtype=torch.complex64, device=dev)
    for n, (kx, ky, y) in enumerate(raw):
        kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device=dev)
        if n < U:
            L.nlinv_psf(plan, n, kxy)
        L.nlinv_grid(plan, kxy, torch.tensor(y, dtype=torch.complex64, device=dev), Ys[n])
    gen = torch.Generator(device=dev)
    gen.manual_seed(5000)
    gv = torch.randn((B, plan.nx), dtype=torch.complex64, device=dev, generator=gen)
    turns = [n % U for n in range(B)]
    st = torch.cuda.current_stream()

    def step():
        Yt = Ys.detach().requires_grad_(True)
        a0 = torch.tensor(1.0, dtype=torch.float64, device=dev, requires_grad=True)
        xs = AG.nlinv_batch(Yt, a0, plan, turns)
        (gv.conj() * xs).real.sum().backward()
        return Yt.grad, a0.grad

    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(st)
    for _ in range(args.c5_steps):
        yg, ag = step()
    e1.record(st)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / args.c5_steps * 1e3
    ms = e0.elapsed_time(e1) / args.c5_steps
    # the forward alone (no graph kept), to split the step into its two halves
    a0c = torch.tensor(1.0, dtype=torch.float64, device=dev)
    with torch.no_grad():
        AG.nlinv_batch(Ys, a0c, plan, turns)
        e0.record(st)
        for _ in range(args.c5_steps):
            AG.nlinv_batch(Ys, a0c, plan, turns)
        e1.record(st)
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / args.c5_steps
    rc = L.nlinv_sync(plan)
    plan.close()
    if rc != 0 or not bool(torch.isfinite(yg).all()) or not math.isfinite(float(ag)):
        raise RuntimeError("C5 step failed")
    return {"value": round(B / (ms / 1e3), 2), "unit": "frames/s (forward + backward)",
            "ms_per_step": round(ms, 3), "wall_ms_per_step": round(wall, 3), "forward_ms": round(fwd, 3),
            "backward_ms": round(ms - fwd, 3), "batch": B, "steps": args.c5_steps,
            "workload": "%d frames N=160 / 320^2 grid, 10 channels, 13 spokes, 7x10 unrolled; "
                        "d/dY and d/dalpha_0 of Re<g, x^_M> through torch.autograd" % B}


# --------------------------------------------------- CPU oracle baseline
def oracle_frames(nframes, seed):
    import oracle as O
    N, J, U = CFG["N"], CFG["J"], CFG["U"]
    G = 2 * N
    raw = make_raw_frames(nframes, seed)
    frames = [(O.grid_data(kx, ky, y, N, G), O.psf_kernel(kx, ky, N, G).real) for kx, ky, y in raw]
    return frames


def cpu_baseline(nframes):
    """The FP64 oracle as it stands, timed on the host cores over a bounded
    sample of the stream (the first `nframes` frames)."""
    import oracle as O
    N, J = CFG["N"], CFG["J"]
    frames = oracle_frames(nframes, CFG["seed"])
    g = O.Geometry(N=N, J=J)
    prm = O.Params(newton_steps=CFG["M"], cg_iters=CFG["CG"])
    t0 = time.perf_counter()
    O.nlinv_stream(frames, g, prm)
    dt = time.perf_counter() - t0
    return {"value": round(nframes / dt, 4), "unit": "frames/s", "cores": O.workers(),
            "kind": "oracle",
            "sample": f"first {nframes} frames of the stream (FP64 NumPy/SciPy, "
                      f"scipy.fft workers={O.workers()})"}


# -------------------------------------- plain per-frame GPU loop (cuFFT)
def plain_gpu_loop(raw, args):
    """The same algorithm as plain eager torch ops (torch.fft = cuFFT, FP32,
    no fusion), one frame at a time: the comparator the metric names."""
    import torch
    N, J, U = CFG["N"], CFG["J"], CFG["U"]
    G = 2 * N
    from paper_1701_08361_gb300 import nlinv as L
    p = L.nlinv_default_params(N, J)
    p.n_turns = U
    plan = L.nlinv_plan(p)
    Gc = plan.Gc
    dev = torch.device("cuda")
    Ys, Ps = [], []
    for n, (kx, ky, y) in enumerate(raw):
        kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device=dev)
        Yd = torch.empty(J * G * G, dtype=torch.complex64, device=dev)
        L.nlinv_grid(plan, kxy, torch.tensor(y, dtype=torch.complex64, device=dev), Yd)
        Ys.append(Yd.view(J, G, G))
        if n < U:
            Pd = torch.empty(G * G, dtype=torch.float32, device=dev)
            L.nlinv_psf(plan, n, kxy, Pd)
            Ps.append(Pd.view(G, G))
    L.nlinv_sync(plan)
    plan.close()
    i = torch.arange(Gc, device=dev)
    f = torch.where(i < (Gc + 1) // 2, i, i - Gc)
    idx = f % G
    k2 = (2.0 * f / G).double()
    D = ((1 + 220.0 * (k2[:, None] ** 2 + k2[None, :] ** 2)) ** -16).float()

    # padded grids allocated once: only the coil band (zc) or the FOV (zi)
    # is ever written, so the rest stays zero without a memset per call
    zc = torch.zeros((J, G, G), dtype=torch.complex64, device=dev)
    zi = torch.zeros((J, G, G), dtype=torch.complex64, device=dev)
    band = (slice(None), idx[:, None], idx[None, :])

    def Winv(ch):
        zc[band] = D * ch
        return torch.fft.ifft2(zc, norm="ortho")[:, :N, :N]

    def WinvH(v):
        zi[:, :N, :N] = v
        return D * torch.fft.fft2(zi, norm="ortho")[band]

    def pad(v):
        zi[:, :N, :N] = v
        return zi

    def frame(Y, P, rho0, ch0, rhor, chr_):
        rho, ch = rho0.clone(), ch0.clone()
        for n in range(CFG["M"]):
            al = 0.5 ** n
            c = Winv(ch)
            Fx = torch.fft.fft2(pad(rho * c), norm="ortho")
            t = torch.fft.ifft2(Y - P * Fx, norm="ortho")[:, :N, :N]
            br = (c.conj() * t).sum(0) - al * (rho - rhor)
            bc = WinvH(rho.conj() * t) - al * (ch - chr_)
            xr, xc = torch.zeros_like(br), torch.zeros_like(bc)
            rr_, rc_ = br.clone(), bc.clone()
            pr, pc = rr_.clone(), rc_.clone()
            rr = (rr_.abs() ** 2).sum().double() + (rc_.abs() ** 2).sum().double()
            for _ in range(CFG["CG"]):
                u = c * pr + rho * Winv(pc)
                tt = torch.fft.ifft2(P * torch.fft.fft2(pad(u), norm="ortho"), norm="ortho")[:, :N, :N]
                qr = (c.conj() * tt).sum(0) + al * pr
                qc = WinvH(rho.conj() * tt) + al * pc
                pq = (pr.conj() * qr).real.sum().double() + (pc.conj() * qc).real.sum().double()
                a = (rr / pq).float()
                xr, xc = xr + a * pr, xc + a * pc
                rr_, rc_ = rr_ - a * qr, rc_ - a * qc
                rn = (rr_.abs() ** 2).sum().double() + (rc_.abs() ** 2).sum().double()
                b = (rn / rr).float()
                pr, pc = rr_ + b * pr, rc_ + b * pc
                rr = rn
            rho, ch = rho + xr, ch + xc
        return rho, ch

    rho = torch.ones((N, N), dtype=torch.complex64, device=dev)
    ch = torch.zeros((J, Gc, Gc), dtype=torch.complex64, device=dev)
    st = torch.cuda.current_stream()
    for n in range(min(3, len(Ys))):
        rho, ch = frame(Ys[n], Ps[n % U], rho, ch, rho, ch)
    torch.cuda.synchronize()
    nf = min(len(Ys), args.plain_frames)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for n in range(nf):
        rho, ch = frame(Ys[n], Ps[n % U], rho, ch, rho, ch)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": round(nf / (ms / 1e3), 2), "unit": "frames/s",
            "kind": "plain torch.fft/cuFFT eager loop, FP32, one frame at a time, padded grids "
                    "allocated once",
            "frames": nf}


# ------------------------------------------------------- reference arm
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    N, J = CFG["N"], CFG["J"]
    g = O.Geometry(N=N, J=J)
    prm = O.Params(newton_steps=CFG["M"], cg_iters=CFG["CG"])
    nf = args.warmup + args.steps
    frames = oracle_frames(nf, CFG["seed"])
    init = O.XVec.initial(g)
    x = init
    times = []
    for s in range(nf):
        Y, P = frames[s]
        t0 = time.perf_counter()
        x = O.nlinv_frame(Y, P, x, x, g, prm)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = len(times) / tot
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot / len(times), 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": "real-time radial stream: N=160, G=320, J=10, 13 spokes x 5 turns, "
                               "7 Newton x 10 CG, moving phantom, sigma=1e-3",
                   "frames_per_step": 1},
        "cpu_baseline": {"value": round(value, 4), "unit": "frames/s", "cores": O.workers(),
                         "kind": "oracle",
                         "sample": "one frame of the stream per step (FP64 NumPy/SciPy oracle)"},
        "e2e": {"value": round(value, 4), "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames-per-step", type=int, default=25)
    ap.add_argument("--exec-mode", type=int, default=0, choices=[0, 1, 2, 3, 4])
    ap.add_argument("--cpu-frames", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-loop", type=int, default=1)
    ap.add_argument("--plain-frames", type=int, default=10)
    ap.add_argument("--unfused-frames", type=int, default=10)
    ap.add_argument("--c3-groups", type=int, default=4)
    ap.add_argument("--c4-frames", type=int, default=3)
    ap.add_argument("--c5-steps", type=int, default=1)
    ap.add_argument("--c5-batch", type=int, default=8, help="frames per C5 step (8: the configuration)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
