"""Measured choice of the grid and the execution path per problem size.

The paper picks the oversampled grid G = 2 gamma N (Eq. 8) from a table of
measured FFT times (Sec. 3.2, Tab. 2) and the parallel set-up from a
database of measured reconstruction times (Sec. 3.3).  Here the unit that is
timed is a whole NLINV frame on this GPU: for an N x N image with J channels
(M Newton steps x K CG iterations) the tuner runs frames for every compiled
grid with gamma in a given range and every execution path a plan can take on
it -- the per-phase frame replayed as a CUDA graph, one launch per fused
phase, the grid kernel, and the cluster kernel for each cluster size whose J
clusters are co-resident -- and keeps the fastest.  The pick and every
candidate's time (CUDA events, median of the timed frames) are stored in a
JSON database keyed by the GPU name, so that later plans for the same sizes
are made from the record (tuned_params) instead of being re-measured.

This module only chooses parameters: every timed frame runs in the library.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import time

import numpy as np
import torch

from . import nlinv as L

DB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_db.json")
CLUSTER_SIZES = (16, 15, 12, 10, 9, 8, 6, 5, 4)


def _key(N, J, M, K):
    return f"N{N}_J{J}_M{M}_K{K}"


def gpu_name() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _params(N, J, M, K, G, exec_mode, cluster_cs, turns=1):
    p = L.nlinv_default_params(N, J)
    p.newton_steps, p.cg_iters = M, K
    p.n_turns = turns
    p.G = G
    p.exec_mode = exec_mode
    p.cluster_cs = cluster_cs
    return p


def candidates(N, J, M=7, K=10, gamma=(1.0, 2.0)):
    """Every (G, exec_mode, cluster_cs) a plan accepts for these sizes, G over
    the compiled grids with 2 N gamma[0] <= G <= 2 N gamma[1]."""
    out = []
    grids = sorted(G for G, n in L.nlinv_grid_list() if n == N and 2 * N * gamma[0] <= G <= 2 * N * gamma[1])
    for G in grids:
        out.append(dict(G=G, exec_mode=4, cluster_cs=0))
        out.append(dict(G=G, exec_mode=2, cluster_cs=0))
        out.append(dict(G=G, exec_mode=1, cluster_cs=0))
        for cs in CLUSTER_SIZES:
            try:
                L.nlinv_plan(_params(N, J, M, K, G, 3, cs)).close()
            except L.NlinvError:
                continue
            out.append(dict(G=G, exec_mode=3, cluster_cs=cs))
    return out


def measure(N, J, cand, M=7, K=10, frames=6, warmup=2, spokes=13, seed=5, batch=1):
    """Median ms per frame of a stream of frames with the candidate's plan
    (batch > 1: `batch` frames in flight per nlinv_batch call, the call's time
    divided by `batch`).  The work of a frame does not depend on the data
    (fixed Newton and CG counts), so the gridded data are seeded random values
    and the PSF comes from a radial trajectory of `spokes` spokes on the
    candidate's grid."""
    from synth import radial_trajectory
    dev = torch.device("cuda")
    G = cand["G"]
    prm = _params(N, J, M, K, G, cand["exec_mode"], cand["cluster_cs"])
    prm.max_batch = max(1, batch)
    plan = L.nlinv_plan(prm)
    kx, ky = radial_trajectory(N, spokes, 5, 0)
    L.nlinv_psf(plan, 0, torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device=dev))
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    Y = torch.randn(J * G * G, dtype=torch.complex64, device=dev, generator=gen) * 1e-2
    x = torch.empty(plan.nx, dtype=torch.complex64, device=dev)
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(frames)]
    if batch > 1:
        xs = torch.empty((batch, plan.nx), dtype=torch.complex64, device=dev)
        L.nlinv_frame(plan, Y, 0, None, x)
        descs = [dict(plan=plan, Y=Y, turn=0, x_prev=x, x_out=xs[f]) for f in range(batch)]
        run = lambda: L.nlinv_batch(descs)
    else:
        run = lambda: L.nlinv_frame(plan, Y, 0, x, x)
        L.nlinv_frame(plan, Y, 0, None, x)
    for n in range(warmup):
        run()
    for n in range(frames):
        ev[n][0].record(st)
        run()
        ev[n][1].record(st)
    torch.cuda.synchronize()
    rc = L.nlinv_sync(plan)
    path = L.nlinv_plan_path(plan)
    plan.close()
    if rc != 0:
        raise L.NlinvError(rc, "tune.measure")
    return statistics.median(a.elapsed_time(b) for a, b in ev) / max(1, batch), path


def _load(db):
    if db and os.path.exists(db):
        with open(db) as f:
            return json.load(f)
    return {}


def tune(N, J, M=7, K=10, gamma=(1.0, 2.0), db=DB_PATH, write=True, frames=6):
    """Time every candidate, keep the fastest; returns the record (and stores
    it under the GPU's name and the sizes when `write`)."""
    rows = []
    for c in candidates(N, J, M, K, gamma):
        ms, path = measure(N, J, c, M, K, frames=frames)
        rows.append(dict(c, ms_per_frame=round(ms, 4), path=path[0], cluster_size=path[1]))
    best = min(rows, key=lambda r: r["ms_per_frame"])
    rec = dict(pick={k: best[k] for k in ("G", "exec_mode", "cluster_cs")}, ms_per_frame=best["ms_per_frame"],
               gamma=[gamma[0], gamma[1]], candidates=rows, frames_timed=frames,
               when=time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()))
    if write and db:
        data = _load(db)
        data.setdefault(gpu_name(), {})[_key(N, J, M, K) + f"_g{gamma[0]}-{gamma[1]}"] = rec
        with open(db, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    return rec


def lookup(N, J, M=7, K=10, gamma=(1.0, 2.0), db=DB_PATH):
    """The stored record for this GPU and these sizes, or None."""
    return _load(db).get(gpu_name(), {}).get(_key(N, J, M, K) + f"_g{gamma[0]}-{gamma[1]}")


def tuned_params(N, J, M=7, K=10, gamma=(1.0, 2.0), db=DB_PATH, measure_if_missing=False):
    """nlinv_params_t with the recorded pick (defaults when there is none and
    `measure_if_missing` is false)."""
    rec = lookup(N, J, M, K, gamma, db)
    if rec is None and measure_if_missing:
        rec = tune(N, J, M, K, gamma, db)
    p = _params(N, J, M, K, 0, 0, 0)
    if rec is not None:
        p.G, p.exec_mode, p.cluster_cs = rec["pick"]["G"], rec["pick"]["exec_mode"], rec["pick"]["cluster_cs"]
    return p


# ------------------------------------------------ compile-time knobs
# Per compiled grid the tile width TW (columns of a column item, rows of a row
# item), the elements per thread and round of the elementwise parts
# (NLINV_EU), the CTAs per SM the frame-indexed phase kernels are compiled
# for (NLINV_PMINB) and the fewest CTAs a phase leaves to its elementwise part
# (NLINV_ELEM_CTAS) are fixed when the library is built.  compile_sweep
# builds one library per variant (only this grid's unit, all variants in
# parallel, each in its own object folder), times each in a child process on
# the default execution path and records every time and the fastest.

def _fits(g1, g2, n, tw, mb, stage_psf=0):
    """Whether Cfg<g1, g2, n, tw, mb> compiles: 16-byte staging chunks, whole
    warps within 1024 threads, the shared memory of one CTA within the limit
    for mb CTAs per SM (the conditions the Cfg static_asserts check)."""
    G, mx = g1 * g2, max(g1, g2)
    bs = (tw * mx + 31) // 32 * 32
    smem = tw * (G + mx) * 8 + 2 * n * tw * 8 + (G * tw * 4 if stage_psf else 0)
    lim = 227 * 1024 if mb == 1 else 228 * 1024 // mb - 1024
    return tw % 4 == 0 and G % 2 == 0 and bs <= 1024 and smem <= lim and 2 * n <= G


def built_in_knob(name):
    """The library's default of a compile-time knob (the #define in the
    kernel sources)."""
    import re
    src = open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "phases.cuh")).read()
    m = re.search(r"#define %s (\d+)" % name, src)
    if not m:
        src = open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "grid.cuh")).read()
        m = re.search(r"#define %s (\d+)" % name, src)
    return int(m.group(1))


# the -D knobs the sweep varies (besides the tile width) and their candidates
KNOBS = {"NLINV_EU": (2, 4, 8), "NLINV_PMINB": (1, 2), "NLINV_ELEM_CTAS": (16, 32, 64)}


def compile_variants(N, G=None, tws=(8, 12, 16), knobs=None):
    """Variants of the compiled grid for (G, N) (G = 2N by default): the
    built-in one, then one knob changed at a time -- each tile width in `tws`
    and each candidate of every -D knob in `knobs` (default KNOBS).  Returns
    dicts with the grid tuple (G1, G2, N, TW, MINB), the knob values and the
    nvcc -D flags."""
    from . import build as B
    G = 2 * N if G is None else G
    knobs = KNOBS if knobs is None else knobs
    base = [t for t in B.grid_sizes() if t[0] * t[1] == G and t[2] == N]
    if not base:
        raise ValueError(f"no compiled grid for G={G}, N={N}")
    g1, g2, n, tw0, mb = base[0]
    k0 = {k: built_in_knob(k) for k in knobs}
    out = [dict(grid=(g1, g2, n, tw0, mb), knobs=dict(k0))]
    out += [dict(grid=(g1, g2, n, tw, mb), knobs=dict(k0)) for tw in tws if tw != tw0]
    for k, cands in knobs.items():
        out += [dict(grid=(g1, g2, n, tw0, mb), knobs=dict(k0, **{k: v})) for v in cands if v != k0[k]]
    out = [v for v in out if _fits(*v["grid"])]
    short = {"NLINV_EU": "eu", "NLINV_PMINB": "pm", "NLINV_ELEM_CTAS": "ec"}
    for v in out:
        v["flags"] = [f"-D{k}={x}" for k, x in sorted(v["knobs"].items())]
        v["name"] = "tw{}_".format(v["grid"][3]) + "_".join(
            "{}{}".format(short.get(k, k.lower()), x) for k, x in sorted(v["knobs"].items()))
    return out


def _time_in_child(lib, N, J, G, M, K, frames, batch=1):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import json, sys; sys.path.insert(0, %r); from paper_1701_08361_gb300 import tune as T; "
            "ms, path = T.measure(%d, %d, dict(G=%d, exec_mode=0, cluster_cs=0), %d, %d, frames=%d, batch=%d); "
            "print(json.dumps(dict(ms=ms, path=list(path))))" % (root, N, J, G, M, K, frames, batch))
    env = dict(os.environ, NLINV_LIB=lib)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return None, r.stderr.strip().splitlines()[-1:] or ["failed"]
    return json.loads(r.stdout.strip().splitlines()[-1])["ms"], None


def compile_sweep(N, J, M=7, K=10, G=None, frames=6, db=DB_PATH, write=True, workdir=None, variants=None,
                  batch=1):
    """Build and time every compile variant (compile_variants) for an N x N
    image with J channels; returns (and records under the GPU's name) the
    times and the fastest variant."""
    import concurrent.futures as cf
    import tempfile
    from . import build as B
    G = 2 * N if G is None else G
    vs = variants if variants is not None else compile_variants(N, G)
    work = workdir or tempfile.mkdtemp(prefix="nlinv_sweep_")
    per = max(1, (os.cpu_count() or 2) // max(1, len(vs)))

    def build_one(v):
        lib = os.path.join(work, f"lib_{v['name']}.so")
        B.build(force=True, extra=v["flags"], sizes=[v["grid"]], lib=lib, obj=os.path.join(work, v["name"]),
                workers=per)
        return lib

    with cf.ThreadPoolExecutor(max_workers=len(vs)) as ex:
        libs = list(ex.map(build_one, vs))
    rows = []
    for v, lib in zip(vs, libs):
        ms, err = _time_in_child(lib, N, J, G, M, K, frames, batch)
        rows.append(dict(name=v["name"], tw=v["grid"][3], knobs=v["knobs"],
                         ms_per_frame=None if ms is None else round(ms, 4), error=err))
    ok = [r for r in rows if r["ms_per_frame"] is not None]
    best = min(ok, key=lambda r: r["ms_per_frame"]) if ok else None
    rec = dict(pick=best, variants=rows, frames_timed=frames, G=G, batch=batch,
               when=time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()))
    if write and db:
        data = _load(db)
        data.setdefault(gpu_name(), {})[_key(N, J, M, K) + f"_G{G}_compile" + (f"_b{batch}" if batch > 1 else "")] = rec
        with open(db, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    return rec


def main():
    ap = argparse.ArgumentParser(description="time NLINV frames per grid and execution path, keep the fastest")
    ap.add_argument("--N", type=int, required=True)
    ap.add_argument("--J", type=int, required=True)
    ap.add_argument("--M", type=int, default=7)
    ap.add_argument("--K", type=int, default=10)
    ap.add_argument("--gamma", type=float, nargs=2, default=(1.0, 2.0))
    ap.add_argument("--frames", type=int, default=6)
    ap.add_argument("--db", default=DB_PATH)
    ap.add_argument("--batch", type=int, default=1, help="frames in flight per call (compile sweep)")
    ap.add_argument("--compile", action="store_true",
                    help="sweep the compile-time knobs of the G = 2N grid instead of grids and paths")
    a = ap.parse_args()
    if a.compile:
        rec = compile_sweep(a.N, a.J, a.M, a.K, frames=a.frames, db=a.db, batch=a.batch)
    else:
        rec = tune(a.N, a.J, a.M, a.K, tuple(a.gamma), a.db, frames=a.frames)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
