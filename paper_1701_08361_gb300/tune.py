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


def measure(N, J, cand, M=7, K=10, frames=6, warmup=2, spokes=13, seed=5):
    """Median ms per frame of a stream of frames with the candidate's plan.
    The work of a frame does not depend on the data (fixed Newton and CG
    counts), so the gridded data are seeded random values and the PSF comes
    from a radial trajectory of `spokes` spokes on the candidate's grid."""
    from synth import radial_trajectory
    dev = torch.device("cuda")
    G = cand["G"]
    plan = L.nlinv_plan(_params(N, J, M, K, G, cand["exec_mode"], cand["cluster_cs"]))
    kx, ky = radial_trajectory(N, spokes, 5, 0)
    L.nlinv_psf(plan, 0, torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device=dev))
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    Y = torch.randn(J * G * G, dtype=torch.complex64, device=dev, generator=gen) * 1e-2
    x = torch.empty(plan.nx, dtype=torch.complex64, device=dev)
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(frames)]
    for n in range(warmup):
        L.nlinv_frame(plan, Y, 0, None if n == 0 else x, x)
    for n in range(frames):
        ev[n][0].record(st)
        L.nlinv_frame(plan, Y, 0, x, x)
        ev[n][1].record(st)
    torch.cuda.synchronize()
    rc = L.nlinv_sync(plan)
    path = L.nlinv_plan_path(plan)
    plan.close()
    if rc != 0:
        raise L.NlinvError(rc, "tune.measure")
    return statistics.median(a.elapsed_time(b) for a, b in ev), path


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


def main():
    ap = argparse.ArgumentParser(description="time NLINV frames per grid and execution path, keep the fastest")
    ap.add_argument("--N", type=int, required=True)
    ap.add_argument("--J", type=int, required=True)
    ap.add_argument("--M", type=int, default=7)
    ap.add_argument("--K", type=int, default=10)
    ap.add_argument("--gamma", type=float, nargs=2, default=(1.0, 2.0))
    ap.add_argument("--frames", type=int, default=6)
    ap.add_argument("--db", default=DB_PATH)
    a = ap.parse_args()
    rec = tune(a.N, a.J, a.M, a.K, tuple(a.gamma), a.db, frames=a.frames)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
