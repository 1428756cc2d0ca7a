"""GPU parity of nlinv_batch (independent frames in flight together, the
temporal decomposition of Sec. 3.3 / Eq. (10)) against the FP64 oracle and
against one-frame launches, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
import synth as S
from gpu_util import make_plan, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = 1e-3


def cart_frames(N, J, n, seed):
    return [S.cartesian_frame(N, J, seed=seed, sigma=1e-3, frame=f)[:2] for f in range(n)]


def test_batch_of_independent_frames_matches_oracle_and_single_launches():
    from paper_1701_08361_gb300 import nlinv as L
    N, J, B = 64, 4, 5
    g = O.Geometry(N=N, J=J)
    frames = cart_frames(N, J, B, seed=11)
    P = frames[0][1]
    plan = make_plan(N, J, psf=P, max_batch=8, exec_mode=2)   # single frames on the batch kernel's arithmetic
    # each frame starts from its own x_prev (frame 0 from the initial value)
    xps = [None] + [O.XVec(S.random_complex((N, N), 40 + f, 0.3) + 1.0,
                           S.random_complex((J, g.gc, g.gc), 50 + f, 20.0)) for f in range(1, B)]
    descs, outs = [], []
    for f, (Y, _) in enumerate(frames):
        xo = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
        img = torch.empty(N * N, dtype=torch.complex64, device="cuda")
        descs.append(dict(plan=plan, Y=to_dev(Y), turn=0,
                          x_prev=None if xps[f] is None else to_dev(xps[f].flat()),
                          x_out=xo, img_out=img))
        outs.append((xo, img))
    L.nlinv_batch(descs)
    assert L.nlinv_sync(plan) == 0
    for f, (Y, _) in enumerate(frames):
        x0 = O.XVec.initial(g) if xps[f] is None else xps[f]
        ref = O.nlinv_frame(Y, P, x0, x0, g, O.Params())
        assert rel(to_np(outs[f][0]), ref.flat()) <= TOL, f
        assert rel(to_np(outs[f][1]), O.image(ref, g)) <= TOL, f
        # the same frame alone
        xs = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
        L.nlinv_frame(plan, descs[f]["Y"], 0, descs[f]["x_prev"], xs)
        assert L.nlinv_sync(plan) == 0
        # the same arithmetic, but a batch group sums its CG inner products over
        # its own (fewer) CTAs: FP32 partial sums round differently, which 7 x 10
        # Newton/CG steps carry to ~1e-5..1e-4 (the bar against FP64 stays 1e-3)
        assert rel(to_np(outs[f][0]), to_np(xs)) <= 1e-4, f


def test_batch_mixes_grid_sizes_and_channel_counts():
    from paper_1701_08361_gb300 import nlinv as L
    specs = [(32, 3, 2), (64, 4, 3), (20, 2, 1)]
    plans, descs, refs = [], [], []
    for i, (N, J, nf) in enumerate(specs):
        g = O.Geometry(N=N, J=J)
        frames = cart_frames(N, J, nf, seed=100 + i)
        P = frames[0][1]
        plan = make_plan(N, J, psf=P, max_batch=nf, newton_steps=5, cg_iters=8)
        plans.append(plan)
        for f, (Y, _) in enumerate(frames):
            xo = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
            descs.append(dict(plan=plan, Y=to_dev(Y), turn=0, x_prev=None, x_out=xo))
            refs.append((g, O.nlinv_frame(Y, P, O.XVec.initial(g), O.XVec.initial(g), g,
                                          O.Params(newton_steps=5, cg_iters=8))))
    L.nlinv_batch(descs)
    for pl in plans:
        assert L.nlinv_sync(pl) == 0
    for d, (g, ref) in zip(descs, refs):
        assert rel(to_np(d["x_out"]), ref.flat()) <= TOL


def test_batch_graph_replays_new_inputs_frame_counts_and_alpha0():
    """The per-phase batch runs from CUDA graphs captured once per frame count
    (and again after nlinv_set_alpha0) that read the frames' pointers from a
    device table: replays with other inputs and outputs, another frame count
    and a changed alpha_0 all match the oracle."""
    from paper_1701_08361_gb300 import nlinv as L
    N, J, M, K = 32, 3, 3, 6
    g = O.Geometry(N=N, J=J)
    frames = cart_frames(N, J, 7, seed=300)
    P = frames[0][1]
    plan = make_plan(N, J, psf=P, max_batch=3, newton_steps=M, cg_iters=K)   # default: CUDA graph
    assert L.nlinv_plan_path(plan)[0] == 4

    def run(idx, alpha0):
        prm = O.Params(newton_steps=M, cg_iters=K, alpha0=alpha0)
        descs = []
        for f in idx:
            xo = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
            descs.append(dict(plan=plan, Y=to_dev(frames[f][0]), turn=0, x_prev=None, x_out=xo))
        L.nlinv_batch(descs)
        assert L.nlinv_sync(plan) == 0
        for f, d in zip(idx, descs):
            ref = O.nlinv_frame(frames[f][0], P, O.XVec.initial(g), O.XVec.initial(g), g, prm)
            assert rel(to_np(d["x_out"]), ref.flat()) <= TOL, (idx, f, alpha0)

    run([0, 1, 2], 1.0)      # captures the 3-frame sequence
    run([3, 4, 5], 1.0)      # replays it on other buffers
    run([6, 0], 1.0)         # a second graph (2 frames)
    L.nlinv_set_alpha0(plan, 0.5)
    run([1, 2, 3], 0.5)      # recaptured with the new alpha_n


# radial stream of the schedule tests: 8 frames N=128, 4 coils, 13 spokes,
# 5 turns; frames 0..2 in order, then 3 in flight (Eq. (10) with o = 3).  At
# N=64 the same trajectory sits on the FP32 floor of the 1e-3 bar (FP32
# operator rounding alone moves the FP64 trajectory by about 1e-3 there).
STREAM = dict(N=128, J=4, K=13, U=5, NF=8, D=3, WU=2)


def radial_stream_on_gpu(last_from_prev):
    """Run the stream through the scheduler; returns (GPU x^ per frame,
    oracle (Y, P) per frame, geometry)."""
    from paper_1701_08361_gb300 import nlinv as L
    from paper_1701_08361_gb300 import stream as ST
    N, J, K, U, NF, D, WU = (STREAM[k] for k in ("N", "J", "K", "U", "NF", "D", "WU"))
    g = O.Geometry(N=N, J=J)
    plan = make_plan(N, J, turns=U, max_batch=D)
    frames_o, Ys, turns = [], [], []
    coils = S.coil_maps(N, J, 9)
    for n in range(NF):
        kx, ky, y, _, _ = S.radial_frame(N, J, K, U, n, seed=9, coils=coils)
        frames_o.append((O.grid_data(kx, ky, y, N, g.G), O.psf_kernel(kx, ky, N, g.G).real))
        kxy = torch.tensor(np.stack([kx, ky], 1), dtype=torch.float64, device="cuda")
        if n < U:
            L.nlinv_psf(plan, n, kxy)
        Yd = torch.empty(J * g.G * g.G, dtype=torch.complex64, device="cuda")
        L.nlinv_grid(plan, kxy, to_dev(y), Yd)
        Ys.append(Yd)
        turns.append(n % U)
    xs = torch.empty((NF, plan.nx), dtype=torch.complex64, device="cuda")
    ST.run([dict(plan=plan, Y=Ys, turns=turns, delay=D, warmup=WU, x=xs, last_from_prev=last_from_prev)])
    assert L.nlinv_sync(plan) == 0
    return [to_np(xs[n]) for n in range(NF)], frames_o, g


def test_scheduled_radial_stream_matches_oracle_stream():
    """Each frame after the warm-up starts from, and is regularised towards,
    the most recent frame finished when its group starts."""
    xs, frames_o, g = radial_stream_on_gpu(False)
    ref = O.nlinv_stream(frames_o, g, O.Params(), delay=STREAM["D"], warmup=STREAM["WU"])
    for n, x in enumerate(xs):
        assert rel(x, ref[n].flat()) <= TOL, n


def test_stream_with_last_step_regularised_to_previous_frame():
    """Eq. (10) with its exception: the last Newton step of frame n is
    regularised towards x^_{n-1}; inside a launch that step waits for the
    frame before it (per-group barriers, device completion flags)."""
    xs, frames_o, g = radial_stream_on_gpu(True)
    kw = dict(delay=STREAM["D"], warmup=STREAM["WU"])
    ref = O.nlinv_stream(frames_o, g, O.Params(), last_from_prev=True, **kw)
    simp = O.nlinv_stream(frames_o, g, O.Params(), **kw)
    for n, x in enumerate(xs):
        assert rel(x, ref[n].flat()) <= TOL, n
    # the exception changes the frames it touches by more than the bar
    assert max(rel(ref[n].flat(), simp[n].flat()) for n in range(len(xs))) > 10 * TOL


def test_batch_rejects_reading_another_frames_output():
    from paper_1701_08361_gb300 import nlinv as L
    plan = make_plan(8, 2, psf=np.ones((16, 16)), max_batch=2)
    Y = torch.zeros(2 * 16 * 16, dtype=torch.complex64, device="cuda")
    xa = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    xb = torch.empty(plan.nx, dtype=torch.complex64, device="cuda")
    a = dict(plan=plan, Y=Y, turn=0, x_prev=None, x_out=xa)
    b = dict(plan=plan, Y=Y, turn=0, x_prev=None, x_out=xb)
    for frames in ([dict(a, x_last=xb), b],       # last step on a LATER frame
                   [a, dict(b, x_prev=xa)]):      # initial value from this call
        with pytest.raises(L.NlinvError) as e:
            L.nlinv_batch(frames)
        assert e.value.code == L.NLINV_EINVAL
    L.nlinv_batch([a, dict(b, x_last=xa)])        # an earlier frame: allowed
    assert L.nlinv_sync(plan) == 0


def test_batch_rejects_more_frames_than_the_plan_holds():
    from paper_1701_08361_gb300 import nlinv as L
    plan = make_plan(8, 2, psf=np.ones((16, 16)), max_batch=2)
    Y = torch.zeros(2 * 16 * 16, dtype=torch.complex64, device="cuda")
    frames = [dict(plan=plan, Y=Y, turn=0, x_prev=None,
                   x_out=torch.empty(plan.nx, dtype=torch.complex64, device="cuda")) for _ in range(3)]
    with pytest.raises(L.NlinvError) as e:
        L.nlinv_batch(frames)
    assert e.value.code == L.NLINV_EINVAL
    frames[0]["turn"] = 1
    with pytest.raises(L.NlinvError):
        L.nlinv_batch(frames[:2])
