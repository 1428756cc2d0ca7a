"""The host scheduler of the temporal decomposition matches the oracle's
schedule and never reads a frame finished in the same launch (CPU only)."""
import oracle as O
from paper_1701_08361_gb300 import stream as ST


def test_sources_match_oracle():
    for D in (1, 2, 3, 11):
        for l in (0, 2, 5):
            for n in range(40):
                assert ST.source(n, D, l) == O.source_frame(n, D, l)


def test_groups_cover_frames_once_and_respect_dependencies():
    for D in (1, 3, 10, 11):
        for l in (0, 5):
            for nf in (1, 7, 32, 60):
                gs = ST.groups(nf, D, l)
                flat = [n for g in gs for n in g]
                assert flat == list(range(nf))
                done = set()
                for g in gs:
                    assert len(g) <= max(D, 1)
                    for n in g:
                        s = ST.source(n, D, l)
                        assert s < 0 or s in done
                    done.update(g)


def test_run_passes_the_last_step_regulariser(monkeypatch):
    """With last_from_prev, every frame whose source is not n - 1 gets
    x_last = x^_{n-1}, which is then either a finished frame of an earlier
    launch or an EARLIER frame of the same launch (the only in-call reference
    the library accepts); x_prev never refers to the same launch."""
    from paper_1701_08361_gb300 import nlinv as L
    calls = []
    monkeypatch.setattr(L, "nlinv_batch", lambda frames, stream=None: calls.append(frames))
    NF, D, WU = 14, 3, 2
    xs = [f"x{n}" for n in range(NF)]        # stand-ins for the output buffers
    ST.run([dict(plan="P", Y=[None] * NF, turns=[0] * NF, delay=D, warmup=WU, x=xs,
                 last_from_prev=True)])
    assert [len(c) for c in calls] == [len(g) for g in ST.groups(NF, D, WU)]
    done = set()
    for frames in calls:
        outs = [f["x_out"] for f in frames]
        for i, f in enumerate(frames):
            n = xs.index(f["x_out"])
            s = ST.source(n, D, WU)
            assert f["x_prev"] == (None if s < 0 else xs[s]) and f["x_prev"] not in outs
            if s == n - 1:
                assert f["x_last"] is None
            else:
                assert f["x_last"] == xs[n - 1]
                assert f["x_last"] in done or f["x_last"] in outs[:i]
        done.update(outs)
    # without the option nothing changes
    calls.clear()
    ST.run([dict(plan="P", Y=[None] * NF, turns=[0] * NF, delay=D, warmup=WU, x=xs)])
    assert all(f["x_last"] is None for c in calls for f in c)
