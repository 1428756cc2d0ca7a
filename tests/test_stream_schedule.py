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
