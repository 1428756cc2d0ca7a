"""Host logic of the autotuner's compile-time sweep (CPU only): the variant
list changes one knob at a time from the compiled grid, every grid the
library compiles passes the fit check that mirrors the Cfg static_asserts,
and every variant's build command carries its flags and only its grid."""
import pytest

from paper_1701_08361_gb300 import build as B
from paper_1701_08361_gb300 import tune as T


def test_every_compiled_grid_fits():
    for g in B.grid_sizes():
        assert T._fits(*g), g


def test_fit_check_rejects_what_cfg_rejects():
    assert not T._fits(16, 20, 160, 6, 1)          # TW not a multiple of 4
    assert not T._fits(16, 32, 256, 64, 1)         # 2048 threads
    assert not T._fits(16, 32, 256, 32, 1)         # shared memory over 227 KB
    assert not T._fits(16, 20, 161, 12, 1)         # FOV over half the grid


@pytest.mark.parametrize("N", [160, 256, 64])
def test_variants_change_one_knob(N):
    vs = T.compile_variants(N)
    base = vs[0]
    assert base["knobs"] == {k: T.built_in_knob(k) for k in T.KNOBS}
    assert base["grid"] in B.grid_sizes()
    names = [v["name"] for v in vs]
    assert len(set(names)) == len(names)
    for v in vs[1:]:
        diff = (v["grid"][3] != base["grid"][3]) + sum(v["knobs"][k] != base["knobs"][k] for k in T.KNOBS)
        assert diff == 1, v
        assert v["grid"][:3] == base["grid"][:3] and v["grid"][4] == base["grid"][4]


def test_variant_build_commands(tmp_path):
    v = T.compile_variants(160)[1]
    jobs = B.units(v["flags"], [v["grid"]], str(tmp_path))
    assert len(jobs) == 2                          # the host unit and this grid's unit
    for obj, cmd in jobs:
        assert obj.startswith(str(tmp_path))
        for f in v["flags"]:
            assert f in cmd
    g1, g2, n, tw, mb = v["grid"]
    grid_cmd = jobs[1][1]
    assert f"-DNLINV_TWU={tw}" in grid_cmd and f"-DNLINV_G1={g1}" in grid_cmd and f"-DNLINV_NR={n}" in grid_cmd
