"""The C-ABI library loads, exports every entry point of include/nlinv.h and
rejects invalid plans on the host (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nlinv.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nlinv_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1701_08361_gb300 import nlinv as L
    if not os.path.exists(L.LIB_PATH):
        pytest.skip("libnlinv.so not built")
    return L.library()


def test_header_declares_the_hot_path_calls():
    names = declared()
    for n in ["nlinv_plan", "nlinv_apply_DF", "nlinv_apply_DFH", "nlinv_apply_normal",
              "nlinv_frame", "nlinv_psf", "nlinv_grid", "nlinv_sync", "nlinv_strerror"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared():
        assert hasattr(lib, n), n


def test_defaults_and_strerror(lib):
    from paper_1701_08361_gb300 import nlinv as L
    p = L.nlinv_default_params(160, 10)
    assert (p.N, p.J, p.Gc, p.newton_steps, p.cg_iters) == (160, 10, 0, 7, 10)
    assert (p.alpha0, p.q, p.damping, p.w_a, p.w_l) == (1.0, 0.5, 1.0, 220.0, 32.0)
    for code in range(0, -7, -1):
        assert L.nlinv_strerror(code)
    assert "unknown" in L.nlinv_strerror(-99)


@pytest.mark.parametrize("field,value,code", [
    ("N", 0, -1), ("N", 100, -6), ("Gc", 1, -1), ("Gc", 1000, -1), ("G", 300, -1), ("G", 500, -6),
    ("newton_steps", 0, -1), ("newton_steps", 33, -1), ("cg_iters", -1, -1),
    ("q", 1.5, -1), ("alpha0", 0.0, -1), ("n_turns", 0, -1), ("exec_mode", 5, -1), ("exec_mode", -1, -1),
])
def test_invalid_plans_are_rejected_on_host(lib, field, value, code):
    from paper_1701_08361_gb300 import nlinv as L
    p = L.nlinv_default_params(160, 10)
    setattr(p, field, value)
    h = ctypes.c_void_p()
    assert lib.nlinv_plan(ctypes.byref(h), ctypes.byref(p), None, None) == code
    assert not h.value


def test_null_arguments_are_rejected(lib):
    assert lib.nlinv_frame(None, None, 0, None, None, None, None, None) == -1
    assert lib.nlinv_apply_DF(None, None, None, None, None) == -1
    assert lib.nlinv_plan(None, None, None, None) == -1


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's nlinv_params_t, nlinv_frame_desc_t and nlinv_stream_desc_t have the C layout
    of include/nlinv.h: sizes and every field offset, from a C program
    compiled against the header (gcc, host only)."""
    import shutil
    import subprocess
    from paper_1701_08361_gb300 import nlinv as L
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"nlinv_params_t": L.nlinv_params_t, "nlinv_frame_desc_t": L.nlinv_frame_desc_t,
               "nlinv_stream_desc_t": L.nlinv_stream_desc_t}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nlinv.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'  printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for sname, cls in structs.items():
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)
