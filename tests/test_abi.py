"""The C ABI: libcc.so builds for sm_103a, loads, and exports every entry
point include/*.h declares (no GPU needed: no compute call is made)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cc_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_1407_7105_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    need = {"cc_init", "cc_timestep_graph", "cc_components", "cc_kick", "cc_drift", "cc_evolve"}
    assert need <= _declared()


def test_library_exports_every_declared_symbol(built):
    from paper_1407_7105_gb300 import cc
    L = cc.lib()
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    assert set(cc.EXPORTS) == _declared()


def test_default_params_without_gpu(built):
    from paper_1407_7105_gb300 import cc
    p = cc.default_params()
    assert p.G == 1.0 and p.eta == 0.03 and p.max_depth == 64 and p.near_tol == 1e-12
    assert p.precision == cc.PREC_FP64


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of cc_params, cc_stats_t, cc_timing_t and
    cc_tune_entry_t have the C structs' sizes and field offsets (a host C
    program built against include/cc.h prints them)."""
    import ctypes as C
    import subprocess

    from paper_1407_7105_gb300 import cc
    structs = {"cc_params": cc.Params, "cc_stats_t": cc.Stats, "cc_timing_t": cc.Timing,
               "cc_tune_entry_t": cc.TuneEntry}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cc.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            a, b, c = ln.split()
            got[(a, b)] = int(c)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
