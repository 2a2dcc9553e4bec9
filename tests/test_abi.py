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
