"""cc_components_noalloc: component labels with no device allocation.

The paper has no counterpart; the entry point exists for callers that
cannot let the library call cudaMalloc (their device memory belongs to
another allocator, or their loop cannot take cudaMalloc's device-wide
synchronisation).  Its scratch is one fixed device array shared by every
call, so these tests call it twice in a row (different sizes, then the
first input again) and require labels identical to the context-based
cc_components each time: integer results, compared bit for bit.
This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(*arrays):
    import torch
    return tuple(torch.tensor(a, device="cuda") for a in arrays)


def _reference(cclib, m, x, v, h):
    ctx = cclib.Context(m, x, v)
    lab, k = ctx.components(h)
    ctx.close()
    return lab, k


def test_noalloc_matches_cc_components_on_consecutive_calls(cclib, plummer_ic):
    import torch
    cases = [(1000, 1.0 / 128), (4099, 1.0 / 256), (1000, 1.0 / 128)]
    for n, h in cases:
        m, x, v = plummer_ic(n, seed=7)
        dm, dx, dv = _dev(m, x, v)
        labels = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        ncomp = torch.full((1,), -5, dtype=torch.int64, device="cuda")
        cclib.components_noalloc(dm, dx, dv, h, labels, ncomp)
        ref, k = _reference(cclib, m, x, v, h)
        assert int(ncomp.item()) == k
        assert np.array_equal(labels.cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_the_array(cclib):
    import torch
    n = 65537
    dm = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    dx = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    labels = torch.zeros(n, dtype=torch.int32, device="cuda")
    ncomp = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(cclib.CCError) as e:
        cclib.components_noalloc(dm, dx, dx, 1.0 / 256, labels, ncomp)
    assert e.value.code == -6
