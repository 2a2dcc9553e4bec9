"""cc_components_noalloc: component labels with no device allocation.

The paper has no counterpart; the entry point exists for callers that
cannot let the library call cudaMalloc (their device memory belongs to
another allocator, or their loop cannot take cudaMalloc's device-wide
synchronisation).  Its scratch is one fixed device array shared by every
call, so these tests call it several times in a row (different sizes, then
the first input again) and require labels identical to the context-based
cc_components each time, and to the oracle's at the array's full size:
integer results, compared bit for bit.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_1407_7105_gb300 import ics

pytestmark = pytest.mark.gpu

CC_E_ARG, CC_E_CAPACITY = -1, -6


def _dev(*arrays):
    import torch
    return tuple(torch.tensor(a, device="cuda") for a in arrays)


def _reference(cclib, m, x, v, h):
    ctx = cclib.Context(m, x, v)
    lab, k = ctx.components(h)
    ctx.close()
    return lab, k


def _run(cclib, m, x, v, h, params=None):
    import torch
    n = m.shape[0]
    dm, dx, dv = _dev(m, x, v)
    labels = torch.full((n,), -5, dtype=torch.int32, device="cuda")
    ncomp = torch.full((1,), -5, dtype=torch.int64, device="cuda")
    cclib.components_noalloc(dm, dx, dv, h, labels, ncomp, params=params)
    return labels.cpu().numpy(), int(ncomp.item())


def test_noalloc_matches_cc_components_on_consecutive_calls(cclib, plummer_ic):
    cases = [(1000, 1.0 / 128), (4099, 1.0 / 256), (1000, 1.0 / 128)]
    for n, h in cases:
        m, x, v = plummer_ic(n, seed=7)
        lab, k = _run(cclib, m, x, v, h)
        ref, rk = _reference(cclib, m, x, v, h)
        assert k == rk
        assert np.array_equal(lab, ref)


def _separated_spheres(nsph=16, nper=4096, spacing=1000.0, hubble=0.1):
    """nsph Plummer spheres of nper bodies on a 4 x (nsph/4) grid, `spacing`
    apart, each moving with the bulk velocity hubble * (its centre): every
    pair of bodies from different spheres recedes."""
    ms, xs, vs, cen = [], [], [], []
    for k in range(nsph):
        m, x, v = ics.plummer(nper, seed=100 + k)
        X = spacing * np.array([k % 4, k // 4, 0.0])
        ms.append(m)
        xs.append(x + X[:, None])
        vs.append(v + hubble * X[:, None])
        cen.append(X)
    return (np.concatenate(ms), np.ascontiguousarray(np.concatenate(xs, axis=1)),
            np.ascontiguousarray(np.concatenate(vs, axis=1)), np.array(cen))


def _no_cross_edges(m, x, v, cen, nper, hubble, eta, h):
    """A proof, from the data, that no pair of bodies from different spheres
    is an edge at h, in either reading of the eta placement.  For spheres k,
    l with centre offset D, radii R (max |x - X|) and internal speeds w (max
    |v - V|), a cross pair has r >= |D| - R_k - R_l, |dv| <= hubble |D| + w_k
    + w_l and dx.dv >= hubble |D|^2 - |D| (hubble (R_k + R_l) + w_k + w_l) -
    (R_k + R_l)(w_k + w_l) > 0.  Receding (dx.dv > 0) makes both time
    derivatives >= 0, so each tau_x >= T_x, and tau >= eta min(sqrt(r^3/mu),
    r/|dv|) with mu <= 2 G max m."""
    nsph = cen.shape[0]
    R = np.zeros(nsph)
    w = np.zeros(nsph)
    for k in range(nsph):
        sl = slice(k * nper, (k + 1) * nper)
        R[k] = np.linalg.norm(x[:, sl] - cen[k][:, None], axis=0).max()
        w[k] = np.linalg.norm(v[:, sl] - hubble * cen[k][:, None], axis=0).max()
    mu = 2.0 * m.max()
    for k in range(nsph):
        for q in range(k + 1, nsph):
            D = np.linalg.norm(cen[k] - cen[q])
            rr, ww = R[k] + R[q], w[k] + w[q]
            rv_lo = hubble * D * D - D * (hubble * rr + ww) - rr * ww
            assert rv_lo > 0.0
            dmin, vmax = D - rr, hubble * D + ww
            tau_lo = eta * min(np.sqrt(dmin ** 3 / mu), dmin / vmax)
            assert tau_lo > 2.0 * h, (k, q, tau_lo)


@pytest.mark.parametrize("eta_outside", [0, 1])
def test_noalloc_matches_oracle_at_full_size(cclib, eta_outside):
    """n = CC_NOALLOC_MAX_N = 65536 in both readings of the eta placement:
    16 receding Plummer spheres, for which the test proves that no edge
    joins two spheres, so the oracle's labels of the whole state are its
    labels of each sphere (run on the full translated state, restricted to
    the sphere's ids).  Then a small call and the full-size call again:
    the array keeps no state that changes a result."""
    nper, hubble, eta, h = 4096, 0.1, 0.03, 1.0 / 256
    m, x, v, cen = _separated_spheres(nper=nper, hubble=hubble)
    n = m.shape[0]
    assert n == 65536
    _no_cross_edges(m, x, v, cen, nper, hubble, eta, h)
    s = O.State(m, x, v)
    op = O.params(eta=eta, eta_outside=bool(eta_outside))
    olab = np.zeros(n, dtype=np.int32)
    ok = 0
    for k in range(cen.shape[0]):
        ids = np.arange(k * nper, (k + 1) * nper, dtype=np.int32)
        lab_k, c_k = O.components(s, op, h, set_ids=ids)
        olab[k * nper:(k + 1) * nper] = lab_k
        ok += c_k
    p = cclib.default_params(eta=eta, eta_outside=eta_outside)
    lab, k = _run(cclib, m, x, v, h, params=p)
    assert k == ok and np.array_equal(lab, olab)
    sm, sx, sv = ics.plummer(300, seed=4)
    _run(cclib, sm, sx, sv, 1.0 / 64, params=p)
    lab2, k2 = _run(cclib, m, x, v, h, params=p)
    assert k2 == ok and np.array_equal(lab2, olab)


def test_noalloc_rejects_sizes_beyond_the_array(cclib):
    import torch
    n = 65537
    dm = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
    dx = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    labels = torch.zeros(n, dtype=torch.int32, device="cuda")
    ncomp = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(cclib.CCError) as e:
        cclib.components_noalloc(dm, dx, dx, 1.0 / 256, labels, ncomp)
    assert e.value.code == CC_E_CAPACITY


def test_noalloc_refuses_host_memory_and_bad_parameters(cclib, plummer_ic):
    """Pageable host memory is refused by the library before any launch
    (through the C ABI directly, past the binding's own checks), and so are
    parameters cc_init would refuse; the binding refuses wrong dtypes and
    short buffers."""
    import torch
    m, x, v = plummer_ic(256)
    n = 256
    lab_h = np.zeros(n, dtype=np.int32)
    nc_h = np.zeros(1, dtype=np.int64)
    p = cclib.default_params()
    L = cclib.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda a: C.c_void_p(a.ctypes.data)  # noqa: E731
    rc = L.cc_components_noalloc(ptr(m), ptr(x), ptr(v), n, C.byref(p), 1.0 / 64, ptr(lab_h), ptr(nc_h), stream)
    assert rc == CC_E_ARG
    dm, dx, dv = _dev(m, x, v)
    dlab = torch.zeros(n, dtype=torch.int32, device="cuda")
    dnc = torch.zeros(1, dtype=torch.int64, device="cuda")
    dptr = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    # device state, host outputs
    rc = L.cc_components_noalloc(dptr(dm), dptr(dx), dptr(dv), n, C.byref(p), 1.0 / 64, ptr(lab_h), ptr(nc_h),
                                 stream)
    assert rc == CC_E_ARG
    for bad in (dict(eta=0.0), dict(G=-1.0), dict(eps=float("nan")), dict(eta_outside=2)):
        rc = L.cc_components_noalloc(dptr(dm), dptr(dx), dptr(dv), n, C.byref(cclib.default_params(**bad)),
                                     1.0 / 64, dptr(dlab), dptr(dnc), stream)
        assert rc == CC_E_ARG, bad
    with pytest.raises(TypeError):
        cclib.components_noalloc(dm, dx, dv, 1.0 / 64, torch.zeros(n, dtype=torch.int64, device="cuda"), dnc)
    with pytest.raises(ValueError):
        cclib.components_noalloc(dm, dx, dv, 1.0 / 64, dlab[:100], dnc)
    with pytest.raises(TypeError):
        cclib.components_noalloc(dm, dx, dv, 1.0 / 64, lab_h, dnc)
    # and a good call right after the refusals
    cclib.components_noalloc(dm, dx, dv, 1.0 / 64, dlab, dnc)
    ref, rk = _reference(cclib, m, x, v, 1.0 / 64)
    assert int(dnc.item()) == rk and np.array_equal(dlab.cpu().numpy(), ref)
