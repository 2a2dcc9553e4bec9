"""The group certificate of the mixed tau kernel (tau_groups_apart and
warp_group_box in csrc/cc_device.cuh / cc_mixed.cu), restated in numpy
float32 and checked against the oracle's FP64 tau: when it certifies two
groups of 32 bodies, every cross pair whose high-part velocity difference
passes the returned threshold must have tau >= h.  Cases: random groups at
many separations and scales, head-on approaching groups with the threshold
swept through the exact tau (the free-fall bound is tight there), slow
approaching pairs around the flyby's lower speed root, softening, and both
readings of the eta placement."""
import numpy as np
import pytest

from oracle import oracle as O

f32 = np.float32
U32 = f32(2.0 ** -24)


def box(x, v, gm):
    """warp_group_box: boxes of the high parts and the largest G m."""
    xh, vh = x.astype(f32), v.astype(f32)
    b = dict(xlo=xh.min(1), xhi=xh.max(1), vlo=vh.min(1), vhi=vh.max(1), gm=f32(gm.astype(f32).max()))
    b["amax"] = f32(max(np.abs(b["xlo"]).max(), np.abs(b["xhi"]).max()))
    b["vabs"] = f32(max(np.abs(b["vlo"]).max(), np.abs(b["vhi"]).max()))
    return b


def groups_apart(A, B, eta_in, etah, hq, eps2=0.0):
    """tau_groups_apart: (certified, vthr2), float32 step by step."""
    M = f32(1.02)
    pad_x = f32(4) * U32 * max(A["amax"], B["amax"])
    pad_v = f32(4) * U32 * max(A["vabs"], B["vabs"])
    d2, w2 = f32(eps2), f32(0)
    for k in range(3):
        g = max(f32(0), f32(max(f32(B["xlo"][k] - A["xhi"][k]), f32(A["xlo"][k] - B["xhi"][k])) - pad_x))
        w = f32(max(f32(0), max(f32(B["vhi"][k] - A["vlo"][k]), f32(A["vhi"][k] - B["vlo"][k]))) + pad_v)
        d2 = f32(g * g + d2)
        w2 = f32(w * w + w2)
    d, vmax = f32(np.sqrt(d2)), f32(np.sqrt(w2))
    mu = f32(f32(A["gm"] + B["gm"]) * f32(1.0001))
    if not (d > 0 and mu > 0):
        return False, 0.0
    X = f32(f32(f32(etah) * d) * f32(np.sqrt(f32(d / mu))))
    q = f32(f32(f32(hq) * vmax) / d)
    if not (f32(X * f32(f32(1) - f32(f32(0.75) * M) * q)) >= M):
        return False, 0.0
    a = f32(f32(M * f32(f32(2) + f32(eta_in))) * d)
    b = f32(f32(f32(2) * f32(etah)) * d2)
    c = f32(f32(M * f32(eta_in)) * mu)
    disc = f32(b * b - f32(f32(4) * a) * c)
    if not disc > 0:
        return False, 0.0
    vp = f32(f32(b + f32(np.sqrt(disc))) / f32(f32(2) * a))
    vm = f32(c / f32(a * vp))
    if not vmax <= f32(vp * f32(0.9999)):
        return False, 0.0
    vt = f32(f32(vm * f32(1.0001)) + f32(f32(4) * pad_v))
    return True, float(f32(vt * vt))


def readings(eta, h, eta_outside):
    eta_in = 1.0 if eta_outside else eta
    etah = eta_in * eta / h if eta_outside else eta / h
    return eta_in, etah, eta_in / etah


def check_groups(xa, va, ma, xb, vb, mb, eta, h, eta_outside=0, eps=0.0):
    """Certify the two groups; if certified, every passing pair has tau >= h.
    Returns (certified, passing pairs)."""
    G = 1.0
    eta_in, etah, hq = readings(eta, h, eta_outside)
    A, B = box(xa, va, G * ma), box(xb, vb, G * mb)
    ok, thr = groups_apart(A, B, eta_in, etah, hq, eps * eps)
    if not ok:
        return False, 0
    dvh = vb.astype(f32)[:, None, :] - va.astype(f32)[:, :, None]
    v2 = (dvh[2] * dvh[2] + (dvh[1] * dvh[1] + dvh[0] * dvh[0])).astype(f32)
    s = O.State(np.concatenate([ma, mb]), np.concatenate([xa, xb], axis=1), np.concatenate([va, vb], axis=1))
    p = O.params(eta=eta, eps=eps, eta_outside=bool(eta_outside))
    na = ma.shape[0]
    npass = 0
    for i in range(na):
        for j in range(mb.shape[0]):
            if v2[i, j] >= thr:
                npass += 1
                t = O.tau_ids(s, p, i, na + j)
                assert t >= h, (t, h, i, j)
    return True, npass


@pytest.mark.parametrize("eta_outside", [0, 1])
def test_random_groups(eta_outside):
    rng = np.random.default_rng(11 + eta_outside)
    certified = 0
    for case in range(60):
        scale = np.exp(rng.uniform(-3, 3))
        sep = scale * np.exp(rng.uniform(-1, 3))
        spread = scale * np.exp(rng.uniform(-4, 0))
        vs = np.sqrt(1.0 / scale) * np.exp(rng.uniform(-3, 1))
        m = np.full(32, 1.0 / 16384) * np.exp(rng.uniform(-2, 2, 32))
        off = rng.standard_normal(3)
        off *= sep / np.linalg.norm(off)
        xa = rng.standard_normal((3, 32)) * spread + rng.standard_normal((3, 1)) * 10 * scale
        xb = xa[:, :1] + off[:, None] + rng.standard_normal((3, 32)) * spread
        va = rng.standard_normal((3, 32)) * vs
        vb = rng.standard_normal((3, 32)) * vs
        h = 2.0 ** -rng.integers(4, 12)
        ok, _ = check_groups(xa, va, m, xb, vb, m[::-1].copy(), 0.03, h, eta_outside)
        certified += ok
    assert certified >= 10  # the test exercises the certified branch


@pytest.mark.parametrize("eta_outside", [0, 1])
def test_head_on_groups_at_the_threshold(eta_outside):
    """Two clumps approaching head on: the free-fall bound is attained (r =
    d, rv = -r v), so thresholds swept through the pair's tau probe the
    margin; a certificate above tau would fail."""
    rng = np.random.default_rng(3)
    tight = 0
    for d, w in ((0.5, 0.05), (1.0, 0.2), (2.0, 0.02), (0.05, 0.001)):
        xa = np.zeros((3, 32)) + rng.standard_normal((3, 32)) * 1e-12
        xb = xa.copy()
        xb[0] += d
        va = np.zeros((3, 32))
        va[0] = w
        vb = -va
        m = np.full(32, 1e-4)
        s = O.State(np.array([1e-4, 1e-4]), np.array([[0.0, d], [0, 0], [0, 0]]),
                    np.array([[w, -w], [0, 0], [0, 0]]))
        tau = O.tau_ids(s, O.params(eta=0.03, eta_outside=bool(eta_outside)), 0, 1)
        for rel in (0.9, 0.97, 0.985, 0.995, 1.0, 1.005, 1.05):
            # above tau (rel > 1) a passing pair fails check_groups' assertion
            ok, npass = check_groups(xa, va, m, xb, vb, m, 0.03, tau * rel, eta_outside)
            tight += rel <= 0.97 and npass > 0
    assert tight > 0  # certified within 3 % of tau somewhere: the margin is not vacuous


def test_slow_pairs_below_the_lower_root():
    """Nearly equal velocities: tau_fb -> 0 as |dv| -> 0 for approaching
    bodies, so pairs slower than the lower root must fail the per-pair
    threshold; pairs passing it are checked against the oracle."""
    rng = np.random.default_rng(7)
    m = np.full(32, 1e-3)
    npass_total = 0
    for case in range(20):
        xa = rng.standard_normal((3, 32)) * 0.01
        xb = xa + np.array([[1.0], [0.0], [0.0]])
        base = rng.standard_normal((3, 1)) * 0.3
        va = base + rng.standard_normal((3, 32)) * 10.0 ** rng.uniform(-9, -3)
        vb = base - np.array([[1.0], [0], [0]]) * 10.0 ** rng.uniform(-8, -4) + \
            rng.standard_normal((3, 32)) * 10.0 ** rng.uniform(-9, -4)
        ok, npass = check_groups(xa, va, m, xb, vb, m, 0.03, 1 / 64)
        npass_total += npass
    assert npass_total > 0


def test_softened_groups():
    rng = np.random.default_rng(9)
    for case in range(20):
        eps = 10.0 ** rng.uniform(-3, -1)
        xa = rng.standard_normal((3, 32)) * 0.02
        xb = xa + rng.standard_normal((3, 1)) * 0.5
        va = rng.standard_normal((3, 32)) * 0.3
        vb = rng.standard_normal((3, 32)) * 0.3
        m = np.full(32, 1.0 / 4096)
        check_groups(xa, va, m, xb, vb, m, 0.03, 1 / 256, 0, eps)


def test_a_dropped_speed_threshold_is_caught():
    """Planted mistake: a certificate that drops the per-pair lower speed
    root (every pair passing) lets slow approaching pairs, which are edges,
    through; check_groups must reject it on the slow-pair cases."""
    global groups_apart
    keep = groups_apart

    def weak(A, B, eta_in, etah, hq, eps2=0.0):
        ok, _ = keep(A, B, eta_in, etah, hq, eps2)
        return ok, 0.0

    groups_apart = weak
    try:
        with pytest.raises(AssertionError):
            test_slow_pairs_below_the_lower_root()
    finally:
        groups_apart = keep
