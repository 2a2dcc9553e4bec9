"""The cheap "certainly apart" test of the mixed tau kernel (tau_quick_apart
in csrc/cc_device.cuh), restated in numpy float32 and checked against the
oracle's FP64 tau: a pair it certifies must have tau >= h, on random pairs
and on pairs built near the threshold (slow approaching pairs, grazing
fly-bys, pairs at tau within a few per mille of h, both eta readings).  The
float32 reciprocal square root here is correctly rounded; the kernel's is
within 2 ulp, which the test's 2 % margin covers with room to spare."""
import numpy as np
import pytest

from oracle import oracle as O

f32 = np.float32


def quick_apart(dx, dv, mu, eta_in, etah, c_x=0.0, c_v=0.0, eps2=0.0):
    dx = dx.astype(f32)
    dv = dv.astype(f32)
    r2 = (dx[2] * dx[2] + (dx[1] * dx[1] + (dx[0] * dx[0] + f32(eps2)))).astype(f32)
    v2 = (dv[2] * dv[2] + (dv[1] * dv[1] + dv[0] * dv[0])).astype(f32)
    with np.errstate(all="ignore"):
        rinv = (f32(1) / np.sqrt(r2)).astype(f32)
        r = (r2 * rinv).astype(f32)
        s1 = (f32(1) / np.sqrt((r * f32(mu)).astype(f32))).astype(f32)
        s2 = (f32(1) / np.sqrt(v2)).astype(f32)
        vn = (v2 * s2).astype(f32)
        Tff = (f32(etah) * r2 * s1).astype(f32)
        q = (f32(eta_in) * vn * rinv / f32(etah)).astype(f32)
        Tfb = (f32(etah) * r * s2).astype(f32)
        g = (f32(mu) * rinv * s2 * s2).astype(f32)
        M = f32(1.02)
        return ((f32(c_x) * rinv <= f32(0.99e-4)) & (v2 > 0) & (f32(c_v) * s2 <= f32(0.99e-4)) &
                (f32(0.75) * M * q < 1) & (Tff * (f32(1) - f32(0.75) * M * q) >= M) &
                (Tfb >= M * (f32(1) + f32(0.5) * f32(eta_in) * (f32(1) + g))))


def oracle_tau(dx, dv, mi, mj, eta, eta_outside):
    p = O.params(eta=eta, eta_outside=eta_outside)
    out = np.empty(dx.shape[1])
    for k in range(dx.shape[1]):
        out[k] = O.tau_parts(np.zeros(3), np.zeros(3), mi, -dx[:, k], -dv[:, k], mj, p)[0]
    return out


def check(dx, dv, mi, mj, eta, h, eta_outside):
    eta_in = 1.0 if eta_outside else eta
    etah = (eta_in * eta / h) if eta_outside else eta / h
    mu = mi + mj
    ok = quick_apart(dx, dv, mu, eta_in, etah)
    tau = oracle_tau(dx[:, ok], dv[:, ok], mi, mj, eta, eta_outside)
    assert np.all(tau >= h), (tau.min(), h)
    return ok.mean()


@pytest.mark.parametrize("eta_outside", [0, 1])
def test_random_pairs(eta_outside):
    rng = np.random.default_rng(5 + eta_outside)
    n = 20000
    dx = rng.standard_normal((3, n)) * np.exp(rng.uniform(-6, 1, n))
    dv = rng.standard_normal((3, n)) * np.exp(rng.uniform(-6, 1, n))
    frac = check(dx, dv, 1e-4, 2e-4, 0.03, 1 / 256, eta_outside)
    assert frac > 0.3  # the test settles a good share of them


@pytest.mark.parametrize("eta_outside", [0, 1])
def test_pairs_near_threshold(eta_outside):
    """Pairs whose tau is within a few per mille of h, or approaching slowly
    (dT/dt strongly negative), are the ones a loose bound could misjudge."""
    rng = np.random.default_rng(11 + eta_outside)
    eta, mi, mj = 0.03, 1e-4, 1e-4
    n = 6000
    dx = rng.standard_normal((3, n)) * np.exp(rng.uniform(-5, 0, n))
    dv = rng.standard_normal((3, n)) * np.exp(rng.uniform(-7, 1, n))
    # make half of them approach head-on (rv < 0, |rv| = r |dv|)
    dv[:, ::2] = -dx[:, ::2] / np.linalg.norm(dx[:, ::2], axis=0) * np.linalg.norm(dv[:, ::2], axis=0)
    tau = oracle_tau(dx, dv, mi, mj, eta, eta_outside)
    eta_in = 1.0 if eta_outside else eta
    # thresholds just above each pair's tau (an edge: the test must not
    # certify it) and just below (not an edge: either answer is allowed)
    for rel in (0.5, 0.9, 0.99, 0.995, 0.998, 0.9995, 1.0005, 1.002, 1.01):
        h = tau / rel
        etah = (eta_in * eta / h) if eta_outside else eta / h
        for k in range(0, n, 7):
            ok = quick_apart(dx[:, k:k + 1], dv[:, k:k + 1], mi + mj, eta_in, etah[k])[0]
            if rel < 1.0:
                assert not ok, (k, rel, tau[k])


@pytest.mark.parametrize("X", [1.0, 30.0, 1000.0])
def test_high_part_differences(X):
    """The kernel forms the test's differences from the rounded high parts
    alone, fl32(x_j) - fl32(x_i), and passes c_x = 7.1 u max|x_i| per pair
    (likewise for v): bodies far from the origin, at separations down to
    where that rounding matters, with thresholds placed just above each
    pair's tau."""
    rng = np.random.default_rng(int(X))
    n = 4000
    u = 2.0 ** -24
    xi = rng.uniform(-X, X, (3, n))
    sep = rng.standard_normal((3, n)) * np.exp(rng.uniform(np.log(X) - 18, np.log(X), n))
    xj = xi + sep
    vi = rng.standard_normal((3, n))
    vj = vi + rng.standard_normal((3, n)) * np.exp(rng.uniform(-8, 0, n))
    dxh = xj.astype(f32) - xi.astype(f32)
    dvh = vj.astype(f32) - vi.astype(f32)
    mi = mj = 1e-4
    eta = 0.03
    tau = oracle_tau(xi - xj, vi - vj, mi, mj, eta, 0)
    for rel in (0.5, 0.98, 0.999):
        h = tau / rel  # every pair an edge: none may be certified apart
        ok = quick_apart(dxh, dvh, mi + mj, eta, eta / h, c_x=7.1 * u * np.abs(xi.astype(f32)).max(axis=0),
                         c_v=7.1 * u * np.abs(vi.astype(f32)).max(axis=0))
        assert not ok.any(), (rel, np.flatnonzero(ok)[:5])
