"""Seeded synthetic initial conditions in N-body units (G = M = 1).

This module is the only code shared by the CUDA path and the CPU oracle:
it draws particle states and holds none of the integrator's arithmetic.
Random numbers come from a counter-based SplitMix64 generator (Steele,
Lea & Flood 2014): for seed q and stream s the key is
b = (q << 32) xor (s * 0x51ED27 mod 2^32), and draw k is
mix64(mix64(b + 1) + (k + 1) * 0x9E3779B97F4A7C15) with SplitMix64's
finaliser mix64, so every draw is reproducible element by element,
independent of the order in which draws are made.

Every generator returns ``(m, x3, v3)``: float64 arrays of shapes (n,),
(3, n), (3, n), C-contiguous, in the centre-of-mass frame unless stated.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _u64(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 output for counter ``idx`` of (seed, stream)."""
    base = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)) ^ np.uint64((stream * 0x51ED27) & 0xFFFFFFFF)
    with np.errstate(over="ignore"):
        z = _mix64(base + np.uint64(1)) + (idx.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        return _mix64(z)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) with 53 random bits, counters offset..offset+n-1."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    return (_u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _isotropic(seed: int, stream: int, n: int, radius: np.ndarray) -> np.ndarray:
    u = uniform(seed, stream, 2 * n)
    cth = 2.0 * u[:n] - 1.0
    phi = 2.0 * math.pi * u[n:]
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([radius * sth * np.cos(phi), radius * sth * np.sin(phi), radius * cth])


def _com_frame(m, x3, v3):
    M = m.sum()
    x3 = x3 - (x3 * m).sum(axis=1, keepdims=True) / M
    v3 = v3 - (v3 * m).sum(axis=1, keepdims=True) / M
    return np.ascontiguousarray(x3), np.ascontiguousarray(v3)


def potential_energy(m, x3, eps: float = 0.0, chunk: int = 2048) -> float:
    """Exact pairwise potential energy (used only to scale initial conditions)."""
    n = m.shape[0]
    W = 0.0
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d = x3[:, s:e, None] - x3[:, None, :]
        r = np.sqrt((d * d).sum(axis=0) + eps * eps)
        mm = m[s:e, None] * m[None, :]
        ii = np.arange(s, e)[:, None]
        jj = np.arange(n)[None, :]
        W -= (mm / np.where(jj > ii, r, np.inf)).sum()
    return float(W)


def scale_to_nbody_units(m, x3, v3, Q: float = 0.5, eps: float = 0.0, exact: bool = True,
                         W: float | None = None):
    """Rescale velocities to virial ratio Q = T/|W| and lengths so E = -1/4."""
    T = 0.5 * float((m * (v3 * v3).sum(axis=0)).sum())
    if W is None:
        W = potential_energy(m, x3, eps) if exact else -3.0 * math.pi / 32.0
    if T > 0.0:
        v3 = v3 * math.sqrt(Q * abs(W) / T)
    E = Q * abs(W) - abs(W)
    beta = E / -0.25
    return np.ascontiguousarray(x3 * beta), np.ascontiguousarray(v3 / math.sqrt(beta))


def plummer(n: int, seed: int = 1, Q: float = 0.5, exact_scale: bool | None = None):
    """Equal-mass Plummer sphere (Aarseth, Henon & Wielen 1974 sampling).

    Radii from the inverted cumulative mass with the outermost 0.1 % of the
    mass excluded; speeds by von Neumann rejection on q^2 (1-q^2)^{7/2};
    isotropic directions; then virial ratio Q and E = -1/4.
    """
    m = np.full(n, 1.0 / n)
    X = 1e-10 + (0.999 - 1e-10) * uniform(seed, 1, n)
    r = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    x3 = _isotropic(seed, 2, n, r)
    q = np.full(n, -1.0)
    todo = np.arange(n)
    k = 0
    while todo.size:
        a = uniform(seed, 3 + 2 * k, n)[todo]
        b = uniform(seed, 4 + 2 * k, n)[todo]
        ok = 0.1 * b < a * a * (1.0 - a * a) ** 3.5
        q[todo[ok]] = a[ok]
        todo = todo[~ok]
        k += 1
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** -0.25
    v3 = _isotropic(seed, 1000, n, q * vesc)
    x3 = x3 * (3.0 * math.pi / 16.0)
    v3 = v3 * math.sqrt(16.0 / (3.0 * math.pi))
    x3, v3 = _com_frame(m, x3, v3)
    if exact_scale is None:
        exact_scale = n <= 20000
    x3, v3 = scale_to_nbody_units(m, x3, v3, Q=Q, exact=exact_scale)
    return m, x3, v3


def orbit_state(m1: float, m2: float, a: float, e: float, E_anom: float,
                inc: float = 0.0, node: float = 0.0, peri: float = 0.0, G: float = 1.0):
    """Relative state (r, v) of particle 1 minus particle 2 on a bound orbit
    with semi-major axis a, eccentricity e, eccentric anomaly E_anom and
    orientation angles (inclination, node, argument of pericentre)."""
    mu = G * (m1 + m2)
    n = math.sqrt(mu / a ** 3)
    cE, sE = math.cos(E_anom), math.sin(E_anom)
    fac = math.sqrt(1.0 - e * e)
    den = 1.0 - e * cE
    p = np.array([a * (cE - e), a * fac * sE, 0.0])
    w = np.array([-a * n * sE / den, a * n * fac * cE / den, 0.0])
    ci, si = math.cos(inc), math.sin(inc)
    cO, sO = math.cos(node), math.sin(node)
    cw, sw = math.cos(peri), math.sin(peri)
    R = np.array([
        [cO * cw - sO * sw * ci, -cO * sw - sO * cw * ci, sO * si],
        [sO * cw + cO * sw * ci, -sO * sw + cO * cw * ci, -cO * si],
        [sw * si, cw * si, ci],
    ])
    return R @ p, R @ w


def binary(m1: float, m2: float, a: float, e: float, E_anom: float = 0.0, **kw):
    """Two-body system in its centre-of-mass frame (for the Kepler tests)."""
    r, v = orbit_state(m1, m2, a, e, E_anom, **kw)
    M = m1 + m2
    x3 = np.stack([m2 / M * r, -m1 / M * r], axis=1)
    v3 = np.stack([m2 / M * v, -m1 / M * v], axis=1)
    return np.array([m1, m2]), np.ascontiguousarray(x3), np.ascontiguousarray(v3)


def _mean_anomaly_E(seed: int, stream: int, e: np.ndarray) -> np.ndarray:
    """Eccentric anomalies distributed as a uniform mean anomaly
    (density proportional to 1 - e cos E), by rejection."""
    n = e.shape[0]
    out = np.zeros(n)
    todo = np.arange(n)
    k = 0
    while todo.size:
        E = 2.0 * math.pi * uniform(seed, stream + 2 * k, n)[todo]
        u = uniform(seed, stream + 2 * k + 1, n)[todo]
        ok = u * (1.0 + e[todo]) < 1.0 - e[todo] * np.cos(E)
        out[todo[ok]] = E[ok]
        todo = todo[~ok]
        k += 1
    return out


def plummer_with_binaries(n: int, seed: int = 1, binary_fraction: float = 0.5,
                          a_min: float = 1e-5, a_max: float = 1e-2):
    """Plummer sphere in which a fraction of the particles are members of
    primordial binaries: n_b = binary_fraction * n / 2 binaries and
    n - 2 n_b single stars, n_b + n_s equal-mass Plummer systems.  Binary
    semi-major axes log-uniform in [a_min, a_max], thermal eccentricities
    f(e) = 2e, isotropic orientations, uniform mean anomaly, mass ratio
    q ~ U(0.1, 1]; the system mass splits as M/(1+q), qM/(1+q)."""
    nb = int(round(binary_fraction * n / 2))
    ns = n - 2 * nb
    nsys = nb + ns
    ms, xs, vs = plummer(nsys, seed=seed, exact_scale=nsys <= 20000)
    u = uniform(seed, 5000, 6 * nb).reshape(6, nb)
    a = np.exp(np.log(a_min) + (np.log(a_max) - np.log(a_min)) * u[0])
    e = np.sqrt(u[1])
    q = 0.1 + 0.9 * (1.0 - u[2])
    cinc = 2.0 * u[3] - 1.0
    node = 2.0 * math.pi * u[4]
    peri = 2.0 * math.pi * u[5]
    Ean = _mean_anomaly_E(seed, 6000, e)
    m = np.zeros(n)
    x3 = np.zeros((3, n))
    v3 = np.zeros((3, n))
    for b in range(nb):
        M = ms[b]
        m1, m2 = M / (1.0 + q[b]), q[b] * M / (1.0 + q[b])
        r, v = orbit_state(m1, m2, a[b], e[b], Ean[b], inc=math.acos(cinc[b]),
                           node=node[b], peri=peri[b])
        m[2 * b], m[2 * b + 1] = m1, m2
        x3[:, 2 * b] = xs[:, b] + m2 / M * r
        x3[:, 2 * b + 1] = xs[:, b] - m1 / M * r
        v3[:, 2 * b] = vs[:, b] + m2 / M * v
        v3[:, 2 * b + 1] = vs[:, b] - m1 / M * v
    m[2 * nb:] = ms[nb:]
    x3[:, 2 * nb:] = xs[:, nb:]
    v3[:, 2 * nb:] = vs[:, nb:]
    x3, v3 = _com_frame(m, x3, v3)
    return m, x3, v3


def salpeter_masses(n: int, seed: int, stream: int, lo: float = 0.1, hi: float = 100.0,
                    slope: float = 2.35) -> np.ndarray:
    """Masses with dN/dm ~ m^-slope on [lo, hi], rescaled to total mass 1."""
    u = uniform(seed, stream, n)
    k = 1.0 - slope
    mm = (lo ** k + u * (hi ** k - lo ** k)) ** (1.0 / k)
    return mm / mm.sum()


def _gauss(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal deviates (Box-Muller on two uniform streams)."""
    u1 = uniform(seed, stream, n)
    u2 = uniform(seed, stream + 1, n)
    return np.sqrt(-2.0 * np.log(1.0 - u1)) * np.cos(2.0 * math.pi * u2)


def box_fractal_raw(n: int, seed: int = 1, D: float = 1.6, max_gen: int = 16):
    """Unscaled box fractal in the manner of Goodwin & Whitworth (2004).

    A cube of side 2 centred on the origin holds the first parent.  Each
    generation halves the cell size: every parent gets 2^3 children at the
    centres of its sub-cubes, displaced by uniform noise of a tenth of the
    new cell size; a child survives as a parent of the next generation with
    probability 2^(D-3).  Velocities: the first generation draws a Gaussian
    velocity, every later child inherits its parent's velocity plus a
    Gaussian component whose scale halves each generation (correlated
    clump velocities).  Generations continue until the children inside the
    unit sphere number at least 1.5 n; n of them are drawn at random.
    Returns positions (3, n) and velocities (3, n), not yet scaled."""
    offs = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)], dtype=float)
    keep = 2.0 ** (D - 3.0)
    for attempt in range(50):
        pos = np.zeros((1, 3))
        vel = np.zeros((1, 3))
        side = 2.0
        leaves = None
        for gen in range(1, max_gen + 1):
            side *= 0.5
            child = (pos[:, None, :] + 0.5 * side * offs[None, :, :]).reshape(-1, 3)
            cvel = np.repeat(vel, 8, axis=0)
            nc = child.shape[0]
            st = 100 * attempt + 10 * gen
            jit = np.stack([uniform(seed, st + q, nc) for q in range(3)], axis=1) - 0.5
            child = child + 0.1 * side * jit
            g = np.stack([_gauss(seed, 5000 + st + 2 * q, nc) for q in range(3)], axis=1)
            cvel = cvel + (0.5 ** (gen - 1)) * g
            inside = (child * child).sum(axis=1) < 1.0
            if inside.sum() >= 1.5 * n:
                leaves = (child[inside], cvel[inside])
                break
            alive = uniform(seed, 9000 + st, nc) < keep if gen > 1 else np.ones(nc, dtype=bool)
            if not alive.any():
                break
            pos, vel = child[alive], cvel[alive]
        if leaves is not None:
            pick = np.argsort(uniform(seed, 777 + attempt, leaves[0].shape[0]), kind="stable")[:n]
            return np.ascontiguousarray(leaves[0][pick].T), np.ascontiguousarray(leaves[1][pick].T)
    raise ValueError("box fractal: branching process died out repeatedly")


def box_fractal(n: int, seed: int = 1, D: float = 1.6, Q: float = 0.3, imf: bool = True,
                W: float | None = None):
    """Box-fractal cluster (Goodwin & Whitworth 2004 recipe, box_fractal_raw)
    with Salpeter masses (0.1-100, total 1) in the centre-of-mass frame,
    scaled to virial ratio Q and E = -1/4.  W, the potential energy of the
    unscaled configuration with these masses, may be passed in (computed
    elsewhere for large n); otherwise it is summed exactly here."""
    x3, v3 = box_fractal_raw(n, seed=seed, D=D)
    m = salpeter_masses(n, seed, 9100) if imf else np.full(n, 1.0 / n)
    x3, v3 = _com_frame(m, x3, v3)
    x3, v3 = scale_to_nbody_units(m, x3, v3, Q=Q, exact=W is None, W=W)
    return m, x3, v3


def hierarchical_triple(seed: int, stream: int, G: float = 1.0):
    """A hierarchical triple in its own N-body units (M = 1): inner binary
    (a_in = 1, e_in ~ U[0, 0.5]) orbited by a third body with outer-to-inner
    period ratio ~ logU[10, 1000], e_out ~ U[0, 0.5], isotropic mutual
    inclination, uniform mean anomalies; masses (0.4, 0.3, 0.3)."""
    u = uniform(seed, stream, 12)
    m1, m2, m3 = 0.4, 0.3, 0.3
    e_in, e_out = 0.5 * u[0], 0.5 * u[1]
    ratio = math.exp(math.log(10.0) + (math.log(1000.0) - math.log(10.0)) * u[2])
    a_in = 1.0
    # P ~ sqrt(a^3 / M): a_out from the period ratio
    a_out = a_in * (ratio ** 2 * (m1 + m2 + m3) / (m1 + m2)) ** (1.0 / 3.0)
    Ei = _mean_anomaly_E(seed, stream + 1000, np.array([e_in]))[0]
    Eo = _mean_anomaly_E(seed, stream + 2000, np.array([e_out]))[0]
    r_in, v_in = orbit_state(m1, m2, a_in, e_in, Ei, inc=math.acos(2 * u[3] - 1), node=2 * math.pi * u[4],
                             peri=2 * math.pi * u[5], G=G)
    r_out, v_out = orbit_state(m1 + m2, m3, a_out, e_out, Eo, inc=math.acos(2 * u[6] - 1),
                               node=2 * math.pi * u[7], peri=2 * math.pi * u[8], G=G)
    mi = m1 + m2
    M = mi + m3
    x = np.zeros((3, 3))
    v = np.zeros((3, 3))
    # inner COM at (m3/M) r_out, third body at -(mi/M) r_out
    ci, cv = (m3 / M) * r_out, (m3 / M) * v_out
    x[:, 0] = ci + (m2 / mi) * r_in
    x[:, 1] = ci - (m1 / mi) * r_in
    x[:, 2] = -(mi / M) * r_out
    v[:, 0] = cv + (m2 / mi) * v_in
    v[:, 1] = cv - (m1 / mi) * v_in
    v[:, 2] = -(mi / M) * v_out
    m = np.array([m1, m2, m3])
    x, v = _com_frame(m, x, v)
    # N-body units: scale lengths so E = -1/4 (virial ratio is what it is)
    T = 0.5 * float((m * (v * v).sum(axis=0)).sum())
    Wt = potential_energy(m, x)
    beta = (T + Wt) / -0.25
    return m, np.ascontiguousarray(x * beta), np.ascontiguousarray(v / math.sqrt(beta))


def small_systems(nsys: int = 4096, seed: int = 1, n_min: int = 3, n_max: int = 512):
    """A batch of independent small systems, each in its own N-body units:
    a fair coin picks a hierarchical triple or an equal-mass Plummer clump
    with round(logU[n_min, n_max]) bodies.  Returns (m, x3, v3, sys_off)
    with system s occupying ids [sys_off[s], sys_off[s+1])."""
    coin = uniform(seed, 31, nsys)
    sizes = np.rint(np.exp(np.log(n_min) + (np.log(n_max) - np.log(n_min)) * uniform(seed, 32, nsys))).astype(int)
    ms, xs, vs, off = [], [], [], [0]
    for s in range(nsys):
        if coin[s] < 0.5:
            m, x, v = hierarchical_triple(seed, 100000 + 37 * s)
        else:
            m, x, v = plummer(int(sizes[s]), seed=seed * 100003 + s, exact_scale=True)
        ms.append(m)
        xs.append(x)
        vs.append(v)
        off.append(off[-1] + m.shape[0])
    return (np.concatenate(ms), np.ascontiguousarray(np.concatenate(xs, axis=1)),
            np.ascontiguousarray(np.concatenate(vs, axis=1)), np.array(off, dtype=np.int64))
