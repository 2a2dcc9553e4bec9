"""Per-body error bounds for the mixed-precision form and the Kepler mode.

The mixed form evaluates the pair forces between components in FP32 (the
FP64 difference of positions rounded, rsqrt with one Newton step, terms
summed in groups of 8 with each group sum added with compensation), so the
error of body i's acceleration is bounded by a small multiple of the unit
roundoff u = 2^-24 times the sum of the absolute pair terms,

    S_i = sum_j G m_j / (|x_i - x_j|^2 + eps^2),

not by a multiple of |a_i| (a body near the centre of a cluster has a small
net force out of large terms).  Per pair: 2u for the rounded difference, 3u
for r^2, 2u for rsqrt and its Newton step, 3u for r^-3, 2u for the factors:
12u; a group of 8 summed in plain FP32 adds at most 7u of the group's
absolute sum, the compensated addition of the group sums 2u of |a_i|.  So
|da_i| <= 21 u S_i.  An outer step of length dt kicks each body once per
recursion level it takes part in, with kicks that add up to dt per level, so
after one step |dv_i| <= 21 u dt S_i (D + 1) for a recursion D levels deep.
The bound used by the tests is K u dt S_i (D + 1) per step with K = 32.

A pair whose tau lies within the rounding of the two trajectories of the
threshold of some split (|tau - h| / h ~ 1e-8) may be an edge in one run and
not in the other; its two bodies are then integrated by a different
splitting and legitimately differ by far more.  The tests let the GPU log
every pair within 1e-6 of a threshold (near_tol) and exempt the bodies of
logged pairs, and only those, from the per-body bound.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53
K_MIXED = 32.0


def abs_accel_sum(m, x3, G: float = 1.0, eps: float = 0.0, chunk: int = 256, groups=None, labels=None, rows=None):
    """S_i = sum_{j != i} G m_j / (r_ij^2 + eps^2) (numpy, chunked).  groups:
    optional system index per body; pairs of different systems are left out
    (independent systems never interact).  labels: optional component label
    per body; only pairs with different labels count (the pairs a kick
    with these labels applies).  rows: optional body indices; S is then
    computed for those bodies only (other entries 0)."""
    n = m.shape[0]
    S = np.zeros(n)
    idx = np.arange(n) if rows is None else np.asarray(rows)
    for s in range(0, idx.shape[0], chunk):
        r = idx[s:s + chunk]
        d = x3[:, r, None] - x3[:, None, :]
        r2 = (d * d).sum(axis=0) + eps * eps
        r2[np.arange(r.shape[0]), r] = np.inf
        w = G * m[None, :] / r2
        if groups is not None:
            w = np.where(groups[r, None] == groups[None, :], w, 0.0)
        if labels is not None:
            w = np.where(labels[r, None] != labels[None, :], w, 0.0)
        S[r] = w.sum(axis=1)
    return S


def abs_accel_sum_systems(m, x3, sys_off, G: float = 1.0, eps: float = 0.0):
    """S_i within each independent system (system by system: O(sum n_s^2))."""
    S = np.zeros(m.shape[0])
    for a, b in zip(sys_off[:-1], sys_off[1:]):
        S[a:b] = abs_accel_sum(m[a:b], x3[:, a:b], G=G, eps=eps)
    return S


def system_index(n, sys_off):
    g = np.zeros(n, dtype=np.int64)
    for k, (a, b) in enumerate(zip(sys_off[:-1], sys_off[1:])):
        g[a:b] = k
    return g


def near_bodies(pairs):
    """Bodies of the GPU's logged near-threshold pairs."""
    return np.unique(np.asarray(pairs, dtype=np.int64).reshape(-1))


def check_velocity_bound(gv, ov, S, dt, depth, steps=1, K=K_MIXED, u=U32, exempt=(), what=""):
    """Assert |gv_i - ov_i| <= K u dt S_i (depth + 1) steps for every body
    not in `exempt`; returns (max ratio over bodies, exempt bodies over bound)."""
    err = np.linalg.norm(gv - ov, axis=0)
    tol = K * u * dt * S * (depth + 1) * steps
    ratio = err / tol
    mask = np.ones(ratio.shape[0], dtype=bool)
    ex = np.asarray(exempt, dtype=np.int64)
    if ex.size:
        mask[ex] = False
    worst = int(np.argmax(np.where(mask, ratio, -1.0)))
    assert ratio[mask].max() <= 1.0, (what, "body", worst, "ratio", float(ratio[worst]), "err", float(err[worst]),
                                      "tol", float(tol[worst]))
    return float(ratio[mask].max()), int((ratio[~mask] > 1.0).sum())


def check_position_bound(gx, ox, S, dt, depth, steps=1, K=K_MIXED, u=U32, exempt=(), what=""):
    """Positions of the mixed form: a body's position is its start plus the
    drifts of the step, each taking a velocity within the bound of
    check_velocity_bound, so |gx_i - ox_i| <= dt (K u dt S_i (depth + 1)
    steps) steps, plus the FP64 roundings of the drifts (at most one ulp of
    |x| per level).  Asserted for every body not in `exempt`; returns the
    largest ratio."""
    err = np.linalg.norm(gx - ox, axis=0)
    tol = dt * steps * (K * u * dt * S * (depth + 1) * steps) + 4 * U64 * (depth + 1) * np.linalg.norm(ox, axis=0)
    ratio = err / tol
    mask = np.ones(ratio.shape[0], dtype=bool)
    ex = np.asarray(exempt, dtype=np.int64)
    if ex.size:
        mask[ex] = False
    worst = int(np.argmax(np.where(mask, ratio, -1.0)))
    assert ratio[mask].max() <= 1.0, (what, "body", worst, "ratio", float(ratio[worst]), "err", float(err[worst]),
                                      "tol", float(tol[worst]))
    return float(ratio[mask].max())
