"""Helpers shared by the GPU parity tests: oracle component arrays built from
the generators' species arrays, and the error metric of the parity bars.

Error metric (per output q at each ray): e_q = |dq| / max(|q_ref|, 1e-3 *
median |q_ref|), with vector norms for alpha and the complex modulus for
gamma; kappa uses the same form.
"""
import numpy as np

import oracle


def comps_points(p):
    p = np.asarray(p, np.float64)
    return oracle.make_components(oracle.POINT, p[:, 0], p[:, 1], p[:, 2])


def comps_gauss(p, q):
    p = np.asarray(p, np.float64)
    return oracle.make_components(oracle.GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], q)


def comps_nfw(p, conc):
    p = np.asarray(p, np.float64)
    return oracle.make_components(oracle.NFW, p[:, 0], p[:, 1], p[:, 2], p[:, 3], conc * p[:, 3])


def rel_errors(got, ref):
    """(alpha, kappa, gamma) error arrays per the metric above."""
    out = []
    for cols in ([0, 1], [2], [3, 4]):
        d = np.linalg.norm(got[:, cols] - ref[:, cols], axis=1)
        r = np.linalg.norm(ref[:, cols], axis=1)
        med = np.median(r)
        out.append(d / np.maximum(r, 1e-3 * med) if med > 0 else d)
    return out


def to_np(outs):
    return np.stack([o.double().cpu().numpy() for o in outs], axis=1)


EPS32 = 2.0 ** -24


def within_fp32_bar(got, ref, absum, rel=1e-5, k=8.0):
    """Per output and ray: |d| <= rel * max(|ref|, 1e-3 median |ref|) or, for
    an ill-conditioned sum, |d| <= k * eps32 * sum |term| (the error any sum
    of FP32-evaluated terms can carry; the oracle's absum is sum |term|).
    Returns (ok mask (nr, 3), fraction of rays that needed the second form)."""
    ok = np.zeros((got.shape[0], 3), bool)
    cond = np.zeros((got.shape[0], 3), bool)
    for j, cols in enumerate(([0, 1], [2], [3, 4])):
        d = np.linalg.norm(got[:, cols] - ref[:, cols], axis=1)
        r = np.linalg.norm(ref[:, cols], axis=1)
        a = np.linalg.norm(absum[:, cols], axis=1)
        floor = 1e-3 * np.median(r) if np.median(r) > 0 else 0.0
        first = d <= rel * np.maximum(r, floor)
        second = d <= k * EPS32 * a
        ok[:, j] = first | second
        cond[:, j] = ~first & second
    return ok, cond.any(axis=1).mean()
