"""Shared helpers of the tests: error metrics and seeded inputs with the
structure of the paper's workloads (random non-overlapping packings at a given
volume fraction, N(0,1) forces, deliberately planted overlapping pairs)."""
import numpy as np

from paper_1205_6333_gb300 import inputs

# Gates (velocity error relative to the largest reference velocity)
TOL = {"fp32c": 1e-5, "fp64": 1e-12, "fp32": 1e-4}


def rel_err(v, ref):
    """max_i |v_i - ref_i|_2 / max_i |ref_i|_2."""
    v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1, 3)
    den = np.linalg.norm(ref, axis=1).max()
    return float(np.linalg.norm(v - ref, axis=1).max() / den)


def l2_rel_err(v, ref):
    v = np.asarray(v, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(v - ref) / np.linalg.norm(ref))


def system_with_overlaps(n, phi=0.05, seed=1, overlaps=3):
    """Non-overlapping cube packing, then `overlaps` particles moved onto a neighbour
    at r in (0.2a, 1.9a) -- the RPY overlap branch and the clamp both get exercised."""
    x, L = inputs.cube_rsa(n, phi, seed)
    rng = np.random.default_rng(seed + 7)
    for k in range(min(overlaps, n // 2)):
        i, j = 2 * k, 2 * k + 1
        d = rng.standard_normal(3)
        x[j] = x[i] + d / np.linalg.norm(d) * rng.uniform(0.2, 1.9)
    return x, L


def periodic_rel_err(v, ref, x, F, box, tensor="rpy", a=1.0, eta=1.0, margin=4e-6, rows=None):
    """rel_err for a periodic box where the nearest image is ambiguous.

    A pair whose separation lies within margin * L of half a period in some
    dimension has two equally near images (Sec. 3.1 footnote: only the nearest one
    interacts), and FP32 separations decide that tie at FP32 precision.  Both
    choices are correct, so for every particle the error is taken against the
    closest of the oracle values with any subset of its tie pairs switched to the
    other image.  With `rows`, v and ref hold those particles' velocities only."""
    import itertools

    import oracle

    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    F = np.asarray(F, dtype=np.float64).reshape(-1, 3)
    v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1, 3)
    L = np.asarray(box, dtype=np.float64)
    per = L > 0
    n = x.shape[0]
    idx = np.arange(n) if rows is None else np.asarray(rows)
    alts = {}   # position in v -> list of velocity changes, one per tie pair
    for i0 in range(0, idx.size, 512):
        d = x[idx[i0:i0 + 512], None, :] - x[None, :, :]
        img = np.where(per, d - L * np.round(d / np.where(per, L, 1.0)), d)
        near_tie = per & (np.abs(np.abs(img) - 0.5 * L) < margin * L)
        for ii, j, k in zip(*np.nonzero(near_tie)):
            if idx[i0 + ii] == j:
                continue
            r1 = img[ii, j]
            r2 = r1.copy()
            r2[k] -= np.sign(r1[k]) * L[k]
            dv = (oracle.pair_tensor(r2, tensor, a, eta) - oracle.pair_tensor(r1, tensor, a, eta)) @ F[j]
            alts.setdefault(int(i0 + ii), []).append(dv)
    den = np.linalg.norm(ref, axis=1).max()
    err = np.linalg.norm(v - ref, axis=1)
    for i, dvs in alts.items():
        best = err[i]
        for m in range(1, len(dvs) + 1):
            for sub in itertools.combinations(dvs, m):
                best = min(best, float(np.linalg.norm(v[i] - ref[i] - sum(sub))))
        err[i] = best
    return float(err.max() / den)
