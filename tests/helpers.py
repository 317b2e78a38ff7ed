"""Shared helpers of the tests: error metrics and seeded inputs with the
structure of the paper's workloads (see the design doc for the recipe)."""
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
