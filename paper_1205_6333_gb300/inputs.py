"""Seeded synthetic inputs for the Stokesian-dynamics workloads.

This module holds geometry and random numbers only -- none of the method's
arithmetic -- so that both the CUDA path and the CPU oracle can be fed the very
same arrays.  It imports neither of them.

Workloads (units a = eta = F = 1 unless stated):

* ``square_cluster``  -- four spheres at the corners of a horizontal square of
  side 4a, each coordinate perturbed by U(-0.01a, 0.01a).
* ``tory_four_spheres`` -- the periodic four-sphere sedimentation start of
  Sec. 4 (Tory's stretched tetrahedron), in the reading
  r1=(5a,0,5a), r2=(0,5a,-5a), r3=(-5a,0,5a), r4=(0,-5a,-5a): the only
  placement consistent with every symmetry the section lists.
* ``cube_rsa``        -- N non-overlapping spheres (r_ij >= 2a) uniform in a cube
  sized for volume fraction phi, by random sequential addition.
* ``ball_rsa_batch``  -- many independent clusters, each uniform in a ball of
  radius a (N/phi)^(1/3) without overlap.
* ``normal_forces``   -- forces with i.i.d. N(0,1) components.
* ``fcc_lattice``     -- the paper's benchmark start, an fcc lattice at number
  density n (Sec. 3.3).

Seeds follow 1205633 + workload index.  numpy's PCG64 gives the same stream on
every platform.
"""
from __future__ import annotations

import math
import numpy as np

SEED_BASE = 1205633


def sphere_volume(a: float = 1.0) -> float:
    return 4.0 / 3.0 * math.pi * a ** 3


def cube_side(n: int, phi: float, a: float = 1.0) -> float:
    """Side L of the cube holding n spheres of radius a at volume fraction phi."""
    return (n * sphere_volume(a) / phi) ** (1.0 / 3.0)


def ball_radius(n: int, phi: float, a: float = 1.0) -> float:
    """Radius R_c = a (n/phi)^(1/3) of the ball holding n spheres at volume fraction phi."""
    return a * (n / phi) ** (1.0 / 3.0)


def square_cluster(seed: int = SEED_BASE + 0, a: float = 1.0, side: float = 4.0, jitter: float = 0.01) -> np.ndarray:
    """Four spheres on a horizontal square of side `side`*a, jittered by U(+-jitter*a)."""
    h = side * a / math.sqrt(2.0)
    x = np.array([[h, 0.0, 0.0], [0.0, h, 0.0], [-h, 0.0, 0.0], [0.0, -h, 0.0]])
    rng = np.random.default_rng(seed)
    return x + rng.uniform(-jitter * a, jitter * a, size=x.shape)


def tory_four_spheres(a: float = 1.0, h: float = 5.0) -> np.ndarray:
    """Start of the periodic four-sphere orbit (Sec. 4), reading described in the module docstring."""
    return a * np.array([[h, 0.0, h], [0.0, h, -h], [-h, 0.0, h], [0.0, -h, -h]], dtype=np.float64)


def _greedy_keep(cand: np.ndarray, dmin: float) -> np.ndarray:
    """Mask keeping, among candidates closer than dmin to each other, the earlier one."""
    from scipy.spatial import cKDTree
    keep = np.ones(len(cand), dtype=bool)
    if len(cand) < 2:
        return keep
    pairs = cKDTree(cand).query_pairs(dmin, output_type="ndarray")
    if len(pairs) == 0:
        return keep
    pairs = np.sort(pairs, axis=1)
    pairs = pairs[np.lexsort((pairs[:, 0], pairs[:, 1]))]
    for i, j in pairs:
        if keep[i]:
            keep[j] = False
    return keep


def cube_rsa(n: int, phi: float, seed: int, a: float = 1.0):
    """n non-overlapping spheres uniform in [0, L)^3, L = cube_side(n, phi).

    Random sequential addition in batches: candidates closer than 2a to an
    accepted sphere, or to an earlier candidate of the same batch, are dropped.
    Returns (x[n, 3] float64, L).
    """
    from scipy.spatial import cKDTree
    L = cube_side(n, phi, a)
    rng = np.random.default_rng(seed)
    dmin = 2.0 * a
    pts = np.empty((0, 3))
    while len(pts) < n:
        m = max(64, int(1.3 * (n - len(pts))) + 16)
        cand = rng.uniform(0.0, L, size=(m, 3))
        if len(pts):
            d, _ = cKDTree(pts).query(cand, k=1, distance_upper_bound=dmin)
            cand = cand[d >= dmin]
        cand = cand[_greedy_keep(cand, dmin)]
        pts = np.concatenate([pts, cand[: n - len(pts)]])
    return pts, L


def normal_forces(n: int, seed: int) -> np.ndarray:
    """Forces with i.i.d. standard-normal components, shape (n, 3)."""
    return np.random.default_rng(seed).standard_normal((n, 3))


def cluster_sizes(nclusters: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Cluster sizes uniform on the integers [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=nclusters).astype(np.int32)


def ball_rsa_batch(sizes, phi: float, seed: int, a: float = 1.0):
    """Independent clusters, cluster c holding sizes[c] spheres uniform in a ball of
    radius ball_radius(sizes[c], phi) about the origin, pairwise r >= 2a.

    All clusters advance in lock step: at step k every cluster still short of
    k+1 spheres draws one candidate and keeps it if it is at least 2a from the
    cluster's accepted spheres.  Returns (x[sum(sizes), 3] float64, offsets[C+1] int32).
    """
    sizes = np.asarray(sizes, dtype=np.int64)
    C = sizes.size
    nmax = int(sizes.max()) if C else 0
    rng = np.random.default_rng(seed)
    R = a * (sizes / phi) ** (1.0 / 3.0)
    buf = np.zeros((C, max(nmax, 1), 3))
    cnt = np.zeros(C, dtype=np.int64)
    dmin2 = (2.0 * a) ** 2
    active = np.nonzero(cnt < sizes)[0]
    while active.size:
        m = active.size
        # uniform in the unit ball: direction from a normal triple, radius u^(1/3)
        g = rng.standard_normal((m, 3))
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        u = rng.uniform(0.0, 1.0, size=m) ** (1.0 / 3.0)
        cand = g * (u * R[active])[:, None]
        k = cnt[active]
        kmax = int(k.max())
        ok = np.ones(m, dtype=bool)
        if kmax > 0:
            d2 = ((buf[active, :kmax, :] - cand[:, None, :]) ** 2).sum(-1)
            valid = np.arange(kmax)[None, :] < k[:, None]
            ok = ~np.any((d2 < dmin2) & valid, axis=1)
        acc = active[ok]
        buf[acc, cnt[acc], :] = cand[ok]
        cnt[acc] += 1
        active = np.nonzero(cnt < sizes)[0]
    offsets = np.zeros(C + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(sizes)
    x = np.concatenate([buf[c, : sizes[c]] for c in range(C)]) if C else np.zeros((0, 3))
    return x, offsets


def fcc_lattice(n_cells: int, density: float = 0.1, a: float = 1.0):
    """4 n_cells^3 sites of an fcc lattice at number density `density`/a^3 (Sec. 3.3 benchmark).
    Returns (x, L)."""
    N = 4 * n_cells ** 3
    L = (N / density) ** (1.0 / 3.0) * a
    c = L / n_cells
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(*[np.arange(n_cells)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = ((g[:, None, :] + base[None]) * c).reshape(-1, 3) + 0.25 * c
    return x, L


def config_inputs(idx: int, n: int | None = None):
    """Inputs of the five named workloads, seeded with SEED_BASE + idx:

      1. four spheres on a horizontal square of side 4a with U(+-0.01a) jitter, gravity;
      2. n = 65,536 spheres uniform in a cube at volume fraction 0.05 without overlap
         (random sequential addition), forces N(0,1) per component, both as float32;
      3. n = 16,384 spheres in a cube at volume fraction 0.10, gravity and the soft
         repulsion eps (2a/r)^12 (eps = 1) cut at 2.5a;
      4. 16,384 clusters of U{4..256} spheres, each uniform in a ball at volume
         fraction 0.05 without overlap, forces N(0,1);
      5. n = 4,096 spheres in a cube at volume fraction 0.05, gravity, and targets
         x(0) + N(0,1) for the loss sum |x(T) - x*|^2.

    Returns a dict of numpy arrays and scalars; positions and forces are float64
    except where the workload specifies float32 inputs (workload 2).
    """
    seed = SEED_BASE + idx
    if idx == 1:
        return {"x": square_cluster(seed), "gravity": np.array([0.0, 0.0, -1.0])}
    if idx == 2:
        n = n or 65536
        x, L = cube_rsa(n, 0.05, seed)
        F = normal_forces(n, seed + 1000)
        return {"x": x.astype(np.float32), "F": F.astype(np.float32), "L": L}
    if idx == 3:
        n = n or 16384
        x, L = cube_rsa(n, 0.10, seed)
        return {"x": x, "L": L, "gravity": np.array([0.0, 0.0, -1.0]), "rep_eps": 1.0, "rep_rc": 2.5}
    if idx == 4:
        C = n or 16384
        sizes = cluster_sizes(C, 4, 256, seed)
        x, off = ball_rsa_batch(sizes, 0.05, seed + 1)
        F = normal_forces(x.shape[0], seed + 2)
        return {"x": x, "offsets": off, "F": F}
    if idx == 5:
        n = n or 4096
        x, L = cube_rsa(n, 0.05, seed)
        target = x + np.random.default_rng(seed + 3).standard_normal(x.shape)
        return {"x": x, "L": L, "gravity": np.array([0.0, 0.0, -1.0]), "target": target}
    raise ValueError("unknown workload %d" % idx)
