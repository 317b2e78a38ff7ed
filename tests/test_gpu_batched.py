"""Batched clusters (one persistent launch per step) against the FP64 oracle run
cluster by cluster."""
import numpy as np
import pytest

import oracle
import paper_1205_6333_gb300 as sd
from paper_1205_6333_gb300 import inputs

pytestmark = pytest.mark.gpu


def _clusters(C, seed, lo=4, hi=256):
    sizes = inputs.cluster_sizes(C, lo, hi, seed)
    x, off = inputs.ball_rsa_batch(sizes, 0.05, seed + 1)
    F = inputs.normal_forces(x.shape[0], seed + 2)
    return x, off, F


def _oracle_batch(x, off, F, nsteps, dt, tensor="rpy"):
    out = np.empty_like(x)
    for c in range(len(off) - 1):
        a, b = off[c], off[c + 1]
        if b > a:
            out[a:b] = oracle.euler(x[a:b], nsteps, dt, fext=F[a:b], tensor=tensor)
    return out


@pytest.mark.parametrize("prec,tol", [("fp32c", 1e-5), ("fp64", 1e-10)])
def test_batched_matches_oracle(prec, tol):
    x, off, F = _clusters(160, inputs.SEED_BASE + 4)
    nsteps, dt = 20, 0.01
    ref = _oracle_batch(x, off, F, nsteps, dt)
    b = sd.Batch(off, prec=prec)
    b.set_positions(x)
    b.set_forces(F)
    b.step(dt, nsteps)
    got = b.get_positions()
    b.close()
    disp = np.abs(ref - x).max()
    assert np.abs(got - ref).max() <= tol * disp


@pytest.mark.parametrize("tensor", ["rpy", "rp", "oseen"])
def test_batched_overlaps_and_odd_sizes(tensor):
    """Clusters of size 0, 1, 2, 31, 32, 33, 255, 256 with overlapping pairs."""
    rng = np.random.default_rng(3)
    sizes = [0, 1, 2, 31, 32, 33, 255, 256, 5]
    xs = []
    for n in sizes:
        p, _ = inputs.cube_rsa(max(n, 1), 0.05, int(rng.integers(1 << 30)))
        p = p[:n]
        if n >= 4:
            p[1] = p[0] + np.array([0.7, 0.3, -0.2])    # r < 2a
            p[3] = p[2] + np.array([1.95, 0.0, 0.0])
        xs.append(p)
    x = np.concatenate(xs)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    F = inputs.normal_forces(x.shape[0], 5)
    ref = _oracle_batch(x, off, F, 3, 0.02, tensor)
    b = sd.Batch(off, tensor=tensor)
    b.set_positions(x)
    b.set_forces(F)
    b.step(0.02, 3)
    got = b.get_positions()
    b.close()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref - x).max()


def _odd_sizes_with_overlaps(seed=3):
    rng = np.random.default_rng(seed)
    sizes = [0, 1, 2, 31, 32, 33, 255, 256, 5, 3, 7, 130, 129]
    xs = []
    for n in sizes:
        p, _ = inputs.cube_rsa(max(n, 1), 0.05, int(rng.integers(1 << 30)))
        p = p[:n]
        if n >= 4:
            p[1] = p[0] + np.array([0.7, 0.3, -0.2])    # r < 2a
            p[3] = p[2] + np.array([1.95, 0.0, 0.0])
        xs.append(p)
    x = np.concatenate(xs)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    return x, off, inputs.normal_forces(x.shape[0], seed + 2)


def _shape_kinds(prec):
    """One shape index per (threads per CTA, targets per thread) the batch offers."""
    b = sd.Batch(np.array([0, 4], dtype=np.int32), prec=prec)
    kinds = {}
    for k, sh in enumerate(b.shapes()):
        kinds.setdefault((sh["threads"], sh["targets_per_thread"]), k)
    b.close()
    return kinds


def test_batched_shapes_include_two_targets_per_thread():
    kinds = _shape_kinds("fp32c")
    assert {(128, 1), (256, 1), (128, 2), (256, 2), (128, 0)} <= set(kinds)
    assert {r for (_, r) in _shape_kinds("fp64")} == {1}
    b = sd.Batch(np.array([0, 4], dtype=np.int32))
    with pytest.raises(sd.SDError):
        b.set_shape(len(b.shapes()))
    b.close()


@pytest.mark.parametrize("threads,r", [(128, 1), (256, 1), (128, 2), (256, 2), (128, 0)])
@pytest.mark.parametrize("tensor", ["rpy", "oseen"])
def test_batched_every_shape_matches_oracle(threads, r, tensor):
    """Each FP32C kernel variant, pinned instead of autotuned (r = 0: the symmetric
    kernel, two clusters per warp): clusters of sizes 0 to 256 (odd and even: the last
    target of an odd cluster has a slot of its own when a thread owns two), overlapping
    pairs, 20 steps (one graph replay and 4 eager steps)."""
    x, off, F = _odd_sizes_with_overlaps()
    ref = _oracle_batch(x, off, F, 20, 0.01, tensor)
    b = sd.Batch(off, tensor=tensor)
    k = next(k for k, sh in enumerate(b.shapes())
             if sh["threads"] == threads and sh["targets_per_thread"] == r)
    b.set_shape(k)
    b.set_positions(x)
    b.set_forces(F)
    b.step(0.01, 20)
    got = b.get_positions()
    b.close()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref - x).max()


def test_batched_coincident_pairs():
    x = np.array([[0.0, 0, 0], [4.0, 0, 0], [4.0, 0, 0], [0.0, 9, 0]])
    off = np.array([0, 3, 4], dtype=np.int32)
    F = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [1, 1, 1.0]])
    b = sd.Batch(off, tensor="rpy", prec="fp64")
    b.set_positions(x)
    b.set_forces(F)
    b.step(0.1, 1)
    got = b.get_positions()
    ref = _oracle_batch(x, off, F, 1, 0.1)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13)
    b2 = sd.Batch(off, tensor="rp")
    b2.set_positions(x)
    b2.set_forces(F)
    # reported by the first synchronising call: the autotuner's (first step) or ours
    with pytest.raises(sd.SDError) as ei:
        b2.step(0.1, 1)
        b2.synchronize()
    assert ei.value.status_name == "SD_ERR_COINCIDENT"
    b2.synchronize()   # error word cleared, batch still usable
    b2.close()
    b.close()


def test_batched_graph_equals_eager_and_autotune():
    x, off, F = _clusters(300, 77)
    b = sd.Batch(off)
    b.set_positions(x)
    b.set_forces(F)
    choice = b.autotune()
    assert choice >= 0
    b.step(0.01, 33)
    a = b.get_positions()
    b.set_positions(x)
    for _ in range(33):
        b.step(0.01, 1)
    np.testing.assert_array_equal(a, b.get_positions())
    c0 = b.launch_count()
    b.step(0.01, 16)
    b.synchronize()
    assert b.launch_count() == c0 + 16
    b.close()


def test_batched_full_workload_sampled_clusters():
    """The batched workload at full size (16,384 clusters, N_c ~ U{4..256}, 2.1M particles)
    in the launch shape the autotuner picks, as timed: 5 FP32C steps, then 48 clusters
    (the 8 largest, the 8 smallest and 32 seeded others) against the oracle run on each
    cluster alone."""
    w = inputs.config_inputs(4)
    x, off, F = w["x"], w["offsets"], w["F"]
    nsteps, dt = 5, 0.01
    b = sd.Batch(off, prec="fp32c")
    b.set_positions(x)
    b.set_forces(F)
    b.step(dt, nsteps)
    got = b.get_positions()
    b.close()
    sizes = np.diff(off)
    order = np.argsort(sizes, kind="stable")
    rng = np.random.default_rng(inputs.SEED_BASE + 40)
    picks = np.unique(np.concatenate([order[:8], order[-8:], rng.choice(len(sizes), 32, replace=False)]))
    for c in picks:
        a, e = off[c], off[c + 1]
        ref = oracle.euler(x[a:e], nsteps, dt, fext=F[a:e])
        disp = np.abs(ref - x[a:e]).max()
        assert np.abs(got[a:e] - ref).max() <= 1e-5 * disp, (int(c), int(e - a))


@pytest.mark.parametrize("tensor", ["rpy", "rp", "oseen"])
def test_batched_symmetric_kernel_overlaps_and_coincident(tensor):
    """The symmetric kernel pinned: many overlapping pairs in clusters of every block
    count (1 to 8 blocks of 32), including pairs inside one 32-block and across blocks,
    and, for RPY, two coincident spheres; 3 steps against the oracle."""
    rng = np.random.default_rng(11)
    sizes = [1, 2, 5, 32, 33, 64, 65, 100, 130, 200, 255, 256, 17]
    xs = []
    for n in sizes:
        p, _ = inputs.cube_rsa(n, 0.05, int(rng.integers(1 << 30)))
        for k in range(0, n - 1, 7):      # an overlapping partner every 7 particles
            j = (k + 1 + 37 * (k // 7)) % n
            if j != k:
                d = rng.standard_normal(3)
                p[j] = p[k] + d / np.linalg.norm(d) * rng.uniform(0.3, 1.9)
        if tensor == "rpy" and n >= 40:
            p[39] = p[38]
        xs.append(p)
    x = np.concatenate(xs)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    F = inputs.normal_forces(x.shape[0], 12)
    ref = _oracle_batch(x, off, F, 3, 0.01, tensor)
    b = sd.Batch(off, tensor=tensor)
    b.set_shape(next(k for k, sh in enumerate(b.shapes()) if sh["targets_per_thread"] == 0))
    b.set_positions(x)
    b.set_forces(F)
    b.step(0.01, 3)
    got = b.get_positions()
    b.close()
    for c in range(len(sizes)):
        a, e = off[c], off[c + 1]
        disp = max(np.abs(ref[a:e] - x[a:e]).max(), 1e-300)
        assert np.abs(got[a:e] - ref[a:e]).max() <= 1e-5 * disp, (c, sizes[c])


def _crowded_cluster(n, side, dmin, rng):
    """n centres uniform in a cube of the given side, none closer than dmin to another
    (random sequential addition): every sphere overlaps several others."""
    pts = []
    while len(pts) < n:
        q = rng.uniform(0.0, side, 3)
        if all(np.sum((q - p) ** 2) >= dmin * dmin for p in pts):
            pts.append(q)
    return np.array(pts)


@pytest.mark.parametrize("tensor", ["rpy", "oseen"])
def test_batched_symmetric_kernel_crowded_clusters(tensor):
    """The symmetric kernel pinned on crowded clusters (about eight overlapping
    partners per sphere, none closer than 0.3a): most tiles meet pairs closer than 2a,
    many lanes of a warp at once and several pairs per target in one tile, in both
    halves of the packed registers, in diagonal and off-diagonal tiles; the two halves
    pair crowded with crowded and crowded with dilute clusters.  3 steps against the
    oracle."""
    rng = np.random.default_rng(21)
    sizes = [256, 256, 250, 249, 200, 64, 33, 32, 31, 2]
    xs = []
    for c, n in enumerate(sizes):
        if c in (3, 6):   # dilute partners for a crowded cluster of (nearly) the same size
            p, _ = inputs.cube_rsa(n, 0.05, int(rng.integers(1 << 30)))
        else:
            p = _crowded_cluster(n, (n / 0.25) ** (1.0 / 3.0), 0.3, rng)
        xs.append(p)
    x = np.concatenate(xs)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    F = inputs.normal_forces(x.shape[0], 22)
    ref = _oracle_batch(x, off, F, 3, 0.002, tensor)
    b = sd.Batch(off, tensor=tensor)
    b.set_shape(next(k for k, sh in enumerate(b.shapes()) if sh["targets_per_thread"] == 0))
    b.set_positions(x)
    b.set_forces(F)
    b.step(0.002, 3)
    got = b.get_positions()
    b.close()
    for c in range(len(sizes)):
        a, e = off[c], off[c + 1]
        disp = max(np.abs(ref[a:e] - x[a:e]).max(), 1e-300)
        assert np.abs(got[a:e] - ref[a:e]).max() <= 1e-5 * disp, (c, sizes[c])
