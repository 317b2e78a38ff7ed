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
