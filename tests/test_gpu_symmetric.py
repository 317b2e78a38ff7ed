"""The symmetric all-pairs kernel (each unordered pair once, mu_ij = mu_ji of
Sec. 2.2) against the FP64 oracle, and against the directed kernel of Sec. 3.2,
through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_1205_6333_gb300 as sd
from paper_1205_6333_gb300 import inputs
from helpers import TOL, periodic_rel_err, rel_err, system_with_overlaps

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32c", "fp32", "fp64"])
@pytest.mark.parametrize("tensor", ["rpy", "rp", "oseen"])
@pytest.mark.parametrize("n", [1, 2, 3, 33, 257, 513, 1500, 4133])
def test_symmetric_matches_oracle(prec, tensor, n):
    """Forced symmetric kernel; sizes below, at and across the blocks (256 particles,
    128 in FP64; ragged last block, padding), overlapping pairs (RPY branch and
    clamp)."""
    x, _ = system_with_overlaps(n, 0.05, seed=300 + n, overlaps=5)
    F = inputs.normal_forces(n, seed=400 + n)
    with sd.System(n, tensor=tensor, prec=prec, dense="symmetric") as s:
        assert s.dense_kernel() == "symmetric"
        s.set_positions(x)
        v = s.mobility_apply(F)
    ref = oracle.mobility_apply(x, F, tensor, nthreads=8)
    assert rel_err(v, ref) <= TOL[prec]


def test_symmetric_close_pairs_across_blocks():
    """Pairs closer than a (the near pass then makes every tile clamp) placed between
    particles of different 256-blocks, i.e. inside off-diagonal tiles."""
    n = 2048
    x, _ = inputs.cube_rsa(n, 0.05, 77)
    rng = np.random.default_rng(78)
    for i, j in [(3, 700), (260, 1900), (1023, 1024), (5, 2047)]:
        d = rng.standard_normal(3)
        x[j] = x[i] + d / np.linalg.norm(d) * rng.uniform(0.1, 0.9)
    F = inputs.normal_forces(n, 79)
    ref = oracle.mobility_apply(x, F, "rpy", nthreads=8)
    for dense in ["symmetric", "directed"]:
        with sd.System(n, dense=dense) as s:
            s.set_positions(x)
            assert rel_err(s.mobility_apply(F), ref) <= TOL["fp32c"], dense


def test_symmetric_and_directed_agree_and_repeat():
    """Same inputs through both kernels: each direction's FP32 term is the same, so
    the results differ only by summation order; each kernel repeats bit for bit."""
    n = 20000
    w = inputs.config_inputs(2, n=n)
    x, F = w["x"].astype(np.float64), w["F"].astype(np.float64)
    out = {}
    for dense in ["directed", "symmetric"]:
        with sd.System(n, dense=dense) as s:
            s.set_positions(x)
            v1 = s.mobility_apply(F)
            v2 = s.mobility_apply(F)
            np.testing.assert_array_equal(v1, v2)
            out[dense] = v1
    assert rel_err(out["symmetric"], out["directed"]) <= 2e-6
    rows = np.arange(0, n, 53, dtype=np.int32)
    ref = oracle.mobility_rows(x, F, rows, "rpy", nthreads=8)
    for dense in out:
        assert rel_err(out[dense][rows], ref) <= TOL["fp32c"], dense


def test_symmetric_euler_steps_match_oracle():
    """Workload-3 physics (gravity + soft repulsion) through sd_step with the
    symmetric kernel: 20 steps at N = 3000 against the oracle's trajectory."""
    n, steps, dt = 3000, 20, 0.05
    x0, _ = inputs.cube_rsa(n, 0.10, 91)
    g = (0.0, 0.0, -1.0)
    ref = oracle.euler(x0, steps, dt, gravity=g, rep_eps=1.0, rep_rc=2.5, nthreads=8)
    with sd.System(n, gravity=g, rep_eps=1.0, rep_rc=2.5, dense="symmetric") as s:
        s.set_positions(x0)
        s.step(dt, steps)
        xT = s.get_positions()
    disp = np.linalg.norm(ref - x0, axis=1).max()
    assert np.linalg.norm(xT - ref, axis=1).max() <= 1e-5 * disp


def test_auto_choice():
    with sd.System(65536) as s:
        assert s.dense_kernel() == "symmetric"
    with sd.System(1024) as s:
        assert s.dense_kernel() == "directed"
    with sd.System(8192) as s:
        assert s.dense_kernel() == "symmetric"
    with sd.System(65536, prec="fp64") as s:
        assert s.dense_kernel() == "symmetric"
    with sd.System(1024, prec="fp64") as s:
        assert s.dense_kernel() == "directed"
    with sd.System(100, prec="fp64", dense="symmetric") as s:
        assert s.dense_kernel() == "symmetric"


def test_fp64_symmetric_and_directed_agree_and_repeat():
    """FP64: each direction's term of the symmetric kernel is bit-identical to the
    directed kernel's; the sums differ by order only (far below the 1e-12 gate)."""
    n = 6000
    x, _ = system_with_overlaps(n, 0.05, seed=81, overlaps=4)
    F = inputs.normal_forces(n, 82)
    out = {}
    for dense in ["directed", "symmetric"]:
        with sd.System(n, prec="fp64", dense=dense) as s:
            assert s.dense_kernel() == dense
            s.set_positions(x)
            v1 = s.mobility_apply(F)
            np.testing.assert_array_equal(v1, s.mobility_apply(F))
            out[dense] = v1
    assert rel_err(out["symmetric"], out["directed"]) <= 1e-14
    rows = np.arange(0, n, 17, dtype=np.int32)
    ref = oracle.mobility_rows(x, F, rows, "rpy", nthreads=8)
    assert rel_err(out["symmetric"][rows], ref) <= TOL["fp64"]


@pytest.mark.parametrize("tensor", ["rpy", "oseen"])
def test_fp64_symmetric_periodic(tensor):
    n = 3000
    x, L = system_with_overlaps(n, 0.05, seed=83, overlaps=4)
    L = max(L, 10.0)
    box = (L, L, L)
    x = x + L * np.random.default_rng(84).integers(-1, 2, x.shape)
    F = inputs.normal_forces(n, 85)
    with sd.System(n, prec="fp64", tensor=tensor, box=box, dense="symmetric") as s:
        s.set_positions(x)
        v = s.mobility_apply(F)
    ref = oracle.mobility_apply(x, F, tensor, box=box, nthreads=8)
    assert periodic_rel_err(v, ref, x, F, box, tensor, margin=1e-12) <= TOL["fp64"]


def test_fp64_symmetric_euler_steps_match_oracle():
    n, steps, dt = 2500, 20, 0.05
    x0, _ = inputs.cube_rsa(n, 0.10, 92)
    g = (0.0, 0.0, -1.0)
    ref = oracle.euler(x0, steps, dt, gravity=g, rep_eps=1.0, rep_rc=2.5, nthreads=8)
    with sd.System(n, prec="fp64", gravity=g, rep_eps=1.0, rep_rc=2.5) as s:
        assert s.dense_kernel() == "symmetric"
        s.set_positions(x0)
        s.step(dt, steps)
        xT = s.get_positions()
    disp = np.linalg.norm(ref - x0, axis=1).max()
    assert np.linalg.norm(xT - ref, axis=1).max() <= 1e-10 * disp


@pytest.mark.parametrize("n", [9000, 33000])   # blocks of 256 x 64 threads, and of 512 x 128 threads
@pytest.mark.parametrize("tensor", ["rpy", "oseen"])
@pytest.mark.parametrize("periodic", [False, True])
def test_four_target_block_shapes(n, tensor, periodic):
    """The block shapes with four targets per thread (mid-size and large N), ragged
    last blocks, overlapping pairs, unbounded and periodic, on sampled rows; the
    overlapping pairs are among the rows."""
    x, L = system_with_overlaps(n, 0.05, seed=500 + n, overlaps=6)
    box = (L, L, L) if periodic else None
    if periodic:
        x = x + L * np.random.default_rng(501).integers(-1, 2, x.shape)   # unwrapped images
    F = inputs.normal_forces(n, seed=502 + n)
    with sd.System(n, tensor=tensor, box=box) as s:
        assert s.dense_kernel() == "symmetric"
        s.set_positions(x)
        v = s.mobility_apply(F)
    rows = np.concatenate([np.arange(12), np.random.default_rng(n).choice(n, 300, replace=False), [n - 1]])
    rows = np.unique(rows).astype(np.int32)
    ref = oracle.mobility_rows(x, F, rows, tensor, box=box, nthreads=8)
    if periodic:
        assert periodic_rel_err(v[rows], ref, x, F, box, tensor, rows=rows) <= TOL["fp32c"]
    else:
        assert rel_err(v[rows], ref) <= TOL["fp32c"]
