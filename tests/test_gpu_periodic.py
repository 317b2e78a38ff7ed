"""Periodic box, nearest image only (Sec. 3.1 footnote), against the FP64 oracle
through the C ABI: mobility apply (both all-pairs kernels), Euler steps with
repulsion and lubrication, and the VJP."""
import numpy as np
import pytest

import oracle
import paper_1205_6333_gb300 as sd
from paper_1205_6333_gb300 import inputs
from helpers import TOL, periodic_rel_err, rel_err

pytestmark = pytest.mark.gpu


def _periodic_system(n, phi, seed, overlaps=4, min_side=10.0):
    """Cube packing of side L (>= min_side); particles shifted by whole periods so
    the state is unwrapped; a few pairs overlapping across the faces of the box."""
    x, L = inputs.cube_rsa(n, phi, seed)
    L = max(L, min_side)
    rng = np.random.default_rng(seed + 11)
    x = x + L * rng.integers(-2, 3, x.shape)          # unwrapped images of the same configuration
    for k in range(min(overlaps, n // 2)):
        i, j = 2 * k, 2 * k + 1
        d = rng.standard_normal(3)
        base = np.array([0.05, rng.uniform(0, L), L - 0.05])   # at the faces x = 0 and z = L
        x[i] = base + L * rng.integers(-1, 2, 3)
        x[j] = base + d / np.linalg.norm(d) * rng.uniform(0.3, 1.9) + L * rng.integers(-1, 2, 3)
    return x, L


@pytest.mark.parametrize("prec", ["fp32c", "fp64", "fp32"])
@pytest.mark.parametrize("tensor", ["rpy", "rp", "oseen"])
@pytest.mark.parametrize("n", [1, 2, 33, 513, 1500, 4133])
def test_periodic_apply_matches_oracle(prec, tensor, n):
    x, L = _periodic_system(n, 0.05, 500 + n)
    F = inputs.normal_forces(n, 600 + n)
    box = (L, L, L)
    with sd.System(n, tensor=tensor, prec=prec, box=box) as s:
        s.set_positions(x)
        v = s.mobility_apply(F)
    ref = oracle.mobility_apply(x, F, tensor, box=box, nthreads=8)
    assert periodic_rel_err(v, ref, x, F, box, tensor) <= TOL[prec]


@pytest.mark.parametrize("dense", ["directed", "symmetric"])
@pytest.mark.parametrize("box", [(1, 1, 0), (0, 0, 1), (1, 0.7, 1.3)])
def test_periodic_slabs_and_boxes(dense, box):
    """Periodic in some dimensions only, unequal sides; both all-pairs kernels."""
    n = 3000
    x, L = _periodic_system(n, 0.05, 700)
    b = tuple(L * f for f in box)
    F = inputs.normal_forces(n, 701)
    with sd.System(n, box=b, dense=dense) as s:
        assert s.dense_kernel() == dense
        s.set_positions(x)
        v = s.mobility_apply(F)
    ref = oracle.mobility_apply(x, F, "rpy", box=b, nthreads=8)
    assert periodic_rel_err(v, ref, x, F, b) <= TOL["fp32c"]


def test_periodic_images_are_equivalent():
    """Moving particles by whole periods does not change the velocities (the state is
    kept unwrapped; only the nearest image interacts)."""
    n = 2048
    x, L = _periodic_system(n, 0.08, 710, overlaps=0)
    F = inputs.normal_forces(n, 711)
    shift = L * np.random.default_rng(712).integers(-3, 4, x.shape)
    with sd.System(n, prec="fp64", box=(L, L, L)) as s:
        s.set_positions(x)
        v1 = s.mobility_apply(F)
        s.set_positions(x + shift)
        v2 = s.mobility_apply(F)
    assert periodic_rel_err(v2, v1, x, F, (L, L, L), margin=1e-12) <= 1e-13


def _odd_lattice(m=13, spacing=2.4, jitter=0.1, seed=720):
    """A jittered simple-cubic lattice filling a periodic cube of m (odd) cells per
    side.  Every separation component is a whole number of spacings plus at most
    2 jitter, while half a period is m/2 spacings, a half-integer number: no pair
    comes within spacing/2 - 2 jitter of a nearest-image tie, at any step of a
    short trajectory."""
    g1 = np.arange(m) * spacing
    x = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    x = x + np.random.default_rng(seed).uniform(-jitter, jitter, x.shape)
    return x, m * spacing


def _min_tie_distance(x, L):
    """Smallest distance, over pairs and dimensions, of a separation component's
    nearest image from half a period."""
    best = np.inf
    for i0 in range(0, x.shape[0], 256):
        d = x[i0:i0 + 256, None, :] - x[None, :, :]
        img = d - L * np.round(d / L)
        best = min(best, float(np.abs(np.abs(img) - 0.5 * L).min()))
    return best


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 2e-6)])
def test_periodic_steps_match_oracle(prec, tol):
    """Gravity + soft repulsion + random forces in a periodic box, 20 Euler steps
    (workload-3 physics, neighbours at 2.4a inside the repulsion range), at the
    gates of unbounded trajectories.  The start is a lattice with an odd number of
    cells per side, so no pair is ever near a nearest-image tie (half a period),
    where FP32 and FP64 separations may pick different, equally correct images;
    the oracle trajectory confirms the margin at the first and last step."""
    x0, L = _odd_lattice()
    n = x0.shape[0]
    box = (L, L, L)
    g = (0.0, 0.0, -1.0)
    fe = inputs.normal_forces(n, 721)
    ref = oracle.euler(x0, 20, 0.01, fe, g, rep_eps=1.0, rep_rc=2.5, box=box, nthreads=8)
    assert min(_min_tie_distance(x0, L), _min_tie_distance(ref, L)) > 0.5
    with sd.System(n, prec=prec, gravity=g, rep_eps=1.0, rep_rc=2.5, box=box) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(0.01, 20)
        xT = s.get_positions()
    disp = np.linalg.norm(ref - x0, axis=1).max()
    assert np.linalg.norm(xT - ref, axis=1).max() <= tol * disp


def test_periodic_random_packing_steps_tie_aware():
    """A random packing has a few pairs per step within FP32 rounding of half a
    period.  Each of 10 FP32C Euler steps is checked on its own: the step's
    velocities (x_{k+1} - x_k) / dt against the oracle's velocities at x_k, with
    the forces of x_k, under the tie-aware error of the apply tests."""
    n = 2500
    x0, L = inputs.cube_rsa(n, 0.10, 722)
    L = L + 2.5          # the packing is non-overlapping across the faces as well
    box = (L, L, L)
    g = (0.0, 0.0, -1.0)
    fe = inputs.normal_forces(n, 723)
    dt = 0.01
    with sd.System(n, prec="fp32c", gravity=g, rep_eps=1.0, rep_rc=2.5, box=box) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        xk = x0
        for k in range(10):
            s.step(dt, 1)
            x1 = s.get_positions()
            F = oracle.forces(xk, fe, g, rep_eps=1.0, rep_rc=2.5, box=box)
            ref = oracle.mobility_apply(xk, F, "rpy", box=box, nthreads=8)
            assert periodic_rel_err((x1 - xk) / dt, ref, xk, F, box) <= TOL["fp32c"], k
            xk = x1


def test_periodic_lubrication_lattice():
    """A jittered lattice filling a periodic box (every sphere has 6 neighbours inside
    the friction window, across the faces too): 10 steps with lubrication."""
    m, spacing = 8, 2.8
    g1 = np.arange(m) * spacing
    x0 = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    x0 = x0 + np.random.default_rng(730).uniform(-0.05, 0.05, x0.shape)
    n, L = x0.shape[0], m * spacing
    box = (L, L, L)
    fe = inputs.normal_forces(n, 731)
    ref = oracle.euler(x0, 10, 0.02, fe, box=box, lubrication=True, nthreads=8)
    with sd.System(n, prec="fp64", box=box, lubrication=True) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(0.02, 10)
        xT = s.get_positions()
    disp = np.linalg.norm(ref - x0, axis=1).max()
    assert np.linalg.norm(xT - ref, axis=1).max() <= 1e-10 * disp


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32c", 1e-5)])
def test_periodic_vjp_matches_oracle(prec, tol):
    n = 700
    x, L = _periodic_system(n, 0.05, 740)
    box = (L, L, L)
    F = inputs.normal_forces(n, 741)
    W = inputs.normal_forces(n, 742)
    with sd.System(n, prec=prec, box=box) as s:
        s.set_positions(x)
        gx, gF = s.vjp(F, W)
    rx, rF = oracle.vjp(x, F, W, "rpy", box=box, nthreads=8)
    assert rel_err(gF, rF) <= tol
    assert rel_err(gx, rx) <= 10 * tol


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_periodic_fcc_lattice_near_pairs(prec):
    """The paper's benchmark geometry (Sec. 3.3): an fcc lattice at number density
    0.1/a^3 in a periodic cube, every sphere with 12 neighbours at 2.42a < r_near
    (the near pass's list holds them all); jittered so that no pair sits at an exact
    half-period tie."""
    x, L = inputs.fcc_lattice(5)
    x = x + np.random.default_rng(750).uniform(-0.05, 0.05, x.shape)
    n = x.shape[0]
    box = (L, L, L)
    F = inputs.normal_forces(n, 751)
    with sd.System(n, prec=prec, box=box) as s:
        s.set_positions(x)
        v = s.mobility_apply(F)
    ref = oracle.mobility_apply(x, F, "rpy", box=box, nthreads=8)
    assert periodic_rel_err(v, ref, x, F, box) <= TOL[prec]
