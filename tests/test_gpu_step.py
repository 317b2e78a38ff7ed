"""Euler time stepping on the GPU (Sec. 3.1: positions, forces, velocities) against
the FP64 oracle; the four-sphere orbit of Sec. 4."""
import json
import os

import numpy as np
import pytest

import oracle
import paper_1205_6333_gb300 as sd
from paper_1205_6333_gb300 import inputs
from helpers import system_with_overlaps

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _run(x0, nsteps, dt, prec, gravity=(0, 0, -1.0), fext=None, rep_eps=0.0, tensor="rpy"):
    n = x0.shape[0]
    with sd.System(n, prec=prec, gravity=gravity, rep_eps=rep_eps, rep_rc=2.5, tensor=tensor) as s:
        s.set_positions(x0)
        if fext is not None:
            s.set_forces(fext)
        s.step(dt, nsteps)
        return s.get_positions()


@pytest.mark.parametrize("dt_unit", ["tau_s", "raw"])
def test_square_cluster_matches_oracle(dt_unit):
    """Four spheres on a horizontal square (side 4a, +-0.01a jitter), F=(0,0,-1),
    20,000 Euler steps; dt = 0.01 in units of tau_s = a/(mu0 F) (Sec. 3.3) or raw."""
    x0 = inputs.config_inputs(1)["x"]
    tau = 1.0 / oracle.mu0()
    dt = 0.01 * tau if dt_unit == "tau_s" else 0.01
    ref = oracle.euler(x0, 20000, dt, gravity=(0, 0, -1.0))
    g64 = _run(x0, 20000, dt, "fp64")
    assert np.abs(g64 - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())
    g32 = _run(x0, 20000, dt, "fp32c")
    assert np.abs(g32 - ref).max() <= 1e-6 * np.abs(ref - x0).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_four_sphere_orbit_on_gpu(prec):
    """Tory's orbit (Sec. 4): period ~517 tau_s, particles 1 and 3 stay in the xz plane."""
    g = json.load(open(os.path.join(GOLDEN, "four_sphere_orbit.json")))
    tau = 1.0 / oracle.mu0()
    dt = g["dt_tau_s"] * tau
    x = np.array(g["start"])
    traj = []
    chunk = 100
    with sd.System(4, prec=prec, tensor="rp", gravity=g["force"]) as s:
        s.set_positions(x)
        for _ in range(int(1000.0 / g["dt_tau_s"]) // chunk):
            s.step(dt, chunk)
            traj.append(s.get_positions())
    traj = np.array(traj)
    x1 = traj[:, 0, 0]
    k = np.nonzero((x1[1:-1] > x1[:-2]) & (x1[1:-1] >= x1[2:]))[0] + 1
    t = (k + 1) * chunk * g["dt_tau_s"]
    assert len(t) >= 2
    assert np.diff(t) == pytest.approx(np.full(len(t) - 1, g["period_tau_s"]), rel=0.01)
    drift = np.abs(traj[:, [0, 2], 1]).max()
    assert drift <= (1e-12 if prec == "fp64" else 1e-5)
    # and the oracle's trajectory at the sampled times
    ref = oracle.euler(np.array(g["start"]), len(traj) * chunk, dt, gravity=g["force"], tensor="rp", every=chunk)[1]
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert np.abs(traj - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 1e-5)])
def test_repulsion_gravity_matches_oracle(prec, tol):
    """Workload-3 physics at a size the oracle integrates in seconds: phi = 0.10,
    gravity + eps (2a/r)^12 repulsion cut at 2.5a, dt = 1e-3, 100 steps."""
    n = 2048
    x0, _ = inputs.cube_rsa(n, 0.10, inputs.SEED_BASE + 3)
    ref = oracle.euler(x0, 100, 1e-3, gravity=(0, 0, -1.0), rep_eps=1.0, rep_rc=2.5, nthreads=8)
    got = _run(x0, 100, 1e-3, prec, rep_eps=1.0)
    assert np.abs(got - ref).max() <= tol * np.abs(ref - x0).max()


def test_repulsion_gravity_full_size_steps():
    """Workload 3 at full size (N = 16,384, phi = 0.10, gravity + repulsion, dt = 1e-3),
    in the FP32C step as the drift run takes it: 16 steps (one replay of the captured
    16-step graph) against the oracle's trajectory."""
    w = inputs.config_inputs(3)
    x0 = w["x"]
    ref = oracle.euler(x0, 16, 1e-3, gravity=(0, 0, -1.0), rep_eps=1.0, rep_rc=2.5, nthreads=8)
    got = _run(x0, 16, 1e-3, "fp32c", rep_eps=1.0)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref - x0).max()


def test_external_forces_and_overlaps_step():
    n = 900
    x0, _ = system_with_overlaps(n, 0.05, seed=21, overlaps=5)
    fe = inputs.normal_forces(n, seed=22)
    ref = oracle.euler(x0, 7, 0.05, fext=fe, gravity=(0.1, 0, -0.5))
    got = _run(x0, 7, 0.05, "fp32c", gravity=(0.1, 0, -0.5), fext=fe)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref - x0).max()


def test_graph_replay_equals_eager_steps():
    """16-step graphs + single-step graphs, single-step graphs alone, and eager
    launches (the profiler's mode) give the same trajectory bit for bit."""
    n = 1000
    x0, _ = inputs.cube_rsa(n, 0.05, 31)
    with sd.System(n, gravity=(0, 0, -1.0), rep_eps=1.0) as s:
        s.set_positions(x0)
        s.step(0.01, 35)          # two 16-step replays + 3 single-step replays
        a = s.get_positions()
        s.set_positions(x0)
        for _ in range(35):
            s.step(0.01, 1)
        b = s.get_positions()
        s.set_positions(x0)
        s.profile(True)           # eager launches, one event pair per kernel family
        s.step(0.01, 35)
        s.profile(False)
        e = s.get_positions()
        np.testing.assert_array_equal(a, e)
        c0 = s.launch_count()
        s.step(0.01, 16)
        s.synchronize()
        assert s.launch_count() > c0
    np.testing.assert_array_equal(a, b)


def test_profiler_times_kernels():
    n = 4096
    x0, _ = inputs.cube_rsa(n, 0.05, 41)
    with sd.System(n, gravity=(0, 0, -1.0)) as s:
        s.set_positions(x0)
        s.profile(True)
        s.step(0.01, 3)
        ms, cnt = s.profile_read(sd.SD_KERNEL_DENSE)
        assert cnt == 3 and ms > 0
        ms_e, cnt_e = s.profile_read(sd.SD_KERNEL_EPILOGUE)
        assert cnt_e == 3 and ms_e > 0
        ms_n, cnt_n = s.profile_read(sd.SD_KERNEL_NEAR)
        assert cnt_n == 3 and ms_n > 0
        s.profile(False)


def test_checkpoint_resume_is_exact():
    """Positions read back and set again resume the trajectory bit for bit."""
    n = 700
    x0, _ = inputs.cube_rsa(n, 0.05, 51)
    with sd.System(n, gravity=(0, 0, -1.0)) as s:
        s.set_positions(x0)
        s.step(0.02, 40)
        full = s.get_positions()
        s.set_positions(x0)
        s.step(0.02, 17)
        mid = s.get_positions()
    with sd.System(n, gravity=(0, 0, -1.0)) as s2:
        s2.set_positions(mid)
        s2.step(0.02, 23)
        np.testing.assert_array_equal(s2.get_positions(), full)


def _verlet_case(n=1500, seed=61):
    """A loose packing under strong random forces: relative displacements pass half
    the skin every few steps, so lists are both reused and rebuilt."""
    x0, _ = inputs.cube_rsa(n, 0.08, seed)
    fe = 40.0 * inputs.normal_forces(n, seed + 1)
    return x0, fe


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_verlet_lists_graph_eager_and_no_reuse_agree(prec):
    """Neighbour lists reused across steps give the same trajectory bit for bit in graph
    replays, single steps and eager steps, and agree with lists built every step
    without a skin to the last bits; against the oracle as usual."""
    x0, fe = _verlet_case()
    n, steps, dt = x0.shape[0], 48, 0.01
    with sd.System(n, prec=prec, gravity=(0, 0, -1.0)) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, steps)                 # three 16-step graph replays
        a = s.get_positions()
        s.set_positions(x0)
        for _ in range(steps):
            s.step(dt, 1)                 # single-step graph replays
        b = s.get_positions()
        s.set_positions(x0)
        s.profile(True)                   # eager launches
        s.step(dt, steps)
        s.profile(False)
        e = s.get_positions()
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, e)
    with sd.System(n, prec=prec, gravity=(0, 0, -1.0), verlet_skin=0) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, steps)
        c = s.get_positions()
    disp = np.abs(a - x0).max()
    rel = (a - x0) - (a[0] - x0[0])
    assert np.linalg.norm(rel, axis=1).max() > 1.0   # relative motion of several half skins
    assert np.abs(a - c).max() <= (1e-13 if prec == "fp64" else 1e-6) * disp
    ref = oracle.euler(x0, steps, dt, fext=fe, gravity=(0, 0, -1.0), nthreads=8)
    assert np.abs(a - ref).max() <= (1e-10 if prec == "fp64" else 1e-5) * np.abs(ref - x0).max()


@pytest.mark.parametrize("dense", ["directed", "symmetric"])
@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_verlet_clamp_flag_from_the_list(prec, dense):
    """A pair driven past each other comes closer than r_safe = 1a and separates again,
    so the all-pairs kernel's clamp-every-tile flag turns on and off during the run.
    In a Verlet step that flag comes from the step's check kernel, which scans the
    last list, while the near pass runs beside the all-pairs kernel.  Graph replays,
    single steps and eager steps agree bit for bit; the lists rebuilt every step
    without a skin and the oracle agree as usual."""
    n, steps, dt = 600, 64, 0.01
    x0, _ = inputs.cube_rsa(n, 0.05, 81)
    x0[1] = x0[0] + np.array([2.0, 0.3, 0.0])   # closer than 1a in steps 14 .. 53 (oracle)
    fe = inputs.normal_forces(n, 82)
    fe[0] = [250.0, 0.0, 0.0]
    fe[1] = [-250.0, 0.0, 0.0]
    runs = []
    with sd.System(n, prec=prec, dense=dense) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, steps)
        runs.append(s.get_positions())
        s.set_positions(x0)
        for _ in range(steps):
            s.step(dt, 1)
        runs.append(s.get_positions())
        s.set_positions(x0)
        s.profile(True)
        s.step(dt, steps)
        s.profile(False)
        runs.append(s.get_positions())
    np.testing.assert_array_equal(runs[0], runs[1])
    np.testing.assert_array_equal(runs[0], runs[2])
    a = runs[0]
    assert np.linalg.norm(a[0] - a[1]) > 1.2 and a[0, 0] - a[1, 0] > 1.0   # passed and apart again
    with sd.System(n, prec=prec, dense=dense, verlet_skin=0) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, steps)
        c = s.get_positions()
    disp = np.abs(a - x0).max()
    assert np.abs(a - c).max() <= (1e-13 if prec == "fp64" else 1e-6) * disp
    ref = oracle.euler(x0, steps, dt, fext=fe, nthreads=8)
    assert np.abs(a - ref).max() <= (1e-10 if prec == "fp64" else 1e-5) * np.abs(ref - x0).max()


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_verlet_lists_with_repulsion(prec):
    """Soft repulsion with Verlet lists: the repulsive pairs come from the near-pair list
    (their cutoff 2.5a equals r_near).  A dense packing under gravity and strong random
    forces, so pairs enter and leave the cutoff and the list is rebuilt.  Graph replays,
    single steps and eager steps agree bit for bit; the cell-list forces of steps
    without a skin and the oracle agree to rounding."""
    n, steps, dt = 1500, 48, 0.005
    x0, _ = inputs.cube_rsa(n, 0.15, 63)
    fe = 20.0 * inputs.normal_forces(n, 64)
    kw = dict(prec=prec, gravity=(0, 0, -1.0), rep_eps=1.0, rep_rc=2.5)
    runs = []
    with sd.System(n, **kw) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, steps)
        runs.append(s.get_positions())
        s.set_positions(x0)
        for _ in range(steps):
            s.step(dt, 1)
        runs.append(s.get_positions())
        s.set_positions(x0)
        s.profile(True)
        s.step(dt, steps)
        s.profile(False)
        runs.append(s.get_positions())
    np.testing.assert_array_equal(runs[0], runs[1])
    np.testing.assert_array_equal(runs[0], runs[2])
    a = runs[0]
    with sd.System(n, verlet_skin=0, **kw) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, steps)
        c = s.get_positions()
    disp = np.abs(a - x0).max()
    assert np.abs(a - c).max() <= (1e-12 if prec == "fp64" else 1e-6) * disp
    ref = oracle.euler(x0, steps, dt, fext=fe, gravity=(0, 0, -1.0), rep_eps=1.0, rep_rc=2.5, nthreads=8)
    assert np.abs(a - ref).max() <= (1e-10 if prec == "fp64" else 1e-5) * np.abs(ref - x0).max()


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_verlet_lists_with_lubrication(prec):
    """Lubrication with Verlet lists: the lubricated pairs (s < 1, r < 3a) come from the
    near-pair list, whose cutoff is then 3a + skin.  A jittered lattice of spacing 2.9a
    (every nearest-neighbour gap inside the friction window) under random forces and
    gravity, dt = 0.02, with the previous step's velocities.  Graph replays and eager
    steps agree bit for bit; the cell-list forces of steps without a skin and the oracle
    agree to rounding."""
    m, spacing, steps, dt = 10, 2.9, 24, 0.02
    rng = np.random.default_rng(65)
    g = np.arange(m) * spacing
    x0 = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + rng.uniform(-0.05, 0.05, (m ** 3, 3))
    n = x0.shape[0]
    fe = inputs.normal_forces(n, 66)
    kw = dict(prec=prec, gravity=(0, 0, -1.0), lubrication=True)
    runs = []
    with sd.System(n, **kw) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, steps)
        runs.append(s.get_positions())
        s.set_positions(x0)
        s.profile(True)
        s.step(dt, steps)
        s.profile(False)
        runs.append(s.get_positions())
    np.testing.assert_array_equal(runs[0], runs[1])
    a = runs[0]
    with sd.System(n, verlet_skin=0, **kw) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, steps)
        c = s.get_positions()
    disp = np.abs(a - x0).max()
    assert np.abs(a - c).max() <= (1e-12 if prec == "fp64" else 1e-6) * disp
    ref = oracle.euler(x0, steps, dt, fext=fe, gravity=(0, 0, -1.0), lubrication=True, nthreads=8)
    assert np.abs(a - ref).max() <= (1e-10 if prec == "fp64" else 1e-4) * np.abs(ref - x0).max()


def test_verlet_lists_periodic_box():
    x0, L = inputs.cube_rsa(2000, 0.08, 71)
    L = L + 2.5
    box = (L, L, L)
    fe = 10.0 * inputs.normal_forces(2000, 72)
    with sd.System(2000, prec="fp64", box=box) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(0.01, 32)
        xT = s.get_positions()
    ref = oracle.euler(x0, 32, 0.01, fext=fe, box=box, nthreads=8)
    assert np.abs(xT - ref).max() <= 1e-10 * np.abs(ref - x0).max()
