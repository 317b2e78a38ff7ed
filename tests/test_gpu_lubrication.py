"""Lubrication friction in sd_step (Sec. 2.3 Eq. lubrication; Sec. 3.1 step 2 with the
previous step's velocities) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_1205_6333_gb300 as sd
from paper_1205_6333_gb300 import inputs

pytestmark = pytest.mark.gpu


def _lattice(m, spacing=2.8, jitter=0.05, seed=0):
    """m^3 spheres on a jittered simple-cubic lattice: nearest-neighbour gaps s ~ 0.7-0.9,
    inside the friction window 0 < s < 1, diagonal neighbours beyond 3a.  The lagged
    friction of Sec. 3.1 is stable there; on closer lattices (spacing <= 2.7a) it
    diverges within tens of steps, in the oracle as on the GPU."""
    rng = np.random.default_rng(inputs.SEED_BASE + 60 + seed)
    g = np.arange(m) * spacing
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    return x + rng.uniform(-jitter, jitter, x.shape)


def _disp_err(xT, ref, x0):
    return np.linalg.norm(xT - ref, axis=1).max() / np.linalg.norm(ref - x0, axis=1).max()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32c", 2e-6)])
@pytest.mark.parametrize("m", [8, 16])   # N = 512 (directed kernel), 4096 (symmetric kernel)
def test_lubrication_trajectory_matches_oracle(prec, tol, m):
    x0 = _lattice(m, seed=m)
    n = x0.shape[0]
    fe = inputs.normal_forces(n, inputs.SEED_BASE + 61 + m)
    g = (0.0, 0.0, -1.0)
    steps, dt = 12, 0.02
    ref = oracle.euler(x0, steps, dt, fe, g, lubrication=True, nthreads=8)
    plain = oracle.euler(x0, steps, dt, fe, g, nthreads=8)
    assert _disp_err(plain, ref, x0) > 1e-3          # the friction changes the motion
    with sd.System(n, prec=prec, gravity=g, lubrication=True) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, steps)
        assert _disp_err(s.get_positions(), ref, x0) <= tol


def test_lubrication_with_repulsion_and_graph_replay():
    """Repulsion and friction in the same neighbour pass; 16 steps replayed from the
    captured graph equal 16 single steps bit for bit."""
    x0 = _lattice(8, seed=3)
    n = x0.shape[0]
    fe = inputs.normal_forces(n, inputs.SEED_BASE + 62)
    g = (0.0, 0.0, -1.0)
    ref = oracle.euler(x0, 16, 0.01, fe, g, rep_eps=0.5, rep_rc=3.0, lubrication=True, nthreads=8)
    out = []
    for chunks in ([16], [1] * 16):
        with sd.System(n, prec="fp64", gravity=g, rep_eps=0.5, rep_rc=3.0, lubrication=True) as s:
            s.set_positions(x0)
            s.set_forces(fe)
            for k in chunks:
                s.step(0.01, k)
            out.append(s.get_positions())
    np.testing.assert_array_equal(out[0], out[1])
    assert _disp_err(out[0], ref, x0) <= 1e-10


def test_set_positions_forgets_previous_velocities():
    """After sd_set_positions the next step has no friction, as at the start."""
    x0 = _lattice(6, seed=4)
    n = x0.shape[0]
    fe = inputs.normal_forces(n, inputs.SEED_BASE + 63)
    with sd.System(n, prec="fp64", lubrication=True) as s:
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(0.02, 5)
        x5 = s.get_positions()
        s.set_positions(x5)
        s.step(0.02, 5)
        xT = s.get_positions()
    ref = oracle.euler(x5, 5, 0.02, fe, lubrication=True)
    assert _disp_err(xT, ref, x5) <= 1e-10


def test_lubrication_unsupported_paths():
    with sd.System(64, prec="fp64", lubrication=True) as s:
        s.set_positions(_lattice(4))
        with pytest.raises(sd.SDError) as ei:
            s.adjoint(0.01, 2, 1, np.ones((64, 3)))
        assert ei.value.status_name == "SD_ERR_UNSUPPORTED"
    cfg, _ = sd._make_config(0, lubrication=True)
    with pytest.raises(sd.SDError) as ei:
        sd.sd_batch_create(cfg, np.array([0, 4], dtype=np.int32))
    assert ei.value.status_name == "SD_ERR_UNSUPPORTED"
