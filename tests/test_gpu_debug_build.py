"""The debug build of the library (libsd_gb300_debug.so, compiled with -DSD_DEBUG):
its kernels check every data-dependent index (cell list, near-pair list,
partial-sum slots and source-side rows, batched staging) and would report a
violation as SD_ERR_INTERNAL.  A child process loads that build (SD_LIBRARY) and
runs the paths that use those indices against the FP64 oracle: both all-pairs
kernels in FP32C and FP64, a periodic box, a near-pair list that overflows, Euler
steps with repulsion, the VJP, tile shards and a batch of clusters.  Every call
must succeed (no check fires on valid input) and match the oracle."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _child():
    sys.path[:0] = [ROOT, HERE]
    import torch

    import oracle
    import paper_1205_6333_gb300 as sd
    from paper_1205_6333_gb300 import _lib, inputs
    from helpers import TOL, periodic_rel_err, rel_err, system_with_overlaps

    assert _lib.LIB_PATH.endswith("libsd_gb300_debug.so"), _lib.LIB_PATH
    n = 3000
    x, L = system_with_overlaps(n, 0.05, seed=980, overlaps=5)
    F = inputs.normal_forces(n, 981)
    ref = oracle.mobility_apply(x, F, "rpy", nthreads=8)
    for prec, dense in [("fp32c", "symmetric"), ("fp32c", "directed"), ("fp64", "symmetric"), ("fp64", "directed")]:
        with sd.System(n, prec=prec, dense=dense) as s:
            s.set_positions(x)
            assert rel_err(s.mobility_apply(F), ref) <= TOL[prec], (prec, dense)
            Ft = torch.tensor(F, device="cuda")
            Pall = torch.stack([s.mobility_apply_part(Ft, r, 3) for r in range(3)])
            assert rel_err(s.mobility_apply_combine(Pall).cpu().numpy(), ref) <= TOL[prec], (prec, dense, "shards")
    box = (max(L, 10.0),) * 3
    xp = x + box[0] * np.random.default_rng(982).integers(-1, 2, x.shape)
    with sd.System(n, box=box) as s:
        s.set_positions(xp)
        v = s.mobility_apply(F)
    assert periodic_rel_err(v, oracle.mobility_apply(xp, F, "rpy", box=box, nthreads=8), xp, F, box) <= 1e-5
    # a crowded cluster: the near-pair list overflows and the in-place path runs
    xc = np.random.default_rng(983).uniform(0.0, 10.0, (1500, 3))
    Fc = inputs.normal_forces(1500, 984)
    with sd.System(1500) as s:
        s.set_positions(xc)
        assert rel_err(s.mobility_apply(Fc), oracle.mobility_apply(xc, Fc, "rpy", nthreads=8)) <= 1e-5
    # Euler steps with gravity and soft repulsion (cell-list walks of the force pass)
    x0, _ = inputs.cube_rsa(2500, 0.10, 985)
    g = (0.0, 0.0, -1.0)
    xr = oracle.euler(x0, 10, 0.02, gravity=g, rep_eps=1.0, rep_rc=2.5, nthreads=8)
    with sd.System(2500, gravity=g, rep_eps=1.0, rep_rc=2.5) as s:
        s.set_positions(x0)
        s.step(0.02, 10)
        xT = s.get_positions()
    assert np.abs(xT - xr).max() <= 1e-5 * np.abs(xr - x0).max()
    # VJP
    W = inputs.normal_forces(n, 986)
    with sd.System(n, prec="fp64") as s:
        s.set_positions(x)
        gx, gF = s.vjp(F, W)
    rx, rF = oracle.vjp(x, F, W, "rpy")
    assert rel_err(gF, rF) <= 1e-11 and rel_err(gx, rx) <= 1e-10
    # a batch of clusters of sizes 0 .. 256
    sizes = inputs.cluster_sizes(200, 0, 256, 987)
    xb, off = inputs.ball_rsa_batch(sizes, 0.05, 988)
    Fb = inputs.normal_forces(xb.shape[0], 989)
    b = sd.Batch(off)
    try:
        b.set_positions(xb)
        b.set_forces(Fb)
        b.step(0.01, 3)
        xb1 = b.get_positions()
    finally:
        b.close()
    for c in range(len(sizes)):
        lo, hi = off[c], off[c + 1]
        if hi > lo:
            rb = oracle.euler(xb[lo:hi], 3, 0.01, fext=Fb[lo:hi])
            assert np.abs(xb1[lo:hi] - rb).max() <= 1e-5 * max(np.abs(rb - xb[lo:hi]).max(), 1e-300), c
    print("debug build ok")


def test_debug_build_runs_clean_against_oracle():
    from paper_1205_6333_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, SD_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "child"], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug build ok" in r.stdout


if __name__ == "__main__" and sys.argv[1:] == ["child"]:
    _child()
