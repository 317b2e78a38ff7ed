"""Adjoint on the GPU: vector-Jacobian products of v = mu(x) F and the reverse
sweep through Euler steps with checkpoints, against the FP64 oracle and central
finite differences."""
import numpy as np
import pytest

import oracle
import paper_1205_6333_gb300 as sd
from paper_1205_6333_gb300 import inputs
from helpers import rel_err, system_with_overlaps

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tensor", ["rpy", "rp", "oseen"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32c", 1e-5)])
def test_vjp_matches_oracle(tensor, prec, tol):
    n = 700
    x, _ = system_with_overlaps(n, 0.05, seed=61 + n, overlaps=4)
    F = inputs.normal_forces(n, 62)
    W = inputs.normal_forces(n, 63)
    with sd.System(n, tensor=tensor, prec=prec) as s:
        s.set_positions(x)
        gx, gF = s.vjp(F, W)
    rx, rF = oracle.vjp(x, F, W, tensor)
    assert rel_err(gF, rF) <= tol
    assert rel_err(gx, rx) <= 10 * tol


def _adjoint_case(n=64, seed=inputs.SEED_BASE + 5):
    x0, L = inputs.cube_rsa(n, 0.05, seed)
    target = x0 + np.random.default_rng(seed + 3).standard_normal(x0.shape)
    return x0, target


def test_adjoint_matches_oracle_n64():
    """Workload 5 protocol on an N=64 system: gravity, dt = 0.01, 1000 steps,
    L = sum |x(T) - x*|^2, checkpoints every 50 steps; full gradients."""
    x0, target = _adjoint_case()
    nsteps, dt, K = 1000, 0.01, 50
    g = (0.0, 0.0, -1.0)
    fe = np.zeros_like(x0)
    xT = oracle.euler(x0, nsteps, dt, fe, g)
    gxT = 2.0 * (xT - target)
    rx0, rF = oracle.adjoint(x0, fe, gxT, nsteps, dt, g)
    for prec, tol in [("fp64", 1e-9), ("fp32c", 1e-4)]:
        with sd.System(64, prec=prec, gravity=g) as s:
            s.set_positions(x0)
            gx0, gF = s.adjoint(dt, nsteps, K, gxT)
            np.testing.assert_array_equal(s.get_positions(), x0)   # state restored
        assert rel_err(gx0, rx0) <= tol, prec
        assert rel_err(gF, rF) <= tol, prec


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_adjoint_graphs_equal_eager(prec):
    """Full checkpoint segments replay cached graphs; with the profiler on every launch
    is eager.  Both give the same gradients bit for bit: a ragged last segment
    (nsteps not a multiple of K), K = 1 (no recompute part), a repeated call, and a
    call after sd_mobility_vjp has reallocated the staging buffer the graphs use."""
    n = 700
    x0, target = _adjoint_case(n, inputs.SEED_BASE + 7)
    g = (0.0, 0.0, -1.0)
    F = inputs.normal_forces(n, 8)
    with sd.System(n, prec=prec, gravity=g) as s:
        s.set_positions(x0)
        xT = x0 + 0.1
        gxT = 2.0 * (xT - target)
        for nsteps, K in [(40, 1), (130, 50), (100, 25)]:   # staging buffer 24n, then 96n (vjp), then 1200n B
            s.profile(True)
            ref = s.adjoint(0.01, nsteps, K, gxT)
            s.profile(False)
            got = s.adjoint(0.01, nsteps, K, gxT)          # captures the segment graphs
            again = s.adjoint(0.01, nsteps, K, gxT)        # replays them
            for a, b, c in zip(ref, got, again):
                np.testing.assert_array_equal(a, b)
                np.testing.assert_array_equal(a, c)
            s.vjp(F, gxT)                                   # host arrays: reallocates the staging buffer
            np.testing.assert_array_equal(s.adjoint(0.01, nsteps, K, gxT)[0], ref[0])
        np.testing.assert_array_equal(s.get_positions(), x0)


def test_adjoint_graphs_survive_host_apply_reallocation():
    """The adjoint's cached segment graphs read the handle's staging buffer.  With
    K = 1 that buffer holds one position array; a host-array mobility apply then
    needs two and reallocates it, which must drop the graphs: the next adjoint
    equals the eager one bit for bit."""
    n = 300
    x0, target = _adjoint_case(n, inputs.SEED_BASE + 9)
    F = inputs.normal_forces(n, 10)
    gxT = 2.0 * (x0 + 0.1 - target)
    with sd.System(n, prec="fp64", gravity=(0.0, 0.0, -1.0)) as s:
        s.set_positions(x0)
        s.profile(True)
        ref = s.adjoint(0.01, 12, 1, gxT)                  # eager
        s.profile(False)
        first = s.adjoint(0.01, 12, 1, gxT)                # captures the K = 1 graphs
        s.mobility_apply(F)                                # host arrays: staging buffer grows
        again = s.adjoint(0.01, 12, 1, gxT)
    for a, b, c in zip(ref, first, again):
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(a, c)


def test_adjoint_finite_differences_fp64():
    """Central differences (h = 1e-4) of the GPU FP64 trajectory loss."""
    x0, target = _adjoint_case()
    nsteps, dt, K, h = 1000, 0.01, 50, 1e-4
    g = (0.0, 0.0, -1.0)
    with sd.System(64, prec="fp64", gravity=g) as s:
        def loss(x, f):
            s.set_positions(x)
            s.set_forces(f)
            s.step(dt, nsteps)
            return float(((s.get_positions() - target) ** 2).sum())

        fe = np.zeros_like(x0)
        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, nsteps)
        xT = s.get_positions()
        s.set_positions(x0)
        gx0, gF = s.adjoint(dt, nsteps, K, 2.0 * (xT - target))
        rng = np.random.default_rng(7)
        for comp in rng.choice(64 * 3, 6, replace=False):
            i, d = divmod(int(comp), 3)
            e = np.zeros_like(x0)
            e[i, d] = h
            fdx = (loss(x0 + e, fe) - loss(x0 - e, fe)) / (2 * h)
            fdF = (loss(x0, fe + e) - loss(x0, fe - e)) / (2 * h)
            assert abs(gx0[i, d] - fdx) <= 1e-6 * max(abs(fdx), np.abs(gx0).max() * 1e-3)
            assert abs(gF[i, d] - fdF) <= 1e-6 * max(abs(fdF), np.abs(gF).max() * 1e-3)


def test_adjoint_finite_differences_workload5_n4096():
    """Workload 5 at its own size: N = 4,096 at volume fraction 0.05, gravity, 1000
    Euler steps at dt = 0.01, loss sum |x(T) - x*|^2, checkpoints every 50 steps.
    The FP64 adjoint against central differences (h = 1e-4) of the GPU FP64
    trajectory on three seeded components of x0 and of F, gate 1e-6."""
    w = inputs.config_inputs(5)
    x0, target = w["x"], w["target"]
    n = x0.shape[0]
    nsteps, dt, K, h = 1000, 0.01, 50, 1e-4
    fe = np.zeros_like(x0)
    with sd.System(n, prec="fp64", gravity=(0.0, 0.0, -1.0)) as s:
        def loss(x, f):
            s.set_positions(x)
            s.set_forces(f)
            s.step(dt, nsteps)
            return float(((s.get_positions() - target) ** 2).sum())

        s.set_positions(x0)
        s.set_forces(fe)
        s.step(dt, nsteps)
        xT = s.get_positions()
        s.set_positions(x0)
        gx0, gF = s.adjoint(dt, nsteps, K, 2.0 * (xT - target))
        rng = np.random.default_rng(inputs.SEED_BASE + 56)
        for comp in rng.choice(3 * n, 3, replace=False):
            i, d = divmod(int(comp), 3)
            e = np.zeros_like(x0)
            e[i, d] = h
            fdx = (loss(x0 + e, fe) - loss(x0 - e, fe)) / (2 * h)
            fdF = (loss(x0, fe + e) - loss(x0, fe - e)) / (2 * h)
            assert abs(gx0[i, d] - fdx) <= 1e-6 * max(abs(fdx), np.abs(gx0).max() * 1e-3), (i, d, gx0[i, d], fdx)
            assert abs(gF[i, d] - fdF) <= 1e-6 * max(abs(fdF), np.abs(gF).max() * 1e-3), (i, d, gF[i, d], fdF)


def test_adjoint_rejects_repulsion():
    with sd.System(8, rep_eps=1.0) as s:
        s.set_positions(np.arange(24, dtype=float).reshape(8, 3) * 3)
        with pytest.raises(sd.SDError) as ei:
            s.adjoint(0.01, 2, 1, np.ones((8, 3)))
        assert ei.value.status_name == "SD_ERR_UNSUPPORTED"


def test_torch_autograd_functions():
    """torch.autograd through the C ABI: the apply's VJP and the Euler trajectory's
    adjoint match the oracle."""
    import torch
    from paper_1205_6333_gb300.autograd import euler_trajectory, mobility_apply
    x0, target = _adjoint_case()
    n = x0.shape[0]
    with sd.System(n, prec="fp64", gravity=(0.0, 0.0, -1.0)) as s:
        x = torch.tensor(x0, device="cuda", requires_grad=True)
        F = torch.tensor(inputs.normal_forces(n, 71), device="cuda", requires_grad=True)
        W = inputs.normal_forces(n, 72)
        v = mobility_apply(s, x, F)
        (v * torch.tensor(W, device="cuda")).sum().backward()
        rx, rF = oracle.vjp(x0, F.detach().cpu().numpy(), W, "rpy")
        assert rel_err(x.grad.cpu().numpy(), rx) <= 1e-10
        assert rel_err(F.grad.cpu().numpy(), rF) <= 1e-10

        x = torch.tensor(x0, device="cuda", requires_grad=True)
        fe = torch.zeros((n, 3), dtype=torch.float64, device="cuda", requires_grad=True)
        xT = euler_trajectory(s, x, fe, 0.01, 200, 25)
        loss = ((xT - torch.tensor(target, device="cuda")) ** 2).sum()
        loss.backward()
        xr = oracle.euler(x0, 200, 0.01, np.zeros_like(x0), (0.0, 0.0, -1.0))
        gx0, gF = oracle.adjoint(x0, np.zeros_like(x0), 2.0 * (xr - target), 200, 0.01, (0.0, 0.0, -1.0))
        assert rel_err(x.grad.cpu().numpy(), gx0) <= 1e-9
        assert rel_err(fe.grad.cpu().numpy(), gF) <= 1e-9
