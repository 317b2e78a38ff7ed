"""Failure detection without a GPU fault: bounded device waits that run out and
allocation failures reported through the allocator callbacks.

The time-out is made on purpose by a host switch (sd_inject_stall): the first CTA
of each all-pairs launch skips the bulk copy of its first tile, so its bounded
waits give up after the watchdog limit; the kernel records the time-out, drains
the copies it did issue and exits.  The context stays usable, and the same handle
then computes correct velocities again."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1205_6333_gb300 as sd
from paper_1205_6333_gb300 import _lib, inputs
from helpers import TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,dense", [("fp32c", "symmetric"), ("fp32c", "directed"), ("fp64", "symmetric"),
                                        ("fp64", "directed")])
def test_bounded_wait_times_out_and_handle_recovers(prec, dense):
    n = 3000
    x, _ = inputs.cube_rsa(n, 0.05, 401)
    F = inputs.normal_forces(n, 402)
    with sd.System(n, prec=prec, dense=dense, gravity=(0.0, 0.0, -1.0)) as s:
        s.set_positions(x)
        s.set_watchdog(2000)
        s.inject_stall(True)
        with pytest.raises(sd.SDError) as ei:
            s.mobility_apply(F)                 # host arrays: synchronises, reads the error word
        assert ei.value.status_name == "SD_ERR_TIMEOUT"
        s.step(0.01, 3)                         # asynchronous, through a step graph captured with the stall
        with pytest.raises(sd.SDError) as ei:
            s.synchronize()
        assert ei.value.status_name == "SD_ERR_TIMEOUT"
        s.synchronize()                         # the error word was cleared when reported
        s.inject_stall(False)
        s.set_watchdog(1 << 22)
        s.set_positions(x)                      # the stalled steps left invalid positions
        v = s.mobility_apply(F)
        s.step(0.01, 1)
        x1 = s.get_positions()
    assert rel_err(v, oracle.mobility_apply(x, F, "rpy", nthreads=8)) <= TOL[prec]
    ref1 = oracle.euler(x, 1, 0.01, gravity=(0.0, 0.0, -1.0), nthreads=8)
    assert np.abs(x1 - ref1).max() <= 10 * TOL[prec] * np.abs(ref1 - x).max()


class _CountingAllocator:
    """Allocator callbacks backed by torch's caching allocator that can be told to fail."""

    def __init__(self):
        import torch
        self.torch = torch
        self.fail = False
        self.fail_after = None      # fail every call after this many
        self.live = set()
        self.calls = 0
        self.alloc_fn = _lib.ALLOC_FN(self._alloc)
        self.free_fn = _lib.FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        self.calls += 1
        if self.fail or (self.fail_after is not None and self.calls > self.fail_after):
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), 0, self.torch.cuda.current_stream(0))
        self.live.add(p)
        return p

    def _free(self, ptr, ctx):
        self.live.discard(ptr)
        self.torch.cuda.caching_allocator_delete(ptr)

    def config(self, n, **kw):
        cfg = sd.sd_config_init()
        cfg.n = n
        for k, v in kw.items():
            setattr(cfg, k, v)
        cfg.alloc, cfg.free = self.alloc_fn, self.free_fn
        return cfg


def test_allocation_failure_in_create_returns_oom():
    al = _CountingAllocator()
    al.fail = True
    with pytest.raises(sd.SDError) as ei:
        sd.sd_create(al.config(1000))
    assert ei.value.status_name == "SD_ERR_OOM"
    assert al.calls >= 1 and not al.live
    with pytest.raises(sd.SDError) as ei:
        sd.sd_batch_create(al.config(0), np.array([0, 10, 30], dtype=np.int32))
    assert ei.value.status_name == "SD_ERR_OOM"
    # failing part-way: the buffers allocated before the failure are released
    al2 = _CountingAllocator()
    al2.fail_after = 5
    with pytest.raises(sd.SDError) as ei:
        sd.sd_create(al2.config(1000))
    assert ei.value.status_name == "SD_ERR_OOM"
    assert al2.calls > 5 and not al2.live


def test_allocation_failure_in_adjoint_returns_oom_then_recovers():
    n, nsteps, dt, K = 64, 40, 0.01, 10
    x0, _ = inputs.cube_rsa(n, 0.05, 411)
    gxT = inputs.normal_forces(n, 412)
    al = _CountingAllocator()
    cfg = al.config(n)
    cfg.prec = sd.SD_PREC_FP64
    cfg.gravity[2] = -1.0
    h = sd.sd_create(cfg)
    try:
        xa = np.ascontiguousarray(x0)
        sd.sd_set_positions(h, xa.ctypes.data, 0)
        g0, gF = np.empty_like(x0), np.empty_like(x0)
        ga = np.ascontiguousarray(gxT)
        al.fail = True                      # the checkpoints are allocated on first use
        with pytest.raises(sd.SDError) as ei:
            sd.sd_adjoint(h, dt, nsteps, K, ga.ctypes.data, g0.ctypes.data, gF.ctypes.data, 0)
        assert ei.value.status_name == "SD_ERR_OOM"
        al.fail = False
        sd.sd_adjoint(h, dt, nsteps, K, ga.ctypes.data, g0.ctypes.data, gF.ctypes.data, 0)
    finally:
        sd.sd_destroy(h)
    assert not al.live                      # every buffer went back through the free callback
    rx0, rF = oracle.adjoint(x0, np.zeros_like(x0), gxT, nsteps, dt, (0.0, 0.0, -1.0))
    assert rel_err(g0, rx0) <= 1e-9
    assert rel_err(gF, rF) <= 1e-9
