"""The allocation-free mobility product, sd_mobility_apply_noalloc.

Some callers cannot allocate GPU memory: code running while a stream is
captured into a CUDA graph, plug-ins held to a fixed device-memory budget, and
loops that cannot take cudaMalloc's synchronisation.  This entry point works
out of a static device array instead of handle buffers.  Its results must agree
with the handle-based sd_mobility_apply (FP32-compensated) within the FP32C
tolerance, call after call, although the second call reuses the scratch array
the first one left behind.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import paper_1205_6333_gb300 as sd
from paper_1205_6333_gb300 import inputs
from helpers import TOL, rel_err, system_with_overlaps

pytestmark = pytest.mark.gpu


def _noalloc(x, F, tensor):
    import torch
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    Ft = torch.tensor(F, dtype=torch.float64, device="cuda")
    Vt = torch.full_like(xt, float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    sd.sd_mobility_apply_noalloc(xt.data_ptr(), Ft.data_ptr(), Vt.data_ptr(), x.shape[0], 1.0, 1.0, tensor, stream)
    torch.cuda.synchronize()
    return Vt.cpu().numpy()


def _handle_apply(x, F, tensor):
    with sd.System(x.shape[0], tensor=tensor, prec="fp32c") as s:
        s.set_positions(x)
        return s.mobility_apply(F)


@pytest.mark.parametrize("tensor", ["rpy", "rp", "oseen"])
def test_noalloc_matches_handle_apply_on_two_calls(tensor):
    # first call: a larger system with overlapping pairs; second call: a smaller
    # one, so it runs over the scratch contents the first call left
    cases = [system_with_overlaps(5000, 0.05, seed=301, overlaps=4)[0],
             system_with_overlaps(1234, 0.10, seed=302, overlaps=2)[0] + 50.0]
    for k, x in enumerate(cases):
        F = inputs.normal_forces(x.shape[0], 303 + k)
        v = _noalloc(x, F, tensor)
        ref = _handle_apply(x, F, tensor)
        assert np.all(np.isfinite(v))
        assert rel_err(v, ref) <= TOL["fp32c"], (k, rel_err(v, ref))
        assert rel_err(v, oracle.mobility_apply(x, F, tensor)) <= TOL["fp32c"]


def test_noalloc_rejects_oversized_systems():
    with pytest.raises(sd.SDError) as ei:
        sd.sd_mobility_apply_noalloc(0, 0, 0, 65537)
    assert ei.value.status_name == "SD_ERR_ARG"
    assert "65536" in sd.sd_last_error()


def test_noalloc_at_its_size_limit():
    # n = 65,536 fills the scratch stride and all eight splits; separations taken
    # relative to particle 0 are least accurate here (cube side 176a)
    x, _ = inputs.cube_rsa(65536, 0.05, seed=311)
    F = inputs.normal_forces(65536, 312)
    v = _noalloc(x, F, "rpy")
    assert np.all(np.isfinite(v))
    assert rel_err(v, _handle_apply(x, F, "rpy")) <= TOL["fp32c"]
    rows = np.sort(np.random.default_rng(313).choice(65536, 192, replace=False))
    ref = oracle.mobility_rows(x, F, rows, "rpy")
    assert rel_err(v[rows], ref) <= TOL["fp32c"]


def test_noalloc_coincident_spheres_rpy():
    # two distinct spheres at the same point: the RPY overlap form gives T(0) = mu0 I
    x, _ = inputs.cube_rsa(300, 0.05, seed=321)
    x[7] = x[3]
    x[11] = x[10] + np.array([0.3, 0.0, 0.0])
    F = inputs.normal_forces(300, 322)
    v = _noalloc(x, F, "rpy")
    assert rel_err(v, oracle.mobility_apply(x, F, "rpy")) <= TOL["fp32c"]
