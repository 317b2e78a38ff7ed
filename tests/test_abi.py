"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every symbol include/sd.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1205_6333_gb300 as sd
    return sd


def _declared():
    txt = open(os.path.join(ROOT, "include", "sd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sd_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["sd_create", "sd_destroy", "sd_set_positions", "sd_get_positions", "sd_set_forces",
                 "sd_mobility_apply", "sd_step", "sd_step_batched", "sd_adjoint", "sd_batch_create",
                 "sd_mobility_vjp", "sd_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(sd):
    lib = sd.lib()
    from paper_1205_6333_gb300 import _lib
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in _lib.PROTOTYPES, "binding lacks " + name


def test_config_defaults(sd):
    cfg = sd.sd_config_init()
    assert cfg.a == 1.0 and cfg.eta == 1.0
    assert cfg.tensor == sd.SD_TENSOR_RPY and cfg.prec == sd.SD_PREC_FP32C
    assert cfg.r_near == 2.5 and cfg.rep_eps == 0.0
    assert list(cfg.box) == [0.0, 0.0, 0.0]
    assert cfg.verlet_skin == 0.5
    assert "sm_103a" in sd.sd_version()


def test_config_struct_layout_matches_c(sd, tmp_path):
    """The ctypes mirror of sd_config has the C compiler's size and field offsets."""
    import subprocess
    fields = [f[0] for f in sd.sd_config._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sd.h"\nint main(void){printf("%zu'
                   + "".join(" %zu" for _ in fields) + '\\n", sizeof(sd_config)'
                   + "".join(", offsetof(sd_config, %s)" % f for f in fields) + ");return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got[0] == ctypes.sizeof(sd.sd_config)
    assert got[1:] == [getattr(sd.sd_config, f).offset for f in fields]


@pytest.mark.parametrize("field,value,status", [
    ("a", 0.0, 1), ("a", float("nan"), 1), ("eta", -1.0, 1), ("tensor", 7, 1), ("prec", 9, 1),
    ("n", -3, 1), ("r_near", 2.0, 1)])
def test_create_rejects_bad_config_on_host(sd, field, value, status):
    cfg = sd.sd_config_init()
    cfg.n = 10
    setattr(cfg, field, value)
    with pytest.raises(sd.SDError) as ei:
        sd.sd_create(cfg)
    assert ei.value.status == status
    assert sd.sd_last_error()


def test_periodic_box_validation(sd):
    """A periodic side shorter than three cell-list cells is an argument error (checked
    before any device work); batches have no periodic mode."""
    for box, lub in [((7.4, 0.0, 0.0), 0), ((20.0, 20.0, 8.9), 1)]:   # 3 x 2.5a, 3 x 3a
        cfg = sd.sd_config_init()
        cfg.n = 10
        cfg.lubrication = lub
        for d in range(3):
            cfg.box[d] = box[d]
        with pytest.raises(sd.SDError) as ei:
            sd.sd_create(cfg)
        assert ei.value.status_name == "SD_ERR_ARG"
    cfg = sd.sd_config_init()
    cfg.box[2] = 20.0
    with pytest.raises(sd.SDError) as ei:
        sd.sd_batch_create(cfg, [0, 4])
    assert ei.value.status_name == "SD_ERR_UNSUPPORTED"


def test_batch_rejects_oversized_clusters(sd):
    cfg = sd.sd_config_init()
    with pytest.raises(sd.SDError) as ei:
        sd.sd_batch_create(cfg, [0, 10, 300])
    assert ei.value.status_name == "SD_ERR_ARG"
    with pytest.raises(sd.SDError):
        sd.sd_batch_create(cfg, [1, 10])


def test_null_handles_are_rejected(sd):
    lib = sd.lib()
    assert lib.sd_step(None, 0.1, 1) == 1
    assert lib.sd_mobility_apply(None, None, None, 0, 0) == 1
    assert lib.sd_adjoint(None, 0.1, 1, 1, None, None, None, 0) == 1
    assert lib.sd_step_batched(None, 0.1, 1) == 1
    assert lib.sd_launch_count(None) == 0


def test_create_without_gpu_fails_cleanly(sd):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = sd.sd_config_init()
    cfg.n = 8
    with pytest.raises(sd.SDError) as ei:
        sd.sd_create(cfg)
    assert ei.value.status_name == "SD_ERR_CUDA"


@pytest.mark.parametrize("args", [
    (4, 0, 0, 64, 128),     # unknown algorithm
    (0, 3, 0, 64, 128),     # unknown map
    (3, 1, 0, 64, 128),     # bulk tiles with the strided map
    (3, 2, 1, 64, 128),     # bulk tiles with the unordered map
    (0, 0, 0, -1, 128),     # n < 0
    (1, 0, 0, 64, 48),      # block not a multiple of 32
    (1, 0, 0, 64, 2048),    # block above 1024
    (2, 0, 1, 64, 0),       # block 0
])
def test_access_study_rejects_bad_arguments_on_host(sd, args):
    """Every argument check of sd_access_run runs before any CUDA call."""
    algo, mp, vec4, n, block = args
    assert sd.lib().sd_access_run(algo, mp, vec4, n, block, 256, 512, None) == 1


def test_access_study_null_and_unaligned_pointers(sd):
    lib = sd.lib()
    assert lib.sd_access_run(0, 0, 0, 64, 128, None, 512, None) == 1
    assert lib.sd_access_run(0, 0, 0, 64, 128, 256, None, None) == 1
    assert lib.sd_access_run(3, 0, 0, 64, 128, 260, 512, None) == 1     # bulk input not 16-byte aligned
    assert lib.sd_access_run(1, 2, 1, 0, 128, None, None, None) == 0    # n = 0: nothing to launch
