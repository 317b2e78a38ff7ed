"""The memory-access study kernels (App. A, Algorithms 3 and 4) against their
oracle through the C ABI: bit-exact on integer-valued inputs, whose FP32
partial sums are all exact, for every kernel, map and element type, on ragged
launches and at the study's largest size on sampled threads."""
import numpy as np
import pytest

import oracle.access as acc
import paper_1205_6333_gb300 as sd

pytestmark = pytest.mark.gpu

COMBOS = [(a, m) for a in acc.ALGOS for m in acc.MAPS if a != "bulk" or m == "linear"]


def _data(n, vec4, seed):
    shape = (n, 4) if vec4 else (n,)
    return np.random.default_rng(seed).integers(-8, 9, shape).astype(np.float32)


def _run(algo, kind, x, block):
    import torch
    d = torch.from_numpy(x).cuda()
    out = sd.access_study(algo, kind, d, block=block)
    torch.cuda.synchronize()
    sd.sd_access_status()
    return out.cpu().numpy()


@pytest.mark.parametrize("vec4", [False, True])
@pytest.mark.parametrize("algo,kind", COMBOS)
@pytest.mark.parametrize("n", [1, 31, 1000, 4133])
def test_access_kernels_match_oracle(algo, kind, vec4, n):
    x = _data(n, vec4, 100 + n)
    got = _run(algo, kind, x, 128)
    want = acc.access_study(algo, kind, x, block=128)
    np.testing.assert_array_equal(got, want.astype(np.float32))


@pytest.mark.parametrize("block", [32, 96, 256, 1024])
@pytest.mark.parametrize("algo,kind", COMBOS)
def test_access_block_sizes(algo, kind, block):
    n = 3 * block + 17
    x = _data(n, True, block)
    np.testing.assert_array_equal(_run(algo, kind, x, block),
                                  acc.access_study(algo, kind, x, block=block).astype(np.float32))


@pytest.mark.parametrize("vec4", [False, True])
@pytest.mark.parametrize("algo,kind", COMBOS)
def test_access_study_size_sampled(algo, kind, vec4):
    """N = 70,000 (the top of the study's range) and 128 threads per block, as timed:
    threads of the first, a middle and the ragged last block against the oracle."""
    n, block = 70000, 128
    x = _data(n, vec4, 7)
    got = _run(algo, kind, x, block)
    rows = np.concatenate([np.arange(0, 130), np.arange(35000, 35130), np.arange(n - 200, n)])
    want = acc.access_study(algo, kind, x, block=block, rows=rows)
    np.testing.assert_array_equal(got[rows], want.astype(np.float32))


def test_access_rejects_unaligned_bulk_input():
    import torch
    d = torch.zeros(65, device="cuda")
    out = torch.zeros(64, device="cuda")
    with pytest.raises(sd.SDError) as ei:
        sd.sd_access_run("bulk", "linear", False, 64, 128, d.data_ptr() + 4, out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    assert ei.value.status_name == "SD_ERR_ARG"
