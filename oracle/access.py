"""Oracle of the memory-access study (App. A, Algorithms 3 and 4) -- test
infrastructure only: the tests, the smoke check and the CPU baseline of the
benchmark use it; the library never does.

What each study kernel computes, written as its definition: thread j of an
N-thread launch (blocks of B threads) returns

    out[j] = in[j] + sum over the N positions q of in[idx(q)]

where idx(q) = map(q, j) for the naive kernel (every thread reads its own
sequence), and for the tiling kernels the element at position q is the one the
thread that loads it fetched: in tiles of T elements (T = B for "tiling" and
the bulk variant, T = 32 for "smalltiling"), position q is loaded by thread
q mod T of the block, whose global index is jl = b B + (q mod T) for block b,
so idx(q) = map(q, jl).  The maps (Sec. A; p = 131, M = 32):

    linear     map(k, j) = k
    strided    map(k, j) = k p mod N
    unordered  map(k, j) = (k p + j M) mod N

float4 elements are summed componentwise.  Sums are formed in float64; with
integer-valued inputs whose partial sums stay below 2^24 in magnitude every
FP32 partial sum is exact as well, so the result does not depend on the order
of the additions and the GPU kernels must match it bit for bit.
"""
import numpy as np

P = 131   # the prime of the strided and unordered maps
M = 32    # the warp size of the unordered map
ALGOS = ("naive", "tiling", "smalltiling", "bulk")
MAPS = ("linear", "strided", "unordered")


def access_map(kind, k, j, N):
    """map(k, j) of App. A for integer arrays k, j (broadcast), as int64."""
    k = np.asarray(k, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    if kind == "linear":
        return np.broadcast_to(k, np.broadcast(k, j).shape) % N
    if kind == "strided":
        return np.broadcast_to(k * P, np.broadcast(k, j).shape) % N
    if kind == "unordered":
        return (k * P + j * M) % N
    raise ValueError(kind)


def access_study(algo, kind, data, block=128, rows=None, chunk=None):
    """out[j] of the study kernel `algo` under map `kind` (definition above).

    data: array of shape (N,) or (N, 4).  rows: the thread indices j to return
    (default all N), so that large launches can be checked on a sample.
    Returns float64 of shape (len(rows),) or (len(rows), 4)."""
    if algo not in ALGOS:
        raise ValueError(algo)
    if algo == "bulk" and kind != "linear":
        raise ValueError("the bulk kernel reads linear tiles only")
    x = np.asarray(data, dtype=np.float64)
    N = x.shape[0]
    rows = np.arange(N, dtype=np.int64) if rows is None else np.asarray(rows, dtype=np.int64)
    out = np.empty((rows.shape[0],) + x.shape[1:], dtype=np.float64)
    if rows.shape[0] == 0:
        return out
    q = np.arange(N, dtype=np.int64)
    tile = 32 if algo == "smalltiling" else block
    chunk = chunk or max(1, (1 << 22) // max(N, 1))   # rows per gather of at most 2^22 elements
    for c0 in range(0, rows.shape[0], chunk):
        j = rows[c0:c0 + chunk]
        if algo == "naive":
            loader = j[:, None]                              # every thread reads for itself
        else:
            loader = (j // block * block)[:, None] + (q % tile)[None, :]   # thread q mod T of j's block
        idx = access_map(kind, q[None, :], loader, N)
        out[c0:c0 + chunk] = x[j] + x[idx].sum(axis=1)
    return out
