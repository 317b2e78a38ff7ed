"""Pins of the memory-access study's oracle (App. A) against facts that do not
come from its own formula: closed forms of the three maps, a thread-by-thread
simulation of the kernels' programs (Algorithms 3 and 4) on tiny launches, and
the statement that "tiling" is "smalltiling" with the warp size replaced by
the block size.  A mutation check plants plausible mistakes in a copy of the
oracle and requires every one to fail a pin."""
import os
import types

import numpy as np
import pytest

import oracle.access as acc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ints(shape, seed, lo=-8, hi=9):
    return np.random.default_rng(seed).integers(lo, hi, shape).astype(np.float64)


def _simulate(algo, kind, x, block):
    """Run the study kernel's program one thread at a time: a shared array per block,
    the load phase and the accumulate phase separated as the barriers separate them."""
    N = x.shape[0]

    def mp(k, j):
        if kind == "linear":
            return k
        if kind == "strided":
            return (131 * k) % N
        return (131 * k + 32 * j) % N

    out = np.zeros_like(x)
    nblocks = -(-N // block)
    for b in range(nblocks):
        threads = range(b * block, (b + 1) * block)
        if algo == "naive":
            for j in threads:
                if j < N:
                    s = x[j].copy()
                    for k in range(N):
                        s = s + x[mp(k, j)]
                    out[j] = s
            continue
        T = 32 if algo == "smalltiling" else block
        sums = {j: (x[j].copy() if j < N else 0.0 * x[0]) for j in threads}
        for m in range(0, N, T):
            shared = [None] * T
            for n, jl in enumerate(threads):          # load phase
                if n < T:
                    shared[n] = x[mp(m + n, jl)] if m + n < N else 0.0 * x[0]
            for j in threads:                         # accumulate phase
                for k in range(T):
                    sums[j] = sums[j] + shared[k]
        for j in threads:
            if j < N:
                out[j] = sums[j]
    return out


def pin_constant_input(mod):
    """in = c everywhere: every kernel under every map returns (N + 1) c."""
    for N in (1, 37, 300):
        for algo in mod.ALGOS:
            for kind in mod.MAPS:
                if algo == "bulk" and kind != "linear":
                    continue
                got = mod.access_study(algo, kind, np.full(N, 3.0), block=64)
                assert np.array_equal(got, np.full(N, 3.0 * (N + 1))), (algo, kind, N)


def pin_permutation_maps(mod):
    """N coprime to 131: k -> k p mod N and k -> (k p + j M) mod N permute 0..N-1, so the
    naive kernel returns in[j] + sum(in) under all three maps."""
    for N in (100, 257, 1000):
        x = _ints((N, 4), N)
        want = x + x.sum(axis=0)
        for kind in mod.MAPS:
            assert np.array_equal(mod.access_study("naive", kind, x), want), (kind, N)


def pin_non_coprime_strided_and_unordered(mod):
    """N = 131 q: k p mod N hits each multiple of 131 exactly 131 times, and
    (k p + j M) mod N hits each index congruent to 32 j (mod 131) 131 times."""
    for q in (2, 3):
        N = 131 * q
        x = _ints(N, q)
        got = mod.access_study("naive", "strided", x)
        assert np.array_equal(got, x + 131 * x[::131].sum()), N
        got = mod.access_study("naive", "unordered", x)
        want = np.array([x[j] + 131 * x[(32 * j) % 131::131].sum() for j in range(N)])
        assert np.array_equal(got, want), N


def pin_simulation(mod):
    """Thread-by-thread runs of the programs on tiny ragged launches."""
    for N, block in ((70, 32), (100, 64), (131, 32)):
        x = _ints(N, 7 * N)
        for algo in ("naive", "tiling", "smalltiling"):
            for kind in mod.MAPS:
                got = mod.access_study(algo, kind, x, block=block)
                assert np.array_equal(got, _simulate(algo, kind, x, block)), (algo, kind, N, block)
        assert np.array_equal(mod.access_study("bulk", "linear", x, block=block),
                              _simulate("tiling", "linear", x, block))


def pin_tiling_is_smalltiling_at_warp_size(mod):
    """Algorithm 4: tiling is smalltiling with warpSize replaced by the block size."""
    x = _ints(500, 3)
    for kind in mod.MAPS:
        assert np.array_equal(mod.access_study("tiling", kind, x, block=32),
                              mod.access_study("smalltiling", kind, x, block=32)), kind


def pin_unordered_tiles_shared_by_block(mod):
    """With tiles every thread of a block adds the same staged elements: out[j] - in[j] is
    constant over each block, and (N coprime to 131, tiles within one block's loaders)
    differs between blocks."""
    N, block = 1000, 128
    x = _ints(N, 11)
    d = mod.access_study("tiling", "unordered", x, block=block) - x
    per_block = [np.unique(d[b:b + block]) for b in range(0, N, block)]
    assert all(u.size == 1 for u in per_block)
    assert len({float(u[0]) for u in per_block}) > 1


def pin_sampled_rows(mod):
    """rows= returns the same values as the whole launch."""
    x = _ints((777, 4), 5)
    rows = np.array([0, 1, 127, 128, 400, 776])
    for algo in ("naive", "tiling", "smalltiling"):
        full = mod.access_study(algo, "unordered", x, block=128)
        assert np.array_equal(mod.access_study(algo, "unordered", x, block=128, rows=rows), full[rows])


PINS = [pin_constant_input, pin_permutation_maps, pin_non_coprime_strided_and_unordered, pin_simulation,
        pin_tiling_is_smalltiling_at_warp_size, pin_unordered_tiles_shared_by_block, pin_sampled_rows]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_access_oracle_pin(pin):
    pin(acc)


def test_rejects_bulk_with_scattered_map():
    with pytest.raises(ValueError):
        acc.access_study("bulk", "strided", np.zeros(8))


def test_empty_launch():
    assert acc.access_study("tiling", "unordered", np.zeros(0)).shape == (0,)


# (name, text in oracle/access.py, replacement); the text must occur exactly once.
MUTANTS = [
    ("prime", "P = 131 ", "P = 127 "),
    ("warp_offset", "M = 32    #", "M = 31    #"),
    ("strided_as_linear", "return np.broadcast_to(k * P, ", "return np.broadcast_to(k * 1, "),
    ("unordered_offset_sign", "return (k * P + j * M) % N", "return (k * P - j * M) % N"),
    ("unordered_without_stride", "return (k * P + j * M) % N", "return (k + j * M) % N"),
    ("own_element_dropped", "out[c0:c0 + chunk] = x[j] + x[idx]", "out[c0:c0 + chunk] = x[idx]"),
    ("loader_is_reader", "loader = (j // block * block)[:, None] + (q % tile)[None, :]",
     "loader = j[:, None] + 0 * q[None, :]"),
    ("loader_block_offset_dropped", "loader = (j // block * block)[:, None] + (q % tile)[None, :]",
     "loader = 0 * j[:, None] + (q % tile)[None, :]"),
    ("smalltile_is_block", "tile = 32 if algo == \"smalltiling\" else block", "tile = block"),
    ("smalltile_is_16", "tile = 32 if algo == \"smalltiling\" else block",
     "tile = 16 if algo == \"smalltiling\" else block"),
    ("naive_uses_tiles", "if algo == \"naive\":\n            loader", "if algo == \"never\":\n            loader"),
    ("last_position_dropped", "q = np.arange(N, dtype=np.int64)", "q = np.arange(max(N - 1, 0), dtype=np.int64)"),
]


def _mutant_module(name, old, new):
    src = open(os.path.join(ROOT, "oracle", "access.py")).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType("access_mutant_" + name)
    exec(compile(src.replace(old, new), "access_mutant_" + name, "exec"), mod.__dict__)
    return mod


def test_pins_kill_every_access_mutant():
    survivors = []
    for name, old, new in MUTANTS:
        mod = _mutant_module(name, old, new)
        killed = False
        for pin in PINS:
            try:
                pin(mod)
            except Exception:
                killed = True
                break
        if not killed:
            survivors.append(name)
    assert not survivors, survivors
