"""The serving loop's device arena (csrc/sell_arena.h), on the CPU.

The server admits a request only if its x block, y block and long-row scratch
fit in one arena allocated at creation, so the HBM budget holds as long as the
arena never hands out overlapping or out-of-range memory.  The arena is
host-only C++; this test builds it with g++ behind a small C harness and runs
random allocate/release sequences against a brute-force model of the same
policy: 256-byte units, first fit over maximal free ranges in offset order.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1307_6209_gb300", "csrc")
UNIT = 256


@pytest.fixture(scope="module")
def arena(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("arena") / "libarena.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(ROOT, "tests", "native", "arena_harness.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    sz = ctypes.c_size_t
    lib.arena_reset.argtypes = [sz]
    lib.arena_alloc.argtypes = [sz, ctypes.POINTER(sz)]
    lib.arena_alloc.restype = ctypes.c_int
    lib.arena_release.argtypes = [sz, sz]
    lib.arena_region.argtypes = [sz]
    lib.arena_region.restype = sz
    lib.arena_free_ranges.argtypes = [ctypes.POINTER(sz), ctypes.POINTER(sz), sz]
    lib.arena_free_ranges.restype = sz
    return lib


def _alloc(lib, n):
    off = ctypes.c_size_t()
    return int(off.value) if lib.arena_alloc(n, ctypes.byref(off)) else None


def _ranges(lib):
    cap = 1 << 16
    offs, lens = (ctypes.c_size_t * cap)(), (ctypes.c_size_t * cap)()
    n = lib.arena_free_ranges(offs, lens, cap)
    assert n <= cap
    return [(int(offs[i]), int(lens[i])) for i in range(n)]


class Model:
    """Brute force: one flag per 256-byte unit."""

    def __init__(self, size):
        self.used = np.zeros(size // UNIT, bool)

    def runs(self):
        free = np.concatenate([[False], ~self.used, [False]]).astype(np.int8)
        d = np.diff(free)
        starts, ends = np.nonzero(d == 1)[0], np.nonzero(d == -1)[0]
        return [(int(s) * UNIT, int(e - s) * UNIT) for s, e in zip(starts, ends)]

    def alloc(self, n):
        k = -(-n // UNIT)
        for off, length in self.runs():
            if length >= k * UNIT:
                self.used[off // UNIT:off // UNIT + k] = True
                return off
        return None

    def release(self, off, n):
        k = -(-n // UNIT)
        assert self.used[off // UNIT:off // UNIT + k].all()
        self.used[off // UNIT:off // UNIT + k] = False


@pytest.mark.parametrize("seed", range(4))
def test_random_sequences_match_first_fit_model(arena, seed):
    rng = np.random.default_rng(seed)
    size = 4096 * UNIT
    arena.arena_reset(size)
    model = Model(size)
    live = []
    for step in range(3000):
        if live and rng.random() < 0.45:
            off, n = live.pop(int(rng.integers(len(live))))
            arena.arena_release(off, n)
            model.release(off, n)
        else:
            n = int(rng.integers(1, 40 * UNIT)) if rng.random() < 0.9 else int(rng.integers(1, size // 3))
            got, want = _alloc(arena, n), model.alloc(n)
            assert got == want, f"step {step}: alloc({n}) gave {got}, first fit gives {want}"
            if got is not None:
                assert got % UNIT == 0 and got + n <= size
                live.append((got, n))
        if step % 50 == 0 or step > 2950:
            assert _ranges(arena) == model.runs()  # maximal, merged, in order
    # everything released: one range covering the arena again
    for off, n in live:
        arena.arena_release(off, n)
    assert _ranges(arena) == [(0, size)]


def test_live_regions_never_overlap(arena):
    rng = np.random.default_rng(9)
    size = 1000 * UNIT
    arena.arena_reset(size)
    live = {}
    for _ in range(2000):
        if live and rng.random() < 0.5:
            off = list(live)[int(rng.integers(len(live)))]
            arena.arena_release(off, live.pop(off))
            continue
        n = int(rng.integers(1, 30 * UNIT))
        off = _alloc(arena, n)
        if off is None:
            # a refusal means no free range is large enough
            assert all(length < -(-n // UNIT) * UNIT for _, length in _ranges(arena))
            continue
        lo, hi = off, off + -(-n // UNIT) * UNIT
        assert 0 <= lo and hi <= size
        for o, m in live.items():
            assert hi <= o or o + -(-m // UNIT) * UNIT <= lo
        live[off] = n
    used = sum(-(-m // UNIT) * UNIT for m in live.values())
    assert used + sum(length for _, length in _ranges(arena)) == size


def test_exact_fill_empty_arena_and_regions(arena):
    arena.arena_reset(8 * UNIT)
    offs = [_alloc(arena, UNIT) for _ in range(8)]
    assert offs == [i * UNIT for i in range(8)]
    assert _alloc(arena, 1) is None and _ranges(arena) == []
    arena.arena_release(3 * UNIT, UNIT)
    arena.arena_release(5 * UNIT, UNIT)
    assert _alloc(arena, 2 * UNIT) is None  # two single free units are not adjacent
    arena.arena_release(4 * UNIT, UNIT)
    assert _ranges(arena) == [(3 * UNIT, 3 * UNIT)]
    assert _alloc(arena, 3 * UNIT) == 3 * UNIT
    arena.arena_reset(0)
    assert _alloc(arena, 1) is None
    # a region of 0 bytes still takes one unit, so every request owns distinct addresses
    assert arena.arena_region(0) == UNIT and arena.arena_region(1) == UNIT
    assert arena.arena_region(UNIT) == UNIT and arena.arena_region(UNIT + 1) == 2 * UNIT
