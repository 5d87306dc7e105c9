"""The binary64 kernels' documented arithmetic, checked bit for bit.

A row of length L <= 64 is one FMA chain in CRS order from y0 (0, or the old
y when accumulating); a longer row is cut into segments of 64 entries, each an
FMA chain (segment 0 from y0, the others from 0), and the segment results are
added in order -- for more than 256 segments first within each group of 256
consecutive segments, then the group results in order.  Here every FMA and every addition is emulated exactly with
rational arithmetic and one correct rounding to binary64 (float(Fraction) is
correctly rounded), so the GPU result must match to the last bit."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1307_6209_gb300 import synth

pytestmark = pytest.mark.gpu
SEG = 64
SUPER = 256


def _rnd(q: Fraction) -> float:
    return float(q)


def _chain(vals, xs, y0):
    s = float(y0)
    for a, b in zip(vals, xs):
        s = _rnd(Fraction(a) * Fraction(b) + Fraction(s))
    return s


def _row_result(vals, xs, y0):
    L = len(vals)
    if L <= SEG:
        return _chain(vals, xs, y0)
    parts = [_chain(vals[s:s + SEG], xs[s:s + SEG], y0 if s == 0 else 0.0) for s in range(0, L, SEG)]

    def fold(ps):
        t = ps[0]
        for p in ps[1:]:
            t = _rnd(Fraction(t) + Fraction(p))
        return t
    if len(parts) <= SUPER:
        return fold(parts)
    # more than 256 segments: fold each group of 256 in order, then the groups
    return fold([fold(parts[g:g + SUPER]) for g in range(0, len(parts), SUPER)])


def _matrix(spread=False):
    """The special lengths in the first 64 rows, or (spread) one every 40 rows,
    so that a chunk of up to 32 rows holds at most one long row -- the long
    rows then run segment by segment across the chunk's threads."""
    lens = [0, 1, 5, 63, 64, 65, 100, 127, 128, 129, 192, 200, 257, 640, 1000, 3, 1500, 2000, 1089, 4096,
            4100, 9000, 16384, 16385, 20000, 33000]
    rng = np.random.default_rng(42)
    n = 40000
    rows = []
    nrows = 64 * 40 if spread else 300
    for i in range(nrows):
        if spread:
            special = i % 40 == 0
            L = lens[(i // 40) % len(lens)] if special else int(rng.integers(0, 40))
        else:
            L = lens[i % len(lens)] if i < 64 else int(rng.integers(0, 40))
        rows.append(np.sort(rng.choice(n, size=L, replace=False)))
    rl = np.array([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    val = rng.standard_normal(col.shape[0])
    rpt = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(rl, out=rpt[1:])
    return synth.CSR(len(rows), n, rpt, col, val)


@pytest.mark.parametrize("spread", [False, True])
@pytest.mark.parametrize("accumulate", [False, True])
def test_f64_rows_match_documented_arithmetic(accumulate, spread):
    import torch
    from paper_1307_6209_gb300 import sell

    A = _matrix(spread)
    x = synth.vector(A.ncols, seed=9)
    y0 = synth.vector(A.nrows, seed=10)
    expect = np.array([
        _row_result(A.val[A.rpt[i]:A.rpt[i + 1]], x[A.col[A.rpt[i]:A.rpt[i + 1]]], y0[i] if accumulate else 0.0)
        for i in range(A.nrows)])
    flags = sell.SELL_SPMV_ACCUMULATE if accumulate else 0
    for C, sigma, block, pipe in [(32, 1, 256, 0), (32, 10 ** 9, 512, 1), (64, 128, 64, 0), (1, 1, 32, 1),
                                  (128, 4, 128, 1), (32, 10 ** 9, 256, 2), (64, 1, 128, 2), (128, 128, 512, 2)]:
        h = sell.sell_build(A, C=C, sigma=sigma)
        sell.sell_set_launch(h, block, 4, pipe)
        xd = torch.from_numpy(x).cuda()
        yd = torch.from_numpy(y0.copy()).cuda()
        sell.sell_spmv(h, xd, yd, flags=flags)
        torch.cuda.synchronize()
        got = yd.cpu().numpy()
        bad = np.nonzero(got.view(np.uint64) != expect.view(np.uint64))[0]
        assert bad.size == 0, f"C={C} sigma={sigma} pipeline={pipe}: rows {bad[:8]} (lengths {np.diff(A.rpt)[bad[:8]]})"


def _round_f32(q: Fraction) -> float:
    """q rounded to the nearest binary32 (ties to even), exactly."""
    if q == 0:
        return 0.0
    sign = -1.0 if q < 0 else 1.0
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()  # 2^(e-1) <= q < 2^(e+1)
    if Fraction(2) ** e > q:
        e -= 1
    e = max(e, -126)  # subnormals share the exponent of the smallest normal
    scale = Fraction(2) ** (e - 23)  # spacing of binary32 numbers in [2^e, 2^(e+1))
    m = q / scale
    n = m.numerator // m.denominator
    rem = m - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sign * float(n * scale)


def _row_result_f32(vals, xs, y0):
    """Binary32 FMA chains per 64-entry segment, the segment results added in
    order in binary64 (two levels beyond 256 segments), one final rounding to
    binary32."""
    def chain(v, x, s):
        s = float(s)
        for a, b in zip(v, x):
            s = _round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(s))
        return s
    L = len(vals)
    if L <= SEG:
        return chain(vals, xs, y0)
    parts = [chain(vals[s:s + SEG], xs[s:s + SEG], y0 if s == 0 else 0.0) for s in range(0, L, SEG)]

    def fold(ps):
        t = ps[0]
        for p in ps[1:]:
            t = _rnd(Fraction(t) + Fraction(p))
        return t
    t = fold(parts) if len(parts) <= SUPER else fold([fold(parts[g:g + SUPER]) for g in range(0, len(parts), SUPER)])
    return float(np.float32(t))


def test_f32_long_rows_fold_in_binary64():
    """Binary32 storage: long rows' segment results are added in binary64 and
    rounded once; checked bit for bit against exact rational emulation."""
    import torch
    import oracle
    from paper_1307_6209_gb300 import sell

    rng = np.random.default_rng(5)
    n = 40000
    lens = [3, 64, 65, 300, 1000, 5000, 17000] + [int(v) for v in rng.integers(0, 30, 57)]
    rows = [np.sort(rng.choice(n, size=L, replace=False)) for L in lens]
    rl = np.array([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    val = rng.standard_normal(col.shape[0])
    rpt = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(rl, out=rpt[1:])
    A = synth.CSR(len(rows), n, rpt, col, val)
    v32 = oracle.round_values(A.val, oracle.F32).astype(np.float32)
    x = synth.vector(n, seed=3).astype(np.float32)
    expect = np.array([_row_result_f32(v32[rpt[i]:rpt[i + 1]], x[col[rpt[i]:rpt[i + 1]]], 0.0)
                       for i in range(len(rows))], dtype=np.float32)
    for C, sigma in [(32, 1), (32, 10 ** 9), (64, 4)]:
        h = sell.sell_build(A, C=C, sigma=sigma, store_type=sell.SELL_F32)
        y = torch.empty(len(rows), dtype=torch.float32, device="cuda")
        sell.sell_spmv(h, torch.from_numpy(x).cuda(), y)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        bad = np.nonzero(got.view(np.uint32) != expect.view(np.uint32))[0]
        assert bad.size == 0, f"C={C} sigma={sigma}: rows {bad[:8]} (lengths {rl[bad[:8]]})"
