"""The oracle's pins catch plausible mistakes.

Each case plants ONE mistake in a copy of oracle/sell_oracle.c -- a dropped
term, a wrong sign, a wrong or transposed index, an ascending or unstable sort,
a lost permutation, an off-by-one in the chunk offsets, a truncating rounding
-- compiles the copy, runs the oracle's Python functions on it, and checks that
the named pins of tests/test_oracle_pins.py fail.  A mistake that no pin
catches would be a gap in the pins.  Every planted mistake keeps all memory
accesses inside the arrays the oracle is given, so a mutant can give wrong
numbers but cannot corrupt the test process.
"""
import os

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sell_oracle.c")

# (name, text in sell_oracle.c, replacement, pins that must fail)
MUTANTS = [
    ("crs: last entry of each row dropped",
     "for (int64_t j = rpt[i]; j < rpt[i + 1]; ++j) {\n            double p = val[j] * x[col[j]];\n"
     "            s = s + p;\n        }\n        y[i] = s;",
     "for (int64_t j = rpt[i]; j < rpt[i + 1] - 1; ++j) {\n            double p = val[j] * x[col[j]];\n"
     "            s = s + p;\n        }\n        y[i] = s;",
     [(pins.test_csr_spmv_within_rounding_of_exact_rational, dict(seed=0)),
      (pins.test_csr_spmv_integer_matrix_is_exact, {}),
      (pins.test_laplace_row_sums_with_unit_x, {})]),
    ("crs: product subtracted",
     "            s = s + p;\n        }\n        y[i] = s;",
     "            s = s - p;\n        }\n        y[i] = s;",
     [(pins.test_csr_spmv_within_rounding_of_exact_rational, dict(seed=1)),
      (pins.test_csr_spmv_dense_brute_force, dict(n=7, m=64))]),
    ("crs: x indexed by the row's first column",
     "double s = accumulate ? y[i] : 0.0;\n        for (int64_t j = rpt[i]; j < rpt[i + 1]; ++j) {\n"
     "            double p = val[j] * x[col[j]];",
     "double s = accumulate ? y[i] : 0.0;\n        for (int64_t j = rpt[i]; j < rpt[i + 1]; ++j) {\n"
     "            double p = val[j] * x[col[rpt[i]]];",
     [(pins.test_csr_spmv_integer_matrix_is_exact, {}),
      (pins.test_csr_spmv_dense_brute_force, dict(n=64, m=64))]),
    ("crs: accumulate ignored",
     "double s = accumulate ? y[i] : 0.0;",
     "double s = 0.0;",
     [(pins.test_csr_accumulate_starts_from_y, {})]),
    ("crs rows: absolute value dropped from the scale",
     "            a = a + fabs(p);",
     "            a = a + p;",
     [(pins.test_csr_rows_matches_full_product_and_absdot, {})]),
    ("absdot: absolute value dropped",
     "a = a + fabs(val[j] * x[col[j]]);",
     "a = a + val[j] * x[col[j]];",
     [(pins.test_absdot_is_dense_abs_product, {})]),
    ("spmmv: X transposed",
     "X[(int64_t)col[j] * ldx + c]",
     "X[(int64_t)c * ldx + col[j]]",
     [(pins.test_spmmv_columns_are_independent_spmv, {})]),
    ("sort: ascending",
     "return (a->len > b->len) ? -1 : 1; /* longer first */",
     "return (a->len < b->len) ? -1 : 1; /* longer first */",
     [(pins.test_sigma_sort_invariants, dict(sigma=64)),
      (pins.test_global_sort_minimises_storage, {})]),
    ("sort: ties reversed (not stable)",
     "return (a->row < b->row) ? -1 : 1; /* stable ties */",
     "return (a->row > b->row) ? -1 : 1; /* stable ties */",
     [(pins.test_sigma_sort_invariants, dict(sigma=8))]),
    ("chunk length: minimum instead of maximum",
     "if (len > m) m = len;",
     "if (m == 0 || (len > 0 && len < m)) m = len;",
     [(pins.test_sell_N_1_is_ellpack, dict(extra=0)),
      (pins.test_laplace_beta_closed_form, {})]),
    ("chunk offsets: one padding column too many",
     "cs[c + 1] = cs[c] + (int64_t)C * m;",
     "cs[c + 1] = cs[c] + (int64_t)C * (m + 1);",
     [(pins.test_sell_1_1_is_crs, dict(seed=0)),
      (pins.test_laplace_beta_closed_form, {})]),
    ("fill: row-major inside the chunk (transposed)",
     "int64_t pos = cs[c] + (int64_t)j * C + l;\n                if (j < len) {",
     "int64_t pos = cs[c] + (int64_t)l * cl[c] + j;\n                if (j < len) {",
     [(pins.test_sell_N_1_is_ellpack, dict(extra=5)),
      (pins.test_format_layout_by_definition, {})]),
    ("fill: padding column is the row's own index",
     "                    scol[pos] = 0;",
     "                    scol[pos] = (int32_t)l;",
     [(pins.test_sell_N_1_is_ellpack, dict(extra=0)),
      (pins.test_format_layout_by_definition, {})]),
    ("fill: columns renumbered with perm instead of its inverse",
     "scol[pos] = inv ? inv[col[src]] : col[src];",
     "scol[pos] = inv ? perm[col[src]] : col[src];",
     [(pins.test_permuted_columns_are_symmetric_permutation, {}),
      (pins.test_sell_spmv_permuted_space, {})]),
    ("sell spmv: result left in sorted order",
     "else y[perm[r]] = tmp[r];",
     "else y[r] = tmp[r];",
     [(pins.test_sell_spmv_bitwise_equals_crs, dict(C=32, sigma=256))]),
    ("sell spmv: accumulate starts from the wrong row",
     "init = permuted_io ? y[r] : y[perm[r]];",
     "init = permuted_io ? y[r] : y[r];",
     [(pins.test_sell_spmv_bitwise_equals_crs, dict(C=64, sigma=4096))]),
    ("beta: stored count without the factor C",
     "stored += (int64_t)C * cl[c];",
     "stored += cl[c];",
     [(pins.test_laplace_beta_closed_form, {}),
      (pins.test_beta_worst_closed_form, dict(N=96, C=8))]),
    ("zeta: sample instead of population deviation",
     "return sqrt(sq / (double)nrows) / mean;",
     "return sqrt(sq / (double)(nrows - 1)) / mean;",
     [(pins.test_zeta_closed_forms, {})]),
    ("rounding: truncation instead of nearest-even",
     "double r = nearbyint(a / q) * q;",
     "double r = floor(a / q) * q;",
     [(pins.test_round_f32_equals_ieee_cast, {}),
      (pins.test_round_bf16_is_nearest, {})]),
    ("rounding: bfloat16 with a 7-bit significand",
     "orc_round_to(in[i], to == 1 ? 24 : 8);",
     "orc_round_to(in[i], to == 1 ? 24 : 7);",
     [(pins.test_round_bf16_hand_derived, dict(value=1.0 + 2 ** -8 + 2 ** -30, bits=0x3F81)),
      (pins.test_round_bf16_is_nearest, {})]),
    ("bfloat16 decoding: bits shifted one place too few",
     "uint32_t bits = (uint32_t)in[i] << 16;",
     "uint32_t bits = (uint32_t)in[i] << 15;",
     [(pins.test_round_bf16_is_nearest, {})]),
    ("rounding: subnormal spacing one binade too fine",
     "if (E < -126) E = -126;",
     "if (E < -127) E = -127;",
     [(pins.test_round_f32_equals_ieee_cast, {}),
      (pins.test_round_bf16_is_nearest, {})]),
]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name,old,new,killers", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, killers, source, tmp_path):
    assert source.count(old) == 1, f"mutation site not unique or missing: {old!r}"
    src = tmp_path / "mutant.c"
    src.write_text(source.replace(old, new))
    lib = oracle.compile_library(str(src), str(tmp_path / "libmutant.so"))
    with oracle.substituted_library(lib):
        for pin, kw in killers:
            with pytest.raises((AssertionError, ValueError)):
                pin(**kw)
    # the unmodified oracle passes the same pins
    for pin, kw in killers:
        pin(**kw)
