"""The pins have teeth: plausible mistakes planted in copies of the oracle
(a dropped term, a wrong sign, a swapped operand, an off-by-one bound, a wrong
divisor) each make at least one pin fail.  Everything here runs on the CPU;
the real oracle is restored after every mutant."""
import os
import subprocess

import pytest

import oracle as O
from tests import test_oracle_algorithms as TA
from tests import test_oracle_applications as TP
from tests import test_oracle_coupled as TC
from tests import test_oracle_f32 as TF
from tests import test_oracle_horner_ew as TH
from tests import test_oracle_reduce as TR
from tests import test_oracle_transforms as TT

SRC = os.path.join(os.path.dirname(O.__file__), "twofold_oracle.c")
SRC32 = os.path.join(os.path.dirname(O.__file__), "twofold_oracle_f32.c")


def _in_function(src, fname, old, new):
    """Replace the first `old` inside the body of C function `fname`."""
    start = src.index(fname + "(")
    brace = src.index("{", start)
    depth, i = 0, brace
    while True:
        if src[i] == "{":
            depth += 1
        elif src[i] == "}":
            depth -= 1
            if depth == 0:
                break
        i += 1
    body = src[brace:i]
    assert old in body, (fname, old)
    return src[:brace] + body.replace(old, new, 1) + src[i:]


DATA = None


def data():
    global DATA
    if DATA is None:
        DATA = TA.make_data()
    return DATA


def _pairs32():
    rng = __import__("numpy").random.default_rng(32)
    return TF.rand32(rng, 6000), TF.rand32(rng, 6000)


MUTANTS = {
    "mtf1_drops_p11": (("tfo_mtf1", "double u = e00 + p11;", "double u = e00;"),
                       [lambda: TA.test_mtf1_budget(data())]),
    "two_diff_printed_signs": (("tfo_two_diff", "double bs = b1 - b;", "double bs = b - b1;"),
                               [lambda: TT.test_two_diff_exact(TT.make_pairs())]),
    "atf1_subtracts_tail": (("tfo_atf1", "double u = x1 + y1;", "double u = x1 - y1;"),
                            [lambda: TA.test_atf1_budget(data())]),
    "dtf1_divides_by_y0": (("tfo_dtf1", "z.z1 = c0 / d0;", "z.z1 = c0 / y0;"),
                           [lambda: TA.test_dtf1_budget(data())]),
    "dtf1_r1_sign": (("tfo_dtf1", "fma(-q, y1, x1)", "fma(q, y1, x1)"),
                     [lambda: TA.test_dtf1_budget(data())]),
    "rpf11_no_factor_two": (("tfo_rpf11", "double w = 2.0 * c;", "double w = c;"),
                            [lambda: TA.test_rpf11_output_coupled(data())]),
    "rtf1_drops_u1": (("tfo_rtf1", "tfo_rpf1(u0, u1)", "tfo_rpf1(u0, 0.0)"),
                      [lambda: TA.test_rtf1_coupled_loose(data()), TA.test_rtf1_budget]),
    "rtf1_input_tail_for_two_sum_tail": (("tfo_rtf1", "tfo_rpf1(u0, u1)", "tfo_rpf1(u0, x1)"),
                                         [TA.test_rtf1_budget]),
    "rtf1_drops_w1": (("tfo_rtf1", "z.z1 = w.z0 + w.z1;", "z.z1 = w.z0;"), [TA.test_rtf1_budget]),
    "rtf1_stf_operands_swapped": (("tfo_rtf1", "tfo_stf11(v.z0, v.z1, z0)", "tfo_stf11(z0, v.z1, v.z0)"),
                                  [TA.test_rtf1_budget]),
    "two_sum_swaps_roles": (("tfo_two_sum", "double b1 = s_ - a;", "double b1 = s_ - b;"),
                            [lambda: TT.test_two_sum_exact(TT.make_pairs())]),
    "leaf_skips_first": (("leaf_reduce", "for (int64_t i = b; i < e; ++i)",
                          "for (int64_t i = b + 1; i < e; ++i)"),
                         [lambda: TR.test_dot_z0_is_plain_order(1000, 256)]),
    "tree_drops_odd_carry": (("tree_reduce", "if (m & 1) nodes[h++] = nodes[m - 1];", ""),
                             [lambda: TR.test_sum_z0_is_plain_order(4097, 256)]),
    "horner_stops_early": (("tfo_horner", "for (int i = k - 1; i >= 0; --i)",
                            "for (int i = k - 1; i >= 1; --i)"),
                           [lambda: TH.test_horner_binomial(5)]),
    "flag_ge": (("tfo_flag", "if (fabs(z1) > lim)", "if (fabs(z1) >= lim)"),
                [TA.test_flag_rel_and_nonfinite]),
    "mtf11_uses_x0": (("tfo_mtf11", "double p10 = x1 * y0;", "double p10 = x0 * y0;"),
                      [lambda: TA.test_atf11_strict(data()),
                       lambda: TH.test_horner_binomial(10)]),
    "stf11_adds_instead": (("tfo_stf11", "tfo_two_diff(x0, y0, &d, &e);",
                            "tfo_two_sum(x0, y0, &d, &e);"),
                           [lambda: TA.test_stf11_strict(data())]),
    "renorm_skipped": (("renorm", "tfo_fast_two_sum(z.z0, z.z1, &r.z0, &r.z1);", "r = z;"),
                       [lambda: TC.test_coupled_outputs_are_coupled(TC.make_coupled(), O.PADD, "add", "tt")]),
    "fast_two_sum_swapped": (("tfo_fast_two_sum", "double b1 = s_ - a;", "double b1 = s_ - b;"),
                             [TC.test_fast_two_sum_exact_when_ordered]),
    "mpf1_drops_p10": (("tfo_mpf1", "double v = p01 + p10;", "double v = p01;"),
                       [lambda: TC.test_mpf1_budget(TC.make_coupled())]),
    "dpf1_r1_sign": (("tfo_dpf1", "fma(-q, y1, x1)", "fma(q, y1, x1)"),
                     [lambda: TC.test_dpf1_budget(TC.make_coupled())]),
    "rpf1_drops_x1": (("tfo_rpf1", "double t = x1 + d;", "double t = d;"),
                      [lambda: TC.test_rpf1_budget(TC.make_coupled())]),
    "f32_two_diff_printed_signs": (("tfof_two_diff", "float bs = b1 - b;", "float bs = b - b1;"),
                                   [lambda: TF.test_exact_transforms32(
                                       (TF.rand32(__import__("numpy").random.default_rng(1), 3000),
                                        TF.rand32(__import__("numpy").random.default_rng(2), 3000)))]),
    "f32_mtf1_drops_p11": (("tfof_mtf1", "float u = e00 + p11;", "float u = e00;"),
                           [lambda: TF.test_mtf1_budget32(_pairs32())]),
    "f32_dtf1_r1_sign": (("tfof_dtf1", "fmaf(-q, y1, x1)", "fmaf(q, y1, x1)"),
                         [lambda: TF.test_dtf1_budget32(_pairs32())]),
    "f32_rtf1_drops_w1": (("tfof_rtf1", "z.z1 = w.z0 + w.z1;", "z.z1 = w.z0;"),
                          [lambda: TF.test_rtf1_budget32(_pairs32())]),
    "f32_atf1_subtracts_tail": (("tfof_atf1", "float u = x1 + y1;", "float u = x1 - y1;"),
                                [lambda: TF.test_atf1_stf1_budget32(
                                    (TF.rand32(__import__("numpy").random.default_rng(1), 3000),
                                     TF.rand32(__import__("numpy").random.default_rng(2), 3000)))]),
    "f32_dot_drops_product_tail": (("tfof_reduce", "acc = tfof_atf1(acc.z0, acc.z1, q.z0, q.z1);",
                                    "acc = tfof_atf11(acc.z0, acc.z1, q.z0);"),
                                   [lambda: TF.test_dot32_single_term_is_two_product(
                                       (TF.rand32(__import__("numpy").random.default_rng(1), 600),
                                        TF.rand32(__import__("numpy").random.default_rng(2), 600)))]),
    "f32_dot_leaf_off_by_one": (("tfof_reduce", "for (int64_t i = j * L; i < e; ++i) {",
                                 "for (int64_t i = j * L + 1; i < e; ++i) {"),
                                [TF.test_dot32_exact_when_everything_is_representable]),
    "f32_plain_tree_drops_carry": (("tfof_reduce_plain", "if (m & 1) nodes[h++] = nodes[m - 1];", ""),
                                   [TF.test_plain32_twin_is_plain_float_arithmetic]),
    "gauss_dtf1_drops_d0": (("tfo_dtf1", "double d0 = y0 + y1;", "double d0 = y0 + y0;"),
                            [lambda: TP.test_gauss_logs("gauss_well3", 0.1, (11.0, 11.0, 1.0)),
                             lambda: TA.test_dtf1_budget(data())]),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    (fname, old, new), checks = MUTANTS[name]
    srcs = [SRC, SRC32]
    k = 1 if fname.startswith("tfof_") else 0          # the binary32 basis lives in its own file
    mutated = tmp_path / "mutant.c"
    mutated.write_text(_in_function(open(srcs[k]).read(), fname, old, new))
    srcs[k] = str(mutated)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", *O.CFLAGS, *srcs, "-o", str(so), "-lm"])
    saved = O.lib()
    O._lib = O.load(str(so))
    failed = 0
    try:
        for chk in checks:
            try:
                chk()
            except AssertionError:
                failed += 1
    finally:
        O._lib = saved
    assert failed > 0, f"mutant {name} survived the pins"
