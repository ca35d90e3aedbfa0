"""The oracle's algorithms perform the operation counts the paper tabulates
(Add/subtract: an exact transform a + b -> s + t takes 6 operations, ATF/STF
1.1 take 7 and ATF/STF 1 take 8; Multiply: a x b -> p + e takes 1 multiply
and 1 FMA, and the table of MTF 1 / MTF 1.1 / MPF 1 counts add/subtract,
multiply and FMA operations separately; the fast renormalisation of the
Dekker arithmetic section takes 3 add/subtract operations).

A static check: the oracle is compiled here for x86-64 without inlining,
and the scalar floating-point instructions of each function (addsd, subsd,
mulsd; calls of fma) are counted in the assembly of that build, following
calls into the other oracle functions.  A dropped or extra operation
anywhere in an algorithm changes its count; the last test plants two such
mistakes in a copy of the source and checks that the counts catch them.
Runs where gcc targets x86-64 (the CPU suite's machine)."""
import collections
import os
import platform
import re
import shutil
import subprocess

import pytest

import oracle as O

pytestmark = pytest.mark.skipif(platform.machine() not in ("x86_64", "AMD64") or shutil.which("gcc") is None,
                                reason="counts the x86-64 instructions of the oracle's own build")

SRC = os.path.join(os.path.dirname(O.__file__), "twofold_oracle.c")
FP_OPS = {"addsd": "add", "subsd": "add", "mulsd": "mul", "divsd": "div", "sqrtsd": "sqrt"}

# The paper's tables (add/subtract counted together).
PAPER = {
    "tfo_two_sum": {"add": 6},
    "tfo_two_diff": {"add": 6},
    "tfo_two_prod": {"mul": 1, "fma": 1},
    "tfo_fast_two_sum": {"add": 3},
    "tfo_atf11": {"add": 7},
    "tfo_stf11": {"add": 7},
    "tfo_atf1": {"add": 8},
    "tfo_stf1": {"add": 8},
    "tfo_mtf1": {"add": 3, "mul": 4, "fma": 1},
    "tfo_mtf11": {"add": 1, "mul": 2, "fma": 1},
    "tfo_mpf1": {"add": 2, "mul": 3, "fma": 1},
}


def assembly(src, tmp):
    out = os.path.join(tmp, "oracle.s")
    flags = [f for f in O.CFLAGS if f not in ("-O2", "-shared")]
    subprocess.check_call(["gcc", "-O1", "-fno-inline", *flags, "-S", src, "-o", out])
    return open(out).read()


def functions(asm):
    """Instruction lines of each global function of the assembly."""
    funcs, cur = {}, None
    for line in asm.splitlines():
        m = re.match(r"^([A-Za-z_]\w*):\s*$", line)
        if m:
            cur = m.group(1)
            funcs[cur] = []
        elif cur is not None and line.startswith("\t"):
            funcs[cur].append(line.strip())
    return funcs


def op_counts(name, funcs, memo=None):
    memo = {} if memo is None else memo
    if name in memo:
        return memo[name]
    c = collections.Counter()
    for ins in funcs[name]:
        parts = ins.split(None, 1)
        if not parts:
            continue
        if parts[0] in FP_OPS:
            c[FP_OPS[parts[0]]] += 1
        elif parts[0] == "call" and len(parts) > 1:
            callee = parts[1].split("@")[0]
            if callee == "fma":
                c["fma"] += 1
            elif callee in funcs:
                c.update(op_counts(callee, funcs, memo))
    memo[name] = c
    return c


def test_counting_sees_the_instructions(tmp_path):
    """The parser finds every counted function and some instructions in each."""
    funcs = functions(assembly(SRC, str(tmp_path)))
    for name in PAPER:
        assert name in funcs and funcs[name], name


@pytest.mark.parametrize("name", sorted(PAPER))
def test_paper_operation_counts(name, tmp_path):
    funcs = functions(assembly(SRC, str(tmp_path)))
    assert dict(op_counts(name, funcs)) == PAPER[name], (name, dict(op_counts(name, funcs)))


def test_counts_catch_planted_mistakes(tmp_path):
    """MTF1 without its x1 y1 product, and ATF1 adding its tail twice: each
    changes the count, so the pin has teeth."""
    src = open(SRC).read()
    for fname, old, new in [("tfo_mtf1", "double u = e00 + p11;", "double u = e00;"),
                            ("tfo_atf1", "z.z1 = u + e;", "z.z1 = (u + e) + e;")]:
        start = src.index(fname + "(")
        body_end = src.index("\n}\n", start)
        assert old in src[start:body_end], (fname, old)
        mutated = src[:start] + src[start:body_end].replace(old, new, 1) + src[body_end:]
        path = tmp_path / f"{fname}.c"
        path.write_text(mutated)
        funcs = functions(assembly(str(path), str(tmp_path)))
        assert dict(op_counts(fname, funcs)) != PAPER[fname], fname
