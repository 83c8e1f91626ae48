"""The constants the device exponentials are typed with, checked on the host
against their definitions (2048/ln 2 and ln 2/2048, derived here with sympy
to 80 digits) and against the precision each step of the methods needs.

The kernels' accuracy is measured on the GPU (tests/test_gpu_exp.py); this
pins the numbers themselves, so that a mistyped digit fails without a GPU."""
import os
import re

import numpy as np
import sympy as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "paper_1309_7327_gb300", "csrc", "chem.cuh")).read()

C = sp.Integer(2048) / sp.log(2)          # 2048 / ln 2
L = sp.log(2) / 2048                      # ln 2 / 2048


def _body(name):
    i = SRC.index(f"__device__ __forceinline__ double {name}(")
    return SRC[i:SRC.index("\n}\n", i)]


def _num(text, pattern):
    m = re.search(pattern, text)
    assert m, pattern
    return m.group(1)


def test_fp64_exponential_reduction_constants():
    """fast_exp: n from x 2048/ln2 (a double rounding of the constant is
    harmless: n only has to be nearest within the reduction's slack) and
    r = x - n (L1 + L2) with L1 holding at most 29 significant bits, so that
    n L1 is exact for |n| < 2^22, and L1 + L2 = ln2/2048 to ~2^-100."""
    body = _body("fast_exp")
    c = float(_num(body, r"fma\(x, ([0-9.]+), shift\)"))
    assert c == float(sp.N(C, 30))
    l1 = float(_num(body, r"L1 = ([0-9.e+-]+),"))
    l2 = float(_num(body, r"L2 = ([0-9.e+-]+);"))
    mant, _ = np.frexp(l1)
    bits = int(mant * 2 ** 53)
    assert bits % (1 << (53 - 29)) == 0, "L1 has more than 29 significant bits"
    err = sp.Rational(l1) + sp.Rational(l2) - L
    assert abs(float(err / L)) < 2.0 ** -75


def test_integer_exponential_constants():
    """exp_alu: CI + CR 2^-64 is 2048/ln2 scaled by 2^52, truncated to 128
    bits (so the fixed-point t is never above the exact one by more than one
    unit of 2^-64); LH + LL is ln2/2048 as a float pair within 2^-46."""
    body = _body("exp_alu")
    ci = int(_num(body, r"CI = (0x[0-9a-f]+)ULL"), 16)
    cr = int(_num(body, r"CR = (0x[0-9a-f]+)ULL"), 16)
    c128 = sp.floor(sp.N(C * sp.Integer(2) ** 116, 90))
    assert ci * 2 ** 64 + cr == int(c128)
    assert ci < 2 ** 64 and cr < 2 ** 64
    lh = float.fromhex(_num(body, r"LH = (0x[0-9a-fp.+-]+)f"))
    ll = float.fromhex(_num(body, r"LL = (-?0x[0-9a-fp.+-]+)f"))
    assert np.float32(lh) == lh and np.float32(ll) == ll       # exact floats
    assert lh == float(np.float32(float(sp.N(L, 30))))           # ln2/2048 rounded to float
    err = sp.Rational(lh) + sp.Rational(ll) - L
    assert abs(float(err / L)) < 2.0 ** -46


def test_integer_exponential_reduction_range():
    """The fixed-point reduction shifts the 117-bit product right by
    s = 1063 - e for biased exponents e of 1003..1032 (|x| from 2^-20 to the
    clamp at 709): s must stay in 1..63 so that both word shifts are defined,
    and the integer part of t must fit an int (|t| < 2^22)."""
    assert "1063 - ef" in _body("exp_alu")
    for ef in range(1023 - 20, 1023 + 9 + 1):
        s = 1063 - ef
        assert 1 <= s <= 63, (ef, s)
    t_max = 709.0 * float(sp.N(C, 20))
    assert t_max < 2 ** 22
