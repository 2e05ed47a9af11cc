"""Double-float arithmetic of the SG_DF64 contraction type, checked on the CPU.

The functions of csrc/sg_df.cuh are host-and-device code; here they are
compiled by the host compiler (with FMA contraction off, as the device code
forbids it through single-rounding intrinsics) and run on seeded inputs,
and every result is compared with the exact rational value:
  * two_sum: s + e equals a + b exactly and s is the rounded sum (Knuth);
  * the split of a double into hi + lo is within 2^-48 of it;
  * df_mul: within 8u^2 of the exact product of the two double-floats
    (u = 2^-24);
  * df_mul with a second factor left unrenormalised by df_fma: the same
    plus u |x| |y_lo|;
  * df_fma: within 8u^2 (|x y| + |c|) of c + x y, cancellation included;
  * a dot product of six terms by df_fma: within 6 * 8u^2 sum |x_k y_k|.
"""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2111_13655_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include "sg_df.cuh"
using sg::df2;
int main() {
    char op[16];
    while (std::scanf("%15s", op) == 1) {
        if (op[0] == 't') {               // two_sum a b
            float a, b, s, e;
            std::scanf("%a %a", &a, &b);
            sg::dfops::two_sum(a, b, s, e);
            std::printf("%a %a\n", s, e);
        } else if (op[0] == 's') {        // split d
            double d;
            std::scanf("%la", &d);
            df2 r(d);
            std::printf("%a %a\n", r.hi, r.lo);
        } else if (op[0] == 'm') {        // df_mul xh xl yh yl
            float a, b, c, d;
            std::scanf("%a %a %a %a", &a, &b, &c, &d);
            df2 r = sg::df_mul(df2(a, b), df2(c, d));
            std::printf("%a %a\n", r.hi, r.lo);
        } else {                          // df_fma xh xl yh yl ch cl
            float a, b, c, d, e, f;
            std::scanf("%a %a %a %a %a %a", &a, &b, &c, &d, &e, &f);
            df2 r = sg::df_fma(df2(a, b), df2(c, d), df2(e, f));
            std::printf("%a %a\n", r.hi, r.lo);
        }
    }
    return 0;
}
"""

U = Fraction(1, 2 ** 24)


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("df")
    src, exe = d / "df.cpp", d / "df"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True, capture_output=True)

    def go(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.split("\n")
        return [tuple(float.fromhex(t) for t in ln.split()) for ln in out if ln.strip()]
    return go


def f32(v):
    """Round a Python float to the nearest FP32 value."""
    return struct.unpack("f", struct.pack("f", v))[0]


def df_of(rng, scale=1.0):
    """A normalised double-float (hi, lo) near scale."""
    d = float(rng.standard_normal()) * scale
    hi = f32(d)
    lo = f32(d - hi)
    return hi, lo


def F(*vals):
    return sum((Fraction(v) for v in vals), Fraction(0))


def test_two_sum_is_exact(run):
    rng = np.random.default_rng(1)
    pairs = []
    for _ in range(400):
        a = f32(float(rng.standard_normal()) * 2.0 ** int(rng.integers(-30, 30)))
        b = f32(float(rng.standard_normal()) * 2.0 ** int(rng.integers(-30, 30)))
        pairs.append((a, b))
    res = run([f"t {a.hex()} {b.hex()}" for a, b in pairs])
    for (a, b), (s, e) in zip(pairs, res):
        assert F(s, e) == F(a, b)
        assert s == f32(a + b)


def test_split_of_a_double(run):
    rng = np.random.default_rng(2)
    ds = [float(rng.standard_normal()) * 2.0 ** int(rng.integers(-40, 40)) for _ in range(400)]
    res = run([f"s {d.hex()}" for d in ds])
    for d, (hi, lo) in zip(ds, res):
        assert hi == f32(d)
        assert abs(F(hi, lo) - Fraction(d)) <= abs(Fraction(d)) * Fraction(1, 2 ** 48)


def test_product(run):
    rng = np.random.default_rng(3)
    xs = [(df_of(rng, 2.0 ** int(rng.integers(-10, 10))), df_of(rng, 2.0 ** int(rng.integers(-10, 10))))
          for _ in range(400)]
    res = run([f"m {x[0].hex()} {x[1].hex()} {y[0].hex()} {y[1].hex()}" for x, y in xs])
    for (x, y), (hi, lo) in zip(xs, res):
        exact = F(*x) * F(*y)
        assert abs(F(hi, lo) - exact) <= 8 * U * U * abs(exact)


def test_product_of_an_unrenormalised_accumulator(run):
    """df_fma leaves its result unrenormalised (lo can exceed ulp(hi)/2; here
    |lo| <= 2^-20 |hi|).  A product taking it rounds the cross term x_hi y_lo
    to FP32: its error gains u |x| |y_lo| over the normalised bound (which is
    about u^2 |x y| again when lo is a few roundings of hi)."""
    rng = np.random.default_rng(6)
    xs = []
    for _ in range(400):
        x = df_of(rng)
        hi = f32(float(rng.standard_normal()))
        lo = f32(hi * float(rng.uniform(-1, 1)) * 2.0 ** -20)
        xs.append((x, (hi, lo)))
    res = run([f"m {x[0].hex()} {x[1].hex()} {y[0].hex()} {y[1].hex()}" for x, y in xs])
    for (x, y), (hi, lo) in zip(xs, res):
        exact = F(*x) * F(*y)
        assert abs(F(hi, lo) - exact) <= 8 * U * U * abs(exact) + 2 * U * abs(F(*x)) * abs(Fraction(y[1]))


def test_fused_multiply_add_with_cancellation(run):
    rng = np.random.default_rng(4)
    cases = []
    for k in range(600):
        x, y = df_of(rng), df_of(rng)
        if k % 3 == 0:      # c close to -x*y: the sum cancels
            prod = -(F(*x) * F(*y)) * (1 + Fraction(int(rng.integers(-1000, 1000)), 2 ** 30))
            hi = f32(float(prod))
            c = (hi, f32(float(prod - Fraction(hi))))
        else:
            c = df_of(rng, 2.0 ** int(rng.integers(-8, 8)))
        cases.append((x, y, c))
    res = run([f"f {x[0].hex()} {x[1].hex()} {y[0].hex()} {y[1].hex()} {c[0].hex()} {c[1].hex()}"
               for x, y, c in cases])
    for (x, y, c), (hi, lo) in zip(cases, res):
        p, cc = F(*x) * F(*y), F(*c)
        assert abs(F(hi, lo) - (p + cc)) <= 8 * U * U * (abs(p) + abs(cc))


def test_dot_product_of_six(run):
    rng = np.random.default_rng(5)
    for _ in range(60):
        xs = [df_of(rng) for _ in range(6)]
        ys = [df_of(rng) for _ in range(6)]
        acc = (0.0, 0.0)
        for x, y in zip(xs, ys):
            (acc,) = run([f"f {x[0].hex()} {x[1].hex()} {y[0].hex()} {y[1].hex()} {acc[0].hex()} {acc[1].hex()}"])
        terms = [F(*x) * F(*y) for x, y in zip(xs, ys)]
        assert abs(F(*acc) - sum(terms)) <= 6 * 8 * U * U * sum(abs(t) for t in terms)
