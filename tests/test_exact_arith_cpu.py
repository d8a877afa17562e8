"""Host checks of the library's exact integer-arithmetic helpers, compiled from the shipped CUDA
sources (the function bodies are taken from the .cu files as they are and built with the host
compiler behind a few definitions of the CUDA intrinsics they call):

- ``exact_fold`` (tensor-core coefficient GEMM): (hi 2^24 + lo) 2^e rounded once to the nearest
  double, ties to even -- checked against exact rational rounding (``fractions.Fraction``, whose
  conversion to float rounds to nearest even), including constructed halfway cases;
- ``dyadic`` (streaming P1 interpolation): k 2^-l as a double, exactly;
- ``half_pos`` (streaming edge weights): v / 2 for positive normal doubles, exactly.
"""
from __future__ import annotations

import os
import random
import re
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_03407_gb300", "csrc")

SHIM = r"""
#include <cstdio>
#include <cstring>
#include <cstdlib>
#define __device__
#define __forceinline__ inline
static inline int __clzll(long long x) { return __builtin_clzll((unsigned long long)x); }
static inline int __clz(int x) { return __builtin_clz((unsigned)x); }
static inline double __longlong_as_double(long long b) { double d; std::memcpy(&d, &b, 8); return d; }
static inline long long __double_as_longlong(double d) { long long b; std::memcpy(&b, &d, 8); return b; }
"""

MAIN = r"""
int main() {
  char op[8];
  while (std::scanf("%7s", op) == 1) {
    if (op[0] == 'f') {
      long long hi, lo; int e;
      if (std::scanf("%lld %lld %d", &hi, &lo, &e) != 3) return 1;
      std::printf("%016llx\n", (unsigned long long)__double_as_longlong(exact_fold(hi, lo, e)));
    } else if (op[0] == 'd') {
      int k, l;
      if (std::scanf("%d %d", &k, &l) != 2) return 1;
      std::printf("%016llx\n", (unsigned long long)__double_as_longlong(dyadic(k, l)));
    } else {
      unsigned long long b;
      if (std::scanf("%llx", &b) != 1) return 1;
      std::printf("%016llx\n", (unsigned long long)__double_as_longlong(half_pos(__longlong_as_double((long long)b))));
    }
  }
  return 0;
}
"""


def _function(path, name):
    """The source text of the device function `name` in `path` (signature through its closing brace)."""
    src = open(path).read()
    m = re.search(r"__device__ __forceinline__ double " + name + r"\(", src)
    assert m, f"{name} not found in {path}"
    i = src.index("{", m.end())
    depth = 0
    for j in range(i, len(src)):
        if src[j] == "{":
            depth += 1
        elif src[j] == "}":
            depth -= 1
            if depth == 0:
                return src[m.start(): j + 1]
    raise AssertionError(f"unbalanced braces in {name}")


@pytest.fixture(scope="module")
def helper(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    code = SHIM + "\n".join([
        _function(os.path.join(CSRC, "mq_tc.cu"), "exact_fold"),
        _function(os.path.join(CSRC, "mq_stream.cu"), "dyadic"),
        _function(os.path.join(CSRC, "mq_stream.cu"), "half_pos"),
    ]) + MAIN
    d = tmp_path_factory.mktemp("exact")
    src, exe = d / "exact.cpp", d / "exact"
    src.write_text(code)
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", str(exe), str(src)], check=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return [struct.unpack("<d", int(h, 16).to_bytes(8, "little"))[0] for h in out.stdout.split()]

    return run


def test_exact_fold_rounds_once_to_nearest_even(helper):
    rng = random.Random(7)
    cases = []
    for _ in range(20000):
        kind = rng.random()
        if kind < 0.4:  # the full ranges of the fold: |hi| < 2^56, |lo| < 2^40
            hi, lo = rng.randint(-(1 << 56) + 1, (1 << 56) - 1), rng.randint(-(1 << 40) + 1, (1 << 40) - 1)
        elif kind < 0.55:  # small high part: leading bit in the low word
            hi, lo = rng.randint(-(1 << 16), 1 << 16), rng.randint(-(1 << 40) + 1, (1 << 40) - 1)
        elif kind < 0.65:
            hi, lo = 0, rng.randint(-(1 << 40) + 1, (1 << 40) - 1)
        else:  # exactly halfway between two doubles: ties go to the even mantissa
            m = rng.randint(1 << 52, (1 << 53) - 1)
            sh = rng.randint(1, 20)
            v = ((2 * m + 1) << (sh - 1)) * rng.choice((1, -1))
            hi, lo = v >> 24, v - ((v >> 24) << 24)
        cases.append((hi, lo, rng.randint(-80, -40)))
    got = helper([f"f {h} {l} {e}" for h, l, e in cases])
    for (h, l, e), g in zip(cases, got):
        assert g == float(Fraction((h << 24) + l) * Fraction(2) ** e), (h, l, e)
    assert helper(["f 0 0 -63"]) == [0.0]


def test_dyadic_fractions(helper):
    cases = [(k, l) for l in range(0, 11) for k in range(1 << l)]
    got = helper([f"d {k} {l}" for k, l in cases])
    for (k, l), g in zip(cases, got):
        assert g == k / (1 << l), (k, l)


def test_half_pos_halves_positive_normals(helper):
    rng = random.Random(3)
    vals = [rng.uniform(1e-3, 1e3) for _ in range(2000)] + [2.0 ** rng.randint(-1000, 1000) for _ in range(200)]
    got = helper(["h " + struct.pack("<d", v)[::-1].hex() for v in vals])
    for v, g in zip(vals, got):
        assert g == v / 2, v
