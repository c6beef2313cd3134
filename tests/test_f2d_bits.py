"""The element kernel widens its FP32 forces to FP64 with integer operations on
the IEEE 754 bit layouts (`f2d_exact` in k_element.cu) instead of the
conversion instruction.  The function's own source text is compiled for the
host here, with the CUDA bit-cast and leading-zero intrinsics defined in C, and
compared bit for bit with C's float -> double conversion over a stride of all
2^32 bit patterns plus the edge cases (signed zeros, subnormals, the largest
and smallest normals, infinities, NaN) and every subnormal."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2408_04066_gb300", "csrc", "k_element.cu")

HARNESS = r"""
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#define __device__
#define __forceinline__ static inline
static inline unsigned __float_as_uint(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
static inline int __clz(int x) { return x ? __builtin_clz((unsigned)x) : 32; }
static inline double __longlong_as_double(long long v) { double d; memcpy(&d, &v, 8); return d; }
%s
static int same(float f) {
    double a = f2d_exact(f), b = (double)f;
    if (a != a && b != b) return 1;   /* NaN: any payload */
    return memcmp(&a, &b, 8) == 0;
}
int main(void) {
    const uint32_t edge[] = {0x00000000u, 0x80000000u, 0x00000001u, 0x807fffffu, 0x00800000u, 0x80800000u,
                             0x7f7fffffu, 0xff7fffffu, 0x3f800000u, 0x7f800000u, 0xff800000u, 0x7fc00000u};
    unsigned long bad = 0, n = 0;
    for (unsigned i = 0; i < sizeof(edge) / sizeof(edge[0]); ++i) {
        float f; memcpy(&f, &edge[i], 4); bad += !same(f); ++n;
    }
    for (uint64_t u = 0; u < (1ull << 32); u += 97) {
        uint32_t v = (uint32_t)u; float f; memcpy(&f, &v, 4); bad += !same(f); ++n;
    }
    for (uint32_t v = 0; v < (1u << 23); ++v) {   /* every subnormal, both signs */
        float f; uint32_t w = v | 0x80000000u;
        memcpy(&f, &v, 4); bad += !same(f); ++n;
        memcpy(&f, &w, 4); bad += !same(f); ++n;
    }
    printf("%%lu %%lu\n", n, bad);
    return 0;
}
"""


def test_f2d_exact_matches_the_conversion(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    text = open(SRC).read()
    m = re.search(r"__device__ __forceinline__ double f2d_exact\(float f\) \{.*?\n\}\n", text, re.S)
    assert m, "f2d_exact not found in k_element.cu"
    c = tmp_path / "f2d.c"
    c.write_text(HARNESS % m.group(0))
    exe = tmp_path / "f2d"
    subprocess.run([gcc, "-O2", "-std=c11", str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    n, bad = int(out[0]), int(out[1])
    assert n > 60_000_000
    assert bad == 0
