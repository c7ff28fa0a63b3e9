"""The integer-pipe conversions between float and double (csrc/semd_convert.cuh) against the
host's IEEE 754 conversions.

The FP32-mixed pass kernel converts every sample of an IMF commit between the working
precision and the FP64 residue with these helpers instead of the hardware conversions, so
they must return exactly what IEEE conversion returns. The header is host-callable; this
test compiles it into a small host program and checks widening on every binary32 bit
pattern and narrowing on structured and random binary64 inputs: ties at every rounding
position, the ends of the normal range, overflow to infinity, subnormal results, zeros,
infinities and NaN.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2106_15319_gb300", "csrc")

PROGRAM = r"""
#include "semd_convert.cuh"
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <random>

static uint32_t fb(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }
static uint64_t db(double d) { uint64_t u; std::memcpy(&u, &d, 8); return u; }
static double dfrom(uint64_t u) { double d; std::memcpy(&d, &u, 8); return d; }
static float ffrom(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }

static long bad = 0;
static void check_narrow(double d) {
    const float want = (float)d, got = semd::narrow_float(d);
    if (std::isnan(want) ? !std::isnan(got) : fb(want) != fb(got)) {
        if (bad < 10) std::printf("narrow %a: want %a got %a\n", d, (double)want, (double)got);
        ++bad;
    }
}

int main() {
    // widening: every binary32 pattern
    for (uint64_t u = 0; u <= 0xffffffffull; ++u) {
        const float f = ffrom((uint32_t)u);
        const double want = (double)f, got = semd::widen(f);
        if (std::isnan(want) ? !std::isnan(got) : db(want) != db(got)) {
            if (bad < 10) std::printf("widen %08x\n", (unsigned)u);
            ++bad;
        }
    }
    // narrowing: every float neighbourhood at the ends and around ties
    const uint32_t anchors[] = {0x00000001u, 0x007fffffu, 0x00800000u, 0x00800001u, 0x3f800000u,
                                0x3f7fffffu, 0x3fffffffu, 0x7f7ffffeu, 0x7f7fffffu, 0x33000000u,
                                0x0c800000u, 0x34000000u};
    for (uint32_t a : anchors) {
        for (int sgn = 0; sgn < 2; ++sgn) {
            const double base = (double)ffrom(a | (sgn ? 0x80000000u : 0u));
            const uint64_t b = db(base);
            for (int64_t k = -70000; k <= 70000; ++k)
                check_narrow(dfrom(b + (uint64_t)k));
            // exact halfway points between base and its float neighbours, and 1 ulp around
            for (int dir = -1; dir <= 1; dir += 2) {
                const double nb = (double)std::nextafter((float)base, dir * INFINITY);
                const double mid = base + (nb - base) / 2;
                for (int j = -3; j <= 3; ++j)
                    check_narrow(dfrom(db(mid) + (uint64_t)(int64_t)j));
            }
        }
    }
    const double specials[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 1e-300, -1e-300, 1e300,
                               3.4028235677973366e38, 3.4028235677973362e38, 1.1754942e-38,
                               1.1754943508222875e-38, 1.401298464324817e-45, 7e-46};
    for (double d : specials)
        check_narrow(d);
    // random patterns, and random doubles in the float range
    std::mt19937_64 g(20210629);
    for (long i = 0; i < 20000000; ++i) {
        check_narrow(dfrom(g()));
        const int e = 1023 + (int)(g() % 300) - 150;
        check_narrow(dfrom(((uint64_t)(g() & 1) << 63) | ((uint64_t)e << 52) | (g() >> 12)));
    }
    std::printf("bad %ld\n", bad);
    return bad ? 1 : 0;
}
"""


def test_conversions_match_ieee(tmp_path):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    inc = None
    for cand in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            inc = os.path.join(cand, "include")
            break
    if inc is None:
        pytest.skip("CUDA headers not found")
    src = tmp_path / "conv.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "conv"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", inc, "-I", CSRC,
                    str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad 0" in r.stdout
