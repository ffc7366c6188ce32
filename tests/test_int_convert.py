"""Host checks of the integer arithmetic the CUDA kernels use in place of FP64 instructions
(no GPU): the fixed-point -> double conversion of the digit-plane GEMM epilogue
(`fix_to_double`) and the combination of the Householder DP4A digit orders (`hd_combine`).
Both functions are taken verbatim from the CUDA sources, compiled for the host with small
stand-ins for the three device intrinsics they call, and compared with exact integer
arithmetic rounded once (the C++ long double conversion of an exactly representable value)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1402_4247_gb300", "csrc")


def _extract(path, start, end):
    text = open(path).read()
    i = text.index(start)
    j = text.index(end, i)
    return text[i:j]


DRIVER = r"""
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <cmath>
#include <random>
#include <algorithm>
using std::max; using std::min;
#define __device__
#define __forceinline__ inline
static int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }
static double __longlong_as_double(long long b) { double d; memcpy(&d, &b, 8); return d; }
%(fix)s
%(comb)s
int main() {
  std::mt19937_64 g(11);
  long bad_fix = 0, bad_comb = 0;
  for (int it = 0; it < 2000000; ++it) {
    const int bits = (int)(g() %% 63);
    long long t = bits ? (long long)(g() >> (64 - bits)) : 0;
    if (it %% 5 == 0) t = ((long long)(g() >> 12) << 11) | 0x400;  // exact ties
    if (g() & 1) t = -t;
    const int ex = (int)(g() %% 600) - 300;
    const bool neg = g() & 1;
    const double r = fix_to_double(t, ex, neg);
    double ref = (double)ldexpl((long double)t, ex);  // t is exact in long double; one rounding
    if (neg) ref = -ref;
    if (!(r == ref || (r == 0 && ref == 0))) ++bad_fix;
  }
  for (int it = 0; it < 1000000; ++it) {
    int R[8];
    const int mag = (int)(g() %% 31);
    for (int k = 0; k < 8; ++k) { const long long x = mag ? (long long)(g() >> (64 - mag)) : 0; R[k] = (int)((g() & 1) ? -x : x); }
    if (it %% 3 == 0) R[0] = R[1] = R[2] = 0;
    const int ex = (int)(g() %% 200) - 100;
    for (int ng = 6; ng <= 8; ng += 2) {  // the digit counts the kernels use
      __int128 T = 0;
      for (int k = 0; k < ng; ++k) T += (__int128)R[k] * ((__int128)1 << (8 * (7 - k)));
      const double ref = (double)ldexpl((long double)T, ex - 56);
      const double r = ng == 8 ? hd_combine<8>(R, ex) : hd_combine<6>(R, ex);
      if (ref == 0) { if (r != 0) ++bad_comb; continue; }
      if (std::fabs((r - ref) / ref) > 0x1p-52) ++bad_comb;  // within one ulp of the exact sum
    }
  }
  printf("%%ld %%ld\n", bad_fix, bad_comb);
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    fix = _extract(os.path.join(CSRC, "nao_internal.cuh"), "__device__ __forceinline__ double fix_to_double(",
                   "\n}\n") + "\n}\n"
    comb = _extract(os.path.join(CSRC, "hetrd.cu"), "template <int NG>\n__device__ __forceinline__ double hd_combine(",
                    "\n}\n") + "\n}\n"
    assert re.search(r"HD_S = 8;", open(os.path.join(CSRC, "hetrd.cu")).read()), "digit count changed"
    d = tmp_path_factory.mktemp("intconv")
    src = d / "drv.cpp"
    src.write_text(DRIVER % {"fix": fix, "comb": comb})
    exe = d / "drv"
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", str(exe), str(src)], check=True)
    return str(exe)


DIGITS_DRIVER = r"""
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <cmath>
#include <random>
#define __device__
#define __forceinline__ inline
static long long __double_as_longlong(double x) { long long b; memcpy(&b, &x, 8); return b; }
%(fixed)s
%(digits)s
template <int S, int DB> static long check(std::mt19937_64& g, int bits) {
  long bad = 0;
  const int half = 1 << (DB - 1);
  for (int it = 0; it < 400000; ++it) {
    const int nb = 1 + (int)(g() %% bits);
    long long q = (long long)(g() >> (64 - nb));
    if (g() & 1) q = -q;
    int d[S];
    oz_digits<S, DB>(q, d);
    __int128 r = 0;
    for (int s = 0; s < S; ++s) r = r * ((__int128)1 << DB) + d[s];
    if (r != (__int128)q) ++bad;
    if (d[0] < -2 * half || d[0] > 2 * half) ++bad;
    for (int s = 1; s < S; ++s) if (d[s] < -half || d[s] >= half) ++bad;
  }
  // q = round(x 2^{DB S - e}) for |x| < 2^e, rounded half away from zero
  for (int it = 0; it < 400000; ++it) {
    const int e = (int)(g() %% 80) - 40;
    double x = ldexp((double)(g() >> 11) / 9007199254740992.0, e);  // [0, 2^e)
    x = ldexp(x, -(int)(g() %% 70));
    if (g() & 1) x = -x;
    const long long q = oz_fixed<S, DB>(x, e);
    const long double y = ldexpl((long double)x, DB * S - e);
    const long long ref = (long long)(y < 0 ? -floorl(-y + 0.5L) : floorl(y + 0.5L));
    if (q != ref) ++bad;
  }
  return bad;
}
int main() {
  std::mt19937_64 g(7);
  printf("%%ld %%ld\n", check<10, 6>(g, 60), check<9, 7>(g, 63));
  return 0;
}
"""


def test_digit_splits():
    """The digit-plane split of the FP64-accurate tensor-core products: q = round(x 2^{DB S - e})
    and its S balanced digits, for ten base-64 digits (60 bits) and nine base-128 digits (63
    bits): exact reconstruction and the digit ranges that the exactness bounds of the FP32
    group sums assume (lower digits in [-2^{DB-1}, 2^{DB-1}), the leading one within 2^DB)."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    src = os.path.join(CSRC, "ozgemm.cu")
    fixed = _extract(src, "template <int S, int DB>\n__device__ __forceinline__ long long oz_fixed(", "\n}\n") + "\n}\n"
    digits = _extract(src, "template <int S, int DB>\n__device__ __forceinline__ void oz_digits(", "\n}\n") + "\n}\n"
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "dig.cpp")
        open(c, "w").write(DIGITS_DRIVER % {"fixed": fixed, "digits": digits})
        exe = os.path.join(d, "dig")
        subprocess.run([cxx, "-O2", "-std=c++17", "-o", exe, c], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    assert out == ["0", "0"], out


def test_fixed_point_conversions(driver):
    out = subprocess.run([driver], check=True, capture_output=True, text=True).stdout.split()
    bad_fix, bad_comb = int(out[0]), int(out[1])
    assert bad_fix == 0, f"fix_to_double: {bad_fix} results differ from the correctly rounded value"
    assert bad_comb == 0, f"hd_combine: {bad_comb} results off by more than one ulp"
