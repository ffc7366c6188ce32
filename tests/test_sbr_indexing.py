"""Host check of the two-stage reduction's reflector indexing (no GPU).  The bulge chase stores
the reflector of sweep j, step k at slot q = j + F(n - 2) - F(n - 2 - j) + k, with
F(T) = sum_{t=0}^{T} floor(t / B) (`floor_sum`), and the stage-2 back-transformation reads the
same slots; each matrix has `sbr_q2_count(n, B)` slots.  Both functions are taken verbatim from
csrc/sbr.cu and compiled for the host.  For every padded order n, problem order m <= n and
band width B, the slots that the chase's steps write (sweeps j = 0 .. m - 2, each running until
its fill block would start past row m - 1) must be distinct and inside [0, sbr_q2_count(n, B))."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SBR = os.path.join(ROOT, "paper_1402_4247_gb300", "csrc", "sbr.cu")

DRIVER = r"""
#include <cstdio>
#include <vector>
#define __host__
#define __device__
%(floor_sum)s
%(count)s
static long long brute(long long T, int B) {
  long long s = 0;
  for (long long t = 0; t <= T; ++t) s += t / B;
  return s;
}
int main() {
  long bad_sum = 0, bad_slot = 0, checked = 0;
  for (int B : {16, 32})
    for (long long T = -3; T < 2000; ++T)
      if (floor_sum(T, B) != (T < 0 ? 0 : brute(T, B))) ++bad_sum;
  for (int B : {16, 32})
    for (int n = 1; n <= 300; ++n) {
      const long long cnt = sbr_q2_count(n, B);
      for (int m : {n, n - 1, (n + 1) / 2, 2, 1}) {
        if (m < 1 || m > n) continue;
        std::vector<char> used((size_t)cnt, 0);
        const long long fs_n = floor_sum(n - 2, B);
        for (int j = 0; j < m - 1; ++j) {
          const long long qbase = j + fs_n - floor_sum(n - 2 - j, B);
          int s1 = j + 1, k = 0;
          while (true) {  // the chase's step loop: one reflector per step
            const int s2 = s1 + B - 1 < m - 1 ? s1 + B - 1 : m - 1;
            const int t0 = s2 + 1;
            const int Lb = m - t0 < B ? m - t0 : B;
            const long long q = qbase + k;
            ++checked;
            if (q < 0 || q >= cnt || used[(size_t)q]) ++bad_slot;
            else used[(size_t)q] = 1;
            if (Lb <= 0) break;
            s1 = t0;
            ++k;
          }
          // the back-transformation's step count for sweep j
          if (k + 1 != (m - 2 - j) / B + 1) ++bad_slot;
        }
      }
    }
  printf("%%ld %%ld %%ld\n", bad_sum, bad_slot, checked);
  return 0;
}
"""


def _extract(text, start, end):
    i = text.index(start)
    j = text.index(end, i)
    return text[i:j + len(end)]


def test_chase_slots_distinct_and_in_range(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    text = open(SBR).read()
    fs = _extract(text, "__host__ __device__ inline long long floor_sum(", "\n}\n")
    cnt = _extract(text, "long long sbr_q2_count(int n, int B) {", "\n}\n")
    src = tmp_path / "drv.cpp"
    src.write_text(DRIVER % {"floor_sum": fs, "count": cnt})
    exe = tmp_path / "drv"
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", str(exe), str(src)], check=True)
    bad_sum, bad_slot, checked = (int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                                                  check=True).stdout.split())
    assert bad_sum == 0
    assert bad_slot == 0
    assert checked > 100000
