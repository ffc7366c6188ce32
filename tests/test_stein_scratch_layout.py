"""Host check of the tridiagonal solver's scratch layout (no GPU).  `launch_stein` carves one
scratch array (`stein_scratch_doubles(n, nprob)` doubles) into the inverse-iteration arrays
(NARR n^2 per problem), which the bisection queue borrows before kernel 2 (qlo, qhi, the int4
entries, the split e^2: one queue slot per eigenvalue of every problem, and one norm per
problem), the eigenvalues by slot (n per problem), the big-cluster list (a count and
`big_capacity(n, nprob)` triples), the MRRR done flags (n ints per problem) and the queue
counter in the last two doubles.  `big_capacity`, `stein_scratch_doubles` and the constants are
taken verbatim from csrc/stein.cu; the carve-out below restates launch_stein's pointer
arithmetic, and every region must lie inside the array without overlapping the next."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEIN = os.path.join(ROOT, "paper_1402_4247_gb300", "csrc", "stein.cu")

DRIVER = r"""
#include <cstdio>
#include <cstddef>
#include <initializer_list>
%(consts)s
%(bigcap)s
%(scratch)s
int main() {
  long bad = 0, checked = 0;
  for (int n = 1; n <= 700; n += (n < 80 ? 1 : 13))
    for (int nprob : {1, 2, 3, 16, 64, 129}) {
      const size_t total = stein_scratch_doubles(n, nprob);           // doubles
      const size_t cap = (size_t)n * nprob;
      const size_t inv = (size_t)NARR * n * n * nprob;                // inverse-iteration arrays
      const size_t queue_end = 5 * cap + nprob;                       // qlo, qhi, qent (2 each), e2g, tng
      const size_t wslot = inv, wslot_end = wslot + cap;
      const size_t big_int0 = 2 * wslot_end;                          // ints from here on
      const size_t bigcap = (size_t)big_capacity(n, nprob);
      const size_t big_end_int = big_int0 + 1 + 3 * bigcap;
      const size_t mdone_int0 = big_int0 + 1 + 3 * bigcap + 1;
      const size_t mdone_end_int = mdone_int0 + cap;
      const size_t qcount_int = 2 * (total - 2);
      ++checked;
      if (queue_end > inv) ++bad;                                     // queue inside the borrowed arrays
      if (big_end_int > mdone_int0) ++bad;
      if (mdone_end_int > qcount_int) ++bad;                          // flags end before the counter
      if (qcount_int + 1 > 2 * total) ++bad;
      // at most n / (BIG + 1) clusters of more than BIG members per problem
      if ((size_t)nprob * (n / (BIG + 1)) > bigcap) ++bad;
    }
  printf("%%ld %%ld\n", bad, checked);
  return 0;
}
"""


def test_scratch_regions_fit(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    text = open(STEIN).read()
    consts = "\n".join(re.search(rf"constexpr int {c} = [^;]+;", text).group(0) for c in ("NARR", "BIG"))
    i = text.index("static int big_capacity(int n, int nprob)")
    bigcap = text[i:text.index("\n", i)]
    j = text.index("size_t stein_scratch_doubles(int n, int nprob) {")
    scratch = text[j:text.index("\n}\n", j) + 3]
    src = tmp_path / "drv.cpp"
    src.write_text(DRIVER % {"consts": consts, "bigcap": bigcap, "scratch": scratch})
    exe = tmp_path / "drv"
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", str(exe), str(src)], check=True)
    bad, checked = (int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                                    check=True).stdout.split())
    assert checked > 500
    assert bad == 0
