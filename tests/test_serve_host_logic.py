"""Host checks of the serving loop's batching rules (no GPU): which queued request may join a
batch (`joins`) and the order and eigenvector count the batch's launch uses (`batch_shape`).
Both are taken verbatim from csrc/serve.cu and compiled for the host with a stand-in for the
request record that carries the fields they read."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SERVE = os.path.join(ROOT, "paper_1402_4247_gb300", "csrc", "serve.cu")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "nao.h"
struct ServeReq { nao_request rq{}; int nb = 0; };
struct Core {
%(rules)s
};
static ServeReq req(int n, int nb, int prec, double s_cut) {
  ServeReq r;
  r.rq.n = n;
  r.rq.precision = prec;
  r.rq.s_cut = s_cut;
  r.nb = nb;
  return r;
}
int main() {
  // joins: head (n, nb, precision; cutoff 1e-10), candidate (n, nb, precision, cutoff), the
  // batch's current order range
  int hn, hnb, prec, rn, rnb, rprec, nlo, nhi;
  double rcut;
  while (scanf("%%d %%d %%d %%d %%d %%d %%lf %%d %%d", &hn, &hnb, &prec, &rn, &rnb, &rprec, &rcut, &nlo, &nhi) == 9) {
    ServeReq h = req(hn, hnb, prec, 1e-10), r = req(rn, rnb, rprec, rcut);
    printf("%%d\n", Core::joins(&h, &r, nlo, nhi) ? 1 : 0);
  }
  // batch_shape on fixed batches
  const int shapes[][4] = {{64, 10, 64, 10}, {100, 100, 120, 120}, {120, 120, 100, 100}, {64, 64, 64, 64}};
  for (const auto& s : shapes) {
    ServeReq a = req(s[0], s[1], 0, 1e-10), b = req(s[2], s[3], 0, 1e-10);
    std::vector<ServeReq*> rs{&a, &b};
    int n = 0, nb = 0;
    Core::batch_shape(rs, &n, &nb);
    printf("shape %%d %%d\n", n, nb);
  }
  return 0;
}
"""


def _rules():
    text = open(SERVE).read()
    i = text.index("  // a batch's launch order n (its largest request's) and eigenvector columns nb")
    j = text.index("\n};\n", i)
    return text[i:j]


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("serve_rules")
    src = d / "drv.cpp"
    src.write_text(DRIVER % {"rules": _rules()})
    exe = d / "drv"
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    return str(exe)


# (head n, head nb, precision, cand n, cand nb, cand precision, cand s_cut, nlo, nhi) -> joins
CASES = [
    ((64, 64, 0, 64, 64, 0, 1e-10, 64, 64), 1),      # equal order, all vectors
    ((64, 10, 0, 64, 10, 0, 1e-10, 64, 64), 1),      # equal order, equal eigenvector subsets
    ((64, 10, 0, 64, 12, 0, 1e-10, 64, 64), 0),      # subsets differ and cannot be padded
    ((64, 64, 0, 64, 64, 2, 1e-10, 64, 64), 0),      # precision differs
    ((64, 64, 0, 64, 64, 0, 1e-8, 64, 64), 0),       # overlap cutoff differs
    ((100, 100, 0, 120, 120, 0, 1e-10, 100, 100), 1),  # 1.20x: padded into one launch
    ((100, 100, 0, 125, 125, 0, 1e-10, 100, 100), 1),  # exactly 1.25x
    ((100, 100, 0, 126, 126, 0, 1e-10, 100, 100), 0),  # beyond 1.25x
    ((100, 100, 0, 90, 90, 0, 1e-10, 100, 120), 0),    # widens the batch's range past 1.25x
    ((100, 100, 0, 110, 110, 0, 1e-10, 100, 120), 1),  # inside the range
    ((100, 100, 0, 110, 50, 0, 1e-10, 100, 100), 0),   # uneven order needs all vectors
    ((100, 60, 0, 110, 110, 0, 1e-10, 100, 100), 0),   # ... of the head too
    ((100, 100, 2, 110, 110, 2, 1e-10, 100, 100), 1),  # mixed precision batches as well
]


def test_joins(driver):
    inp = "".join(" ".join(str(v) for v in c) + "\n" for c, _ in CASES)
    out = subprocess.run([driver], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    got = [int(x) for x in out[:len(CASES)]]
    for (case, want), g in zip(CASES, got):
        assert g == want, f"joins{case} = {g}, expected {want}"


def test_batch_shape(driver):
    out = subprocess.run([driver], input="", capture_output=True, text=True, check=True).stdout.split("\n")
    shapes = [tuple(int(v) for v in line.split()[1:]) for line in out if line.startswith("shape")]
    # equal orders keep the requests' eigenvector count; uneven batches launch at the largest
    # order with all vectors
    assert shapes == [(64, 10), (120, 120), (120, 120), (64, 64)]
