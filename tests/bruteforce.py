"""Exact (rational) characteristic-polynomial roots of small generalized Hermitian pencils.

Independent witness for the oracle: the double inputs are converted exactly to Gaussian
rationals, det(H - lambda S) is evaluated exactly at n + 1 integer points, the polynomial is
recovered by exact Lagrange interpolation, and its real roots are isolated with a Sturm
sequence and bisected in exact arithmetic."""
from fractions import Fraction


class CQ:
    """Exact complex rational a + b i."""
    __slots__ = ("a", "b")

    def __init__(self, a, b=Fraction(0)):
        self.a = Fraction(a)
        self.b = Fraction(b)

    def __add__(self, o):
        return CQ(self.a + o.a, self.b + o.b)

    def __sub__(self, o):
        return CQ(self.a - o.a, self.b - o.b)

    def __mul__(self, o):
        return CQ(self.a * o.a - self.b * o.b, self.a * o.b + self.b * o.a)

    def __truediv__(self, o):
        den = o.a * o.a + o.b * o.b
        return CQ((self.a * o.a + self.b * o.b) / den, (self.b * o.a - self.a * o.b) / den)

    def iszero(self):
        return self.a == 0 and self.b == 0


def _det(M):
    n = len(M)
    M = [row[:] for row in M]
    det = CQ(1)
    for c in range(n):
        piv = next((r for r in range(c, n) if not M[r][c].iszero()), None)
        if piv is None:
            return CQ(0)
        if piv != c:
            M[c], M[piv] = M[piv], M[c]
            det = CQ(0) - det
        det = det * M[c][c]
        for r in range(c + 1, n):
            if M[r][c].iszero():
                continue
            fac = M[r][c] / M[c][c]
            for j in range(c, n):
                M[r][j] = M[r][j] - fac * M[c][j]
    return det


def char_poly(H, S):
    """Coefficients (low to high, exact Fractions) of p(l) = det(H - l S); checks Im p = 0."""
    n = H.shape[0]
    Hq = [[CQ(Fraction(float(H[i, j].real)), Fraction(float(H[i, j].imag))) for j in range(n)] for i in range(n)]
    Sq = [[CQ(Fraction(float(S[i, j].real)), Fraction(float(S[i, j].imag))) for j in range(n)] for i in range(n)]
    xs = list(range(n + 1))
    ys = []
    for x in xs:
        lam = CQ(x)
        ys.append(_det([[Hq[i][j] - lam * Sq[i][j] for j in range(n)] for i in range(n)]))
    # Lagrange interpolation into monomial coefficients
    coef_re = [Fraction(0)] * (n + 1)
    coef_im = [Fraction(0)] * (n + 1)
    for i, xi in enumerate(xs):
        basis = [Fraction(1)]
        denom = Fraction(1)
        for j, xj in enumerate(xs):
            if j == i:
                continue
            basis = [Fraction(0)] + basis
            for t in range(len(basis) - 1):
                basis[t] -= xj * basis[t + 1]
            denom *= (xi - xj)
        for t in range(n + 1):
            coef_re[t] += ys[i].a * basis[t] / denom
            coef_im[t] += ys[i].b * basis[t] / denom
    return coef_re, coef_im


def _peval(c, x):
    r = Fraction(0)
    for a in reversed(c):
        r = r * x + a
    return r


def _prem(a, b):
    a = a[:]
    while len(a) >= len(b) and any(a):
        if a[-1] == 0:
            a.pop()
            continue
        f = a[-1] / b[-1]
        sh = len(a) - len(b)
        for t in range(len(b)):
            a[sh + t] -= f * b[t]
        a.pop()
    while a and a[-1] == 0:
        a.pop()
    return a


def _sturm(p):
    dp = [i * p[i] for i in range(1, len(p))]
    seq = [p, dp]
    while True:
        r = _prem(seq[-2], seq[-1])
        if not r:
            break
        seq.append([-x for x in r])
    return seq


def _changes(seq, x):
    vals = [_peval(s, x) for s in seq]
    vals = [v for v in vals if v != 0]
    return sum(1 for u, v in zip(vals, vals[1:]) if (u < 0) != (v < 0))


def real_roots(p, rel=1e-15):
    """All real roots (ascending floats) of a real polynomial with distinct roots."""
    while p and p[-1] == 0:
        p = p[:-1]
    seq = _sturm(p)
    bound = 1 + max(abs(c / p[-1]) for c in p[:-1])
    lo0, hi0 = -bound, bound
    roots = []

    def isolate(lo, hi):
        cnt = _changes(seq, lo) - _changes(seq, hi)
        if cnt == 0:
            return
        if cnt == 1:
            while hi - lo > Fraction(rel) * max(Fraction(1), abs(lo), abs(hi)):
                mid = (lo + hi) / 2
                if _changes(seq, lo) - _changes(seq, mid) == 1:
                    hi = mid
                else:
                    lo = mid
            roots.append(float((lo + hi) / 2))
            return
        mid = (lo + hi) / 2
        isolate(lo, mid)
        isolate(mid, hi)

    isolate(lo0, hi0)
    return sorted(roots)
