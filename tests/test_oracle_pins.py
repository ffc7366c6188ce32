"""Pins for the CPU oracle: values fixed by the paper's definitions and by mathematics,
never by the oracle itself (CPU only)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.optimize

import oracle
from paper_1402_4247_gb300 import synth
from tests import bruteforce

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _expr(s):
    return float(eval(s, {"__builtins__": {}}, {"sqrt": math.sqrt}))


def _frac(s):
    return float(Fraction(s))


# ----------------------------------------------------------------------------- Part 1

def test_bloch_sum_hand_values():
    """Sec. 3 Part 1 against hand-worked phases (tests/golden/bloch_hand.txt)."""
    R = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0]], dtype=np.int32)
    M = np.array([[[1, 2], [2, 3]], [[0, 5], [7, 0]], [[0, 7], [5, 0]], [[4, 0], [0, 0]], [[4, 0], [0, 0]]],
                 dtype=np.float64)
    rows = []
    with open(os.path.join(GOLDEN, "bloch_hand.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            k, ij, re, im = [t.strip() for t in line.split("|")]
            rows.append(([_frac(x) for x in k.split()], [int(x) for x in ij.split()], _expr(re), _expr(im)))
    assert len(rows) == 12
    for k, (i, j), re, im in rows:
        Mk = oracle.bloch_sum(M, R, np.array([k]))[0]
        assert abs(Mk[i, j] - complex(re, im)) < 1e-13, (k, i, j, Mk[i, j], re, im)


def test_bloch_sum_hermitian_on_cells():
    inp = synth.tiny_cell()
    Hk = oracle.bloch_sum(inp.HR, inp.R, inp.kpts)
    Sk = oracle.bloch_sum(inp.SR, inp.R, inp.kpts)
    for M in (Hk[0], Sk):
        for A in M:
            assert np.array_equal(A, A.conj().T) or np.abs(A - A.conj().T).max() < 1e-15


# ----------------------------------------------------------------------------- Eigen_HH

@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_tridiagonalization_preserves_spectrum_exact(n):
    """Eigen_HH step 1: the real tridiagonal (d, e) has exactly A's characteristic roots."""
    rng = np.random.Generator(np.random.PCG64(100 + n))
    A, _ = synth.random_hermitian_pair(rng, n)
    d, e, us, hs, delta = oracle.householder_tridiagonalize(A)
    cre, cim = bruteforce.char_poly(A, np.eye(n))
    assert all(c == 0 for c in cim)
    exact = bruteforce.real_roots(cre)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    got = np.sort(np.linalg.eigvalsh(T))
    assert len(exact) == n
    assert np.allclose(got, exact, rtol=0, atol=1e-13 * max(1.0, np.abs(exact).max()))
    assert np.all(e >= 0)


# Eigen_HH step 2: the oracle's own tridiagonal eigensolver (implicit QL), pinned on its own

def _tri(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 100, 301])
def test_ql_discrete_laplacian_closed_form(n):
    """tridiag(-1, 2, -1): eigenvalues 2 - 2 cos(j pi/(n+1)), eigenvectors sin(i j pi/(n+1))
    (distinct eigenvalues, so each column is fixed up to sign)."""
    w, Z = oracle.tridiagonal_eigensolve(2.0 * np.ones(n), -np.ones(n - 1))
    j = np.arange(1, n + 1)
    exact = 2.0 - 2.0 * np.cos(j * np.pi / (n + 1))
    assert np.abs(w - exact).max() <= 8e-15 * n
    zs = np.sin(np.outer(np.arange(1, n + 1), j) * np.pi / (n + 1))
    zs /= np.linalg.norm(zs, axis=0)
    dots = np.abs(np.sum(zs * Z, axis=0))
    assert np.abs(dots - 1.0).max() <= 1e-12


@pytest.mark.parametrize("n", [2, 5, 8, 33])
def test_ql_clement_matrix_integer_spectrum(n):
    """Zero diagonal, off-diagonals sqrt(i (n - i)): the eigenvalues are exactly
    -(n-1), -(n-3), ..., n-1 (the Clement / Kac-Sylvester matrix)."""
    i = np.arange(1, n)
    w, Z = oracle.tridiagonal_eigensolve(np.zeros(n), np.sqrt(i * (n - i)))
    exact = np.arange(-(n - 1), n, 2, dtype=float)
    assert np.abs(w - exact).max() <= 1e-13 * n


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_ql_exact_sturm_roots(n):
    """Random tridiagonals against the exact roots of det(T - l I) (rational arithmetic),
    with the residual and orthogonality of the eigenvectors."""
    rng = np.random.Generator(np.random.PCG64(300 + n))
    d = rng.standard_normal(n)
    e = rng.standard_normal(n - 1)
    T = _tri(d, e)
    cre, cim = bruteforce.char_poly(T.astype(complex), np.eye(n))
    exact = np.array(bruteforce.real_roots(cre))
    w, Z = oracle.tridiagonal_eigensolve(d, e)
    assert len(exact) == n
    assert np.abs(w - exact).max() <= 1e-14 * max(1.0, np.abs(exact).max())
    assert np.abs(Z.T @ Z - np.eye(n)).max() <= 1e-14
    assert np.abs(T @ Z - Z * w[None, :]).max() <= 1e-14 * max(1.0, np.abs(w).max())


def test_ql_split_blocks_clusters_and_grading():
    """Zero off-diagonals split T (the diagonal entries are eigenvalues); a Wilkinson W21+
    matrix has pairs of eigenvalues equal to ~1e-13 (orthogonality must survive); a graded
    matrix spans 1e-8 .. 1e8.  Residual and orthogonality at working precision."""
    cases = []
    d = np.array([3.0, 1.0, -2.0, 5.0, 0.5])
    cases.append((d, np.zeros(4), np.sort(d)))
    d = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    e = np.array([0.5, 0.0, 0.25, 0.0, 1.0])
    ex = np.sort(np.concatenate([np.linalg.eigvalsh(_tri(d[:2], e[:1])), np.linalg.eigvalsh(_tri(d[2:4], e[2:3])),
                                 np.linalg.eigvalsh(_tri(d[4:], e[4:]))]))
    cases.append((d, e, ex))
    cases.append((np.abs(np.arange(-10, 11)).astype(float), np.ones(20), None))
    g = 10.0 ** np.linspace(-8, 8, 12)
    cases.append((g, np.sqrt(g[:-1] * g[1:]) * 0.3, None))
    for d, e, ex in cases:
        w, Z = oracle.tridiagonal_eigensolve(d, e)
        T = _tri(d, e)
        nrm = np.abs(w).max()
        if ex is not None:
            assert np.abs(w - ex).max() <= 1e-14 * nrm
        assert np.all(np.diff(w) >= 0)
        assert np.abs(Z.T @ Z - np.eye(len(d))).max() <= 1e-13
        assert np.abs(T @ Z - Z * w[None, :]).max() <= 1e-14 * nrm * len(d)
    # W21+: the two largest eigenvalues agree to ~1e-13 and still get orthogonal vectors
    w, Z = oracle.tridiagonal_eigensolve(np.abs(np.arange(-10, 11)).astype(float), np.ones(20))
    assert w[-1] - w[-2] < 1e-12
    assert abs(Z[:, -1] @ Z[:, -2]) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_generalized_eigenvalues_vs_exact_char_poly(n):
    """Parts 2-4 against exact roots of det(H - l S) (Gaussian-rational arithmetic)."""
    rng = np.random.Generator(np.random.PCG64(200 + n))
    H, S = synth.random_hermitian_pair(rng, n, cond=20.0)
    cre, cim = bruteforce.char_poly(H, S)
    assert all(c == 0 for c in cim), "Im det(H - l S) must vanish for a Hermitian pencil"
    exact = np.array(bruteforce.real_roots(cre))
    eps, C, m, s = oracle.generalized_eigensolve(H, S)
    assert m == n and len(exact) == n
    assert np.abs(eps - exact).max() <= 1e-13 * max(1.0, np.abs(exact).max())
    assert np.abs(C.conj().T @ S @ C - np.eye(n)).max() < 1e-12
    assert np.abs(H @ C - S @ C * eps[None, :]).max() < 1e-12 * max(1.0, np.abs(eps).max())


@pytest.mark.parametrize("N,alpha,beta,s,k", [
    (7, 0.3, -0.5, 0.1, 0.0), (7, 0.3, -0.5, 0.1, 0.13), (10, -0.2, 0.4, 0.0, 0.5),
    (33, 0.1, -0.25, 0.3, 0.37), (64, 0.0, -1.0, 0.45, 0.0), (129, 0.05, -0.7, 0.2, 0.21)])
def test_chain_closed_form(N, alpha, beta, s, k):
    """One-orbital chain: eps_j = (alpha + 2 beta cos t_j) / (1 + 2 s cos t_j)."""
    inp = synth.chain_1orb(N, alpha, beta, s, np.array([[k, 0.0, 0.0]]))
    Hk = oracle.bloch_sum(inp.HR, inp.R, inp.kpts)[0, 0]
    Sk = oracle.bloch_sum(inp.SR, inp.R, inp.kpts)[0]
    t = 2 * np.pi * (k + np.arange(N)) / N
    exact = np.sort((alpha + 2 * beta * np.cos(t)) / (1 + 2 * s * np.cos(t)))
    eps, C, m, _ = oracle.generalized_eigensolve(Hk, Sk)
    assert m == N
    assert np.abs(eps - exact).max() < 1e-13 * max(1.0, np.abs(exact).max())


def test_chain_exactly_singular_overlap_cuts_one_direction():
    """s = 1/2 at t = pi: S has one exact null direction, so m = n - 1 (Part 2 cutoff)."""
    N = 8
    inp = synth.chain_1orb(N, 0.2, -0.6, 0.5, np.array([[0.0, 0.0, 0.0]]))
    Hk = oracle.bloch_sum(inp.HR, inp.R, inp.kpts)[0, 0]
    Sk = oracle.bloch_sum(inp.SR, inp.R, inp.kpts)[0]
    eps, C, m, s = oracle.generalized_eigensolve(Hk, Sk, s_cut=1e-10)
    assert m == N - 1
    t = 2 * np.pi * np.arange(N) / N
    keep = np.abs(np.cos(t) + 1) > 1e-9
    exact = np.sort((0.2 - 1.2 * np.cos(t[keep])) / (1 + np.cos(t[keep])))
    assert np.abs(eps - exact).max() < 1e-12 * max(1.0, np.abs(exact).max())


@pytest.mark.parametrize("k", [0.0, 0.17, 0.25, 0.5, 0.81])
def test_two_orbital_chain_closed_form(k):
    """Complex off-diagonal H_AB(k): eps = (-b +- sqrt(b^2 - 4ac)) / 2a, a = det S(k),
    b = -(h_AA s_BB + h_BB s_AA - 2 Re(h_AB conj(s_AB))), c = det H(k)."""
    eA, eB, t1, t2, s1, s2 = 0.3, -0.4, -0.7, -0.35, 0.2, 0.15
    inp = synth.chain_2orb(eA, eB, t1, t2, s1, s2, np.array([[k, 0.0, 0.0]]))
    Hk = oracle.bloch_sum(inp.HR, inp.R, inp.kpts)[0, 0]
    Sk = oracle.bloch_sum(inp.SR, inp.R, inp.kpts)[0]
    ph = np.exp(-2j * np.pi * k)
    hab = t1 + t2 * ph
    sab = s1 + s2 * ph
    assert abs(Hk[0, 1] - hab) < 1e-15 and abs(Sk[0, 1] - sab) < 1e-15
    a = 1.0 - abs(sab) ** 2
    b = -(eA + eB - 2 * (hab * np.conj(sab)).real)
    c = eA * eB - abs(hab) ** 2
    disc = math.sqrt(b * b - 4 * a * c)
    exact = np.sort([(-b - disc) / (2 * a), (-b + disc) / (2 * a)])
    eps, C, m, _ = oracle.generalized_eigensolve(Hk, Sk)
    assert np.abs(eps - exact).max() < 1e-14


def test_special_cases():
    rng = np.random.Generator(np.random.PCG64(7))
    # S = I: a standard Hermitian problem
    H, _ = synth.random_hermitian_pair(rng, 9)
    eps, C, m, _ = oracle.generalized_eigensolve(H, np.eye(9, dtype=complex))
    cre, _ = bruteforce.char_poly(H[:4, :4], np.eye(4))
    e4, _, _, _ = oracle.generalized_eigensolve(H[:4, :4], np.eye(4, dtype=complex))
    assert np.abs(e4 - np.array(bruteforce.real_roots(cre))).max() < 1e-13
    assert abs(eps.sum() - np.trace(H).real) < 1e-12
    # n = 1: eps = H / S
    eps, C, m, _ = oracle.generalized_eigensolve(np.array([[2.5 + 0j]]), np.array([[0.5 + 0j]]))
    assert m == 1 and abs(eps[0] - 5.0) < 1e-15 and abs(abs(C[0, 0]) - math.sqrt(2.0)) < 1e-15
    # diagonal H, S: eps = h_ii / s_ii
    h = np.array([3.0, -1.0, 0.5, 2.0, -4.0])
    s = np.array([1.0, 0.5, 2.0, 0.25, 1.5])
    eps, C, m, _ = oracle.generalized_eigensolve(np.diag(h).astype(complex), np.diag(s).astype(complex))
    assert np.abs(eps - np.sort(h / s)).max() < 1e-14


def test_invariants_tiny_cell():
    inp = synth.tiny_cell()
    out = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT)
    for p in range(inp.nprob):
        H, S = out["Hk"][0, p], out["Sk"][p]
        eps, C = out["eps"][p], out["C"][p]
        assert out["m"][p] == inp.n
        assert np.abs(C.conj().T @ S @ C - np.eye(inp.n)).max() < 1e-11
        hn = np.linalg.norm(H, 2)
        assert np.linalg.norm(H @ C - S @ C * eps[None, :]) / (inp.n * hn) < 1e-12
        tr = np.trace(np.linalg.solve(S, H)).real
        assert abs(eps.sum() - tr) < 1e-12 * max(abs(tr), np.abs(eps).sum())
        assert np.all(np.diff(eps) >= 0)
    # electron count and band energy through rho(R) (Part 6) and S(R), H(R)
    rho = out["rho"]
    ne = sum((rho[0, r] * inp.SR[r]).sum() for r in range(inp.nR))
    eb = sum((rho[0, r] * inp.HR[0, r]).sum() for r in range(inp.nR))
    assert abs(ne - inp.n_electrons) < 1e-9
    assert abs(eb - out["eband"]) < 1e-9 * max(1.0, abs(out["eband"]))
    for p in range(inp.nprob):
        f = out["f"][p]
        assert np.all((f >= 0) & (f <= 1))
    # energy density matrix (Part 6): sum E(R) S(R) = E_band and sum E(R) H(R) = g sum w f eps^2
    # (c^H S c = 1 and c^H H c = eps for each eigenvector)
    edm = out["edm"]
    es = sum((edm[0, r] * inp.SR[r]).sum() for r in range(inp.nR))
    eh = sum((edm[0, r] * inp.HR[0, r]).sum() for r in range(inp.nR))
    m2 = 2.0 * sum(inp.wk[p] * np.sum(out["f"][p] * out["eps"][p] ** 2) for p in range(inp.nprob))
    assert abs(es - out["eband"]) < 1e-9 * max(1.0, abs(out["eband"]))
    assert abs(eh - m2) < 1e-9 * max(1.0, abs(m2))


def test_two_spin_identities():
    inp = synth.small_cell(11, 1, 2, kgrid=(2, 1, 1), nspin=2)
    out = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT)
    rho = out["rho"]
    ne = sum((rho[sg, r] * inp.SR[r]).sum() for sg in range(2) for r in range(inp.nR))
    eb = sum((rho[sg, r] * inp.HR[sg, r]).sum() for sg in range(2) for r in range(inp.nR))
    assert out["g"] == 1.0
    assert abs(ne - inp.n_electrons) < 1e-9
    assert abs(eb - out["eband"]) < 1e-9 * max(1.0, abs(out["eband"]))


# ----------------------------------------------------------------------------- Part 5

def test_fermi_single_level_closed_form():
    kT = 0.01
    for f0 in (0.65, 0.05, 0.999):
        mu, f, eb = oracle.fermi_occupations([np.array([0.3])], [1.0], 2.0, 2.0 * f0, kT)
        assert abs(mu - (0.3 - kT * math.log(1.0 / f0 - 1.0))) < 1e-13
        assert abs(f[0][0] - f0) < 1e-12
        assert abs(eb - 2.0 * f0 * 0.3) < 1e-12


def test_fermi_symmetric_levels_half_filling():
    mu, f, eb = oracle.fermi_occupations([np.array([-0.2, 0.2]), np.array([-0.05, 0.05])], [0.5, 0.5], 2.0, 2.0,
                                         0.03)
    assert abs(mu) < 1e-14
    assert abs(eb - 2.0 * (0.5 * (-0.2 * f[0][0] + 0.2 * f[0][1]) + 0.5 * (-0.05 * f[1][0] + 0.05 * f[1][1]))) < 1e-15


# ----------------------------------------------------------------------------- Part 6

@pytest.mark.parametrize("N,k", [(6, 0.1), (9, 0.37)])
def test_density_matrix_plane_waves(N, k):
    """S = I chain at one non-symmetric k: eigenvectors are plane waves, so
    rho(R)_ab = Re[(g/N) sum_j f_j e^{i t_j (a-b)} e^{-2 pi i k R}] with t_j = 2 pi (k+j)/N.
    The occupations come from an independent root find on the closed-form bands."""
    alpha, beta, kT, Ne = 0.1, -0.5, 0.02, 5.0
    inp = synth.chain_1orb(N, alpha, beta, 0.0, np.array([[k, 0.0, 0.0]]), n_electrons=Ne, kT=kT)
    t = 2 * np.pi * (k + np.arange(N)) / N
    ej = alpha + 2 * beta * np.cos(t)

    def count(mu):
        return 2.0 * np.sum(1.0 / (1.0 + np.exp((ej - mu) / kT))) - Ne

    mu = scipy.optimize.brentq(count, ej.min() - 1, ej.max() + 1, xtol=1e-15, rtol=1e-15)
    fj = 1.0 / (1.0 + np.exp((ej - mu) / kT))
    out = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT)
    assert abs(out["mu"] - mu) < 1e-12
    a = np.arange(N)
    P = (fj[None, None, :] * np.exp(1j * t[None, None, :] * (a[:, None, None] - a[None, :, None]))).sum(-1) / N
    for ir, Rv in enumerate(inp.R):
        want = (2.0 * P * np.exp(-2j * np.pi * k * Rv[0])).real
        assert np.abs(out["rho"][0, ir] - want).max() < 1e-12
    # the energy density matrix: the same plane waves weighted by f_j eps_j
    PE = ((fj * ej)[None, None, :] * np.exp(1j * t[None, None, :] * (a[:, None, None] - a[None, :, None]))).sum(-1) / N
    for ir, Rv in enumerate(inp.R):
        want = (2.0 * PE * np.exp(-2j * np.pi * k * Rv[0])).real
        assert np.abs(out["edm"][0, ir] - want).max() < 1e-12
