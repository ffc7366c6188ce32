"""Plain numpy FP64 oracle of Band_DFT_Col (Sec. 3, Parts 1-6) -- test infrastructure only.

Readings of the paper taken here (each also listed in the design notes):

* Part 1, k-dependence: M(k) = sum_R exp(+2 pi i k.R) M(R), k fractional, R integer
  cell vectors (the form H(k) = sum_R e^{ik.R} H(R) of Sec. 3 Part 1).
* Procedure 2 ("subtract s from the i-th element"): the element is the first one below the
  diagonal and s carries the phase -x_0/|x_0|, so u_0 = x_0 + e^{i arg x_0} |x|: no
  cancellation.
* Procedure 4 ("p' = B u / (2 u^2)"): the textbook normalisation p = B u / h with
  h = |u|^2 / 2 (any consistent normalisation gives the same reflector).
* Procedure 5 (q' only defined in a missing reference): q = p - K u with K = u^H p / (2h),
  which makes Procedure 6, B <- B - q u^H - u q^H, the two-sided reflector update.
* The complex subdiagonal left by the procedures is made real by a diagonal unitary
  phase matrix before the tridiagonal solve.
* The LAPACK step of Eigen_HH: the paper allows dstevx, dstedc or dstegr; the oracle writes
  out the implicit QL method with Wilkinson shifts (no library eigensolver), so it reaches
  the tridiagonal eigenpairs by a different route from the GPU's bisection + inverse
  iteration.
* Part 2's "rearrange S": canonical orthogonalisation X = U_m diag(s_m^{-1/2}) over the
  eigenvalues s_j >= s_cut (absolute cutoff; negative s_j are cut as well).
* Part 3's "S^dagger H S" is X^H H X.
* Part 5: Fermi-Dirac occupations f = 1 / (1 + exp((eps - mu) / kT)), spin degeneracy
  g = 2 for one spin channel and 1 for two, mu by bisection on the electron count.
* Part 6: rho_sigma(R) = Re[ g sum_k w_k sum_n f_nk c_n c_n^H exp(-2 pi i k.R) ], the
  real-space matrix whose pairing with S(R) counts the electrons.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg.blas import drot as _rot


# --------------------------------------------------------------------------------------
# Part 1: giving k dependence to S and H
# --------------------------------------------------------------------------------------

def bloch_sum(MR: np.ndarray, R: np.ndarray, kpts: np.ndarray) -> np.ndarray:
    """Sec. 3 Part 1: M(k) = sum_R exp(2 pi i k.R) M(R).

    MR: [..., nR, n, n] real; R: [nR, 3] int; kpts: [nk, 3] fractional.
    Returns complex [..., nk, n, n]."""
    phase = np.exp(2j * np.pi * (np.asarray(kpts, dtype=np.float64) @ np.asarray(R, dtype=np.float64).T))
    return np.einsum("kr,...rij->...kij", phase, MR)


# --------------------------------------------------------------------------------------
# Eigen_HH step 1: Householder tridiagonalization, Procedures 1-6
# --------------------------------------------------------------------------------------

def householder_tridiagonalize(A: np.ndarray):
    """Sec. 3, Eigen_HH step 1 (Procedures 1-6) on a Hermitian matrix A.

    Returns (d, e, us, hs, delta): real tridiagonal (d, e) with
    D^H Q^H A Q D = tridiag(e, d, e), the reflectors u_i and scalars h_i that define
    P_i = I - u_i u_i^H / h_i acting on rows/columns i+1..n-1 (Q = P_0 P_1 ... P_{n-2}),
    and the diagonal phase delta of D."""
    B = np.array(A, dtype=np.complex128, copy=True)
    n = B.shape[0]
    us, hs = [], []
    b = np.zeros(max(n - 1, 0), dtype=np.complex128)
    for i in range(n - 1):
        u = B[i + 1:, i].copy()                         # Procedure 1
        s = np.linalg.norm(u)                           # Procedure 2
        if s == 0.0:
            us.append(None)
            hs.append(0.0)
            b[i] = 0.0
            continue
        ph = u[0] / abs(u[0]) if u[0] != 0 else 1.0 + 0.0j
        u[0] += ph * s
        h = 0.5 * np.vdot(u, u).real
        us.append(u)                                    # Procedure 3
        hs.append(h)
        B22 = B[i + 1:, i + 1:]
        p = (B22 @ u) / h                               # Procedure 4
        K = np.vdot(u, p).real / (2.0 * h)
        q = p - K * u                                   # Procedure 5
        B22 -= np.outer(q, u.conj()) + np.outer(u, q.conj())   # Procedure 6
        b[i] = -ph * s
        B[i + 1:, i] = 0.0
        B[i, i + 1:] = 0.0
        B[i + 1, i] = b[i]
        B[i, i + 1] = np.conj(b[i])
    d = B.diagonal().real.copy()
    e = np.abs(b)
    delta = np.ones(n, dtype=np.complex128)
    for j in range(n - 1):
        delta[j + 1] = delta[j] * (b[j] / abs(b[j]) if b[j] != 0 else 1.0)
    return d, e, us, hs, delta


# --------------------------------------------------------------------------------------
# Eigen_HH step 2: the tridiagonal eigensolver (implicit QL with Wilkinson shifts)
# --------------------------------------------------------------------------------------

_EPS = float(np.finfo(np.float64).eps)
_TINY = float(np.finfo(np.float64).tiny)


def tridiagonal_eigensolve(d: np.ndarray, e: np.ndarray, max_sweeps_per_value: int = 30):
    """Sec. 3, Eigen_HH step 2: all eigenpairs of the real symmetric tridiagonal T with
    diagonal d[0..n) and off-diagonal e[0..n-1), eigenvalues ascending.

    The paper hands this step to LAPACK (dstevx, dstedc or dstegr).  The oracle takes the
    implicit QL method with Wilkinson shifts instead, written out here, with the plane
    rotations accumulated into Z (T = Z diag(w) Z^T), so that it reaches the eigenpairs by a
    route of its own, different from the CUDA path's bisection + inverse iteration:

    * Deflation: an off-diagonal e_i with |e_i| <= eps (|d_i| + |d_{i+1}|) is set to zero,
      which splits T.  The eigenvalue at the top of the unreduced block [l, m] is found
      when the block shrinks to one row (l = m); then l moves down by one.
    * Shift: the eigenvalue of the leading 2 x 2 block [[d_l, e_l], [e_l, d_{l+1}]] that lies
      closer to d_l (Wilkinson's choice), sigma = d_l - e_l^2 / (delta + sign(delta)
      sqrt(delta^2 + e_l^2)) with delta = (d_{l+1} - d_l) / 2.
    * One QL sweep on T[l..m]: the first rotation, in the plane (m-1, m), is the one that
      annihilates entry (m-1, m) of P (T - sigma I); applied to T as T <- P T P^T it leaves a
      bulge at (m-2, m).  Each further rotation in the plane (i, i+1), i = m-2 .. l, removes
      the bulge at (i, i+2) and creates the next at (i-1, i+1), until it leaves the block at
      the top.  Z <- Z P^T accumulates every rotation: columns (z_i, z_{i+1}) become
      (c z_i + s z_{i+1}, -s z_i + c z_{i+1}).
    The scalar recurrences run on Python floats (IEEE doubles); the columns of Z are rows of
    a C-ordered array, and each plane rotation of a pair of them is the BLAS level-1 routine
    drot (x, y <- c x + s y, c y - s x), a library primitive.
    """
    dl = [float(x) for x in np.asarray(d, dtype=np.float64)]
    n = len(dl)
    off = [float(x) for x in np.asarray(e, dtype=np.float64)] + [0.0]  # off[i] couples rows i, i+1
    Zt = np.eye(n)                               # rows of Zt are the columns of Z
    hypot = math.hypot
    for l in range(n):
        sweeps = 0
        while True:
            # end m of the unreduced block that starts at l
            m = l
            while m < n - 1:
                if abs(off[m]) <= _EPS * (abs(dl[m]) + abs(dl[m + 1])) or abs(off[m]) <= _TINY:
                    off[m] = 0.0
                    break
                m += 1
            if m == l:
                break                            # dl[l] is an eigenvalue
            sweeps += 1
            if sweeps > max_sweeps_per_value:
                raise np.linalg.LinAlgError("implicit QL: no convergence")
            # Wilkinson shift from the leading 2 x 2 block
            delta = 0.5 * (dl[l + 1] - dl[l])
            root = hypot(delta, off[l])
            sigma = dl[l] - off[l] * off[l] / (delta + (root if delta >= 0.0 else -root))
            # first rotation, plane (m-1, m): zero (m-1, m) of P (T - sigma I)
            x, z = dl[m] - sigma, off[m - 1]
            for i in range(m - 1, l - 1, -1):
                r = hypot(x, z)
                if r > 0.0:
                    c, s = x / r, -z / r
                else:
                    c, s = 1.0, 0.0
                if i < m - 1:
                    off[i + 1] = r                # (i+1, i+2) once the bulge at (i, i+2) is gone
                a, b, dd = dl[i], off[i], dl[i + 1]
                cs2 = 2.0 * c * s * b
                dl[i] = c * c * a + cs2 + s * s * dd
                dl[i + 1] = s * s * a - cs2 + c * c * dd
                off[i] = c * s * (dd - a) + (c * c - s * s) * b
                if i > l:                          # new bulge at (i-1, i+1)
                    bulge = -s * off[i - 1]
                    off[i - 1] = c * off[i - 1]
                    x, z = off[i], bulge           # the next rotation zeroes the bulge
                _rot(Zt[i], Zt[i + 1], c, s, overwrite_x=1, overwrite_y=1)
    w = np.array(dl)
    order = np.argsort(w, kind="stable")
    return w[order], np.ascontiguousarray(Zt[order].T)


# --------------------------------------------------------------------------------------
# Eigen_HH steps 3-4: rearrangement (back-transformation) and normalization
# --------------------------------------------------------------------------------------

def rearrange_eigenvectors(Z: np.ndarray, us, hs, delta) -> np.ndarray:
    """Sec. 3, Eigen_HH steps 3 and 4: U = Q D Z with Q = P_0 ... P_{n-2} applied from the
    last reflector to the first, then every column scaled to unit 2-norm."""
    V = delta[:, None] * np.asarray(Z, dtype=np.complex128)
    for i in range(len(us) - 1, -1, -1):
        u = us[i]
        if u is None:
            continue
        blk = V[i + 1:, :]
        blk -= np.outer(u, (u.conj() @ blk) / hs[i])
    V /= np.linalg.norm(V, axis=0)[None, :]
    return V


def eigen_hh(A: np.ndarray, tridiagonal=None):
    """Sec. 3 Eigen_HH: eigenvalues (ascending) and orthonormal eigenvectors of Hermitian A.
    ``tridiagonal`` replaces the step-2 solver (a function (d, e) -> (w, Z)) when a test
    wants another route through the same steps 1, 3 and 4."""
    d, e, us, hs, delta = householder_tridiagonalize(A)
    w, Z = (tridiagonal or tridiagonal_eigensolve)(d, e)
    return w, rearrange_eigenvectors(Z, us, hs, delta)


# --------------------------------------------------------------------------------------
# Parts 2-4: the generalized eigenproblem H C = S C eps
# --------------------------------------------------------------------------------------

def generalized_eigensolve(H: np.ndarray, S: np.ndarray, s_cut: float = 1e-10, tridiagonal=None):
    """Sec. 3 Parts 2-4.

    Part 2: Eigen_HH(S) -> s, U; X = U_m s_m^{-1/2} over s_j >= s_cut.
    Part 3: H' = X^H H X (made exactly Hermitian from its lower triangle).
    Part 4: Eigen_HH(H') -> eps, V; C = X V.
    Returns (eps [m], C [n, m], m, s [n])."""
    s, U = eigen_hh(S, tridiagonal)
    keep = s >= s_cut
    X = U[:, keep] / np.sqrt(s[keep])[None, :]
    Hp = X.conj().T @ H @ X
    L = np.tril(Hp, -1)
    Hp = L + L.conj().T + np.diag(Hp.diagonal().real)
    m = int(keep.sum())
    if m == 0:
        return np.zeros(0), np.zeros((H.shape[0], 0), dtype=np.complex128), 0, s
    eps, V = eigen_hh(Hp, tridiagonal)
    return eps, X @ V, m, s


# --------------------------------------------------------------------------------------
# Part 5: chemical potential and band energy
# --------------------------------------------------------------------------------------

def _fermi(x: np.ndarray) -> np.ndarray:
    """f(x) = 1 / (1 + e^x), evaluated without overflow."""
    out = np.empty_like(x)
    neg = x <= 0.0
    out[neg] = 1.0 / (1.0 + np.exp(x[neg]))
    ex = np.exp(-x[~neg])
    out[~neg] = ex / (1.0 + ex)
    return out


def fermi_occupations(eps_list, w_list, g: float, n_electrons: float, kT: float,
                      max_iter: int = 200):
    """Sec. 3 Part 5: mu with g sum_p w_p sum_n f((eps_pn - mu)/kT) = N_e, by bisection.

    eps_list: per problem, its m_p eigenvalues; w_list: the problem's k weight.
    Returns (mu, [f_p], E_band) with E_band = g sum_p w_p sum_n f_pn eps_pn."""
    allv = np.concatenate([np.asarray(e, dtype=np.float64) for e in eps_list])
    cap = g * sum(w * len(e) for e, w in zip(eps_list, w_list))
    if not (0.0 <= n_electrons <= cap):
        raise ValueError("electron count outside [0, number of states]")

    def count(mu):
        return g * sum(w * _fermi((np.asarray(e) - mu) / kT).sum() for e, w in zip(eps_list, w_list))

    lo = allv.min() - 40.0 * kT
    hi = allv.max() + 40.0 * kT
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi or hi - lo <= 1e-15 * max(1.0, abs(mid)):
            break
        if count(mid) < n_electrons:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    f = [_fermi((np.asarray(e) - mu) / kT) for e in eps_list]
    eband = g * sum(w * float(np.dot(fp, e)) for fp, e, w in zip(f, eps_list, w_list))
    return mu, f, eband


# --------------------------------------------------------------------------------------
# Part 6: charge density matrix
# --------------------------------------------------------------------------------------

def density_matrix(C_list, f_list, w_list, kpts_of_prob, R: np.ndarray, g: float) -> np.ndarray:
    """Sec. 3 Part 6: rho(R) = Re[ g sum_p w_p (C_p diag(f_p) C_p^H) exp(-2 pi i k_p.R) ]
    summed over the problems of one spin channel.  Returns real [nR, n, n]."""
    n = C_list[0].shape[0]
    Rf = np.asarray(R, dtype=np.float64)
    rho = np.zeros((Rf.shape[0], n, n))
    for C, f, w, k in zip(C_list, f_list, w_list, kpts_of_prob):
        P = (C * f[None, :]) @ C.conj().T
        ph = np.exp(-2j * np.pi * (Rf @ np.asarray(k, dtype=np.float64)))
        rho += g * w * (ph[:, None, None] * P[None, :, :]).real
    return rho


# --------------------------------------------------------------------------------------
# Band_DFT_Col, single pass (Parts 1-6)
# --------------------------------------------------------------------------------------

def band_step(HR, SR, R, kpts, wk, n_electrons: float, kT: float, s_cut: float = 1e-10,
              problems=None):
    """Sec. 3 Band_DFT_Col on real-space inputs HR [nspin][nR][n][n], SR [nR][n][n].

    Problem p = sigma * nk + k.  Returns a dict with Hk, Sk, eps, C, m, mu, f, eband, rho
    and edm (the energy density matrix).
    ``problems`` restricts Parts 2-4 to a subset (then mu/f/rho are not computed)."""
    nspin = HR.shape[0]
    nk = kpts.shape[0]
    g = 2.0 if nspin == 1 else 1.0
    Hk = bloch_sum(HR, R, kpts)           # [nspin][nk][n][n]
    Sk = bloch_sum(SR, R, kpts)           # [nk][n][n]
    plist = range(nspin * nk) if problems is None else problems
    eps, C, m = {}, {}, {}
    for p in plist:
        sg, k = divmod(p, nk)
        eps[p], C[p], m[p], _ = generalized_eigensolve(Hk[sg, k], Sk[k], s_cut)
    out = dict(Hk=Hk, Sk=Sk, eps=eps, C=C, m=m)
    if problems is not None:
        return out
    ps = list(range(nspin * nk))
    mu, f, eband = fermi_occupations([eps[p] for p in ps], [wk[p % nk] for p in ps], g, n_electrons, kT)
    rho = np.stack([
        density_matrix([C[p] for p in ps if p // nk == sg], [f[p] for p in ps if p // nk == sg],
                       [wk[p % nk] for p in ps if p // nk == sg], [kpts[p % nk] for p in ps if p // nk == sg],
                       R, g)
        for sg in range(nspin)])
    # Part 6's second output, the energy density matrix: the same sum with weights f eps
    edm = np.stack([
        density_matrix([C[p] for p in ps if p // nk == sg], [f[p] * eps[p] for p in ps if p // nk == sg],
                       [wk[p % nk] for p in ps if p // nk == sg], [kpts[p % nk] for p in ps if p // nk == sg],
                       R, g)
        for sg in range(nspin)])
    out.update(mu=mu, f={p: f[i] for i, p in enumerate(ps)}, eband=eband, rho=rho, edm=edm, g=g)
    return out
