"""Seeded synthetic inputs for the NAO band step: real-space H(R), S(R), images, k-points.

This module only *makes inputs*.  It holds none of the band step's arithmetic (no Bloch
sum, no eigensolve, no occupations), so both the CUDA path and the CPU oracle can take
their inputs from it without sharing any of the method.

Model (a stand-in for a numerical-atomic-orbital basis, Sec. 3 of the paper: magnetite,
56 atoms, collinear spin, 64 k-points):

* atoms at seeded uniform positions in a cubic cell of side ``L`` (Angstrom) with a
  minimum-image separation of at least 1.8 A (rejection sampling);
* every atom carries ``norb`` s-like Gaussian orbitals with widths sigma_i drawn per
  orbital; orbitals of one atom are contiguous, atoms in generation order;
* overlap: the Gram matrix of the Gaussians over lattice images R,
  ``G_ij(R) = (2 s_i s_j / (s_i^2 + s_j^2))^{3/2} exp(-|r_i - r_j - R|^2 / (s_i^2 + s_j^2))``
  (equal widths give ``exp(-|d|^2 / (2 s^2))``), regularised so it is positive definite:
  ``S(R) = D^{-1/2} (G(R) + delta_{R,0} diag(eta)) D^{-1/2}``, ``D = diag(1 + eta)``, so
  ``S_ii(0) = 1``;
* Hamiltonian: ``H_ij(R) = -t_ij exp(-|r_i - r_j - R|^2 / (s_i^2 + s_j^2))`` with a
  symmetric hopping scale ``t_ij ~ U[0.5, 2] eV`` plus an onsite ``eps_i ~ N(0, 3 eV)`` at
  R = 0; a second spin channel adds ``Delta_i ~ U[1, 3] eV`` on the heavy-site orbitals;
* energies are stored in Hartree (1 Ha = 27.211386245988 eV).

``H_ij(R) = H_ji(-R)`` and ``S_ij(R) = S_ji(-R)`` hold exactly (the image set is symmetric
and the pair terms are computed once per unordered pair), so every Bloch sum is Hermitian.

The ``chain_*`` builders give the closed-form test systems (one- and two-orbital chains).
"""
from __future__ import annotations

import dataclasses
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HARTREE_EV = 27.211386245988
KT_001_EV = 0.01 / HARTREE_EV


@dataclasses.dataclass
class BandInput:
    """One band-step workload (all arrays C-contiguous, float64 unless noted).

    HR:   [nspin][nR][n][n]   real-space Hamiltonian blocks (Ha)
    SR:   [nR][n][n]          real-space overlap blocks
    R:    int32 [nR][3]       lattice images (integer cell vectors), symmetric under R -> -R
    kpts: [nk][3]             fractional k-points (units of the reciprocal lattice)
    wk:   [nk]                k weights, summing to 1
    """

    n: int
    nspin: int
    HR: np.ndarray
    SR: np.ndarray
    R: np.ndarray
    kpts: np.ndarray
    wk: np.ndarray
    n_electrons: float
    kT: float
    name: str = ""

    @property
    def nR(self) -> int:
        return int(self.R.shape[0])

    @property
    def nk(self) -> int:
        return int(self.kpts.shape[0])

    @property
    def nprob(self) -> int:
        return self.nspin * self.nk


def image_cube(r: int) -> np.ndarray:
    """All integer images with components in [-r, r], ordered lexicographically."""
    rng = range(-r, r + 1)
    return np.array([(a, b, c) for a in rng for b in rng for c in rng], dtype=np.int32)


def monkhorst_pack(q1: int, q2: int, q3: int) -> tuple[np.ndarray, np.ndarray]:
    """Monkhorst-Pack grid k_i = (2r - q - 1) / (2q), r = 1..q; equal weights."""
    axes = [np.array([(2 * r - q - 1) / (2.0 * q) for r in range(1, q + 1)]) for q in (q1, q2, q3)]
    k = np.array([(a, b, c) for a in axes[0] for b in axes[1] for c in axes[2]], dtype=np.float64)
    w = np.full(k.shape[0], 1.0 / k.shape[0])
    return k, w


def _positions(rng: np.random.Generator, natom: int, L: float, dmin: float) -> np.ndarray:
    pos = np.zeros((natom, 3))
    placed = 0
    tries = 0
    while placed < natom:
        tries += 1
        if tries > 2_000_000:
            raise RuntimeError("could not place atoms with the requested minimum separation")
        p = rng.uniform(0.0, L, size=3)
        if placed:
            d = pos[:placed] - p
            d -= L * np.round(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < dmin * dmin:
                continue
        pos[placed] = p
        placed += 1
    return pos


def make_cell(
    seed: int,
    L: float,
    species: list[tuple[int, int, float, float, bool]],
    image_radius: int,
    kgrid: tuple[int, int, int] | np.ndarray,
    nspin: int,
    eta_log10: tuple[float, float],
    n_electrons: float | None = None,
    kT: float = KT_001_EV,
    dup_every: int | None = None,
    name: str = "",
) -> BandInput:
    """Gaussian-orbital cell; ``species`` = [(natom, norb, sigma_lo, sigma_hi, heavy)].

    ``dup_every``: if set, one orbital in every ``dup_every`` (the last orbital of the
    atom it falls on, when that atom has another orbital) becomes an exact copy of its
    neighbour on the same atom: its whole row and column of S(R) and H(R), including the
    regularisation, equal the sibling's, so S(k) has exactly that many null directions.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    natom = sum(s[0] for s in species)
    pos = _positions(rng, natom, L, 1.8)
    centers, sig, heavy = [], [], []
    a = 0
    for (cnt, norb, lo, hi, hv) in species:
        for _ in range(cnt):
            for _o in range(norb):
                centers.append(pos[a])
                sig.append(rng.uniform(lo, hi))
                heavy.append(hv)
            a += 1
    centers = np.array(centers)
    sig = np.array(sig)
    heavy = np.array(heavy)
    n = centers.shape[0]
    R = image_cube(image_radius)
    nR = R.shape[0]

    t = rng.uniform(0.5, 2.0, size=(n, n))
    t = np.triu(t) + np.triu(t, 1).T  # symmetric per unordered pair
    onsite = rng.normal(0.0, 3.0, size=n)
    eta = 10.0 ** rng.uniform(eta_log10[0], eta_log10[1], size=n)
    delta = np.where(heavy, rng.uniform(1.0, 3.0, size=n), 0.0)

    s2 = sig[:, None] ** 2 + sig[None, :] ** 2
    pref = (2.0 * sig[:, None] * sig[None, :] / s2) ** 1.5
    dvec = centers[:, None, :] - centers[None, :, :]  # r_i - r_j

    SR = np.empty((nR, n, n))
    HR = np.empty((nspin, nR, n, n))
    r0 = next(ir for ir in range(nR) if not R[ir].any())
    th = -(t / HARTREE_EV)

    def image(ir):  # the images are independent: threads fill their own slices
        d = dvec - L * R[ir].astype(np.float64)[None, None, :]
        g = np.exp(-np.einsum("ijx,ijx->ij", d, d) / s2)
        SR[ir] = pref * g
        HR[0, ir] = th * g

    if n >= 256:
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(image, range(nR)))
    else:
        for ir in range(nR):
            image(ir)
    SR[r0] += np.diag(eta)
    HR[0, r0] += np.diag(onsite / HARTREE_EV)

    if dup_every:
        bounds = []
        o = 0
        for (cnt, norb, *_r) in species:
            for _ in range(cnt):
                bounds.append((o, o + norb))
                o += norb
        for target in range(dup_every - 1, n, dup_every):
            lo, hi = next(b for b in bounds if b[0] <= target < b[1])
            src = target - 1 if target - 1 >= lo else target + 1
            if not (lo <= src < hi):
                continue
            for M in (SR, HR[0]):
                M[..., target, :] = M[..., src, :]
                M[..., :, target] = M[..., :, src]
            eta[target] = eta[src]
            delta[target] = delta[src]

    dinv = 1.0 / np.sqrt(1.0 + eta)
    SR *= dinv[None, :, None] * dinv[None, None, :]
    if nspin == 2:
        HR[1] = HR[0]
        HR[1, r0] += np.diag(delta / HARTREE_EV)

    if isinstance(kgrid, tuple):
        kpts, wk = monkhorst_pack(*kgrid)
    else:
        kpts = np.ascontiguousarray(kgrid, dtype=np.float64)
        wk = np.full(kpts.shape[0], 1.0 / kpts.shape[0])
    if n_electrons is None:
        n_electrons = 2.0 * (n // 4)
    return BandInput(n=n, nspin=nspin, HR=np.ascontiguousarray(HR), SR=np.ascontiguousarray(SR),
                     R=R, kpts=kpts, wk=wk, n_electrons=float(n_electrons), kT=kT, name=name)


# ---------------------------------------------------------------------------------------
# The workloads.  Seeds follow the workload index (tiny = 1, magnetite-shaped = 2, ...).
# ---------------------------------------------------------------------------------------

def tiny_cell(seed: int = 1) -> BandInput:
    """8 atoms x 8 orbitals (n = 64) in an 8 A cube, 27 images, 2x2x1 k, 1 spin, 20 e."""
    return make_cell(seed, 8.0, [(8, 8, 0.8, 1.4, False)], 1, (2, 2, 1), 1, (-3.0, -1.0),
                     n_electrons=20.0, name="tiny n=64 nk=4 nspin=1")


def magnetite_cell(seed: int = 2, kgrid=(4, 4, 4), nspin: int = 2) -> BandInput:
    """Magnetite-shaped: 24 heavy x 13 + 32 light x 8 orbitals (n = 568), 8.4 A cube,
    125 images, 4x4x4 k, 2 spins (128 problems), N_e = 2 floor(n/4)."""
    return make_cell(seed, 8.4, [(24, 13, 1.0, 1.8, True), (32, 8, 0.7, 1.2, False)], 2, kgrid,
                     nspin, (-3.0, -1.0), name=f"magnetite-shaped n=568 nk={np.prod(kgrid) if isinstance(kgrid, tuple) else len(kgrid)} nspin={nspin}")


def scaled_cell(n: int, seed: int = 3, kgrid=(4, 4, 1), nspin: int = 1, ill_conditioned: bool = True,
                image_radius: int = 2) -> BandInput:
    """Same generator on a larger cell: n/25 heavy and 3n/50 light atoms (13h + 8l = n),
    L = 8.4 ((h + l)/56)^{1/3} A.  ``ill_conditioned`` pushes eta to ~1e-8 and duplicates one
    orbital in 50 (exact null directions of S), exercising the s^{-1/2} cutoff."""
    if n % 50:
        raise ValueError("n must be a multiple of 50")
    h, l = n // 25, 3 * n // 50
    L = 8.4 * ((h + l) / 56.0) ** (1.0 / 3.0)
    if ill_conditioned:
        return make_cell(seed, L, [(h, 13, 1.0, 2.2, True), (l, 8, 0.7, 1.2, False)], image_radius, kgrid,
                         nspin, (-8.5, -7.5), dup_every=50, name=f"large-basis n={n} ill-conditioned")
    return make_cell(seed, L, [(h, 13, 1.0, 1.8, True), (l, 8, 0.7, 1.2, False)], image_radius, kgrid,
                     nspin, (-3.0, -1.0), name=f"large-basis n={n}")


def small_cell(seed: int, natom_heavy: int, natom_light: int, kgrid=(2, 1, 1), nspin: int = 2,
               L: float | None = None, image_radius: int = 1) -> BandInput:
    """Reduced magnetite-like cell for parity tests (n = 13 h + 8 l, ragged sizes)."""
    if L is None:
        L = 8.4 * max((natom_heavy + natom_light) / 56.0, 0.15) ** (1.0 / 3.0) + 2.0
    sp = []
    if natom_heavy:
        sp.append((natom_heavy, 13, 1.0, 1.8, True))
    if natom_light:
        sp.append((natom_light, 8, 0.7, 1.2, False))
    return make_cell(seed, L, sp, image_radius, kgrid, nspin, (-3.0, -1.0),
                     name=f"small h={natom_heavy} l={natom_light}")


# ---------------------------------------------------------------------------------------
# Closed-form chains (for pins).  Supercell of N sites along x, lattice constant 1 cell.
# ---------------------------------------------------------------------------------------

def chain_1orb(N: int, alpha: float, beta: float, s: float, kpts: np.ndarray, nspin: int = 1,
               n_electrons: float = 0.0, kT: float = KT_001_EV) -> BandInput:
    """One orbital per site, onsite alpha, nearest-neighbour hopping beta and overlap s,
    periodic via the images R = (+-1, 0, 0).  Eigenvalues at supercell k:
    (alpha + 2 beta cos t_j) / (1 + 2 s cos t_j), t_j = 2 pi (k_x + j) / N."""
    R = np.array([[-1, 0, 0], [0, 0, 0], [1, 0, 0]], dtype=np.int32)
    H = np.zeros((3, N, N))
    S = np.zeros((3, N, N))
    for a in range(N):
        H[1, a, a] = alpha
        S[1, a, a] = 1.0
    for a in range(N - 1):
        H[1, a, a + 1] = H[1, a + 1, a] = beta
        S[1, a, a + 1] = S[1, a + 1, a] = s
    # wrap: orbital N-1 in cell 0 couples to orbital 0 in cell +1 (and the mirror)
    if N == 1:
        H[2, 0, 0] = H[0, 0, 0] = beta
        S[2, 0, 0] = S[0, 0, 0] = s
    elif N == 2:
        H[2, 1, 0] += beta
        H[0, 0, 1] += beta
        S[2, 1, 0] += s
        S[0, 0, 1] += s
    else:
        H[2, N - 1, 0] = beta
        H[0, 0, N - 1] = beta
        S[2, N - 1, 0] = s
        S[0, 0, N - 1] = s
    HR = np.repeat(H[None], nspin, axis=0)
    kpts = np.ascontiguousarray(np.atleast_2d(kpts), dtype=np.float64)
    wk = np.full(kpts.shape[0], 1.0 / kpts.shape[0])
    return BandInput(n=N, nspin=nspin, HR=HR, SR=S, R=R, kpts=kpts, wk=wk,
                     n_electrons=float(n_electrons), kT=kT, name=f"chain1 N={N}")


def chain_2orb(eA: float, eB: float, t1: float, t2: float, s1: float, s2: float,
               kpts: np.ndarray, n_electrons: float = 0.0, kT: float = KT_001_EV) -> BandInput:
    """Two orbitals A, B per cell: onsite eA, eB; intracell A-B hopping t1 / overlap s1;
    intercell coupling of A in cell 0 to B in cell -1 (t2, s2) only, so H_AB(k) is complex."""
    R = np.array([[-1, 0, 0], [0, 0, 0], [1, 0, 0]], dtype=np.int32)
    H = np.zeros((3, 2, 2))
    S = np.zeros((3, 2, 2))
    H[1] = [[eA, t1], [t1, eB]]
    S[1] = [[1.0, s1], [s1, 1.0]]
    H[0, 0, 1] = t2  # A(0) - B(-1)
    S[0, 0, 1] = s2
    H[2, 1, 0] = t2  # mirror: B(0) - A(+1)
    S[2, 1, 0] = s2
    kpts = np.ascontiguousarray(np.atleast_2d(kpts), dtype=np.float64)
    wk = np.full(kpts.shape[0], 1.0 / kpts.shape[0])
    return BandInput(n=2, nspin=1, HR=H[None], SR=S, R=R, kpts=kpts, wk=wk,
                     n_electrons=float(n_electrons), kT=kT, name="chain2")


def random_hermitian_pair(rng: np.random.Generator, n: int, cond: float = 10.0):
    """Dense complex Hermitian H and Hermitian positive-definite S (k-space, for solver tests)."""
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    H = (A + A.conj().T) / 2.0
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    s = np.logspace(0.0, -math.log10(cond), n) if n > 1 else np.ones(1)
    S = (Q * s) @ Q.conj().T
    S = (S + S.conj().T) / 2.0
    return np.ascontiguousarray(H), np.ascontiguousarray(S)
