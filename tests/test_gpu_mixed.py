"""Mixed-precision band step vs the CPU oracle (GPU only).

The mixed mode runs the back-transformations, X^H H X, the rank-2k updates of H' and X V
with reduced-precision tensor-core products (36 bits by default) and the Householder
matrix-vector products of H' with 46-bit digits, then refines with FP64-accurate products
of the input H and S.  The workload statement bounds it by |d eps| <= 1e-9 Ha over all kept
eigenvalues of every problem.  Each case runs raw (no refinement), with Rayleigh quotients
only (the default), and with 1 and 2 Ritz (Ogita-Aishima) sweeps: the quotients and every
sweep meet the eigenvalue bound, and each sweep squares the vector error (up to a factor
||H'|| / gap), which the test checks; the printed line reports the errors before and
after."""
import numpy as np
import pytest

import oracle
from paper_1402_4247_gb300 import synth
from tests.gpu_helpers import TOL_RHO, gpu_band_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_MIXED_EPS_HA = 1e-9
NAO_MIXED_TF32, NAO_MIXED_BF16X3 = 1, 2


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4247_gb300.nao import Context
    c = Context(0)
    yield c
    c.close()


def _errors(inp, g, ref):
    de = res = orth = 0.0
    for p in range(inp.nprob):
        sg, k = divmod(p, inp.nk)
        H, S = ref["Hk"][sg, k], ref["Sk"][k]
        m = int(g["m"][p])
        assert m == ref["m"][p]
        e = g["eps"][p][:m]
        de = max(de, np.abs(e - ref["eps"][p]).max())
        C = g["C"][p][:, :m]
        n = H.shape[0]
        res = max(res, np.linalg.norm(H @ C - S @ C * e[None, :]) / (n * np.linalg.norm(H, 2)))
        orth = max(orth, np.abs(C.conj().T @ S @ C - np.eye(m)).max())
    return de, res, orth


@pytest.mark.parametrize("maker", [
    lambda: synth.tiny_cell(),
    lambda: synth.small_cell(32, 3, 5, kgrid=(2, 2, 1), nspin=1),       # n = 79
    lambda: synth.small_cell(33, 5, 8, kgrid=(1, 2, 1), nspin=2),       # n = 129: several tiles + ragged tail
], ids=["tiny64", "n79", "n129"])
def test_mixed_refined_matches_oracle(ctx, maker):
    inp = maker()
    ref = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT)
    runs = {}
    for sweeps in (-1, 0, 1, 2):
        ctx.nao_set_refinement(sweeps)
        runs[sweeps] = gpu_band_step(ctx, inp, torch, DEV, precision=NAO_MIXED_BF16X3, density=sweeps == 2)
    ctx.nao_set_refinement(0)
    err = {k: _errors(inp, g, ref) for k, g in runs.items()}
    names = {-1: "raw", 0: "Rayleigh quotients", 1: "1 sweep", 2: "2 sweeps"}
    print("\n" + inp.name + ": " + "; ".join(
        f"{names[k]}: |d eps| {e[0]:.2e} Ha, residual {e[1]:.2e}, C^H S C - I {e[2]:.2e}" for k, e in err.items()))
    for g in runs.values():
        assert (g["status"] == 0).all()
        d = np.diff(g["eps"], axis=1)
        assert np.all(d[np.isfinite(d)] >= 0)
    # eigenvalues to the mixed-mode bound from the quotients alone and after each sweep; the
    # vector errors fall quadratically (e_{k+1} <= C e_k^2 with C ~ ||H'|| / gap, at most ~1e2
    # on these cells)
    (de0, res0, orth0), (deq, resq, orthq) = err[-1], err[0]
    (de1, res1, orth1), (de2, res2, orth2) = err[1], err[2]
    for de in (deq, de1, de2):
        assert de <= TOL_MIXED_EPS_HA, f"refined eigenvalues differ by {de:.3e} Ha"
    assert orth1 <= 1e3 * orth0 ** 2 + 1e-12 and orth2 <= 1e3 * orth1 ** 2 + 1e-12  # + rounding floor
    assert res1 < res0 and res2 <= max(res1, 1e-13)  # a second sweep stays at the rounding floor
    # Parts 5-6 on the twice-refined eigenpairs: rho to the FP64 bound, or to the first
    # order of the remaining vector error where that is larger
    g = runs[2]
    assert int(g["rstatus"][0]) == 0
    assert abs(g["eband"][0] - ref["eband"]) <= 1e-9 * max(1.0, abs(ref["eband"]))
    drho = np.abs(g["rho"] - ref["rho"]).max() / max(1.0, np.abs(ref["rho"]).max())
    assert drho <= max(TOL_RHO, 10 * orth2), f"rho differs by {drho:.3e} (relative)"


def test_mixed_precision_arguments(ctx):
    from paper_1402_4247_gb300.nao import NaoError
    inp = synth.tiny_cell()
    with pytest.raises(NaoError):
        gpu_band_step(ctx, inp, torch, DEV, precision=NAO_MIXED_TF32, density=False)
    with pytest.raises(NaoError):
        ctx.nao_set_refinement(3)
    with pytest.raises(NaoError):
        ctx.nao_set_refinement(-2)
    with pytest.raises(NaoError):
        gpu_band_step(ctx, inp, torch, DEV, precision=7, density=False)


def _host_norm2(H, iters=60):
    """||H||_2 of a Hermitian matrix by power iteration (an estimate from below, good to a
    few digits: enough for a residual's normalisation)."""
    v = np.random.default_rng(0).standard_normal(H.shape[0]) + 0j
    lam = 0.0
    for _ in range(iters):
        w = H @ v
        lam = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    return lam


def test_mixed_full_size_magnetite_against_oracle(ctx):
    """The magnetite-shaped step (n = 568, 128 problems in one call, the bench's launch
    configuration) in mixed precision: sampled problems against the oracle at the mixed-mode
    bound |d eps| <= 1e-9 Ha; residual and S-orthonormality after the one sweep."""
    inp = synth.magnetite_cell()
    ctx.nao_set_refinement(1)
    g = gpu_band_step(ctx, inp, torch, DEV, precision=NAO_MIXED_BF16X3)
    ctx.nao_set_refinement(0)
    gq = gpu_band_step(ctx, inp, torch, DEV, precision=NAO_MIXED_BF16X3, density=False)
    assert (g["status"] == 0).all() and int(g["rstatus"][0]) == 0
    sample = [3, 42, 64 + 17, 126]
    ref = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT, problems=sample)
    worst = {}
    for p in sample:
        sg, k = divmod(p, inp.nk)
        H, S = ref["Hk"][sg, k], ref["Sk"][k]
        m = int(g["m"][p])
        assert m == ref["m"][p]
        de = np.abs(g["eps"][p][:m] - ref["eps"][p]).max()
        C = g["C"][p][:, :m]
        res = np.linalg.norm(H @ C - S @ C * g["eps"][p][:m][None, :]) / (inp.n * _host_norm2(H))
        orth = np.abs(C.conj().T @ S @ C - np.eye(m)).max()
        deq = np.abs(gq["eps"][p][:m] - ref["eps"][p]).max()
        worst[p] = (de, res, orth, deq)
        assert de <= TOL_MIXED_EPS_HA, f"p={p}: |d eps| = {de:.3e} Ha"
        assert deq <= TOL_MIXED_EPS_HA, f"p={p}: |d eps| = {deq:.3e} Ha (Rayleigh quotients)"
        assert res <= 1e-9 and orth <= 1e-7, (p, res, orth)
    print("\nmagnetite mixed: " + "; ".join(f"p={p}: Rayleigh quotients |d eps| {v[3]:.2e} Ha; 1 sweep |d eps| "
                                            f"{v[0]:.2e} Ha, residual {v[1]:.2e}, C^H S C - I {v[2]:.2e}"
                                            for p, v in worst.items()))


def test_mixed_n2000_against_oracle_golden(ctx):
    """Two problems of the n = 2000 mixed-precision workload (4x4x4 k, seed 4) against the
    oracle's eigenvalues stored by tests/golden/make_mixed_n2000_oracle.py (oracle/ only):
    the mixed path (Rayleigh quotients) within 1e-9 Ha, the FP64 path within 1e-10 ||H'||."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "mixed_n2000_oracle_eps.txt")
    rows = np.loadtxt(path, comments="#")
    inp = synth.scaled_cell(2000, seed=4, kgrid=(4, 4, 4), nspin=1, ill_conditioned=False)
    probs = [int(p) for p in np.unique(rows[:, 0])]
    sub = inp.kpts[probs]
    HR = torch.from_numpy(inp.HR).to(DEV)
    SR = torch.from_numpy(inp.SR)[None].to(DEV)
    R = torch.from_numpy(inp.R).to(DEV)
    k = torch.from_numpy(np.ascontiguousarray(sub)).to(DEV)
    Hk = ctx.nao_bloch_sum(HR, R, k)[0]
    Sk = ctx.nao_bloch_sum(SR, R, k)[0]
    del HR, SR
    ctx.nao_set_refinement(0)
    for prec, tol in ((0, None), (NAO_MIXED_BF16X3, TOL_MIXED_EPS_HA)):
        eps, C, m, st = ctx.nao_gen_eig(Hk, Sk, precision=prec, want_vectors=False)
        torch.cuda.synchronize()
        assert int(st.abs().sum()) == 0
        e = eps.cpu().numpy()
        for i, p in enumerate(probs):
            r = rows[rows[:, 0] == p]
            mo = int(r[0, 1])
            eo = r[np.argsort(r[:, 2]), 3]
            assert int(m[i]) == mo
            bound = tol if tol is not None else 1e-10 * np.abs(eo).max()
            de = np.abs(e[i][:mo] - eo).max()
            assert de <= bound, (prec, p, de, bound)
            print(f"\nn2000 p={p} precision={prec}: |d eps| = {de:.2e} Ha (bound {bound:.1e})")
