"""Two-stage Householder reduction (dense -> band -> tridiagonal, nao_config.band_width 16 or
32) against the CPU oracle, element by element on the same seeded inputs (GPU only).

The oracle reduces straight to tridiagonal form (the paper's Procedures 1-6), so agreement
is evidence for the band reduction, the bulge chase and both back-transformations."""
import numpy as np
import pytest

import oracle
from paper_1402_4247_gb300 import synth
from tests.gpu_helpers import TOL_RHO, check_problem, gpu_band_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", params=[(32, 1), (16, 1), (32, 0)], ids=["b32-tc", "b16-tc", "b32-fp64"])
def ctx(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4247_gb300.nao import Context
    bw, method = request.param
    c = Context(0, config={"band_width": bw})
    c.nao_set_gemm_method(method)
    assert c.nao_get_config()["band_width"] == bw
    yield c
    c.close()


@pytest.mark.parametrize("maker", [
    lambda: synth.tiny_cell(),                                          # n = 64: two panels of 32
    lambda: synth.small_cell(31, 1, 2, kgrid=(2, 1, 1), nspin=2),       # n = 29: no panel at B = 32
    lambda: synth.small_cell(32, 3, 5, kgrid=(2, 2, 1), nspin=1),       # n = 79: ragged last panel
    lambda: synth.small_cell(33, 5, 8, kgrid=(1, 2, 1), nspin=2),       # n = 129: several WY blocks
], ids=["tiny64", "n29", "n79", "n129"])
def test_two_stage_band_step_matches_oracle(ctx, maker):
    inp = maker()
    g = gpu_band_step(ctx, inp, torch, DEV)
    ref = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT)
    for p in range(inp.nprob):
        sg, k = divmod(p, inp.nk)
        check_problem(ref["Hk"][sg, k], ref["Sk"][k], g["eps"][p], g["C"][p], int(g["m"][p]), ref["eps"][p],
                      ref["C"][p], ref["m"][p], label=f"{inp.name} p={p}")
        assert int(g["status"][p]) == 0
    assert int(g["rstatus"][0]) == 0
    drho = np.abs(g["rho"] - ref["rho"]).max()
    assert drho <= TOL_RHO * max(1.0, np.abs(ref["rho"]).max()), f"rho differs by {drho:.3e}"


@pytest.mark.parametrize("n", [1, 2, 17, 33, 65, 130])
def test_two_stage_random_pencils(ctx, n):
    rng = np.random.Generator(np.random.PCG64(700 + n))
    H, S = synth.random_hermitian_pair(rng, n, cond=100.0)
    Ht = torch.from_numpy(np.ascontiguousarray(H[None])).to(DEV)
    St = torch.from_numpy(np.ascontiguousarray(S[None])).to(DEV)
    eps, C, m, st = ctx.nao_gen_eig(Ht, St)
    torch.cuda.synchronize()
    eo, Co, mo, _ = oracle.generalized_eigensolve(H, S)
    assert int(st[0]) == 0
    check_problem(H, S, eps.cpu().numpy()[0], C.cpu().numpy()[0], int(m[0]), eo, Co, mo, label=f"random n={n}")


def test_two_stage_cut_directions_and_subset(ctx):
    """Exactly singular overlap (H' of order m = n - 1 inside an n x n array: the rows and
    columns past m must not leak into the band reduction) and an eigenvector subset."""
    N = 40
    inp = synth.chain_1orb(N, 0.2, -0.6, 0.5, np.array([[0.0, 0.0, 0.0]]))
    g = gpu_band_step(ctx, inp, torch, DEV, density=False)
    assert int(g["m"][0]) == N - 1
    t = 2 * np.pi * np.arange(N) / N
    keep = np.abs(np.cos(t) + 1) > 1e-9
    exact = np.sort((0.2 - 1.2 * np.cos(t[keep])) / (1 + np.cos(t[keep])))
    assert np.abs(g["eps"][0][:N - 1] - exact).max() <= 1e-10 * np.abs(exact).max()
    assert np.isinf(g["eps"][0][N - 1])
    inp = synth.small_cell(34, 2, 2, kgrid=(2, 1, 1), nspin=1)  # n = 42
    g = gpu_band_step(ctx, inp, torch, DEV, nb=17, density=False)
    ref = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT,
                           problems=list(range(inp.nprob)))
    for p in range(inp.nprob):
        check_problem(ref["Hk"][0, p], ref["Sk"][p], g["eps"][p], g["C"][p], int(g["m"][p]), ref["eps"][p],
                      ref["C"][p], ref["m"][p], label=f"nb17 p={p}")


def test_two_stage_equals_one_stage_magnetite_sample():
    """The full n = 568 magnetite-shaped cell (4 k-points x 2 spins): the two-stage results
    against the one-stage ones and, for two problems, against the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4247_gb300.nao import Context
    inp = synth.magnetite_cell(kgrid=(2, 2, 1))
    c1 = Context(0)
    c2 = Context(0, config={"band_width": 32})
    g1 = gpu_band_step(c1, inp, torch, DEV, density=False)
    g2 = gpu_band_step(c2, inp, torch, DEV, density=False)
    c1.close()
    c2.close()
    assert np.array_equal(g1["m"], g2["m"])
    hn = np.abs(g1["eps"][np.isfinite(g1["eps"])]).max()
    assert np.abs(g1["eps"][np.isfinite(g1["eps"])] - g2["eps"][np.isfinite(g2["eps"])]).max() <= 2e-10 * hn
    ref = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT, problems=[0, 5])
    for p in (0, 5):
        sg, k = divmod(p, inp.nk)
        check_problem(ref["Hk"][sg, k], ref["Sk"][k], g2["eps"][p], g2["C"][p], int(g2["m"][p]), ref["eps"][p],
                      ref["C"][p], ref["m"][p], label=f"magnetite two-stage p={p}")


@pytest.mark.parametrize("bw", [32, 16])
def test_two_stage_mixed_precision_meets_mixed_bound(bw):
    """The mixed mode on the two-stage reduction (its stage-1 products of H' with the mixed
    planes, then the default Rayleigh-quotient refinement): eigenvalues within the mixed-mode
    bound of 1e-9 Ha of the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4247_gb300.nao import Context
    inp = synth.small_cell(33, 5, 8, kgrid=(1, 2, 1), nspin=2)  # n = 129
    ref = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT)
    c = Context(0, config={"band_width": bw})
    g = gpu_band_step(c, inp, torch, DEV, precision=2, density=False)
    c.close()
    for p in range(inp.nprob):
        m = int(g["m"][p])
        assert m == ref["m"][p] and int(g["status"][p]) == 0
        assert np.abs(g["eps"][p][:m] - ref["eps"][p]).max() <= 1e-9
