"""Eigenvalues only, and eigenvectors of a lowest subset of bands (the paper's two-pass form,
dstevx's index range), against the oracle (GPU only)."""
import numpy as np
import pytest

import oracle
from paper_1402_4247_gb300 import synth
from tests.gpu_helpers import TOL_EPS, TOL_RHO, check_problem, gpu_band_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4247_gb300.nao import Context
    c = Context(0)
    yield c
    c.close()


def test_eigenvalues_only(ctx):
    inp = synth.small_cell(33, 5, 8, kgrid=(1, 2, 1), nspin=2)
    t = dict(HR=torch.from_numpy(inp.HR).to(DEV), SR=torch.from_numpy(inp.SR).to(DEV)[None],
             R=torch.from_numpy(inp.R).to(DEV), k=torch.from_numpy(inp.kpts).to(DEV))
    n = inp.n
    Hk = ctx.nao_bloch_sum(t["HR"], t["R"], t["k"]).reshape(-1, n, n)
    Sk = ctx.nao_bloch_sum(t["SR"], t["R"], t["k"])[0]
    smap = torch.arange(inp.nprob, dtype=torch.int32, device=DEV) % inp.nk
    eps, C, m, st = ctx.nao_gen_eig(Hk, Sk, s_of_prob=smap, want_vectors=False)
    assert C is None
    eps, m, st = eps.cpu().numpy(), m.cpu().numpy(), st.cpu().numpy()
    ref = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT)
    for p in range(inp.nprob):
        assert st[p] == 0 and m[p] == ref["m"][p]
        e = ref["eps"][p]
        assert np.abs(eps[p][:m[p]] - e).max() <= TOL_EPS * np.abs(e).max()


@pytest.mark.parametrize("nb", [1, 40, 97])
def test_lowest_bands_only(ctx, nb):
    """nb eigenvectors of the lowest bands: the same eigenpairs (projectors) as the full solve,
    and Parts 5-6 unchanged while every occupied band lies below nb."""
    inp = synth.small_cell(33, 5, 8, kgrid=(1, 2, 1), nspin=2)
    g = gpu_band_step(ctx, inp, torch, DEV, nb=nb, density=nb >= 97)
    ref = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT)
    for p in range(inp.nprob):
        sg, k = divmod(p, inp.nk)
        check_problem(ref["Hk"][sg, k], ref["Sk"][k], g["eps"][p], g["C"][p], int(g["m"][p]), ref["eps"][p],
                      ref["C"][p], ref["m"][p], label=f"nb={nb} p={p}")
    if nb >= 97:
        assert int(g["rstatus"][0]) == 0
        assert np.abs(g["rho"] - ref["rho"]).max() <= TOL_RHO * max(1.0, np.abs(ref["rho"]).max())
        assert np.abs(g["edm"] - ref["edm"]).max() <= TOL_RHO * max(1.0, np.abs(ref["edm"]).max())
