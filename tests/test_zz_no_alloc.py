"""The allocation-free Fermi-level entry point gives the same mu, occupations and band energy
as the regular path (GPU only).

Callers that cannot let the library allocate device memory (a host code with its own fixed
memory pool, or a loop that must not synchronise the device) use nao_fermi_level_noalloc,
whose scratch is a static array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_1402_4247_gb300 import synth
from tests.gpu_helpers import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _regular(ctx, inp):
    t = to_dev(inp, torch, DEV)
    n = inp.n
    Hk = ctx.nao_bloch_sum(t["HR"], t["R"], t["k"]).reshape(-1, n, n)
    Sk = ctx.nao_bloch_sum(t["SR"], t["R"], t["k"])[0]
    smap = torch.arange(inp.nprob, dtype=torch.int32, device=DEV) % inp.nk
    eps, C, m, st = ctx.nao_gen_eig(Hk, Sk, s_of_prob=smap)
    mu, eb, f, rho, rst = ctx.nao_density_matrix(t["w"], t["k"], eps, C, m, inp.n_electrons, inp.kT, t["R"],
                                                 inp.nspin)
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0 and int(rst[0]) == 0
    return t, eps, m, C.shape[2], float(mu[0]), float(eb[0]), f.cpu().numpy()


def test_noalloc_fermi_matches_regular_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4247_gb300.nao import Context, nao_fermi_level_noalloc
    ctx = Context(0)
    # two calls in a row on different workloads (1 spin x 4 k, then 2 spins x 2 k), so a
    # second call that read stale scratch from the first would show
    for inp in (synth.tiny_cell(), synth.small_cell(31, 1, 2, kgrid=(2, 1, 1), nspin=2)):
        t, eps, m, nb, mu_ref, eb_ref, f_ref = _regular(ctx, inp)
        f = torch.full((inp.nprob, inp.n), -1.0, dtype=torch.float64, device=DEV)
        mu = torch.empty(1, dtype=torch.float64, device=DEV)
        eb = torch.empty(1, dtype=torch.float64, device=DEV)
        st = torch.full((1,), 12345, dtype=torch.int32, device=DEV)
        nao_fermi_level_noalloc(t["w"], eps, m, nb, inp.n_electrons, inp.kT, inp.nspin, f, mu, eb, st)
        torch.cuda.synchronize()
        assert int(st[0]) == 0
        # the tolerances of the parity tests: occupations 1e-9, band energy 1e-9 relative,
        # mu through the electron count it implies
        assert np.abs(f.cpu().numpy() - f_ref).max() <= 1e-9
        assert abs(float(eb[0]) - eb_ref) <= 1e-9 * max(1.0, abs(eb_ref))
        e = eps.cpu().numpy()
        g = 2.0 if inp.nspin == 1 else 1.0
        with np.errstate(over="ignore"):
            cnt = g * sum(inp.wk[p % inp.nk] * (1.0 / (1.0 + np.exp((e[p][np.isfinite(e[p])] - float(mu[0])) / inp.kT))).sum()
                          for p in range(inp.nprob))
        assert abs(cnt - inp.n_electrons) <= 1e-9 * max(1.0, inp.n_electrons)
    ctx.close()


def test_noalloc_rejects_oversized_problem_count():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4247_gb300.nao import NaoError, nao_fermi_level_noalloc
    nk = 40000  # 2 spins x 40000 k > 65536 problems
    wk = torch.full((nk,), 1.0 / nk, dtype=torch.float64, device=DEV)
    eps = torch.zeros((2 * nk, 1), dtype=torch.float64, device=DEV)
    m = torch.ones(2 * nk, dtype=torch.int32, device=DEV)
    f = torch.empty_like(eps)
    one = torch.empty(1, dtype=torch.float64, device=DEV)
    st = torch.empty(1, dtype=torch.int32, device=DEV)
    with pytest.raises(NaoError, match="fixed scratch limit"):
        nao_fermi_level_noalloc(wk, eps, m, 1, 1.0, 0.01, 2, f, one, one.clone(), st)
