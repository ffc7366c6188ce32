"""Failure detection on the device, driven by the context's settings (nao_config) and never by
a GPU fault: every device-side loop and wait is bounded, and a bound that runs out turns into
a per-problem status the host reads, while the context stays usable.

* inverse_iteration_max = 0: no eigenvector of the tridiagonal solve (Eigen_HH step 2) may pass
  its growth test, so every problem reports NAO_E_NOCONV; the vectors are still written and the
  eigenvalues (bisection) are unaffected.  Back at the default, the same call is clean again.
* tc_wait_cycles below 1024: each wait of a tensor-core product's copy/MMA pipeline is one
  non-blocking test, which the first copies cannot pass; the product's blocks let their copies
  land, free their tensor memory and raise the context's timeout flag.  The next nao_gen_eig
  (or nao_density_matrix) reports NAO_E_TIMEOUT once; the call after that is clean.
* hbm_budget_bytes: a call whose workspace would exceed the budget fails on the host with
  NAO_E_NOMEM before any launch."""
import numpy as np
import pytest

from paper_1402_4247_gb300 import synth
from tests.gpu_helpers import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _ctx(**kw):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4247_gb300.nao import Context
    return Context(0, **kw)


def _problems(ctx, inp):
    t = to_dev(inp, torch, DEV)
    n = inp.n
    Hk = ctx.nao_bloch_sum(t["HR"], t["R"], t["k"]).reshape(-1, n, n)
    Sk = ctx.nao_bloch_sum(t["SR"], t["R"], t["k"])[0]
    smap = torch.arange(inp.nprob, dtype=torch.int32, device=DEV) % inp.nk
    return t, Hk, Sk, smap


def test_inverse_iteration_cap_zero_reports_noconv():
    from paper_1402_4247_gb300.nao import NAO_E_NOCONV
    inp = synth.small_cell(21, 2, 3, kgrid=(2, 2, 1), nspin=2)   # n = 50, 8 problems
    ref = _ctx()
    _, Hk, Sk, smap = _problems(ref, inp)
    e0, C0, m0, s0 = ref.nao_gen_eig(Hk, Sk, s_of_prob=smap)
    torch.cuda.synchronize()
    assert int(s0.abs().sum()) == 0
    ctx = _ctx(config={"inverse_iteration_max": 0})
    assert ctx.nao_get_config()["inverse_iteration_max"] == 0
    e1, C1, m1, s1 = ctx.nao_gen_eig(Hk, Sk, s_of_prob=smap)
    torch.cuda.synchronize()
    assert (s1.cpu().numpy() == NAO_E_NOCONV).all(), s1
    assert torch.isfinite(C1).all()
    # the overlap eigenvalues come from bisection: the kept count is unaffected
    assert torch.equal(m1, m0)
    # the same context at the default cap: clean, and the same result as a fresh context
    ctx.nao_set_config(inverse_iteration_max=5)
    e2, C2, m2, s2 = ctx.nao_gen_eig(Hk, Sk, s_of_prob=smap)
    torch.cuda.synchronize()
    assert int(s2.abs().sum()) == 0
    fin = torch.isfinite(e0)
    assert torch.equal(fin, torch.isfinite(e2))
    assert float((e2[fin] - e0[fin]).abs().max()) <= 1e-12 * float(e0[fin].abs().max())
    ctx.close()
    ref.close()


def test_tensor_core_wait_expiry_reports_timeout_once():
    from paper_1402_4247_gb300.nao import NAO_E_TIMEOUT, NAO_GEMM_TC
    inp = synth.small_cell(23, 2, 3, kgrid=(2, 2, 1), nspin=1)   # n = 50, 4 problems
    ctx = _ctx()
    t, Hk, Sk, smap = _problems(ctx, inp)
    e0, C0, m0, s0 = ctx.nao_gen_eig(Hk, Sk, s_of_prob=smap)
    torch.cuda.synchronize()
    assert int(s0.abs().sum()) == 0
    default_wait = ctx.nao_get_config()["tc_wait_cycles"]
    # a product whose pipeline waits are single non-blocking tests: they expire
    rng = np.random.default_rng(5)
    A = torch.from_numpy(rng.standard_normal((2, 256, 512)) + 1j * rng.standard_normal((2, 256, 512))).to(DEV)
    B = torch.from_numpy(rng.standard_normal((2, 512, 128)) + 1j * rng.standard_normal((2, 512, 128))).to(DEV)
    ctx.nao_set_config(tc_wait_cycles=16)
    ctx.nao_zgemm(A, B, method=NAO_GEMM_TC)
    torch.cuda.synchronize()  # the product returned: no hang, no fault
    ctx.nao_set_config(tc_wait_cycles=default_wait)
    # reported by the next eigensolve (whose own products run normally) ...
    e1, C1, m1, s1 = ctx.nao_gen_eig(Hk, Sk, s_of_prob=smap)
    torch.cuda.synchronize()
    assert (s1.cpu().numpy() == NAO_E_TIMEOUT).all(), s1
    fin = torch.isfinite(e0)
    assert float((e1[fin] - e0[fin]).abs().max()) <= 1e-12 * float(e0[fin].abs().max())
    # ... once
    e2, C2, m2, s2 = ctx.nao_gen_eig(Hk, Sk, s_of_prob=smap)
    torch.cuda.synchronize()
    assert int(s2.abs().sum()) == 0
    # the density matrix reports a pending expiry the same way
    ctx.nao_set_config(tc_wait_cycles=16)
    ctx.nao_zgemm(A, B, method=NAO_GEMM_TC)
    ctx.nao_set_config(tc_wait_cycles=default_wait)
    mu, eb, f, rho, rst = ctx.nao_density_matrix(t["w"], t["k"], e2, C2, m2, inp.n_electrons, inp.kT, t["R"],
                                                 inp.nspin)
    torch.cuda.synchronize()
    assert int(rst[0]) == NAO_E_TIMEOUT
    mu, eb, f, rho, rst = ctx.nao_density_matrix(t["w"], t["k"], e2, C2, m2, inp.n_electrons, inp.kT, t["R"],
                                                 inp.nspin)
    torch.cuda.synchronize()
    assert int(rst[0]) == 0
    ctx.close()


def test_hbm_budget_refuses_oversized_workspace():
    from paper_1402_4247_gb300.nao import NAO_E_NOMEM, NaoError
    inp = synth.small_cell(25, 2, 3, kgrid=(2, 1, 1), nspin=1)
    ctx = _ctx(hbm_budget_bytes=1 << 16)   # far below one problem's workspace
    t = to_dev(inp, torch, DEV)
    n = inp.n
    # the Bloch sums below 8 k-points need no workspace
    Hk = ctx.nao_bloch_sum(t["HR"], t["R"], t["k"]).reshape(-1, n, n)
    Sk = ctx.nao_bloch_sum(t["SR"], t["R"], t["k"])[0]
    with pytest.raises(NaoError) as ei:
        ctx.nao_gen_eig(Hk, Sk)
    assert f"({NAO_E_NOMEM})" in str(ei.value) and "budget" in str(ei.value)
    assert ctx.workspace_bytes() == 0
    ctx.close()
    # the same call fits a budget of its own workspace size
    probe = _ctx()
    need = probe.nao_gen_eig_workspace(n, inp.nprob, inp.nprob)
    probe.close()
    ctx = _ctx(hbm_budget_bytes=need)
    eps, C, m, st = ctx.nao_gen_eig(Hk, Sk)
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0
    assert ctx.workspace_bytes() <= need
    ctx.close()


def test_config_range_checks():
    from paper_1402_4247_gb300.nao import NaoError, nao_config_defaults
    d = nao_config_defaults()
    assert d["inverse_iteration_max"] == 5 and d["f_min"] == 1e-16 and d["tc_wait_cycles"] == 4_000_000_000
    assert d["mixed_planes"] == 6 and d["overlap_mrrr"] == 1
    with pytest.raises(NaoError):
        _ctx(config={"inverse_iteration_max": -1})
    ctx = _ctx()
    for bad in ({"f_min": 0.5}, {"tc_wait_cycles": 0}, {"inverse_iteration_max": 65}, {"mixed_planes": 4},
                {"mixed_planes": 10}, {"overlap_mrrr": 2}):
        with pytest.raises(NaoError):
            ctx.nao_set_config(**bad)
    assert ctx.nao_get_config() == d
    ctx.close()
