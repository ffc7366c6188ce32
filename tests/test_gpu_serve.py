"""Serving through nao_serve_* (GPU only): continuous batching of band steps of mixed basis
size.  Each result must be the same alone and in a mix (where requests whose basis sizes lie
within a factor 1.25 share one eigensolve launch, the smaller ones padded, and batches overlap
on two slots), within the parity tolerances; admission follows the HBM budget; inputs may live
on the host or the device."""
import numpy as np
import pytest

import oracle
from paper_1402_4247_gb300 import synth
from tests.gpu_helpers import TOL_EPS, TOL_RHO, check_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
GB = 1 << 30


def _context(budget=8 * GB, max_batch=64, slots=2):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_4247_gb300.nao import Context
    c = Context(0)
    c.nao_serve_config(budget, max_batch, slots)
    return c


def _submit(ctx, inp, on_device=True, precision=0, nb=0):
    dev = DEV if on_device else "cpu"
    t = dict(HR=torch.from_numpy(inp.HR).to(dev), SR=torch.from_numpy(inp.SR).to(dev),
             R=torch.from_numpy(inp.R).to(dev), k=torch.from_numpy(inp.kpts).to(dev),
             w=torch.from_numpy(inp.wk).to(dev))
    torch.cuda.synchronize()
    return ctx.nao_serve_submit(t["HR"], t["SR"], t["R"], t["k"], t["w"], inp.n_electrons, inp.kT,
                                precision=precision, nb=nb)


def _collect(ctx, ticket):
    res = ctx.nao_serve_poll(ticket, -1)
    assert res.status == 0, f"request failed ({res.status})"
    out = {k: (v.cpu().numpy() if v is not None else None) for k, v in ctx.serve_result_tensors(res).items()}
    out["batch_requests"] = res.batch_requests
    out["latency_ms"] = res.latency_ms
    ctx.nao_serve_release(ticket)
    return out


CELLS = {
    "A64": lambda: synth.tiny_cell(),
    "B79": lambda: synth.small_cell(32, 3, 5, kgrid=(2, 2, 1), nspin=1),
    "C79": lambda: synth.small_cell(41, 3, 5, kgrid=(2, 1, 1), nspin=2),
    "D129": lambda: synth.small_cell(33, 5, 8, kgrid=(1, 2, 1), nspin=2),
}


def _same(a, b, label):
    fin = np.isfinite(b["eps"])
    assert np.array_equal(fin, np.isfinite(a["eps"])), label
    hn = np.abs(b["eps"][fin]).max()
    assert np.abs(a["eps"][fin] - b["eps"][fin]).max() <= TOL_EPS * hn, label
    assert np.array_equal(a["m"], b["m"]), label
    rmax = max(1.0, np.abs(b["rho"]).max())
    assert np.abs(a["rho"] - b["rho"]).max() <= TOL_RHO * rmax, label
    assert abs(a["mu"][0] - b["mu"][0]) <= 1e-9 and abs(a["eband"][0] - b["eband"][0]) <= 1e-9 * max(1, abs(b["eband"][0]))


def test_alone_and_in_the_mix():
    cells = {k: f() for k, f in CELLS.items()}
    ctx = _context(slots=1)
    try:
        alone = {k: _collect(ctx, _submit(ctx, inp)) for k, inp in cells.items()}
        for k, r in alone.items():
            assert r["batch_requests"] == 1, k
        # the mix: queued together while admission is held, B79, C79 and both copies of A64
        # (n = 64 padded to 79) share one launch; D129 is too large to join them
        order = ["D129", "B79", "A64", "C79", "A64"]
        ctx.nao_serve_pause(True)
        tickets = [(k, _submit(ctx, cells[k], on_device=(i % 2 == 0))) for i, k in enumerate(order)]
        ctx.nao_serve_pause(False)
        mixed = [(k, _collect(ctx, t)) for k, t in tickets]
    finally:
        ctx.close()
    for k, r in mixed:
        _same(r, alone[k], f"{k} in the mix")
    shared = {k: r["batch_requests"] for k, r in mixed}
    assert shared["B79"] == 4 and shared["C79"] == 4 and shared["A64"] == 4 and shared["D129"] == 1, shared
    # and two of them (one at the launch's order, one padded into it) against the oracle
    for name in ("B79", "A64"):
        inp = cells[name]
        ref = oracle.band_step(inp.HR, inp.SR, inp.R, inp.kpts, inp.wk, inp.n_electrons, inp.kT)
        r = dict(mixed)[name]
        assert r["eps"].shape == (inp.nprob, inp.n) and r["C"].shape == (inp.nprob, inp.n, inp.n)
        for p in range(inp.nprob):
            sg, k = divmod(p, inp.nk)
            check_problem(ref["Hk"][sg, k], ref["Sk"][k], r["eps"][p], r["C"][p], int(r["m"][p]), ref["eps"][p],
                          ref["C"][p], ref["m"][p], label=f"served {name} p={p}")
        assert np.abs(r["rho"] - ref["rho"]).max() <= TOL_RHO * max(1.0, np.abs(ref["rho"]).max())


def test_two_slots_match():
    cells = {k: f() for k, f in CELLS.items()}
    ctx = _context(slots=2)
    try:
        alone = {k: _collect(ctx, _submit(ctx, inp)) for k, inp in cells.items()}
        tickets = [(k, _submit(ctx, cells[k])) for k in ["D129", "A64", "B79", "C79", "D129", "A64"]]
        mixed = [(k, _collect(ctx, t)) for k, t in tickets]
        used, peak, queued, running = ctx.nao_serve_stats()
    finally:
        ctx.close()
    for k, r in mixed:
        _same(r, alone[k], f"{k} (two slots)")
    assert queued == 0 and running == 0 and peak > 0


def test_budget_admission():
    from paper_1402_4247_gb300.nao import NAO_E_NOMEM
    inp = synth.small_cell(33, 5, 8, kgrid=(1, 2, 1), nspin=2)
    # a budget far below one request: the request fails, nothing hangs
    ctx = _context(budget=1 << 20)
    try:
        res = ctx.nao_serve_poll(_submit(ctx, inp), -1)
        assert res.status == NAO_E_NOMEM
    finally:
        ctx.close()
    # room for about one request at a time: all complete, and the scheduler stays inside it
    ws = None
    ctx = _context(budget=256 << 20, slots=2)
    try:
        ws = ctx.nao_gen_eig_workspace(inp.n, inp.nprob, inp.nk)
        one = ws + 3 * inp.nprob * inp.n * inp.n * 16 + 4 * inp.nR * inp.n * inp.n * 8
        ctx.close()
        ctx = _context(budget=int(one * 1.6), slots=2)
        tickets = [_submit(ctx, inp) for _ in range(4)]
        outs = [_collect(ctx, t) for t in tickets]
        _, peak, _, _ = ctx.nao_serve_stats()
        assert peak <= int(one * 1.6)
        for o in outs[1:]:
            _same(o, outs[0], "budget-limited copy")
    finally:
        ctx.close()


def test_mixed_precision_request():
    inp = synth.small_cell(32, 3, 5, kgrid=(2, 2, 1), nspin=1)
    ctx = _context()
    try:
        a = _collect(ctx, _submit(ctx, inp, precision=0))
        b = _collect(ctx, _submit(ctx, inp, precision=2, on_device=False))
    finally:
        ctx.close()
    fin = np.isfinite(a["eps"])
    assert np.abs(a["eps"][fin] - b["eps"][fin]).max() <= 1e-9  # Ha, the mixed-mode bound
