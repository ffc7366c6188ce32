"""Argument checks of the Python binding (CPU): every shape, dtype and device the library
entry points read is verified before a pointer reaches a kernel.  The checks take the device
as an argument, so they run here on CPU tensors; the shapes are the ones the band step, the
benchmark and the tests pass."""
import pytest

torch = pytest.importorskip("torch")

from paper_1402_4247_gb300 import synth  # noqa: E402
from paper_1402_4247_gb300.nao import (check_bloch_sum_args, check_density_matrix_args,  # noqa: E402
                                       check_gen_eig_args, check_serve_request_args, check_zgemm_args)

CPU = torch.device("cpu")
C128, F64, I32 = torch.complex128, torch.float64, torch.int32


def _step_tensors(nspin=2):
    """The band step's tensors for a small cell, shaped as the benchmark allocates them."""
    inp = synth.small_cell(25, 2, 3, kgrid=(2, 1, 1), nspin=nspin)
    n, nk, nR, nprob = inp.n, inp.nk, inp.nR, inp.nprob
    t = dict(HR=torch.from_numpy(inp.HR), SR=torch.from_numpy(inp.SR)[None], R=torch.from_numpy(inp.R),
             k=torch.from_numpy(inp.kpts), w=torch.from_numpy(inp.wk))
    t.update(Hk=torch.empty((nspin, nk, n, n), dtype=C128), Sk=torch.empty((1, nk, n, n), dtype=C128),
             eps=torch.empty((nprob, n), dtype=F64), C=torch.empty((nprob, n, n), dtype=C128),
             m=torch.empty(nprob, dtype=I32), st=torch.empty(nprob, dtype=I32),
             smap=torch.arange(nprob, dtype=I32) % nk,
             dens=(torch.empty(1, dtype=F64), torch.empty(1, dtype=F64), torch.empty((nprob, n), dtype=F64),
                   torch.empty((nspin, nR, n, n), dtype=F64), torch.empty(1, dtype=I32)))
    return inp, t


def test_band_step_shapes_pass():
    inp, t = _step_tensors()
    n, nprob = inp.n, inp.nprob
    check_bloch_sum_args(t["SR"], t["R"], t["k"], t["Sk"], CPU)
    check_bloch_sum_args(t["HR"], t["R"], t["k"], t["Hk"], CPU)
    check_bloch_sum_args(t["HR"], t["R"], t["k"], None, CPU)
    check_gen_eig_args(t["Hk"].view(nprob, n, n), t["Sk"][0], t["smap"], n, (t["eps"], t["C"], t["m"], t["st"]),
                       None, CPU)
    check_gen_eig_args(t["Hk"].view(nprob, n, n), t["Sk"][0], t["smap"], n, None, None, CPU)
    check_density_matrix_args(t["w"], t["k"], t["eps"], t["C"], t["m"], t["R"], inp.nspin, t["dens"], None, CPU)
    edm = torch.empty((inp.nspin, inp.nR, n, n), dtype=F64)
    check_density_matrix_args(t["w"], t["k"], t["eps"], t["C"], t["m"], t["R"], inp.nspin, None, edm, CPU)
    # eigenvectors of the lowest nb bands only
    nb = 7
    C_sub = torch.empty((nprob, n, nb), dtype=C128)
    check_gen_eig_args(t["Hk"].view(nprob, n, n), t["Sk"][0], t["smap"], nb, (t["eps"], C_sub, t["m"], t["st"]),
                       None, CPU)
    check_density_matrix_args(t["w"], t["k"], t["eps"], C_sub, t["m"], t["R"], inp.nspin, t["dens"], None, CPU)
    # eigenvalues only: no C in the outputs
    check_gen_eig_args(t["Hk"].view(nprob, n, n), t["Sk"][0], t["smap"], n, (t["eps"], None, t["m"], t["st"]),
                       None, CPU)
    # one S per problem, padded orders
    H = torch.zeros((3, 40, 40), dtype=C128)
    check_gen_eig_args(H, H.clone(), None, 40, None, torch.tensor([40, 33, 1], dtype=I32), CPU)


def test_gen_eig_rejects():
    inp, t = _step_tensors()
    n, nprob = inp.n, inp.nprob
    H, S, smap = t["Hk"].view(nprob, n, n), t["Sk"][0], t["smap"]
    out = (t["eps"], t["C"], t["m"], t["st"])
    bad = [
        dict(H=H.real.contiguous()),                               # real H
        dict(H=H[:, :, : n - 1].contiguous()),                     # not square
        dict(S=S[:, : n - 1, : n - 1].contiguous()),               # order differs from H
        dict(S=S.to(torch.complex64)),                             # single precision
        dict(smap=smap.long()),                                    # int64 map
        dict(smap=smap[:-1].contiguous()),                         # one entry short
        dict(smap=None),                                           # nS != nprob without a map
        dict(nb=0), dict(nb=n + 1),
        dict(out=(t["eps"][:, :-1].contiguous(), t["C"], t["m"], t["st"])),
        dict(out=(t["eps"], t["C"][:, :, :-1].contiguous(), t["m"], t["st"])),  # C narrower than nb
        dict(out=(t["eps"], t["C"], t["m"].long(), t["st"])),
        dict(out=(t["eps"], t["C"], t["m"], t["st"][:-1].contiguous())),
        dict(s_size=torch.ones(nprob, dtype=I32)),                 # s_size needs one entry per S
        dict(H=H.transpose(1, 2)),                                 # not contiguous
    ]
    for b in bad:
        a = dict(H=H, S=S, smap=smap, nb=n, out=out, s_size=None)
        a.update(b)
        with pytest.raises(ValueError):
            check_gen_eig_args(a["H"], a["S"], a["smap"], a["nb"], a["out"], a["s_size"], CPU)
    with pytest.raises(ValueError, match="must be on"):
        check_gen_eig_args(H.to("meta"), S, smap, n, None, None, CPU)


def test_bloch_and_density_reject():
    inp, t = _step_tensors()
    n, nprob = inp.n, inp.nprob
    for args in ((t["SR"][0], t["R"], t["k"], None),                      # 3-d M(R)
                 (t["SR"], t["R"].long(), t["k"], None),                  # int64 images
                 (t["SR"], t["R"][:-1].contiguous(), t["k"], None),       # one image short
                 (t["SR"], t["R"], t["k"][:, :2].contiguous(), None),     # 2-d k-points
                 (t["HR"], t["R"], t["k"], t["Sk"]),                      # output for one spin only
                 (t["SR"], t["R"], t["k"], t["Sk"].real.contiguous())):   # real output
        with pytest.raises(ValueError):
            check_bloch_sum_args(*args, CPU)
    base = dict(wk=t["w"], kpts=t["k"], eps=t["eps"], C=t["C"], m=t["m"], R=t["R"], nspin=inp.nspin,
                out=t["dens"], edm=None)
    mu, eb, f, rho, st = t["dens"]
    bad = [
        dict(nspin=1),                                             # nprob != nspin nk
        dict(wk=t["w"][:-1].contiguous()),
        dict(kpts=t["k"].float()),
        dict(eps=t["eps"][:-1].contiguous()),
        dict(m=t["m"].long()),
        dict(R=t["R"].double()),
        dict(C=None),
        dict(out=(mu, eb, f, rho[:, :-1].contiguous(), st)),       # rho short of one image
        dict(out=(mu, eb, f[:, :-1].contiguous(), rho, st)),
        dict(out=(mu, eb, f, rho, st.long())),
        dict(edm=torch.empty((inp.nspin, inp.nR, n, n - 1), dtype=F64)),
    ]
    for b in bad:
        a = dict(base)
        a.update(b)
        with pytest.raises(ValueError):
            check_density_matrix_args(a["wk"], a["kpts"], a["eps"], a["C"], a["m"], a["R"], a["nspin"], a["out"],
                                      a["edm"], CPU)
    assert nprob == inp.nspin * inp.nk


@pytest.mark.parametrize("tA,tB", [(0, 0), (1, 0), (0, 2), (2, 1)])
def test_zgemm_shapes(tA, tB):
    M, K, N = 5, 7, 3
    A = torch.zeros((2, K, M) if tA else (2, M, K), dtype=C128)
    B = torch.zeros((2, N, K) if tB else (2, K, N), dtype=C128)
    check_zgemm_args(A, B, None, tA, tB, CPU)
    check_zgemm_args(A, B, torch.zeros((2, M, N), dtype=C128), tA, tB, CPU)
    with pytest.raises(ValueError):   # inner extents differ
        Bbad = torch.zeros((2, N, K + 1) if tB else (2, K + 1, N), dtype=C128)
        check_zgemm_args(A, Bbad, None, tA, tB, CPU)
    with pytest.raises(ValueError):   # C of the wrong shape
        check_zgemm_args(A, B, torch.zeros((2, N, M), dtype=C128), tA, tB, CPU)
    with pytest.raises(ValueError):   # batch sizes differ
        check_zgemm_args(A, B[:1].contiguous(), None, tA, tB, CPU)


def test_serve_request_shapes():
    inp, t = _step_tensors()
    SR = t["SR"][0]
    META = torch.device("meta")
    # host tensors are accepted whatever the context's device
    check_serve_request_args(t["HR"], SR, t["R"], t["k"], t["w"], META)
    check_serve_request_args(t["HR"][:1].contiguous(), SR, t["R"], t["k"], t["w"], META)
    # device tensors must all be on the context's device
    on = {k: v.to("meta") for k, v in dict(HR=t["HR"], SR=SR, R=t["R"], k=t["k"], w=t["w"]).items()}
    check_serve_request_args(on["HR"], on["SR"], on["R"], on["k"], on["w"], META)
    for args in ((t["HR"], t["SR"], t["R"], t["k"], t["w"]),                    # S(R) with a spin axis
                 (t["HR"][0], SR, t["R"], t["k"], t["w"]),                      # H(R) without one
                 (t["HR"], SR, t["R"].long(), t["k"], t["w"]),
                 (t["HR"], SR, t["R"], t["k"], t["w"][:-1].contiguous()),       # one weight short
                 (t["HR"], SR.float(), t["R"], t["k"], t["w"]),
                 (t["HR"], on["SR"], t["R"], t["k"], t["w"])):                   # host and device mixed
        with pytest.raises(ValueError):
            check_serve_request_args(*args, META)
