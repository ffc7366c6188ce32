"""Shared helpers of the GPU parity tests: run the CUDA band step through the C ABI binding
and compare it with the oracle by the parity tolerances stated for the workload."""
import numpy as np

# Tolerances (floating point): eigenvalues |d eps| <= 1e-10 * ||H'|| with ||H'|| = max |eps|
# (the norm of X^H H X, the matrix whose eigenvalues are computed); residual
# ||H C - S C eps||_F / (n ||H||_2) <= 1e-12; ||C^H S C - I||_max <= 1e-11; rho elementwise
# <= 1e-10 max(1, max|rho|) (rho reaches ~1e3 here: |c_i| ~ s_min^{-1/2}); spectral projectors
# of eigenvalue clusters <= 1e-9 max(1, ||P||).
TOL_EPS = 1e-10
TOL_RES = 1e-12
TOL_ORTH = 1e-11
TOL_RHO = 1e-10
TOL_PROJ = 1e-9


def to_dev(inp, torch, dev):
    return dict(HR=torch.from_numpy(inp.HR).to(dev), SR=torch.from_numpy(inp.SR).to(dev)[None],
                R=torch.from_numpy(inp.R).to(dev), k=torch.from_numpy(inp.kpts).to(dev),
                w=torch.from_numpy(inp.wk).to(dev))


def gpu_band_step(ctx, inp, torch, dev, nb=None, s_cut=1e-10, density=True, precision=0):
    t = to_dev(inp, torch, dev)
    n = inp.n
    Hk = ctx.nao_bloch_sum(t["HR"], t["R"], t["k"]).reshape(-1, n, n)
    Sk = ctx.nao_bloch_sum(t["SR"], t["R"], t["k"])[0]
    smap = torch.arange(inp.nprob, dtype=torch.int32, device=dev) % inp.nk
    eps, C, m, st = ctx.nao_gen_eig(Hk, Sk, s_of_prob=smap, s_cut=s_cut, nb=nb, precision=precision)
    out = dict(Hk=Hk, Sk=Sk, eps=eps, C=C, m=m, status=st)
    if density:
        edm = torch.empty((inp.nspin, inp.nR, n, n), dtype=torch.float64, device=dev)
        mu, eb, f, rho, rst = ctx.nao_density_matrix(t["w"], t["k"], eps, C, m, inp.n_electrons, inp.kT, t["R"],
                                                     inp.nspin, edm=edm)
        out.update(mu=mu, eband=eb, f=f, rho=rho, edm=edm, rstatus=rst)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


def clusters(e, gap):
    groups, cur = [], [0]
    for j in range(1, len(e)):
        if e[j] - e[j - 1] >= gap:
            groups.append(cur)
            cur = []
        cur.append(j)
    groups.append(cur)
    return groups


def check_problem(H, S, eps_g, C_g, m_g, eps_o, C_o, m_o, label=""):
    """Compare one generalized eigenproblem's GPU result with the oracle's."""
    n = H.shape[0]
    assert m_g == m_o, f"{label}: m {m_g} vs {m_o}"
    m = m_o
    e = eps_g[:m]
    assert np.all(np.isinf(eps_g[m:])), label
    hn = max(np.abs(eps_o).max(), 1e-300)
    de = np.abs(e - eps_o).max()
    assert de <= TOL_EPS * hn, f"{label}: eigenvalues differ by {de:.3e} (bound {TOL_EPS * hn:.3e})"
    if C_g is None:
        return de
    nbv = C_g.shape[1]
    C = C_g[:, :min(m, nbv)]
    ee = e[:C.shape[1]]
    h2 = np.linalg.norm(H, 2)
    res = np.linalg.norm(H @ C - S @ C * ee[None, :]) / (n * h2)
    assert res <= TOL_RES, f"{label}: residual {res:.3e}"
    orth = np.abs(C.conj().T @ S @ C - np.eye(C.shape[1])).max()
    assert orth <= TOL_ORTH, f"{label}: C^H S C - I = {orth:.3e}"
    if m < nbv:
        assert np.all(C_g[:, m:] == 0), label
    # spectral projectors of clusters fully inside the returned columns
    for g in clusters(eps_o, 1e-8 * hn):
        if g[-1] >= C.shape[1]:
            continue
        Pg = C[:, g] @ C[:, g].conj().T
        Po = C_o[:, g] @ C_o[:, g].conj().T
        dp = np.abs(Pg - Po).max()
        assert dp <= TOL_PROJ * max(1.0, np.abs(Po).max()), f"{label}: projector of {g[:3]}.. differs {dp:.3e}"
    return de
