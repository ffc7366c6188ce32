#!/usr/bin/env python3
"""Benchmark of the band step (Band_DFT_Col, Sec. 3 Parts 1-6) on the magnetite-shaped cell.

One step = Bloch sums of S and H (Part 1), 128 generalized eigensolves (2 spins x 64 k,
Parts 2-4), chemical potential, occupations and the density matrix (Parts 5-6), all through
the C ABI of libnao.so.  Inputs are seeded synthetic stand-ins for the paper's magnetite
system (n = 568 basis functions, 125 lattice images, 4x4x4 k-grid); they are generated on
the host, copied to the GPU once, and stay resident (total working set > 8 GB, far above the
L2 size, so no explicit L2 flush is needed).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "k-point generalized eigensolves/s (FP64, n=568)"
UNIT = "solves/s"
FP64_PEAK_TFLOPS = 4 * 152 * 2.070e9 / 1e12  # 2 FP64 FMA/clk/SM x 152 SMs at 2070 MHz


def _hbm_peak():
    """Measured copy bandwidth of the GB300s (GB/s) and where it came from."""
    try:
        v = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        return v, "of measured (MEASURED_PEAKS.json hbm_gbs: STREAM-style copy)"
    except Exception:
        return 6800.0, "of fallback (6.8 TB/s, one earlier GB300 measurement)"


# ------------------------------------------------------------------------------ helpers

def _workload_config(inp, extra=None):
    cfg = {
        "workload": "magnetite-shaped cell: n=568 (24 heavy x 13 + 32 light x 8 orbitals), 125 images, "
                    "4x4x4 k, 2 spins = 128 generalized eigensolves + mu + rho per step",
        "n": inp.n, "nk": inp.nk, "nspin": inp.nspin, "nR": inp.nR, "problems_per_step": inp.nprob,
        "n_electrons": inp.n_electrons, "kT_Ha": inp.kT, "precision": "fp64",
        "l2": "inputs larger than L2 (H(R)+S(R) 968 MB; working set > 8 GB), no flush needed",
    }
    if extra:
        cfg.update(extra)
    return cfg


def _oracle_worker(args):
    """One (spin, k) problem of the workload through the oracle (Parts 1-4), timed."""
    path_h, path_s, path_r, path_k, p, nk = args
    import numpy as np
    import oracle
    HR = np.load(path_h, mmap_mode="r")
    SR = np.load(path_s, mmap_mode="r")
    R = np.load(path_r)
    kp = np.load(path_k)
    sg, q = divmod(p, nk)
    t0 = time.perf_counter()
    Hk = oracle.bloch_sum(HR[sg], R, kp[q:q + 1])[0]
    Sk = oracle.bloch_sum(SR, R, kp[q:q + 1])[0]
    eps, C, m, _ = oracle.generalized_eigensolve(Hk, Sk)
    return time.perf_counter() - t0, int(m)


def _cpu_model():
    """The host CPU's model string (lscpu, else /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


class OracleSampler:
    """Spawned process pool (created before any GPU call) running the oracle one problem per
    core with single-threaded BLAS."""

    def __init__(self, inp, cores):
        self.tmp = tempfile.mkdtemp(prefix="nao_bench_")
        import numpy as np
        self.paths = []
        for name, arr in (("HR", inp.HR), ("SR", inp.SR), ("R", inp.R), ("k", inp.kpts)):
            pth = os.path.join(self.tmp, name + ".npy")
            np.save(pth, arr)
            self.paths.append(pth)
        self.nk = inp.nk
        self.nprob = inp.nprob
        self.cores = cores
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        self.pool = mp.get_context("spawn").Pool(cores)
        self.next = 0

    def run(self):
        probs = [(self.next + i) % self.nprob for i in range(self.cores)]
        self.next += self.cores
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(*self.paths, p, self.nk) for p in probs])
        wall = time.perf_counter() - t0
        return len(probs), wall, max(r[0] for r in res)

    def close(self):
        self.pool.close()
        self.pool.join()
        import shutil
        shutil.rmtree(self.tmp, ignore_errors=True)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _stage_flops(stage, inp, m_mean, nocc_mean):
    """Algorithmic FLOPs of one step for a traced stage (FP64, real-flop count)."""
    n, ns, npb, nR, nk = inp.n, inp.nk, inp.nprob, inp.nR, inp.nk
    m = m_mean
    if stage == "hetrd":       # panel kernel: the Hermitian matvec half of 16/3 n^3 (digit products)
        return ns * 8.0 / 3.0 * n ** 3 + npb * 8.0 / 3.0 * m ** 3
    if stage == "hetrd_update":  # rank-2NB updates: the other half, tensor cores
        return ns * 8.0 / 3.0 * n ** 3 + npb * 8.0 / 3.0 * m ** 3
    if stage == "backtransform":  # Q Z with Q from n-1 complex reflectors: 8 n^2 per column
        return ns * 8.0 * n * n * m + npb * 8.0 * m ** 3
    if stage == "ortho_ns":    # Z (3I - Z^T Z)/2: two real n^3 GEMMs
        return ns * 4.0 * n ** 3 + npb * 4.0 * m ** 3
    if stage == "zgemm_HX":
        return npb * 8.0 * n * n * m
    if stage == "zgemm_XHY":   # lower triangle of X^H (H X)
        return npb * 4.0 * n * m * m
    if stage == "zgemm_XV":
        return npb * 8.0 * n * m * m
    if stage == "zgemm_P":     # Hermitian C f C^H over occupied bands
        return npb * 4.0 * n * n * nocc_mean
    if stage == "bloch_sum":   # (1 + nspin) matrices, lower triangle, complex phase x real
        return (1 + inp.nspin) * nk * nR * 4.0 * n * (n + 1) / 2
    if stage == "rho_phase":
        return inp.nspin * nk * nR * 4.0 * n * n
    return None


def _sum_sq(k):
    """sum_{L=1}^{k-1} L^2: the trailing orders of the columns of a reduction of order k."""
    k = float(k)
    return (k - 1.0) * k * (2.0 * k - 1.0) / 6.0


def _panel_bytes(inp, m_mean):
    """Algorithmic DRAM bytes of the Householder reductions of one step: every column's
    Hermitian matrix-vector product reads the trailing matrix once in half storage (the
    lower triangle, FP64 complex: 16 B per entry, L^2 / 2 entries), i.e. 8 sum_L L^2 ~
    (8/3) n^3 bytes per reduction (nk overlap matrices of order n, nprob H' of order m)."""
    return 8.0 * (inp.nk * _sum_sq(inp.n) + inp.nprob * _sum_sq(m_mean))


def _digit_stream_bytes(inp, m_mean):
    """Bytes the digit form of the panel kernel streams by design: 8-bit digits of both
    triangles (8 digits x (re, im) = 16 B per entry, L^2 entries), 16 sum_L L^2 per matrix:
    twice the algorithmic bytes, the price of per-row digit scales."""
    return 16.0 * (inp.nk * _sum_sq(inp.n) + inp.nprob * _sum_sq(m_mean))


def _load_traffic(stage, units_per_launch):
    """DRAM bytes per launch of a stage's kernel: the per-unit figure of a committed ncu
    capture (a smaller case) times the units one launch processes, provided the kernel
    source has not changed since the capture."""
    import hashlib
    pth = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(pth):
        return None
    try:
        data = json.load(open(pth))
        ent = data.get(stage)
        if not ent:
            return None
        src = os.path.join(ROOT, "paper_1402_4247_gb300", "csrc", ent["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return ent["bytes_per_unit"] * units_per_launch if h == ent["source_sha256_16"] else None
    except Exception:
        return None


def run_serve_stated(local_rank, n_requests=12, seed=5, ncells=4):
    """The serving workload at its stated distribution, on a bounded sample: n log-uniform in
    [200, 4000] (four seeded cells of the same generator, n rounded to a multiple of 50, 27
    images so that a request's real-space inputs stay a few GB), 1-32 mirrored random
    k-points, 1 or 2 spins, FP64 or mixed; offline capacity first, then Poisson arrivals at
    0.7x that rate; latencies from submit to finished on the GPU."""
    return run_serve(local_rank, n_requests=n_requests, seed=seed, ncells=ncells, n_range=(200, 4000), nk_max=32,
                     stated=True)


def run_serve(local_rank, n_requests=48, seed=5, ncells=6, n_range=(128, 768), nk_max=8, stated=False):
    """Serving stream (a scaled-down form of the serving workload: fewer requests, n up to 768):
    cells with n log-uniform in [128, 768], 1-8 random k-points mirrored to +-k (Gamma added
    when odd), 1 or 2 spins, FP64 or mixed precision.  First the offline capacity (all
    requests queued at once), then Poisson arrivals at 0.7x that rate; latencies are the
    library's submit -> finished-on-GPU times."""
    import numpy as np
    import torch
    from paper_1402_4247_gb300 import synth
    from paper_1402_4247_gb300.nao import Context

    rng = np.random.default_rng(seed)
    cells = []
    for i in range(ncells):
        nt = float(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]))))
        if stated:
            cells.append(synth.scaled_cell(max(50, int(round(nt / 50.0)) * 50), seed=600 + i, kgrid=(1, 1, 1), nspin=2,
                                           ill_conditioned=False, image_radius=1))
        else:
            h, l = max(1, round(nt / 25)), max(1, round(3 * nt / 50))
            cells.append(synth.small_cell(500 + i, h, l, kgrid=(1, 1, 1), nspin=2))
    reqs = []
    for _ in range(n_requests):
        c = cells[int(rng.integers(len(cells)))]
        nk = int(rng.integers(1, nk_max + 1))
        half = rng.uniform(-0.5, 0.5, size=(nk // 2, 3))
        k = np.concatenate([half, -half] + ([np.zeros((1, 3))] if nk % 2 else []))
        nspin = int(rng.integers(1, 3))
        reqs.append(dict(HR=torch.from_numpy(np.ascontiguousarray(c.HR[:nspin])), SR=torch.from_numpy(c.SR),
                         R=torch.from_numpy(c.R), k=torch.from_numpy(k), w=torch.full((nk,), 1.0 / nk, dtype=torch.float64),
                         ne=c.n_electrons, kT=c.kT, prec=int(rng.integers(0, 2)) * 2, nprob=nspin * nk, n=c.n))
    ctx = Context(local_rank)

    def submit(q):
        return ctx.nao_serve_submit(q["HR"], q["SR"], q["R"], q["k"], q["w"], q["ne"], q["kT"], precision=q["prec"])

    # warm-up: one request of every cell (workspaces, allocator pool)
    for c in cells:
        q = dict(reqs[0], HR=torch.from_numpy(c.HR[:1].copy()), SR=torch.from_numpy(c.SR), R=torch.from_numpy(c.R),
                 ne=c.n_electrons, kT=c.kT)
        t = submit(q)
        ctx.nao_serve_poll(t, -1)
        ctx.nao_serve_release(t)
    ok = True
    # offline capacity
    ctx.nao_serve_pause(True)
    tickets = [submit(q) for q in reqs]
    t0 = time.perf_counter()
    ctx.nao_serve_pause(False)
    batch = []
    for t in tickets:
        r = ctx.nao_serve_poll(t, -1)
        ok = ok and r.status == 0
        batch.append(r.batch_requests)
        ctx.nao_serve_release(t)
    t_off = time.perf_counter() - t0
    cap = n_requests / t_off
    # online: Poisson arrivals at 0.7x capacity
    rate = 0.7 * cap
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    tickets = []
    t0 = time.perf_counter()
    due = t0
    for q, g in zip(reqs, gaps):
        due += g
        while time.perf_counter() < due:
            time.sleep(min(1e-3, max(0.0, due - time.perf_counter())))
        tickets.append(submit(q))
    lat = []
    for t in tickets:
        r = ctx.nao_serve_poll(t, -1)
        ok = ok and r.status == 0
        lat.append(r.latency_ms)
        ctx.nao_serve_release(t)
    _, peak, _, _ = ctx.nao_serve_stats()
    ctx.close()
    return {"workload": f"{n_requests} requests: n log-uniform in [{n_range[0]}, {n_range[1]}] over {ncells} cells (n = "
                        + ", ".join(str(c.n) for c in cells) + f", {cells[0].nR} images), 1-{nk_max} mirrored random "
                        "k-points, 1-2 spins, FP64 or mixed 50/50, Parts 1-6 each; 2 slots, batches up to 256 problems",
            "requests": n_requests, "capacity_req_per_s": cap,
            "solves_per_s_offline": sum(q["nprob"] for q in reqs) / t_off,
            "rate_req_per_s": rate, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_batch_requests_offline": float(np.mean(batch)), "peak_hbm_bytes": peak, "status_ok": ok}


def _band_step_timed(ctx, inp, dev, steps, warmup, precision=0, density=True):
    """Run the band step (Parts 1-6; Parts 1-4 when density is False) of one cell through the
    public binding: ``warmup`` untimed steps, then ``steps`` steps timed by CUDA events on the
    launching stream with the library's per-stage trace.  Returns (ms per step, stages,
    outputs of the last step)."""
    import torch
    n, nk, nprob = inp.n, inp.nk, inp.nprob
    d = {"HR": torch.from_numpy(inp.HR).to(dev), "SR": torch.from_numpy(inp.SR)[None].to(dev),
         "R": torch.from_numpy(inp.R).to(dev), "k": torch.from_numpy(inp.kpts).to(dev),
         "w": torch.from_numpy(inp.wk).to(dev)}
    Hk = torch.empty((inp.nspin, nk, n, n), dtype=torch.complex128, device=dev)
    Sk = torch.empty((1, nk, n, n), dtype=torch.complex128, device=dev)
    eps = torch.empty((nprob, n), dtype=torch.float64, device=dev)
    C = torch.empty((nprob, n, n), dtype=torch.complex128, device=dev)
    m = torch.empty(nprob, dtype=torch.int32, device=dev)
    st = torch.empty(nprob, dtype=torch.int32, device=dev)
    smap = (torch.arange(nprob, dtype=torch.int32) % nk).to(dev)
    dens = None
    if density:
        dens = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty(1, dtype=torch.float64, device=dev),
                torch.empty((nprob, n), dtype=torch.float64, device=dev),
                torch.empty((inp.nspin, inp.nR, n, n), dtype=torch.float64, device=dev),
                torch.empty(1, dtype=torch.int32, device=dev))
    stream = torch.cuda.current_stream(dev)

    def step():
        ctx.nao_bloch_sum(d["SR"], d["R"], d["k"], out=Sk)
        ctx.nao_bloch_sum(d["HR"], d["R"], d["k"], out=Hk)
        ctx.nao_gen_eig(Hk.view(nprob, n, n), Sk[0], s_of_prob=smap, precision=precision, out=(eps, C, m, st))
        if density:
            ctx.nao_density_matrix(d["w"], d["k"], eps, C, m, inp.n_electrons, inp.kT, d["R"], inp.nspin, out=dens)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ctx.nao_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.nao_profile_read()
    ctx.nao_profile_enable(False)
    ms = e0.elapsed_time(e1) / steps
    stages = {k_: round(v[0] / steps, 3) for k_, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    ok = int(st.abs().sum()) == 0 and (not density or int(dens[4][0]) == 0)
    return ms, stages, {"eps": eps, "C": C, "m": m, "status_ok": ok, "Hk": Hk, "Sk": Sk}


def _oracle_golden(path):
    """{problem: (m, eps)} from a golden file written by a committed oracle-only script."""
    import numpy as np
    out = {}
    if not os.path.exists(path):
        return out
    rows = np.loadtxt(path, comments="#")
    for p in np.unique(rows[:, 0]).astype(int):
        r = rows[rows[:, 0] == p]
        out[int(p)] = (int(r[0, 1]), r[np.argsort(r[:, 2]), 3])
    return out


def run_mixed_n2000(local_rank, steps=2, warmup=1):
    """The mixed-precision workload: n = 2000, 4x4x4 k, one spin (64 problems + mu + rho), seed 4.
    The FP64 step and the mixed step (NAO_MIXED_BF16X3 + one Ritz sweep) are timed alike; the
    eigenvalues of two fixed problems are compared with the oracle's (a golden file written by
    tests/golden/make_mixed_n2000_oracle.py), for the mixed path before and after its
    refinement sweep, with residual and S-orthonormality on the host."""
    import numpy as np
    import torch
    from paper_1402_4247_gb300 import synth
    from paper_1402_4247_gb300.nao import Context
    dev = torch.device("cuda", local_rank)
    inp = synth.scaled_cell(2000, seed=4, kgrid=(4, 4, 4), nspin=1, ill_conditioned=False)
    gold = _oracle_golden(os.path.join(ROOT, "tests", "golden", "mixed_n2000_oracle_eps.txt"))
    ctx = Context(local_rank)
    res = {"workload": "n=2000 (80 heavy x 13 + 120 light x 8 orbitals), 125 images, 4x4x4 k, 1 spin, seed 4: "
                       "64 generalized eigensolves + mu + rho per step", "n": inp.n, "problems_per_step": inp.nprob}
    checks = {}

    def errors(out, label):
        eps, C, m = out["eps"].cpu().numpy(), out["C"], out["m"].cpu().numpy()
        for p, (mo, eo) in gold.items():
            e = checks.setdefault(p, {})
            e[f"{label}_m_equal"] = bool(int(m[p]) == mo)
            e[f"{label}_max_abs_deps_Ha"] = float(np.abs(eps[p][:mo] - eo).max()) if int(m[p]) == mo else None
            H = out["Hk"].view(-1, inp.n, inp.n)[p].cpu().numpy()
            S = out["Sk"][0, p].cpu().numpy()
            Cp = C[p, :, :mo].cpu().numpy()
            ep = eps[p][:mo]
            v = np.random.default_rng(0).standard_normal(inp.n) + 0j  # ||H||_2 by power iteration
            for _ in range(60):
                w_ = H @ v
                hn = np.linalg.norm(w_) / np.linalg.norm(v)
                v = w_ / np.linalg.norm(w_)
            e[f"{label}_residual"] = float(np.linalg.norm(H @ Cp - (S @ Cp) * ep[None, :]) / (inp.n * hn))
            e[f"{label}_orth"] = float(np.abs(Cp.conj().T @ S @ Cp - np.eye(mo)).max())

    ms64, st64, out = _band_step_timed(ctx, inp, dev, steps, warmup, precision=0)
    res["fp64"] = {"value": inp.nprob / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64, "stages_ms": st64,
                   "status_ok": out["status_ok"]}
    errors(out, "fp64")
    del out
    ctx.nao_set_refinement(-1)
    msr, _, out = _band_step_timed(ctx, inp, dev, 1, 0, precision=2)
    errors(out, "mixed_raw")
    del out
    ctx.nao_set_refinement(1)
    ms1, st1, out = _band_step_timed(ctx, inp, dev, 1, 0, precision=2)
    res["mixed_one_sweep"] = {"value": inp.nprob / (ms1 * 1e-3), "unit": UNIT, "ms_per_step": ms1,
                              "precision": "NAO_MIXED_BF16X3 + one Ritz sweep + Rayleigh quotients"}
    errors(out, "mixed_sweep")
    del out
    ctx.nao_set_refinement(0)
    msm, stm, out = _band_step_timed(ctx, inp, dev, steps, warmup, precision=2)
    res["mixed"] = {"value": inp.nprob / (msm * 1e-3), "unit": UNIT, "ms_per_step": msm, "stages_ms": stm,
                    "precision": "NAO_MIXED_BF16X3 (36-bit products, 46-bit H' Householder digits) + Rayleigh "
                                 "quotients with FP64-accurate S C and H C (the default refinement)",
                    "status_ok": out["status_ok"]}
    errors(out, "mixed_refined")
    del out
    ctx.close()
    torch.cuda.empty_cache()
    res["mixed_over_fp64_speed"] = res["mixed"]["value"] / res["fp64"]["value"]
    res["vs_oracle"] = {"problems": sorted(gold), "per_problem": checks,
                        "source": "tests/golden/mixed_n2000_oracle_eps.txt (oracle/ only)"}
    worst = [c.get("mixed_refined_max_abs_deps_Ha") for c in checks.values()]
    res["mixed_bound_Ha"] = 1e-9
    res["mixed_meets_bound"] = bool(worst and all(w is not None and w <= 1e-9 for w in worst))
    return res


def run_large_basis(local_rank, sizes=(1000, 2000, 3000), steps=1, warmup=0, two_stage_sizes=(1000,)):
    """The large-basis FP64 sweep: n in {1000, 2000, 3000}, 4x4x1 k, one spin, seed 3, overlap
    condition ~1e8 plus one orbital in 50 duplicated (exact null directions; m = n - n/50).
    Per size: solves/s of the band step (Parts 1-6) and its per-stage split; the Householder
    panel kernel's achieved HBM rate by its algorithmic bytes; at two_stage_sizes, the same
    step with the two-stage reduction."""
    import torch
    from paper_1402_4247_gb300 import synth
    from paper_1402_4247_gb300.nao import Context
    dev = torch.device("cuda", local_rank)
    hbm, _ = _hbm_peak()
    rows = []
    for n in sizes:
        inp = synth.scaled_cell(n, seed=3, kgrid=(4, 4, 1), nspin=1, ill_conditioned=True)
        ctx = Context(local_rank)
        ms, stages, out = _band_step_timed(ctx, inp, dev, steps, warmup)
        m_mean = float(out["m"].double().mean())
        ctx.close()
        del out
        torch.cuda.empty_cache()
        row = {"n": n, "problems_per_step": inp.nprob, "value": inp.nprob / (ms * 1e-3), "unit": UNIT,
               "ms_per_step": ms, "m_mean": m_mean, "stages_ms": stages}
        if "hetrd" in stages:
            row["panel_hbm_frac"] = _panel_bytes(inp, m_mean) / (stages["hetrd"] * 1e-3) / 1e9 / hbm
        if n in two_stage_sizes:  # the same step with the two-stage reduction (band width 32)
            ctx = Context(local_rank, config={"band_width": 32})
            ms2, stages2, out = _band_step_timed(ctx, inp, dev, steps, warmup)
            ctx.close()
            del out
            torch.cuda.empty_cache()
            row["two_stage_b32"] = {"value": inp.nprob / (ms2 * 1e-3), "unit": UNIT, "ms_per_step": ms2,
                                    "stages_ms": stages2}
        rows.append(row)
    return {"workload": "large-basis cells (n/25 heavy x 13 + 3n/50 light x 8 orbitals), 125 images, 4x4x1 k, "
                        "1 spin, eta ~ 1e-8 and one orbital in 50 duplicated (kappa(S) ~ 1e8, exact null "
                        "directions), seed 3", "sizes": rows}


# ------------------------------------------------------------------------------ arms

def run_reference(args, rank, world):
    """CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from paper_1402_4247_gb300 import synth
    inp = synth.magnetite_cell()
    cores = min(os.cpu_count() or 1, args.cpu_cores)
    sampler = OracleSampler(inp, cores)
    for _ in range(args.warmup):
        sampler.run()
    tot, wall = 0, 0.0
    for _ in range(args.steps):
        c, w, _ = sampler.run()
        tot += c
        wall += w
    sampler.close()
    value = tot / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _workload_config(inp, {"sample": f"{cores} problems (one per core) per step, Parts 1-4"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "nproc": os.cpu_count(), "cpu_model": _cpu_model(),
                         "sample": f"{cores} of 128 (spin, k) problems per step through Parts 1-4 "
                                   f"(Bloch sum for one k + generalized eigensolve), one per process, "
                                   f"single-threaded BLAS"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    from paper_1402_4247_gb300 import synth

    inp = synth.magnetite_cell()

    import torch
    from paper_1402_4247_gb300.nao import Context

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ctx = Context(local_rank)
    n, nk, nspin, nprob, nR = inp.n, inp.nk, inp.nspin, inp.nprob, inp.nR

    # pinned host inputs (for the end-to-end arm) and resident device copies
    h_in = {"HR": torch.from_numpy(inp.HR).pin_memory(), "SR": torch.from_numpy(inp.SR)[None].pin_memory(),
            "R": torch.from_numpy(inp.R).pin_memory(), "k": torch.from_numpy(inp.kpts).pin_memory(),
            "w": torch.from_numpy(inp.wk).pin_memory()}
    d_in = {k_: v.to(dev) for k_, v in h_in.items()}
    Hk = torch.empty((nspin, nk, n, n), dtype=torch.complex128, device=dev)
    Sk = torch.empty((1, nk, n, n), dtype=torch.complex128, device=dev)
    eps = torch.empty((nprob, n), dtype=torch.float64, device=dev)
    C = torch.empty((nprob, n, n), dtype=torch.complex128, device=dev)
    m = torch.empty(nprob, dtype=torch.int32, device=dev)
    st = torch.empty(nprob, dtype=torch.int32, device=dev)
    mu = torch.empty(1, dtype=torch.float64, device=dev)
    eb = torch.empty(1, dtype=torch.float64, device=dev)
    f = torch.empty((nprob, n), dtype=torch.float64, device=dev)
    rho = torch.empty((nspin, nR, n, n), dtype=torch.float64, device=dev)
    rst = torch.empty(1, dtype=torch.int32, device=dev)
    smap = (torch.arange(nprob, dtype=torch.int32) % nk).to(dev)
    stream = torch.cuda.current_stream(dev)

    def step(src, precision=0, eps_out=eps, before_eig=None, before_density=None, c=None):
        c = c or ctx
        c.nao_bloch_sum(src["SR"], src["R"], src["k"], out=Sk)
        c.nao_bloch_sum(src["HR"], src["R"], src["k"], out=Hk)
        if before_eig:
            before_eig()
        c.nao_gen_eig(Hk.view(nprob, n, n), Sk[0], s_of_prob=smap, precision=precision, out=(eps_out, C, m, st))
        if before_density:
            before_density()
        c.nao_density_matrix(src["w"], src["k"], eps_out, C, m, inp.n_electrons, inp.kT, src["R"], nspin,
                             out=(mu, eb, f, rho, rst))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(d_in)
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0 and int(rst[0]) == 0, "band step reported a failure status"

    clocks = ClockSampler(local_rank)
    barrier()
    ctx.nao_profile_enable(True)
    l0 = ctx.nao_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(d_in)
    e1.record(stream)
    barrier()
    ms_total = e0.elapsed_time(e1)
    launches = ctx.nao_launch_count() - l0
    prof = ctx.nao_profile_read()
    ctx.nao_profile_enable(False)
    clk = clocks.stop()

    # end to end through the public API: pinned host inputs -> device, step, results -> host
    out_h = {"eps": torch.empty_like(eps, device="cpu").pin_memory(), "m": torch.empty_like(m, device="cpu").pin_memory(),
             "mu": torch.empty_like(mu, device="cpu").pin_memory(), "eb": torch.empty_like(eb, device="cpu").pin_memory(),
             "rho": torch.empty_like(rho, device="cpu").pin_memory()}
    h2d = sum(v.numel() * v.element_size() for v in h_in.values())
    d2h = sum(v.numel() * v.element_size() for v in out_h.values())
    # Pipelined: a copy stream brings step i+1's inputs into the other of two device input
    # slots while step i computes, and copies step i's results out while step i+1 runs (its
    # eigensolve waits for the small results' copy, its density matrix for rho's).  Every
    # step still copies its own inputs in and reads its own results back, inside the timed
    # region, which ends when the last step's results are on the host.
    d_e2e = [{k_: torch.empty_like(v) for k_, v in d_in.items()} for _ in range(2)]
    k_e2e = max(1, args.steps)  # as many steps as the device-resident arm: the first copy in and
                                # the last copy out are the only ones not overlapped
    cs = torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_used = [torch.cuda.Event() for _ in range(2)]
    ev_small, ev_rho = torch.cuda.Event(), torch.cuda.Event()

    def copy_in(slot):
        with torch.cuda.stream(cs):
            for k_, v in h_in.items():
                d_e2e[slot][k_].copy_(v, non_blocking=True)
            ev_in[slot].record(cs)

    def copy_out():
        ev_done = torch.cuda.Event()
        ev_done.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_done)
            for k_, v in (("eps", eps), ("m", m), ("mu", mu), ("eb", eb)):
                out_h[k_].copy_(v, non_blocking=True)
            ev_small.record(cs)
            out_h["rho"].copy_(rho, non_blocking=True)
            ev_rho.record(cs)

    barrier()
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record(stream)
    cs.wait_event(x0)
    copy_in(0)
    for i in range(k_e2e):
        sl = i % 2
        if i + 1 < k_e2e:
            if i >= 1:
                cs.wait_event(ev_used[1 - sl])  # step i-1 is done with that slot
            copy_in(1 - sl)
        stream.wait_event(ev_in[sl])
        step(d_e2e[sl], before_eig=(lambda: stream.wait_event(ev_small)) if i else None,
             before_density=(lambda: stream.wait_event(ev_rho)) if i else None)
        ev_used[sl].record(stream)
        copy_out()
        if i:
            ev_prev.synchronize()  # step i-1's results are on the host (step i is queued already)
            _ = float(out_h["mu"][0])
        ev_prev = torch.cuda.Event()
        ev_prev.record(cs)
    stream.wait_event(ev_rho)
    x1.record(stream)
    x1.synchronize()
    _ = float(out_h["mu"][0])
    barrier()
    e2e_ms = x0.elapsed_time(x1) / k_e2e

    # the mixed-precision form of the same step: reduced-precision products where the mixed mode allows
    # them, then the default refinement (NAO_MIXED_BF16X3); its eigenvalues are compared
    # with the FP64 step's
    eps_mx = torch.empty_like(eps)
    step(d_in, 2, eps_mx)
    barrier()
    y0, y1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    y0.record(stream)
    for _ in range(args.steps):
        step(d_in, 2, eps_mx)
    y1.record(stream)
    barrier()
    mixed_ms = y0.elapsed_time(y1) / args.steps
    fin = torch.isfinite(eps)
    mixed = {"value": nprob * world / (mixed_ms * 1e-3), "unit": UNIT, "ms_per_step": mixed_ms,
             "precision": "NAO_MIXED_BF16X3: six BF16 digit planes (36 bits) for the back-transformations, "
                          "X^H H X, the H' rank-2k updates and X V, 46-bit digits for the H' Householder "
                          "matrix-vector products; Rayleigh quotients with FP64-accurate S C and H C",
             "max_abs_deps_vs_fp64_Ha": float((eps_mx - eps)[fin].abs().max()),
             "status_ok": bool(int(st.abs().sum()) == 0 and int(rst[0]) == 0)}

    # the paper's two-pass form: eigenvectors only for the bands the density matrix uses
    # (the most occupied bands of any problem on the FP64 step, plus a margin of 8)
    nb_sub = min(n, int((f > 1e-16).sum(1).max()) + 8)
    C_sub = torch.empty((nprob, n, nb_sub), dtype=torch.complex128, device=dev)
    eps_sub = torch.empty_like(eps)

    def step_sub(src):
        ctx.nao_bloch_sum(src["SR"], src["R"], src["k"], out=Sk)
        ctx.nao_bloch_sum(src["HR"], src["R"], src["k"], out=Hk)
        ctx.nao_gen_eig(Hk.view(nprob, n, n), Sk[0], s_of_prob=smap, nb=nb_sub, out=(eps_sub, C_sub, m, st))
        ctx.nao_density_matrix(src["w"], src["k"], eps_sub, C_sub, m, inp.n_electrons, inp.kT, src["R"], nspin,
                               out=(mu, eb, f, rho, rst))

    step_sub(d_in)
    barrier()
    z0, z1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    z0.record(stream)
    for _ in range(args.steps):
        step_sub(d_in)
    z1.record(stream)
    barrier()
    sub_ms = z0.elapsed_time(z1) / args.steps
    subset = {"value": nprob * world / (sub_ms * 1e-3), "unit": UNIT, "ms_per_step": sub_ms, "nb": nb_sub,
              "note": "eigenvectors of H' only for the lowest nb bands (most occupied bands of any problem + 8), "
                      "eigenvalues all; the density-matrix status confirms no occupied band lies beyond nb",
              "status_ok": bool(int(st.abs().sum()) == 0 and int(rst[0]) == 0)}

    def alternative(config):
        """The same FP64 step on a context with other nao_config settings: timed steps, stage
        split and eigenvalue distance from the default step's."""
        c2 = Context(local_rank, config=config)
        eps_alt = torch.empty_like(eps)
        step(d_in, 0, eps_alt, c=c2)
        barrier()
        c2.nao_profile_enable(True)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(d_in, 0, eps_alt, c=c2)
        t1.record(stream)
        barrier()
        alt_ms = t0.elapsed_time(t1) / args.steps
        aprof = c2.nao_profile_read()
        c2.close()
        return {"value": nprob * world / (alt_ms * 1e-3), "unit": UNIT, "ms_per_step": alt_ms,
                "over_default_speed": ms_total / args.steps / alt_ms,
                "stages_ms": {k_: round(v[0] / args.steps, 3) for k_, v in sorted(aprof.items(), key=lambda kv: -kv[1][0])},
                "max_abs_deps_vs_default_Ha": float((eps_alt - eps)[fin].abs().max()),
                "status_ok": bool(int(st.abs().sum()) == 0 and int(rst[0]) == 0)}

    # the two-stage Householder reduction (dense -> band -> tridiagonal, then the second
    # back-transformation) at both band widths; eigenvectors of both tridiagonals from
    # relatively robust representations (dstegr's method) wherever the relative gap allows
    two_stage = {f"band_width_{bw}": alternative({"band_width": bw}) for bw in (32, 16)}
    mrrr_vectors = alternative({"mrrr_all": 1})
    # Parts 3-4 as two staggered halves of the problems on two streams
    split_hprime = alternative({"split_hprime": 2})

    serve = run_serve(local_rank) if (world == 1 and not args.no_serve) else None
    serve_stated = run_serve_stated(local_rank) if (world == 1 and not args.no_serve and not args.quick) else None
    mixed_n2000 = run_mixed_n2000(local_rank) if (world == 1 and not args.quick) else None
    large_basis = run_large_basis(local_rank) if (world == 1 and not args.quick) else None

    t_max = ms_total
    e2e_max = e2e_ms
    if dist is not None:
        tt = torch.tensor([ms_total, e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max, e2e_max = float(tt[0]), float(tt[1])

    cpu = None
    sampler = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's process pool starts only now (spawn, so it is safe after the CUDA
        # calls), so that it cannot overlap any GPU measurement
        sampler = OracleSampler(inp, min(os.cpu_count() or 1, args.cpu_cores))
    if sampler is not None:
        cnt, wall, _ = sampler.run()
        sampler.close()
        cpu = {"value": cnt / wall, "unit": UNIT, "cores": sampler.cores, "kind": "oracle",
               "nproc": os.cpu_count(), "cpu_model": _cpu_model(),
               "sample": f"{cnt} of 128 (spin, k) problems through Parts 1-4 (Bloch sum for one k + "
                         f"generalized eigensolve), one per process on each of {sampler.cores} host cores, "
                         f"single-threaded BLAS, {wall:.1f} s wall"}

    if rank == 0:
        m_mean = float(m.double().mean())
        nocc_mean = float((f > 1e-16).sum(1).double().mean())
        stages = {}
        for name, (tms, calls, nl) in prof.items():
            fl = _stage_flops(name, inp, m_mean, nocc_mean)
            stages[name] = {"ms_per_step": tms / args.steps, "launches_per_step": nl / args.steps,
                            "share": tms / max(sum(v[0] for v in prof.values()), 1e-9)}
            if fl is not None:
                stages[name]["gflop_per_step"] = fl / 1e9
        dom = max(prof.items(), key=lambda kv: kv[1][0])
        dname, (dms, dcalls, dl) = dom
        per_launch_ms = dms / max(dl, 1)
        if dname == "hetrd":
            # the Householder panel kernel against HBM: algorithmic bytes = the trailing
            # matrix in half storage once per column, (8/3) n^3 per reduction
            hbm, hsrc = _hbm_peak()
            byts = _panel_bytes(inp, m_mean) * args.steps / max(dl, 1)
            achieved = byts / (per_launch_ms * 1e-3) / 1e9
            roof = {"kernel": "hetrd_panel_kernel", "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": _load_traffic(dname, (inp.nk + inp.nprob) / (dl / args.steps)),
                    "peak_source": hsrc, "algorithmic_bytes_per_launch": byts,
                    "algorithmic_bytes": "8 sum_L L^2 ~ (8/3) n^3 per reduction: the trailing matrix in half "
                                         "storage (FP64 complex) once per column",
                    "digit_stream_bytes_per_launch": _digit_stream_bytes(inp, m_mean) * args.steps / max(dl, 1),
                    "ms_per_step": dms / args.steps}
        else:
            fl = _stage_flops(dname, inp, m_mean, nocc_mean)
            achieved = (fl * args.steps / max(dl, 1)) / (per_launch_ms * 1e-3) / 1e12 if fl else None
            roof = {"kernel": dname, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None, "traffic": None,
                    "peak_source": "FP64 FMA pipe: 2 FMA/clk/SM x 152 SMs x 2070 MHz (derived; 1.20 TFLOP/s "
                                   "measured by a DFMA microbenchmark)"}
        value = nprob * world * args.steps / (t_max * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _workload_config(inp, {"parallelism": "replicas" if world > 1 else "single GPU"}),
            "roofline": roof, "stages": stages,
            "e2e": {"value": nprob * world / (e2e_max * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu, "mixed": mixed, "subset": subset, "serve": serve,
            "mixed_n2000": mixed_n2000, "large_basis": large_basis, "serve_stated": serve_stated,
            "two_stage": two_stage, "mrrr_vectors": mrrr_vectors, "split_hprime": split_hprime,
            "status_ok": bool(int(st.abs().sum()) == 0 and int(rst[0]) == 0),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-stream measurement")
    ap.add_argument("--quick", action="store_true",
                    help="skip the n = 2000 mixed-precision and large-basis measurements")
    ap.add_argument("--cpu-cores", type=int, default=os.cpu_count() or 1,
                    help="host cores for the oracle (default: all of them)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
