"""Run the band step once (or a few times) on a magnetite-shaped cell of chosen size.

A small driver for tracing and profiling one configuration through the public binding:

    python -m paper_1402_4247_gb300.run_case --kgrid 4 2 2 --nspin 2 --repeat 1 [--band-width 32]
    python -m paper_1402_4247_gb300.run_case --large-basis 1000 --kgrid 1 1 1 --nspin 1

prints the time per step and the per-stage times recorded by the library's CUDA-event tracing
(after --warmup untraced steps; when Parts 3-4 run as two halves (--split) the stages of the
two streams overlap, so their sum exceeds the step).  --band-width selects the two-stage Householder reduction and --mrrr-all the
relatively robust representations for the eigenvectors of both tridiagonals (nao_config);
--large-basis n takes the large-basis cell of order n (overlap condition ~1e8, one orbital
in 50 duplicated) instead of the magnetite-shaped one.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import synth
from .nao import Context


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kgrid", type=int, nargs=3, default=[4, 2, 2])
    ap.add_argument("--nspin", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--band-width", type=int, default=0, choices=[0, 16, 32])
    ap.add_argument("--large-basis", type=int, default=0, metavar="N")
    ap.add_argument("--mrrr-all", action="store_true",
                    help="eigenvectors of both tridiagonals from relatively robust representations")
    ap.add_argument("--split", type=int, default=0, choices=[0, 1, 2],
                    help="Parts 3-4 as two halves on two streams: 0 never, 1 always, 2 from 32 problems")
    args = ap.parse_args()
    if args.large_basis:
        inp = synth.scaled_cell(args.large_basis, seed=3, kgrid=tuple(args.kgrid), nspin=args.nspin,
                                ill_conditioned=True)
    else:
        inp = synth.magnetite_cell(seed=args.seed, kgrid=tuple(args.kgrid), nspin=args.nspin)
    dev = torch.device("cuda:0")
    ctx = Context(0, config={"band_width": args.band_width, "mrrr_all": int(args.mrrr_all),
                             "split_hprime": args.split})
    n, nk, nprob = inp.n, inp.nk, inp.nprob
    HR = torch.from_numpy(inp.HR).to(dev)
    SR = torch.from_numpy(inp.SR)[None].to(dev)
    R = torch.from_numpy(inp.R).to(dev)
    k = torch.from_numpy(inp.kpts).to(dev)
    w = torch.from_numpy(inp.wk).to(dev)
    smap = (torch.arange(nprob, dtype=torch.int32) % nk).to(dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for it in range(args.warmup + args.repeat):
        if it == args.warmup:
            torch.cuda.synchronize()
            ctx.nao_profile_enable(True)
            t0.record()
        Sk = ctx.nao_bloch_sum(SR, R, k)[0]
        Hk = ctx.nao_bloch_sum(HR, R, k).reshape(nprob, n, n)
        eps, C, m, st = ctx.nao_gen_eig(Hk, Sk, s_of_prob=smap)
        mu, eb, f, rho, rst = ctx.nao_density_matrix(w, k, eps, C, m, inp.n_electrons, inp.kT, R, inp.nspin)
    t1.record()
    torch.cuda.synchronize()
    prof = ctx.nao_profile_read()
    ok = int(st.abs().sum()) == 0 and int(rst[0]) == 0
    print(json.dumps({"n": n, "problems": nprob, "band_width": args.band_width, "status_ok": ok, "mu": float(mu[0]),
                      "ms_per_step": round(t0.elapsed_time(t1) / max(args.repeat, 1), 3),
                      "stages_ms": {k_: round(v[0] / args.repeat, 3) for k_, v in prof.items()}}))
    ctx.close()
    if not ok:
        raise SystemExit(1)


if __name__ == "__main__":
    main()
