"""Run one fragment solve through the C-ABI (for profiling with external tools such as ncu).

    python -m paper_2407_11258_gb300.profile_case --nocc 16 --nvir 120 --naux 480 --iters 4 [--mlp-guess]

Builds the integrals, runs `--iters` CCSD iterations (mixed precision unless --fp64), the fragment
energies and the (T) energy on a seeded synthetic fragment, and prints the timings the library reports.
"""
import argparse
import sys
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nocc", type=int, default=16)
    ap.add_argument("--nvir", type=int, default=120)
    ap.add_argument("--naux", type=int, default=480)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--no-triples", action="store_true")
    ap.add_argument("--mlp-guess", action="store_true", help="also run the learned-guess kernel once (initial weights)")
    a = ap.parse_args(argv)
    import torch

    from paper_2407_11258_gb300 import build, lnocc, synth
    build.build()
    fr = synth.make_fragment(a.nocc, a.nvir, a.naux, a.seed, decay=20.0, frag=(0, 1) if a.nocc > 1 else (0,))
    eps = torch.tensor(fr.eps, device="cuda")
    B = torch.tensor(fr.B, device="cuda")
    U = torch.tensor(fr.U_frag, device="cuda")
    prec = lnocc.LNOCC_PREC_FP64 if a.fp64 else lnocc.LNOCC_PREC_MIXED
    f = lnocc.lnocc_build_ints(fr.nocc, fr.nvir, fr.naux, eps, B, lnocc.default_opts(precision=prec, max_iter=a.iters))
    t0 = time.perf_counter()
    e, it, st = lnocc.lnocc_ccsd(f, allow_noconv=True)
    t1 = time.perf_counter()
    ec, em = lnocc.lnocc_fragment_energy(f, U)
    out = f"ccsd {it} iterations {1e3 * (t1 - t0):.1f} ms E={e:.12f} E_frag={ec:.12f}"
    if a.mlp_guess:
        m = lnocc.Mlp(synth.mlp_init())
        t2g = torch.empty(a.nocc, a.nocc, a.nvir, a.nvir, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        tg = time.perf_counter()
        lnocc.lnocc_mlp_guess(f, m, t2g)
        torch.cuda.synchronize()
        out += f"; learned guess {1e3 * (time.perf_counter() - tg):.2f} ms"
        m.free()
    if not a.no_triples:
        et, etf = lnocc.lnocc_triples(f, U)
        inf = f.info()
        out += (f"; (T) device {inf.t_triples_ms:.1f} ms (contractions {inf.t_triples_gemm_ms:.1f} ms)"
                f" E_T={et:.12f} E_T_frag={etf:.12f}")
    f.free()
    print(out, flush=True)


if __name__ == "__main__":
    sys.exit(main())
