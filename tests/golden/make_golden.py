"""Write the stored oracle energies under tests/golden/ (calls only `oracle/` and the input generator).

    python tests/golden/make_golden.py small        # nocc=4/nvir=24, (T) at nocc=12/nvir=96, batch subset
    python tests/golden/make_golden.py diamond      # nocc=16, nvir=240, naux=960, CCSD only (about 1.5 h)
    python tests/golden/make_golden.py half         # nocc=16, nvir=120, naux=480 with (T) (about 30 min)
    python tests/golden/make_golden.py half_li      # same sizes, lithium-like small-gap energies, with (T)

Each file records the generator call that rebuilds the inputs, the oracle's
energies (FP64) and its convergence data.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ccsd, fragment, triples  # noqa: E402
from paper_2407_11258_gb300 import synth  # noqa: E402


def solve(fr, with_t=True, log=None):
    t0 = time.time()
    r = ccsd.ccsd(fr.eps, fr.B, fr.nocc, tol_t=1e-10, tol_e=1e-12,
                  callback=(lambda it, e, d: log(f"  it {it:3d} E={e:.14f} dt={d:.2e} ({time.time()-t0:.0f}s)"))
                  if log else None)
    Ec = ccsd.pair_energy_matrix(r["t1"], r["t2"], fr.B, fr.nocc)
    t2mp2 = ccsd.mp2_amplitudes(fr.eps, fr.B, fr.nocc)
    Emp2 = ccsd.pair_energy_matrix(np.zeros_like(r["t1"]), t2mp2, fr.B, fr.nocc)
    out = dict(nocc=fr.nocc, nvir=fr.nvir, naux=fr.naux, seed=fr.seed, kind=fr.kind, frag=list(fr.frag),
               e_mp2=float(np.trace(Emp2)), e_ccsd=r["e_corr"], n_iter=r["n_iter"],
               converged=r["converged"],
               e_mp2_frag=fragment.project(Emp2, fr.U_frag),
               e_ccsd_frag=fragment.project(Ec, fr.U_frag),
               ccsd_seconds=time.time() - t0)
    if with_t:
        t1 = time.time()
        Et = triples.pair_matrix(r["t1"], r["t2"], fr.eps, fr.B, fr.nocc)
        out.update(e_t=float(np.trace(Et)), e_t_frag=fragment.project(Et, fr.U_frag),
                   t_seconds=time.time() - t1)
    return out


def main(tier):
    log = lambda s: print(s, flush=True)  # noqa: E731
    if tier == "small":
        res = {"single_fp64": dict(gen="synth.single_fp64()", **solve(synth.single_fp64()))}
        res["triples_scaled"] = dict(gen="synth.triples_large(scaled=True)",
                                     **solve(synth.triples_large(scaled=True)))
        shrink = lambda o, v: (max(2, o // 3), max(8, v // 10))  # noqa: E731
        bat = []
        for f in range(16):
            fr = synth.batch_fragment(f, scale_shape=shrink)
            bat.append(dict(gen=f"synth.batch_fragment({f}, scale_shape=shrink)", **solve(fr)))
        res["batch_shrunk"] = bat
        path = os.path.join(HERE, "oracle_small.json")
    elif tier == "diamond":
        fr = synth.diamond_like()
        res = {"diamond_like": dict(gen="synth.diamond_like()", **solve(fr, with_t="--no-t" not in sys.argv, log=log))}
        path = os.path.join(HERE, "oracle_diamond.json")
    elif tier == "half":
        # the diamond-like generator at half the virtual space: (T) at the production nocc against the oracle
        fr = synth.make_fragment(16, 120, 480, 2000, occ_range=(-1.2, -0.4), vir_range=(0.3, 4.0), decay=20.0,
                                 frag=(0, 1))
        gen = ("synth.make_fragment(16, 120, 480, 2000, occ_range=(-1.2, -0.4), vir_range=(0.3, 4.0), "
               "decay=20.0, frag=(0, 1))")
        res = {"half_diamond": dict(gen=gen, **solve(fr, log=log))}
        path = os.path.join(HERE, "oracle_half_diamond.json")
    elif tier == "half_li":
        # lithium-like (small-gap) energies at the half-diamond sizes: the regime where the mixed path's
        # residual noise floor and slow convergence could break the 1e-6 Eh budget (seed 2505: gap 0.040 Eh, the
        # smallest of the lithium-like range 2 * U[0.02, 0.1])
        fr = synth.make_fragment(16, 120, 480, 2505, decay=20.0, small_gap=True, frag=(0, 1))
        gen = "synth.make_fragment(16, 120, 480, 2505, decay=20.0, small_gap=True, frag=(0, 1))"
        res = {"half_lithium": dict(gen=gen, gap=float(fr.eps[16] - fr.eps[15]), **solve(fr, log=log))}
        path = os.path.join(HERE, "oracle_half_lithium.json")
    else:
        raise SystemExit(__doc__)
    res["_note"] = "written by tests/golden/make_golden.py from oracle/ only"
    with open(path, "w") as fh:
        json.dump(res, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "")
