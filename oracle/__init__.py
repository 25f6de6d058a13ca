"""ORACLE: plain, slow FP64 CPU reference for the fragment CCSD(T) hot path.

This package is test infrastructure. Only `tests/`, `__graft_entry__.smoke()`
and the CPU-baseline / reference legs of `bench.py` may import it; the
product library never does, and it shares no code, header or table with the
CUDA path. Every function cites the passage of Ye & Berkelbach, "Periodic
Local Coupled-Cluster Theory for Insulators and Metals" (arXiv 2407.11258) or
the published formulation it follows.

Modules
  ccsd      closed-shell CCSD (T1-transformed form), MP2, energies      -- Sec. II.B, Eq. 7, 12-13, 21
  triples   LNO-(T) intermediates and the projected (T) energy          -- Eq. 14-16, SI Sec. S1
  fragment  projection of an occupied-pair energy matrix onto LOs       -- Eq. 7-8, Eq. 12, Eq. 15
  mp2       full-system MP2 and the MP2 composite correction            -- Eq. 17, Eq. 12-13, Eq. 21
  lno       local active space: SVD split, MP2 / CBNO densities, LNOs   -- Sec. II.C-E, Eq. 18-26, Eq. 28
  fci       brute-force two-electron FCI (pin for CCSD)
  spinorb   spin-orbital CCSD and (T) (independent pin for the closed-shell forms)
"""
from . import ccsd, triples, fragment, fci, spinorb, mp2, lno  # noqa: F401
