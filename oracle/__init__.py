"""Plain FP64 CPU oracle for the screened Lasso solve (Dantas & Gribonval, arXiv 1812.06635).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import or run it.  It shares no code
with the CUDA library; the two meet only through the seeded inputs of ``synthetic``.

Modules:
  lasso         problem, dual, dual scalings, safe spheres and tests (Sections I-III, Table I)
  dictionaries  dense, sum-of-Kronecker and sparse-factor operators, BF16 / per-atom FP8
                quantisers, error bounds eps_j, relative complexity, step size (Sections III-A,
                IV-B, V-A, VI)
  solvers       FISTA / ISTA with (stable) GAP or Dynamic Safe screening over a ladder of
                approximate dictionaries (Algorithms 1-2), KKT polish, brute force
  backward      derivative of the solution w.r.t. y and A through the support system
  regions       l_p spheres and l_q error zones with C_{p,q} (Section III-B), Lemma 2 with l_q
                errors, and dome regions (a safe sphere cut by a dual constraint)

Pins: every function is checked by ``tests/test_oracle_*.py`` against closed forms, brute
force, the lemmas and theorem of Section III, or library routines.  Parity unpinned: the
iterate-level switching trajectory of Algorithm 2 (the paper prints no values for it; only
its invariants are pinned) and the easy/moderate/hard decay weights of the Kronecker
variants (Section V-A gives them only as a figure).
"""
