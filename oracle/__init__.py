"""Plain FP64 CPU oracle for the deflated SAP-GCR Wilson-clover solver.

TEST INFRASTRUCTURE ONLY.  This package is a slow, obviously-correct
restatement of what the CUDA path computes, written from the paper
(Luescher, "Local coherence and deflation of the low quark modes in
lattice QCD").  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import it.  The
product path never calls it and it shares no code with ``csrc/``.

Modules
-------
lattice    geometry, parity, shifts, gamma matrices
dirac      clover field strength, Wilson-clover operator D, even-odd pieces
krylov     GCR (restarted, optionally flexible/preconditioned), MR
sap        block decomposition and the Schwarz alternating procedure
deflation  subspace generation (5.1), block projection (4.1)-(4.2),
           little Dirac operator (3.2)/(A.1), projectors (3.3)-(3.4)
little     even-odd little operator (A.2), global-mode deflation (A.3),
           little GCR (A.4)
solver     deflated, SAP-preconditioned flexible GCR (6.2) with adapted
           little-solve precision (A.5)

Parity status: every function is pinned by a test in ``tests/`` against a
closed form, an identity of the paper or a brute-force dense computation,
except where its docstring says "parity unpinned".
"""
