"""FP64 CPU oracle for all-edge spanning centrality (TGT / TGT+).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or execute anything in this package. The CUDA library never imports it,
and this package imports nothing from the CUDA library: the two share no code.
The only inputs they share come from the seeded generators in ``graphgen``.

Modules:
  exact       exact SC = effective resistance (Kirchhoff enumeration, matrix-tree
              theorem, grounded-Laplacian Cholesky, sparse LU, CG)
  series      truncated series of Eq. (2) by Algorithm 2, half sums of Eq. (9),
              end-corrected estimator and a-posteriori tail bounds
  truncation  eigenvalue extremes and the truncation length of Eq. (5)-(6);
              CalTau (Algorithm 1) with omega eigenpairs, Eq. (7)-(8)
  philox      Philox4x32-10 counter-based generator (Salmon et al., SC'11)
  tgtplus     the TGT+ pieces: CalChi (Alg. 3), walk counts (Eq. 13), walk
              estimator (Eq. 11), switch rule (Eq. 14)
  learned     FP64 reference MLP (features, forward, backward, Adam) for the
              learned truncation length, its certified labels, and on bipartite
              graphs the power-law tail estimate and its extension loop
"""
from . import exact, learned, philox, series, tgtplus, truncation  # noqa: F401
