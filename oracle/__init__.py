"""FP64 CPU oracle for the separated fast-spectral Boltzmann collision operator.

TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the benchmark's CPU
baseline leg are the only code allowed to import it.  It shares no code with
the CUDA library (`paper_2112_02695_gb300`), which must never import it.

Modules:
  quadrature  Gauss-Legendre by Newton, circle rule, octahedral sphere rules
              derived from their moment equations.
  collision   the separated algorithm step by step (plain separable DFTs),
              the brute-force direct sum, projection and moments.
  lowrank     the low-rank step pieces that consume the batch: K- and
              L-step collision terms, weighted QR, SVD rank truncation.
  mott_smith  the strong-shock closure alpha, beta of Sec. 4.2.
  carleman    the Carleman-form fast spectral operator for gamma = d - 2
              (the Mouhot-Pareschi algorithm the paper's experiments use).
  shock       the 1D normal shock end to end: full-tensor upwind scheme and
              the adaptive low-rank K-S-L scheme with its boundary treatment.
"""
from . import quadrature, collision, lowrank, mott_smith, carleman, shock  # noqa: F401
