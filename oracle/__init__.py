"""FP64 CPU oracle for compressed NMF / SNMF (Tepper & Sapiro).

TEST INFRASTRUCTURE.  A plain, slow, obviously correct restatement of what
the GPU path computes, used only by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py``.  The product path
(the CUDA library and its Python binding) never imports, links or calls
anything here, and nothing here imports the product package: the two share
only the seeded input generator in ``synth``.

Modules (each cites the passage it follows):
  philox    -- counter-based Gaussian test matrices (Alg. 1 first step)
  compress  -- structured random compression, one- and two-sided (Alg. 1,
               Sec. III definitions of L, R, A-check, A-tilde)
  admm      -- compressed ADMM NMF (Alg. 4) and plain ADMM (L = I, R = I)
  snmf      -- compressed SNMF column selection with SPA (Alg. 3)
  residual  -- relative reconstruction error, compressed objective, SVD floor

Parity unpinned: the speed of ADMM convergence for a given (lam, phi) -- the
paper gives no theory for it beyond Proposition 1 (limit points are KKT).
"""
from . import philox, compress, admm, snmf, residual  # noqa: F401
