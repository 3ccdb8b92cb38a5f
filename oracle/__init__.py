"""Plain FP64 CPU oracle for the sketching hot path (TEST INFRASTRUCTURE).

This package is the checker, not the product.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and its
``--impl reference`` arm) may import it.  The CUDA library under
``paper_2203_02798_gb300/`` never imports, links or calls anything here, and
nothing here imports the CUDA library: the two share no code.  The only
module both sides use is ``workloads/`` (seeded synthetic inputs, which holds
none of the method's arithmetic).

Every function is the plain definition (or the paper's algorithm, step by
step), evaluated in float64 on numpy arrays.  Section / algorithm / equation
numbers in the docstrings refer to Sobczyk & Gallopoulos, "pylspack: Parallel
algorithms and data structures for sketching, column subset selection,
regression and leverage scores" (arXiv 2203.02798).

Modules
-------
philox      Philox-4x32-10 (Salmon et al. SC'11), the counter-based generator
            every random draw of the method comes from.
countsketch CountSketch S (Def. 3): hash/sign spec, explicit S, S*A (Alg. 2).
gaussian    Gaussian G (Alg. 3 / csrcgs scaling 1/sqrt(m)), G*(S*A).
gram        A^T A (Alg. 5 / Alg. 7 semantics, csrrk).
rownorms    squared row norms of A*B (Alg. 8, csrsqn / rmsqn).
qr          Householder QR, sign-normalised R, R^-1, full-rank check.
leverage    sketched (Alg. 15 without Pi) and exact (Alg. 13) leverage scores.
lsq         sketch-and-precondition least squares (Alg. 12) with LSQR.
"""
from . import philox, countsketch, gaussian, gram, rownorms, qr, leverage, lsq  # noqa: F401
