"""CPU FP64 oracle for the ChASE hot path of arXiv 2006.08498.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import, call, link or execute anything in this
package.  The product path (paper_2006_08498_gb300) never imports it and
shares no code with it: the synthetic generator, the random streams and every
step of the solver are written here independently of the CUDA kernels.

structured.py holds the exact eigenvalue count of the synthetic Hamiltonian
(Sylvester's inertia law on its block + low-rank structure), bisection for its
lowest eigenvalues at any size, and its product H V as an operator, so that
the plain oracle ChASE runs at the full benchmark sizes.

Parity pins (tests/test_oracle_*.py) tie each function to something other
than itself: closed forms, the paper's printed tables, brute force on tiny
inputs, and library routines used as test-time cross-checks.
"""
from ._lib import build  # noqa: F401
from . import structured  # noqa: F401
from .chase import (  # noqa: F401
    STREAM_EXCHANGE, STREAM_LANCZOS, STREAM_START, STREAM_THETA, STREAM_XI,
    bse_elements, bse_tables, build_h, chase, chebyshev_filter, cholesky, cholqr,
    convergence_rate, damping, default_model, degree_cap, degrees, eigh, filter_interval, group_degrees, grown_nex, count_point,
    lanczos_bounds, lock_count, nex_regression, normalize_phase, qr, random_block,
    rayleigh_ritz, residuals, splitmix64, tridiag_eig, uniform)
