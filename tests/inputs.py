"""Seeded synthetic inputs shared by the oracle side and the CUDA side of
the parity tests.  Nothing here performs any step of the method: these are
random Hermitian matrices and blocks of the shapes the solver sees."""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def hermitian(n, seed, spread=(0.5, 12.0)):
    """Dense Hermitian n x n (Fortran order) with eigenvalues uniform in
    `spread`, built as U diag(lam) U^H from a seeded unitary U."""
    r = rng(seed)
    lam = np.sort(r.uniform(spread[0], spread[1], n))
    X = r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))
    U, _ = np.linalg.qr(X)
    A = (U * lam) @ U.conj().T
    A = (A + A.conj().T) / 2
    return np.asfortranarray(A), lam


def block(n, m, seed):
    """Seeded complex n x m block (Fortran order), entries N(0,1) + i N(0,1)."""
    r = rng(seed)
    return np.asfortranarray(r.standard_normal((n, m)) + 1j * r.standard_normal((n, m)))


def degrees(m, seed, lo=1, hi=36):
    """Ascending per-column degrees in [lo, hi]."""
    return np.sort(rng(seed).integers(lo, hi + 1, size=m)).astype(np.int32)


def orthonormal(n, k, seed):
    Q, _ = np.linalg.qr(block(n, k, seed))
    return np.asfortranarray(Q)
