"""Pins of the oracle's dense Hermitian eigensolver and tridiagonal QR."""
import math

import numpy as np
import pytest

import oracle


def _rng(seed):
    return np.random.default_rng(seed)


def _random_unitary(n, seed, reflectors=16):
    """Product of seeded Householder reflectors I - 2 u u^H."""
    r = _rng(seed)
    Q = np.eye(n, dtype=np.complex128)
    for _ in range(reflectors):
        u = r.standard_normal(n) + 1j * r.standard_normal(n)
        u /= np.linalg.norm(u)
        Q = Q - 2.0 * np.outer(Q @ u, u.conj())
    return Q


def test_tridiagonal_toeplitz_closed_form():
    """tridiag(b, a, b) of order n has eigenvalues a + 2 b cos(k pi/(n+1))."""
    n, a, b = 40, 1.5, -0.7
    w, Z = oracle.tridiag_eig(np.full(n, a), np.full(n - 1, b))
    exact = np.sort([a + 2 * b * math.cos(k * math.pi / (n + 1)) for k in range(1, n + 1)])
    assert np.allclose(w, exact, rtol=0, atol=1e-14)
    T = np.diag(np.full(n, a)) + np.diag(np.full(n - 1, b), 1) + np.diag(np.full(n - 1, b), -1)
    assert np.linalg.norm(T @ Z - Z * w) < 1e-13
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) < 1e-13


def test_tridiagonal_wilkinson_matrix():
    """W21+ has pairs of eigenvalues agreeing to ~1e-14: a hard case for
    deflation; check against brute-force characteristic polynomial sign
    changes (Sturm count) at the computed values."""
    n = 21
    d = np.abs(np.arange(n) - 10).astype(float)
    e = np.ones(n - 1)
    w = oracle.tridiag_eig(d, e, vectors=False)

    def sturm(x):   # number of eigenvalues < x
        q, cnt = d[0] - x, int(d[0] - x < 0)
        for i in range(1, n):
            q = d[i] - x - e[i - 1] ** 2 / (q if q != 0 else 1e-300)
            cnt += q < 0
        return cnt
    for i, lam in enumerate(w):
        assert sturm(lam - 1e-9) <= i and sturm(lam + 1e-9) >= i + 1
    assert w[-1] == pytest.approx(10.746194182903393, abs=1e-12)


def test_two_by_two_closed_form():
    a, dd, b = 1.25, -0.5, 0.3 - 0.4j
    A = np.array([[a, np.conj(b)], [b, dd]])
    w, Z = oracle.eigh(A)
    r = math.sqrt(((a - dd) / 2) ** 2 + abs(b) ** 2)
    assert np.allclose(w, [(a + dd) / 2 - r, (a + dd) / 2 + r], rtol=0, atol=1e-15)
    assert np.linalg.norm(A @ Z - Z * w) < 1e-15


def test_four_by_four_brute_force():
    """det(A - lambda I) = 0 at every computed eigenvalue (4x4 by cofactor
    expansion) and the computed eigenvalues sum to the trace."""
    r = _rng(3)
    X = r.standard_normal((4, 4)) + 1j * r.standard_normal((4, 4))
    A = (X + X.conj().T) / 2

    def det(M):
        if M.shape[0] == 1:
            return M[0, 0]
        return sum((-1) ** j * M[0, j] * det(np.delete(M[1:], j, axis=1))
                   for j in range(M.shape[0]))
    w, Z = oracle.eigh(A)
    for lam in w:
        dlam = 1e-7
        slope = (det(A - (lam + dlam) * np.eye(4)) - det(A - (lam - dlam) * np.eye(4))) / (2 * dlam)
        assert abs(det(A - lam * np.eye(4))) / abs(slope) < 1e-12
    assert np.sum(w) == pytest.approx(np.trace(A).real, abs=1e-13)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64])
def test_known_spectrum(n):
    """Q Lambda Q^H with Q a product of 16 seeded Householder reflectors."""
    r = _rng(n)
    lam = np.sort(r.uniform(0.5, 12.0, n))
    if n >= 17:
        lam[3] = lam[4]              # an exactly degenerate pair
    Q = _random_unitary(n, n + 100)
    A = (Q * lam) @ Q.conj().T
    A = (A + A.conj().T) / 2
    w, Z = oracle.eigh(A)
    assert np.allclose(w, np.sort(lam), rtol=0, atol=2e-13)
    assert np.linalg.norm(Z.conj().T @ Z - np.eye(n)) < 1e-12
    assert np.linalg.norm(A @ Z - Z * w) < 1e-12


def test_matches_lapack_on_bse_matrix():
    """Cross-check against LAPACK (numpy) on a synthetic BSE matrix."""
    H = oracle.build_h(0, 20, 4, 4)
    w, Z = oracle.eigh(H, 10)
    assert np.allclose(w, np.linalg.eigvalsh(H), rtol=0, atol=1e-12)
    assert np.linalg.norm(H @ Z - Z * w[:10]) < 1e-12
