"""Pins of the structured eigenvalue oracle (oracle/structured.py): the
Sylvester/Haynsworth eigenvalue count and the structured product H V are
checked against the dense oracle (its own Householder + implicit QR
eigensolver), LAPACK, brute-force counts and the circulant closed form."""
import math

import numpy as np
import pytest

import oracle
from oracle import structured

CASES = [
    ((125, 4, 4), None),                                          # C1 matrix
    ((7, 3, 5), None),                                            # ragged N = 105
    ((24, 1, 1), dict(dispersion=0.0, jitter=0.0, x0=0.0)),        # degenerate circulant
    ((9, 2, 2), dict(rank_x=1, w0=0.0)),                          # rank-1 exchange only
    ((5, 4, 3), dict(rank_x=0, w0=0.7, band_gap=3.0)),            # no exchange
    ((10, 2, 3), dict(rank_x=20)),                                # rank above the block size
    ((16, 4, 4), dict(w0=1.5, x0=3.0)),                           # strong coupling
]


@pytest.mark.parametrize("shape,model", CASES)
def test_count_matches_dense_spectrum(shape, model):
    """#{lambda < sigma} equals the brute-force count from the dense
    oracle's eigenvalues at every midpoint between distinct eigenvalues and
    outside the spectrum."""
    H = oracle.build_h(3, *shape, model)
    w, _ = oracle.eigh(H, 0)
    B = structured.bse_blocks(3, *shape, model)
    gaps = np.diff(w)
    sig = np.concatenate([(w[:-1] + 0.5 * gaps)[gaps > 1e-10], [w[0] - 1.0, w[-1] + 1.0]])
    assert np.array_equal(structured.eig_count(B, sig), np.searchsorted(w, sig))


@pytest.mark.parametrize("shape,model", CASES)
def test_bisection_eigenvalues_match_dense(shape, model):
    H = oracle.build_h(3, *shape, model)
    w, _ = oracle.eigh(H, 0)
    k = min(60, len(w))
    lam = structured.lowest_eigenvalues(structured.bse_blocks(3, *shape, model), k)
    assert np.max(np.abs(lam - w[:k])) <= 1e-13 * np.max(np.abs(w))
    assert np.max(np.abs(lam - np.linalg.eigvalsh(H)[:k])) <= 1e-13 * np.max(np.abs(w))


def test_count_on_exact_block_eigenvalue():
    """x0 = 0 and flat bands: the spectrum is the circulant closed form
    E0 - w0 sum_d K(d) cos(2 pi q d / Nk) (exact double eigenvalues); counts
    just below and above each distinct value step by its multiplicity."""
    Nk, w0 = 24, 0.3
    md = dict(dispersion=0.0, jitter=0.0, x0=0.0, w0=w0)
    lam = []
    for q in range(Nk):
        s = sum(math.cos(2 * math.pi * q * d / Nk) / (min(d, Nk - d) ** 2 + 0.5)
                for d in range(Nk))
        lam.append(2.0 - w0 * s)
    lam = np.sort(lam)
    B = structured.bse_blocks(9, Nk, 1, 1, md)
    distinct = np.unique(np.round(lam, 12))
    for x in distinct:
        mult = int(np.sum(np.abs(lam - x) < 1e-9))
        lo = structured.eig_count(B, x - 1e-9)[0]
        hi = structured.eig_count(B, x + 1e-9)[0]
        assert hi - lo == mult
    assert np.allclose(structured.lowest_eigenvalues(B, Nk), lam, rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape,model", CASES)
def test_operator_matches_dense_product(shape, model):
    H = oracle.build_h(3, *shape, model)
    op = structured.BseOperator(3, *shape, model)
    V = oracle.random_block(1, 5, H.shape[0], 9)
    ref = H @ V
    assert op.shape == H.shape
    assert np.max(np.abs(op @ V - ref)) <= 2e-15 * np.max(np.abs(H)) * np.max(np.sum(np.abs(V), 0))
    v = V[:, 3].copy()
    assert np.max(np.abs(op @ v - H @ v)) <= 2e-15 * np.max(np.abs(H)) * np.sum(np.abs(v))


def test_oracle_chase_on_operator_matches_dense():
    """The plain oracle ChASE run on the structured operator reaches the
    dense eigenvalues (it only uses H @ V and H.shape)."""
    H = oracle.build_h(0, 30, 4, 4)
    w, _ = oracle.eigh(H, 0)
    r = oracle.chase(structured.BseOperator(0, 30, 4, 4), 40, 16, tol=1e-10)
    assert r["status"] == "ok"
    assert np.max(np.abs(r["evals"] - w[:40]) / np.abs(w[:40])) < 1e-10
    assert np.linalg.norm(H @ r["evecs"] - r["evecs"] * r["evals"]) / np.max(np.abs(w)) < 1e-9
