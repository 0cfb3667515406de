"""Pins of the oracle's RNG and synthetic Eq. (1) Hamiltonian."""
import math

import numpy as np
import pytest

import oracle
from conftest import golden


def test_splitmix64_published_vector():
    for key, hexval in golden("splitmix64.txt"):
        assert oracle.splitmix64(int(key)) == int(hexval, 16)


def test_uniform_range_and_moments():
    u = np.array([oracle.uniform(7, 2, i) for i in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1.0 / 12.0) < 0.005


def test_random_block_layout_and_streams():
    V = oracle.random_block(3, 5, 6, 4)
    W = oracle.random_block(3, 5, 6, 5)
    assert np.array_equal(V, W[:, :4])         # column j depends on (j, i) only
    assert V.flags["F_CONTIGUOUS"]
    assert np.all(np.abs(V.real) <= 1) and np.all(np.abs(V.imag) <= 1)
    assert not np.array_equal(V, oracle.random_block(3, 4, 6, 4))


@pytest.mark.parametrize("Nk,Nv,Nc", [(5, 2, 3), (16, 4, 4), (7, 1, 1)])
def test_hermitian_exact(Nk, Nv, Nc):
    H = oracle.build_h(11, Nk, Nv, Nc)
    assert H.shape == (Nk * Nv * Nc,) * 2
    assert np.array_equal(H, H.conj().T)        # bit-exact mirror
    assert np.all(np.diag(H).imag == 0.0)


def test_no_coupling_no_spectrum_change():
    """x0 = w0 = 0: H is diagonal and its spectrum is the sorted transition
    energies E_c(k) - E_v(k)."""
    md = dict(x0=0.0, w0=0.0)
    H = oracle.build_h(2, 10, 3, 2, md)
    assert np.count_nonzero(H - np.diag(np.diag(H))) == 0
    w, _ = oracle.eigh(H, 0)
    assert np.allclose(w, np.sort(np.diag(H).real), rtol=0, atol=1e-14)


def test_transition_energies_closed_form():
    """dE(k, v, c) = gap + c + v/2 + 5 s(k) + j xi with s = (1 - cos 2 pi k/Nk)/2."""
    Nk, Nv, Nc = 8, 2, 3
    dE, _, _ = oracle.bse_tables(5, Nk, Nv, Nc, dict(jitter=0.0))
    for k in range(Nk):
        s = (1 - math.cos(2 * math.pi * k / Nk)) / 2
        for v in range(Nv):
            for c in range(Nc):
                I = (k * Nv + v) * Nc + c
                assert dE[I] == pytest.approx(2.0 + c + 0.5 * v + 5 * s, abs=1e-14)
    assert dE.min() >= 2.0 - 1e-14


def test_direct_term_circulant_spectrum():
    """Nv = Nc = 1, flat bands, no jitter, no exchange: H = E0 I - w0 Phi C
    Phi^H with C circulant, so the eigenvalues are
    E0 - w0 * sum_d K(d) cos(2 pi q d / Nk) with K(d) = 1/(d^2 + 1/2) and d
    the ring distance."""
    Nk, w0 = 24, 0.3
    H = oracle.build_h(9, Nk, 1, 1, dict(dispersion=0.0, jitter=0.0, x0=0.0, w0=w0))
    E0 = 2.0
    lam = []
    for q in range(Nk):
        s = 0.0
        for d in range(Nk):
            dr = min(d, Nk - d)
            s += math.cos(2 * math.pi * q * d / Nk) / (dr * dr + 0.5)
        lam.append(E0 - w0 * s)
    w, _ = oracle.eigh(H, 0)
    assert np.allclose(w, np.sort(lam), rtol=0, atol=1e-13)
    assert min(lam) > 0.0   # K is positive definite on the ring: W is PSD


def test_exchange_rank1_secular_equation():
    """w0 = 0, rank-1 exchange: H = D + 2 a a^H, and every eigenvalue is a
    root of the secular equation 1 = 2 sum_i |a_i|^2 / (lambda - d_i)."""
    Nk, Nv, Nc = 6, 2, 2
    md = dict(w0=0.0, rank_x=1, x0=0.5)
    H = oracle.build_h(4, Nk, Nv, Nc, md)
    dE, a, _ = oracle.bse_tables(4, Nk, Nv, Nc, md)
    w, _ = oracle.eigh(H, 0)
    a2 = np.abs(a[:, 0]) ** 2
    for lam in w:
        f = 1.0 - 2.0 * np.sum(a2 / (lam - dE))
        # f is monotone between poles; its derivative scales the residual
        fp = 2.0 * np.sum(a2 / (lam - dE) ** 2)
        assert abs(f) / fp < 1e-10
    # interlacing: lambda_i in [d_(i), d_(i+1)] (rank-one positive update)
    d = np.sort(dE)
    assert np.all(w >= d - 1e-12)
    assert np.all(w[:-1] <= d[1:] + 1e-12)


def test_exchange_sparsity_and_trace():
    """trace(H) = sum dE + sum X_II - N w0 K(0) and equals sum of eigenvalues;
    the direct term couples only equal (v, c)."""
    Nk, Nv, Nc = 9, 2, 2
    md = dict(x0=0.0)
    H = oracle.build_h(1, Nk, Nv, Nc, md)
    for I in range(H.shape[0]):
        for J in range(H.shape[0]):
            if I % (Nv * Nc) != J % (Nv * Nc):
                assert H[I, J] == 0
    H = oracle.build_h(1, Nk, Nv, Nc)
    dE, a, _ = oracle.bse_tables(1, Nk, Nv, Nc)
    X_diag = 2.0 * np.sum(np.abs(a) ** 2, axis=1)
    tr = np.sum(dE) + np.sum(X_diag) - H.shape[0] * 0.3 * 2.0
    assert np.trace(H).real == pytest.approx(tr, rel=1e-13)
    w, _ = oracle.eigh(H, 0)
    assert np.sum(w) == pytest.approx(tr, rel=1e-12)


def test_exchange_magnitude():
    """E |a_r(I)|^2 = x0 / N, so the exchange term 2 A A^H has trace ~ 2 R x0."""
    Nk, Nv, Nc = 125, 4, 4
    _, a, _ = oracle.bse_tables(0, Nk, Nv, Nc)
    tr = 2.0 * np.sum(np.abs(a) ** 2)
    assert tr == pytest.approx(2 * 8 * 0.5, rel=0.05)
