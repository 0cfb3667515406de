"""Pins of the oracle ChASE phases against closed forms, the paper's
printed tables and brute force."""
import math

import numpy as np
import pytest

import oracle
from conftest import golden


def _cheb(d, x):
    """T_d(x) from the closed forms T_d(cos t) = cos(d t), T_d(+-cosh p) =
    (+-1)^d cosh(d p)."""
    if abs(x) <= 1.0:
        return math.cos(d * math.acos(x))
    s = 1.0 if x > 0 or d % 2 == 0 else -1.0
    return s * math.cosh(d * math.acosh(abs(x)))


@pytest.mark.parametrize("table", ["nex25.txt", "nex100.txt"])
def test_interval_and_rate_match_paper_tables(table):
    """Supplement Tables S8/S9: c, e from (alpha, beta) and 1/rho_nev from
    Eq. (S1) with gamma = lambda_nev, to the printed 5 decimals."""
    for row in golden(table):
        lam, alpha, beta, c, e, inv_rho = map(float, row[1:7])
        cc, ee = oracle.filter_interval(alpha, beta)
        assert cc == pytest.approx(c, abs=1.01e-5)
        assert ee == pytest.approx(e, abs=1.01e-5)
        assert 1.0 / oracle.convergence_rate(lam, cc, ee) == pytest.approx(inv_rho, abs=1.01e-5)


def test_rate_inside_interval_is_one():
    assert oracle.convergence_rate(5.0, 5.0, 2.0) == 1.0
    assert oracle.convergence_rate(3.0, 5.0, 2.0) == 1.0


@pytest.mark.parametrize("degs", [[1], [2, 2, 2], [2, 4, 4, 7, 12], [3, 36]])
def test_filter_diagonal_closed_form(degs):
    """On a diagonal H the filter maps component i of column j to
    T_d((lam_i - c)/e) / T_d((lower - c)/e) times itself."""
    lam = np.linspace(0.5, 12.0, 23)
    H = np.diag(lam).astype(np.complex128)
    m = len(degs)
    V = oracle.random_block(1, 5, len(lam), m)
    lower, alpha, beta = 0.45, 3.0, 12.5
    c, e = oracle.filter_interval(alpha, beta)
    Y, mv = oracle.chebyshev_filter(H, V, degs, lower, c, e)
    assert mv == sum(degs)
    for j, d in enumerate(degs):
        scale = np.array([_cheb(d, (x - c) / e) / _cheb(d, (lower - c) / e) for x in lam])
        assert np.allclose(Y[:, j], scale * V[:, j], rtol=1e-12, atol=1e-14)


def test_filter_is_polynomial_in_h():
    """Filtering with a non-diagonal H equals U p_d(Lam) U^H V."""
    r = np.random.default_rng(0)
    n = 30
    X = r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))
    A = (X + X.conj().T) / 4
    lam, U = np.linalg.eigh(A)
    V = oracle.random_block(2, 5, n, 3)
    lower = lam[0]
    c, e = oracle.filter_interval(lam[5], lam[-1] + 0.1)
    Y, _ = oracle.chebyshev_filter(A, V, [4, 6, 6], lower, c, e)
    for j, d in enumerate([4, 6, 6]):
        p = np.array([_cheb(d, (x - c) / e) / _cheb(d, (lower - c) / e) for x in lam])
        assert np.allclose(Y[:, j], U @ (p * (U.conj().T @ V[:, j])), rtol=1e-10, atol=1e-12)


def test_cholesky_unique_factor():
    """R from G = R^H R equals numpy's QR R with a positive real diagonal."""
    r = np.random.default_rng(5)
    X = r.standard_normal((40, 9)) + 1j * r.standard_normal((40, 9))
    R = oracle.cholesky(X.conj().T @ X)
    _, R2 = np.linalg.qr(X)
    ph = np.diag(R2) / np.abs(np.diag(R2))
    R2 = R2 / ph[:, None]
    assert np.allclose(R, R2, rtol=0, atol=1e-12)
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R).imag == 0)
    assert oracle.cholesky(-np.eye(3, dtype=complex)) is None


def test_qr_ill_conditioned_and_locked():
    """Shifted CholeskyQR3 orthonormalises a kappa ~ 1e12 block, keeps its
    span, and removes the locked directions."""
    r = np.random.default_rng(7)
    n, m, k = 300, 12, 4
    L, _ = np.linalg.qr(r.standard_normal((n, k)) + 1j * r.standard_normal((n, k)))
    A = r.standard_normal((n, m)) + 1j * r.standard_normal((n, m))
    U, _, Wh = np.linalg.svd(A, full_matrices=False)
    A = (U * np.logspace(0, -12, m)) @ Wh + L @ (r.standard_normal((k, m)))
    Q = oracle.qr(L, A)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(m)) < 1e-13
    assert np.linalg.norm(L.conj().T @ Q) < 1e-13
    # span: the projection of A (minus its locked part) onto span(Q) is exact
    P = A - L @ (L.conj().T @ A)
    assert np.linalg.norm(P - Q @ (Q.conj().T @ P)) < 1e-10 * np.linalg.norm(P)


def test_rayleigh_ritz_exact_on_invariant_subspace():
    """RR on an exact invariant subspace returns its eigenvalues and zero
    residuals."""
    r = np.random.default_rng(9)
    n = 50
    X = r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))
    A = (X + X.conj().T) / 2
    lam, U = np.linalg.eigh(A)
    M = U[:, :6] @ (r.standard_normal((6, 6)) + 1j * r.standard_normal((6, 6)))
    Q, _ = np.linalg.qr(M)
    th, V, HV = oracle.rayleigh_ritz(A, Q)
    assert np.allclose(th, lam[:6], rtol=0, atol=1e-12)
    assert np.max(oracle.residuals(HV, V, th, 1.0)) < 1e-12


def test_lanczos_full_steps_recovers_spectrum():
    """With k = N steps from a generic start, the Ritz values of T are the
    eigenvalues of H (small N, no breakdown), so mu_1 = lambda_1 and beta
    bounds lambda_N."""
    r = np.random.default_rng(2)
    lam = np.sort(r.uniform(1.0, 9.0, 8))
    Q = np.linalg.qr(r.standard_normal((8, 8)) + 1j * r.standard_normal((8, 8)))[0]
    A = (Q * lam) @ Q.conj().T
    est = oracle.lanczos_bounds(A, 3, seed=1, n_runs=2, k_steps=8)
    assert est["mu_1"] == pytest.approx(lam[0], abs=1e-9)
    assert est["beta"] >= lam[-1] - 1e-9
    assert lam[0] - 1e-9 <= est["mu_m"] <= lam[-1] + 1e-9


def test_lanczos_bounds_on_bse_matrix():
    H = oracle.build_h(0, 40, 4, 4)
    w = np.linalg.eigvalsh(H)
    est = oracle.lanczos_bounds(H, 60, seed=0)
    assert est["beta"] >= w[-1]                     # upper bound
    assert w[0] - 1e-9 <= est["mu_1"] <= w[0] + 0.05
    assert w[0] <= est["mu_m"] <= w[-1]


def test_degree_rule():
    c, e, tol = 8.0, 5.0, 1e-10
    th = np.array([0.8, 2.0, 2.9, 3.0])            # last one at alpha -> rho = 1
    res = np.array([1e-3, 1e-6, 1e-12, 1e-4])
    d = oracle.degrees(th, res, c, e, tol, 36)
    assert d[3] == 36 and d[2] == 2
    assert np.all(d % 2 == 0) and np.all((d >= 2) & (d <= 36))
    for j in range(2):
        rho = oracle.convergence_rate(th[j], c, e)
        # the degree is the smallest even one that damps r_j below tol
        assert res[j] * rho ** (-float(d[j])) <= tol
        assert res[j] * rho ** (-float(d[j] - 2)) > tol


def test_lock_contiguous_from_bottom():
    assert oracle.lock_count(np.array([1e-11, 1e-12, 1e-3, 1e-13]), 1e-10, 0, 10) == 2
    assert oracle.lock_count(np.array([1e-11, 1e-12, 1e-13]), 1e-10, 8, 10) == 2
    assert oracle.lock_count(np.array([1e-3, 1e-12]), 1e-10, 0, 10) == 0


def _subspace_gap(A, B):
    """sin of the largest principal angle between span(A) and span(B) (equal
    dimensions): ||(I - Qa Qa^H) Qb||_2, accurate for small angles."""
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    return float(np.linalg.norm(Qb - Qa @ (Qa.conj().T @ Qb), 2))


@pytest.mark.parametrize("Nk,nev,nex", [(16, 20, 10), (30, 40, 16)])
def test_chase_matches_dense(Nk, nev, nex):
    H = oracle.build_h(0, Nk, 4, 4)
    w, Z = oracle.eigh(H, nev + 1)
    r = oracle.chase(H, nev, nex, tol=1e-10, deg_max=36)
    assert r["status"] == "ok"
    assert 2 <= r["iters"] <= 15
    assert np.max(np.abs(r["evals"] - w[:nev]) / np.abs(w[:nev])) < 1e-10
    assert np.max(r["resid"]) <= 1e-10
    V = r["evecs"]
    assert np.linalg.norm(V.conj().T @ V - np.eye(nev)) < 1e-12
    assert np.linalg.norm(H @ V - V * r["evals"]) / np.linalg.norm(H, 2) < 1e-9
    # Davis-Kahan sin-theta bound: the angle to the exact invariant subspace
    # is at most ||H V - V Lambda||_F / (lambda_{nev+1} - max computed).
    gap = w[nev] - r["evals"][-1]
    if gap > 1e-6:
        bound = np.linalg.norm(H @ V - V * r["evals"]) / gap
        assert _subspace_gap(V, Z[:, :nev]) <= 1.01 * bound + 1e-12


def test_chase_warm_start_saves_iterations():
    H = oracle.build_h(0, 30, 4, 4)
    cold = oracle.chase(H, 30, 15)
    warm = oracle.chase(H, 30, 15, V0=cold["evecs"])
    assert warm["status"] == "ok" and warm["iters"] < cold["iters"]
    assert np.allclose(warm["evals"], cold["evals"], rtol=1e-10, atol=0)


def test_chase_noconv_reports_inf():
    H = oracle.build_h(0, 16, 4, 4)
    r = oracle.chase(H, 20, 10, max_iter=1)
    assert r["status"] == "noconv"
    assert np.all(np.isinf(r["resid"]))


def test_degree_cap_bounds_amplification():
    """The cap is the largest even degree with |T_d((lower-c)/e)| <= 1e12."""
    lower, c, e = 0.5, 8.0, 5.0
    d = oracle.degree_cap(lower, c, e)
    t = (lower - c) / e
    assert abs(_cheb(d, t)) <= 1e12 < abs(_cheb(d + 2, t))
    assert d % 2 == 0
    assert oracle.degree_cap(5.0, 8.0, 5.0) is None          # inside the interval
    assert oracle.degree_cap(-1e6, 8.0, 1e-3) == 2            # floor of 2


def test_chase_full_search_space():
    """m = N: the capped filter keeps the block full rank and Rayleigh-Ritz
    on the whole space is exact."""
    H = oracle.build_h(5, 3, 4, 4)                           # N = 48
    w = np.linalg.eigvalsh(H)
    r = oracle.chase(H, 40, 8)
    assert r["status"] == "ok"
    assert np.max(np.abs(r["evals"] - w[:40])) < 1e-12


@pytest.mark.parametrize("width", [0, 1, 4, 48])
def test_group_degrees_properties(width):
    rng = np.random.default_rng(width + 3)
    deg = np.sort(rng.integers(1, 19, size=75) * 2)
    g = oracle.group_degrees(deg, width)
    assert np.all(np.diff(g) >= 0) and np.all(g >= deg)
    if width <= 1:
        assert np.array_equal(g, deg)
        return
    # groups of `width` from the top share the group's largest degree
    hi = len(deg)
    while hi > 0:
        lo = max(0, hi - width)
        assert np.all(g[lo:hi] == deg[hi - 1])
        hi = lo
    # every filter step's active set is a union of whole groups from the top
    allowed = {min(k * width, len(g)) for k in range(len(g) // width + 2)}
    for t in range(1, int(g.max()) + 1):
        assert int(np.sum(g >= t)) in allowed


def test_chase_grouped_degrees_matches_dense():
    """Grouped degrees only add filtering: the solve reaches the same
    eigenpairs as the dense eigensolver, in no more iterations."""
    H = oracle.build_h(0, 30, 4, 4)
    w, _ = oracle.eigh(H, 41)
    plain = oracle.chase(H, 40, 16)
    r = oracle.chase(H, 40, 16, degree_group=48)
    assert r["status"] == "ok" and r["iters"] <= plain["iters"]
    assert np.max(np.abs(r["evals"] - w[:40]) / np.abs(w[:40])) < 1e-10
    assert np.max(r["resid"]) <= 1e-10


def _lanczos_closed_form(N, n_runs, seed):
    """H = Q diag(lam) Q^H with a known spectrum, and the closed-form
    quantities of k = N Lanczos steps from the oracle's start vectors: the
    Ritz values of each run are the eigenvalues, and the weight of Ritz value
    lam_i is tau_i = |q_i^H v_0|^2 (the first component of the eigenvector of
    T is the overlap of the start vector with the eigenvector of H).  The
    estimated count at lam_j is C_j = N * mean_runs sum_{i <= j} tau_i."""
    r = np.random.default_rng(seed)
    lam = np.sort(r.uniform(1.0, 9.0, N))
    Q = np.linalg.qr(r.standard_normal((N, N)) + 1j * r.standard_normal((N, N)))[0]
    A = (Q * lam) @ Q.conj().T
    V0 = oracle.random_block(1, oracle.STREAM_LANCZOS, N, n_runs)
    tau = np.abs(Q.conj().T @ (V0 / np.linalg.norm(V0, axis=0))) ** 2      # N x runs
    C = N * np.cumsum(tau.mean(axis=1))
    return A, lam, tau, C


def test_lanczos_mu_m_interpolates_the_count_one_run():
    """One run of N steps: mu_m is the point where the count N sum tau_i
    reaches m, linear between consecutive Ritz values (closed form from the
    eigenvectors, not from the tridiagonal), and clamps at both ends."""
    N = 8
    A, lam, tau, C = _lanczos_closed_form(N, 1, 2)
    for j in range(1, N):
        for frac in (0.2, 0.5, 0.9):
            m = C[j - 1] + frac * (C[j] - C[j - 1])
            want = lam[j - 1] + frac * (lam[j] - lam[j - 1])
            est = oracle.lanczos_bounds(A, m, seed=1, n_runs=1, k_steps=N)
            assert est["mu_m"] == pytest.approx(want, abs=1e-9)
    assert oracle.lanczos_bounds(A, 0.5 * C[0], seed=1, n_runs=1, k_steps=N)["mu_m"] == \
        pytest.approx(lam[0], abs=1e-9)
    assert oracle.lanczos_bounds(A, N + 3, seed=1, n_runs=1, k_steps=N)["mu_m"] == \
        pytest.approx(lam[-1], abs=1e-9)


@pytest.mark.parametrize("n_runs", [2, 3])
def test_lanczos_mu_m_pooled_runs_closed_form(n_runs):
    """Several runs of N steps: every run's Ritz values are the eigenvalues,
    so the pooled list holds each lam_j n_runs times, with weights
    (N / n_runs) tau_j^(l).  A target count just below C_j (by less than the
    smallest of those weights) is crossed inside the group of copies of lam_j,
    so mu_m = lam_j.  A weight of N (not N / n_runs), or tau taken from the
    last component of the eigenvector of T, moves the crossing elsewhere."""
    N = 8
    A, lam, tau, C = _lanczos_closed_form(N, n_runs, 2)
    for j in range(N):
        w = (N / n_runs) * tau[j]
        m = C[j] - 0.5 * float(np.min(w))
        est = oracle.lanczos_bounds(A, m, seed=1, n_runs=n_runs, k_steps=N)
        assert est["mu_m"] == pytest.approx(lam[j], abs=1e-9)
        assert est["mu_1"] == pytest.approx(lam[0], abs=1e-9)


def test_nex_regression_reproduces_table_s10():
    """Eq. (S2) against every entry of Table S10.  The text names E_cut-high =
    12.82 eV, but at 12.82 the table prints 76 and 106, not nex_high; the
    printed values are those of E_cut-high in (14.311, 14.334] eV rounded to
    the nearest integer (reading: E_cut-high = 14.32 eV).  With 12.82 the last
    row would be nex_high itself."""
    for row in golden("nex_dyn.txt"):
        e_cut, n100, n150 = float(row[1]), int(row[2]), int(row[3])
        for nex_high, printed in ((100, n100), (150, n150)):
            v = oracle.nex_regression(e_cut, 10.54, 14.32, 40, nex_high)
            assert int(math.floor(v + 0.5)) == printed
            assert abs(v - printed) <= 0.5
    # the interpolation's end points and its linearity
    assert oracle.nex_regression(10.54, 10.54, 14.32, 40, 150) == 40
    assert oracle.nex_regression(14.32, 10.54, 14.32, 40, 150) == pytest.approx(150)
    assert oracle.nex_regression(12.43, 10.54, 14.32, 40, 100) == pytest.approx(70)
    assert oracle.nex_regression(12.82, 10.54, 12.82, 40, 100) == pytest.approx(100)


def test_damping_matches_tables_s8_s9():
    """damping(lambda_nev, alpha, beta) = 1/rho_nev of Tables S8 and S9."""
    for table in ("nex25.txt", "nex100.txt"):
        for row in golden(table):
            lam, alpha, beta, inv_rho = float(row[1]), float(row[2]), float(row[3]), float(row[6])
            assert oracle.damping(lam, alpha, beta) == pytest.approx(inv_rho, abs=1.01e-5)


def test_grown_nex_limits():
    assert oracle.grown_nex(40, 100, 20000) == 80
    assert oracle.grown_nex(3, 10, 1000) == 11
    assert oracle.grown_nex(200, 300, 20000) == 212        # m <= 512
    assert oracle.grown_nex(10, 40, 56) == 16              # m <= N


def test_chase_nex_tuner():
    """nev = 50, nex = 10 on the N = 2000 matrix: the settled damping of the
    last wanted pair (about 0.81) exceeds a target of 0.75, so nex doubles
    once; the solve reaches the dense eigenvalues in fewer iterations.  A
    target above the damping changes nothing, bit for bit."""
    H = oracle.build_h(0, 125, 4, 4)
    w, _ = oracle.eigh(H, 0)
    plain = oracle.chase(H, 50, 10, trace=True)
    tuned = oracle.chase(H, 50, 10, nex_damping=0.75)
    assert plain["nex"] == 10 and tuned["nex"] == 20
    assert tuned["status"] == "ok" and tuned["iters"] < plain["iters"]
    assert np.max(np.abs(tuned["evals"] - w[:50]) / np.abs(w[:50])) < 1e-10
    assert np.max(tuned["resid"]) <= 1e-10
    # the damping the tuner saw settles near the value of the exact spectrum
    h = plain["history"][-1]
    d_last = oracle.damping(h["theta"][50 - 1 - h["locked"]], h["theta"][-1], h["beta"])
    assert d_last == pytest.approx(oracle.damping(w[49], w[59], h["beta"]), abs=0.01)
    same = oracle.chase(H, 50, 10, nex_damping=0.99)
    assert same["nex"] == 10 and np.array_equal(same["evals"], plain["evals"])
