"""Plain CPU FP64 ChASE (Chebyshev-accelerated subspace iteration).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (arXiv 2006.08498) names the solver's phases but does not list
its steps; each function below cites the passage that defines its phase and
states the reading taken where the paper is silent:

  lanczos_bounds   Supplement, "Lanczos" item of the ChASE timing breakdown
                   (spectral-density estimate of lambda_1, lambda_{nev+nex},
                   lambda_N; run once); beta is fixed for the whole solve
                   (Supplement, discussion of Tables S8/S9).
  filter_interval  Supplement, Tables S8/S9: c and e are the centre and
                   half-width of the damped interval [alpha, beta].
  chebyshev_filter Sec. 3 (three-term Chebyshev recurrence run as BLAS-3)
                   and the Supplement's "Filter" item (repeated HEMM).
  qr               Supplement, "QR" item (orthonormalise the filtered block).
  rayleigh_ritz    Supplement, "RR" item (project, reduced eig, back-transform).
  residuals, lock  Supplement, "Resid" item (residuals, deflation, locking).
  degrees          Eq. (S1) (convergence ratio rho) and Sec. 3 ("pre-computing
                   and minimizing the total FLOP count").

Matrix products use numpy's matmul (a library primitive); the small
Hermitian eigensolver and the Cholesky factorisation are the oracle's own C
routines.  Nothing is blocked, fused or reordered beyond what each step
states.
"""
import math

import numpy as np
import scipy.linalg

from . import _lib
from ._lib import Model, fortran, ptr

U = 2.0 ** -53                 # unit roundoff of IEEE double

STREAM_XI, STREAM_EXCHANGE, STREAM_THETA = 1, 2, 3
STREAM_LANCZOS, STREAM_START = 4, 5


# ----------------------------------------------------------------- inputs

def default_model():
    """Synthetic-model defaults: gap 2 eV, w0 0.3 eV, x0 0.5 eV, 0.01 eV
    jitter, unit dispersion, rank-8 exchange."""
    return dict(band_gap=2.0, w0=0.3, x0=0.5, jitter=0.01, dispersion=1.0,
                rank_x=8)


def _model(model):
    md = default_model()
    if model:
        md.update(model)
    return Model(md["band_gap"], md["w0"], md["x0"], md["jitter"],
                 md["dispersion"], int(md["rank_x"]))


def build_h(seed, Nk, Nv, Nc, model=None):
    """The synthetic Eq. (1) Hamiltonian, N = Nk*Nv*Nc, complex128,
    column-major (numpy Fortran order)."""
    N = Nk * Nv * Nc
    H = np.zeros((N, N), dtype=np.complex128, order="F")
    md = _model(model)
    _lib.lib().or_bse_build(seed, Nk, Nv, Nc, md, ptr(H), N)
    return H


def bse_elements(seed, Nk, Nv, Nc, I, J, model=None):
    """H[I[t], J[t]] of the synthetic Hamiltonian without forming H."""
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    out = np.zeros(len(I), dtype=np.complex128)
    _lib.lib().or_bse_elements(seed, Nk, Nv, Nc, _model(model), len(I), ptr(I), ptr(J),
                               ptr(out))
    return out


def bse_tables(seed, Nk, Nv, Nc, model=None):
    """(dE[N], a[N, R], theta[N]) of the synthetic model."""
    N = Nk * Nv * Nc
    md = _model(model)
    R = md.rank_x
    dE = np.zeros(N)
    a = np.zeros((N, max(R, 1)), dtype=np.complex128)  # row-major: a[I, r]
    th = np.zeros(N)
    _lib.lib().or_bse_tables(seed, Nk, Nv, Nc, md, ptr(dE), ptr(a), ptr(th))
    return dE, a[:, :R], th


def random_block(seed, stream, n, m):
    """Seeded n x m complex block with entries (2u-1) + i(2u'-1)."""
    V = np.zeros((n, m), dtype=np.complex128, order="F")
    if n and m:
        _lib.lib().or_random_block(seed, stream, n, m, ptr(V), n)
    return V


def uniform(seed, stream, idx):
    return _lib.lib().or_uniform(seed, stream, idx)


def splitmix64(key):
    return _lib.lib().or_splitmix64(key)


# ------------------------------------------------------ dense eigensolver

def tridiag_eig(d, e, vectors=True):
    """Eigen-decomposition of the real symmetric tridiagonal matrix with
    diagonal d and off-diagonal e (implicit QR, Wilkinson shift).  Returns
    ascending eigenvalues and (optionally) the n x n eigenvector matrix."""
    n = len(d)
    dd = np.array(d, dtype=np.float64)
    ee = np.zeros(max(n, 1))
    ee[:n - 1] = e
    Z = np.eye(n) if vectors else None  # row-major n x n
    rc = _lib.lib().or_tridiag_eig(n, ptr(dd), ptr(ee), ptr(Z) if vectors else None)
    if rc != 0:
        raise RuntimeError("tridiagonal QR did not converge")
    return (dd, Z) if vectors else dd


def eigh(A, nz=None):
    """All eigenvalues (ascending) of the Hermitian A, and the eigenvectors
    of the nz smallest (all if nz is None): Householder tridiagonalisation,
    phase to real tridiagonal, implicit QR, back-transformation."""
    A = fortran(A, np.complex128).copy(order="F")
    n = A.shape[0]
    nz = n if nz is None else nz
    w = np.zeros(n)
    Z = np.zeros((n, max(nz, 1)), dtype=np.complex128, order="F")
    rc = _lib.lib().or_heev(n, ptr(A), n, ptr(w), ptr(Z), n, nz)
    if rc != 0:
        raise RuntimeError("dense eigensolver did not converge")
    return w, Z[:, :nz]


def cholesky(G):
    """Upper R with G = R^H R (real positive diagonal), or None if G is not
    numerically positive definite."""
    R = fortran(G, np.complex128).copy(order="F")
    n = R.shape[0]
    rc = _lib.lib().or_cholesky(n, ptr(R), n)
    return None if rc != 0 else R


# ------------------------------------------------------------- the phases

def lanczos_bounds(H, m, seed, n_runs=4, k_steps=25):
    """Spectral estimate of lambda_1, lambda_m and lambda_N.

    n_runs independent Lanczos runs of k_steps steps each (no
    re-orthogonalisation) from seeded unit vectors (stream 4, column l for
    run l).  For run l the tridiagonal T_l has Ritz values theta_i and
    weights tau_i = (first component of its eigenvector)^2.  Readings (the
    paper names only the three estimates):
      beta    = max over runs of (max theta + |last off-diagonal|): an upper
                bound of lambda_N;
      mu_1    = min over runs of min theta;
      mu_m    = the point where the estimated eigenvalue count
                N * mean_l sum_{theta_i <= x} tau_i reaches m, interpolated
                linearly between consecutive pooled Ritz values;
      norm_est = max(|mu_1|, |beta|).
    """
    N = H.shape[0]
    V0 = random_block(seed, STREAM_LANCZOS, N, n_runs)
    k = min(k_steps, N)
    thetas, taus, uppers = [], [], []
    for l in range(n_runs):
        v = V0[:, l] / np.linalg.norm(V0[:, l])
        v_prev = np.zeros(N, dtype=np.complex128)
        b_prev = 0.0
        a_list, b_list = [], []
        for j in range(k):
            w = H @ v
            a_j = float(np.real(np.vdot(v, w)))
            w = w - a_j * v - b_prev * v_prev
            b_j = float(np.linalg.norm(w))
            a_list.append(a_j)
            b_list.append(b_j)
            if b_j == 0.0:
                break
            v_prev, v = v, w / b_j
            b_prev = b_j
        th, Z = tridiag_eig(a_list, b_list[:-1])
        thetas.append(th)
        taus.append(Z[0, :] ** 2)
        uppers.append(th[-1] + abs(b_list[-1]))
    beta = max(uppers)
    mu_1 = min(t[0] for t in thetas)
    allt = np.concatenate(thetas)
    allw = np.concatenate(taus) * (N / n_runs)
    order = np.argsort(allt, kind="stable")
    xs, cnt = allt[order], np.cumsum(allw[order])
    return dict(beta=beta, mu_1=mu_1, mu_m=count_point(xs, cnt, m),
                norm_est=max(abs(mu_1), abs(beta)), density=(xs, cnt))


def count_point(xs, cnt, m):
    """The point where the estimated eigenvalue count (cumulative weights cnt
    at the pooled Ritz values xs, ascending) reaches m, linear between
    consecutive Ritz values; the end values outside the range."""
    i = int(np.searchsorted(cnt, m, side="left"))
    if i >= len(xs):
        return xs[-1]
    if i == 0:
        return xs[0]
    return xs[i - 1] + (m - cnt[i - 1]) * (xs[i] - xs[i - 1]) / (cnt[i] - cnt[i - 1])


def filter_interval(alpha, beta):
    """Centre c and half-width e of the damped interval [alpha, beta]."""
    return (alpha + beta) / 2.0, (beta - alpha) / 2.0


def convergence_rate(gamma, c, e):
    """|rho| of Eq. (S1): max over +- of |t +- sqrt(t^2 - 1)|, t=(gamma-c)/e.
    Inside the damped interval (|t| <= 1) both roots have modulus 1."""
    t = (gamma - c) / e
    if abs(t) <= 1.0:
        return 1.0
    return abs(t) + math.sqrt(t * t - 1.0)


def chebyshev_filter(H, V, degrees, lower, c, e):
    """Filter each column j of V with the degree-d_j scaled Chebyshev
    polynomial p_d(x) = T_d((x - c)/e) / T_d((lower - c)/e) of H.

    Three-term recurrence (scaled so the component at `lower` stays O(1)):
      sigma_1 = e/(lower - c);  Y_1 = (sigma_1/e)(H Y_0 - c Y_0)
      sigma_{t+1} = 1/(2/sigma_1 - sigma_t)
      Y_{t+1} = (2 sigma_{t+1}/e)(H Y_t - c Y_t) - sigma_t sigma_{t+1} Y_{t-1}
    Degrees are ascending along the columns, so at step t the columns still
    being filtered (d_j > t) are a trailing block; column j's result is
    Y_{d_j}.  Returns (filtered block, number of H*vector products)."""
    degrees = np.asarray(degrees, dtype=np.int64)
    m = V.shape[1]
    if m == 0:
        return V.copy(), 0
    assert np.all(np.diff(degrees) >= 0) and degrees[0] >= 1
    sigma1 = e / (lower - c)
    Yprev = V.copy()
    Y = (sigma1 / e) * (H @ V - c * V)
    matvecs = m
    sigma = sigma1
    for t in range(1, int(degrees[-1])):
        s = int(np.searchsorted(degrees, t, side="right"))  # first d_j > t
        sigma_new = 1.0 / (2.0 / sigma1 - sigma)
        Ya = Y[:, s:]
        Ynew = (2.0 * sigma_new / e) * (H @ Ya - c * Ya) - (sigma * sigma_new) * Yprev[:, s:]
        Yprev[:, s:] = Ya
        Y[:, s:] = Ynew
        matvecs += m - s
        sigma = sigma_new
    return Y, matvecs


def _trsm_right_upper(V, R):
    """V R^{-1} for upper-triangular R: X R = V is R^T X^T = V^T, a triangular
    solve (LAPACK trtrs through scipy, a library primitive)."""
    X = scipy.linalg.solve_triangular(R, np.asarray(V).T, trans="T", lower=False,
                                      check_finite=False)
    return np.asfortranarray(X.T)


def cholqr(V, shift=0.0):
    """One (shifted) Cholesky QR pass: G = V^H V + shift I = R^H R,
    Q = V R^{-1}.  Returns Q, or None if the factorisation fails."""
    G = V.conj().T @ V
    if shift:
        G = G + shift * np.eye(G.shape[0])
    R = cholesky(G)
    if R is None:
        return None
    return _trsm_right_upper(V, R)


def qr(V_locked, V_act):
    """Orthonormalise the filtered block against the locked vectors and
    itself.  Reading (ChASE ran LAPACK Householder QR on the host; the paper
    fixes only that the filtered vectors are orthonormalised):
      1. V -= V_L (V_L^H V), done twice (block classical Gram-Schmidt, CGS2);
      2. each column scaled to unit 2-norm (does not change the span);
      3. shifted Cholesky QR, shift 11 (N m + m(m+1)) u ||V||_F^2 (Fukaya,
         Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SISC 2020);
      4. twice: V -= V_L (V_L^H V) once, then a plain Cholesky QR pass
         (shifted CholeskyQR3, each pass preceded by a projection so that
         rounding in the first projection cannot leave locked directions)."""
    V = V_act.copy()
    has_locked = V_locked is not None and V_locked.shape[1] > 0

    def project(X):
        return X - V_locked @ (V_locked.conj().T @ X) if has_locked else X

    V = project(project(V))
    V = V / np.linalg.norm(V, axis=0)
    N, m = V.shape
    fro2 = float(np.sum(np.abs(V) ** 2))
    shift = 11.0 * (N * m + m * (m + 1)) * U * fro2
    Q = cholqr(V, shift)
    if Q is None:
        raise FloatingPointError("shifted Cholesky QR failed")
    for _ in range(2):
        Q = cholqr(project(Q))
        if Q is None:
            raise FloatingPointError("Cholesky QR failed")
    return Q


def rayleigh_ritz(H, Q):
    """W = H Q; G = Q^H W made exactly Hermitian as (G + G^H)/2; G = Y Theta
    Y^H with Theta ascending; returns (Theta, V = Q Y, HV = W Y)."""
    W = H @ Q
    G = Q.conj().T @ W
    G = (G + G.conj().T) / 2.0
    theta, Y = eigh(G)
    return theta, Q @ Y, W @ Y


def residuals(HV, V, theta, norm_est):
    """r_j = ||H v_j - theta_j v_j||_2 / ||H||_est (reading: relative to the
    Lanczos norm estimate)."""
    return np.linalg.norm(HV - V * theta[None, :], axis=0) / norm_est


def lock_count(resid, tol, locked, nev):
    """Number of newly locked pairs: the longest run of converged pairs
    (r_j <= tol) starting from the lowest unlocked Ritz value, capped so
    that no more than nev pairs are locked in total."""
    n = 0
    while n < len(resid) and locked + n < nev and resid[n] <= tol:
        n += 1
    return n


def degrees(theta, resid, c, e, tol, deg_max):
    """Per-vector filter degree from Eq. (S1): with rho_j the convergence
    ratio of Ritz value theta_j for the interval (c, e), the degree that
    brings residual r_j to tol is ln(r_j/tol)/ln(rho_j).  Reading: ceil,
    at least 2, rounded up to even, at most deg_max; a ratio of 1 (theta_j
    inside the damped interval) gets deg_max."""
    out = np.empty(len(theta), dtype=np.int64)
    for j, (th, r) in enumerate(zip(theta, resid)):
        rho = convergence_rate(th, c, e)
        if rho <= 1.0:
            d = deg_max
        elif r <= tol:
            d = 2
        else:
            d = max(2, int(math.ceil(math.log(r / tol) / math.log(rho))))
        d += d & 1
        out[j] = min(d, deg_max)
    return out


KAPPA_MAX = 1e12


def degree_cap(lower, c, e, kappa_max=KAPPA_MAX):
    """Largest even degree d (at least 2) with |T_d((lower - c)/e)| <=
    kappa_max.  The filtered block's condition number is about
    |T_d((lower - c)/e)| (components at `lower` keep their size, those at
    alpha are divided by it), so the cap keeps the block numerically full
    rank for Cholesky QR.  Returns None when no cap applies."""
    t = abs((lower - c) / e)
    if t <= 1.0:
        return None
    d = int(math.floor(math.acosh(kappa_max) / math.acosh(t)))
    d -= d & 1
    return max(2, d)


def normalize_phase(V):
    """Make the largest-modulus entry of each column (smallest index on
    ties) real and positive."""
    V = V.copy()
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        V[:, j] *= np.conj(V[i, j]) / abs(V[i, j])
    return V


# -------------------------------------------------------------- the solve

def group_degrees(deg, width):
    """Degrees in groups of `width`: with the degrees ascending, the columns
    are taken in groups of `width` from the highest degree down, and every
    degree of a group is raised to the group's largest.  A filter step costs
    the same for any number of columns within one group, so this adds
    filtering (never removes it) at no cost on such hardware.  width <= 0:
    unchanged."""
    deg = np.array(deg, dtype=np.int64, copy=True)
    if width <= 0:
        return deg
    hi = len(deg)
    while hi > 0:
        lo = max(0, hi - width)
        deg[lo:hi] = deg[hi - 1]
        hi = lo
    return deg


def nex_regression(e_cut, e_low, e_high, nex_low, nex_high):
    """Eq. (S2): nex interpolated linearly in the energy cut-off between
    (E_cut-low, nex_low) and (E_cut-high, nex_high)."""
    return nex_low + (nex_high - nex_low) / (e_high - e_low) * (e_cut - e_low)


def damping(gamma, alpha, beta):
    """1/rho of Eq. (S1) for the value gamma with the damped interval
    [alpha, beta]: the factor by which one filter degree shrinks the
    component at gamma relative to the one at the interval's edge."""
    c, e = filter_interval(alpha, beta)
    return 1.0 / convergence_rate(gamma, c, e)


def grown_nex(nex, nev, N, m_max=512):
    """The larger nex of the nex tuner: doubled (and at least 8 more), within
    the search-space limit nev + nex <= min(N, m_max)."""
    return min(max(2 * nex, nex + 8), min(N, m_max) - nev)


NEX_SETTLED = 0.02


def chase(H, nev, nex, tol=1e-10, deg_max=36, deg_init=20, max_iter=50,
          seed=0, V0=None, lanczos_runs=4, lanczos_steps=25, trace=False,
          degree_group=0, nex_damping=0.0):
    """Lowest nev eigenpairs of the Hermitian H by ChASE.

    Lanczos estimate, then per iteration: interval (c, e) from (alpha,
    beta); filter the unlocked columns with their degrees; QR; Rayleigh-
    Ritz; residuals; lock; alpha <- largest Ritz value, lower <- min(lower,
    smallest Ritz value); new degrees; unlocked columns sorted by degree.
    degree_group > 0 raises the degrees in groups (group_degrees) before
    each filter; 0 keeps the degrees of Eq. (S1).
    nex_damping > 0 turns on the nex tuner (reading of the Supplement's nex
    study: the damping 1/rho_nev of the last wanted pair, Eq. (S1) with
    gamma = lambda_nev, sets the convergence rate, and a larger nex lowers
    it).  After each Rayleigh-Ritz from the second on, the damping is
    evaluated with gamma = the nev-th Ritz value and alpha = the largest;
    once two consecutive values differ by at most NEX_SETTLED (the first
    iterations' Ritz values above lambda_nev are still far off) and the value
    exceeds nex_damping, nex grows once to grown_nex.  The new columns are the
    seeded start block's next columns, filtered with deg_max.
    Returns a dict with ascending eigenvalues, eigenvectors (phase-
    normalised), residuals, iteration and matvec counts, and a status
    ("ok" or "noconv")."""
    N = H.shape[0]
    m = nev + nex
    if not (0 < nev and nex >= 0 and m <= N):
        raise ValueError("need 0 < nev, 0 <= nex, nev + nex <= N")
    est = lanczos_bounds(H, m, seed, lanczos_runs, lanczos_steps)
    beta, lower, alpha = est["beta"], est["mu_1"], est["mu_m"]
    norm_est = est["norm_est"]
    V = random_block(seed, STREAM_START, N, m)
    if V0 is not None:
        V0 = np.asarray(V0)
        V[:, :V0.shape[1]] = V0
    deg = np.full(m, deg_init + (deg_init & 1), dtype=np.int64)
    deg = np.minimum(deg, deg_max)
    locked = 0
    lam = np.zeros(m)
    res = np.full(m, np.inf)
    matvecs = min(lanczos_steps, N) * lanczos_runs
    history = []
    it = 0
    status = "noconv"
    damp_prev, grown = None, False
    while it < max_iter:
        it += 1
        c, e = filter_interval(alpha, beta)
        cap = degree_cap(lower, c, e)
        if cap is not None:
            deg = np.minimum(deg, cap)
        deg = group_degrees(deg, degree_group)
        Vf, mv = chebyshev_filter(H, V[:, locked:], deg, lower, c, e)
        matvecs += mv
        locked0 = locked
        Q = qr(V[:, :locked], Vf)
        theta, Vr, HVr = rayleigh_ritz(H, Q)
        matvecs += Q.shape[1]
        r = residuals(HVr, Vr, theta, norm_est)
        nl = lock_count(r, tol, locked, nev)
        V[:, locked:] = Vr
        lam[locked:] = theta
        res[locked:] = r
        if trace:
            history.append(dict(alpha=alpha, beta=beta, c=c, e=e, lower=lower,
                                degrees=deg.copy(), locked=locked,
                                new_locked=nl, theta=theta.copy(), resid=r.copy()))
        locked += nl
        alpha = float(theta[-1])
        lower = min(lower, float(theta[0]))
        if locked >= nev:
            status = "ok"
            break
        c2, e2 = filter_interval(alpha, beta)
        th_u, r_u = theta[nl:], r[nl:]
        d = degrees(th_u, r_u, c2, e2, tol, deg_max)
        perm = np.argsort(d, kind="stable")
        V[:, locked:] = V[:, locked:][:, perm]
        lam[locked:] = th_u[perm]
        res[locked:] = r_u[perm]
        deg = d[perm]
        if nex_damping > 0.0 and not grown and nev - 1 - locked0 >= 0:
            dmp = damping(theta[nev - 1 - locked0], alpha, beta)
            if (damp_prev is not None and abs(dmp - damp_prev) <= NEX_SETTLED
                    and dmp > nex_damping):
                grown = True
                nex2 = grown_nex(nex, nev, N)
                if nex2 > nex:
                    m2 = nev + nex2
                    V = np.concatenate([V, random_block(seed, STREAM_START, N, m2)[:, m:]], axis=1)
                    lam = np.concatenate([lam, np.full(m2 - m, alpha)])
                    res = np.concatenate([res, np.full(m2 - m, np.inf)])
                    deg = np.concatenate([deg, np.full(m2 - m, deg_max, dtype=np.int64)])
                    nex, m = nex2, m2
            damp_prev = dmp
    k = nev
    res_out = res[:k].copy()
    res_out[locked:] = np.inf          # not converged: reported as +inf
    order = np.argsort(lam[:k], kind="stable")
    evals = lam[:k][order]
    evecs = normalize_phase(V[:, :k][:, order])
    resid = res_out[order]
    return dict(evals=evals, evecs=evecs, resid=resid, iters=it,
                matvecs=matvecs, status=status, lanczos=est, history=history,
                nex=nex)
