"""Exact spectral facts of the synthetic Eq. (1) Hamiltonian from its structure.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The synthetic Hamiltonian (Sec. 2, Eq. (1) with the generator's reading) is

    H = D - W + U U^H,

  D = diag(dE)                          transition energies,
  W_IJ = w0 K(d(k,k')) [v=v', c=c'] e^{i(theta_I - theta_J)}
                                        screened direct term, K(d) = 1/(d^2 + 1/2),
  U = sqrt(2) [a_1 .. a_R]              exchange term 2 sum_r a_r a_r^H (rank R).

Ordered by band pair b = (v, c), D - W is block diagonal with Nv*Nc blocks
of size Nk, and block b is Phi_b (D_b - w0 K) Phi_b^H with Phi_b =
diag(e^{i theta}) unitary and K the real symmetric circulant matrix of the
ring.  So the blocks are diagonalised by real symmetric eigensolvers of
size Nk:  D_b - w0 K = Q_b diag(mu_b) Q_b^T.

Two textbook facts then give the eigenvalue count of H below any sigma
without factoring the N x N matrix:
  - Sylvester's law of inertia: congruent Hermitian matrices have the same
    numbers of negative, zero and positive eigenvalues;
  - the Haynsworth inertia additivity of the Schur complement: for the
    bordered matrix M = [[B, U], [U^H, -I_R]],
        In(M) = In(-I_R) + In(B + U U^H) = In(B) + In(-I_R - U^H B^-1 U).
With B = D - W - sigma I, B + U U^H = H - sigma I, so

    #{lambda(H) < sigma} = #{mu < sigma} + #{eig(S(sigma)) < 0} - R,
    S(sigma) = -I_R - sum_i conj(w_i) w_i^T / (mu_i - sigma),

where w_i are the rows of W_b = Q_b^T Phi_b^H U_b over all blocks (an R x R
Hermitian matrix per sigma).  Bisection on this count gives every
eigenvalue of H, in FP64, at any N the generator supports (N = 50000 in
seconds): the eigenvalue oracle at sizes where no dense eigensolver runs.

The same structure gives H V in O(N (log Nk + R)) per column (the circulant
K applied by FFT), which lets the plain oracle ChASE of chase.py run at the
full benchmark sizes: BseOperator.

The block eigensolver and the FFT are library primitives (numpy, scipy); nothing
else is blocked or reordered beyond the formulas above.
"""
import os

import numpy as np
import scipy.fft

from .chase import _model, bse_tables


def ring_kernel(Nk):
    """First column of the circulant K: K(d) = 1/(d^2 + 1/2) with d the
    distance on the periodic ring of Nk k-points."""
    k = np.arange(Nk)
    d = np.minimum(k, Nk - k).astype(np.float64)
    return 1.0 / (d * d + 0.5)


def _params(model):
    md = _model(model)
    return md.w0, md.rank_x


def bse_blocks(seed, Nk, Nv, Nc, model=None):
    """The block decomposition of the synthetic H (module docstring).

    Returns a dict with
      mu  (N,)   eigenvalues of the blocks D_b - w0 K, block after block,
      W   (N, R) rows w_i = (Q_b^T Phi_b^H U_b)_i matching mu,
      R          the exchange rank,
      trace_x    trace(U U^H) (bounds the shift of every eigenvalue)."""
    w0, R = _params(model)
    dE, a, th = bse_tables(seed, Nk, Nv, Nc, model)
    nb = Nv * Nc
    k0 = ring_kernel(Nk)
    idx = np.arange(Nk)
    K = k0[np.abs(idx[:, None] - idx[None, :])]          # symmetric circulant
    U = np.sqrt(2.0) * a                                    # N x R
    mu_all, W_all = [], []
    for b in range(nb):
        rows = idx * nb + b                                 # I = k*Nv*Nc + b
        M = np.diag(dE[rows]) - w0 * K
        mu, Q = np.linalg.eigh(M)
        phase = np.exp(-1j * th[rows])                      # Phi_b^H
        mu_all.append(mu)
        W_all.append(Q.T @ (phase[:, None] * U[rows, :]))
    mu = np.concatenate(mu_all)
    W = np.concatenate(W_all, axis=0) if R > 0 else np.zeros((len(mu), 0), np.complex128)
    return dict(mu=mu, W=W, R=R, trace_x=float(np.sum(np.abs(U) ** 2)))


def eig_count(blocks, sigmas, chunk=256):
    """#{lambda(H) < sigma} for each sigma (Sylvester + Haynsworth)."""
    sigmas = np.atleast_1d(np.asarray(sigmas, dtype=np.float64)).copy()
    mu, W, R = blocks["mu"], blocks["W"], blocks["R"]
    # B must be nonsingular: a sigma equal to a block eigenvalue moves up by
    # ulps until it equals none (the count is then that of the moved sigma)
    mus = np.sort(mu)
    for _ in range(64):
        pos = np.clip(np.searchsorted(mus, sigmas), 0, len(mus) - 1)
        hit = mus[pos] == sigmas
        if not np.any(hit):
            break
        sigmas[hit] = np.nextafter(sigmas[hit], np.inf)
    below = np.searchsorted(mus, sigmas, side="left")   # #{mu < sigma}
    if R == 0:
        return below.astype(np.int64)
    # P_i = conj(w_i) w_i^T, flattened: S(sigma) = -I - sum_i P_i / (mu_i - sigma)
    P = (W.conj()[:, :, None] * W[:, None, :]).reshape(len(mu), R * R)
    out = np.empty(len(sigmas), dtype=np.int64)
    eye = np.eye(R)
    for s0 in range(0, len(sigmas), chunk):
        sg = sigmas[s0:s0 + chunk]
        Dinv = 1.0 / (mu[:, None] - sg[None, :])           # N x s
        T = (P.T @ Dinv).T.reshape(len(sg), R, R)
        S = -eye[None, :, :] - T
        S = 0.5 * (S + np.conj(np.swapaxes(S, 1, 2)))
        neg = np.sum(np.linalg.eigvalsh(S) < 0.0, axis=1)
        out[s0:s0 + chunk] = below[s0:s0 + chunk] + neg - R
    return out


def lowest_eigenvalues(blocks, k, rel=2e-16, max_steps=80):
    """The k smallest eigenvalues of H by bisection on eig_count, all at
    once.  Brackets: lambda_j >= mu_(j) (U U^H is positive semidefinite) and
    lambda_j <= mu_(j) + trace(U U^H) (Weyl), mu_(j) the j-th smallest block
    eigenvalue.  Each bracket is halved until its width is below rel |x| (or
    a few ulps)."""
    mus = np.sort(blocks["mu"])
    lo = mus[:k].copy() - 1e-12 * (1.0 + np.abs(mus[:k]))
    hi = mus[:k] + blocks["trace_x"] + 1e-12 * (1.0 + np.abs(mus[:k]))
    j = np.arange(1, k + 1)
    for _ in range(max_steps):
        mid = 0.5 * (lo + hi)
        cnt = eig_count(blocks, mid)
        up = cnt >= j                     # lambda_j < mid
        hi = np.where(up, mid, hi)
        lo = np.where(up, lo, mid)
        if np.all(hi - lo <= np.maximum(rel * np.abs(hi), 4 * np.spacing(np.abs(hi)))):
            break
    return 0.5 * (lo + hi)


class BseOperator:
    """H of the synthetic model as a linear operator: H @ V for an N x m
    (or N) complex block, from the structure of the module docstring:
    H V = dE * V + U (U^H V) - (block b) Phi_b w0 K Phi_b^H V_b, the
    circulant K applied by FFT along the k-points.  Supports `@` and
    `.shape`, which is all the oracle ChASE (chase.chase) uses of H."""

    def __init__(self, seed, Nk, Nv, Nc, model=None):
        self.w0, self.R = _params(model)
        dE, a, th = bse_tables(seed, Nk, Nv, Nc, model)
        self.Nk, self.nb = Nk, Nv * Nc
        self.N = Nk * self.nb
        self.shape = (self.N, self.N)
        self.dE = dE
        self.U = np.sqrt(2.0) * a
        self.phase = np.exp(1j * th)                        # diag of Phi
        self.k_hat = np.fft.fft(ring_kernel(Nk))            # real, symmetric kernel

    def __matmul__(self, V):
        V = np.asarray(V)
        vec = V.ndim == 1
        X = V.reshape(self.N, -1)
        out = self.dE[:, None] * X
        if self.R > 0:
            out = out + self.U @ (self.U.conj().T @ X)
        # rows of band pair b sit at k*nb + b: view as (Nk, nb, m)
        Y = (self.phase.conj()[:, None] * X).reshape(self.Nk, self.nb, -1)
        nw = os.cpu_count() or 1
        KY = scipy.fft.ifft(self.k_hat[:, None, None] * scipy.fft.fft(Y, axis=0, workers=nw),
                            axis=0, workers=nw)
        out = out - self.w0 * (self.phase[:, None] * KY.reshape(self.N, -1))
        return out[:, 0] if vec else out
