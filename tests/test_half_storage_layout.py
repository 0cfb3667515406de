"""Host-side checks of the half-storage layout of H's tensor-core slices
(no GPU): the index arithmetic the slicing kernels and the product kernel's
producer use, restated here and run on small matrices, and the bound of the
symmetric scaling that lets one exponent serve every row.

Layout: tile (b, kc) of 128 rows x 64 columns (row tile b, K chunk kc) is
stored iff kc <= 2b + 1, at slot b (b + 1) + kc of each part.  Row tile br
reads chunk kc > 2br + 1 as the conjugate transpose of rows 64 (kc mod 2) ..
+ 63 of the stored tiles (kc / 2, 2 br) and (kc / 2, 2 br + 1)."""
import numpy as np
import pytest

BM, KC = 128, 64


def slot(b, kc):
    return b * (b + 1) + kc


def store(S):
    """The stored tiles of the Hermitian S (Np x Np, Np = 128 T)."""
    T = S.shape[0] // BM
    tiles = np.zeros((T * (T + 1), BM, KC), dtype=S.dtype)
    for b in range(T):
        for kc in range(2 * b + 2):
            tiles[slot(b, kc)] = S[b * BM:(b + 1) * BM, kc * KC:(kc + 1) * KC]
    return tiles


def a_tile(tiles, br, kc):
    """The 128 x 64 A tile of row tile br and chunk kc, as the producer loads
    it: one stored tile, or (above the stored triangle) two 64-row boxes read
    transposed and conjugated."""
    if kc <= 2 * br + 1:
        return tiles[slot(br, kc)]
    bc, y = kc // 2, 64 * (kc % 2)
    box0 = tiles[slot(bc, 2 * br)][y:y + 64]        # rows c of chunk kc, columns 128 br + 0..63
    box1 = tiles[slot(bc, 2 * br + 1)][y:y + 64]    # columns 128 br + 64..127
    return np.concatenate([box0, box1], axis=1).T.conj()


@pytest.mark.parametrize("T", [1, 2, 3, 7])
def test_slots_enumerate_the_lower_tiles_once(T):
    seen = sorted(slot(b, kc) for b in range(T) for kc in range(2 * b + 2))
    assert seen == list(range(T * (T + 1)))


@pytest.mark.parametrize("T,seed", [(1, 0), (2, 1), (3, 2), (5, 3)])
def test_every_a_tile_is_the_hermitian_matrix(T, seed):
    rng = np.random.default_rng(seed)
    n = BM * T
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    S = A + A.conj().T
    tiles = store(S)
    for br in range(T):
        for kc in range(2 * T):
            got = a_tile(tiles, br, kc)
            assert np.array_equal(got, S[br * BM:(br + 1) * BM, kc * KC:(kc + 1) * KC]), (br, kc)
            if kc > 2 * br + 1:                      # the mirror tiles exist and are stored
                assert kc // 2 > br and 2 * br + 1 <= 2 * (kc // 2) + 1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_symmetric_scaling_bound(seed):
    """t_i = sqrt(M_i)(1 + 2^-20), M_i = max_k max(|Re H_ik|, |Im H_ik|): every
    entry of S = T^-1 H T^-1 is below 1 in both parts (so one exponent, 0,
    serves all rows), also for rows of very different size and a zero row."""
    rng = np.random.default_rng(seed)
    n = 300
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    d = np.logspace(-8, 8, n)
    X = d[:, None] * (A + A.conj().T) * d[None, :]
    H = np.tril(X, -1)                               # exactly Hermitian: mirrored,
    H = H + H.conj().T + np.diag(X.diagonal().real)  # with a real diagonal
    H[7, :] = 0
    H[:, 7] = 0
    M = np.maximum(np.abs(H.real), np.abs(H.imag)).max(axis=1)
    t = np.where(M > 0, np.sqrt(M) * (1 + 2.0 ** -20), 1.0)
    s = 1.0 / t
    S = H * (s[:, None] * s[None, :])
    assert np.max(np.abs(S.real)) < 1 and np.max(np.abs(S.imag)) < 1
    assert np.array_equal(S, S.conj().T)             # Hermitian bit for bit
