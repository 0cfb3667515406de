"""The allocation-free Gram entry point (chase_gram_noalloc), called through
the C ABI, against the regular chase_gram.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test.  It builds everything it needs
itself, so it also passes alone in a fresh process."""
import numpy as np
import pytest

from inputs import block

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2006_08498_gb300 as pkg  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).cuda().T


def test_gram_noalloc_matches_gram_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_08498_gb300 import build
    build.build()
    K, m1, m2 = 20000, 140, 140
    A, B = _dev(block(K, m1, 21)), _dev(block(K, m2, 22))
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    bound = np.abs(Ah).T @ np.abs(Bh)
    with pkg.Context(0) as ctx:
        ref = ctx.gram(A, B).cpu().numpy()
    for call in range(2):                        # the shared array keeps old contents
        G = pkg.colmajor_empty(m1, m2, device=A.device)
        G.fill_(float("nan"))
        assert pkg.gram_noalloc(A, B, G) == pkg.BSE_OK
        torch.cuda.synchronize()
        got = G.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * bound), "call %d" % call
    # a different shape right after, then the first one again
    C = _dev(block(K, 7, 23))
    G2 = pkg.colmajor_empty(m1, 7, device=A.device)
    assert pkg.gram_noalloc(A, C, G2) == pkg.BSE_OK
    torch.cuda.synchronize()
    ref2 = Ah.conj().T @ C.cpu().numpy()
    assert np.all(np.abs(G2.cpu().numpy() - ref2) <= 1e-12 * (np.abs(Ah).T @ np.abs(C.cpu().numpy())))


def test_gram_noalloc_self_product_and_side_stream():
    """A^H A with the same pointer for both operands (the upper-tile path of
    the Gram kernel and its mirrored reduction, the Cholesky QR use) at an
    odd width, against chase_gram and numpy, twice; then one call on a side
    stream."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_08498_gb300 import build
    build.build()
    K, m = 5001, 137
    A = _dev(block(K, m, 31))
    Ah = A.cpu().numpy()
    ref_np = Ah.conj().T @ Ah
    bound = np.abs(Ah).T @ np.abs(Ah)
    with pkg.Context(0) as ctx:
        ref = ctx.gram(A, A).cpu().numpy()
    assert np.all(np.abs(ref - ref_np) <= 1e-12 * bound)
    for call in range(2):
        G = pkg.colmajor_empty(m, m, device=A.device)
        G.fill_(float("nan"))
        assert pkg.gram_noalloc(A, A, G) == pkg.BSE_OK
        torch.cuda.synchronize()
        got = G.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * bound), "call %d" % call
        assert np.all(np.abs(got - ref_np) <= 1e-12 * bound), "call %d" % call
    side = torch.cuda.Stream(device=A.device)
    side.wait_stream(torch.cuda.current_stream(A.device))
    G = pkg.colmajor_empty(m, m, device=A.device)
    with torch.cuda.stream(side):
        G.fill_(float("nan"))
        assert pkg.gram_noalloc(A, A, G, stream=side) == pkg.BSE_OK
    side.synchronize()
    assert np.all(np.abs(G.cpu().numpy() - ref) <= 1e-12 * bound)


def test_gram_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A = torch.zeros((513, 600), dtype=torch.complex128, device="cuda").T   # 600 x 513
    G = pkg.colmajor_empty(513, 513, device=A.device)
    assert pkg.gram_noalloc(A, A, G) == pkg.BSE_EINVAL
