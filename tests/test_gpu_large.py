"""N = 100000 on one GPU: the synthetic Eq. (1) Hamiltonian solved without
storing it, on the half-storage slices of its lower triangle (12 N^2 bytes for
all of H), against its exact eigenvalues from the structured oracle
(tests/golden/bse_exact_nk6250.txt, written by make_bse_exact.py)."""
import numpy as np
import pytest
import torch

from conftest import golden
import paper_2006_08498_gb300 as pkg

pytestmark = pytest.mark.gpu


def test_solve_n100000_without_h_on_half_storage():
    """nev = 200, nex = 80, tol 1e-10, degree groups of 48: every eigenvalue
    within 1e-10 of the exact one (so none below lambda_200 was missed),
    residuals within the tolerance, orthonormal eigenvectors."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_08498_gb300 import build
    build.build()
    torch.cuda.empty_cache()
    lam = np.array([float(r[0]) for r in golden("bse_exact_nk6250.txt")])
    nev, nex = 200, 80
    with pkg.Context(0) as ctx:
        ev, Vd, r, st = ctx.solve_bse(0, 6250, 4, 4, nev, nex, tol=1e-10, deg_max=36,
                                      degree_group=48, half_storage=True)
        assert np.all(np.diff(ev) >= 0) and np.max(r) <= 1e-10
        assert np.max(np.abs(ev - lam[:nev]) / np.abs(lam[:nev])) <= 1e-10
        assert lam[nev] > ev[-1]
        G = ctx.gram(Vd, Vd)
        eye = torch.eye(nev, dtype=torch.complex128, device=G.device)
        assert torch.linalg.norm(G - eye).item() <= 1e-11
        assert st["iters"] <= 20
