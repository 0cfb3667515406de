"""The boundary from plain C: tests/c_abi_solve.c, compiled with a C compiler
against include/bsechase.h and linked with the CUDA runtime and
libbsechase.so, solves the N = 2000 synthetic Hamiltonian through
chase_solve and chase_solve_bse (half storage); its eigenvalues match the
dense oracle's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import paper_2006_08498_gb300 as pkg

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def test_c_program_solves_through_the_abi(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    from paper_2006_08498_gb300 import build
    build.build()
    libdir = os.path.dirname(pkg.library_path())
    exe = str(tmp_path / "c_abi_solve")
    r = subprocess.run([cc, "-std=c99", "-O2", "-Wall", "-Werror",
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
                        os.path.join(ROOT, "tests", "c_abi_solve.c"), "-o", exe,
                        "-L", libdir, "-lbsechase", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
                        "-Wl,-rpath," + libdir, "-Wl,-rpath," + os.path.join(CUDA, "lib64")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    nev, nex = 40, 20
    out = subprocess.run([exe, "125", str(nev), str(nex)], capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.split("\n")
    w, _ = oracle.eigh(oracle.build_h(0, 125, 4, 4), 0)
    for k, name in enumerate(("solve", "solve_bse")):
        head = lines[k * (nev + 1)].split()
        assert head[0] == name and int(head[1]) == pkg.BSE_OK
        vals = np.array([[float(x) for x in ln.split()] for ln in
                         lines[k * (nev + 1) + 1:(k + 1) * (nev + 1)]])
        assert np.max(vals[:, 1]) <= 1e-10
        assert np.max(np.abs(vals[:, 0] - w[:nev]) / np.abs(w[:nev])) <= 1e-10
