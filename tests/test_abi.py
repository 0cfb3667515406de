"""The C ABI library builds, loads and exports every symbol its header
declares (no GPU needed: no compute calls are made)."""
import ctypes
import os
import re

import pytest

import paper_2006_08498_gb300 as pkg
from paper_2006_08498_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            if not m.group(0).lstrip().startswith(("typedef", "#")):
                names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return pkg.load()


def test_header_declares_expected_entry_points():
    names = declared_functions()
    assert set(names) == set(pkg.ABI_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(pkg.library_path())
    for name in declared_functions():
        assert hasattr(raw, name), name


def test_strerror_and_dim(lib):
    assert lib.bsechase_strerror(0) == b"success"
    assert lib.bsechase_strerror(-3) == b"not converged"
    assert lib.bse_dim(125, 4, 4) == 2000
    assert lib.bse_dim(3125, 4, 4) == 50000
    assert lib.bse_dim(0, 4, 4) == -1


def test_null_context_is_rejected(lib):
    assert lib.bse_build_hamiltonian(None, 0, 1, 1, 1, None, None, 1) == pkg.BSE_EINVAL
    assert lib.chase_solve(None, None, 1, 1, 1, 0, 1e-10, 36, 0, None, None, None, 1,
                           None, None) == pkg.BSE_EINVAL
    lib.bsechase_destroy(None)  # ignored


def test_enum_values_match_binding():
    """The status and precision values of the header are the binding's;
    precision 2 is CHASE_MIXED_BF16X3 and native FP64 is 3."""
    src = open(os.path.join(ROOT, "include", "bsechase.h")).read()
    vals = {m.group(1): int(m.group(2))
            for m in re.finditer(r"\b((?:BSE|CHASE)_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    for name, v in vals.items():
        assert getattr(pkg, name) == v, name
    assert vals["CHASE_MIXED_BF16X3"] == 2 and vals["CHASE_FP64_DFMA"] == 3


_CTYPES = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
           "double": ctypes.c_double}


def header_structs():
    """Field names and C types of every `typedef struct { ... } name;` of the
    header, in declaration order (comments removed; `T a, b;` gives two)."""
    src = open(os.path.join(ROOT, "include", "bsechase.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"typedef struct \{(.*?)\}\s*(\w+);", src, flags=re.S):
        fields = []
        for decl in m.group(1).split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            mt = re.match(r"((?:const )?[A-Za-z_]\w*(?: \*|\*)*)\s*(.*)", decl)
            ctype, names = mt.group(1), mt.group(2)
            for nm in names.split(","):
                nm = nm.strip()
                ptr = ctype.endswith("*") or nm.startswith("*")
                fields.append((nm.lstrip("*").strip(), "ptr" if ptr else ctype.split()[-1]))
        out[m.group(2)] = fields
    return out


@pytest.mark.parametrize("cname,pyname", [("bse_model", "Model"), ("chase_opts", "Opts"),
                                          ("chase_stats", "Stats"), ("chase_request", "Request"),
                                          ("chase_result", "Result")])
def test_struct_layouts_match_binding(cname, pyname):
    """The ctypes structures of the binding declare the header's fields in the
    header's order with matching types (appended fields included)."""
    hdr = header_structs()[cname]
    py = getattr(pkg, pyname)._fields_
    assert [n for n, _ in hdr] == [n for n, _ in py]
    for (n, t), (_, pt) in zip(hdr, py):
        if t == "ptr":
            assert pt is ctypes.c_void_p or hasattr(pt, "contents") or pt is ctypes.c_char_p, n
        elif t in _CTYPES:
            assert ctypes.sizeof(pt) == ctypes.sizeof(_CTYPES[t]) and pt is _CTYPES[t], n
        else:                                            # a nested struct
            assert issubclass(pt, ctypes.Structure), n


def test_argument_checks_before_any_device_call(lib):
    """Entry points added later reject bad arguments without touching a GPU."""
    p = ctypes.c_void_p()
    assert lib.bsechase_host_alloc(None, 16) == pkg.BSE_EINVAL
    assert lib.bsechase_host_alloc(ctypes.byref(p), 0) == pkg.BSE_EINVAL
    assert lib.bsechase_host_free(None) == pkg.BSE_OK
    assert lib.chase_hemm_slices(None, None, 1, 1, None, 1, 1, None, 1, 6, 0) == pkg.BSE_EINVAL
    assert lib.chase_solve_bse(None, 0, 1, 1, 1, None, 1, 0, 1e-10, 36, 0, None, None, None, 1,
                               None, None) == pkg.BSE_EINVAL


def test_header_compiles_as_c99(tmp_path):
    """The boundary is a C ABI: the header compiles as plain C99, warnings
    as errors."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "bsechase.h"\nint main(void) { chase_stats s; chase_opts o; '
                   'chase_request r; (void)s; (void)o; (void)r; return 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o",
                        str(tmp_path / "use_header.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
