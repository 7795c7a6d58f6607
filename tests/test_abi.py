"""C ABI checks that need no GPU: the library builds and loads, exports every
entry point include/nrsense.h declares, and the ctypes structures match the C
layout (checked with a small C program compiled by gcc against the header)."""

import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nrsense.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    # function-pointer typedefs declare types, not entry points
    txt = re.sub(r"typedef\s+nrsense_status\s*\(\*\s*\w+\)\s*\([^)]*\)\s*;", "", txt)
    return sorted(set(re.findall(r"\b(nrsense_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2501_16713_gb300 import nrsense
    return nrsense.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "nrsense_plan_create" in names and "nrsense_apply_normal" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2501_16713_gb300 import nrsense
    assert set(_declared()) == set(nrsense.exported_symbols())


def test_status_strings(lib):
    lib.nrsense_status_string.restype = ctypes.c_char_p
    assert lib.nrsense_status_string(0) == b"ok"
    assert lib.nrsense_status_string(-1) == b"invalid argument"
    assert lib.nrsense_status_string(-123) == b"unknown status"


def test_null_arguments_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    assert lib.nrsense_plan_create(None, None, None, None, None, None, ctypes.byref(h)) == -1
    assert lib.nrsense_apply_forward(None, None, None, None) == -1
    assert lib.nrsense_plan_destroy(None) == 0


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_struct_layout_matches_header(tmp_path):
    from paper_2501_16713_gb300 import nrsense
    src = tmp_path / "layout.c"
    src.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu\\n", sizeof(nrsense_desc), offsetof(nrsense_desc, kb_beta),
         offsetof(nrsense_desc, n_phases), offsetof(nrsense_desc, flags), sizeof(nrsense_c64));
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(nrsense_info), offsetof(nrsense_info, kb_beta),
         offsetof(nrsense_info, tile), offsetof(nrsense_info, n_tiles),
         offsetof(nrsense_info, device_bytes), offsetof(nrsense_info, phase_chunk));
  printf("%zu\\n", offsetof(nrsense_desc, phase_chunk));
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    d = [int(v) for v in out[0].split()]
    i = [int(v) for v in out[1].split()]
    D, I = nrsense.Desc, nrsense.Info
    assert d == [ctypes.sizeof(D), D.kb_beta.offset, D.n_phases.offset, D.flags.offset, 8]
    assert i == [ctypes.sizeof(I), I.kb_beta.offset, I.tile.offset, I.n_tiles.offset,
                 I.device_bytes.offset, I.phase_chunk.offset]
    assert int(out[2]) == D.phase_chunk.offset


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_every_mirrored_field_matches_header(tmp_path):
    """Each ctypes mirror of a header struct: size and the offset of every
    field, as the C compiler lays them out (fields appended to the header
    structs must be appended to the mirrors in the same order)."""
    from paper_2501_16713_gb300 import nrsense
    pairs = [("nrsense_desc", nrsense.Desc), ("nrsense_info", nrsense.Info),
             ("nrsense_tuning", nrsense.Tuning)]
    lines = []
    for cname, cls in pairs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "fields.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n"
                   f'#include "{HEADER}"\nint main(void) {{\n' + "\n".join(lines) +
                   "\n  return 0;\n}\n")
    exe = tmp_path / "fields"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    got = [int(v) for v in
           subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for _, cls in pairs:
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f, _ in cls._fields_]
    assert got == want


def test_host_symmetric_eigen_matches_numpy(lib):
    """The Jacobi eigen-solver behind nrsense_deflation_from_solve (host only)
    against numpy's on a CG-Lanczos-shaped tridiagonal and on a dense matrix:
    eigenvalues, orthonormal eigenvectors, A V = V diag(vals)."""
    import numpy as np
    from paper_2501_16713_gb300 import nrsense
    rng = np.random.default_rng(181)
    m = 40
    T = np.diag(rng.uniform(0.5, 3.0, m)) - np.diag(rng.uniform(0.1, 1.0, m - 1), 1)
    T = T + np.triu(T, 1).T
    X = rng.standard_normal((12, 12))
    for A in (T, X + X.T):
        vals, vecs = nrsense.symmetric_eigen(A)
        ref = np.linalg.eigvalsh(A)
        scale = np.abs(ref).max()
        assert np.allclose(vals, ref, rtol=0, atol=1e-12 * scale)
        assert np.allclose(vecs.T @ vecs, np.eye(A.shape[0]), atol=1e-12)
        assert np.allclose(A @ vecs, vecs * vals, atol=1e-11 * scale)
    with pytest.raises(nrsense.NrsenseError):
        nrsense.symmetric_eigen(np.zeros((0, 0)))
