"""Host-side checks of libpff (no GPU): the C-ABI library loads, exports every
symbol that include/pff.h declares, and its quadtree / node / constraint
construction agrees with the independent oracle mesh."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "pff.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(pff_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_03265_gb300 import _lib
    return _lib.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2404_03265_gb300 import _lib
    assert set(names) <= set(_lib.exported_names()) | {"pff_params_default"}


def declared_prototypes():
    """name -> number of parameters of every function prototype in include/pff.h."""
    txt = open(os.path.join(ROOT, "include", "pff.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(pff_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", txt):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_header():
    """Every ctypes signature of the binding passes as many arguments as the
    header's prototype of the same function declares."""
    from paper_2404_03265_gb300 import _lib
    protos = declared_prototypes()
    for name, _, args in _lib._SIGS:
        assert name in protos, name
        assert len(args) == protos[name], (name, len(args), protos[name])


def test_binding_constants_match_header():
    """Every PFF_* integer constant the binding names has the header's value (a
    #define or an enumerator)."""
    from paper_2404_03265_gb300 import _lib
    txt = open(os.path.join(ROOT, "include", "pff.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(PFF_[A-Z0-9_]+)\s+(-?\d+)\b", txt)}
    defs.update({k: int(v) for k, v in re.findall(r"\b(PFF_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt)})
    named = [k for k in dir(_lib) if k.startswith("PFF_") and isinstance(getattr(_lib, k), int)]
    assert {"PFF_PHIT_PREVIOUS", "PFF_PHIT_EXTRAPOLATED", "PFF_F32"} <= set(named)
    for k in named:
        assert k in defs, k
        assert getattr(_lib, k) == defs[k], (k, getattr(_lib, k), defs[k])


@pytest.mark.parametrize("name,k", [("tiny", 1), ("small", 1), ("tiny", 2), ("small", 2), ("band4_2_4", 1),
                                    ("band4_2_4", 2)])
def test_mesh_matches_oracle(name, k):
    from harness import Pair
    P = Pair(name, k)
    om, lm = P.om, P.lm
    inf = lm.info
    assert inf["n_nodes"] == om.nn
    assert inf["n_leaf_cells"] == len(om.cells)
    assert inf["n_hanging"] == len(om.hanging)
    assert inf["x_max"] == om.Xmax and inf["y_max"] == om.Ymax
    assert abs(inf["h_min"] - om.h_min_diag()) < 1e-15
    F = P.slot_F[P.slots]
    # hanging and boundary flags agree node by node
    assert np.array_equal((F & 4) != 0, om.is_hanging[P.onode])
    assert np.array_equal((F & 2) != 0, om.dirichlet[P.onode])
    # leaf cells in canonical order
    assert np.array_equal(lm.leaf_cells(), om.cells.astype(np.int32))


def test_refine_marked_and_errors():
    from paper_2404_03265_gb300 import Mesh, PffError
    m = Mesh(-1, 1, -1, 1, 2, 2)
    m.refine_global(1)
    n = m.n_leaves()
    marks = np.zeros(n, np.uint8)
    marks[0] = 1
    m.refine_marked(marks)
    with pytest.raises(PffError):
        m.refine_marked(np.zeros(3, np.uint8))
    m.finalize(1)
    with pytest.raises(PffError):
        m.refine_global(1)
    with pytest.raises(PffError):
        Mesh(1, -1, 0, 1, 1, 1)


@pytest.mark.parametrize("py_name,c_name", [("MeshInfo", "pff_mesh_info"), ("Params", "pff_params"),
                                            ("SolveInfo", "pff_solve_info"), ("NewtonOpts", "pff_newton_opts")])
def test_binding_struct_layouts_match_header(py_name, c_name, tmp_path):
    """Every ctypes structure of the binding has the size and field offsets that
    a C compiler gives the struct of the same name in include/pff.h."""
    import ctypes
    import shutil
    import subprocess
    from paper_2404_03265_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cls = getattr(_lib, py_name)
    fields = [f[0] for f in cls._fields_]
    src = ['#include <stddef.h>', '#include <stdio.h>', '#include "pff.h"', "int main(void) {",
           '  printf("%%zu\\n", sizeof(%s));' % c_name]
    src += ['  printf("%%zu\\n", offsetof(%s, %s));' % (c_name, f) for f in fields]
    src += ["  return 0;", "}"]
    (tmp_path / "layout.c").write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(tmp_path / "layout.c"), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(cls), (c_name, got[0], ctypes.sizeof(cls))
    for f, off in zip(fields, got[1:]):
        assert getattr(cls, f).offset == off, (c_name, f, off, getattr(cls, f).offset)
