"""CPU checks of the C-ABI library: it loads without a GPU and exports every
entry point that include/*.h declares; the binding's struct matches the
header's field list."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\(", txt, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2303_03529_gb300 import build
    path = build.build()
    assert os.path.exists(path)
    return path


def test_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared()
    assert "sxl_create" in names and "xlbomd_step" in names and "scf_solve" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(libpath):
    from paper_2303_03529_gb300 import sxl
    names = _declared()
    assert set(names) <= set(sxl.EXPORTS), set(names) - set(sxl.EXPORTS)
    sxl.load_library(libpath)


def test_params_struct_matches_header():
    from paper_2303_03529_gb300 import sxl
    txt = open(os.path.join(ROOT, "include", "sxl.h")).read()
    body = txt[txt.index("typedef struct {"):txt.index("} sxl_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.replace("typedef struct {", "").strip()
        if not decl:
            continue
        parts = decl.split(None, 1)
        for item in parts[1].split(","):
            fields.append(item.strip().split("[")[0])
    assert fields == [f for f, _ in sxl.Params._fields_]


def test_scf_opts_struct_matches_header():
    from paper_2303_03529_gb300 import sxl
    txt = open(os.path.join(ROOT, "include", "sxl.h")).read()
    body = txt[txt.rindex("typedef struct {", 0, txt.index("} sxl_scf_opts;")):txt.index("} sxl_scf_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S).replace("typedef struct {", "")
    fields = [d.split()[-1] for d in body.split(";") if d.strip()]
    assert fields == [f for f, _ in sxl.ScfOpts._fields_]
    assert sxl.MIXERS == {"kernel": 0, "linear": 1, "diis": 2}
