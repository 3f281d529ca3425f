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


def test_create_rejects_bad_parameters_without_a_gpu(libpath):
    """sxl_create checks its parameters before any CUDA call, so every
    refusal can be checked on the CPU: SXL_E_ARG and no context."""
    from dataclasses import replace

    import numpy as np
    from paper_2303_03529_gb300 import sxl
    from paper_2303_03529_gb300 import workload as wl
    lib = sxl.load_library(libpath)
    w = wl.fe16()

    def code(mp=None, n_atoms=16, cell=None, **kw):
        p = sxl.make_params(mp or w.params, n_atoms, w.cell if cell is None else cell, **kw)
        h = ctypes.c_void_p()
        rc = lib.sxl_create(ctypes.byref(p), None, ctypes.byref(h))
        assert not h.value
        return rc

    E_ARG = -1
    assert code(n_atoms=1) == E_ARG                              # fewer than 2 atoms
    assert code(cell=np.array([3.0, 5.74, 5.74])) == E_ARG       # 1.5 L <= r_cut
    assert code(precision="fp16", foe_steps=41) == E_ARG
    assert code(mp=replace(w.params, kmax=0)) == E_ARG
    assert code(mp=replace(w.params, krylov_rank=0)) == E_ARG
    assert code(mp=replace(w.params, n_elec_per_atom=0.0)) == E_ARG
    assert code(mp=replace(w.params, kT=0.0)) == E_ARG
    h = ctypes.c_void_p()
    assert lib.sxl_batch_create(None, 0, ctypes.byref(h)) == E_ARG
    assert lib.scf_solve_ex(None, None, None, 1e-8, 10, None, None, None, None) == E_ARG
    assert lib.bomd_step(None, 1, None, 1e-8, 10, None, None) == E_ARG
