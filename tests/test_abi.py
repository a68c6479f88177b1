"""The C-ABI library builds, loads without a GPU, and exports every function
that include/d2.h declares; the binding rejects bad arguments before any call."""
import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "d2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    names = []
    for stmt in src.split(";"):
        stmt = " ".join(stmt.split())
        if "typedef" in stmt or "#" in stmt or "{" in stmt or "}" in stmt:
            stmt = stmt.split("}")[-1]
        m = re.match(r"^(?:extern\s+\"C\"\s*)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", stmt.strip())
        if m and "typedef" not in stmt:
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1510_00012_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("d2_cost", "badmm_barycenter", "d2_assign", "d2_cluster", "d2_create", "d2_destroy",
                 "d2_merge_init", "d2_prune_train", "d2_prune_loss_grad"):
        assert must in names, names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(libpath):
    import paper_1510_00012_gb300 as d2
    names = set(declared_functions())
    assert names <= set(d2._SIGS), names - set(d2._SIGS)


def test_binding_rejects_host_tensors(libpath):
    import paper_1510_00012_gb300 as d2
    with pytest.raises((ValueError, TypeError)):
        d2.DeviceBags(torch.tensor([0, 2]), torch.tensor([0.5, 0.5]), 1, supp=torch.zeros(2, 1))
    with pytest.raises(TypeError):
        d2._need(torch.zeros(3, dtype=torch.float64), torch.float32, "x")
