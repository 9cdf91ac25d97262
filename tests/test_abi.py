"""The C ABI library builds, loads, and exports every function that
include/hcgrid.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "hcgrid.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hcg_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_calls():
    names = declared()
    for must in ["hcg_create", "hcg_destroy", "hcg_set_kernel", "hcg_set_grid", "hcg_load_samples", "hcg_grid",
                 "hcg_fetch", "hcg_batch_create", "hcg_batch_add", "hcg_batch_grid", "hcg_set_tuning",
                 "hcg_debug_pix", "hcg_debug_neighbours", "hcg_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2012_13173_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    import paper_2012_13173_gb300 as H
    lib = H.load()
    names = set(declared()) - {"hcg_last_error"}
    assert names <= set(H._SIGS), sorted(names - set(H._SIGS))
    assert lib.hcg_last_error() is not None
