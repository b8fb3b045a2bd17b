"""The C-ABI library builds, loads and exports every entry point of include/mr.h
(no compute call: these run without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "mr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mr_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1902_00088_gb300 import build as b
    b.build()
    import paper_1902_00088_gb300 as m
    return m.load_library()


def test_header_declares_the_boundary():
    syms = header_symbols()
    for name in ("mr_init_tree", "mr_set_rhs", "mr_rk_step", "mr_sync_ghosts", "mr_adapt",
                 "mr_get_blocks", "mr_step", "mr_create", "mr_destroy"):
        assert name in syms


def test_library_exports_every_header_symbol(lib):
    missing = [s for s in header_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_signatures_cover_header(lib):
    import paper_1902_00088_gb300 as m
    assert set(header_symbols()) == set(m.SIGNATURES)


def test_relation_counts_without_device(lib):
    # Sec. 2.2: 16 relations in 2D, 74 in 3D (pure host function)
    assert lib.mr_num_relations(2) == 16 and lib.mr_num_relations(3) == 74
