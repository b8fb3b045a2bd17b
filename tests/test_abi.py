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


def test_every_kernel_waits_for_its_predecessor_first():
    # Kernels may be launched with programmatic dependent launch: each one must
    # wait for the previous kernel (pdl_enter) before it touches memory.
    src = os.path.join(ROOT, "paper_1902_00088_gb300", "csrc")
    n = 0
    for f in sorted(os.listdir(src)):
        if not f.endswith((".cu", ".cuh")):
            continue
        txt = open(os.path.join(src, f)).read()
        for m in re.finditer(r"__global__", txt):
            i = m.end()
            # end of the parameter list: the first ')' closing the '(' after the kernel name
            j = txt.index("(", i)
            while txt[i:j].rstrip().endswith("__launch_bounds__"):
                depth, k = 0, j
                while True:
                    depth += {"(": 1, ")": -1}.get(txt[k], 0)
                    if depth == 0:
                        break
                    k += 1
                i, j = k + 1, txt.index("(", k + 1)
            depth, k = 0, j
            while True:
                depth += {"(": 1, ")": -1}.get(txt[k], 0)
                if depth == 0:
                    break
                k += 1
            rest = txt[k + 1:].lstrip()
            if rest.startswith(";"):
                continue  # declaration
            assert rest.startswith("{"), (f, txt[m.start():m.start() + 80])
            body = rest[1:].lstrip()
            assert body.startswith("pdl_enter();"), (f, txt[m.start():m.start() + 80])
            n += 1
    assert n > 40


def test_missing_library_fails_loudly(tmp_path):
    # No CPU fallback: without the built library the binding raises instead of
    # running anything else.
    import paper_1902_00088_gb300 as m
    saved, m._lib = m._lib, None  # the loaded library is cached per process
    try:
        with pytest.raises(ImportError):
            m.load_library(str(tmp_path / "absent" / "libmr.so"))
    finally:
        m._lib = saved
