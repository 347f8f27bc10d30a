"""The C-ABI library builds, loads and exports every symbol include/gbqr.h
declares; host-side argument checks that need no GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbqr.h")


def declared_functions(path=HEADER):
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"GBQR_API\s+[\w\s\*]+?\b(gbqr_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_1805_05278_gb300 as gb
    gb.build()
    return gb.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gbqr_create", "gbqr_destroy", "gbqr_factor", "gbqr_apply_qt", "gbqr_apply_q",
                     "gbqr_form_q", "gbqr_ls_solve", "gbqr_workspace_bytes", "gbqr_strerror", "gbqr_sync"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = []
    for name in declared_functions():
        try:
            getattr(lib, name)
        except AttributeError:
            missing.append(name)
    assert not missing, missing


def test_binding_covers_the_header(lib):
    import paper_1805_05278_gb300 as gb
    assert set(declared_functions()) == set(gb.SIGNATURES)


def test_strerror(lib):
    import paper_1805_05278_gb300 as gb
    assert gb.gbqr_strerror(0) == b"ok"
    assert gb.gbqr_strerror(1) == b"invalid argument"
    assert gb.gbqr_strerror(99) == b"unknown status"


def test_workspace_query(lib):
    import paper_1805_05278_gb300 as gb
    assert gb.gbqr_workspace_bytes(10, 20, gb.GBQR_T_FULL, None) > 0           # wide (Section 2.1)
    assert gb.gbqr_workspace_bytes(-1, 0, gb.GBQR_T_FULL, None) == 0
    assert gb.gbqr_workspace_bytes(100, 10, 7, None) == 0                     # bad layout
    bad = gb.opts(cutoff_b=65)
    assert gb.gbqr_workspace_bytes(100, 10, gb.GBQR_T_PANEL, ctypes.byref(bad)) == 0
    small = gb.gbqr_workspace_bytes(1024, 128, gb.GBQR_T_PANEL, None)
    big = gb.gbqr_workspace_bytes(8192, 8192, gb.GBQR_T_PANEL, None)
    assert 0 < small < big
    # the square 8192 workspace stays a small multiple of the matrix itself
    assert big < 4 * 8192 * 8192 * 8


def test_fanout_range(lib):
    """TSQR fan-out: 0 (the planner's choice) or 2..16; anything else is an
    invalid option.  Any valid fan-out, the widest cutoff included, gets a
    workspace: the planner bounds it over every fan-out it may pick."""
    import paper_1805_05278_gb300 as gb
    for k in (0, 2, 3, 8, 13, 16):
        for b in (16, 64):
            o = gb.opts(fanout=k, cutoff_b=b)
            assert gb.gbqr_workspace_bytes(32768, 2048, gb.GBQR_T_PANEL, ctypes.byref(o)) > 0, (k, b)
    for k in (1, 17, -1):
        o = gb.opts(fanout=k)
        assert gb.gbqr_workspace_bytes(32768, 2048, gb.GBQR_T_PANEL, ctypes.byref(o)) == 0, k
    # the bound over every fan-out covers the adaptive and the fixed choices
    w0 = gb.gbqr_workspace_bytes(32768, 2048, gb.GBQR_T_PANEL, ctypes.byref(gb.opts(fanout=0)))
    w16 = gb.gbqr_workspace_bytes(32768, 2048, gb.GBQR_T_PANEL, ctypes.byref(gb.opts(fanout=16)))
    assert w0 == w16


def test_default_panel(lib):
    import paper_1805_05278_gb300 as gb
    assert gb.gbqr_default_panel_nb(1000, 77) == 77
    assert gb.gbqr_default_panel_nb(8192, 8192) >= 16


def test_null_and_invalid_arguments_without_gpu(lib):
    import paper_1805_05278_gb300 as gb
    assert gb.gbqr_create(None, 0, None) == gb.GBQR_EINVAL
    assert gb.gbqr_destroy(None) == gb.GBQR_EINVAL
    assert gb.gbqr_factor(None, 4, 2, None, 4, None, 2, 0, None) == gb.GBQR_EINVAL
    assert gb.gbqr_sync(None, None) == gb.GBQR_EINVAL
    assert gb.gbqr_autotune(None, 100, 10, 1, 0, 1.0, None, None) == gb.GBQR_EINVAL
    assert gb.gbqr_autotune_batched(None, 1, None, None, 0, 1.0, None, None) == gb.GBQR_EINVAL
    assert gb.gbqr_tuned_lookup(None, 0, 100, 10, 1, 0, None) == gb.GBQR_EINVAL


def test_create_fails_loudly_without_a_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1805_05278_gb300 as gb
    h = ctypes.c_void_p()
    st = gb.gbqr_create(ctypes.byref(h), 0, None)
    assert st in (gb.GBQR_ECUDA, gb.GBQR_EINVAL)
    with pytest.raises(Exception):
        gb.Context(0)
