"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/flowref.h declares; the binding refuses to run without it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "flowref.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    from paper_1012_0006_gb300 import flowref
    return flowref


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ("fr_build_corridor", "fr_maxflow", "fr_extract_cut", "fr_refine_pair", "fr_refine_batch"):
        assert name in fns


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built.LIB_PATH)
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(built):
    assert set(declared_functions()) <= set(built.SYMBOLS)


def test_context_creation_fails_loudly_without_gpu(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert built.lib().fr_create(ctypes.byref(h), 0, 0, None) == built.FR_ERR_CUDA
    with pytest.raises(built.FlowRefError):
        built.Context(0)


def test_missing_library_is_an_error(built, monkeypatch):
    monkeypatch.setattr(built, "_LIB", None)
    monkeypatch.setattr(built, "LIB_PATH", "/nonexistent/libflowref.so")
    with pytest.raises(RuntimeError):
        built.lib()


def test_default_options(built):
    o = built.default_options()
    assert (o.mb, o.mb_reps, o.adaptive, o.max_iters, o.alpha_max, o.pulse_cap) == (0, 1, 0, 10, 1.0, 1 << 20)
    assert (o.fm_permille, o.mt_alpha) == (0, 0)


def test_status_strings(built):
    for st in range(8):
        assert built.lib().fr_status_string(st)


def test_struct_layouts_match_the_header(built):
    """The binding's ctypes structs have the sizes the compiled library uses."""
    F = built
    structs = [F.Graph, F.Options, F.PairResult, F.BatchResult, F.ProfileInfo, F.ServerConfig, F.Request,
               F.Response, F.MtResult, F.VcycleResult, F.CycleResult]
    for i, st in enumerate(structs):
        assert F.lib().fr_struct_size(i) == ctypes.sizeof(st), st.__name__
    assert F.lib().fr_struct_size(len(structs)) == -1


def declared_arities():
    """Parameter count of every function declaration in the header."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(fr_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
        name, params = m.group(1), m.group(2).strip()
        if name.endswith("_t"):
            continue
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(built):
    arities = declared_arities()
    assert len(arities) >= 20
    wrong = {name: (n, len(built.SYMBOLS[name][1])) for name, n in arities.items()
             if name in built.SYMBOLS and len(built.SYMBOLS[name][1]) != n}
    assert not wrong, wrong
