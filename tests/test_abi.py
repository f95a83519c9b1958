"""The C-ABI library builds for sm_103a and exports every declared symbol.
No compute call is made here (no GPU is needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2103_14688_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        names += re.findall(r"^\s*(?:int|const char \*)\s*(cfpq_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["cfpq_create", "cfpq_destroy", "cfpq_load_graph", "cfpq_load_rsm", "cfpq_run",
                 "cfpq_get_reachable", "cfpq_extract_paths", "cfpq_status_string"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    lib = ctypes.CDLL(B.build())
    lib.cfpq_status_string.restype = ctypes.c_char_p
    assert lib.cfpq_status_string(0) == b"ok"
    assert lib.cfpq_status_string(-4).startswith(b"iteration")
    assert lib.cfpq_status_string(12345) == b"unknown status"


def test_binding_names_match_the_header():
    from paper_2103_14688_gb300 import cfpq
    src = open(cfpq.__file__).read()
    for n in _declared():
        assert f'"{n}"' in src, n


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes mirrors of the header's structs have the header's
    size and field offsets (a C program built with gcc prints them)."""
    from paper_2103_14688_gb300 import cfpq
    structs = [cfpq.cfpq_options, cfpq.cfpq_rsm, cfpq.cfpq_run_stats, cfpq.cfpq_tuning, cfpq.cfpq_query]
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "cfpq.h"', "int main(void) {"]
    for S in structs:
        lines.append(f'    printf("{S.__name__} sizeof %zu\\n", sizeof({S.__name__}));')
        for f, _ in S._fields_:
            lines.append(f'    printf("{S.__name__} {f} %zu\\n", offsetof({S.__name__}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", inc, "-o", str(exe), str(src)])
    got = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for S in structs:
        assert ctypes.sizeof(S) == got[(S.__name__, "sizeof")], S.__name__
        for f, _ in S._fields_:
            assert getattr(S, f).offset == got[(S.__name__, f)], (S.__name__, f)


def test_default_options_reject_unknown_names():
    from paper_2103_14688_gb300 import cfpq
    o = cfpq.default_options(closure_mode=cfpq.CFPQ_CLOSURE_TC_FP4, tile_format=cfpq.CFPQ_TILES_NVFP4, tile_ratio=64)
    assert (o.closure_mode, o.tile_format, o.tile_ratio) == (cfpq.CFPQ_CLOSURE_TC_FP4, cfpq.CFPQ_TILES_NVFP4, 64)
    assert o.struct_size == ctypes.sizeof(cfpq.cfpq_options) and o.loop_mode == cfpq.CFPQ_LOOP_DEVICE
    with pytest.raises(TypeError):
        cfpq.default_options(tile_fromat=2)


def test_create_validates_its_options_before_touching_a_device():
    """Options out of range are refused with INVALID_ARG (or UNSUPPORTED) before
    any CUDA call, so this runs on a machine without a GPU."""
    from paper_2103_14688_gb300 import cfpq
    lib = cfpq.load()

    def create(**kw):
        o = cfpq.default_options(**kw)
        h = ctypes.c_void_p()
        return lib.cfpq_create(ctypes.byref(h), ctypes.byref(o), None)

    assert create(closure_mode=99) == cfpq.CFPQ_ERR_INVALID_ARG
    assert create(tile_format=99) == cfpq.CFPQ_ERR_INVALID_ARG
    assert create(loop_mode=7) == cfpq.CFPQ_ERR_INVALID_ARG
    assert create(profile=1) == cfpq.CFPQ_ERR_INVALID_ARG  # profiling needs the host-driven loop
    assert create(closure_mode=cfpq.CFPQ_CLOSURE_TC_I8) == cfpq.CFPQ_ERR_UNSUPPORTED
    assert create(struct_size=3) == cfpq.CFPQ_ERR_INVALID_ARG


def test_create_fails_loudly_without_a_gpu():
    """No CPU path: without a CUDA device the context cannot be created."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2103_14688_gb300 import cfpq
    lib = cfpq.load()
    o = cfpq.default_options()
    h = ctypes.c_void_p()
    assert lib.cfpq_create(ctypes.byref(h), ctypes.byref(o), None) == cfpq.CFPQ_ERR_CUDA
    assert not h.value


def test_null_and_size_checks_without_gpu():
    """Calls refuse NULL handles and wrong struct sizes with INVALID_ARG,
    before any CUDA call."""
    from paper_2103_14688_gb300 import cfpq
    lib = cfpq.load()
    t = cfpq.cfpq_tuning()
    t.struct_size = ctypes.sizeof(cfpq.cfpq_tuning)
    assert lib.cfpq_tune(None, 0, ctypes.byref(t)) == cfpq.CFPQ_ERR_INVALID_ARG
    assert lib.cfpq_run(None, None) == cfpq.CFPQ_ERR_INVALID_ARG
    assert lib.cfpq_destroy(None) == cfpq.CFPQ_OK
    h = ctypes.c_void_p()
    e = (ctypes.c_uint32 * 1)(0)
    for kw in ({"closure_mode": 99}, {"tile_format": 99}, {"struct_size": 3},
               {"closure_mode": cfpq.CFPQ_CLOSURE_TC_I8}):
        o = cfpq.default_options(**kw)
        rc = lib.cfpq_server_create(ctypes.byref(h), ctypes.byref(o), None, 4, 1, 1, e, e, e)
        assert rc in (cfpq.CFPQ_ERR_INVALID_ARG, cfpq.CFPQ_ERR_UNSUPPORTED), (kw, rc)
        assert not h.value
