"""The C-ABI library builds, loads, and exports every entry point include/lr.h declares;
host-side argument checks work without a GPU (no compute calls are made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(lr_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2405_13364_gb300 import _binding
    return _binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lr_create", "lr_destroy", "lr_workspace_size", "lr_render", "lr_render_batch",
                     "lr_render_backward", "lr_get_stats", "lr_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2405_13364_gb300 import _binding
    assert declared_functions() <= set(_binding._SIGNATURES)


def test_struct_sizes_match_header_layout(lib):
    from paper_2405_13364_gb300 import _binding as B
    # plain C layout expectations (x86-64 and aarch64 LP64 agree)
    assert ctypes.sizeof(B.lr_config) == 10 * 4
    assert ctypes.sizeof(B.lr_quads) == 6 * 8
    assert ctypes.sizeof(B.lr_camera) == 18 * 4
    assert ctypes.sizeof(B.lr_target) == 5 * 8
    assert ctypes.sizeof(B.lr_view) == 48 + 72 + 8 + 40 + 8 + 8


def test_struct_layouts_match_the_c_compiler(tmp_path):
    # every binding struct against gcc's layout of the same struct from include/lr.h
    import subprocess
    from paper_2405_13364_gb300 import _binding as B
    names = ["lr_config", "lr_quads", "lr_camera", "lr_target", "lr_view", "lr_stats", "lr_ws_layout",
             "lr_server_config", "lr_request_info", "lr_server_stats"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lr.h"', "int main(void) {"]
    for n in names:
        lines.append(f'  printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in getattr(B, n)._fields_:
            lines.append(f'  printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for n in names:
        st = getattr(B, n)
        assert int(out[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(out[f"{n}.{f}"]) == getattr(st, f).offset, f"{n}.{f}"


def test_host_side_argument_errors(lib):
    from paper_2405_13364_gb300 import _binding as B
    assert lib.lr_create(None, None) == B.LR_ERR_INVALID_ARG
    assert lib.lr_destroy(None) == B.LR_ERR_INVALID_ARG
    assert lib.lr_last_error(None) == b"null context"
    n = ctypes.c_size_t()
    assert lib.lr_workspace_size(None, 10, 64, 64, ctypes.byref(n)) == B.LR_ERR_INVALID_ARG
    assert lib.lr_get_stats(None, None) == B.LR_ERR_INVALID_ARG
    assert lib.lr_render(None, None, None, 1, 1, None, None, 0, None) == B.LR_ERR_INVALID_ARG
    assert lib.lr_render_backward(None, None, None, 1, 1, None, None, None, None, None, 0, None) == \
        B.LR_ERR_INVALID_ARG


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2405_13364_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lr_oracle" not in text, f
