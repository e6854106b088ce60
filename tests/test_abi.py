"""The C-ABI library loads and exports every entry point include/*.h declares
(no compute call: this runs without a GPU)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mm_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_five_calls():
    names = declared_functions()
    for n in ("mm_model_create", "mm_schedule_set", "mm_eval_moves", "mm_topk", "mm_apply_move"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2511_18296_b300 as mm
    L = ctypes.CDLL(mm.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2511_18296_b300 as mm
    bound = {name for name, _, _ in mm.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2511_18296_b300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(f).read()
            assert "import oracle" not in txt and "from oracle" not in txt, f
            assert "liboracle" not in txt, f


def test_error_path_without_model():
    import paper_2511_18296_b300 as mm
    L = mm.lib()
    # NULL model pointer: argument checks run on the host and return an error code
    assert L.mm_eval_moves(None, None, 0, None, None, None) == 1
    assert L.mm_last_error().decode() != ""


@pytest.mark.parametrize("struct,cls", [("mm_model_desc", "MMModelDesc"), ("mm_move", "MMMove")])
def test_binding_struct_layout_matches_header(struct, cls, tmp_path):
    """The ctypes structures have the header's field offsets and size (a C
    program built against include/mm.h prints them)."""
    import subprocess
    import paper_2511_18296_b300 as mm
    C = getattr(mm, cls)
    names = [f[0] for f in C._fields_]
    cnames = {"lam": "lambda"}
    prog = ["#include <stddef.h>", "#include <stdio.h>", '#include "mm.h"', "int main(void) {",
            f'  printf("%zu\\n", sizeof({struct}));']
    prog += [f'  printf("%zu\\n", offsetof({struct}, {cnames.get(n, n)}));' for n in names]
    prog += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(C)
    assert out[1:] == [getattr(C, n).offset for n in names]
