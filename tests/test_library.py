"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/tddft.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tddft.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tddft_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1507_08157_gb300 import build
    return build.build()


def test_header_declares_the_three_calls():
    names = _declared()
    for n in ("tddft_apply", "tddft_pcg_step", "tddft_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tddft_[a-z_0-9]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_declares_all(lib_path):
    from paper_1507_08157_gb300 import tddft
    lib = tddft.load(lib_path)
    for n in _declared():
        assert hasattr(lib, n)
    assert sorted(tddft.SYMBOLS) == _declared()


def test_default_options_without_gpu(lib_path):
    from paper_1507_08157_gb300 import tddft
    o = tddft._options()
    assert o.precision == tddft.FP64 and o.precond_maxit == 50 and abs(o.precond_tol - 1e-4) < 1e-18
    assert o.reapply_every == 10 and o.restart_every == 10
    assert o.spin_limit_cycles == 0


def test_options_struct_layout_matches_the_header(lib_path, tmp_path):
    # the binding's mirror of tddft_options must have the layout the C compiler gives the header
    import ctypes
    from paper_1507_08157_gb300 import tddft
    src = tmp_path / "layout.c"
    fields = [f for f, _ in tddft._Options._fields_]
    body = "".join(f'printf("%zu ", offsetof(tddft_options, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "tddft.h"\n'
                   'int main(void) { ' + body + 'printf("%zu", sizeof(tddft_options)); return 0; }\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[:-1] == [getattr(tddft._Options, f).offset for f in fields]
    assert got[-1] == ctypes.sizeof(tddft._Options)



@pytest.mark.parametrize("struct", ["tddft_options", "tddft_tuning_entry", "tddft_stage_stats"])
def test_struct_layouts_match_the_header(lib_path, tmp_path, struct):
    # every ctypes mirror of a boundary struct has the layout the C compiler gives the header
    import ctypes
    from paper_1507_08157_gb300 import tddft
    mirror = {"tddft_options": tddft._Options, "tddft_tuning_entry": tddft.TuningEntry,
              "tddft_stage_stats": tddft.StageStats}[struct]
    src = tmp_path / "layout.c"
    fields = [f for f, _ in mirror._fields_]
    body = "".join(f'printf("%zu ", offsetof({struct}, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "tddft.h"\n'
                   'int main(void) { ' + body + f'printf("%zu", sizeof({struct})); return 0; }}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[:-1] == [getattr(mirror, f).offset for f in fields]
    assert got[-1] == ctypes.sizeof(mirror)

def test_product_code_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1507_08157_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, flags=re.M), f
                assert "oracle/" not in text, f
