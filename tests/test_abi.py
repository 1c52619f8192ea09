"""The C-ABI library loads, exports every symbol include/mpm.h declares, and its
structs have the layout the Python binding marshals.  No GPU compute here."""
import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpm.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(mpm_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2502_18437_gb300 import build

    return build.build()


def test_header_declares_the_five_calls_of_the_boundary():
    syms = declared_symbols()
    for name in ("mpm_create", "mpm_add_particles", "mpm_set_rigid", "mpm_substep", "mpm_read_state"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    L = ct.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mpm_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_binding_mirrors_every_declared_symbol():
    from paper_2502_18437_gb300 import mpm

    for s in declared_symbols():
        assert s in mpm._SIGS, s
        assert callable(getattr(mpm, s)), s


def test_status_strings_without_gpu(libpath):
    from paper_2502_18437_gb300 import mpm

    assert mpm.mpm_status_string(0) == "ok"
    assert "timed out" in mpm.mpm_status_string(-8)


def test_struct_layout_matches_header(tmp_path):
    from paper_2502_18437_gb300 import mpm

    src = tmp_path / "layout.c"
    fields_cfg = [f[0] for f in mpm.mpm_config._fields_]
    fields_rig = [f[0] for f in mpm.mpm_rigid._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpm.h"', "int main(void){"]
    lines.append('printf("cfg %zu\\n", sizeof(mpm_config));')
    lines.append('printf("rig %zu\\n", sizeof(mpm_rigid));')
    for f in fields_cfg:
        lines.append(f'printf("cfg.{f} %zu\\n", offsetof(mpm_config, {f}));')
    for f in fields_rig:
        lines.append(f'printf("rig.{f} %zu\\n", offsetof(mpm_rigid, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    assert int(got["cfg"]) == ct.sizeof(mpm.mpm_config)
    assert int(got["rig"]) == ct.sizeof(mpm.mpm_rigid)
    for f in fields_cfg:
        assert int(got[f"cfg.{f}"]) == getattr(mpm.mpm_config, f).offset, f
    for f in fields_rig:
        assert int(got[f"rig.{f}"]) == getattr(mpm.mpm_rigid, f).offset, f


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2502_18437_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "mpm_oracle" not in text and "liboracle" not in text, fn
