"""The C-ABI library builds, loads and exports every symbol include/lb.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lb\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_0911_0459_gb300 import build
    return build.build()


def test_header_declares_the_interface():
    names = declared_functions()
    for n in ("lb_create", "lb_step", "lb_fields", "lb_filled_length", "lb_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches_header(libpath):
    from paper_0911_0459_gb300 import lb
    lib = lb.library()
    for n in declared_functions():
        assert hasattr(lib, n)
    assert set(lb.exported_symbols()) <= set(declared_functions())


def test_struct_layouts_match_header(libpath, tmp_path):
    """Compile a C probe of sizeof/offsetof and compare with the ctypes structs."""
    from paper_0911_0459_gb300 import lb
    probe = tmp_path / "p.c"
    fields = {"lb_walls": [f[0] for f in lb.LbWalls._fields_], "lb_params": [f[0] for f in lb.LbParams._fields_],
              "lb_grid": [f[0] for f in lb.LbGrid._fields_], "lb_alloc": [f[0] for f in lb.LbAlloc._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lb.h"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "p"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    py = {"lb_walls": lb.LbWalls, "lb_params": lb.LbParams, "lb_grid": lb.LbGrid, "lb_alloc": lb.LbAlloc}
    for s, cls in py.items():
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f in fields[s]:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_product_wall_gradient_matches_oracle_closed_form():
    from oracle import analysis as an
    from paper_0911_0459_gb300 import binary_wall_gradient
    for th in (30.0, 45.0, 60.0, 80.0):
        for A in (0.03, 0.04, 0.05):
            assert abs(binary_wall_gradient(th, A, A) - an.binary_wall_gradient_for_angle(th, A, A)) < 1e-10


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_0911_0459_gb300 import lb
    monkeypatch.setattr(lb, "_lib", None)
    monkeypatch.setattr(lb, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lb.library()
