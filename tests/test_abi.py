"""CPU checks of the C ABI library: it builds, loads, and exports every declared entry point."""
import ctypes
import os
import re
import subprocess

from paper_2506_10257_gb300 import build as B
from paper_2506_10257_gb300 import rpca

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(rpca_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 9
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(rpca.EXPORTED) <= set(names)


def test_status_strings_and_defaults_without_gpu():
    lib = rpca.load()
    assert rpca.status_str(rpca.OK) == "ok"
    assert "budget" in rpca.status_str(rpca.ERR_BUDGET)
    p = rpca.default_params(4096, 20)
    assert (p.m, p.T, p.max_iter, p.tol, p.rho, p.mu0_scale) == (4096, 20, 500, 1e-7, 1.5, 1.25)
    assert lib is rpca.load()


def test_ctypes_mirrors_match_the_header(tmp_path):
    # compile a probe against include/rpca.h with the host compiler and compare layouts
    fields_p = [f for f, _ in rpca.Params._fields_]
    fields_r = [f for f, _ in rpca.Result._fields_]
    fields_w = [f for f, _ in rpca.Window._fields_]
    cname = {"lambda_": "lambda"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rpca.h"', 'int main(void) {',
             'printf("%zu %zu %zu\\n", sizeof(rpca_params), sizeof(rpca_result), sizeof(rpca_window));']
    for f in fields_p:
        lines.append(f'printf("%zu\\n", offsetof(rpca_params, {cname.get(f, f)}));')
    for f in fields_r:
        lines.append(f'printf("%zu\\n", offsetof(rpca_result, {cname.get(f, f)}));')
    for f in fields_w:
        lines.append(f'printf("%zu\\n", offsetof(rpca_window, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals[0] == ctypes.sizeof(rpca.Params) and vals[1] == ctypes.sizeof(rpca.Result)
    assert vals[2] == ctypes.sizeof(rpca.Window)
    offs = [getattr(rpca.Params, f).offset for f in fields_p] + [getattr(rpca.Result, f).offset for f in fields_r]
    offs += [getattr(rpca.Window, f).offset for f in fields_w]
    assert vals[3:] == offs
