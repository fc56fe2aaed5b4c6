"""The C-ABI library builds, loads without a GPU, and exports every declared entry point."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:gtap_status|const char\*)\s+(gtap_\w+)\s*\(", text, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2604_05982_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    declared = _declared_functions()
    assert len(declared) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(gtap_\w+)", out))
    missing = [n for n in declared if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(lib_path):
    from paper_2604_05982_gb300 import gtap as G
    lib = G.load_library()
    for name in _declared_functions():
        assert hasattr(lib, name)
        assert name in G.exported_symbols(), f"binding lacks {name}"
    assert G.gtap_status_string(0) == "ok"
    assert G.gtap_status_string(3) == "task-record pool exhausted"


def test_struct_layouts_match_header(lib_path, tmp_path):
    from paper_2604_05982_gb300 import gtap as G
    # sizes and field offsets as the C compiler lays out include/gtap.h
    structs = {"gtap_config": G.gtap_config, "gtap_stats": G.gtap_stats, "gtap_error_info": G.gtap_error_info,
               "gtap_kclique_args": G.gtap_kclique_args, "gtap_uts_args": G.gtap_uts_args,
               "gtap_mergesort_args": G.gtap_mergesort_args, "gtap_fib_args": G.gtap_fib_args,
               "gtap_nqueens_args": G.gtap_nqueens_args, "gtap_bintree_args": G.gtap_bintree_args,
               "gtap_integrate_args": G.gtap_integrate_args, "gtap_tune_trial": G.gtap_tune_trial}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gtap.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
    assert ctypes.sizeof(G.gtap_fib_args) == 16
    assert ctypes.sizeof(G.gtap_uts_args) == 32
    assert ctypes.sizeof(G.gtap_mergesort_args) == 40
    assert ctypes.sizeof(G.gtap_integrate_args) == 24
