"""The C-ABI library builds, loads and exports every symbol include/drgraph.h
declares; the Python Params mirror matches the C struct.  No GPU needed: no
call here reaches the device."""
import ctypes as C
import os
import re
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def drg():
    from paper_2008_07799_gb300 import build
    build.build()
    import paper_2008_07799_gb300 as m
    m.lib()
    return m


def _declared():
    src = open(os.path.join(ROOT, "include", "drgraph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(drg_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(drg):
    declared = _declared()
    assert len(declared) >= 25
    L = drg.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(drg.EXPORTS) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", drg.LIB_PATH], capture_output=True, text=True).stdout
    for name in declared:
        assert re.search(r"\bT " + name + r"\b", out), name


def test_params_layout_and_defaults(drg):
    p = drg.Params.default()
    assert (p.k, p.M, p.epochs, p.substeps, p.stop_nodes, p.match_rounds, p.max_levels) == (1, 5, 400, 16, 1000, 8, 32)
    assert abs(p.gamma - 0.1) < 1e-7 and abs(p.gamma_coarsest - 0.01) < 1e-9
    assert p.b == 1.0 and p.lr0 == 1.0 and p.sigma == 1.0 and p.clip == 5.0 and abs(p.rho - 0.8) < 1e-7
    assert p.init_scale == float(np.float32(1e-4))
    assert p.seed == 0 and p.mode == 0 and p.precision == 0 and p.multilevel == 1 and p.coarsen == 0 and p.level_tables == 0 and p.perplexity == 0.0
    assert p.row_cap == 0
    assert C.sizeof(drg.Params) == 104


def test_params_mirror_matches_the_header(drg, tmp_path):
    # the ctypes mirror against the C compiler's own layout of drg_params
    fields = [f for f, _ in drg.Params._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'    printf("%zu\\n", offsetof(drg_params, {f}));\n' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "drgraph.h"\nint main(void) {\n'
                   '    printf("%zu\\n", sizeof(drg_params));\n' + body + '    return 0;\n}\n')
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == C.sizeof(drg.Params)
    assert got[1:] == [getattr(drg.Params, f).offset for f in fields]


def test_status_strings_and_null_arguments(drg):
    L = drg.lib()
    assert L.drg_status_string(0) == b"ok"
    assert L.drg_status_string(1) == b"invalid argument"
    assert L.drg_status_string(6) == b"graph has no edges"
    # argument checks happen before any device work
    assert L.drg_create(None, 0, None) == 1
    assert L.drg_destroy(None) == 1
    assert L.drg_graph_destroy(None) == 1
    assert L.drg_layout(None, None, None, None) == 1
    assert L.drg_kernel_launches(None) == 0
    assert L.drg_probe_memory(None, 0, 1 << 25, 1000, 1, None, None) == 1
    assert L.drg_autotune_enable(None, 1) == 1
    assert L.drg_autotune_read(0, None, None, None, None) == 1


def test_missing_library_fails_loudly():
    # no CPU fallback: without the built library the first call raises
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_2008_07799_gb300 as m\n"
            "m._lib = None\n"
            "m.LIB_PATH = '/nonexistent/libdrgraph.so'\n"
            "try:\n"
            "    m.Context(0)\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert "raised:" in out.stdout and "missing" in out.stdout, (out.stdout, out.stderr)


def test_python_constants_match_the_header(drg):
    # every DRG_PROBE_*, DRG_MODE_*, DRG_PREC_* and DRG_PROF_* value the
    # binding names is the header's #define
    src = open(os.path.join(ROOT, "include", "drgraph.h")).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+DRG_([A-Z0-9_]+)\s+(\d+)\b", src)}
    probes = {k: v for k, v in defines.items() if k.startswith("PROBE_")}
    assert len(probes) == 6
    for name, value in probes.items():
        assert getattr(drg, name) == value, name
    for name, value in defines.items():
        if hasattr(drg, name) and isinstance(getattr(drg, name), int):
            assert getattr(drg, name) == value, name
