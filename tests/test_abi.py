"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, and the ctypes structures match the C layout."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:mc_status|void|const\s+char\s*\*)\s*(mc_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2209_01158_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        from paper_2209_01158_gb300.build import build
        build()
    return _native.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mc_setup", "mc_step_decoupled", "mc_step_coupled", "mc_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2209_01158_gb300 import _native
    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a prototype for every header function
    assert names <= set(_native.SIGNATURES), names - set(_native.SIGNATURES)
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(mc_\w+)\b", out))
    assert names <= exported, names - exported


def test_struct_layout_matches_c(tmp_path):
    from paper_2209_01158_gb300 import _native as N
    import ctypes
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mc.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mc_opts), sizeof(mc_stats),'
                   ' sizeof(mc_grid), offsetof(mc_stats, rel_residual), offsetof(mc_opts, spin_limit),'
                   ' offsetof(mc_opts, inner_form), offsetof(mc_stats, mass_defect));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(N.mc_opts), ctypes.sizeof(N.mc_stats), ctypes.sizeof(N.mc_grid),
                    N.mc_stats.rel_residual.offset, N.mc_opts.spin_limit.offset,
                    N.mc_opts.inner_form.offset, N.mc_stats.mass_defect.offset]


def test_host_only_calls(lib):
    """Calls that need no device: defaults, status strings, argument errors
    caught before any CUDA work."""
    import ctypes
    import paper_2209_01158_gb300 as mc
    o = mc.mc_default_opts()
    assert o.precision == 0 and o.rtol == 1e-12 and o.max_iter > 0
    assert lib.mc_status_string(4) == b"no convergence within max_iter"
    out = ctypes.c_void_p()
    g = mc.N.mc_grid(0, 4)
    assert lib.mc_setup(ctypes.byref(g), 1, None, None, None, None, 1.0, None, None,
                        ctypes.byref(out)) == mc.N.MC_E_ARG
    assert b"grid" in lib.mc_last_error(None)
    assert lib.mc_step_decoupled(None, 0, 1, None) == mc.N.MC_E_ARG


def test_binding_constants_match_the_header():
    """Every integer constant the header defines (#define or enumerator) has
    the same value in the Python binding."""
    from paper_2209_01158_gb300 import _native
    vals = {}
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*#define\s+(MC_[A-Z0-9_]+)\s+(-?\d+)\s*$", text, re.M):
            vals[m.group(1)] = int(m.group(2))
        for m in re.finditer(r"\b(MC_[A-Z0-9_]+)\s*=\s*(-?\d+)", text):
            vals[m.group(1)] = int(m.group(2))
    assert len(vals) >= 20, vals
    missing = [k for k in vals if not hasattr(_native, k)]
    assert not missing, missing
    wrong = {k: (v, getattr(_native, k)) for k, v in vals.items() if getattr(_native, k) != v}
    assert not wrong, wrong
