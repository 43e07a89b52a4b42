"""The C-ABI library builds, loads and exports every entry point include/ctaux.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ctaux.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ctaux_[A-Za-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for need in ("ctaux_init", "ctaux_sweep", "ctaux_measure_G", "ctaux_recompute",
                 "ctaux_get_stats", "ctaux_get_trace", "ctaux_get_config", "ctaux_set_config",
                 "ctaux_destroy", "ctaux_last_error"):
        assert need in syms


def test_library_builds_loads_and_exports_every_symbol():
    from paper_1010_3690_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1010_3690_gb300 import ctaux
    assert sorted(ctaux.EXPORTED) == declared_symbols()


def test_struct_layouts_match_header_sizes():
    from paper_1010_3690_gb300 import ctaux
    # ctaux_trace_rec: 8+4+4+8+4+4+16+8+8
    assert ctypes.sizeof(ctaux.TraceRec) == 64
    assert ctaux.TRACE_DTYPE.itemsize == 64
    assert ctypes.sizeof(ctaux.ChainParams) == 4 * 3 + 4 + 8 * 2 + 8 * 3 + 4 * 2 + 8 + 4 + 4


def test_init_rejects_bad_arguments_without_a_gpu():
    """Argument checks run before any device call, so they work on a CPU-only host."""
    from paper_1010_3690_gb300 import ctaux
    from workloads import configs
    ch = configs.aim1(K=1.0, k_max=8, capacity=32)
    bad = configs.aim1(K=1.0, k_max=8, capacity=32)
    bad.k_max = 999
    with pytest.raises(ctaux.CtauxError) as ei:
        ctaux.Context([bad])
    assert ei.value.code == 1
    with pytest.raises(ctaux.CtauxError):
        ctaux.Context([ch], p_insert=0.9, p_flip=0.3)


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every field of the ctypes mirrors sits at the offset the C compiler gives
    it in include/ctaux.h, and the structs have the same sizes (host C, no GPU)."""
    import shutil
    import subprocess
    from paper_1010_3690_gb300 import ctaux
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("ctaux_chain_params", ctaux.ChainParams), ("ctaux_params", ctaux.Params),
             ("ctaux_stats", ctaux.Stats), ("ctaux_trace_rec", ctaux.TraceRec)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ctaux.h"', "int main(void) {"]
    expect = []
    for cname, cls in pairs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {fname}));')
            expect.append(getattr(cls, fname).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == expect
