"""The C ABI library builds, loads and exports every entry point of include/kpm.h.

CPU only: no compute call is made (there may be no GPU here); kpm_create is
expected to refuse cleanly when no device is present.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_05685_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("kpm_build_H", "kpm_observables", "rmft_iterate", "kpm_bounds", "kpm_peierls_phases",
                     "kpm_create", "kpm_destroy", "kpm_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2212_05685_gb300 import kpm
    for name in _declared():
        assert name in kpm._SIGNATURES, name


def test_strerror_and_refusals_without_gpu(lib):
    from paper_2212_05685_gb300 import kpm
    k = kpm.load()
    assert k.kpm_strerror(0) == b"ok"
    assert k.kpm_strerror(kpm.KPM_EINVAL) == b"invalid argument"
    assert k.kpm_strerror(12345) == b"unknown status"
    # null output handle is refused before any CUDA call
    assert k.kpm_create(None, 0) == kpm.KPM_EINVAL
    # null context is refused by every entry point
    m = kpm.make_model(4, 4)
    assert k.kpm_peierls_phases(None, ctypes.byref(m), None, None) == kpm.KPM_EINVAL
    assert k.kpm_destroy(None) == kpm.KPM_EINVAL


def test_struct_layouts_match_header(tmp_path):
    """Field offsets and sizes of the ctypes structures equal those the C
    compiler gives the header's structures."""
    import shutil
    import subprocess
    from paper_2212_05685_gb300 import kpm
    structs = [kpm.kpm_model, kpm.kpm_opts, kpm.kpm_rmft_opts, kpm.kpm_rmft_stats]
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kpm.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'  printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(got[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(st, f).offset, (n, f)
