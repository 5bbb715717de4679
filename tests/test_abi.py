"""CPU checks of the boundary: the C-ABI library builds for sm_103a, loads,
and exports every symbol that include/dpm.h declares; the Python binding
covers exactly those symbols.  No CUDA call is made here."""
import ctypes
import os
import re

import pytest

from paper_0910_0329_gb300 import build_lib, dpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(dpm_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary_calls():
    names = declared_symbols()
    for required in ["dpm_load_phantom", "dpm_build_tables", "dpm_run", "dpm_read_dose"]:
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    path = build_lib.build()
    L = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_exactly_the_declared_symbols():
    assert sorted(dpm._SIGS) == declared_symbols()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(dpm, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(dpm, "_lib", None)
    with pytest.raises(ImportError):
        dpm.lib()


def test_struct_layouts_match_header():
    # sizes of the ABI structs as laid out by the C compiler (x86-64 / aarch64 LP64)
    assert ctypes.sizeof(dpm.dpm_material) == 4 + 4 + 3 * 8 * 8 + 8 + 8
    assert ctypes.sizeof(dpm.dpm_table_params) == 7 * 8 + 8
    assert ctypes.sizeof(dpm.dpm_source) == 8 + 8 + 3 * 8 + 4 * 8
    assert ctypes.sizeof(dpm.dpm_run_opts) == 6 * 4 + 8 + 5 * 4 + 4  # trailing padding to 8
    assert ctypes.sizeof(dpm.dpm_job) == 4 + 4 + ctypes.sizeof(dpm.dpm_source) + 3 * 8
    assert ctypes.sizeof(dpm.dpm_run_stats) == 8 + 2 * 4 + 4 * 8 + 5 * 8 + 2 * 8 + 2 * 8


ABI_STRUCTS = ["dpm_material", "dpm_table_params", "dpm_source", "dpm_run_opts", "dpm_run_stats", "dpm_job",
               "dpm_serve_opts", "dpm_request_status", "dpm_server_info"]


def test_struct_fields_match_the_c_compiler(tmp_path):
    """Every binding struct against the header as gcc lays it out: the same
    field names, offsets and total size."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dpm.h"', "int main(void) {"]
    expect = []
    for name in ABI_STRUCTS:
        cls = getattr(dpm, name)
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        expect.append(ctypes.sizeof(cls))
        for field, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {field}));')
            expect.append(getattr(cls, field).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect


def test_every_entry_point_rejects_a_null_handle_without_a_gpu():
    """The header's error contract for a null context or server: DPM_EINVAL
    from every call that takes one, before any CUDA call (so this runs on a
    machine without a GPU); destroy calls are no-ops and the last error of a
    null context is a fixed message."""
    L = ctypes.CDLL(build_lib.build())
    skip = {"dpm_host_tables_build", "dpm_host_tables_get", "dpm_host_tables_free", "dpm_serve_next_chunk",
            "dpm_serve_select", "dpm_last_error", "dpm_destroy", "dpm_server_destroy"}
    checked = 0
    for name, (res, args) in sorted(dpm._SIGS.items()):
        if name in skip:
            continue
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
        vals = []
        for a in args:
            if a in (ctypes.c_double, ctypes.c_float):
                vals.append(0.0)
            elif a in (ctypes.c_int, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64,
                       ctypes.c_size_t):
                vals.append(0)
            else:
                vals.append(None)
        assert f(*vals) == dpm.DPM_EINVAL, name
        checked += 1
    assert checked == len([n for n in dpm._SIGS if n not in skip]) and checked > 20
    for name in ("dpm_destroy", "dpm_server_destroy"):
        f = getattr(L, name)
        f.restype, f.argtypes = None, [ctypes.c_void_p]
        f(None)
    f = L.dpm_last_error
    f.restype, f.argtypes = ctypes.c_char_p, [ctypes.c_void_p]
    assert f(None) == b"null context"
    # the pure policies: no options size nothing, an empty queue selects nothing
    assert L.dpm_serve_next_chunk(None, ctypes.c_uint64(10), ctypes.c_double(0.1)) == 0
