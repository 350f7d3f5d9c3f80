"""The C-ABI library builds, loads and exports every symbol that
include/*.h declares; the ctypes structs match the C layout.  No GPU needed
(no compute call is made)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"^SPTRSV_API\s+[^;(]*?\b(sptrsv_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_11445_gb300 import binding as B
    return B.load()


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("sptrsv_analyze", "sptrsv_transform", "sptrsv_solve", "sptrsv_check"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_exports_nothing_else():
    from paper_2103_11445_gb300 import binding as B
    out = subprocess.run(["nm", "-D", "--defined-only", B.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = sorted(set(re.findall(r" T (sptrsv_\w+)", out)))
    assert exported == declared_functions()


def test_binding_covers_every_declared_symbol():
    from paper_2103_11445_gb300 import binding as B
    assert sorted(B._SIGS) == declared_functions()


def test_struct_layout_matches_c(tmp_path):
    from paper_2103_11445_gb300 import binding as B
    probe = tmp_path / "probe.c"
    fields_p = [f for f, _ in B.TransformParams._fields_]
    fields_i = [f for f, _ in B.Info._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sptrsv.h"', "int main(void){"]
    lines.append('printf("%zu %zu\\n", sizeof(sptrsv_transform_params_t), sizeof(sptrsv_info_t));')
    for f in fields_p:
        lines.append(f'printf("%zu ", offsetof(sptrsv_transform_params_t, {f}));')
    lines.append('printf("\\n");')
    for f in fields_i:
        lines.append(f'printf("%zu ", offsetof(sptrsv_info_t, {f}));')
    lines.append('printf("\\n"); return 0; }')
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sp, si = map(int, out[0].split())
    assert sp == ctypes.sizeof(B.TransformParams) and si == ctypes.sizeof(B.Info)
    assert [int(v) for v in out[1].split()] == [getattr(B.TransformParams, f).offset for f in fields_p]
    assert [int(v) for v in out[2].split()] == [getattr(B.Info, f).offset for f in fields_i]


def test_status_strings_and_defaults(lib):
    from paper_2103_11445_gb300 import binding as B
    for code in range(11):
        assert B._status_string(code)
    prm = B.sptrsv_default_params()
    assert prm.select_mode == B.SELECT_HEURISTIC
    assert prm.max_depth == 8 and abs(prm.flop_budget - 0.10) < 1e-15


def test_host_side_argument_errors(lib):
    from paper_2103_11445_gb300 import binding as B
    out = ctypes.c_void_p()
    assert lib.sptrsv_analyze(-1, 0, None, None, None, None, ctypes.byref(out)) == 1
    assert lib.sptrsv_analyze(4, 4, None, None, None, None, ctypes.byref(out)) == 1
    assert lib.sptrsv_analyze(0, 0, None, None, None, None, None) == 1
    assert lib.sptrsv_solve(None, None, None, 1, None) == 1
    assert lib.sptrsv_transform(None, None, None) == 1
    assert lib.sptrsv_check(None, None) == 1
    lib.sptrsv_plan_destroy(None)


def test_pcg_host_side_argument_errors(lib):
    """The preconditioned-CG entry points refuse bad arguments before any
    device work (no GPU needed): null output, empty matrix, null arrays, an
    unknown preconditioner, a null object."""
    from paper_2103_11445_gb300 import binding as B
    out = ctypes.c_void_p()
    fake = ctypes.c_void_p(16)   # never dereferenced: the checks come first
    assert lib.sptrsv_pcg_create(4, 4, fake, fake, fake, 0, None, None, None, None) == 1
    assert lib.sptrsv_pcg_create(0, 4, fake, fake, fake, 0, None, None, None,
                                 ctypes.byref(out)) == 1
    assert out.value is None
    assert lib.sptrsv_pcg_create(4, 0, fake, fake, fake, 0, None, None, None,
                                 ctypes.byref(out)) == 1
    assert lib.sptrsv_pcg_create(4, 4, None, fake, fake, 0, None, None, None,
                                 ctypes.byref(out)) == 1
    assert lib.sptrsv_pcg_create(4, 4, fake, fake, fake, 2, None, None, None,
                                 ctypes.byref(out)) == 1
    assert lib.sptrsv_pcg_create(4, 4, fake, fake, fake, -1, None, None, None,
                                 ctypes.byref(out)) == 1
    it, rel = ctypes.c_int32(7), ctypes.c_double(7.0)
    assert lib.sptrsv_pcg_solve(None, fake, fake, 1e-8, 10, ctypes.byref(it),
                                ctypes.byref(rel), None) == 1
    lo, up = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.sptrsv_pcg_get_plans(None, ctypes.byref(lo), ctypes.byref(up)) == 1
    nnz = ctypes.c_int64()
    assert lib.sptrsv_pcg_get_factor(None, ctypes.byref(nnz), None, None) == 1
    lib.sptrsv_pcg_destroy(None)
    assert (B.PRECOND_SGS, B.PRECOND_IC0) == (0, 1)


def test_network_files_are_checked_before_any_device_work(tmp_path, lib):
    """Missing, foreign and short network files are refused with
    SPTRSV_ERR_INVALID_ARG, and saving the process-wide model when none is
    loaded with SPTRSV_ERR_BAD_STATE -- all before any device call."""
    from paper_2103_11445_gb300 import binding as B
    missing = str(tmp_path / "missing.bin")
    foreign = tmp_path / "foreign.bin"
    foreign.write_bytes(b"NOTANET!" + bytes(64))
    short = tmp_path / "short.bin"
    import struct
    short.write_bytes(b"SPTRSVNN" + struct.pack("<4i", 1, 17, 64, 1) + bytes(40))
    for path in (missing, str(foreign), str(short)):
        out = ctypes.c_void_p()
        assert lib.sptrsv_mlp_load(os.fsencode(path), ctypes.byref(out)) == 1
        assert not out.value
        assert lib.sptrsv_costmodel_load(os.fsencode(path)) == 1
    assert lib.sptrsv_costmodel_save(os.fsencode(str(tmp_path / "x.bin"))) == 9
    with pytest.raises(B.SptrsvError):
        B.sptrsv_costmodel_save(str(tmp_path / "y.bin"))
