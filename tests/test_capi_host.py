"""Host-only checks of the C ABI: the library loads without a GPU, exports
every entry point declared in include/fcoo.h, and rejects bad arguments
before touching the device."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fc():
    import paper_1705_09905_gb300 as fc

    return fc


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fcoo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][A-Za-z0-9_ \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


def test_every_declared_symbol_is_exported(fc):
    names = declared_functions()
    assert "spmttkrp" in names and "fcoo_build" in names and len(names) >= 20, names
    missing = [n for n in names if not hasattr(fc.lib, n)]
    assert not missing, f"declared in include/fcoo.h but not exported: {missing}"


def test_table2_bytes_golden(fc):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "table2_storage.json")))
    for row in g["rows"]:
        assert fc.table2_bytes(1, row["nnz"], row["threadlen"]) == row["fcoo_ttm"]
        assert fc.table2_bytes(2, row["nnz"], row["threadlen"]) == row["fcoo_mttkrp"]
        assert row["fcoo_mttkrp"] < row["coo"]
        assert fc.table2_bytes(1, row["nnz"], row["threadlen"], index_bytes=2) == row["fcoo_ttm_idx16"]
        assert fc.table2_bytes(2, row["nnz"], row["threadlen"], index_bytes=2) == row["fcoo_mttkrp_idx16"]
    assert fc.table2_bytes(2, 1000, 8, index_bytes=3) == -1
    assert fc.table2_bytes(2, 1000, 7) == -1
    assert fc.table2_bytes(2, 1000, 128) == -1
    assert fc.table2_bytes(0, 1000, 8) == -1


def test_status_strings(fc):
    assert fc.lib.fcoo_status_string(0) == b"FCOO_OK"
    assert fc.lib.fcoo_status_string(-3) == b"FCOO_ERR_DUPLICATE"
    assert fc.lib.fcoo_version() >= 10000


@pytest.mark.parametrize("case", ["nmodes", "dims0", "mode", "op", "threadlen", "nullidx", "nnz", "nnz_max", "dims9"])
def test_build_rejects_bad_arguments_without_device_work(fc, case):
    lib = fc.lib
    dims = (ctypes.c_uint32 * 3)(4, 5, 6)
    a = (ctypes.c_uint32 * 2)(0, 1)
    v = (ctypes.c_float * 2)(1.0, 2.0)
    idx = (ctypes.c_void_p * 3)(ctypes.addressof(a), ctypes.addressof(a), ctypes.addressof(a))
    args = dict(nmodes=3, dims=ctypes.addressof(dims), nnz=2, idx=idx, val=ctypes.addressof(v), mode=0, op=0,
                threadlen=8)
    if case == "nmodes":
        args["nmodes"] = 1
    elif case == "dims0":
        dims[1] = 0
    elif case == "mode":
        args["mode"] = 3
    elif case == "op":
        args["op"] = 7
    elif case == "threadlen":
        args["threadlen"] = 12
    elif case == "nullidx":
        idx[2] = None
    elif case == "nnz":
        args["nnz"] = -5
    elif case == "nnz_max":  # one past FCOO_MAX_NNZ (the padded streams must stay below 2^31)
        args["nnz"] = 2147479552 + 1
    elif case == "dims9":  # more modes than FCOO_MAX_MODES
        args["nmodes"] = 9
    out = ctypes.c_void_p(1234)
    st = lib.fcoo_build(args["nmodes"], args["dims"], args["nnz"], ctypes.cast(idx, ctypes.POINTER(ctypes.c_void_p)),
                        args["val"], args["mode"], args["op"], args["threadlen"], None, ctypes.byref(out))
    assert st == -1, (case, st)
    assert out.value is None
    assert lib.fcoo_last_error().startswith(b"fcoo_build:")


def test_compute_entry_points_reject_null_handles(fc):
    lib = fc.lib
    assert lib.spmttkrp(None, None, 0, 16, None, None) == -1
    assert lib.spttm(None, None, 0, 16, None, None) == -1
    assert lib.spttmc(None, None, 0, 16, None, None) == -1
    assert lib.spttmc_plan_create(None, 0, 8, 8, None, None) == -1
    assert lib.spttmc_plan_run(None, None, 0, None, None) == -1
    assert lib.spttmc_plan_info(None, None, None) == -1
    assert lib.tucker_hooi_iter(None, None, None) == -1
    assert lib.cp_state_use_fibres(None, None, 8, None) == -1
    assert lib.tucker_state_stats(None, None, None, None, None, None) == -1
    assert lib.tucker_state_copy_factor(None, 0, None, None) == -1
    assert b"NULL" in lib.fcoo_last_error()
    assert lib.spttmc_plan_destroy(None) == 0
    assert lib.fcoo_destroy(None) == 0


def test_noalloc_rejects_bad_arguments_without_device_work(fc):
    # every check of spmttkrp_noalloc runs on the host before any CUDA call,
    # so fake (never dereferenced) 256-byte-aligned addresses stand in for
    # the caller's device buffers
    from paper_1705_09905_gb300 import _lib

    lib = fc.lib
    fake = 1 << 20

    def view(**kw):
        v = _lib.FcooView()
        v.nmodes, v.mode, v.threadlen, v.nnz, v.nseg = 3, 0, 8, 1000, 10
        for k, d in enumerate((50, 40, 30)):
            v.dims[k] = d
        v.pidx[0] = v.pidx[1] = v.val = v.bf = v.sf = v.segrow = v.hcount = fake
        for k, x in kw.items():
            setattr(v, k, x)
        return v

    F = (ctypes.c_void_p * 3)(fake, fake, fake)
    Fp = ctypes.cast(F, ctypes.POINTER(ctypes.c_void_p))

    def call(v, R=32, out=fake, dtype=0):
        return lib.spmttkrp_noalloc(ctypes.byref(v), Fp, dtype, R, out, None)

    assert call(view(), out=fake + 2) == _lib.FCOO_ERR_INVALID_ARG  # out not 4-byte aligned
    assert b"aligned" in lib.fcoo_last_error()
    assert call(view(), out=None) == _lib.FCOO_ERR_INVALID_ARG
    assert call(view(mode=3)) == _lib.FCOO_ERR_INVALID_ARG
    assert call(view(nseg=51)) == _lib.FCOO_ERR_INVALID_ARG  # more segments than rows
    assert b"nseg" in lib.fcoo_last_error()
    assert call(view(threadlen=3)) == _lib.FCOO_ERR_INVALID_ARG
    assert call(view(), dtype=5) == _lib.FCOO_ERR_INVALID_ARG
    assert call(view(), R=_lib.NOALLOC_MAX_RANK + 8) == _lib.FCOO_ERR_UNSUPPORTED
    assert b"scratch limit" in lib.fcoo_last_error()


def test_header_is_plain_c_and_links(tmp_path):
    """include/fcoo.h compiles as strict C99 and a C program links against
    libfcoo.so and calls it (host-only entry points, and argument errors that
    are returned before any device work): the boundary needs no C++ or torch."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "abi.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "fcoo.h"
int main(void) {
    if (fcoo_version() <= 0) return 1;
    if (strcmp(fcoo_status_string(FCOO_ERR_INVALID_ARG), "") == 0) return 2;
    if (fcoo_table2_bytes(2, 32 * 8, 8) != (4 + 8) * 256 + 256 / 8 + 256 / 64) return 3;
    if (spmttkrp(NULL, NULL, FCOO_F32, 16, NULL, NULL) != FCOO_ERR_INVALID_ARG) return 4;
    if (spttmc(NULL, NULL, FCOO_F32, 4, NULL, NULL) != FCOO_ERR_INVALID_ARG) return 5;
    if (cp_als_iter(NULL, NULL, NULL) != FCOO_ERR_INVALID_ARG) return 6;
    if (tucker_hooi_iter(NULL, NULL, NULL) != FCOO_ERR_INVALID_ARG) return 7;
    if (strstr(fcoo_last_error(), "NULL") == NULL) return 8;
    printf("ok\n");
    return 0;
}
""")
    libdir = os.path.join(ROOT, "paper_1705_09905_gb300", "lib")
    exe = tmp_path / "abi"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           str(src), "-L", libdir, "-lfcoo", f"-Wl,-rpath,{libdir}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
