"""spmttkrp_noalloc: SpMTTKRP for callers that must not allocate device memory
while they run (their memory is reserved up front by a framework allocator or
a fixed arena, or allocation after start-up is forbidden).  The caller passes
the F-COO layout in buffers it owns; the entry point keeps its carry scratch
in a fixed array inside the library.

Checked through the C ABI, on two calls in a row (the second call finds the
first call's leftovers in the shared scratch), element by element against the
FP64 oracle and against the regular spmttkrp on the same layout: 2-, 3- and
4-way tensors (each takes a different instantiation of the streaming kernel),
R = 8 (four-column lanes), 32 (eight-column lanes) and 128 (the largest rank
the scratch holds), FP32 and BF16 factors.

This file is collected last (tests/test_zz_*), so a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from helpers import REL_FRO, assert_close_abs, cuda, host_factors, rel_fro

pytestmark = pytest.mark.gpu


def _view(fc, X, keep):
    """Copy X's layout into fresh caller-owned device buffers and describe them."""
    lay = X.layout()
    n = X.nnz
    npad = ((n + 31) // 32) * 32
    dev = cuda()

    def dev_u32(a, length):
        t = torch.zeros(max(length, 4), dtype=torch.int32, device=dev)
        t[: len(a)] = torch.as_tensor(a.view(np.int32))
        keep.append(t)
        return t.data_ptr()

    bf = lay["bf"]
    nchunk = (n + 1023) // 1024
    pop = np.array([bin(int(w)).count("1") for w in bf], dtype=np.int64)
    csum = np.concatenate([[0], np.cumsum(pop)])
    hcount = np.array([csum[min(32 * c, len(bf))] for c in range(nchunk + 1)], dtype=np.uint32)
    v = fc._lib.FcooView()
    v.nmodes, v.mode, v.threadlen = X.nmodes, X.mode, X.threadlen
    v.nnz, v.nseg = n, X.nseg
    for k, d in enumerate(X.dims):
        v.dims[k] = d
    for m in range(len(X.prod_modes)):
        v.pidx[m] = dev_u32(lay["pidx"][m], npad)
    v.val = dev_u32(lay["val"].view(np.uint32), npad)
    v.bf = dev_u32(bf, len(bf))
    v.sf = dev_u32(lay["sf"], len(lay["sf"]))
    v.segrow = dev_u32(lay["segkeys"][:, 0].copy(), X.nseg)
    v.hcount = dev_u32(hcount, len(hcount))
    return v


def _call(fc, v, F, R, dtype, out):
    ptrs = (ctypes.c_void_p * len(F))(*[f.data_ptr() if f is not None else None for f in F])
    return fc.lib.spmttkrp_noalloc(ctypes.byref(v), ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)), dtype, R,
                                   out.data_ptr(), torch.cuda.current_stream().cuda_stream)


CASES = [
    # (name, dims, nnz, mode, R, factor dtype)
    ("3-way Zipf, R=32", (1200, 900, 2800), 400_003, 0, 32, torch.float32),
    ("3-way Zipf, R=32, last mode", (1200, 900, 2800), 400_003, 2, 32, torch.float32),
    ("3-way Zipf, R=32, BF16", (1200, 900, 2800), 400_003, 1, 32, torch.bfloat16),
    ("3-way Zipf, R=8", (1200, 900, 2800), 300_001, 1, 8, torch.float32),
    ("3-way Zipf, R=128", (1200, 900, 2800), 200_003, 0, 128, torch.float32),
    ("2-way, R=8", (3000, 2500), 150_001, 1, 8, torch.float32),
    ("2-way, R=32", (3000, 2500), 150_001, 0, 32, torch.float32),
    ("4-way, R=32", (60, 50, 40, 30), 100_003, 2, 32, torch.float32),
    ("4-way, R=128", (60, 50, 40, 30), 60_001, 3, 128, torch.float32),
]


@pytest.mark.parametrize("name,dims,nnz,mode,R,dtype", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_oracle_and_spmttkrp_on_two_calls(oracle, name, dims, nnz, mode, R, dtype):
    import paper_1705_09905_gb300 as fc

    if len(dims) == 3:
        T = synth.make_tensor(synth.scaled(synth.CONFIGS["skewed3"], nnz, dims=dims))
    else:
        T = synth.random_small(dims, nnz, seed=len(dims) * 10 + mode)
    F = [f.to(cuda()).to(dtype) for f in synth.make_factors(dims, R, seed=1)]
    code = fc.BF16 if dtype == torch.bfloat16 else fc.F32
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), dims, mode, "mttkrp", 8)
    ref_dev = fc.spmttkrp(X, F).cpu().numpy()
    # the oracle is fed the exact stored factor values (BF16-rounded for BF16)
    Fh = host_factors(F)
    idx = T.idx_u32()
    val = T.val.double().numpy()
    ref = oracle.mttkrp(dims, idx, val, Fh, mode)
    absref = oracle.mttkrp(dims, idx, np.abs(val), [np.abs(f) for f in Fh], mode)
    keep = []
    v = _view(fc, X, keep)
    fl = [None if k == mode else F[k] for k in range(len(dims))]
    for call in range(2):
        out = torch.full((dims[mode], R), float("nan"), device=cuda())
        assert _call(fc, v, fl, R, code, out) == 0, fc.lib.fcoo_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), (name, call)
        assert_close_abs(got, ref, absref)
        assert rel_fro(got, ref_dev) <= REL_FRO, (name, call)
    del keep


def test_noalloc_rejects_ranks_over_its_scratch():
    import paper_1705_09905_gb300 as fc
    from paper_1705_09905_gb300 import _lib

    T = synth.random_small((50, 40, 30), 2000, seed=3)
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 1, "mttkrp", 8)
    keep = []
    v = _view(fc, X, keep)
    R = _lib.NOALLOC_MAX_RANK + 8
    F = [torch.zeros(d, R, device=cuda()) for d in T.dims]
    out = torch.empty(T.dims[1], R, device=cuda())
    assert _call(fc, v, [F[0], None, F[2]], R, fc.F32, out) == _lib.FCOO_ERR_UNSUPPORTED
    assert b"scratch limit" in fc.lib.fcoo_last_error()
