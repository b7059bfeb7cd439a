"""spmttkrp_noalloc: SpMTTKRP for callers that must not allocate device memory
while they run (their memory is reserved up front by a framework allocator or
a fixed arena, or allocation after start-up is forbidden).  The caller passes
the F-COO layout in buffers it owns; the entry point keeps its carry scratch
in a fixed array inside the library.  Checked through the C ABI against the
regular spmttkrp on the same layout, on two calls in a row (the second call
finds the first call's leftovers in the shared scratch).

This file is collected last (tests/test_zz_*), so a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from helpers import REL_FRO, cuda, rel_fro

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
    st = fc.lib.spmttkrp_noalloc(ctypes.byref(v), ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)), dtype, R,
                                 out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_noalloc_matches_spmttkrp_on_two_calls(dtype):
    import paper_1705_09905_gb300 as fc

    cfg = synth.scaled(synth.CONFIGS["skewed3"], 400_003, dims=(1200, 900, 2800))
    T = synth.make_tensor(cfg)
    R = 32
    F = [f.to(cuda()).to(dtype) for f in synth.make_factors(cfg.dims, R, seed=1)]
    code = fc.BF16 if dtype == torch.bfloat16 else fc.F32
    for mode in (0, 2):
        X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), cfg.dims, mode, "mttkrp", 8)
        ref = fc.spmttkrp(X, F)
        keep = []
        v = _view(fc, X, keep)
        fl = [None if k == mode else F[k] for k in range(3)]
        for call in range(2):
            out = torch.full((cfg.dims[mode], R), float("nan"), device=cuda())
            assert _call(fc, v, fl, R, code, out) == 0, fc.lib.fcoo_last_error()
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert rel_fro(out.cpu().numpy(), ref.cpu().numpy()) <= REL_FRO, (mode, call)
        del keep


def test_noalloc_rejects_ranks_over_its_scratch():
    import paper_1705_09905_gb300 as fc

    T = synth.random_small((50, 40, 30), 2000, seed=3)
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 1, "mttkrp", 8)
    keep = []
    v = _view(fc, X, keep)
    R = fc.lib.spmttkrp_noalloc and 136  # over FCOO_NOALLOC_MAX_RANK (128)
    F = [torch.zeros(d, R, device=cuda()) for d in T.dims]
    out = torch.empty(T.dims[1], R, device=cuda())
    assert _call(fc, v, [F[0], None, F[2]], R, fc.F32, out) == -9
    assert b"scratch limit" in fc.lib.fcoo_last_error()
