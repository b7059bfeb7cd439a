"""spmttkrp_gather_bound: the factor-row loads of SpMTTKRP (Eq. 6) on a 3-way
handle and nothing else, a measurement aid for the gather bound.  Its only
result is the number of rows it loaded, which is checked against the rows
SpMTTKRP must read, counted on the host from the F-COO layout: one C row per
nonzero, and one B row wherever the first product-mode index changes or a
segment starts.  A lane group also loads a B row where its range of nonzeros
starts, so the count may exceed that by at most one per extra range; a
tensor of at most 32 nonzeros is one range and is counted exactly.  Also the
rejected shapes and arguments."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from helpers import cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import paper_1705_09905_gb300 as fc

    return fc


def rows_needed(X):
    """C rows (one per nonzero) plus B rows (first nonzero, index change or
    segment head) from the handle's layout."""
    lay = X.layout()
    n = X.nnz
    j = lay["pidx"][0].astype(np.int64)
    heads = np.unpackbits(lay["bf"].view(np.uint8), bitorder="little")[:n].astype(bool)
    change = np.ones(n, bool)
    change[1:] = j[1:] != j[:-1]
    return n + int(np.count_nonzero(change | heads))


@pytest.mark.parametrize("R,dtype", [(32, torch.float32), (8, torch.float32), (16, torch.float32),
                                     (64, torch.float32), (128, torch.float32), (256, torch.float32),
                                     (32, torch.bfloat16), (64, torch.bfloat16)])
def test_rows_loaded(fc, R, dtype):
    T = synth.make_tensor(synth.scaled(synth.CONFIGS["skewed3"], 200_003, dims=(1200, 900, 2800)))
    F = [f.to(cuda()).to(dtype) for f in synth.make_factors(T.dims, R, seed=1)]
    for mode in range(3):
        X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, mode, "mttkrp", 8)
        need = rows_needed(X)
        got = int(fc.spmttkrp_gather_bound(X, F).item())
        nchunk = (X.nnz + 31) // 32
        assert need <= got <= need + nchunk, (mode, need, got)
        X.close()


@pytest.mark.parametrize("nnz", [1, 7, 32])
def test_one_range_is_exact(fc, nnz):
    T = synth.random_small((40, 30, 20), nnz, seed=nnz)
    F = [f.to(cuda()) for f in synth.make_factors(T.dims, 32, seed=2)]
    for mode in range(3):
        X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, mode, "mttkrp", 8)
        assert int(fc.spmttkrp_gather_bound(X, F).item()) == rows_needed(X)
        X.close()


def test_rejected(fc):
    from paper_1705_09905_gb300 import _lib

    lib = fc.lib
    cnt = torch.zeros(1, dtype=torch.int64, device=cuda())
    s = torch.cuda.current_stream().cuda_stream

    def call(X, F, R, dtype=fc.F32, count=None):
        ptrs = (ctypes.c_void_p * len(F))(*[f.data_ptr() if f is not None else None for f in F])
        return lib.spmttkrp_gather_bound(X.handle, ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)), dtype, R,
                                         cnt.data_ptr() if count is None else count, s)

    T4 = synth.random_small((20, 20, 20, 20), 500, seed=1)
    F4 = [torch.zeros(d, 32, device=cuda()) for d in T4.dims]
    X4 = fc.FCOO.build(T4.idx_u32(), T4.val.numpy(), T4.dims, 0, "mttkrp", 8)
    assert call(X4, F4, 32) == _lib.FCOO_ERR_UNSUPPORTED
    X4.close()
    T = synth.random_small((50, 40, 30), 2000, seed=3)
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 1, "mttkrp", 8)
    F24 = [torch.zeros(d, 24, device=cuda()) for d in T.dims]
    assert call(X, F24, 24) == _lib.FCOO_ERR_UNSUPPORTED
    F = [torch.zeros(d, 32, device=cuda()) for d in T.dims]
    assert call(X, F, 32, count=0) == _lib.FCOO_ERR_INVALID_ARG
    assert call(X, F, 32, count=cnt.data_ptr() + 4) == _lib.FCOO_ERR_INVALID_ARG
    assert call(X, [F[0], None, None], 32) == _lib.FCOO_ERR_INVALID_ARG
    # a factor whose rows start off the 32-byte lane boundary
    Fs = torch.zeros(T.dims[0] * 32 + 1, device=cuda())[1:].view(T.dims[0], 32)
    assert call(X, [Fs, None, F[2]], 32) == _lib.FCOO_ERR_UNSUPPORTED
    assert call(X, F, 32) == 0
    torch.cuda.synchronize()
    assert int(cnt.item()) >= X.nnz
    Y = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 0, "ttm", 8)
    assert call(Y, F, 32) == _lib.FCOO_ERR_INVALID_ARG
    Y.close()
    X.close()
