"""Index compression (Table II with 16-bit product-mode indices): handles after
fcoo_compress_indices, through the C ABI, against the same handles before it
(bitwise: the kernel sums the same terms in the same order, only the index
loads differ) and against the FP64 oracle element by element.  Covers every
mode of a 3-way tensor, every lane layout that takes the 16-bit streams
(eight FP32 columns per lane for R = 24..256, four for R = 16, BF16 rows),
ragged tails and threadlen values, SpTTM of a 4-way tensor, a CP-ALS sweep,
indices at the 16-bit limit, and the rejected shapes."""
import numpy as np
import pytest
import torch

import synth
from helpers import assert_close_abs, cuda, host_factors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import paper_1705_09905_gb300 as fc

    return fc


def bits(t):
    return t.cpu().numpy().view(np.uint32)


def oracle_check(oracle, T, F, mode, got):
    Fh = host_factors(F)
    idx, val = T.idx_u32(), T.val.double().numpy()
    ref = oracle.mttkrp(T.dims, idx, val, Fh, mode)
    absref = oracle.mttkrp(T.dims, idx, np.abs(val), [np.abs(f) for f in Fh], mode)
    assert_close_abs(got.cpu().numpy(), ref, absref)


@pytest.mark.parametrize("R,dtype", [(32, torch.float32), (16, torch.float32), (64, torch.float32),
                                     (24, torch.float32), (256, torch.float32), (32, torch.bfloat16),
                                     (64, torch.bfloat16)])
def test_spmttkrp_compressed_is_bitwise_and_matches_oracle(fc, oracle, R, dtype):
    T = synth.make_tensor(synth.scaled(synth.CONFIGS["skewed3"], 300_007, dims=(1200, 900, 2800)))
    F = [f.to(cuda()).to(dtype) for f in synth.make_factors(T.dims, R, seed=1)]
    for mode in range(3):
        X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, mode, "mttkrp", 8)
        a = fc.spmttkrp(X, F)
        X.compress_indices()
        assert X.compressed and X.bytes["pidx16"] == 2 * 2 * X.nnz
        b = fc.spmttkrp(X, F)
        torch.cuda.synchronize()
        assert np.array_equal(bits(a), bits(b)), (R, mode)
        oracle_check(oracle, T, F, mode, b)
        X.close()


@pytest.mark.parametrize("nnz,tl", [(1, 8), (33, 8), (4097, 16), (70_001, 1), (70_001, 64)])
def test_ragged_sizes_and_threadlen(fc, oracle, nnz, tl):
    T = synth.random_small((300, 200, 400), nnz, seed=nnz + tl)
    F = [f.to(cuda()) for f in synth.make_factors(T.dims, 32, seed=2)]
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, nnz % 3, "mttkrp", tl)
    a = fc.spmttkrp(X, F)
    X.compress_indices()
    b = fc.spmttkrp(X, F)
    torch.cuda.synchronize()
    assert np.array_equal(bits(a), bits(b))
    oracle_check(oracle, T, F, nnz % 3, b)


def test_indices_at_the_16_bit_limit(fc, oracle):
    # product-mode dimensions of exactly 65,536: the largest index is 0xffff
    n = 20_000
    rng = np.random.default_rng(5)
    idx = [rng.integers(0, 50, n), rng.integers(0, 65536, n), rng.integers(0, 65536, n)]
    idx[1][:3] = 65535
    idx[2][:3] = [65535, 0, 65534]
    lin = (idx[0] * 65536 + idx[1]) * 65536 + idx[2]
    _, keep = np.unique(lin, return_index=True)
    T = synth.SparseTensor((50, 65536, 65536), [torch.as_tensor(a[keep]) for a in idx],
                           torch.rand(len(keep), generator=torch.Generator().manual_seed(3)))
    F = [f.to(cuda()) for f in synth.make_factors(T.dims, 16, seed=4)]
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 0, "mttkrp", 8)
    a = fc.spmttkrp(X, F)
    X.compress_indices()
    b = fc.spmttkrp(X, F)
    torch.cuda.synchronize()
    assert np.array_equal(bits(a), bits(b))
    oracle_check(oracle, T, F, 0, b)


@pytest.mark.parametrize("mode", [0, 3])
def test_spttm_compressed(fc, oracle, mode):
    cfg = synth.scaled(synth.CONFIGS["ttm4"], 300_000, dims=(500, 400, 300, 5000))
    T = synth.make_tensor(cfg)
    U = synth.make_factors([cfg.dims[mode]], 16, seed=11)[0].to(cuda())
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), cfg.dims, mode, "ttm", 8)
    a = fc.spttm(X, U)
    X.compress_indices()
    assert X.bytes["pidx16"] == 2 * X.nnz
    b = fc.spttm(X, U)
    torch.cuda.synchronize()
    assert np.array_equal(bits(a), bits(b))
    idx, val = T.idx_u32(), T.val.double().numpy()
    Uh = host_factors([U])[0]
    keys, ref = oracle.ttm(cfg.dims, idx, val, Uh, mode)
    _, absref = oracle.ttm(cfg.dims, idx, np.abs(val), np.abs(Uh), mode)
    np.testing.assert_array_equal(X.fibre_indices(), keys)
    assert_close_abs(b.cpu().numpy(), ref, absref)


def test_cp_als_sweep_on_compressed_handles(fc):
    cfg = synth.CONFIGS["tiny"]
    T = synth.make_tensor(cfg)
    init = synth.make_factors(T.dims, 8, seed=3, kind="uniform")
    runs = []
    for compress in (False, True):
        Xs = [fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, n, "mttkrp", 8) for n in range(3)]
        if compress:
            for X in Xs:
                X.compress_indices()
        st = fc.CPState(T.dims, 8, init)
        st.iterate(Xs, sweeps=3)
        runs.append((st.stats()["fit"], [st.factor(k).cpu().numpy() for k in range(3)]))
        st.close()
    assert runs[0][0] == runs[1][0]
    for a, b in zip(runs[0][1], runs[1][1]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_rejected_and_repeated(fc):
    from paper_1705_09905_gb300 import _lib

    T = synth.random_small((40, 70_000, 30), 5000, seed=8)
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 0, "mttkrp", 8)
    with pytest.raises(fc.FcooError) as e:
        X.compress_indices()
    assert e.value.status == _lib.FCOO_ERR_UNSUPPORTED
    assert not X.compressed
    # the index mode may be wide: only product modes are narrowed
    X1 = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 1, "mttkrp", 8)
    X1.compress_indices()
    X1.compress_indices()  # a second call is a no-op
    assert X1.bytes["pidx16"] == 2 * 2 * X1.nnz
