"""SpTTMc (Eq. 4, Table I row 3) through the C ABI vs the FP64 oracle, element
by element, on seeded inputs spanning several CTAs and ragged tails; every
lane layout (eight-column lanes for 3-way R = 8 and 16, four-column lanes for
R = 4, scalar lanes for the other ranks, for 2-way and 4-way tensors and for
factors that are not 32-byte aligned), BF16 factors, the edge cases (empty tensor, one hot
slice, rejected shapes), determinism; the by-fibre plan (SpTTM into fibre
sums, then Eq. 4 over the fibres) on every mode; and at the full skewed
3-way size in the launch configuration bench.py times: every column
r_a = r_b (the SpMTTKRP diagonal) of every row and every column of sampled
rows."""
import ctypes

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


def check_ttmc(fc, oracle, T, R, mode, tl=8, seed=1, factors=None, dtype=torch.float32):
    dims = T.dims
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), dims, mode, "mttkrp", tl)
    if factors is None:
        factors = [f.to(cuda()).to(dtype) for f in synth.make_factors(dims, R, seed=seed)]
    got = fc.spttmc(X, factors)
    torch.cuda.synchronize()
    Fh = host_factors(factors)
    idx = T.idx_u32()
    val = T.val.double().numpy()
    ref = oracle.ttmc(dims, idx, val, Fh, mode)
    absref = oracle.ttmc(dims, idx, np.abs(val), [np.abs(f) for f in Fh], mode)
    assert_close_abs(got.cpu().numpy(), ref, absref)
    return X, factors, got


@pytest.mark.parametrize("R", [4, 8, 16])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_tiny_config_vector_lanes(fc, oracle, R, mode):
    cfg = synth.CONFIGS["tiny"]
    T = synth.make_tensor(cfg)
    check_ttmc(fc, oracle, T, R, mode)


@pytest.mark.parametrize("R,mode", [(8, 0), (16, 1), (16, 2), (5, 0), (3, 2)])
def test_bf16_factors(fc, oracle, R, mode):
    # the oracle gets the same BF16-rounded factor values upcast to FP64
    T = synth.random_small((60, 50, 40), 8000, seed=40 + R)
    check_ttmc(fc, oracle, T, R, mode, dtype=torch.bfloat16)


@pytest.mark.parametrize("R", [1, 2, 3, 5, 10, 12, 15])
def test_scalar_lanes_3way(fc, oracle, R):
    T = synth.random_small((60, 50, 40), 6000, seed=R)
    check_ttmc(fc, oracle, T, R, R % 3)


@pytest.mark.parametrize("R,mode", [(2, 0), (4, 3), (6, 1)])
def test_4way(fc, oracle, R, mode):
    T = synth.random_small((30, 20, 25, 15), 6000, seed=11 + R)
    check_ttmc(fc, oracle, T, R, mode, tl=16)


def test_2way_is_spmm(fc, oracle):
    # one product mode: the output is the sparse matrix times the factor
    T = synth.random_small((300, 200), 5000, seed=5)
    X, factors, got = check_ttmc(fc, oracle, T, 24, 0)
    ref = fc.spmttkrp(X, factors)
    torch.cuda.synchronize()
    torch.testing.assert_close(got, ref, rtol=2e-5, atol=1e-5)


def test_unaligned_factors_take_scalar_lanes(fc, oracle):
    # factors as views one element into a buffer: not 32-byte aligned
    T = synth.random_small((70, 60, 50), 9000, seed=2)
    R = 8
    fs = []
    for f in synth.make_factors(T.dims, R, seed=3):
        buf = torch.empty(f.numel() + 1, dtype=torch.float32, device=cuda())
        v = buf[1:].view(f.shape)
        v.copy_(f.to(cuda()))
        fs.append(v)
    check_ttmc(fc, oracle, T, R, 1, factors=fs)


@pytest.mark.parametrize("R,tl", [(8, 8), (16, 32), (5, 8)])
def test_skewed_zipf_spanning_many_ctas(fc, oracle, R, tl):
    cfg = synth.scaled(synth.CONFIGS["skewed3"], 400_003, dims=(1200, 900, 2800))
    T = synth.make_tensor(cfg)
    for mode in range(3):
        check_ttmc(fc, oracle, T, R, mode, tl=tl)


def test_single_hot_slice_and_empty_rows(fc, oracle):
    n = 200_000
    rng = np.random.default_rng(4)
    lin = rng.choice(700 * 800, size=n, replace=False)
    j, k = np.unravel_index(lin, (700, 800))
    i = np.full(n, 37)
    T = synth.SparseTensor((64, 700, 800), [torch.from_numpy(a.astype(np.int64)) for a in (i, j, k)],
                           torch.from_numpy(rng.uniform(0.0, 1.0, n).astype(np.float32)))
    X, _, got = check_ttmc(fc, oracle, T, 16, 0)
    g = got.cpu()
    assert torch.all(g[:37] == 0) and torch.all(g[38:] == 0)


def test_single_nonzero_and_ragged_sizes(fc, oracle):
    for nnz in (1, 2, 31, 33, 1023, 2049, 4097):
        T = synth.random_small((20, 30, 40), nnz, seed=nnz)
        check_ttmc(fc, oracle, T, 8 if nnz % 2 else 6, nnz % 3)


def test_diagonal_is_spmttkrp_and_repeatable(fc, oracle):
    T = synth.random_small((80, 70, 60), 12000, seed=9)
    R = 8
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 2, "mttkrp", 8)
    F = [f.to(cuda()) for f in synth.make_factors(T.dims, R, seed=4)]
    Y1 = fc.spttmc(X, F)
    Y2 = fc.spttmc(X, F)
    M = fc.spmttkrp(X, F)
    torch.cuda.synchronize()
    assert torch.equal(Y1, Y2)
    diag = [r * R + r for r in range(R)]
    Fh = host_factors(F)
    absref = oracle.mttkrp(T.dims, T.idx_u32(), np.abs(T.val.double().numpy()), [np.abs(f) for f in Fh], 2)
    assert_close_abs(Y1[:, diag].cpu().numpy(), M.cpu().double().numpy(), absref)


def test_empty_tensor_writes_zeros(fc):
    X = fc.FCOO.build([np.zeros(0, np.uint32)] * 3, np.zeros(0, np.float32), (5, 6, 7), 1, "mttkrp", 8)
    F = [torch.ones(d, 4, device=cuda()) for d in (5, 6, 7)]
    out = torch.full((6, 16), 7.0, device=cuda())
    fc.spttmc(X, F, out=out)
    torch.cuda.synchronize()
    assert torch.all(out == 0)


def test_rejected_shapes(fc):
    lib = fc.lib
    T = synth.random_small((30, 20, 10), 500, seed=1)
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 0, "mttkrp", 8)
    Xt = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 0, "ttm", 8)
    out = torch.empty(30, 17 * 17, device=cuda())
    F = [torch.zeros(d, 17, device=cuda()) for d in T.dims]
    arr = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in F])
    assert lib.spttmc(X.handle, arr, fc.F32, 17, out.data_ptr(), None) == -9  # R^2 > 256: unsupported
    assert b"above" in lib.fcoo_last_error()
    assert lib.spttmc(Xt.handle, arr, fc.F32, 4, out.data_ptr(), None) == -1
    assert lib.spttmc(X.handle, arr, fc.F32, 0, out.data_ptr(), None) == -1
    assert lib.spttmc(X.handle, arr, fc.F32, 4, None, None) == -1


# ---------------------------------------------------------------- by fibres (SpTTMcPlan)


def check_plan(fc, oracle, T, R, mode, tl=8, seed=1, factors=None):
    b = 1 if mode == 2 else 2
    Xt = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, b, "ttm", tl)
    plan = fc.SpTTMcPlan(Xt, mode, R, tl)
    assert plan.nfib == Xt.nseg
    if factors is None:
        factors = [f.to(cuda()) for f in synth.make_factors(T.dims, R, seed=seed)]
    got = plan.run(factors)
    torch.cuda.synchronize()
    Fh = host_factors(factors)
    idx = T.idx_u32()
    val = T.val.double().numpy()
    ref = oracle.ttmc(T.dims, idx, val, Fh, mode)
    absref = oracle.ttmc(T.dims, idx, np.abs(val), [np.abs(f) for f in Fh], mode)
    assert_close_abs(got.cpu().numpy(), ref, absref)
    return plan, factors, got


@pytest.mark.parametrize("R", [1, 4, 5, 8, 16])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_plan_every_mode(fc, oracle, R, mode):
    T = synth.random_small((60, 50, 40), 12000, seed=30 + R)
    check_plan(fc, oracle, T, R, mode)


@pytest.mark.parametrize("R,tl", [(16, 8), (8, 32)])
def test_plan_skewed_long_fibres(fc, oracle, R, tl):
    # Zipf indices: long fibres and hot slices spanning many CTAs
    cfg = synth.scaled(synth.CONFIGS["skewed3"], 400_003, dims=(300, 200, 2800))
    T = synth.make_tensor(cfg)
    for mode in range(3):
        check_plan(fc, oracle, T, R, mode, tl=tl)


def test_plan_single_nonzero_and_empty(fc, oracle):
    T = synth.random_small((20, 30, 40), 1, seed=1)
    check_plan(fc, oracle, T, 8, 1)
    Xt = fc.FCOO.build([np.zeros(0, np.uint32)] * 3, np.zeros(0, np.float32), (5, 6, 7), 2, "ttm", 8)
    plan = fc.SpTTMcPlan(Xt, 0, 4)
    assert plan.nfib == 0
    out = torch.full((5, 16), 3.0, device=cuda())
    plan.run([None, torch.ones(6, 4, device=cuda()), torch.ones(7, 4, device=cuda())], out=out)
    torch.cuda.synchronize()
    assert torch.all(out == 0)


def test_plan_rejects(fc):
    lib = fc.lib
    T = synth.random_small((30, 20, 10), 500, seed=1)
    Xm = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 0, "mttkrp", 8)
    X0 = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 0, "ttm", 8)
    X2 = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 2, "ttm", 8)
    for X, mode, R in ((Xm, 0, 8), (X0, 0, 8), (X2, 2, 8), (X2, 3, 8)):
        with pytest.raises(fc.FcooError) as e:
            fc.SpTTMcPlan(X, mode, R)
        assert e.value.status == -1
    with pytest.raises(fc.FcooError) as e:
        fc.SpTTMcPlan(X2, 0, 17)
    assert e.value.status == -9
    plan = fc.SpTTMcPlan(X2, 1, 4)
    F = [torch.zeros(d, 4, device=cuda()) for d in T.dims]
    arr = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in F])
    out = torch.empty(20, 16, device=cuda())
    assert lib.spttmc_plan_run(plan._h, arr, fc.BF16, out.data_ptr(), None) == -9
    arr2 = (ctypes.c_void_p * 3)(F[0].data_ptr(), F[1].data_ptr(), None)
    assert lib.spttmc_plan_run(plan._h, arr2, fc.F32, out.data_ptr(), None) == -1


# ---------------------------------------------------------------- full size


def test_spttmc_full_size_sampled_rows(fc, oracle):
    """The skewed 3-way tensor (76M nonzeros) at R = 16 (256 output columns)
    and R = 8, mode 0, as bench.py runs it (spttmc, and the by-fibre plan at
    R = 16): the r_a = r_b columns of every row against the FP64 SpMTTKRP,
    and all columns of 48 sampled rows (uniform over the rows, plus the 50th
    and 500th hottest) against the oracle on the nonzeros of those rows."""
    cfg = synth.CONFIGS["skewed3"]
    dev = torch.device("cuda", 0)
    T = synth.make_tensor(cfg, device=dev)
    X = fc.FCOO.build([a.to(torch.int32).contiguous() for a in T.idx], T.val, cfg.dims, 0, "mttkrp", 8)
    idx = [a.cpu().numpy().astype(np.uint32) for a in T.idx]
    val = T.val.double().cpu().numpy()
    counts = np.bincount(idx[0], minlength=cfg.dims[0])
    order = np.argsort(-counts, kind="stable")
    rng = np.random.default_rng(12)
    rows = np.unique(np.concatenate([rng.choice(cfg.dims[0], 46, replace=False), order[[50, 500]]]))
    sel = np.isin(idx[0], rows)
    sidx = [a[sel] for a in idx]
    sval = val[sel]
    Xt = fc.FCOO.build([a.to(torch.int32).contiguous() for a in T.idx], T.val, cfg.dims, 2, "ttm", 8)
    del T
    plan = fc.SpTTMcPlan(Xt, 0, 16)
    try:
        for R in (16, 8):
            F = [f.to(dev) for f in synth.make_factors(cfg.dims, R, seed=R)]
            Fh = host_factors(F)
            absF = [np.abs(f) for f in Fh]
            Ys = [fc.spttmc(X, F)] + ([plan.run(F)] if R == 16 else [])
            torch.cuda.synchronize()
            diag = [r * R + r for r in range(R)]
            ref = oracle.mttkrp(cfg.dims, idx, val, Fh, 0)
            absref = oracle.mttkrp(cfg.dims, idx, np.abs(val), absF, 0)
            sref = oracle.ttmc(cfg.dims, sidx, sval, Fh, 0)[rows]
            sabs = oracle.ttmc(cfg.dims, sidx, np.abs(sval), absF, 0)[rows]
            for Y in Ys:
                assert_close_abs(Y[:, diag].cpu().numpy(), ref, absref)
                assert_close_abs(Y[torch.from_numpy(rows).to(dev)].cpu().numpy(), sref, sabs)
            del Ys
    finally:
        plan.close()
        Xt.close()
        X.close()
        torch.cuda.empty_cache()
