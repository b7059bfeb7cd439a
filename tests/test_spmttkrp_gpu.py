"""SpMTTKRP (Eq. 6) and SpTTM (Eq. 3) through the C ABI vs the FP64 oracle,
element by element, on seeded inputs spanning several CTAs and ragged tails."""
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


def run_mttkrp(fc, oracle, T, R, mode, dtype=torch.float32, tl=8, seed=1, factors=None):
    dims = T.dims
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), dims, mode, "mttkrp", tl)
    if factors is None:
        factors = [f.to(cuda()).to(dtype) for f in synth.make_factors(dims, R, seed=seed)]
    got = fc.spmttkrp(X, factors)
    torch.cuda.synchronize()
    Fh = host_factors(factors)
    idx = T.idx_u32()
    val = T.val.double().numpy()
    ref = oracle.mttkrp(dims, idx, val, Fh, mode)
    absref = oracle.mttkrp(dims, idx, np.abs(val), [np.abs(f) for f in Fh], mode)
    assert_close_abs(got.cpu().numpy(), ref, absref)
    return X, factors, got


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_tiny_config_all_modes(fc, oracle, mode):
    cfg = synth.CONFIGS["tiny"]
    T = synth.make_tensor(cfg)
    run_mttkrp(fc, oracle, T, cfg.R, mode)


@pytest.mark.parametrize("R", [1, 3, 4, 8, 16, 24, 32, 40, 64, 100, 128, 200, 256])
def test_ranks(fc, oracle, R):
    T = synth.random_small((60, 50, 40), 8000, seed=R)
    run_mttkrp(fc, oracle, T, R, R % 3)


@pytest.mark.parametrize("R", [8, 16, 32, 64, 6, 33])
def test_bf16_factors(fc, oracle, R):
    # oracle gets the same bf16-rounded factor values upcast to FP64
    T = synth.random_small((60, 50, 40), 8000, seed=100 + R)
    run_mttkrp(fc, oracle, T, R, 1, dtype=torch.bfloat16)


@pytest.mark.parametrize("R", [32, 64])
def test_bf16_skewed_many_ctas(fc, oracle, R):
    # the BF16 value pass (four-nonzero quarters) over a Zipf tensor large
    # enough for every CTA, run and stage, with a ragged last stage, all modes
    T = synth.make_tensor(synth.scaled(synth.CONFIGS["skewed3"], 1_000_003, dims=(3000, 2000, 5000)))
    for mode in range(3):
        run_mttkrp(fc, oracle, T, R, mode, dtype=torch.bfloat16, seed=R)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_4way(fc, oracle, mode):
    T = synth.random_small((30, 20, 25, 15), 9000, seed=7 + mode)
    run_mttkrp(fc, oracle, T, 16, mode, tl=16)


def test_5way_runtime_product_count(fc, oracle):
    T = synth.random_small((9, 8, 7, 6, 5), 4000, seed=3)
    run_mttkrp(fc, oracle, T, 8, 2)


def test_skewed_zipf_spanning_many_ctas(fc, oracle):
    # one hot slice holds a large share: its segment spans many CTAs
    cfg = synth.scaled(synth.CONFIGS["skewed3"], 1_500_003, dims=(1200, 900, 2800))
    T = synth.make_tensor(cfg)
    for mode in range(3):
        run_mttkrp(fc, oracle, T, 32, mode)


def test_single_slice_and_empty_slices(fc, oracle):
    # all nonzeros in one slice (one segment spanning the whole grid), other rows empty
    n = 300_000
    rng = np.random.default_rng(0)
    lin = rng.choice(700 * 800, size=n, replace=False)
    j, k = np.unravel_index(lin, (700, 800))
    T = synth.SparseTensor((50, 700, 800), [torch.full((n,), 17), torch.as_tensor(j), torch.as_tensor(k)],
                           torch.rand(n, generator=torch.Generator().manual_seed(1)))
    _, _, got = run_mttkrp(fc, oracle, T, 32, 0)
    g = got.cpu().numpy()
    assert np.count_nonzero(g[:17]) == 0 and np.count_nonzero(g[18:]) == 0
    # sparse rows: most slices empty
    T = synth.random_small((5000, 30, 30), 3000, seed=9)
    run_mttkrp(fc, oracle, T, 16, 0)


def test_single_nonzero_and_ragged_sizes(fc, oracle):
    for nnz in (1, 2, 31, 33, 1023, 2049, 4097):
        T = synth.random_small((20, 30, 40), nnz, seed=nnz)
        run_mttkrp(fc, oracle, T, 16, nnz % 3)


@pytest.mark.parametrize("tl", [1, 2, 4, 8, 16, 32, 64])
def test_threadlen_values(fc, oracle, tl):
    T = synth.random_small((100, 90, 80), 50_000, seed=tl)
    run_mttkrp(fc, oracle, T, 32, 0, tl=tl)


@pytest.mark.parametrize("R,dtype", [(32, torch.float32), (16, torch.float32), (64, torch.bfloat16)])
def test_deterministic_rows_and_output_overwrite(fc, oracle, R, dtype):
    # the header promises bitwise identical results for repeated calls: a
    # multi-CTA launch (segments cut by runs and CTAs, carries combined in a
    # fixed order), compared bit for bit, into an output pre-filled with NaN
    T = synth.make_tensor(synth.scaled(synth.CONFIGS["skewed3"], 600_001, dims=(800, 700, 900)))
    X, F, a = run_mttkrp(fc, oracle, T, R, 2, dtype=dtype)
    assert X.nnz > 64 * 32 * 2  # several CTAs at this size
    for _ in range(2):
        out = torch.full_like(a, float("nan"))
        b = fc.spmttkrp(X, F, out=out)
        torch.cuda.synchronize()
        assert torch.isfinite(b).all()
        assert np.array_equal(a.cpu().numpy().view(np.uint32), b.cpu().numpy().view(np.uint32))


# ---------------------------------------------------------------- SpTTM


def run_ttm(fc, oracle, T, R, mode, dtype=torch.float32, tl=8):
    dims = T.dims
    X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), dims, mode, "ttm", tl)
    U = synth.make_factors([dims[mode]], R, seed=11)[0].to(cuda()).to(dtype)
    got = fc.spttm(X, U)
    torch.cuda.synchronize()
    idx = T.idx_u32()
    val = T.val.double().numpy()
    Uh = host_factors([U])[0]
    keys, ref = oracle.ttm(dims, idx, val, Uh, mode)
    _, absref = oracle.ttm(dims, idx, np.abs(val), np.abs(Uh), mode)
    np.testing.assert_array_equal(X.fibre_indices(), keys)
    assert_close_abs(got.cpu().numpy(), ref, absref)


@pytest.mark.parametrize("R,dtype", [(32, torch.float32), (16, torch.float32), (32, torch.bfloat16)])
def test_unaligned_factor_rows_take_the_scalar_path(fc, oracle, R, dtype):
    # factor storage starting 4 (2) bytes past an aligned address: the vector
    # lane layouts need 16/32-byte aligned rows, so the scalar lanes run
    T = synth.make_tensor(synth.scaled(synth.CONFIGS["skewed3"], 200_000, dims=(300, 200, 400)))
    base = synth.make_factors(T.dims, R, seed=6)
    factors = []
    for f in base:
        buf = torch.empty(f.numel() + 1, dtype=dtype, device="cuda")
        v = buf[1:].view(f.shape)
        v.copy_(f.to(dtype))
        assert v.data_ptr() % 16 != 0
        factors.append(v)
    for mode in range(3):
        run_mttkrp(fc, oracle, T, R, mode, dtype=dtype, factors=factors)


def test_ttm_tiny_config(fc, oracle):
    cfg = synth.CONFIGS["tiny"]
    run_ttm(fc, oracle, synth.make_tensor(cfg), 16, 2)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_ttm_4way_zipf(fc, oracle, mode):
    cfg = synth.scaled(synth.CONFIGS["ttm4"], 400_000, dims=(500, 400, 300, 5000))
    run_ttm(fc, oracle, synth.make_tensor(cfg), 16, mode)


@pytest.mark.parametrize("R,dtype", [(1, torch.float32), (7, torch.float32), (16, torch.bfloat16),
                                     (32, torch.bfloat16), (64, torch.bfloat16), (64, torch.float32),
                                     (256, torch.float32)])
def test_ttm_ranks(fc, oracle, R, dtype):
    T = synth.random_small((40, 30, 50), 12_000, seed=R)
    run_ttm(fc, oracle, T, R, 2, dtype=dtype)


@pytest.mark.parametrize("R,dtype", [(16, torch.float32), (64, torch.bfloat16)])
def test_ttm_one_long_fibre(fc, oracle, R, dtype):
    n = 200_000
    k = np.random.default_rng(1).choice(1_000_000, size=n, replace=False)
    T = synth.SparseTensor((3, 4, 1_000_000), [torch.full((n,), 2), torch.full((n,), 3), torch.as_tensor(k)],
                           torch.rand(n, generator=torch.Generator().manual_seed(2)))
    run_ttm(fc, oracle, T, R, 2, dtype=dtype)
