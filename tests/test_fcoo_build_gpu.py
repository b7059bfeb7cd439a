"""F-COO layout built on the GPU vs the oracle's definition (Sec. IV-B,
Table I, Fig. 2): bit-exact permutation, flags, start-flags and segment keys;
Table II byte counts; error statuses."""
import json
import os

import numpy as np
import pytest
import torch

import synth
from helpers import cuda

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def fc():
    import paper_1705_09905_gb300 as fc

    return fc


def unpack_bits(words, n):
    return ((words[np.arange(n) // 32] >> (np.arange(n) % 32).astype(np.uint32)) & 1).astype(np.uint8)


def check_against_oracle(fc, oracle, dims, idx, val, mode, op, tl, device_inputs=False):
    ins = [torch.as_tensor(a.astype(np.int64)).to(cuda()) for a in idx] if device_inputs else idx
    v = torch.as_tensor(val).to(cuda()) if device_inputs else val
    X = fc.FCOO.build(ins, v, dims, mode, op, tl)
    lay = X.layout()
    ref = oracle.fcoo_layout(dims, idx, mode, op, tl)
    n = len(val)
    np.testing.assert_array_equal(lay["perm"], ref["perm"])
    np.testing.assert_array_equal(unpack_bits(lay["bf"], n), ref["head"])
    npart = (n + tl - 1) // tl
    np.testing.assert_array_equal(unpack_bits(lay["sf"], npart), ref["sf"])
    np.testing.assert_array_equal(lay["segkeys"], ref["segkeys"])
    assert X.nseg == ref["nseg"]
    for m, k in enumerate(X.prod_modes):
        np.testing.assert_array_equal(lay["pidx"][m], idx[k][ref["perm"]])
    np.testing.assert_array_equal(lay["val"], np.asarray(val, np.float32)[ref["perm"]])
    return X


def test_golden_fig2(fc, oracle):
    g = json.load(open(os.path.join(GOLD, "fig2_fcoo_3x3x3.json")))
    coords = np.array(g["coords_input_order"], dtype=np.uint32)
    idx = [coords[:, k].copy() for k in range(3)]
    val = np.array(g["vals_input_order"], np.float32)
    for key, op, mode in (("mttkrp_mode0", "mttkrp", 0), ("ttm_mode2", "ttm", 2)):
        X = check_against_oracle(fc, oracle, g["dims"], idx, val, mode, op, g["threadlen"])
        assert list(unpack_bits(X.layout()["bf"], 12)) == g[key]["head"]


@pytest.mark.parametrize("dims,nnz,mode,op,tl", [
    ((200, 150, 100), 10_000, 0, "mttkrp", 8),
    ((200, 150, 100), 10_000, 1, "mttkrp", 16),
    ((200, 150, 100), 10_000, 2, "ttm", 32),
    ((40, 30, 20, 50), 20_001, 3, "ttm", 64),
    ((40, 30, 20, 50), 20_001, 2, "mttkrp", 8),
    ((3, 70_000), 5_000, 1, "mttkrp", 8),
])
def test_random_layouts_bit_exact(fc, oracle, dims, nnz, mode, op, tl):
    T = synth.random_small(dims, nnz, seed=nnz + mode)
    idx = T.idx_u32()
    check_against_oracle(fc, oracle, dims, idx, T.val.numpy(), mode, op, tl, device_inputs=(mode % 2 == 1))


def test_zipf_layout_and_wide_keys(fc, oracle):
    cfg = synth.scaled(synth.CONFIGS["skewed3"], 200_000, dims=(12_000, 9_000, 28_000))
    T = synth.make_tensor(cfg)
    check_against_oracle(fc, oracle, cfg.dims, T.idx_u32(), T.val.numpy(), 0, "mttkrp", 8)
    # 5-way with dims whose key bits exceed 64: multi-word sort
    dims = (70_000, 60_000, 50_000, 40_000, 65_000)
    rng = np.random.default_rng(5)
    coords = np.unique(np.stack([rng.integers(0, d, 3000) for d in dims], 1), axis=0)
    coords = coords[rng.permutation(len(coords))]
    idx = [coords[:, k].astype(np.uint32).copy() for k in range(5)]
    check_against_oracle(fc, oracle, dims, idx, rng.uniform(size=len(coords)).astype(np.float32), 2, "ttm", 8)


def test_table2_bytes_of_built_handle(fc):
    g = json.load(open(os.path.join(GOLD, "table2_storage.json")))
    for row in g["rows"]:
        T = synth.random_small((64, 64, 64), row["nnz"], seed=row["nnz"])
        for op, key in (("ttm", "fcoo_ttm"), ("mttkrp", "fcoo_mttkrp")):
            X = fc.FCOO.build(T.idx_u32(), T.val.numpy(), (64, 64, 64), 0, op, row["threadlen"])
            assert X.bytes["table2"] == row[key]
            assert X.bytes["table2"] < row["coo"]


def test_errors(fc):
    idx = [np.array([0, 1, 0], np.uint32), np.array([2, 2, 2], np.uint32), np.array([1, 0, 1], np.uint32)]
    with pytest.raises(fc.FcooError) as e:
        fc.FCOO.build(idx, np.ones(3, np.float32), (2, 3, 2), 0)
    assert e.value.status == -3
    with pytest.raises(fc.FcooError) as e:
        fc.FCOO.build(idx, np.ones(3, np.float32), (2, 2, 2), 0)
    assert e.value.status == -2 and "idx[1]" in e.value.message


def test_empty_tensor(fc):
    X = fc.FCOO.build([np.zeros(0, np.uint32)] * 3, np.zeros(0, np.float32), (5, 6, 7), 1)
    assert X.nnz == 0 and X.nseg == 0
    F = [torch.randn(d, 8, device=cuda()) for d in (5, 6, 7)]
    out = torch.full((6, 8), 7.0, device=cuda())
    fc.spmttkrp(X, F, out=out)
    assert torch.count_nonzero(out).item() == 0
