"""The seeded generators produce what their recipe states (exact nnz, distinct
coordinates, in range, seeded, Zipf skew)."""
import numpy as np
import torch

import synth


def test_distinct_exact_and_seeded():
    cfg = synth.scaled(synth.CONFIGS["skewed3"], 20_000, dims=(300, 200, 400))
    a = synth.make_tensor(cfg)
    b = synth.make_tensor(cfg)
    assert a.nnz == 20_000
    for k in range(3):
        assert torch.equal(a.idx[k], b.idx[k])
        assert int(a.idx[k].min()) >= 0 and int(a.idx[k].max()) < cfg.dims[k]
    lin = (a.idx[0] * cfg.dims[1] + a.idx[1]) * cfg.dims[2] + a.idx[2]
    assert torch.unique(lin).numel() == a.nnz
    assert torch.equal(a.val, b.val)


def test_zipf_skew_visible():
    cfg = synth.scaled(synth.CONFIGS["skewed3"], 50_000, dims=(2000, 2000, 2000))
    t = synth.make_tensor(cfg)
    counts = np.sort(np.bincount(t.idx[0].numpy(), minlength=2000))[::-1]
    # the most frequent index holds a share close to the Zipf(1.1) head mass
    share = counts[0] / t.nnz
    assert 0.5 * synth.zipf_mass(2000, 1.1, 1) < share < 1.5 * synth.zipf_mass(2000, 1.1, 1)


def test_kruskal_values_follow_truth():
    t = synth.make_tensor(synth.CONFIGS["fit3_fd"])
    A, B, C = (x.double() for x in t.truth)
    model = (A[t.idx[0]] * B[t.idx[1]] * C[t.idx[2]]).sum(1)
    resid = t.val.double() - model
    assert t.nnz == 500
    assert 0.005 < float(resid.std()) < 0.02
