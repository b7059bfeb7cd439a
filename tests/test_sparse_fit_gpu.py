"""Differentiation on the device: the sparse CP-fit loss and gradients
(kind 0) and the adjoint of SpMTTKRP (kind 1) vs the FP64 oracle, a
directional finite-difference check of the GPU gradient, the autograd
wrappers, and an Adam fit that drives the loss down."""
import numpy as np
import pytest
import torch

import synth
from helpers import assert_close_abs, cuda, host_factors, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import paper_1705_09905_gb300 as fc

    return fc


def handles(fc, T):
    return [fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, n, "mttkrp", 8) for n in range(T.nmodes)]


def start_factors(dims, R, seed, dtype=torch.float32):
    return [(f * R ** (-1.0 / 6.0)).to(cuda()).to(dtype) for f in synth.make_factors(dims, R, seed=seed)]


@pytest.mark.parametrize("cfgname,dims,nnz,R,dtype", [
    ("fit3_fd", None, None, 4, torch.float32),
    ("fit3", (500, 400, 300), 60_000, 32, torch.float32),
    ("fit3", (500, 400, 300), 60_000, 16, torch.bfloat16),
    ("fit3", (300, 200, 100), 30_000, 7, torch.float32),
])
def test_loss_grads_dvals_vs_oracle(fc, oracle, cfgname, dims, nnz, R, dtype):
    cfg = synth.CONFIGS[cfgname]
    if dims is not None:
        cfg = synth.scaled(cfg, nnz, dims=dims)
    T = synth.make_tensor(cfg)
    Xs = handles(fc, T)
    F = start_factors(T.dims, R, seed=2, dtype=dtype)
    loss, grads, dv = fc.sparse_fit_grad(Xs, F, want_dvals=True)
    torch.cuda.synchronize()
    Fh = host_factors(F)
    idx, val = T.idx_u32(), T.val.double().numpy()
    rl, rg, rdv = oracle.sparse_fit(T.dims, idx, val, Fh)
    assert abs(loss.item() - rl) <= 1e-5 * rl
    np.testing.assert_allclose(dv.cpu().numpy(), rdv, rtol=1e-4, atol=1e-5 * np.abs(rdv).max())
    # element-wise bound from the same sums taken over absolute values
    e = np.abs(rdv)
    for n in range(3):
        absn = oracle.mttkrp(T.dims, idx, e, [np.abs(f) for f in Fh], n)
        assert_close_abs(grads[n].cpu().numpy(), rg[n], absn + 1e-30, rel_abs=2e-5)
    assert float(fc.sparse_cp_loss(Xs[1], F).item()) == pytest.approx(rl, rel=1e-5)


def test_partial_gradients_and_reused_residuals(fc, oracle):
    """Gradients of a subset of the factors: the residuals are computed on the
    first requested mode and gathered into the others' order through a cached
    position map; changing the first requested mode on the same handles must
    rebuild the maps.  A single requested gradient takes the direct path."""
    cfg = synth.scaled(synth.CONFIGS["fit3"], 60_000, dims=(500, 400, 300))
    T = synth.make_tensor(cfg)
    Xs = handles(fc, T)
    F = start_factors(T.dims, 16, seed=5)
    Fh = host_factors(F)
    idx, val = T.idx_u32(), T.val.double().numpy()
    rl, rg, rdv = oracle.sparse_fit(T.dims, idx, val, Fh)
    e = np.abs(rdv)
    for modes in ((1, 2), (0, 1, 2), (2, 0), (2,), (1, 2)):
        loss, grads, dv = fc.sparse_fit_grad(Xs, F, want_dvals=True, modes=modes)
        torch.cuda.synchronize()
        assert abs(loss.item() - rl) <= 1e-5 * rl, modes
        np.testing.assert_allclose(dv.cpu().numpy(), rdv, rtol=1e-4, atol=1e-5 * e.max())
        for n in range(3):
            if n not in modes:
                assert grads[n] is None
                continue
            absn = oracle.mttkrp(T.dims, idx, e, [np.abs(f) for f in Fh], n)
            assert_close_abs(grads[n].cpu().numpy(), rg[n], absn + 1e-30, rel_abs=2e-5)


def test_gradient_directional_finite_difference(fc):
    T = synth.make_tensor(synth.CONFIGS["fit3_fd"])
    Xs = handles(fc, T)
    F = start_factors(T.dims, 4, seed=3)
    _, grads, _ = fc.sparse_fit_grad(Xs, F)
    g = torch.Generator(device="cpu").manual_seed(0)
    D = [torch.randn(f.shape, generator=g).to(cuda()) for f in F]
    h = 1e-3
    lp = fc.sparse_cp_loss(Xs[0], [f + h * d for f, d in zip(F, D)]).item()
    lm = fc.sparse_cp_loss(Xs[0], [f - h * d for f, d in zip(F, D)]).item()
    fd = (lp - lm) / (2 * h)
    an = sum(float((gk * dk).sum()) for gk, dk in zip(grads, D))
    assert abs(fd - an) <= 1e-3 * max(1.0, abs(an)), (fd, an)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_adjoint_kind1_vs_oracle(fc, oracle, mode):
    T = synth.random_small((80, 60, 70), 20_000, seed=mode)
    Xs = handles(fc, T)
    F = [f.to(cuda()) for f in synth.make_factors(T.dims, 16, seed=5)]
    G = torch.randn(T.dims[mode], 16, generator=torch.Generator().manual_seed(1)).to(cuda())
    grads, dv = fc.spmttkrp_adjoint(Xs, F, mode, G)
    torch.cuda.synchronize()
    idx, val = T.idx_u32(), T.val.double().numpy()
    Fh = host_factors(F)
    rgrads, rdv = oracle.mttkrp_adjoint(T.dims, idx, val, Fh, mode, G.double().cpu().numpy())
    for k in range(3):
        if k == mode:
            assert grads[k] is None
            continue
        fl = [np.abs(f) for f in Fh]
        fl[mode] = np.abs(G.double().cpu().numpy())
        absk = oracle.mttkrp(T.dims, idx, np.abs(val), fl, k)
        assert_close_abs(grads[k].cpu().numpy(), rgrads[k], absk)
    assert rel_fro(dv.cpu().numpy(), rdv) <= 1e-5


def test_autograd_functions(fc, oracle):
    T = synth.random_small((40, 30, 20), 3000, seed=11)
    Xs = handles(fc, T)
    F = [f.to(cuda()).requires_grad_(True) for f in synth.make_factors(T.dims, 8, seed=12)]
    # SpMTTKRP with its adjoint as backward: d/dF of <M, W>
    W = torch.randn(T.dims[0], 8, generator=torch.Generator().manual_seed(2)).to(cuda())
    M = fc.SpMTTKRPFunction.apply(Xs, 0, *F)
    (M * W).sum().backward()
    assert F[0].grad is None
    rg, _ = oracle.mttkrp_adjoint(T.dims, T.idx_u32(), T.val.double().numpy(), host_factors(F), 0,
                                  W.double().cpu().numpy())
    for k in (1, 2):
        assert rel_fro(F[k].grad.cpu().numpy(), rg[k]) <= 1e-5
    # sparse CP loss
    for f in F:
        f.grad = None
    loss = fc.SparseCPLoss.apply(Xs, *F)
    (3.0 * loss).backward()
    _, rg, _ = oracle.sparse_fit(T.dims, T.idx_u32(), T.val.double().numpy(), host_factors(F))
    for k in range(3):
        assert rel_fro(F[k].grad.cpu().numpy(), 3.0 * rg[k]) <= 1e-5


def test_adam_fit_reduces_loss(fc):
    cfg = synth.scaled(synth.CONFIGS["fit3"], 40_000, dims=(400, 300, 200), kruskal_rank=8)
    T = synth.make_tensor(cfg)
    Xs = handles(fc, T)
    F = [f.requires_grad_(True) for f in start_factors(T.dims, 8, seed=13)]
    opt = torch.optim.Adam(F, lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    first = None
    for step in range(200):
        opt.zero_grad()
        loss = fc.SparseCPLoss.apply(Xs, *F)
        loss.backward()
        opt.step()
        if first is None:
            first = loss.item()
    last = fc.sparse_cp_loss(Xs[0], [f.detach() for f in F]).item()
    assert last < 0.25 * first, (first, last)
