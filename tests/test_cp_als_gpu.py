"""CP-ALS (Algorithm 1) on the device vs the FP64 oracle: factors, lambda and
fit per sweep (FP32), the BF16 path against the oracle fed the same rounded
factors step by step, the fibre reuse of modes 0 and 1 (FP32 and BF16), the
pseudo-inverse fallback, monotone fit, exact recovery of a low-rank tensor,
checkpoint / resume."""
import numpy as np
import pytest
import torch

import synth
from helpers import cuda, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import paper_1705_09905_gb300 as fc

    return fc


def handles(fc, T, tl=8):
    return [fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, n, "mttkrp", tl) for n in range(T.nmodes)]


def test_fp32_sweeps_match_oracle(fc, oracle):
    cfg = synth.CONFIGS["tiny"]
    T = synth.make_tensor(cfg)
    Xs = handles(fc, T)
    R = 8
    init = synth.make_factors(T.dims, R, seed=3, kind="uniform")
    st = fc.CPState(T.dims, R, init)
    idx, val = T.idx_u32(), T.val.double().numpy()
    F = [f.double().numpy() for f in init]
    fits = []
    for sweep in range(4):
        st.iterate(Xs)
        s = st.stats()
        for n in range(3):
            # the bound below rests on well-conditioned normal equations: the
            # FP32 rounding of M (about 1e-7) moves the solution by at most
            # cond(V) times that; measured cond(V) <= 14 on this case
            V = np.ones((R, R))
            for k in range(3):
                if k != n:
                    V *= oracle.gram(F[k])
            assert np.linalg.cond(V) <= 100, (sweep, n, np.linalg.cond(V))
            F, lam, _, _ = oracle.cp_als_mode(T.dims, idx, val, F, n)
        ref_fit = oracle.cp_fit(T.dims, idx, val, F, lam)
        assert abs(s["fit"] - ref_fit) <= 1e-5, (sweep, s["fit"], ref_fit)
        assert rel_fro(s["lambda"], lam) <= 1e-5
        for k in range(3):
            assert rel_fro(st.factor(k).cpu().numpy(), F[k]) <= 1e-5, (sweep, k)
        fits.append(s["fit"])
        assert s["iters"] == sweep + 1
    assert all(b >= a - 1e-6 for a, b in zip(fits, fits[1:])), fits


def test_bf16_sweep_matches_oracle_with_same_rounding(fc, oracle):
    cfg = synth.CONFIGS["tiny"]
    T = synth.make_tensor(cfg)
    Xs = handles(fc, T)
    R = 16
    init = synth.make_factors(T.dims, R, seed=4, kind="uniform")
    st = fc.CPState(T.dims, R, init, dtype=torch.bfloat16)
    idx, val = T.idx_u32(), T.val.double().numpy()
    rnd = lambda a: torch.as_tensor(a).to(torch.bfloat16).double().numpy()  # round to nearest even
    F = [rnd(f.numpy()) for f in init]
    for sweep in range(2):
        st.iterate(Xs)
        for n in range(3):
            F, lam, _, _ = oracle.cp_als_mode(T.dims, idx, val, F, n)
            F[n] = rnd(F[n])
        s = st.stats()
        ref_fit = oracle.cp_fit(T.dims, idx, val, F, lam)
        assert abs(s["fit"] - ref_fit) <= 1e-4, (sweep, s["fit"], ref_fit)
        for k in range(3):
            # a few entries may round to the neighbouring bf16 value (FP32 vs FP64 near a tie)
            assert rel_fro(st.factor(k).cpu().numpy(), F[k]) <= 2e-3, (sweep, k)


def test_mixed_schedule_switches_storage(fc, oracle):
    """BF16 sweeps, then cp_state_set_dtype(FP32) and FP32 sweeps: the switch
    keeps the factors exactly (BF16 -> FP32 is exact) and the FP32 sweeps
    that follow match the oracle continued from the same factors."""
    cfg = synth.CONFIGS["tiny"]
    T = synth.make_tensor(cfg)
    Xs = handles(fc, T)
    R = 8
    init = synth.make_factors(T.dims, R, seed=5, kind="uniform")
    st = fc.CPState(T.dims, R, init, dtype=torch.bfloat16)
    st.iterate(Xs, sweeps=2)
    before = [st.factor(k).cpu().numpy() for k in range(3)]
    lam0 = st.stats()["lambda"]
    st.set_dtype(torch.float32)
    after = [st.factor(k).cpu().numpy() for k in range(3)]
    for k in range(3):
        assert np.array_equal(before[k], after[k])
        t = torch.from_numpy(after[k])
        assert torch.equal(t.to(torch.bfloat16).float(), t)  # still the BF16 values
    idx, val = T.idx_u32(), T.val.double().numpy()
    F = [b.astype(np.float64) for b in before]
    lam = lam0
    for sweep in range(2):
        st.iterate(Xs)
        for n in range(3):
            F, lam, _, _ = oracle.cp_als_mode(T.dims, idx, val, F, n)
        s = st.stats()
        assert abs(s["fit"] - oracle.cp_fit(T.dims, idx, val, F, lam)) <= 1e-5
        for k in range(3):
            assert rel_fro(st.factor(k).cpu().numpy(), F[k]) <= 1e-4, (sweep, k)
    # and back: FP32 -> BF16 rounds to nearest even
    f32 = [st.factor(k).cpu() for k in range(3)]
    st.set_dtype(torch.bfloat16)
    for k in range(3):
        assert torch.equal(st.factor(k).cpu(), f32[k].to(torch.bfloat16).float())
    st.iterate(Xs)
    assert np.isfinite(st.stats()["fit"])


def skewed_small():
    # Zipf indices: fibres hold several nonzeros, as on the full workload
    return synth.make_tensor(synth.scaled(synth.CONFIGS["skewed3"], 200_003, dims=(300, 250, 700)))


@pytest.mark.parametrize("R", [8, 16])
def test_fibre_reuse_fp32_matches_oracle(fc, oracle, R):
    """Modes 0 and 1 through the mode-2 fibre sums (cp_state_use_fibres).
    Each mode update of each sweep is checked on its own against the oracle's
    update from the factors the device held when it made it (the Zipf
    tensor's normal matrices are ill-conditioned, so errors compounded over
    sweeps say nothing about one update).  The bound is FP32 rounding times
    cond(V), at least 1e-4.  The fit is checked against the oracle and the
    direct path on the device."""
    T = skewed_small()
    Xs = handles(fc, T)
    Xt = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 2, "ttm", 8)
    assert Xt.nseg < 0.7 * T.nnz
    init = synth.make_factors(T.dims, R, seed=3, kind="uniform")
    st = fc.CPState(T.dims, R, init).use_fibres(Xt)
    direct = fc.CPState(T.dims, R, init)
    idx, val = T.idx_u32(), T.val.double().numpy()
    for sweep in range(3):
        before = [st.factor(k).cpu().double().numpy() for k in range(3)]
        st.iterate(Xs)
        direct.iterate(Xs)
        after = [st.factor(k).cpu().double().numpy() for k in range(3)]
        for n in range(3):
            inputs = [after[k] if k < n else before[k] for k in range(3)]
            V = np.ones((R, R))
            for k in range(3):
                if k != n:
                    V *= inputs[k].T @ inputs[k]
            tol = max(1e-4, 5e-8 * np.linalg.cond(V))
            Fo, lam, _, _ = oracle.cp_als_mode(T.dims, idx, val, inputs, n)
            assert rel_fro(after[n], Fo[n]) <= tol, (sweep, n, rel_fro(after[n], Fo[n]), tol)
        s, d = st.stats(), direct.stats()
        assert abs(s["fit"] - oracle.cp_fit(T.dims, idx, val, after, s["lambda"])) <= 1e-5, sweep
        assert abs(s["fit"] - d["fit"]) <= 1e-6, sweep


def test_fibre_reuse_bf16_and_off(fc, oracle):
    """BF16 storage through the fibre sums (the BF16 factor widened to FP32,
    the fibre sums gathered from BF16 C): each mode update against the
    oracle's update from the device's (BF16) factors of that moment, rounded
    to BF16 like the device's; then the reuse turned off mid-run continues on
    the direct path."""
    T = skewed_small()
    Xs = handles(fc, T)
    Xt = fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 2, "ttm", 8)
    R = 16
    init = synth.make_factors(T.dims, R, seed=4, kind="uniform")
    st = fc.CPState(T.dims, R, init, dtype=torch.bfloat16).use_fibres(Xt)
    idx, val = T.idx_u32(), T.val.double().numpy()
    rnd = lambda a: torch.as_tensor(a).to(torch.bfloat16).double().numpy()
    for sweep in range(2):
        before = [st.factor(k).cpu().double().numpy() for k in range(3)]
        st.iterate(Xs)
        after = [st.factor(k).cpu().double().numpy() for k in range(3)]
        for n in range(3):
            inputs = [after[k] if k < n else before[k] for k in range(3)]
            V = np.ones((R, R))
            for k in range(3):
                if k != n:
                    V *= inputs[k].T @ inputs[k]
            # a few entries may round to the neighbouring BF16 value
            tol = max(2e-3, 5e-8 * np.linalg.cond(V))
            Fo, _, _, _ = oracle.cp_als_mode(T.dims, idx, val, inputs, n)
            assert rel_fro(after[n], rnd(Fo[n])) <= tol, (sweep, n, rel_fro(after[n], rnd(Fo[n])), tol)
        s = st.stats()
        assert abs(s["fit"] - oracle.cp_fit(T.dims, idx, val, after, s["lambda"])) <= 1e-4, sweep
    st.use_fibres(None)
    st.iterate(Xs)
    assert np.isfinite(st.stats()["fit"])
    with pytest.raises(fc.FcooError):
        st.use_fibres(fc.FCOO.build(T.idx_u32(), T.val.numpy(), T.dims, 1, "ttm", 8))


@pytest.mark.parametrize("R", [112, 120])
def test_wide_rank_solves(fc, oracle, R):
    """R = 112 is the largest rank whose solve runs in shared memory; R = 120
    takes the global-memory solve.  Both match the oracle's mode updates."""
    cfg = synth.scaled(synth.CONFIGS["tiny"], 30_000, dims=(400, 300, 250))
    T = synth.make_tensor(cfg)
    Xs = handles(fc, T)
    init = synth.make_factors(T.dims, R, seed=6)
    st = fc.CPState(T.dims, R, init)
    st.iterate(Xs)
    s = st.stats()
    idx, val = T.idx_u32(), T.val.double().numpy()
    F = [f.double().numpy() for f in init]
    for n in range(3):
        F, lam, _, used = oracle.cp_als_mode(T.dims, idx, val, F, n)
        assert not used
    assert s["npinv"] == 0
    for k in range(3):
        assert rel_fro(st.factor(k).cpu().numpy(), F[k]) <= 1e-4, k
    assert abs(s["fit"] - oracle.cp_fit(T.dims, idx, val, F, lam)) <= 1e-5


def test_pseudo_inverse_fallback(fc, oracle):
    # modes 1 and 2 of size 1: the mode-0 normal matrix G1 * G2 has rank 1 < R
    T = synth.random_small((50, 1, 1), 30, seed=5)
    Xs = handles(fc, T)
    R = 3
    init = synth.make_factors(T.dims, R, seed=6, kind="uniform")
    st = fc.CPState(T.dims, R, init)
    st.iterate(Xs)
    s = st.stats()
    F, lam, fits, npinv = oracle.cp_als(T.dims, T.idx_u32(), T.val.double().numpy(),
                                        [f.double().numpy() for f in init], 1)
    assert s["npinv"] == npinv > 0
    # this tensor is fitted exactly (fit 1): the Grams identity for the fit then
    # subtracts nearly equal terms, so FP32 inputs (~1e-7) give ~sqrt(1e-7) there
    assert abs(s["fit"] - fits[0]) <= 1e-3
    for k in range(3):
        assert rel_fro(st.factor(k).cpu().numpy(), F[k]) <= 1e-4


def test_low_rank_recovery_4way(fc):
    rng = np.random.default_rng(7)
    dims = (12, 10, 9, 8)
    A = [rng.standard_normal((d, 2)) for d in dims]
    X = np.einsum("ir,jr,kr,lr->ijkl", *A)
    idx = [a.ravel().astype(np.uint32) for a in np.indices(dims)]
    T = synth.SparseTensor(dims, [torch.as_tensor(a.astype(np.int64)) for a in idx],
                           torch.as_tensor(X.ravel().astype(np.float32)))
    Xs = handles(fc, T)
    st = fc.CPState(dims, 2, synth.make_factors(dims, 2, seed=8, kind="uniform"))
    st.iterate(Xs, sweeps=60)
    assert st.fit > 1 - 1e-4


def test_checkpoint_resume_is_bitwise(fc):
    T = synth.make_tensor(synth.scaled(synth.CONFIGS["skewed3"], 100_000, dims=(500, 400, 600)))
    Xs = handles(fc, T)
    init = synth.make_factors(T.dims, 16, seed=9, kind="uniform")
    a = fc.CPState(T.dims, 16, init)
    a.iterate(Xs, sweeps=2)
    blob = a.save()
    a.iterate(Xs, sweeps=2)
    b = fc.CPState(T.dims, 16, init).load(blob)
    assert b.stats()["iters"] == 2
    b.iterate(Xs, sweeps=2)
    sa, sb = a.stats(), b.stats()
    assert sa["fit"] == sb["fit"] and sb["iters"] == 4
    for k in range(3):
        assert torch.equal(a.factor(k), b.factor(k))


def test_argument_errors(fc):
    T = synth.random_small((20, 30, 40), 500, seed=1)
    Xs = handles(fc, T)
    with pytest.raises(fc.FcooError):
        fc.CPState((20, 30, 41), 4, synth.make_factors((20, 30, 41), 4, seed=1)).iterate(Xs)
    with pytest.raises(fc.FcooError):
        fc.CPState(T.dims, 4, synth.make_factors(T.dims, 4, seed=1)).iterate([Xs[1], Xs[0], Xs[2]])
