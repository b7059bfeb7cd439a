"""Tucker by HOOI around SpTTMc (Eq. 4, Sec. II) through the C ABI against the
FP64 oracle.

Each mode update is checked on its own: the oracle's update (SpTTMc, then a
numpy SVD) from the factors the device held when it made that update: the
start factors and the device's own earlier updates of the same iteration.
Inputs are sparse samples of a tensor of planted multilinear rank plus
noise, so the R leading singular values are well separated and each factor
column is unique up to the shared sign convention.  Also: the fit, the
orthonormality of the factors, a fit that never decreases, exact recovery,
4-way tensors (scalar SpTTMc lanes), a matrix (two modes: the truncated SVD),
rejected shapes, and the full skewed
3-way tensor (76M nonzeros) against a numpy SVD of the device's SpTTMc."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import paper_1705_09905_gb300 as fc

    return fc


def planted(dims, R, density, seed, noise=0.05):
    """Coordinates drawn uniformly; values of a tensor with multilinear rank
    (R, ..., R) and a core with decaying entries, plus N(0, noise^2)."""
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    nnz = int(total * density)
    lin = rng.choice(total, size=nnz, replace=False)
    idx = [a.astype(np.uint32) for a in np.unravel_index(lin, dims)]
    # a dominant superdiagonal with distinct entries: every unfolding has R
    # well separated singular values
    core = 0.3 * rng.standard_normal([R] * len(dims))
    for r in range(R):
        core[(r,) * len(dims)] += 2.0 * R - r
    Fs = [np.linalg.qr(rng.standard_normal((d, R)))[0] * np.sqrt(d) for d in dims]
    val = np.zeros(nnz)
    letters = "abcdefgh"[: len(dims)]
    for start in range(0, nnz, 1 << 16):
        sl = slice(start, start + (1 << 16))
        rows = [F[ix[sl]] for F, ix in zip(Fs, idx)]
        val[sl] = np.einsum(f"{letters}," + ",".join(f"z{c}" for c in letters) + "->z", core, *rows)
    val += noise * rng.standard_normal(nnz) * np.std(val)
    return idx, val.astype(np.float32)


def build_all(fc, dims, idx, val):
    return [fc.FCOO.build(idx, val, dims, n, "mttkrp", 8) for n in range(len(dims))]


def start_factors(dims, R, seed=5):
    g = torch.Generator().manual_seed(seed)
    return [torch.randn(d, R, generator=g) for d in dims]


def check_isolated_updates(oracle, dims, idx, val, init, dev_factors, R, fit_dev):
    """Mode n's device factor against the oracle's update from (device factors
    of modes < n, start factors of modes > n); the fit from the last one."""
    v64 = val.astype(np.float64)
    N = len(dims)
    for n in range(N):
        inputs = [dev_factors[k] if k < n else init[k] for k in range(N)]
        ref, sig2 = oracle.hooi_mode(dims, idx, v64, inputs, n, R)
        got = dev_factors[n]
        err = np.max(np.abs(got - ref))
        assert err < 2e-4, (n, err)
    x2 = float(np.sum(v64 ** 2))
    fit_ref = 1.0 - np.sqrt(max(0.0, x2 - float(np.sum(sig2)))) / np.sqrt(x2)
    assert abs(fit_dev - fit_ref) < 2e-5, (fit_dev, fit_ref)


@pytest.mark.parametrize("R", [2, 3, 4, 8, 11])
def test_hooi_mode_updates_3way(fc, oracle, R):
    dims = (60, 50, 40)
    idx, val = planted(dims, R, 0.3, seed=R)
    Xn = build_all(fc, dims, idx, val)
    init = [f.numpy().astype(np.float64) for f in start_factors(dims, R)]
    st = fc.TuckerState(dims, R, [f.astype(np.float32) for f in init])
    st.iterate(Xn, 1)
    s = st.stats()
    assert s["iters"] == 1 and s["null_directions"] == 0
    dev = [st.factor(n).astype(np.float64) for n in range(3)]
    init32 = [f.astype(np.float32).astype(np.float64) for f in init]
    check_isolated_updates(oracle, dims, idx, val, init32, dev, R, s["fit"])
    for U in dev:
        np.testing.assert_allclose(U.T @ U, np.eye(R), atol=2e-5)


@pytest.mark.parametrize("R,dims", [(3, (20, 15, 12, 10)), (2, (14, 12, 10, 9, 8))])
def test_hooi_mode_updates_nway(fc, oracle, R, dims):
    idx, val = planted(dims, R, 0.3 if len(dims) == 4 else 0.15, seed=len(dims))
    Xn = build_all(fc, dims, idx, val)
    init = [f.numpy().astype(np.float64) for f in start_factors(dims, R, seed=2)]
    st = fc.TuckerState(dims, R, [f.astype(np.float32) for f in init])
    st.iterate(Xn, 1)
    dev = [st.factor(n).astype(np.float64) for n in range(len(dims))]
    check_isolated_updates(oracle, dims, idx, val, init, dev, R, st.stats()["fit"])


def test_hooi_converges_monotone_and_matches_oracle_fit(fc, oracle):
    dims, R = (70, 60, 50), 4
    idx, val = planted(dims, R, 0.2, seed=11, noise=0.3)
    Xn = build_all(fc, dims, idx, val)
    init = start_factors(dims, R, seed=9)
    st = fc.TuckerState(dims, R, init)
    fits = []
    for _ in range(8):
        st.iterate(Xn, 1)
        fits.append(st.stats()["fit"])
    assert all(b >= a - 2e-6 for a, b in zip(fits, fits[1:])), fits
    _, ofits = oracle.hooi(dims, idx, val.astype(np.float64), [f.double().numpy() for f in init], 8)
    assert abs(fits[-1] - ofits[-1]) < 2e-5, (fits[-1], ofits[-1])


def test_hooi_exact_recovery(fc):
    # every entry of a tensor of multilinear rank (3, 3, 3) stored: fit 1 to FP32 level
    dims, R = (24, 20, 16), 3
    idx, val = planted(dims, R, 1.0, seed=3, noise=0.0)
    Xn = build_all(fc, dims, idx, val)
    st = fc.TuckerState(dims, R, start_factors(dims, R, seed=1))
    st.iterate(Xn, 2)
    assert st.stats()["fit"] > 0.999


def test_hooi_2way_is_truncated_svd(fc):
    """Two modes: HOOI alternates U0 <- lead(X U1), U1 <- lead(X^T U0), a
    subspace iteration that converges to the R leading singular subspaces of
    X; the fit then equals the truncated SVD's (numpy)."""
    dims, R = (300, 200), 5
    idx, val = planted(dims, R, 0.5, seed=21, noise=0.02)
    Xn = build_all(fc, dims, idx, val)
    st = fc.TuckerState(dims, R, start_factors(dims, R, seed=6))
    st.iterate(Xn, 15)
    X = np.zeros(dims)
    X[idx[0], idx[1]] = val
    U, sv, Vt = np.linalg.svd(X)
    x2 = float(np.sum(val.astype(np.float64) ** 2))
    fit_ref = 1 - np.sqrt(max(0.0, x2 - float(np.sum(sv[:R] ** 2)))) / np.sqrt(x2)
    assert abs(st.stats()["fit"] - fit_ref) < 1e-5
    P = U[:, :R] @ U[:, :R].T
    U0 = st.factor(0).astype(np.float64)
    np.testing.assert_allclose(U0 @ U0.T, P, atol=1e-4)


def test_hooi_rejects(fc):
    dims = (30, 20, 10)
    idx, val = planted(dims, 2, 0.2, seed=1)
    Xn = build_all(fc, dims, idx, val)
    with pytest.raises(fc.FcooError) as e:
        fc.TuckerState(dims, 12, start_factors(dims, 12))  # R^2 = 144 > 128
    assert e.value.status == -9
    st = fc.TuckerState(dims, 2, start_factors(dims, 2))
    with pytest.raises(fc.FcooError) as e:
        st.iterate([Xn[1], Xn[0], Xn[2]], 1)
    assert e.value.status == -1
    with pytest.raises(fc.FcooError) as e:
        st.iterate(Xn[:2] + [fc.FCOO.build(idx, val, dims, 2, "ttm", 8)], 1)
    assert e.value.status == -1


def test_hooi_full_size_last_mode_against_numpy_svd(fc):
    """The skewed 3-way tensor (76M nonzeros), R = 8: after one iteration the
    factors are orthonormal, and the last factor equals the leading left
    singular vectors (numpy SVD, sign convention applied) of SpTTMc of the
    last mode taken with the device's other factors."""
    import oracle as orc

    cfg = synth.CONFIGS["skewed3"]
    dev = torch.device("cuda", 0)
    T = synth.make_tensor(cfg, device=dev)
    idx32 = [a.to(torch.int32).contiguous() for a in T.idx]
    Xn = [fc.FCOO.build(idx32, T.val, cfg.dims, n, "mttkrp", 8) for n in range(3)]
    x2 = float(torch.sum(T.val.double() ** 2))
    del T, idx32
    R = 8
    try:
        st = fc.TuckerState(cfg.dims, R, start_factors(cfg.dims, R, seed=4))
        st.iterate(Xn, 2)
        s = st.stats()
        assert s["null_directions"] == 0
        U = [st.factor(n) for n in range(3)]
        for u in U:
            np.testing.assert_allclose(u.T.astype(np.float64) @ u, np.eye(R), atol=2e-5)
        Y = fc.spttmc(Xn[2], [torch.from_numpy(u).to(dev) for u in U]).cpu().double().numpy()
        Us, sv, _ = np.linalg.svd(Y, full_matrices=False)
        ref = orc.sign_fix(Us[:, :R])
        assert np.max(np.abs(U[2] - ref)) < 2e-4
        fit_ref = 1 - np.sqrt(max(0.0, x2 - float(np.sum(sv[:R] ** 2)))) / np.sqrt(x2)
        assert abs(s["fit"] - fit_ref) < 2e-5
    finally:
        for X in Xn:
            X.close()
        torch.cuda.empty_cache()
