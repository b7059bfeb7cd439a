"""Pins for the FP64 oracle against things other than itself.

Each check is chosen so that a plausible mistake in the oracle (a dropped
factor, a wrong index or mode, a transposed operand, a wrong normalisation or
fit formula) fails at least one of them:

* brute force on tiny tensors: densify, unfold X_(n) (Sec. II), build the
  Khatri-Rao product explicitly column by column from Kronecker products
  (Eq. 1, Eq. 2) and multiply (Eq. 5); SpTTM via a dense n-mode product (Eq. 3);
  SpTTMc via chained dense n-mode products and via X_(n) times a Kronecker
  product (Eq. 4);
* closed forms for a full Kruskal tensor;
* hand-derived golden values (tests/golden, Fig. 2 / Table I / Eq. 3 / Eq. 6);
* special cases (R=1 all-ones factors give slice sums, identity U);
* invariants (linearity in values, mode permutation, nonzero order);
* Algorithm 1: fit never decreases, fit formula equals the dense residual,
  one sweep equals a numpy pinv re-derivation, exact recovery of a low-rank
  tensor, pseudo-inverse fallback against numpy.linalg.pinv;
* sparse-fit gradients against central finite differences, adjoint identity;
* HOOI: exact recovery of a tensor of multilinear rank (2, 2, 2), orthonormal
  factors, a fit that never decreases and equals the dense residual of the
  projected tensor.
"""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rand_coo(rng, dims, nnz):
    total = int(np.prod(dims))
    lin = rng.choice(total, size=nnz, replace=False)
    idx = list(np.unravel_index(lin, dims))
    val = rng.uniform(0.1, 1.0, size=nnz)
    return [a.astype(np.uint32) for a in idx], val


def densify(dims, idx, val):
    X = np.zeros(dims)
    for p in range(len(val)):
        X[tuple(int(a[p]) for a in idx)] += val[p]
    return X


def unfold(X, n):
    """Mode-n matricization: rows are i_n, columns enumerate the other modes in
    ascending order with the lowest mode varying fastest (Sec. II, Eq. 5)."""
    return np.reshape(np.moveaxis(X, n, 0), (X.shape[n], -1), order="F")


def khatri_rao(mats):
    """Column-wise Kronecker product (Eq. 2) of mats listed left to right."""
    R = mats[0].shape[1]
    cols = []
    for r in range(R):
        c = mats[0][:, r]
        for M in mats[1:]:
            c = np.kron(c, M[:, r])  # Eq. 1 block structure
        cols.append(c)
    return np.stack(cols, axis=1)


def brute_mttkrp(X, factors, n):
    others = [k for k in range(X.ndim) if k != n]
    kr = khatri_rao([factors[k] for k in reversed(others)])  # e.g. C (.) B for mode 1 of 3
    return unfold(X, n) @ kr


# ---------------------------------------------------------------- SpMTTKRP


@pytest.mark.parametrize("dims", [(6, 5, 4), (4, 3, 5, 2)])
def test_mttkrp_matches_unfolding_times_khatri_rao(oracle, dims):
    rng = np.random.default_rng(1)
    nnz = int(np.prod(dims) * 0.4)
    idx, val = rand_coo(rng, dims, nnz)
    R = 3
    F = [rng.standard_normal((d, R)) for d in dims]
    X = densify(dims, idx, val)
    for n in range(len(dims)):
        got = oracle.mttkrp(dims, idx, val, F, n)
        ref = brute_mttkrp(X, F, n)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_mttkrp_kruskal_closed_form(oracle):
    rng = np.random.default_rng(2)
    dims, Rt = (7, 6, 5), 3
    A, B, C = (rng.standard_normal((d, Rt)) for d in dims)
    lam = rng.uniform(0.5, 2.0, Rt)
    X = np.einsum("r,ir,jr,kr->ijk", lam, A, B, C)
    idx = [a.astype(np.uint32).ravel() for a in np.indices(dims)]
    val = X.ravel()
    # MTTKRP_1 of a full Kruskal tensor is A diag(lambda) (B^T B * C^T C)
    got = oracle.mttkrp(dims, idx, val, [A, B, C], 0)
    np.testing.assert_allclose(got, A @ np.diag(lam) @ ((B.T @ B) * (C.T @ C)), rtol=1e-11, atol=1e-11)
    got2 = oracle.mttkrp(dims, idx, val, [A, B, C], 2)
    np.testing.assert_allclose(got2, C @ np.diag(lam) @ ((A.T @ A) * (B.T @ B)), rtol=1e-11, atol=1e-11)


def test_mttkrp_rank1_ones_gives_slice_sums(oracle):
    rng = np.random.default_rng(3)
    dims = (5, 6, 7)
    idx, val = rand_coo(rng, dims, 60)
    F = [np.ones((d, 1)) for d in dims]
    for n in range(3):
        got = oracle.mttkrp(dims, idx, val, F, n)[:, 0]
        ref = np.bincount(idx[n].astype(np.int64), weights=val, minlength=dims[n])
        np.testing.assert_allclose(got, ref, rtol=1e-13)


def test_mttkrp_single_nonzero(oracle):
    dims = (4, 3, 2)
    idx = [np.array([2], np.uint32), np.array([1], np.uint32), np.array([0], np.uint32)]
    val = np.array([2.5])
    rng = np.random.default_rng(4)
    F = [rng.standard_normal((d, 5)) for d in dims]
    got = oracle.mttkrp(dims, idx, val, F, 1)
    ref = np.zeros((3, 5))
    ref[1] = 2.5 * F[0][2] * F[2][0]
    np.testing.assert_allclose(got, ref, rtol=1e-15)


def test_mttkrp_linear_in_values_and_order_invariant(oracle):
    rng = np.random.default_rng(5)
    dims = (9, 8, 7)
    idx, v1 = rand_coo(rng, dims, 150)
    v2 = rng.standard_normal(150)
    F = [rng.standard_normal((d, 4)) for d in dims]
    a, b = 1.7, -0.3
    lhs = oracle.mttkrp(dims, idx, a * v1 + b * v2, F, 0)
    rhs = a * oracle.mttkrp(dims, idx, v1, F, 0) + b * oracle.mttkrp(dims, idx, v2, F, 0)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    perm = rng.permutation(150)
    shuf = oracle.mttkrp(dims, [x[perm] for x in idx], v1[perm], F, 1)
    np.testing.assert_allclose(shuf, oracle.mttkrp(dims, idx, v1, F, 1), rtol=1e-12, atol=1e-12)


def test_mttkrp_mode_permutation(oracle):
    rng = np.random.default_rng(6)
    dims = (5, 4, 6, 3)
    idx, val = rand_coo(rng, dims, 100)
    F = [rng.standard_normal((d, 3)) for d in dims]
    perm = [2, 0, 3, 1]  # new mode q is old mode perm[q]
    pdims = tuple(dims[k] for k in perm)
    pidx = [idx[k] for k in perm]
    pF = [F[k] for k in perm]
    for q in range(4):
        np.testing.assert_allclose(oracle.mttkrp(pdims, pidx, val, pF, q), oracle.mttkrp(dims, idx, val, F, perm[q]),
                                   rtol=1e-12, atol=1e-12)


def test_mttkrp_golden_fig2(oracle):
    g = json.load(open(os.path.join(GOLD, "fig2_fcoo_3x3x3.json")))
    coords = np.array(g["coords_input_order"], dtype=np.uint32)
    idx = [coords[:, k] for k in range(3)]
    val = np.array(g["vals_input_order"])
    m = g["mttkrp_mode0"]
    F = [np.ones((3, 1)), np.array(m["B_col"])[:, None], np.array(m["C_col"])[:, None]]
    np.testing.assert_array_equal(oracle.mttkrp(g["dims"], idx, val, F, 0), np.array(m["M"]))


# ---------------------------------------------------------------- SpTTM


@pytest.mark.parametrize("dims,mode", [((6, 5, 4), 2), ((6, 5, 4), 0), ((4, 3, 5, 3), 3), ((4, 3, 5, 3), 1)])
def test_ttm_matches_dense_nmode_product(oracle, dims, mode):
    rng = np.random.default_rng(7)
    nnz = int(np.prod(dims) * 0.3)
    idx, val = rand_coo(rng, dims, nnz)
    U = rng.standard_normal((dims[mode], 3))
    keys, Y = oracle.ttm(dims, idx, val, U, mode)
    X = densify(dims, idx, val)
    Yd = np.moveaxis(np.tensordot(X, U, axes=([mode], [0])), -1, -1)  # other modes ascending, then R
    others = [k for k in range(len(dims)) if k != mode]
    # keys: exactly the distinct index tuples that hold nonzeros, lexicographically sorted
    present = sorted(set(tuple(int(idx[k][p]) for k in others) for p in range(nnz)))
    assert [tuple(int(x) for x in k) for k in keys] == present
    for f, key in enumerate(keys):
        np.testing.assert_allclose(Y[f], Yd[tuple(int(x) for x in key)], rtol=1e-12, atol=1e-12)
    # every fibre without nonzeros is zero in the dense product
    mask = np.ones(Yd.shape[:-1], dtype=bool)
    for key in keys:
        mask[tuple(int(x) for x in key)] = False
    assert np.all(Yd[mask] == 0.0)


def test_ttm_identity_densifies_and_kruskal_closed_form(oracle):
    rng = np.random.default_rng(8)
    dims = (5, 4, 6)
    idx, val = rand_coo(rng, dims, 40)
    keys, Y = oracle.ttm(dims, idx, val, np.eye(6), 2)
    X = densify(dims, idx, val)
    for f, (i, j) in enumerate(keys):
        np.testing.assert_array_equal(Y[f], X[i, j, :])
    # full Kruskal tensor: Y(i,j,:) = sum_r lam_r A(i,r) B(j,r) (U^T C(:,r))
    A, B, C = (rng.standard_normal((d, 2)) for d in dims)
    lam = np.array([1.5, 0.7])
    Xk = np.einsum("r,ir,jr,kr->ijk", lam, A, B, C)
    fidx = [a.astype(np.uint32).ravel() for a in np.indices(dims)]
    U = rng.standard_normal((6, 3))
    keys, Y = oracle.ttm(dims, fidx, Xk.ravel(), U, 2)
    ref = np.einsum("r,ir,jr,qr->ijq", lam, A, B, U.T @ C)
    np.testing.assert_allclose(Y, ref.reshape(-1, 3), rtol=1e-11, atol=1e-11)


def test_ttm_golden_fig2(oracle):
    g = json.load(open(os.path.join(GOLD, "fig2_fcoo_3x3x3.json")))
    coords = np.array(g["coords_input_order"], dtype=np.uint32)
    idx = [coords[:, k] for k in range(3)]
    val = np.array(g["vals_input_order"])
    t = g["ttm_mode2"]
    keys, Y = oracle.ttm(g["dims"], idx, val, np.array(t["U"]), 2)
    np.testing.assert_array_equal(keys, np.array(t["segkeys"]))
    np.testing.assert_array_equal(Y, np.array(t["Y"]))


# ---------------------------------------------------------------- SpTTMc


def dense_ttmc(X, U, n):
    """Eq. 4 on a dense tensor: X times U_k^T on every mode k != n, the product
    modes kept in ascending order; reshaped so the first product mode varies
    slowest in the output column."""
    Y = X
    for k in sorted((k for k in range(X.ndim) if k != n), reverse=True):
        Y = np.moveaxis(np.tensordot(Y, U[k], axes=([k], [0])), -1, k)
    Y = np.moveaxis(Y, n, 0)
    return Y.reshape(X.shape[n], -1)


@pytest.mark.parametrize("dims,mode", [((6, 5, 4), 0), ((6, 5, 4), 1), ((6, 5, 4), 2), ((4, 3, 5, 3), 0),
                                       ((4, 3, 5, 3), 2)])
def test_ttmc_matches_dense_products(oracle, dims, mode):
    rng = np.random.default_rng(21)
    nnz = int(np.prod(dims) * 0.35)
    idx, val = rand_coo(rng, dims, nnz)
    R = 3
    U = [rng.standard_normal((d, R)) for d in dims]
    U[mode] = np.full((dims[mode], R), np.nan)  # the index mode's factor is never read
    got = oracle.ttmc(dims, idx, val, U, mode)
    X = densify(dims, idx, val)
    np.testing.assert_allclose(got, dense_ttmc(X, U, mode), rtol=1e-12, atol=1e-12)
    # the same through the unfolding: X_(n) times the Kronecker product of the
    # product-mode factors (Eq. 1), lowest mode fastest in both; then the
    # column digits reversed so the first product mode is the slowest
    others = [k for k in range(len(dims)) if k != mode]
    K = U[others[-1]]
    for k in reversed(others[:-1]):
        K = np.kron(K, U[k])
    Yu = (unfold(X, mode) @ K).reshape([dims[mode]] + [R] * len(others))
    Yu = np.transpose(Yu, [0] + list(range(len(others), 0, -1))).reshape(dims[mode], -1)
    np.testing.assert_allclose(got, Yu, rtol=1e-12, atol=1e-12)


def test_ttmc_identity_densifies_and_kruskal_closed_form(oracle):
    rng = np.random.default_rng(22)
    dims = (4, 5, 5)
    idx, val = rand_coo(rng, dims, 50)
    U = [np.zeros((4, 5)), np.eye(5), np.eye(5)]
    got = oracle.ttmc(dims, idx, val, U, 0)
    np.testing.assert_array_equal(got, densify(dims, idx, val).reshape(4, 25))
    # full Kruskal tensor: Y(i, p, q) = sum_r lam_r A(i,r) (U1^T B)(p,r) (U2^T C)(q,r)
    dims = (6, 5, 4)
    A, B, C = (rng.standard_normal((d, 2)) for d in dims)
    lam = np.array([1.3, -0.6])
    Xk = np.einsum("r,ir,jr,kr->ijk", lam, A, B, C)
    fidx = [a.astype(np.uint32).ravel() for a in np.indices(dims)]
    U1, U2 = rng.standard_normal((5, 3)), rng.standard_normal((4, 3))
    got = oracle.ttmc(dims, fidx, Xk.ravel(), [np.zeros((6, 3)), U1, U2], 0)
    ref = np.einsum("r,ir,pr,qr->ipq", lam, A, U1.T @ B, U2.T @ C).reshape(6, 9)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("dims,mode", [((6, 5, 4), 1), ((4, 3, 5, 3), 3)])
def test_ttmc_diagonal_is_mttkrp(oracle, dims, mode):
    rng = np.random.default_rng(23)
    idx, val = rand_coo(rng, dims, int(np.prod(dims) * 0.4))
    R = 3
    U = [rng.standard_normal((d, R)) for d in dims]
    Y = oracle.ttmc(dims, idx, val, U, mode)
    nprod = len(dims) - 1
    diag = [sum(r * R ** e for e in range(nprod)) for r in range(R)]
    np.testing.assert_allclose(Y[:, diag], oracle.mttkrp(dims, idx, val, U, mode), rtol=1e-12, atol=1e-12)


def test_ttmc_single_nonzero_and_empty(oracle):
    dims = (3, 4, 2)
    idx = [np.array([2], np.uint32), np.array([1], np.uint32), np.array([0], np.uint32)]
    U = [np.zeros((3, 2)), np.array([[0, 0], [2.0, 3.0], [0, 0], [0, 0]]), np.array([[5.0, 7.0], [0, 0]])]
    Y = oracle.ttmc(dims, idx, np.array([0.5]), U, 0)
    ref = np.zeros((3, 4))
    ref[2] = 0.5 * np.array([2 * 5, 2 * 7, 3 * 5, 3 * 7])
    np.testing.assert_array_equal(Y, ref)
    empty = [np.zeros(0, np.uint32)] * 3
    np.testing.assert_array_equal(oracle.ttmc(dims, empty, np.zeros(0), U, 0), np.zeros((3, 4)))


# ---------------------------------------------------------------- Tucker (HOOI)


def orthonormal(rng, n, r):
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def test_hooi_recovers_exact_multilinear_rank(oracle):
    # X = G x1 A x2 B x3 C with orthonormal A, B, C: one sweep from a random
    # start finds span(A), span(B), span(C) and fit 1
    rng = np.random.default_rng(31)
    dims, R = (8, 7, 6), 2
    A, B, C = (orthonormal(rng, d, R) for d in dims)
    G = rng.standard_normal((R, R, R))
    X = np.einsum("abc,ia,jb,kc->ijk", G, A, B, C)
    idx = [a.astype(np.uint32).ravel() for a in np.indices(dims)]
    init = [rng.standard_normal((d, R)) for d in dims]
    F, fits = oracle.hooi(dims, idx, X.ravel(), init, 2)
    assert abs(fits[0] - 1.0) < 1e-7 and abs(fits[1] - 1.0) < 1e-7
    for Un, T in zip(F, (A, B, C)):
        np.testing.assert_allclose(Un @ Un.T, T @ T.T, atol=1e-10)


def test_hooi_orthonormal_monotone_and_core_identity(oracle):
    rng = np.random.default_rng(32)
    dims, R = (12, 10, 9), 3
    idx, val = rand_coo(rng, dims, 300)
    init = [rng.standard_normal((d, R)) for d in dims]
    F, fits = oracle.hooi(dims, idx, val, init, 6)
    for Un in F:
        np.testing.assert_allclose(Un.T @ Un, np.eye(R), atol=1e-12)
    assert all(b >= a - 1e-12 for a, b in zip(fits, fits[1:]))
    # the fit from the singular values equals the dense residual of the
    # projection X x_k U_k U_k^T
    X = densify(dims, idx, val)
    Gc = np.einsum("ijk,ia,jb,kc->abc", X, *F)
    Xh = np.einsum("abc,ia,jb,kc->ijk", Gc, *F)
    fit_dense = 1.0 - np.linalg.norm(X - Xh) / np.linalg.norm(X)
    assert abs(fits[-1] - fit_dense) < 1e-10
    # each factor's columns are signed so that their largest entry is positive
    for Un in F:
        for r in range(R):
            assert Un[np.argmax(np.abs(Un[:, r])), r] > 0


# ---------------------------------------------------------------- F-COO layout


def test_fcoo_layout_golden_fig2(oracle):
    g = json.load(open(os.path.join(GOLD, "fig2_fcoo_3x3x3.json")))
    coords = np.array(g["coords_input_order"], dtype=np.uint32)
    idx = [coords[:, k] for k in range(3)]
    for key, op, mode in (("mttkrp_mode0", "mttkrp", 0), ("ttm_mode2", "ttm", 2)):
        lay = oracle.fcoo_layout(g["dims"], idx, mode, op, g["threadlen"])
        np.testing.assert_array_equal(coords[lay["perm"]], np.array(g["sorted_coords"]))
        np.testing.assert_array_equal(lay["head"], g[key]["head"])
        np.testing.assert_array_equal(lay["sf"], g[key]["sf"])
        np.testing.assert_array_equal(lay["segkeys"], np.array(g[key]["segkeys"]))
        # the paper's toggling bit-flag marks the same segment starts
        tog = np.array(g[key]["bf_toggle"])
        head_from_toggle = np.concatenate([[1], (tog[1:] != tog[:-1]).astype(np.uint8)])
        np.testing.assert_array_equal(head_from_toggle, lay["head"])


@pytest.mark.parametrize("op,mode", [("mttkrp", 0), ("mttkrp", 1), ("mttkrp", 3), ("ttm", 3), ("ttm", 0)])
def test_fcoo_layout_against_lexsort(oracle, op, mode):
    rng = np.random.default_rng(9)
    dims = (7, 5, 6, 4)
    idx, _ = rand_coo(rng, dims, 300)
    tl = 8
    lay = oracle.fcoo_layout(dims, idx, mode, op, tl)
    N = len(dims)
    if op == "mttkrp":
        order = [mode] + [k for k in range(N) if k != mode]
        nidx = 1
    else:
        order = [k for k in range(N) if k != mode] + [mode]
        nidx = N - 1
    ref_perm = np.lexsort([idx[k] for k in reversed(order)])  # last key is primary
    np.testing.assert_array_equal(lay["perm"], ref_perm)
    keys = np.stack([idx[k][ref_perm] for k in order[:nidx]], 1)
    head = np.ones(300, np.uint8)
    head[1:] = np.any(keys[1:] != keys[:-1], axis=1)
    np.testing.assert_array_equal(lay["head"], head)
    np.testing.assert_array_equal(lay["sf"], head[::tl])
    np.testing.assert_array_equal(lay["segkeys"], keys[head.astype(bool)])


def test_fcoo_layout_rejects_duplicates(oracle):
    idx = [np.array([0, 1, 0], np.uint32), np.array([2, 2, 2], np.uint32), np.array([1, 0, 1], np.uint32)]
    with pytest.raises(oracle.OracleError, match="duplicate"):
        oracle.fcoo_layout((2, 3, 2), idx, 0, "mttkrp", 8)
    with pytest.raises(oracle.OracleError, match="range"):
        oracle.mttkrp((2, 3, 1), idx, np.ones(3), [np.ones((2, 1)), np.ones((3, 1)), np.ones((1, 1))], 0)


# ---------------------------------------------------------------- Algorithm 1


def dense_kruskal(lam, F):
    letters = "abcdefgh"[: len(F)]
    return np.einsum("r," + ",".join(f"{c}r" for c in letters) + "->" + letters, lam, *F)


def test_spd_solve_cholesky_and_pinv(oracle):
    rng = np.random.default_rng(10)
    A = rng.standard_normal((30, 6))
    V = A.T @ A
    M = rng.standard_normal((11, 6))
    X, used = oracle.spd_solve(V, M)
    assert not used
    np.testing.assert_allclose(X, np.linalg.solve(V, M.T).T, rtol=1e-10, atol=1e-10)
    A[:, 5] = A[:, 4]  # rank deficient
    V = A.T @ A
    X, used = oracle.spd_solve(V, M)
    assert used
    np.testing.assert_allclose(X, M @ np.linalg.pinv(V, rcond=1e-12, hermitian=True), rtol=1e-8, atol=1e-9)


def test_cp_als_one_sweep_matches_pinv_rederivation(oracle):
    rng = np.random.default_rng(11)
    dims = (8, 7, 6)
    idx, val = rand_coo(rng, dims, 120)
    R = 3
    init = [rng.uniform(0, 1, (d, R)) for d in dims]
    F, lam, fits, _ = oracle.cp_als(dims, idx, val, init, 1)
    X = densify(dims, idx, val)
    G = [f.copy() for f in init]
    for n in range(3):
        V = np.ones((R, R))
        for k in range(3):
            if k != n:
                V *= G[k].T @ G[k]
        Fn = brute_mttkrp(X, G, n) @ np.linalg.pinv(V)
        nrm = np.linalg.norm(Fn, axis=0)
        G[n] = Fn / nrm
    for n in range(3):
        np.testing.assert_allclose(F[n], G[n], rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(lam, nrm, rtol=1e-9)
    # fit formula against the dense residual
    Xh = dense_kruskal(lam, F)
    fit_direct = 1.0 - np.linalg.norm(X - Xh) / np.linalg.norm(X)
    np.testing.assert_allclose(fits[0], fit_direct, rtol=1e-9, atol=1e-11)


def test_cp_als_fit_monotone_and_exact_recovery(oracle):
    rng = np.random.default_rng(12)
    dims = (9, 8, 7)
    idx, val = rand_coo(rng, dims, 200)
    init = [rng.uniform(0, 1, (d, 4)) for d in dims]
    _, _, fits, _ = oracle.cp_als(dims, idx, val, init, 15)
    assert np.all(np.diff(fits) >= -1e-12), fits
    # a full rank-2 tensor is recovered (fit -> 1) with R = 2
    A, B, C = (rng.standard_normal((d, 2)) for d in dims)
    Xk = dense_kruskal(np.array([2.0, 1.0]), [A, B, C])
    fidx = [a.astype(np.uint32).ravel() for a in np.indices(dims)]
    init = [rng.uniform(0, 1, (d, 2)) for d in dims]
    F, lam, fits, _ = oracle.cp_als(dims, fidx, Xk.ravel(), init, 60)
    assert fits[-1] > 1 - 1e-8, fits[-5:]
    np.testing.assert_allclose(dense_kruskal(lam, F), Xk, atol=1e-6)
    for f in F:
        np.testing.assert_allclose(np.linalg.norm(f, axis=0), 1.0, rtol=1e-12)


def test_cp_als_pinv_fallback_on_deficient_gram(oracle):
    # two modes of size 1 with R = 2 make their Grams rank-1; their Hadamard
    # product (the V of mode 0) has rank <= 1 < R and the pseudo-inverse is used
    rng = np.random.default_rng(13)
    dims = (6, 1, 1)
    idx, val = rand_coo(rng, dims, 5)
    init = [rng.uniform(0, 1, (d, 2)) for d in dims]
    F, lam, fits, npinv = oracle.cp_als(dims, idx, val, init, 3)
    assert npinv > 0
    assert np.all(np.isfinite(fits))


# ---------------------------------------------------------------- sparse fit and adjoint


def test_sparse_fit_loss_bruteforce_and_finite_differences(oracle):
    import synth

    cfg = synth.CONFIGS["fit3_fd"]
    T = synth.make_tensor(cfg)
    dims = T.dims
    idx = T.idx_u32()
    val = T.val.double().numpy()
    rng = np.random.default_rng(14)
    F = [rng.standard_normal((d, cfg.R)) * cfg.R ** (-1 / 6) for d in dims]
    loss, dF, dv = oracle.sparse_fit(dims, idx, val, F)
    model = dense_kruskal(np.ones(cfg.R), F)
    e = model[tuple(a.astype(np.int64) for a in idx)] - val
    np.testing.assert_allclose(loss, 0.5 * np.sum(e * e), rtol=1e-12)
    np.testing.assert_allclose(dv, -e, rtol=1e-12, atol=1e-14)
    h = 1e-6
    for n in range(3):
        for (i, r) in [(0, 0), (dims[n] - 1, cfg.R - 1), (dims[n] // 2, 1)]:
            Fp = [f.copy() for f in F]
            Fm = [f.copy() for f in F]
            Fp[n][i, r] += h
            Fm[n][i, r] -= h
            fd = (oracle.sparse_fit(dims, idx, val, Fp, False, False)[0]
                  - oracle.sparse_fit(dims, idx, val, Fm, False, False)[0]) / (2 * h)
            assert abs(fd - dF[n][i, r]) <= 1e-6 * max(1.0, abs(fd)), (n, i, r, fd, dF[n][i, r])
    for p in (0, 17, len(val) - 1):
        vp = val.copy()
        vm = val.copy()
        vp[p] += h
        vm[p] -= h
        fd = (oracle.sparse_fit(dims, idx, vp, F, False, False)[0]
              - oracle.sparse_fit(dims, idx, vm, F, False, False)[0]) / (2 * h)
        assert abs(fd - dv[p]) <= 1e-6 * max(1.0, abs(fd))


def test_mttkrp_adjoint_identity(oracle):
    rng = np.random.default_rng(15)
    dims = (6, 5, 4, 3)
    idx, val = rand_coo(rng, dims, 90)
    R = 3
    F = [rng.standard_normal((d, R)) for d in dims]
    n = 1
    G = rng.standard_normal((dims[n], R))
    dF, dv = oracle.mttkrp_adjoint(dims, idx, val, F, n, G)
    # <MTTKRP(dval), G> = <dval, dvals>: exact, MTTKRP is linear in the values
    dval = rng.standard_normal(len(val))
    X = densify(dims, idx, dval)
    np.testing.assert_allclose(np.sum(brute_mttkrp(X, F, n) * G), np.dot(dval, dv), rtol=1e-11)
    # multilinear in each other factor: <MTTKRP(F with F_k := D), G> = <D, dF_k>
    Xv = densify(dims, idx, val)
    for k in range(4):
        if k == n:
            assert dF[k] is None
            continue
        D = rng.standard_normal(F[k].shape)
        Fk = [f.copy() for f in F]
        Fk[k] = D
        np.testing.assert_allclose(np.sum(brute_mttkrp(Xv, Fk, n) * G), np.sum(D * dF[k]), rtol=1e-11)


def test_cp_als_mode_steps_compose_to_a_sweep_and_fit_matches_dense(oracle):
    rng = np.random.default_rng(16)
    dims = (7, 6, 5)
    idx, val = rand_coo(rng, dims, 90)
    init = [rng.uniform(0, 1, (d, 3)) for d in dims]
    F_ref, lam_ref, fits, _ = oracle.cp_als(dims, idx, val, init, 2)
    F = [f.copy() for f in init]
    for _ in range(2):
        for n in range(3):
            F, lam, M, _ = oracle.cp_als_mode(dims, idx, val, F, n)
    for a, b in zip(F, F_ref):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(lam, lam_ref, rtol=1e-12)
    fit = oracle.cp_fit(dims, idx, val, F, lam)
    np.testing.assert_allclose(fit, fits[-1], rtol=1e-12)
    X = densify(dims, idx, val)
    direct = 1.0 - np.linalg.norm(X - dense_kruskal(lam, F)) / np.linalg.norm(X)
    np.testing.assert_allclose(fit, direct, rtol=1e-10)


# ---------------------------------------------------------------- multi-threaded build


@pytest.mark.parametrize("dims", [(40, 30, 20), (9, 8, 7, 6)])
def test_mttkrp_rows_is_bitwise_the_oracle_loop(oracle, dims):
    # each output row summed by one thread, in input order, is the serial
    # loop term for term: equal bit for bit in FP64, on every mode (empty
    # slices, a hot slice and a single-nonzero slice included)
    rng = np.random.default_rng(3)
    n = 3000
    idx = [rng.integers(0, d, size=n).astype(np.uint32) for d in dims]
    idx[0][:500] = 2  # one hot slice
    idx[0][500] = dims[0] - 1  # a slice with one nonzero
    idx[0][501:] %= max(dims[0] - 2, 1)  # the slice dims[0] - 2 stays empty
    val = rng.standard_normal(n)
    F = [rng.standard_normal((d, 7)) for d in dims]
    for mode in range(len(dims)):
        rows = oracle.ModeRows(dims, idx, mode)
        a = oracle.mttkrp(dims, idx, val, F, mode)
        b = oracle.mttkrp_rows(rows, val, F)
        assert np.array_equal(a, b), mode
        c = oracle.mttkrp_rows(rows, val.astype(np.float32), [f.astype(np.float32) for f in F], fp32=True)
        absref = oracle.mttkrp(dims, idx, np.abs(val), [np.abs(f) for f in F], mode)
        assert np.all(np.abs(c - a) <= 1e-5 * absref + 1e-30), mode  # FP32 sums of at most 3000 terms


def test_cp_als_rows_matches_cp_als(oracle):
    # Algorithm 1 driven from Python over the multi-threaded loop: the same
    # sweeps as the C oracle
    rng = np.random.default_rng(4)
    dims = (30, 25, 20)
    n = 4000
    lin = rng.choice(np.prod(dims), size=n, replace=False)
    idx = [a.astype(np.uint32) for a in np.unravel_index(lin, dims)]
    val = rng.random(n)
    init = [rng.random((d, 6)) for d in dims]
    f1, l1, fit1, p1 = oracle.cp_als(dims, idx, val, init, 6)
    f2, l2, fit2, p2 = oracle.cp_als_rows(dims, idx, val, init, 6)
    assert np.max(np.abs(fit1 - fit2)) <= 1e-12
    assert p1 == p2
    assert np.max(np.abs(l1 - l2)) <= 1e-10 * np.max(np.abs(l1))
    for a, b in zip(f1, f2):
        assert np.max(np.abs(a - b)) <= 1e-10
