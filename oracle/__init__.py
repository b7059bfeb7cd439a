"""FP64 CPU oracle for the F-COO sparse tensor operations (arXiv 1705.09905).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  The
product library (``paper_1705_09905_gb300``) never imports, links or calls it,
and the two share no code: this wrapper loads ``liboracle.so`` built from
``fcoo_oracle.c`` by plain gcc.

Functions take numpy arrays (or anything ``np.asarray`` accepts); indices are
converted to uint32 per mode and values/factors to float64.  See the C source
for the passage of the paper each routine follows:

* ``mttkrp``        -- Eq. 5 / Eq. 6, Table I row 2 (SpMTTKRP on mode n)
* ``ttm``           -- Eq. 3, Table I row 1 (SpTTM, semi-sparse output)
* ``ttmc``          -- Eq. 4, Table I row 3 (SpTTMc, dense Kronecker-row output)
* ``hooi``          -- Tucker by HOOI around SpTTMc (Sec. II), numpy SVD per mode
* ``fcoo_layout``   -- Sec. IV-B, Table I, Fig. 2 caption (sort order, flags)
* ``cp_als``        -- Algorithm 1 (CP-ALS), N-way
* ``spd_solve``     -- the ``V^dagger`` of Algorithm 1 (Cholesky / pinv)
* ``sparse_fit``    -- loss and gradients of the observed-entry CP fit
* ``mttkrp_adjoint``-- adjoint of Eq. 6 for a given output cotangent
* ``mttkrp_rows``   -- the SpMTTKRP loop of ``mttkrp`` with each output row
                       summed by one OpenMP thread (``fcoo_oracle_omp.c``,
                       gcc -O3 -fopenmp): bitwise equal to ``mttkrp`` in FP64;
                       an FP32 variant times the FP32 CPU baseline
* ``cp_als_rows``   -- Algorithm 1 as ``cp_als``, its MTTKRPs by
                       ``mttkrp_rows``, for runs too large for one core

Parity status: all functions pinned (see tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fcoo_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC_OMP = os.path.join(_HERE, "fcoo_oracle_omp.c")
_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C99, -O2, no vector intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def build_omp(force: bool = False) -> str:
    """Compile liboracle_omp.so (the multi-threaded SpMTTKRP loop) with gcc
    -O3 -fopenmp; contraction into FMAs is off, as in the ISO C99 build of
    liboracle.so, so both round every product and sum alike."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO_OMP) or os.path.getmtime(_SO_OMP) < os.path.getmtime(_SRC_OMP):
        tmp = _SO_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                               tmp, _SRC_OMP])
        os.replace(tmp, _SO_OMP)
    return _SO_OMP


def _load_omp():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            lib = ctypes.CDLL(build_omp())
            for f in ("orp_num_threads", "orp_mode_rows", "orp_mttkrp_f64", "orp_mttkrp_f32"):
                getattr(lib, f).restype = ctypes.c_int
            _lib_omp = lib
    return _lib_omp


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_mttkrp.restype = ctypes.c_int
            lib.orc_ttm.restype = ctypes.c_int64
            lib.orc_ttmc.restype = ctypes.c_int
            lib.orc_fcoo_layout.restype = ctypes.c_int
            lib.orc_cp_als.restype = ctypes.c_int
            lib.orc_spd_solve.restype = ctypes.c_int
            lib.orc_sparse_fit.restype = ctypes.c_int
            lib.orc_mttkrp_adjoint.restype = ctypes.c_int
            lib.orc_gram.restype = None
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _check(st):
    if st < 0:
        raise OracleError({-1: "invalid argument", -2: "index out of range", -3: "duplicate coordinate",
                           -4: "out of memory"}.get(int(st), f"error {st}"))
    return st


class _Coo:
    """Keeps contiguous uint32 index arrays alive and builds the C pointer tables."""

    def __init__(self, dims, idx):
        self.dims = np.ascontiguousarray(np.asarray(dims, dtype=np.uint32))
        self.idx = [np.ascontiguousarray(np.asarray(a, dtype=np.uint32)) for a in idx]
        self.nmodes = len(self.idx)
        self.nnz = int(self.idx[0].shape[0]) if self.nmodes else 0
        self.idx_ptrs = (_u32p * self.nmodes)(*[a.ctypes.data_as(_u32p) for a in self.idx])
        self.dims_ptr = self.dims.ctypes.data_as(_u32p)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr_table(arrs):
    return (_f64p * len(arrs))(*[(a.ctypes.data_as(_f64p) if a is not None else None) for a in arrs])


def mttkrp(dims, idx, val, factors, mode):
    """SpMTTKRP on ``mode`` (Eq. 6): returns dims[mode] x R float64."""
    lib = _load()
    c = _Coo(dims, idx)
    val = _f64(val)
    R = int(np.asarray(factors[(mode + 1) % c.nmodes]).shape[1])
    fs = [(_f64(f) if k != mode else np.zeros((1, R))) for k, f in enumerate(factors)]
    out = np.empty((int(c.dims[mode]), R), dtype=np.float64)
    _check(lib.orc_mttkrp(c.nmodes, c.dims_ptr, ctypes.c_int64(c.nnz), c.idx_ptrs, val.ctypes.data_as(_f64p),
                          _ptr_table(fs), R, mode, out.ctypes.data_as(_f64p)))
    return out


def ttmc(dims, idx, val, factors, mode):
    """SpTTMc on ``mode`` (Eq. 4): returns dims[mode] x R^(N-1) float64, the
    output column of (r_a, r_b, ...) over the product modes in ascending order
    being ((r_a * R) + r_b) * R + ... (first product mode slowest)."""
    lib = _load()
    c = _Coo(dims, idx)
    val = _f64(val)
    R = int(np.asarray(factors[(mode + 1) % c.nmodes]).shape[1])
    fs = [(_f64(f) if k != mode else np.zeros((1, R))) for k, f in enumerate(factors)]
    out = np.empty((int(c.dims[mode]), R ** (c.nmodes - 1)), dtype=np.float64)
    _check(lib.orc_ttmc(c.nmodes, c.dims_ptr, ctypes.c_int64(c.nnz), c.idx_ptrs, val.ctypes.data_as(_f64p),
                        _ptr_table(fs), R, mode, out.ctypes.data_as(_f64p)))
    return out


def ttm(dims, idx, val, U, mode):
    """SpTTM on ``mode`` (Eq. 3): returns (keys nfib x (N-1) uint32, Y nfib x R float64),
    fibres in lexicographic order of the index-mode tuple."""
    lib = _load()
    c = _Coo(dims, idx)
    val = _f64(val)
    U = _f64(U)
    R = int(U.shape[1])
    cap = max(c.nnz, 1)
    keys = np.empty((cap, c.nmodes - 1), dtype=np.uint32)
    out = np.empty((cap, R), dtype=np.float64)
    nfib = _check(lib.orc_ttm(c.nmodes, c.dims_ptr, ctypes.c_int64(c.nnz), c.idx_ptrs, val.ctypes.data_as(_f64p),
                              U.ctypes.data_as(_f64p), R, mode, keys.ctypes.data_as(_u32p),
                              out.ctypes.data_as(_f64p)))
    return keys[:nfib].copy(), out[:nfib].copy()


def fcoo_layout(dims, idx, mode, op, threadlen):
    """F-COO definition (Sec. IV-B): returns dict with perm (F-COO order -> original
    position), head (uint8 per nonzero), sf (uint8 per partition), segkeys
    (nseg x n_index_modes uint32)."""
    lib = _load()
    c = _Coo(dims, idx)
    opi = {"mttkrp": 0, "ttm": 1}.get(op, op)
    nidx = 1 if opi == 0 else c.nmodes - 1
    cap = max(c.nnz, 1)
    perm = np.empty(cap, dtype=np.int64)
    head = np.empty(cap, dtype=np.uint8)
    npart = (c.nnz + threadlen - 1) // threadlen
    sf = np.empty(max(npart, 1), dtype=np.uint8)
    segkeys = np.empty((cap, nidx), dtype=np.uint32)
    nseg = ctypes.c_int64(0)
    _check(lib.orc_fcoo_layout(c.nmodes, c.dims_ptr, ctypes.c_int64(c.nnz), c.idx_ptrs, mode, opi, threadlen,
                               perm.ctypes.data_as(_i64p), head.ctypes.data_as(_u8p), sf.ctypes.data_as(_u8p),
                               segkeys.ctypes.data_as(_u32p), ctypes.byref(nseg)))
    n = c.nnz
    return {"perm": perm[:n].copy(), "head": head[:n].copy(), "sf": sf[:npart].copy(),
            "segkeys": segkeys[:nseg.value].copy(), "nseg": int(nseg.value)}


def gram(F):
    lib = _load()
    F = _f64(F)
    R = int(F.shape[1])
    G = np.empty((R, R), dtype=np.float64)
    lib.orc_gram(F.ctypes.data_as(_f64p), ctypes.c_int64(F.shape[0]), R, G.ctypes.data_as(_f64p))
    return G


def spd_solve(V, M):
    """X = M V^dagger (Algorithm 1's pseudo-inverse reading); returns (X, used_pinv)."""
    lib = _load()
    V = _f64(V)
    M = _f64(M)
    R = int(V.shape[0])
    X = np.empty_like(M)
    used = lib.orc_spd_solve(V.ctypes.data_as(_f64p), R, M.ctypes.data_as(_f64p), ctypes.c_int64(M.shape[0]),
                             X.ctypes.data_as(_f64p))
    return X, bool(used)


def cp_als(dims, idx, val, init_factors, iters):
    """Algorithm 1 for ``iters`` sweeps from ``init_factors``.
    Returns (factors, lambda, fits per sweep, number of pseudo-inverse solves)."""
    lib = _load()
    c = _Coo(dims, idx)
    val = _f64(val)
    fs = [_f64(f).copy() for f in init_factors]
    R = int(fs[0].shape[1])
    lam = np.empty(R, dtype=np.float64)
    fits = np.empty(max(iters, 1), dtype=np.float64)
    npinv = ctypes.c_int(0)
    _check(lib.orc_cp_als(c.nmodes, c.dims_ptr, ctypes.c_int64(c.nnz), c.idx_ptrs, val.ctypes.data_as(_f64p), R,
                          iters, _ptr_table(fs), lam.ctypes.data_as(_f64p), fits.ctypes.data_as(_f64p),
                          ctypes.byref(npinv)))
    return fs, lam, fits[:iters].copy(), int(npinv.value)


def sparse_fit(dims, idx, val, factors, want_dfactors=True, want_dvals=True):
    """Observed-entry CP loss and its gradients.  Returns (loss, dfactors, dvals)."""
    lib = _load()
    c = _Coo(dims, idx)
    val = _f64(val)
    fs = [_f64(f) for f in factors]
    R = int(fs[0].shape[1])
    dfs = [np.empty_like(f) for f in fs] if want_dfactors else None
    dv = np.empty(c.nnz, dtype=np.float64) if want_dvals else None
    loss = ctypes.c_double(0.0)
    _check(lib.orc_sparse_fit(c.nmodes, c.dims_ptr, ctypes.c_int64(c.nnz), c.idx_ptrs, val.ctypes.data_as(_f64p),
                              _ptr_table(fs), R, ctypes.byref(loss), _ptr_table(dfs) if dfs else None,
                              dv.ctypes.data_as(_f64p) if dv is not None else None))
    return float(loss.value), dfs, dv


def mttkrp_adjoint(dims, idx, val, factors, mode, G):
    """Adjoint of SpMTTKRP_mode for cotangent G.  Returns (dfactors with None at
    ``mode``, dvals)."""
    lib = _load()
    c = _Coo(dims, idx)
    val = _f64(val)
    G = _f64(G)
    R = int(G.shape[1])
    fs = [(_f64(f) if k != mode else np.zeros((1, R))) for k, f in enumerate(factors)]
    dfs = [(np.empty((int(c.dims[k]), R)) if k != mode else None) for k in range(c.nmodes)]
    dv = np.empty(c.nnz, dtype=np.float64)
    _check(lib.orc_mttkrp_adjoint(c.nmodes, c.dims_ptr, ctypes.c_int64(c.nnz), c.idx_ptrs,
                                  val.ctypes.data_as(_f64p), _ptr_table(fs), R, mode, G.ctypes.data_as(_f64p),
                                  _ptr_table(dfs), dv.ctypes.data_as(_f64p)))
    return dfs, dv


def cp_als_mode(dims, idx, val, factors, n):
    """One mode update of Algorithm 1 (in place on a copy).  Returns
    (factors, lambda, M, used_pinv)."""
    lib = _load()
    lib.orc_cp_als_mode.restype = ctypes.c_int
    c = _Coo(dims, idx)
    val = _f64(val)
    fs = [_f64(f).copy() for f in factors]
    R = int(fs[0].shape[1])
    lam = np.empty(R, dtype=np.float64)
    M = np.empty((int(c.dims[n]), R), dtype=np.float64)
    used = _check(lib.orc_cp_als_mode(c.nmodes, c.dims_ptr, ctypes.c_int64(c.nnz), c.idx_ptrs,
                                      val.ctypes.data_as(_f64p), R, n, _ptr_table(fs), lam.ctypes.data_as(_f64p),
                                      M.ctypes.data_as(_f64p)))
    return fs, lam, M, bool(used)


def cp_fit(dims, idx, val, factors, lam):
    """Fit 1 - |X - [lambda; F]| / |X| of Algorithm 1's model (Grams identity)."""
    lib = _load()
    lib.orc_cp_fit.restype = ctypes.c_double
    c = _Coo(dims, idx)
    val = _f64(val)
    fs = [_f64(f) for f in factors]
    lam = _f64(lam)
    return float(lib.orc_cp_fit(c.nmodes, c.dims_ptr, ctypes.c_int64(c.nnz), c.idx_ptrs, val.ctypes.data_as(_f64p),
                                int(fs[0].shape[1]), _ptr_table(fs), lam.ctypes.data_as(_f64p)))


def sign_fix(U):
    """Column sign convention shared by the Tucker factors of both sides:
    each column's entry of largest magnitude (the first, on ties) is made
    positive.  Singular vectors are defined only up to sign."""
    U = np.array(U, dtype=np.float64, copy=True)
    for r in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, r])))
        if U[i, r] < 0:
            U[:, r] = -U[:, r]
    return U


def hooi_mode(dims, idx, val, factors, n, R):
    """One HOOI factor update (Sec. II; Eq. 4 as its TTM chain): Y_(n) =
    SpTTMc of mode n with the other factors, then the R leading left singular
    vectors of Y_(n) (numpy SVD), sign-fixed.  Returns (U_n, sigma^2 of the
    R leading singular values)."""
    Y = ttmc(dims, idx, val, factors, n)
    U, s, _ = np.linalg.svd(Y, full_matrices=False)
    k = min(R, U.shape[1])
    Un = np.zeros((int(dims[n]), R))
    Un[:, :k] = U[:, :k]
    sig2 = np.zeros(R)
    sig2[:k] = s[:k] ** 2
    return sign_fix(Un), sig2


def hooi(dims, idx, val, init_factors, iters):
    """Tucker decomposition by higher-order orthogonal iteration: `iters`
    sweeps over the modes in order, each mode replaced by hooi_mode with the
    latest factors.  The core is G = Y_(N-1) times U_(N-1)^T, so |G|^2 is the
    sum of the last mode's sigma^2, and fit = 1 - sqrt(max(0, |X|^2 -
    |G|^2)) / |X| (the factors are orthonormal).  Returns (factors, fits)."""
    F = [np.array(f, dtype=np.float64) for f in init_factors]
    R = F[0].shape[1]
    x2 = float(np.sum(np.asarray(val, dtype=np.float64) ** 2))
    fits = []
    for _ in range(iters):
        for n in range(len(dims)):
            F[n], sig2 = hooi_mode(dims, idx, val, F, n, R)
        g2 = float(np.sum(sig2))
        fits.append(1.0 - np.sqrt(max(0.0, x2 - g2)) / np.sqrt(x2))
    return F, fits


# ---------------------------------------------------------------- multi-threaded loop


def num_threads() -> int:
    """Threads the OpenMP build runs on (OMP_NUM_THREADS, else all cores)."""
    return int(_load_omp().orp_num_threads())


class ModeRows:
    """The nonzeros of a COO tensor grouped by their index in ``mode`` (stable:
    each row keeps its nonzeros in input order): rowptr (dims[mode] + 1) and
    order (nnz), for ``mttkrp_rows``."""

    def __init__(self, dims, idx, mode):
        lib = _load_omp()
        self.coo = _Coo(dims, idx)
        self.mode = int(mode)
        self.rowptr = np.empty(int(self.coo.dims[mode]) + 1, dtype=np.int64)
        self.order = np.empty(max(self.coo.nnz, 1), dtype=np.int64)
        _check(lib.orp_mode_rows(ctypes.c_int64(self.coo.nnz), self.coo.idx[mode].ctypes.data_as(_u32p),
                                 ctypes.c_uint32(int(self.coo.dims[mode])), self.rowptr.ctypes.data_as(_i64p),
                                 self.order.ctypes.data_as(_i64p)))


def mttkrp_rows(rows: ModeRows, val, factors, fp32: bool = False):
    """SpMTTKRP (Eq. 6) on rows.mode with every output row summed by one
    thread: FP64 (bitwise equal to ``mttkrp``), or with FP32 values, factors
    and sums when fp32 is set.  Returns dims[mode] x R."""
    lib = _load_omp()
    c, mode = rows.coo, rows.mode
    R = int(np.asarray(factors[(mode + 1) % c.nmodes]).shape[1])
    if fp32:
        dt, ptr, fn = np.float32, ctypes.POINTER(ctypes.c_float), lib.orp_mttkrp_f32
    else:
        dt, ptr, fn = np.float64, _f64p, lib.orp_mttkrp_f64
    val = np.ascontiguousarray(np.asarray(val, dtype=dt))
    fs = [(np.ascontiguousarray(np.asarray(f, dtype=dt)) if k != mode else np.zeros((1, R), dt))
          for k, f in enumerate(factors)]
    table = (ptr * len(fs))(*[f.ctypes.data_as(ptr) for f in fs])
    out = np.empty((int(c.dims[mode]), R), dtype=dt)
    _check(fn(c.nmodes, c.dims_ptr, c.idx_ptrs, val.ctypes.data_as(ptr), table, R, mode,
              rows.rowptr.ctypes.data_as(_i64p), rows.order.ctypes.data_as(_i64p), out.ctypes.data_as(ptr)))
    return out


def cp_als_rows(dims, idx, val, init_factors, iters, rows=None):
    """Algorithm 1 for ``iters`` sweeps from ``init_factors``, the steps of
    ``cp_als`` in its order: M = SpMTTKRP_n (``mttkrp_rows``, FP64), V = the
    Hadamard product of the other modes' Grams, F_n = M V^dagger
    (``spd_solve``), columns normalised by their 2-norms (lambda = the norms of
    the last mode), and after each sweep fit = 1 - sqrt(max(0, |X|^2 +
    lambda^T (Hadamard of all Grams) lambda - 2 <X, Xhat>)) / |X| with
    <X, Xhat> = sum_r lambda_r sum_i M_last(i, r) F_last(i, r).  ``rows``: one
    ModeRows per mode (built here if None).  Returns (factors, lambda, fits,
    number of pseudo-inverse solves)."""
    N = len(dims)
    val = _f64(val)
    rows = rows or [ModeRows(dims, idx, n) for n in range(N)]
    F = [_f64(f).copy() for f in init_factors]
    R = F[0].shape[1]
    x2 = float(np.dot(val, val))
    lam = np.ones(R)
    fits, npinv = [], 0
    M = None
    for _ in range(iters):
        for n in range(N):
            M = mttkrp_rows(rows[n], val, F)
            V = np.ones((R, R))
            for k in range(N):
                if k != n:
                    V *= gram(F[k])
            F[n], used = spd_solve(V, M)
            npinv += int(used)
            nrm = np.sqrt(np.einsum("ir,ir->r", F[n], F[n]))
            lam = nrm.copy()
            F[n] = np.where(nrm > 0, F[n] / np.where(nrm > 0, nrm, 1.0), F[n])
        V = np.ones((R, R))
        for k in range(N):
            V *= gram(F[k])
        xhat2 = float(lam @ V @ lam)
        inner = float(np.dot(lam, np.einsum("ir,ir->r", M, F[N - 1])))
        fits.append(1.0 - np.sqrt(max(0.0, x2 + xhat2 - 2.0 * inner)) / np.sqrt(x2))
    return F, lam, np.array(fits), npinv
