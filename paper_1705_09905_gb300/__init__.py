"""GB300 (sm_103a) implementation of the F-COO sparse tensor kernels of
"A Unified Optimization Approach for Sparse Tensor Operations on GPUs"
(Liu, Wen, Sarwate, Mehri Dehnavi, 2017).

This module is argument marshalling over the C ABI of ``libfcoo.so``
(``include/fcoo.h``): every step of SpMTTKRP, SpTTM, CP-ALS and the sparse-fit
adjoint runs in the library's CUDA kernels.  PyTorch provides device memory
and the current stream.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from ._lib import FcooError, FcooInfo, check, lib, ptr_array

__all__ = ["FCOO", "FcooError", "spmttkrp", "spmttkrp_gather_bound", "spttm", "table2_bytes", "MTTKRP", "TTM", "F32", "BF16", "lib"]

MTTKRP, TTM = 0, 1
F32, BF16 = 0, 1
_OPS = {"mttkrp": MTTKRP, "ttm": TTM, MTTKRP: MTTKRP, TTM: TTM}


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"factor dtype {t.dtype} not supported (float32 or bfloat16)")


def _as_u32(a):
    """Index array -> (pointer, keepalive): uint32 bits, host or device."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            t = a.to(torch.int64).to(torch.int32).contiguous() if a.dtype != torch.int32 else a.contiguous()
            return t.data_ptr(), t
        a = a.numpy()
    arr = np.ascontiguousarray(np.asarray(a).astype(np.uint32, copy=False))
    return arr.ctypes.data, arr


def _as_f32(a):
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            t = a.to(torch.float32).contiguous()
            return t.data_ptr(), t
        a = a.numpy()
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return arr.ctypes.data, arr


def table2_bytes(nprod: int, nnz: int, threadlen: int, index_bytes: int = 4) -> int:
    """Bytes of the Table II arrays for ``nnz`` nonzeros with ``index_bytes``
    (4, or 2 after index compression) per product-mode index (host only)."""
    return int(lib.fcoo_table2_bytes_ex(nprod, nnz, threadlen, index_bytes))


class FCOO:
    """A device-resident F-COO tensor for one operation on one mode (Sec. IV-B)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        info = FcooInfo()
        check(lib.fcoo_info(self._h, ctypes.byref(info)))
        self.nmodes = info.nmodes
        self.mode = info.mode
        self.op = info.op
        self.threadlen = info.threadlen
        self.nnz = int(info.nnz)
        self.nseg = int(info.nseg)
        self.nfib = int(info.nfib)
        self.dims = tuple(int(info.dims[k]) for k in range(info.nmodes))
        self.prod_modes = tuple(int(info.prod_modes[k]) for k in range(info.nprod))
        self.idx_modes = tuple(int(info.idx_modes[k]) for k in range(info.nidx))
        self.bytes = {k: int(getattr(info, "bytes_" + k)) for k in
                      ("val", "pidx", "bf", "sf", "table2", "segmap", "aux", "scratch", "pidx16")}
        self.compressed = self.bytes["pidx16"] > 0

    @classmethod
    def build(cls, idx: Sequence, val, dims: Sequence[int], mode: int, op="mttkrp", threadlen: int = 8,
              stream=None) -> "FCOO":
        """Build from per-mode index arrays (numpy / torch, host or device) and values."""
        dims = [int(d) for d in dims]
        N = len(dims)
        if len(idx) != N:
            raise ValueError("need one index array per mode")
        keep = []
        ptrs = []
        for a in idx:
            p, k = _as_u32(a)
            ptrs.append(p)
            keep.append(k)
        vp, vk = _as_f32(val)
        keep.append(vk)
        nnz = int(len(vk)) if not isinstance(vk, torch.Tensor) else int(vk.numel())
        dims_arr = (ctypes.c_uint32 * N)(*dims)
        pp, _pk = ptr_array(ptrs)
        out = ctypes.c_void_p()
        st = lib.fcoo_build(N, ctypes.cast(dims_arr, ctypes.c_void_p), nnz, pp, vp, int(mode), _OPS[op],
                            int(threadlen), _stream(stream) if torch.cuda.is_available() else None,
                            ctypes.byref(out))
        check(st)
        return cls(out.value)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            lib.fcoo_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compress_indices(self, stream=None) -> "FCOO":
        """Add 16-bit copies of the product-mode index streams (every
        product-mode dimension <= 65,536); SpMTTKRP and SpTTM then read them
        where their kernel takes them (Table II with 2-byte indices)."""
        check(lib.fcoo_compress_indices(self._h, _stream(stream) if torch.cuda.is_available() else None))
        info = FcooInfo()
        check(lib.fcoo_info(self._h, ctypes.byref(info)))
        self.bytes["pidx16"] = int(info.bytes_pidx16)
        self.compressed = True
        return self

    def layout(self) -> dict:
        """Copy the F-COO arrays to host numpy arrays."""
        n = self.nnz
        nw = (n + 31) // 32
        nsfw = ((n + self.threadlen - 1) // self.threadlen + 31) // 32
        perm = np.empty(n, np.uint32)
        bf = np.empty(nw, np.uint32)
        sf = np.empty(nsfw, np.uint32)
        segkeys = np.empty(self.nseg * len(self.idx_modes), np.uint32)
        pidx = np.empty(len(self.prod_modes) * n, np.uint32)
        val = np.empty(n, np.float32)
        check(lib.fcoo_copy_layout(self._h, perm.ctypes.data, bf.ctypes.data, sf.ctypes.data, segkeys.ctypes.data,
                                   pidx.ctypes.data, val.ctypes.data, _stream(None)))
        return {"perm": perm, "bf": bf, "sf": sf, "segkeys": segkeys.reshape(self.nseg, len(self.idx_modes)),
                "pidx": pidx.reshape(len(self.prod_modes), n), "val": val}

    def fibre_indices(self) -> np.ndarray:
        keys = np.empty(self.nseg * len(self.idx_modes), np.uint32)
        check(lib.fcoo_fibre_indices(self._h, keys.ctypes.data, _stream(None)))
        return keys.reshape(self.nseg, len(self.idx_modes))


def _check_factor(t: torch.Tensor, rows: int, R: int, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.shape != (rows, R) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {rows}x{R} tensor, got {tuple(t.shape)}")


def spmttkrp(X: FCOO, factors: Sequence[Optional[torch.Tensor]], out: Optional[torch.Tensor] = None,
             stream=None) -> torch.Tensor:
    """SpMTTKRP on the handle's mode (Eq. 6): dims[mode] x R float32 result."""
    if X.op != MTTKRP:
        raise ValueError("handle was built for SpTTM")
    ref = factors[X.prod_modes[0]]
    R = int(ref.shape[1])
    dt = _dtype_code(ref)
    ptrs = []
    for k in range(X.nmodes):
        if k == X.mode:
            ptrs.append(None)
            continue
        f = factors[k]
        _check_factor(f, X.dims[k], R, f"factors[{k}]")
        if f.dtype != ref.dtype:
            raise TypeError("all factors must share one dtype")
        ptrs.append(f.data_ptr())
    if out is None:
        out = torch.empty((X.dims[X.mode], R), dtype=torch.float32, device=ref.device)
    pp, _keep = ptr_array(ptrs)
    check(lib.spmttkrp(X.handle, pp, dt, R, out.data_ptr(), _stream(stream)))
    return out


def spmttkrp_gather_bound(X: FCOO, factors: Sequence[Optional[torch.Tensor]], count: Optional[torch.Tensor] = None,
                          stream=None) -> torch.Tensor:
    """The factor-row loads of spmttkrp on this 3-way handle and nothing else
    (a measurement aid for the gather bound of Eq. 6).  Returns a one-element
    int64 device tensor that receives the number of rows loaded."""
    if X.op != MTTKRP:
        raise ValueError("handle was built for SpTTM")
    ref = factors[X.prod_modes[0]]
    R = int(ref.shape[1])
    dt = _dtype_code(ref)
    ptrs = []
    for k in range(X.nmodes):
        if k == X.mode:
            ptrs.append(None)
            continue
        f = factors[k]
        _check_factor(f, X.dims[k], R, f"factors[{k}]")
        if f.dtype != ref.dtype:
            raise TypeError("all factors must share one dtype")
        ptrs.append(f.data_ptr())
    if count is None:
        count = torch.empty(1, dtype=torch.int64, device=ref.device)
    pp, _keep = ptr_array(ptrs)
    check(lib.spmttkrp_gather_bound(X.handle, pp, dt, R, count.data_ptr(), _stream(stream)))
    return count


def spttm(X: FCOO, U: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """SpTTM on the handle's mode (Eq. 3): nfib x R float32 semi-sparse result,
    rows in the order of ``X.fibre_indices()``."""
    if X.op != TTM:
        raise ValueError("handle was built for SpMTTKRP")
    R = int(U.shape[1])
    _check_factor(U, X.dims[X.mode], R, "U")
    if out is None:
        out = torch.empty((X.nseg, R), dtype=torch.float32, device=U.device)
    check(lib.spttm(X.handle, U.data_ptr(), _dtype_code(U), R, out.data_ptr(), _stream(stream)))
    return out


def spttmc(X: FCOO, factors: Sequence[Optional[torch.Tensor]], out: Optional[torch.Tensor] = None,
           stream=None) -> torch.Tensor:
    """SpTTMc on the handle's mode (Eq. 4) with factors of one rank R and one
    dtype (float32 or bfloat16): dims[mode] x R^(N-1) float32, column
    ((r_a * R) + r_b) * R + ... over the other modes a < b < ... (the first
    slowest).  Takes an SpMTTKRP handle."""
    if X.op != MTTKRP:
        raise ValueError("SpTTMc takes a handle built for SpMTTKRP")
    ref = factors[X.prod_modes[0]]
    R = int(ref.shape[1])
    dt = _dtype_code(ref)
    ptrs = []
    for k in range(X.nmodes):
        if k == X.mode:
            ptrs.append(None)
            continue
        f = factors[k]
        _check_factor(f, X.dims[k], R, f"factors[{k}]")
        if f.dtype != ref.dtype:
            raise TypeError("all factors must share one dtype")
        ptrs.append(f.data_ptr())
    if out is None:
        out = torch.empty((X.dims[X.mode], R ** (X.nmodes - 1)), dtype=torch.float32, device=ref.device)
    pp, _keep = ptr_array(ptrs)
    check(lib.spttmc(X.handle, pp, dt, R, out.data_ptr(), _stream(stream)))
    return out


__all__ += ["spttmc"]


class SpTTMcPlan:
    """SpTTMc of a 3-way tensor by fibres (Eq. 4 regrouped through Eq. 3):
    an SpTTM along the last product mode b into fibre sums, then Eq. 4 over
    the fibres.  ``Xttm`` is the SpTTM handle along b (b = 2 for mode 0 or 1,
    1 for mode 2); it must stay open while the plan is used."""

    def __init__(self, Xttm: FCOO, mode: int, R: int, threadlen: int = 8, stream=None):
        out = ctypes.c_void_p()
        check(lib.spttmc_plan_create(Xttm.handle, int(mode), int(R), int(threadlen), ctypes.byref(out),
                                     _stream(stream)))
        self._h = out
        self._X = Xttm  # keeps the handle alive
        self.mode, self.R, self.dims = int(mode), int(R), tuple(Xttm.dims)
        nf, nb = ctypes.c_int64(), ctypes.c_int64()
        check(lib.spttmc_plan_info(self._h, ctypes.byref(nf), ctypes.byref(nb)))
        self.nfib, self.device_bytes = nf.value, nb.value

    def run(self, factors: Sequence[Optional[torch.Tensor]], out: Optional[torch.Tensor] = None,
            stream=None) -> torch.Tensor:
        """dims[mode] x R^2 float32, columns r_a * R + r_b (a < b the other modes)."""
        ptrs = []
        ref = None
        for k in range(3):
            if k == self.mode:
                ptrs.append(None)
                continue
            f = factors[k]
            _check_factor(f, self.dims[k], self.R, f"factors[{k}]")
            if f.dtype != torch.float32:
                raise TypeError("SpTTMc takes float32 factors")
            ptrs.append(f.data_ptr())
            ref = f
        if out is None:
            out = torch.empty((self.dims[self.mode], self.R * self.R), dtype=torch.float32, device=ref.device)
        pp, _keep = ptr_array(ptrs)
        check(lib.spttmc_plan_run(self._h, pp, F32, out.data_ptr(), _stream(stream)))
        return out

    def close(self):
        if self._h is not None and self._h.value:
            lib.spttmc_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ += ["SpTTMcPlan"]


# ---------------------------------------------------------------- CP-ALS (Algorithm 1)


class CPState:
    """Device state of a rank-R CP decomposition driven by ``cp_als_iter``."""

    def __init__(self, dims: Sequence[int], R: int, init: Sequence, dtype=torch.float32, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.R = int(R)
        self.dtype = dtype
        code = BF16 if dtype == torch.bfloat16 else F32
        keep = []
        ptrs = []
        for k, f in enumerate(init):
            if isinstance(f, torch.Tensor):
                t = f.detach().to(torch.float32).contiguous()
                if not t.is_cuda:
                    t = t.numpy()
            else:
                t = np.ascontiguousarray(np.asarray(f, dtype=np.float32))
            if tuple(t.shape) != (self.dims[k], self.R):
                raise ValueError(f"init[{k}] must be {self.dims[k]}x{self.R}")
            keep.append(t)
            ptrs.append(t.data_ptr() if isinstance(t, torch.Tensor) else t.ctypes.data)
        dims_arr = (ctypes.c_uint32 * len(self.dims))(*self.dims)
        pp, _pk = ptr_array(ptrs)
        out = ctypes.c_void_p()
        check(lib.cp_state_create(len(self.dims), ctypes.cast(dims_arr, ctypes.c_void_p), self.R, code, pp,
                                  _stream(stream), ctypes.byref(out)))
        self._h = out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.cp_state_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def use_fibres(self, Xttm: Optional[FCOO], threadlen: int = 8, stream=None):
        """3-way only: modes 0 and 1 reuse the mode-2 fibre sums (``Xttm`` is
        the SpTTM handle along mode 2; None turns the reuse off)."""
        check(lib.cp_state_use_fibres(self._h, Xttm.handle if Xttm is not None else None, int(threadlen),
                                      _stream(stream)))
        self._fib = Xttm  # keeps the handle alive
        return self

    def iterate(self, Xn: Sequence[FCOO], sweeps: int = 1, stream=None):
        """Run ``sweeps`` sweeps of Algorithm 1 (asynchronous on the stream)."""
        hs = (ctypes.c_void_p * len(Xn))(*[x.handle.value for x in Xn])
        for _ in range(int(sweeps)):
            check(lib.cp_als_iter(ctypes.cast(hs, ctypes.POINTER(ctypes.c_void_p)), self._h, _stream(stream)))
        return self

    def set_dtype(self, dtype, stream=None):
        """Change the factor storage type in place (``cp_state_set_dtype``):
        BF16 -> FP32 is exact, FP32 -> BF16 rounds and recomputes the Grams."""
        code = BF16 if dtype == torch.bfloat16 else F32
        check(lib.cp_state_set_dtype(self._h, code, _stream(stream)))
        self.dtype = dtype
        return self

    def stats(self, stream=None):
        lam = np.empty(self.R, np.float64)
        fit = ctypes.c_double()
        iters = ctypes.c_int()
        npinv = ctypes.c_int()
        check(lib.cp_state_stats(self._h, lam.ctypes.data, ctypes.byref(fit), ctypes.byref(iters),
                                 ctypes.byref(npinv), _stream(stream)))
        return {"lambda": lam, "fit": fit.value, "iters": iters.value, "npinv": npinv.value}

    @property
    def fit(self) -> float:
        return self.stats()["fit"]

    def factor(self, k: int, device="cuda") -> torch.Tensor:
        out = torch.empty((self.dims[k], self.R), dtype=torch.float32, device=device)
        check(lib.cp_state_copy_factor(self._h, int(k), out.data_ptr(), _stream(None)))
        return out

    def save(self) -> bytes:
        n = int(lib.cp_state_blob_size(self._h))
        buf = ctypes.create_string_buffer(n)
        check(lib.cp_state_save(self._h, buf, n, _stream(None)))
        return buf.raw

    def load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        check(lib.cp_state_load(self._h, buf, len(blob), _stream(None)))
        return self


__all__ += ["CPState"]


class TuckerState:
    """Device state of a rank-(R, ..., R) Tucker decomposition driven by
    ``tucker_hooi_iter`` (HOOI around SpTTMc, Eq. 4)."""

    def __init__(self, dims: Sequence[int], R: int, init: Sequence, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.R = int(R)
        keep, ptrs = [], []
        for k, f in enumerate(init):
            if isinstance(f, torch.Tensor):
                t = f.detach().to(torch.float32).contiguous()
                if not t.is_cuda:
                    t = t.numpy()
            else:
                t = np.ascontiguousarray(np.asarray(f, dtype=np.float32))
            if tuple(t.shape) != (self.dims[k], self.R):
                raise ValueError(f"init[{k}] must be {self.dims[k]}x{self.R}")
            keep.append(t)
            ptrs.append(t.data_ptr() if isinstance(t, torch.Tensor) else t.ctypes.data)
        dims_arr = (ctypes.c_uint32 * len(self.dims))(*self.dims)
        pp, _pk = ptr_array(ptrs)
        out = ctypes.c_void_p()
        check(lib.tucker_state_create(len(self.dims), ctypes.cast(dims_arr, ctypes.c_void_p), self.R, pp,
                                      _stream(stream), ctypes.byref(out)))
        self._h = out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.tucker_state_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self, Xn: Sequence[FCOO], iters: int = 1, stream=None):
        """Run ``iters`` HOOI iterations (asynchronous on the stream)."""
        hs = (ctypes.c_void_p * len(Xn))(*[x.handle.value for x in Xn])
        for _ in range(int(iters)):
            check(lib.tucker_hooi_iter(ctypes.cast(hs, ctypes.POINTER(ctypes.c_void_p)), self._h, _stream(stream)))
        return self

    def stats(self, stream=None) -> dict:
        fit, g2 = ctypes.c_double(), ctypes.c_double()
        it, nnull = ctypes.c_int(), ctypes.c_int()
        check(lib.tucker_state_stats(self._h, ctypes.byref(fit), ctypes.byref(g2), ctypes.byref(it),
                                     ctypes.byref(nnull), _stream(stream)))
        return {"fit": fit.value, "core_sq": g2.value, "iters": it.value, "null_directions": nnull.value}

    def factor(self, n: int, stream=None) -> np.ndarray:
        out = np.empty((self.dims[n], self.R), dtype=np.float32)
        check(lib.tucker_state_copy_factor(self._h, int(n), out.ctypes.data, _stream(stream)))
        return out


__all__ += ["TuckerState"]


# ---------------------------------------------------------------- differentiation


def _factor_ptrs(factors, dims, R):
    ref = next(f for f in factors if f is not None)
    ptrs = []
    for k, f in enumerate(factors):
        if f is None:
            ptrs.append(None)
            continue
        _check_factor(f, dims[k], R, f"factors[{k}]")
        if f.dtype != ref.dtype:
            raise TypeError("all factors must share one dtype")
        ptrs.append(f.data_ptr())
    return ptrs, _dtype_code(ref)


def _handles(Xn):
    arr = (ctypes.c_void_p * len(Xn))(*[x.handle.value for x in Xn])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def sparse_fit_grad(Xn: Sequence[FCOO], factors: Sequence[torch.Tensor], want_dvals: bool = False, stream=None,
                    modes: Optional[Sequence[int]] = None):
    """Loss 1/2 sum_obs (model - x)^2 and its gradients w.r.t. the factors of
    ``modes`` (default: every factor; the others are None) and the values, in
    the caller's COO order -- kind 0 of spmttkrp_backward."""
    dims = Xn[0].dims
    R = int(factors[0].shape[1])
    ptrs, dt = _factor_ptrs(factors, dims, R)
    dev = factors[0].device
    want = set(range(len(dims)) if modes is None else (int(m) for m in modes))
    grads = [torch.empty((d, R), dtype=torch.float32, device=dev) if n in want else None for n, d in enumerate(dims)]
    dvals = torch.empty(Xn[0].nnz, dtype=torch.float32, device=dev) if want_dvals else None
    loss = torch.empty((), dtype=torch.float64, device=dev)
    hp, _k1 = _handles(Xn)
    fp, _k2 = ptr_array(ptrs)
    gp, _k3 = ptr_array([g.data_ptr() if g is not None else None for g in grads])
    check(lib.spmttkrp_backward(hp, fp, dt, R, None, 0, 0, gp, dvals.data_ptr() if dvals is not None else None,
                                loss.data_ptr(), _stream(stream)))
    return loss, grads, dvals


def sparse_cp_loss(X: FCOO, factors: Sequence[torch.Tensor], stream=None) -> torch.Tensor:
    """Forward value 1/2 sum_obs (model - x)^2 (device float64 scalar)."""
    R = int(factors[0].shape[1])
    ptrs, dt = _factor_ptrs(factors, X.dims, R)
    loss = torch.empty((), dtype=torch.float64, device=factors[0].device)
    fp, _k = ptr_array(ptrs)
    check(lib.sparse_cp_loss(X.handle, fp, dt, R, loss.data_ptr(), _stream(stream)))
    return loss


def spmttkrp_adjoint(Xn: Sequence[FCOO], factors: Sequence[torch.Tensor], mode: int, gradM: torch.Tensor,
                     want_dvals: bool = True, stream=None):
    """Adjoint of SpMTTKRP_mode for cotangent gradM (kind 1): gradients of every
    other factor (None at `mode`) and of the values (caller's COO order)."""
    dims = Xn[0].dims
    R = int(gradM.shape[1])
    _check_factor(gradM, dims[mode], R, "gradM")
    fl = [None if k == mode else factors[k] for k in range(len(dims))]
    ptrs, dt = _factor_ptrs(fl, dims, R)
    dev = gradM.device
    grads = [None if k == mode else torch.empty((dims[k], R), dtype=torch.float32, device=dev)
             for k in range(len(dims))]
    dvals = torch.empty(Xn[0].nnz, dtype=torch.float32, device=dev) if want_dvals else None
    hp, _k1 = _handles(Xn)
    fp, _k2 = ptr_array(ptrs)
    gp, _k3 = ptr_array([g.data_ptr() if g is not None else None for g in grads])
    check(lib.spmttkrp_backward(hp, fp, dt, R, gradM.data_ptr(), 1, int(mode), gp,
                                dvals.data_ptr() if dvals is not None else None, None, _stream(stream)))
    return grads, dvals


class SparseCPLoss(torch.autograd.Function):
    """loss = 1/2 sum over observed entries of (sum_r prod_k F_k(i_k, r) - x)^2.

    ``Xn`` holds one SpMTTKRP handle per mode of the observed tensor.  The
    forward pass runs the fused residual + adjoint kernels once and keeps the
    gradients; backward scales them by the incoming gradient."""

    @staticmethod
    def forward(ctx, Xn, *factors):
        if any(ctx.needs_input_grad[1:]):
            loss, grads, _ = sparse_fit_grad(Xn, [f.detach() for f in factors])
            ctx.save_for_backward(*grads)
        else:
            loss = sparse_cp_loss(Xn[0], [f.detach() for f in factors])
        return loss

    @staticmethod
    def backward(ctx, gout):
        grads = ctx.saved_tensors
        return (None,) + tuple((g * gout.to(g.dtype)).to(torch.float32) for g in grads)


class SpMTTKRPFunction(torch.autograd.Function):
    """M = SpMTTKRP_mode(X, F) with the hand-written adjoint as backward.

    ``Xn`` holds one SpMTTKRP handle per mode (the adjoint of factor k runs on
    the mode-k copy); float32 factors."""

    @staticmethod
    def forward(ctx, Xn, mode, *factors):
        ctx.Xn = Xn
        ctx.mode = mode
        ctx.save_for_backward(*[f.detach() for f in factors])
        fl = [None if k == mode else f.detach() for k, f in enumerate(factors)]
        return spmttkrp(Xn[mode], fl)

    @staticmethod
    def backward(ctx, gM):
        factors = ctx.saved_tensors
        grads, _ = spmttkrp_adjoint(ctx.Xn, list(factors), ctx.mode, gM.contiguous().float(), want_dvals=False)
        return (None, None) + tuple(grads)


__all__ += ["sparse_fit_grad", "sparse_cp_loss", "spmttkrp_adjoint", "SparseCPLoss", "SpMTTKRPFunction"]
