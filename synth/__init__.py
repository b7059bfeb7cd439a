"""Seeded synthetic sparse tensors shaped like the paper's workloads.

This module is the single input source shared by the FP64 oracle (``oracle/``)
and the CUDA path (``paper_1705_09905_gb300``).  It holds none of the method's
arithmetic: it draws coordinates, values and dense factor matrices, nothing
else (the one exception, clearly separated below, evaluates a ground-truth
Kruskal model to *define* the observed values of the sparse-fit workload).

Recipe (all draws from one ``torch.Generator`` seeded with ``seed`` on the
device the tensor is built on; CPU and CUDA draws therefore differ, the
distributions do not):

* coordinates per mode are either uniform over ``[0, I_k)`` or bounded Zipf:
  rank ``k in 1..I_k`` with probability proportional to ``k**-s`` sampled by
  inverse CDF, mapped to an index through a seeded permutation of ``[0, I_k)``;
* coordinates are drawn in rounds and merged (values of repeated coordinates
  are summed, COO coalesce semantics) until at least ``nnz`` distinct
  coordinates exist; the surplus is dropped by a seeded random choice, so the
  tensor has exactly ``nnz`` nonzeros, in random order;
* values are U(0,1) or lognormal(0,1) per draw;
* dense factors are N(0,1) float32 (or U(0,1) for CP-ALS initialisation).

The stand-in workloads (the paper's FROSTT tensors are not available) are in
``CONFIGS``; ``scaled()`` shrinks one while keeping its distributions.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional, Sequence, Tuple, Union

import torch

Dist = Union[str, Tuple[str, float]]  # "uniform" or ("zipf", s)


@dataclass(frozen=True)
class TensorConfig:
    name: str
    dims: Tuple[int, ...]
    nnz: int
    dists: Tuple[Dist, ...]
    values: str = "uniform"  # "uniform" | "lognormal" | "kruskal"
    R: int = 16
    seed: int = 0
    kruskal_rank: int = 0
    noise_std: float = 0.0
    note: str = ""


CONFIGS = {
    # tiny plain case: SpMTTKRP on all modes and SpTTM along the last mode
    "tiny": TensorConfig("tiny", (200, 150, 100), 10_000, ("uniform",) * 3, "uniform", R=16, seed=0,
                         note="3-way 200x150x100, 10k distinct uniform coordinates, U(0,1) values, R=16"),
    # skewed 3-way SpMTTKRP, stand-in for nell2 (12K x 9K x 29K, 77M nnz)
    "skewed3": TensorConfig("skewed3", (12_000, 9_000, 28_000), 76_000_000, (("zipf", 1.1),) * 3, "uniform",
                            R=32, seed=0,
                            note="3-way 12000x9000x28000, 76M nnz, Zipf(1.1) per mode, U(0,1), R=32"),
    # 4-way SpTTM along the last mode
    "ttm4": TensorConfig("ttm4", (5_000, 4_000, 3_000, 50_000), 100_000_000,
                         (("zipf", 1.0), ("zipf", 1.0), ("zipf", 1.0), "uniform"), "lognormal", R=16, seed=0,
                         note="4-way 5000x4000x3000x50000, 100M nnz, Zipf(1.0) x3 + uniform, lognormal"),
    # CP-ALS on the skewed 3-way tensor at R=64
    "cp64": TensorConfig("cp64", (12_000, 9_000, 28_000), 76_000_000, (("zipf", 1.1),) * 3, "uniform",
                         R=64, seed=0, note="skewed3 tensor, CP-ALS R=64, 20 sweeps"),
    # differentiable sparse CP fit: observed entries of a rank-32 Kruskal tensor plus noise
    "fit3": TensorConfig("fit3", (50_000, 40_000, 30_000), 20_000_000, (("zipf", 1.1),) * 3, "kruskal", R=32,
                         seed=0, kruskal_rank=32, noise_std=0.01,
                         note="3-way 50000x40000x30000, 20M Zipf(1.1) coords, rank-32 Kruskal + N(0,0.01^2)"),
    # finite-difference copy of the fit workload
    "fit3_fd": TensorConfig("fit3_fd", (30, 20, 10), 500, ("uniform",) * 3, "kruskal", R=4, seed=0,
                            kruskal_rank=4, noise_std=0.01, note="30x20x10, 500 nnz, FD check copy"),
}


def scaled(cfg: TensorConfig, nnz: int, dims: Optional[Sequence[int]] = None, **kw) -> TensorConfig:
    """Same recipe with fewer nonzeros (and optionally smaller dims)."""
    d = tuple(dims) if dims is not None else cfg.dims
    if int(nnz) == cfg.nnz and d == cfg.dims:
        note = cfg.note
    else:
        note = f"{cfg.note}; scaled to {'x'.join(str(x) for x in d)}, {int(nnz)} nnz"
    return replace(cfg, nnz=int(nnz), dims=d, name=f"{cfg.name}@{nnz}", note=note, **kw)


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def _zipf_cdf(dim: int, s: float, device) -> torch.Tensor:
    k = torch.arange(1, dim + 1, dtype=torch.float64, device=device)
    w = k.pow(-float(s))
    c = torch.cumsum(w, 0)
    return c / c[-1]


def _draw_mode(gen, n: int, dim: int, dist: Dist, cdf, perm, device) -> torch.Tensor:
    if dist == "uniform":
        return torch.randint(0, dim, (n,), generator=gen, device=device, dtype=torch.int64)
    u = torch.rand(n, generator=gen, device=device, dtype=torch.float64)
    r = torch.searchsorted(cdf, u, right=True).clamp_(max=dim - 1)
    return perm[r]


def _draw_values(gen, n: int, kind: str, device) -> torch.Tensor:
    if kind == "lognormal":
        return torch.exp(torch.randn(n, generator=gen, device=device, dtype=torch.float64))
    return torch.rand(n, generator=gen, device=device, dtype=torch.float64)


@dataclass
class SparseTensor:
    dims: Tuple[int, ...]
    idx: list  # per-mode int64 tensors (values < 2**32)
    val: torch.Tensor  # float32
    cfg: Optional[TensorConfig] = None
    truth: Optional[list] = field(default=None, repr=False)  # ground-truth factors (kruskal)

    @property
    def nnz(self) -> int:
        return int(self.val.shape[0])

    @property
    def nmodes(self) -> int:
        return len(self.dims)

    def idx_u32(self):
        """Per-mode index arrays as numpy uint32 (host)."""
        return [a.to("cpu").numpy().astype("uint32") for a in self.idx]

    def to(self, device):
        return SparseTensor(self.dims, [a.to(device) for a in self.idx], self.val.to(device), self.cfg,
                            None if self.truth is None else [t.to(device) for t in self.truth])


def distinct_coords(dims, nnz: int, dists, gen, device, values: str = "uniform"):
    """Draw coordinates in rounds until >= nnz distinct ones exist (values of repeats
    summed), then keep a seeded random subset of exactly nnz.  Returns (idx list, val f64)."""
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    total = 1
    for d in dims:
        total *= d
    if nnz > total:
        raise ValueError(f"nnz={nnz} exceeds the number of cells {total}")
    if total >= 2 ** 62:
        raise ValueError("dims too large for 64-bit linear keys")
    strides = [1] * N
    for k in range(N - 2, -1, -1):
        strides[k] = strides[k + 1] * dims[k + 1]
    cdfs, perms = [], []
    for k in range(N):
        if dists[k] == "uniform":
            cdfs.append(None)
            perms.append(None)
        else:
            cdfs.append(_zipf_cdf(dims[k], dists[k][1], device))
            perms.append(torch.randperm(dims[k], generator=gen, device=device))
    keys = torch.empty(0, dtype=torch.int64, device=device)
    vals = torch.empty(0, dtype=torch.float64, device=device)
    factor = 1.25
    while keys.numel() < nnz:
        need = nnz - keys.numel()
        m = int(need * factor) + 1024
        key = torch.zeros(m, dtype=torch.int64, device=device)
        for k in range(N):
            key += _draw_mode(gen, m, dims[k], dists[k], cdfs[k], perms[k], device) * strides[k]
        v = _draw_values(gen, m, values, device)
        before = keys.numel()
        allk = torch.cat([keys, key])
        allv = torch.cat([vals, v])
        del key, v
        keys, inv = torch.unique(allk, sorted=True, return_inverse=True)
        vals = torch.zeros(keys.numel(), dtype=torch.float64, device=device).scatter_add_(0, inv, allv)
        del allk, allv, inv
        gained = keys.numel() - before
        if gained < 0.5 * m:
            factor *= 2.0
    keep = torch.randperm(keys.numel(), generator=gen, device=device)[:nnz]
    keys = keys[keep]
    vals = vals[keep]
    idx = []
    for k in range(N):
        idx.append(torch.div(keys, strides[k], rounding_mode="floor") % dims[k])
    return idx, vals


def make_tensor(cfg: TensorConfig, device="cpu") -> SparseTensor:
    """Build the sparse tensor of a config (exactly cfg.nnz distinct nonzeros)."""
    gen = _gen(cfg.seed, device)
    vkind = "uniform" if cfg.values == "kruskal" else cfg.values
    idx, vals = distinct_coords(cfg.dims, cfg.nnz, cfg.dists, gen, device, vkind)
    truth = None
    if cfg.values == "kruskal":
        R = cfg.kruskal_rank
        scale = R ** (-1.0 / 6.0)
        truth = [torch.randn(d, R, generator=gen, device=device, dtype=torch.float64) * scale for d in cfg.dims]
        vals = _kruskal_values(idx, truth)
        vals = vals + cfg.noise_std * torch.randn(vals.shape[0], generator=gen, device=device, dtype=torch.float64)
        truth = [t.float() for t in truth]
    return SparseTensor(tuple(cfg.dims), idx, vals.float(), cfg, truth)


def _kruskal_values(idx, truth, chunk: int = 1 << 22):
    """Data definition of the sparse-fit workload: the entries of the ground-truth
    Kruskal tensor [[A, B, C]] at the drawn coordinates (float64)."""
    n = idx[0].shape[0]
    out = torch.empty(n, dtype=torch.float64, device=idx[0].device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        prod = None
        for k, F in enumerate(truth):
            rows = F[idx[k][s:e]]
            prod = rows if prod is None else prod * rows
        out[s:e] = prod.sum(1)
    return out


def make_factors(dims, R: int, seed: int = 1, device="cpu", kind: str = "normal", dtype=torch.float32):
    """Dense factor matrices I_k x R (row-major, contiguous)."""
    gen = _gen(seed, device)
    out = []
    for d in dims:
        if kind == "uniform":
            f = torch.rand(int(d), R, generator=gen, device=device, dtype=torch.float64)
        else:
            f = torch.randn(int(d), R, generator=gen, device=device, dtype=torch.float64)
        out.append(f.to(dtype).contiguous())
    return out


def coo_from_lists(dims, coords, vals, device="cpu") -> SparseTensor:
    """Hand-made small tensor from a list of coordinate tuples."""
    N = len(dims)
    idx = [torch.tensor([c[k] for c in coords], dtype=torch.int64, device=device) for k in range(N)]
    return SparseTensor(tuple(dims), idx, torch.tensor(vals, dtype=torch.float32, device=device))


def random_small(dims, nnz: int, seed: int, dists=None, values="uniform", device="cpu") -> SparseTensor:
    """Small random tensor with exactly nnz distinct coordinates."""
    dists = dists or ("uniform",) * len(dims)
    gen = _gen(seed, device)
    idx, vals = distinct_coords(dims, nnz, dists, gen, device, values)
    return SparseTensor(tuple(dims), idx, vals.float())


def zipf_mass(dim: int, s: float, top: int) -> float:
    """Probability mass of the `top` most frequent ranks of a bounded Zipf."""
    w = [k ** (-s) for k in range(1, dim + 1)]
    return sum(w[:top]) / sum(w)


__all__ = ["TensorConfig", "CONFIGS", "scaled", "make_tensor", "make_factors", "SparseTensor", "distinct_coords",
           "coo_from_lists", "random_small", "zipf_mass"]
