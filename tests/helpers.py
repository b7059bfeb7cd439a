"""Shared test helpers: tolerances, oracle comparisons, seeded inputs."""
import numpy as np
import torch

# tolerance for FP32 paths: relative Frobenius error vs the FP64 oracle
REL_FRO = 1e-5
# element-wise: error relative to the sum of absolute terms of that element
REL_ABS = 2e-5


def rel_fro(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def assert_close_abs(got, ref, absref, rel_abs=REL_ABS, rel_fro_tol=REL_FRO):
    """got vs ref: relative Frobenius error <= rel_fro_tol and every element within
    rel_abs * (sum of absolute values of the terms that element adds up)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.all(np.isfinite(got))
    e = rel_fro(got, ref)
    assert e <= rel_fro_tol, f"relative Frobenius error {e:.3e} > {rel_fro_tol}"
    bad = np.abs(got - ref) > rel_abs * np.asarray(absref) + 1e-30
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{bad.sum()} elements off; first {tuple(i)}: got {got[tuple(i)]} ref {ref[tuple(i)]} "
                             f"abs-sum {np.asarray(absref)[tuple(i)]}")


def host_factors(factors):
    """Factor tensors (float32 or bfloat16, any device) -> float64 numpy of the exact stored values."""
    return [f.detach().float().cpu().double().numpy() for f in factors]


def cuda():
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    return torch.device("cuda:0")
