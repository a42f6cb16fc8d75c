"""Shared helpers of the GPU parity tests (no arithmetic of the method here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype).contiguous()


def real_dtype(prec):
    from paper_2507_22128_gb300 import rix
    return torch.float64 if prec == rix.FP64 else torch.float32


def cplx_dtype(prec):
    from paper_2507_22128_gb300 import rix
    return torch.complex128 if prec == rix.FP64 else torch.complex64


def sparse_model(n, k, seed, lo=0.15, hi=0.85):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, n))
    idx = rng.integers(int(lo * n), int(hi * n), (k, 2))
    x[idx[:, 0], idx[:, 1]] = rng.uniform(0.05, 1.0, k)
    return x
