"""Test helpers: building/loading the CUDA library and moving states between
numpy (the oracle's arrays) and torch device tensors (the library's buffers)."""
import functools

import numpy as np
import pytest


@functools.lru_cache(maxsize=1)
def built_library():
    from paper_1303_6615_gb300 import build
    return build.build()


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_library()
    return torch


def to_dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def to_host(t) -> np.ndarray:
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_l2(got: np.ndarray, ref: np.ndarray) -> float:
    """Relative L2 error over all entries (Parseval weights cancel in the ratio
    only approximately, so plain coefficient L2 is used)."""
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((got - ref).ravel()) / (den if den > 0 else 1.0))


def per_state_rel_l2(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    d = np.linalg.norm((got - ref).reshape(got.shape[0], -1), axis=1)
    n = np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)
    return d / np.where(n > 0, n, 1.0)
