"""Helpers for GPU parity tests: move seeded host inputs to the device and
bring packed results back as uint32 numpy arrays."""
import numpy as np
import torch


def dev():
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    return torch.device("cuda", torch.cuda.current_device())


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64)).to(dev())


def bits_np(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def u64_np(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def bit_at(bits: np.ndarray, k) -> np.ndarray:
    k = np.asarray(k, dtype=np.int64)
    return (bits[k // 32] >> (k % 32).astype(np.uint32)) & 1
