"""Shared helpers of the GPU parity tests: the library context, tensor
conversion, and the basis-invariant error measures used against the oracle."""

from __future__ import annotations

import numpy as np
import pytest
import torch


def cuda_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_CTX = None


def context():
    global _CTX
    cuda_or_skip()
    if _CTX is None:
        from paper_2504_03373_gb300 import binding
        from paper_2504_03373_gb300.build import build
        build()
        _CTX = binding.Context(0)
    return _CTX


def dev(a: np.ndarray) -> torch.Tensor:
    """complex numpy -> contiguous complex64 CUDA tensor."""
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


def max_rel(x, ref) -> float:
    """max |x - ref| / max |ref| (max-normalised relative error)."""
    x = np.asarray(x, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    return float(np.abs(x - ref).max() / np.abs(ref).max())


def projector(E: np.ndarray, Ns: int) -> np.ndarray:
    En = np.asarray(E, dtype=np.complex128)[..., :, Ns:]
    return np.matmul(En, np.conj(np.swapaxes(En, -1, -2)))


def signal_gap(lam: np.ndarray, Ns: int) -> np.ndarray:
    """Relative gap between the last signal and the first noise singular value."""
    return (lam[..., Ns - 1] - lam[..., Ns]) / lam[..., 0]
