"""Helpers shared by the GPU parity tests: move seeded inputs to the device, round them the way
the device stores them, and measure relative errors against the FP64 oracle."""
import numpy as np
import torch

import paper_2207_14589_gb300 as sped

DEV = "cuda"
TOL = {torch.float64: 1e-12, torch.float32: 1e-5, torch.bfloat16: 1e-2}


def to_block(A, dtype, device=DEV):
    """Padded device block holding A (n x k)."""
    n, k = A.shape
    T = sped.alloc_block(n, k, dtype, device)
    T[:, :k] = torch.from_numpy(np.ascontiguousarray(A)).to(device=device, dtype=dtype)
    return T


def stored(A, dtype):
    """A as the device stores it (rounded to dtype), back in float64."""
    return torch.from_numpy(np.ascontiguousarray(A)).to(dtype).to(torch.float64).numpy()


def host(T, k):
    return T[:, :k].to(torch.float64).cpu().numpy()


def rel(got, want):
    d = np.linalg.norm(want)
    return float(np.linalg.norm(got - want) / (d if d > 0 else 1.0))
