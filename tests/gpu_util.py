"""Helpers shared by the GPU tests: device copies in column-major layout."""
import numpy as np
import torch


def dev_colmajor(A: np.ndarray) -> torch.Tensor:
    """A numpy matrix as a column-major CUDA tensor (strides (1, n))."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A).T)).cuda().t()


def dev_vec(v: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()
