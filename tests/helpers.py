"""Shared helpers for the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np

import oracle as orc


def pair(M, w, L, n_min, n_max, p_list=None):
    """The CUDA space and the oracle space over the same sector list."""
    import paper_2111_00050_gb300 as qb

    qs = qb.Space(M, w, L, n_min, n_max, p_list)
    os_ = orc.Space(M, qs.sectors)
    assert os_.total == qs.total
    return qs, os_


def to_dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def to_host(t):
    return t.detach().cpu().numpy()


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def random_state(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return x / np.linalg.norm(x)
