"""Shared helpers of the GPU parity tests: fields from the seeded generators,
the library binding, and error measures."""
import numpy as np
import torch

import synth

KAPPA = 0.12
BC = (1, 1, 1, -1)


def lib():
    import paper_2111_04457_b300 as bpp
    return bpp


def dev():
    return torch.device("cuda", 0)


def to_dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev(), dtype=dtype)


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def gauge(L, U=None, seed=1):
    bpp = lib()
    if U is None:
        U = synth.random_links(L, seed=seed)
    return bpp.Gauge(to_dev(U), L, BC), U


def rel_err(a, b):
    """Norm-relative error ||a - b|| / ||b||."""
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def max_err(a, b):
    """Element-wise error max |a - b| / max |b|."""
    return float(np.abs(a - b).max() / np.abs(b).max())


def round32(a):
    return a.astype(np.complex64).astype(np.complex128)


def eo_split(L, full):
    import oracle
    return full[oracle.parity_sites(L, 0)], full[oracle.parity_sites(L, 1)]
