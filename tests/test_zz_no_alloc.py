"""bpp_dslash_noalloc: the even/odd hopping term for callers that cannot let a
library allocate device memory (an application whose memory manager owns the
GPU, or code that must not risk an allocation failing or stalling midway).
Through the C ABI, two calls in a row with different inputs must match the
allocating bpp_dslash within the parity tolerances used elsewhere (FP64 1e-13,
FP32 1e-6, FP16-storage 5e-3), the device's free memory must not change
across them, and a request beyond the fixed scratch size must be refused with
an error.  This file is collected last so a failure here cannot hide others."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import KAPPA, gauge, lib, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 1e-6, 2: 5e-3}


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_matches_dslash_twice(prec):
    bpp = lib()
    L = (6, 6, 6, 10)
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    dt = torch.complex128 if prec == 0 else torch.complex64
    psis = [to_dev(synth.gaussian_spinor(L, seed=s)[:Vh], dt) for s in (11, 12)]
    out = torch.empty_like(psis[0])
    bpp.dslash_noalloc(g, psis[0], KAPPA, 0, prec, out=out)     # first call on the device: address lookup
    torch.cuda.synchronize()
    for parity in (0, 1):
        for psi in psis:
            ref = bpp.dslash(g, psi, KAPPA, parity, prec)
            rc = bpp._lib.bpp_dslash_noalloc(g.handle, bpp._ptr(psi), bpp._ptr(out), KAPPA, parity, prec, 1,
                                             bpp._stream())
            assert rc == 0
            torch.cuda.synchronize()
            assert rel_err(to_np(out), to_np(ref)) <= TOL[prec]
    torch.cuda.synchronize()
    bpp.release_workspace()


def test_noalloc_no_device_allocation():
    bpp = lib()
    L = (8, 8, 8, 8)
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psi = to_dev(synth.gaussian_spinor(L, seed=13, nrhs=3)[:, :Vh])
    out = torch.empty_like(psi)
    bpp.dslash_noalloc(g, psi, KAPPA, 1, bpp.F64, out=out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        bpp.dslash_noalloc(g, psi, KAPPA, 1, bpp.F64, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref = oracle.hop_eo(U, synth.gaussian_spinor(L, seed=13, nrhs=3)[1, :Vh], KAPPA, L, 1)
    assert rel_err(to_np(out[1]), ref) <= 1e-13


def test_noalloc_rejects_oversize():
    bpp = lib()
    L = (16, 16, 16, 32)       # FP64 half fields: 2 x 65536 x 192 B x 2 RHS > 32 MiB
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psi = torch.zeros((2, Vh, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(bpp.BppError) as e:
        bpp.dslash_noalloc(g, psi, KAPPA, 0, bpp.F64)
    assert e.value.code == -1 and "static maximum" in str(e.value)
    # one RHS fits
    out = bpp.dslash_noalloc(g, psi[0], KAPPA, 0, bpp.F64)
    assert torch.count_nonzero(out) == 0
