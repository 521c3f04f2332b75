"""bpp_dslash_noalloc: the even/odd hopping term for callers that cannot let a
library allocate device memory (an application whose memory manager owns the
GPU, or code that must not risk an allocation failing or stalling midway).
Through the C ABI, two calls in a row with different inputs must match the
allocating bpp_dslash within the parity tolerances used elsewhere (FP64 1e-13,
FP32 1e-6, FP16-storage 5e-3), for every right-hand side of a multi-RHS call;
the device's free memory must not change from just before the first call on
a new gauge field to after the second; a bad output tensor and a request
beyond the fixed scratch size must be refused with an error.  This file is
collected last so a failure here cannot hide others."""
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


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_first_call_allocates_nothing(prec):
    """Free device memory is recorded after the gauge field is created and
    before the first bpp_dslash_noalloc call on it: the scratch array must
    already be in place (the gauge creation placed it), so the first call and
    the second leave free memory unchanged.  The allocating bpp_dslash runs
    first only to load the kernels both entry points share."""
    bpp = lib()
    L = (8, 8, 8, 8)
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    dt = torch.complex128 if prec == 0 else torch.complex64
    psi_np = synth.gaussian_spinor(L, seed=13, nrhs=3)[:, :Vh]
    psi = to_dev(psi_np, dt)
    ref = bpp.dslash(g, psi, KAPPA, 1, prec)
    out = torch.empty_like(psi)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        bpp.dslash_noalloc(g, psi, KAPPA, 1, prec, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for r in range(3):
        assert rel_err(to_np(out[r]), to_np(ref[r])) <= TOL[prec]
    if prec == 0:
        assert rel_err(to_np(out[1]), oracle.hop_eo(U, psi_np[1], KAPPA, L, 1)) <= 1e-13


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_multi_rhs_every_rhs(prec):
    """Three right-hand sides per call in every storage format: each one at its
    own offset of the shared array (FP16 with its per-site scales) must match
    the allocating bpp_dslash, on two calls in a row with different inputs."""
    bpp = lib()
    L = (4, 6, 6, 8)
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    dt = torch.complex128 if prec == 0 else torch.complex64
    out = torch.empty((3, Vh, 4, 3), dtype=dt, device="cuda")
    for seed in (21, 22):
        psi = to_dev(synth.gaussian_spinor(L, seed=seed, nrhs=3)[:, :Vh], dt)
        for parity in (0, 1):
            ref = bpp.dslash(g, psi, KAPPA, parity, prec)
            bpp.dslash_noalloc(g, psi, KAPPA, parity, prec, out=out)
            torch.cuda.synchronize()
            for r in range(3):
                assert rel_err(to_np(out[r]), to_np(ref[r])) <= TOL[prec], (seed, parity, r)


def test_noalloc_checks_out():
    """A caller-supplied out of the wrong dtype, size, device or layout, or one
    overlapping psi, is refused before the library writes through it."""
    bpp = lib()
    L = (4, 4, 4, 4)
    g, U = gauge(L)
    Vh = oracle.volume(L) // 2
    psi = torch.zeros((Vh, 4, 3), dtype=torch.complex128, device="cuda")
    bad = [torch.empty((Vh, 4, 3), dtype=torch.complex64, device="cuda"),
           torch.empty((Vh // 2, 4, 3), dtype=torch.complex128, device="cuda"),
           torch.empty((Vh, 4, 3), dtype=torch.complex128),
           torch.empty((3, 4, Vh), dtype=torch.complex128, device="cuda").permute(2, 1, 0),
           psi]
    for out in bad:
        with pytest.raises(ValueError):
            bpp.dslash_noalloc(g, psi, KAPPA, 0, bpp.F64, out=out)


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
