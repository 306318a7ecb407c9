"""afqmc_local_energy_static: the local-energy entry point for callers that
cannot allocate device memory (for example while a framework's caching
allocator owns the device, or under a fixed memory budget).  It must give the
same energies as afqmc_local_energy, call after call, from its fixed device
array, and refuse requests larger than that array.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2403_02542_gb300.inputs import make_fields, make_system

pytestmark = pytest.mark.gpu
RTOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    from paper_2403_02542_gb300 import _lib, build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _lib


def _static_energy(L, ctx, w, e0, tau):
    e_loc = torch.full((w.n, 2), float("nan"), dtype=torch.float64, device=ctx.device)
    e_mix = torch.full((4,), float("nan"), dtype=torch.float64, device=ctx.device)
    ctx._bind_stream()
    cw = w.c_struct()
    st = L.lib().afqmc_local_energy_static(ctx._h, ctypes.byref(cw), float(e0), float(tau),
                                           e_loc.data_ptr(), e_mix.data_ptr())
    return st, e_loc, e_mix


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_scratch_energy_matches_allocating_entry_point(lib, precision):
    from paper_2403_02542_gb300.api import Context
    s = make_system(24, 3, 3, 40, rho=0.8, seed=77)
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision=precision)
    nw, tau, e0 = 16, 0.05, -10.0
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    for k in range(2):  # move the walkers away from the trial
        x = torch.as_tensor(make_fields(31, k, nw, s.G), device=ctx.device)
        ctx.step(w, x, tau, e0, expm="taylor", order=6)
    ref_loc, ref_mix = ctx.local_energy(w, e0, tau)
    torch.cuda.synchronize()
    for _ in range(2):  # two calls in a row share the array
        st, e_loc, e_mix = _static_energy(lib, ctx, w, e0, tau)
        assert st == lib.AFQMC_OK
        torch.cuda.synchronize()
        assert torch.isfinite(e_loc).all() and torch.isfinite(e_mix).all()
        err = float(((e_loc - ref_loc).norm(dim=1) / ref_loc.norm(dim=1)).max())
        assert err <= RTOL, err
        assert torch.allclose(e_mix, ref_mix, rtol=RTOL, atol=0.0)
    ctx.close()


def test_static_scratch_rejects_requests_beyond_its_size(lib):
    from paper_2403_02542_gb300.api import Context
    s = make_system(24, 3, 3, 40, rho=0.8, seed=77)
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="fp64")
    per_walker = 6 * 24 * 16 + 32 + 128 + 40 * 64 + 8
    nw = lib.STATIC_SCRATCH_BYTES // per_walker + 64
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    st, e_loc, e_mix = _static_energy(lib, ctx, w, -10.0, 0.05)
    assert st == lib.AFQMC_EINVAL
    torch.cuda.synchronize()
    assert torch.isnan(e_mix).all()   # nothing was launched
    ctx.close()
