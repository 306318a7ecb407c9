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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_scratch_on_a_fresh_context_allocates_nothing(lib, precision):
    """The case the entry point is for: a context whose workspace was never
    sized, asked for more walkers than any earlier call on it.  Free device
    memory is the same before and after the call, and the energies equal
    those of afqmc_local_energy called afterwards (which does allocate)."""
    from paper_2403_02542_gb300.api import Context
    s = make_system(24, 3, 3, 40, rho=0.8, seed=78)
    e0, tau = -10.0, 0.05
    # load every module the call uses (kernels and the scratch array) on a
    # throw-away context first, so that lazy module loading is not counted
    warm = Context(s.h1, s.L, s.trial, s.na, s.nb, precision=precision)
    ww = warm.new_walkers(2)
    warm.init_walkers(ww)
    warm.local_energy(ww, e0, tau)
    assert _static_energy(lib, warm, ww, e0, tau)[0] == lib.AFQMC_OK
    torch.cuda.synchronize()
    warm.close()
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision=precision)
    nw = 96
    w = ctx.new_walkers(nw)
    g = torch.Generator(device=ctx.device).manual_seed(3)
    psi = torch.as_tensor(s.trial.T, device=ctx.device).to(ctx.ctype).unsqueeze(0).repeat(nw, 1, 1)
    noise = torch.randn(nw, s.na + s.nb, s.h1.shape[0], 2, dtype=torch.float64, device=ctx.device, generator=g)
    w.psi.copy_(psi + 0.2 * torch.view_as_complex(noise).to(ctx.ctype))
    w.weight.copy_(torch.rand(nw, dtype=torch.float64, device=ctx.device, generator=g) + 0.5)
    w.logovl.zero_()
    w.status.zero_()
    e_loc = torch.full((nw, 2), float("nan"), dtype=torch.float64, device=ctx.device)
    e_mix = torch.full((4,), float("nan"), dtype=torch.float64, device=ctx.device)
    cw = w.c_struct()
    ctx._bind_stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(ctx.device)
    st = lib.lib().afqmc_local_energy_static(ctx._h, ctypes.byref(cw), e0, tau, e_loc.data_ptr(),
                                             e_mix.data_ptr())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(ctx.device)
    assert st == lib.AFQMC_OK
    assert free1 == free0, (free0, free1)
    ref_loc, ref_mix = ctx.local_energy(w, e0, tau)
    torch.cuda.synchronize()
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


def _header_scratch_bytes(nw, N, na, nb, G, mixed):
    """The scratch size of afqmc_local_energy_static as the header states it:
    each term rounded up to a multiple of 256 bytes, the two split Theta planes
    for mixed contexts with 1 <= na == nb <= 64 (tensor-core exchange)."""
    def up(x):
        return (x + 255) // 256 * 256
    nc = na + nb
    total = up(nw * nc * N * (8 if mixed else 16)) + up(nw * 32) + up(nw * 128) + up(nw * G * 64) + up(nw * 8)
    if mixed and 1 <= na == nb <= 64:
        Kp = (N + 63) // 64 * 64
        total += 2 * up(8 * nw * na * Kp)
    return total


def test_static_scratch_limit_follows_the_header_formula_above_128_orbitals(lib):
    """A mixed context with N = 160 (tensor-core exchange with the streamed
    Theta operand): the largest walker count whose scratch, by the header's
    formula, fits in AFQMC_STATIC_SCRATCH_BYTES is accepted, one more is
    refused with nothing launched."""
    from paper_2403_02542_gb300.api import Context
    N, n, G = 160, 8, 20
    s = make_system(N, n, n, G, rho=0.9, seed=160)
    ctx = Context(s.h1, s.L, s.trial, n, n, precision="mixed")
    nw = 1
    while _header_scratch_bytes(nw + 1, N, n, n, G, True) <= lib.STATIC_SCRATCH_BYTES:
        nw += 1
    assert _header_scratch_bytes(nw, N, n, n, G, True) <= lib.STATIC_SCRATCH_BYTES
    w = ctx.new_walkers(nw + 1)
    ctx.init_walkers(w)
    big = type(w)(w.psi, w.weight, w.logovl, w.status)
    small = type(w)(w.psi[:nw], w.weight[:nw], w.logovl[:nw], w.status[:nw])
    st, e_loc, e_mix = _static_energy(lib, ctx, big, -10.0, 0.05)
    assert st == lib.AFQMC_EINVAL
    torch.cuda.synchronize()
    assert torch.isnan(e_mix).all()
    st, e_loc, e_mix = _static_energy(lib, ctx, small, -10.0, 0.05)
    assert st == lib.AFQMC_OK
    torch.cuda.synchronize()
    assert torch.isfinite(e_loc).all() and torch.isfinite(e_mix).all()
    ctx.close()
