"""Population control (comb, reading R8) on the GPU vs the oracle's comb:
selected indices are integers and must match exactly; the copies and the new
weights are exact (no arithmetic beyond the same FP64 cumulative sum)."""
import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import make_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx_fp64():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_02542_gb300.api import Context
    s = make_system(12, 2, 2, 10, rho=0.7, seed=5)
    return Context(s.h1, s.L, s.trial, 2, 2, precision="fp64")


def _population(ctx, nw, seed, zero=()):
    g = np.random.default_rng(seed)
    psi = g.standard_normal((nw, ctx.nc, ctx.N)) + 1j * g.standard_normal((nw, ctx.nc, ctx.N))
    W = g.uniform(0.0, 3.0, nw)
    for z in zero:
        W[z] = 0.0
    lo = g.standard_normal((nw, 2))
    w = ctx.new_walkers(nw)
    w.psi.copy_(torch.as_tensor(psi).to(ctx.ctype))
    w.weight.copy_(torch.as_tensor(W))
    w.logovl.copy_(torch.as_tensor(lo))
    w.status.copy_(torch.arange(nw, dtype=torch.int32))
    return w, psi, W, lo


@pytest.mark.parametrize("nw,u", [(37, 0.37), (1024, 0.0), (1, 0.9), (3000, 0.5)])
def test_comb_matches_oracle(ctx_fp64, nw, u):
    ctx = ctx_fp64
    zero = (0, nw // 2, nw - 1) if nw > 3 else ()
    w, psi, W, lo = _population(ctx, nw, seed=nw, zero=zero)
    idx_dev = torch.empty(nw, dtype=torch.int32, device=ctx.device)
    ctx.population_control(w, u, idx_dev)
    torch.cuda.synchronize()
    ref = R.comb(torch.as_tensor(W), u).numpy()
    got = idx_dev.cpu().numpy()
    assert np.array_equal(got, ref)
    for z in zero:
        assert z not in set(got.tolist())
    total = 0.0
    for x in W:
        total = total + float(x)
    assert torch.all(w.weight.cpu() == total / nw)
    assert np.array_equal(w.psi.cpu().numpy(), psi[ref].astype(np.complex128))
    assert np.array_equal(w.logovl.cpu().numpy(), lo[ref])
    assert np.array_equal(w.status.cpu().numpy(), ref.astype(np.int32))


def test_comb_with_no_weight_leaves_population(ctx_fp64):
    ctx = ctx_fp64
    w, psi, W, lo = _population(ctx, 8, seed=1, zero=range(8))
    idx_dev = torch.zeros(8, dtype=torch.int32, device=ctx.device)
    ctx.population_control(w, 0.5, idx_dev)
    torch.cuda.synchronize()
    assert torch.all(idx_dev.cpu() == -1)
    assert np.array_equal(w.psi.cpu().numpy(), psi)
    assert torch.all(w.weight.cpu() == 0.0)


def test_comb_rejects_bad_u(ctx_fp64):
    from paper_2403_02542_gb300 import _lib as L
    w, *_ = _population(ctx_fp64, 4, seed=2)
    for u in (1.0, -0.1):
        with pytest.raises(L.AfqmcError):
            ctx_fp64.population_control(w, u)
