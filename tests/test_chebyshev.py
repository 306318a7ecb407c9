"""Chebyshev action of the one-body exponential (Sec. IV.B, reading R23) in
the CUDA library against the CPU oracle on the same seeded systems and common
random fields: FP64 element by element (1e-10 relative, as the other FP64
parity tests) with the Split-2 and Split-1 propagators, complex64 walkers
within the mixed energy bar (1e-4 Ha per walker), and the argument checks."""
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import config_system, make_system
from walk_helpers import compare, gpu_walk, oracle_walk

pytestmark = pytest.mark.gpu
RTOL = 1e-10
E_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _e0(s):
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb)
    return float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)


@pytest.mark.parametrize("N,n,G,nw,order,reo,prop", [
    (40, 4, 70, 6, 6, 2, "split2"),
    (40, 4, 70, 6, 10, 0, "split1"),
    (72, 5, 150, 5, 2, 0, "split2"),     # several tiles with ragged tails
    (40, 4, 70, 5, 1, 0, "split2"),      # order 1: c_0 + c_1 A only
    (18, 2, 24, 3, 0, 0, "split2"),      # order 0: c_0 Psi only
])
def test_chebyshev_fp64_matches_oracle(N, n, G, nw, order, reo, prop):
    from paper_2403_02542_gb300.api import Context
    s = make_system(N, n, n, G, rho=0.85 if G < 100 else 1e-5 ** (1 / G), seed=N + order)
    tau = 0.05
    e0 = _e0(s)
    ref, ties = oracle_walk(s, nw, 3, tau, e0, "chebyshev", order, reo, seed=41 + order, propagator=prop)
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    got, _ = gpu_walk(ctx, nw, 3, tau, e0, "chebyshev", order, reo, seed=41 + order, propagator=prop)
    for g, r in zip(got, ref):
        compare(g, r, RTOL, what=f"Chebyshev k={order} {prop} step {g['k']}")
    ctx.close()


def test_chebyshev_mixed_large_workload_energy():
    """Complex64 walkers on the large workload (N=128, 20+20, 640 vectors):
    E_L after two Split-2 steps with the order-8 Chebyshev action within
    1e-4 Ha of the oracle."""
    from paper_2403_02542_gb300.api import Context
    s = config_system("large")
    tau = 0.05
    e0 = _e0(s)
    nw = 4
    ref, ties = oracle_walk(s, nw, 2, tau, e0, "chebyshev", 8, 0, seed=43)
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="mixed")
    got, _ = gpu_walk(ctx, nw, 2, tau, e0, "chebyshev", 8, 0, seed=43)
    dE = max(float((g["El"] - r["El"]).abs().max()) for g, r in zip(got, ref))
    print(f"Chebyshev mixed vs oracle: max|dE_L| = {dE:.2e} Ha")
    assert dE <= E_TOL
    ctx.close()


def test_chebyshev_argument_checks():
    from paper_2403_02542_gb300 import _lib as Lb
    from paper_2403_02542_gb300.api import Context
    s = make_system(12, 2, 2, 10, rho=0.8, seed=1)
    ctx = Context(s.h1, s.L, s.trial, 2, 2, precision="fp64")
    w = ctx.new_walkers(2)
    ctx.init_walkers(w)
    x = torch.zeros(2, s.G, dtype=torch.float64, device=ctx.device)
    for order in (-1, 65):
        with pytest.raises(Lb.AfqmcError):
            ctx.step(w, x, 0.05, -1.0, expm="chebyshev", order=order)
    with pytest.raises(Lb.AfqmcError):
        ctx.step(w, x, 0.05, -1.0, expm="chebyshev", order=4, propagator="taylor")
    ctx.step(w, x, 0.05, -1.0, expm="chebyshev", order=64)
    ctx.sync()
    ctx.close()
