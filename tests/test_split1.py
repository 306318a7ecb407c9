"""Split-1 propagator (Sec. III: the interaction exponential first, then the
whole one-body step e^{-tau h''} as two half steps) of the CUDA library
against the CPU oracle on the same seeded systems and common random fields:
FP64 element by element (1e-10 relative, as the other FP64 parity tests) with
each action of the exponential, and complex64 walkers within the mixed energy
bar (1e-4 Ha per walker)."""
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


@pytest.mark.parametrize("expm,order,reo", [("krylov", 8, 2), ("taylor", 6, 0), ("bkrylov", 3, 0)])
def test_split1_fp64_matches_oracle(expm, order, reo):
    from paper_2403_02542_gb300.api import Context
    s = make_system(40, 4, 4, 70, rho=0.85, seed=11)
    tau = 0.05
    e0 = _e0(s)
    ref, ties = oracle_walk(s, 6, 3, tau, e0, expm, order, reo, seed=17, propagator="split1")
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    got, _ = gpu_walk(ctx, 6, 3, tau, e0, expm, order, reo, seed=17, propagator="split1")
    for g, r in zip(got, ref):
        compare(g, r, RTOL, what=f"Split-1 {expm} step {g['k']}")
    # the two propagators differ at this time step
    two, _ = gpu_walk(ctx, 6, 1, tau, e0, expm, order, 0, seed=17)
    assert float((two[0]["psi"] - got[0]["psi"]).abs().max()) > 1e-6
    ctx.close()


def test_split1_mixed_large_workload_energy():
    """Complex64 walkers on the large workload (N=128, 20+20, 640 vectors):
    E_L after two Split-1 steps within 1e-4 Ha of the oracle."""
    from paper_2403_02542_gb300.api import Context
    s = config_system("large")
    tau = 0.05
    e0 = _e0(s)
    nw = 4
    ref, ties = oracle_walk(s, nw, 2, tau, e0, "krylov", 10, 0, seed=23, propagator="split1")
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="mixed")
    got, _ = gpu_walk(ctx, nw, 2, tau, e0, "krylov", 10, 0, seed=23, propagator="split1")
    dE = max(float((g["El"] - r["El"]).abs().max()) for g, r in zip(got, ref))
    print(f"Split-1 mixed vs oracle: max|dE_L| = {dE:.2e} Ha")
    assert dE <= E_TOL
    ctx.close()
