"""FP64 CUDA path vs the CPU oracle, element by element on the same seeded
Hamiltonians and common random fields.  Bar: 1e-10 relative per walker for
walkers, weights, log-overlaps and local energies (FP64 differs only in
summation order)."""
import math

import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import config_system, make_fields, make_system
from walk_helpers import compare, gpu_walk, oracle_walk

pytestmark = pytest.mark.gpu
RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ctx(sys_, precision="fp64", trial=None, na=None, nb=None):
    from paper_2403_02542_gb300.api import Context
    return Context(sys_.h1, sys_.L, sys_.trial if trial is None else trial,
                   sys_.na if na is None else na, sys_.nb if nb is None else nb,
                   sys_.e_const, precision=precision)


def test_small_workload_200_step_trajectory():
    """N=8, 2+2 electrons, 32 vectors (0.5^g), 64 walkers, tau=0.01, Split-2
    Taylor-6, QR every 5 steps: the whole 200-step trajectory."""
    s = config_system("small")
    tau, e0, steps = 0.01, -7.1, 200
    ref, ties = oracle_walk(s, 64, steps, tau, e0, "taylor", 6, 5, seed=101)
    assert ties == 0
    ctx = _ctx(s)
    rec = set(range(0, steps, 10)) | {steps - 1}
    got, _ = gpu_walk(ctx, 64, steps, tau, e0, "taylor", 6, 5, seed=101, record=rec)
    for g in got:
        r = ref[g["k"]]
        compare(g, r, RTOL, what=f"step {g['k']}")
        assert abs(float(g["emix"][2]) - r["emix"]) <= RTOL * abs(r["emix"])
        assert abs(float(g["emix"][1]) - r["wsum"]) <= RTOL * r["wsum"]


def test_krylov_ragged_tiles_dead_walker_and_qr():
    """Sizes that span several GEMM tiles with ragged tails (N=72, G=150),
    Krylov k=6, a dead walker that must stay untouched, QR at step 3."""
    s = make_system(72, 5, 5, 150, rho=1e-5 ** (1 / 150), seed=4242)
    tau, e0 = 0.05, -20.0
    ref, ties = oracle_walk(s, 13, 4, tau, e0, "krylov", 6, 3, seed=7, dead=(3,))
    assert ties == 0
    ctx = _ctx(s)
    got, w = gpu_walk(ctx, 13, 4, tau, e0, "krylov", 6, 3, seed=7, dead=(3,))
    for g, r in zip(got, ref):
        compare(g, r, RTOL, what=f"step {g['k']}")
    # the dead walker is bit-identical to the trial and keeps W = 0
    trial = torch.as_tensor(s.trial, dtype=torch.complex128)
    assert torch.equal(got[-1]["psi"][3], trial)
    assert float(got[-1]["W"][3]) == 0.0


def test_taylor_unequal_spins_and_order_zero():
    s = make_system(20, 3, 3, 24, rho=0.8, seed=99)
    trial = np.concatenate([s.trial[:, :3], s.trial[:, :1]], axis=1)     # 3 alpha, 1 beta
    tau, e0 = 0.05, -5.0
    for order in (0, 5):
        ref, ties = oracle_walk(s, 5, 3, tau, e0, "taylor", order, 2, seed=3, trial=trial, na=3, nb=1)
        assert ties == 0
        ctx = _ctx(s, trial=trial, na=3, nb=1)
        got, _ = gpu_walk(ctx, 5, 3, tau, e0, "taylor", order, 2, seed=3)
        for g, r in zip(got, ref):
            compare(g, r, RTOL, what=f"order {order} step {g['k']}")


def test_empty_beta_spin():
    s = make_system(12, 2, 2, 10, rho=0.7, seed=5)
    trial = np.ascontiguousarray(s.trial[:, :2])
    ref, ties = oracle_walk(s, 4, 3, 0.05, -3.0, "krylov", 4, 0, seed=11, trial=trial, na=2, nb=0)
    ctx = _ctx(s, trial=trial, na=2, nb=0)
    got, _ = gpu_walk(ctx, 4, 3, 0.05, -3.0, "krylov", 4, 0, seed=11)
    for g, r in zip(got, ref):
        compare(g, r, RTOL, what=f"nb=0 step {g['k']}")


def test_krylov_dimension_beyond_N_is_exact():
    """k >= N: the Krylov space is the whole space (k clamped to N); the step
    then equals the one with the exact exponential."""
    s = make_system(6, 1, 1, 8, rho=0.7, seed=8)
    tau, e0 = 0.1, -3.0
    ref, _ = oracle_walk(s, 3, 2, tau, e0, "exact", 0, 0, seed=5)
    ctx = _ctx(s)
    got, _ = gpu_walk(ctx, 3, 2, tau, e0, "krylov", 9, 0, seed=5)
    for g, r in zip(got, ref):
        compare(g, r, 1e-9, what=f"step {g['k']}")


def test_single_walker_and_local_energy_entry_point():
    s = make_system(10, 2, 2, 12, rho=0.7, seed=12)
    ctx = _ctx(s)
    w = ctx.new_walkers(1)
    ctx.init_walkers(w)
    e_loc, e_mix = ctx.local_energy(w, -4.0, 0.05)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, 2, 2)
    ref = complex(R.local_energy(ham, ham.trial.to(torch.complex128)))
    got = complex(float(e_loc[0, 0]), float(e_loc[0, 1]))
    assert abs(got - ref) <= RTOL * abs(ref)
    assert abs(float(e_mix[1]) - 1.0) == 0.0 and float(e_mix[3]) == 1.0
    assert float(w.logovl.abs().max()) < 1e-13


def test_large_workload_sampled_walkers():
    """Full size of the large-step workload (N=128, 20+20 electrons, 640
    vectors, 1024 walkers, Krylov 10, tau=0.05) in the benchmark's launch
    configuration; two steps.  Walkers are independent, so the oracle follows
    a sample of them one by one with the same fields."""
    s = config_system("large")
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb)
    tau, k = 0.05, 10
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    nw = 1024
    ctx = _ctx(s)
    got, w = gpu_walk(ctx, nw, 2, tau, e0, "krylov", k, 0, seed=2024)
    sample = [0, 517, 1023]
    ref, ties = oracle_walk(s, len(sample), 2, tau, e0, "krylov", k, 0, seed=None,
                            field_fn=lambda step: make_fields(2024, step, nw, s.G)[sample])
    assert ties == 0
    for step in range(2):
        g = {key: got[step][key][sample] for key in ("psi", "lo", "W", "El")}
        compare(g, ref[step], RTOL, what=f"sampled step {step}")
