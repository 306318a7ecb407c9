"""The multi-rank paths on CPU with two gloo ranks (127.0.0.1).  The benchmark
reduces its timings to the slowest rank, reports the whole-job rate from it
and draws different fields per rank: the step shards by walkers and has no
collective on its data path.  An energy run sharded over ranks exchanges one
pair of numbers per step (the global mixed estimate) and combs each rank's
walkers locally; driven here through the oracle-backed context, it must give
the per-step global weights, estimates and E_0 of the same protocol run in
lockstep in one process."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    walkers, steps = 1024, 3
    t = bench.slowest_rank(1.5 + rank, world, torch.device("cpu"))   # rank 1 is slower
    rate = bench.job_rate(walkers * steps, world, t)
    seed = bench.shard_seed(1234, rank)
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(4, generator=g)
    dist.barrier()
    q.put((rank, t, rate, seed, x.tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_slowest_time_job_rate_and_distinct_fields():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, rate0, s0, x0), (r1, t1, rate1, s1, x1) = out
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 2.5                       # both ranks see the slowest time
    assert rate0 == rate1 == pytest.approx(world * 1024 * 3 / 2.5)
    assert s0 != s1 and x0 != x1                 # each rank its own fields


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank(0.75, 1, torch.device("cpu")) == 0.75
    assert bench.job_rate(1024 * 20, 1, 0.5) == 1024 * 20 / 0.5
    assert bench.shard_seed(1234, 0) == 1234


NW, N_STEPS, N_EQ, ORDER, REO, POP, SEED, TAU = 6, 12, 4, 6, 3, 4, 5, 0.05


def _energy_rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import afqmc_ref as R
    from oracle_context import OracleContext
    from paper_2403_02542_gb300 import energy as S
    from paper_2403_02542_gb300.inputs import make_fields, make_system
    s = make_system(10, 2, 2, 16, rho=0.8, seed=12)
    octx = OracleContext(s)
    e0 = float(R.local_energy(octx.ham, octx.ham.trial.to(torch.complex128)).real)
    w = octx.new_walkers(NW)
    octx.init_walkers(w)
    out = S.energy_run(octx, w, TAU, e0, N_STEPS, fields=lambda k: torch.as_tensor(make_fields(77 + rank, k, NW, s.G)),
                       n_eq=N_EQ, expm="krylov", order=ORDER, reortho_every=REO, pop_every=POP, seed=SEED,
                       update_e0=True, group=dist.group.WORLD)
    q.put((rank, out["W"], out["E"], out["e0"], out["W_local"]))
    dist.barrier()
    dist.destroy_process_group()


def _lockstep_reference(world):
    """Both ranks' populations stepped in one process with the oracle: the
    global estimate per step, each population combed with PCG64([seed, rank]),
    E_0 from the global estimates."""
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import afqmc_ref as R
    from paper_2403_02542_gb300 import energy as S
    from paper_2403_02542_gb300.inputs import make_fields, make_system
    s = make_system(10, 2, 2, 16, rho=0.8, seed=12)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb, s.e_const)
    Lbar = R.mean_field_shift(ham)
    hpp, ec = R.propagation_h1(ham, Lbar)
    B = R.half_step_propagator(hpp, TAU)
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    pops = [list(R.init_walkers(ham, NW)) for _ in range(world)]
    rngs = [np.random.Generator(np.random.PCG64([SEED, r])) for r in range(world)]
    Ws, Es, E0s = [], [], []
    for k in range(N_STEPS):
        reo = (k + 1) % REO == 0
        num = den = 0.0
        for r in range(world):
            psi, lo, W = pops[r]
            psi, lo, W, _ = R.step(ham, psi, lo, W, make_fields(77 + r, k, NW, ham.G), TAU, e0, method="krylov",
                                   k=ORDER, reortho=reo, B=B, L_bar=Lbar, ec=ec)
            pops[r] = [psi, lo, W]
            emix, wsum = R.mixed_energy(W, R.energy_window(R.local_energy(ham, psi), e0, TAU, ham.na + ham.nb))
            num += float(wsum) * float(emix) if float(wsum) > 0 else 0.0
            den += float(wsum)
        E0s.append(e0)
        Ws.append(den)
        Es.append(num / den)
        if (k + 1) % POP == 0:
            for r in range(world):
                psi, lo, W, _ = R.population_control(*pops[r], float(rngs[r].random()))
                pops[r] = [psi, lo, W]
            e0 = Es[-1] if k < N_EQ else S.time_average(Ws, Es, N_EQ)[0]
    return Ws, Es, E0s


def test_sharded_energy_run_matches_the_lockstep_protocol():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_energy_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    Wr, Er, E0r = _lockstep_reference(world)
    for rank, W, E, e0s, W_local in out:
        assert W == pytest.approx(Wr, rel=1e-13), rank
        assert E == pytest.approx(Er, rel=1e-13), rank
        assert e0s == pytest.approx(E0r, rel=1e-13), rank
    assert out[0][4] != out[1][4]                          # the ranks hold different walkers
    assert [a + b for a, b in zip(out[0][4], out[1][4])] == pytest.approx(Wr, rel=1e-13)
