"""The benchmarked trajectory schedule against the FP64 oracle.

bench.py times 16^3 x 32 trajectories with this exact parameter set:
kappa = 0.1575, beta = 5.6, tau = 1, slabs of thickness l0 = 4, three
Omelyan levels (lambda = 0.1932) with n = (2, 4, 8) for the gauge, W1 and
boundary (Schur) forces, the W1 slab solves by the geometric series (Sec. 3),
chronological initial guesses, the molecular dynamics replayed as a CUDA
graph, single-precision inner storage with double defect correction to
1e-10, Metropolis and the x0 shift (Sec. 2).  Here the same set runs on a
field prepared the same way (links exp(i 0.6 H), pure-gauge HMC at
beta = 5.6) on an 8 x 4^3 lattice (two slabs of thickness 4): one oracle
trajectory of this schedule already takes about two minutes of host time
there (its CGNR solves need several hundred matrix applications each on a
thermalised field), so 16 x 8^3 (about half an hour) is out of reach of a
test.  Tolerances: |dH_gpu - dH_oracle| <= 1e-4 (the stated bound),
the same Metropolis decision and shift, links within 1e-6.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0710_0066_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0710_0066_gb300 import lqcd  # noqa: E402

LAM = 0.1931833275037836
KAPPA, BETA = 0.1575, 5.6


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def bench_params():
    return lqcd.hmc_params(BETA, KAPPA, 1.0, 3, (lqcd.SW, lqcd.SW, lqcd.SW), (2, 4, 8), 0, 1, 2, lam=LAM,
                           roll=1, metropolis=1, precision=lqcd.PREC_F32, tol=1e-10, max_iter=20000,
                           use_graph=1, chrono=1, block_solver=lqcd.SOLVER_SERIES)


def test_bench_schedule_trajectory_matches_oracle():
    L, l0, seed = (8, 4, 4, 4), 4, 2009
    lat = lqcd.Lattice(L, l0, -1)
    U = syn.random_links_torch(L, 0.6, seed, "cuda").contiguous()
    # input preparation: pure-gauge HMC at beta = 5.6 (20 trajectories
    # without accept/reject, 10 with)
    pg = lqcd.hmc_params(BETA, 0.0, 1.0, 1, (lqcd.SW,), (10,), 0, -1, -1, lam=LAM, roll=0, metropolis=0,
                         precision=lqcd.PREC_F64, tol=1e-10)
    for t in range(30):
        pg.metropolis = 1 if t >= 20 else 0
        U, _ = lat.hmc_trajectory(U, pg, seed, 1000000 + t)
    prm = bench_params()
    # one trajectory first, so that the compared one replays an already
    # recorded MD graph
    U, _ = lat.hmc_trajectory(U, prm, seed, 0)
    U_in = U.clone()
    U1, res = lat.hmc_trajectory(U, prm, seed, 1)
    olat = O.Lattice(L, l0, -1)
    oprm = O.hmc_params(BETA, KAPPA, 1.0, 3, (O.SW, O.SW, O.SW), [2, 4, 8], 0, 1, 2, lam=LAM, roll=1,
                        metropolis=1, tol=1e-11, maxit=50000)
    Uo, ores, st = olat.hmc_trajectory(U_in.cpu().numpy(), oprm, seed, 1)
    assert st == 0
    assert abs(res.dH - ores.dH) < 1e-4, (res.dH, ores.dH)
    assert res.accepted == ores.accepted and res.shift == ores.shift
    assert rel(U1, Uo) < 1e-6
    assert abs(res.plaq - ores.plaq) < 1e-9
    lat.close()
