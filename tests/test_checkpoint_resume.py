"""Checkpoint and resume of an HMC chain.

The chain's whole state between trajectories is the FP64 gauge field (the
x0 shift of the last trajectory is already applied to it) and the
counters of the counter-based generator, (seed, trajectory index): the
heatbath, momenta, Metropolis uniform and shift of trajectory t draw from
Philox4x32-10 at counter (index, stream, t) under key seed.  A checkpoint
is therefore U with (seed, next t).  Checked: a chain of three trajectories
and the same chain stopped after the first, written to an .npz file, read
back and continued give bit-identical fields, dH and decisions on the FP64
oracle (CPU), and the same fields to 1e-12, dH to 1e-10 and the same
decisions through the library with the molecular dynamics replayed as a
CUDA graph and chronological guesses on (GPU; the resumed half runs on a
fresh handle, as after a process restart).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0710_0066_gb300 import synthetic as syn

L, L0_SLAB, KAPPA, BETA = (4, 4, 4, 4), 2, 0.15, 5.6
SEED = 2301


def _oprm():
    return O.hmc_params(BETA, KAPPA, 0.5, 2, (O.SW, O.LF), [2, 2], 0, 0, 1, roll=1, tol=1e-13)


def test_oracle_chain_resumes_bit_identically(tmp_path):
    U0 = syn.random_links(L, 0.3, SEED)
    olat = O.Lattice(L, L0_SLAB, -1)
    prm = _oprm()
    # uninterrupted: trajectories 0, 1, 2
    U, ref = U0.copy(), []
    for t in range(3):
        U, res, st = olat.hmc_trajectory(U, prm, SEED, t)
        assert st == 0
        ref.append((res.dH, res.accepted, res.shift))
    U_ref = U
    # stopped after trajectory 0, checkpointed to disk, resumed
    U, res, st = olat.hmc_trajectory(U0.copy(), prm, SEED, 0)
    ck = tmp_path / "chain.npz"
    np.savez(ck, U=U, seed=np.uint64(SEED), next_traj=np.uint32(1))
    del U
    d = np.load(ck)
    U, seed, t0 = d["U"], int(d["seed"]), int(d["next_traj"])
    olat2 = O.Lattice(L, L0_SLAB, -1)
    got = []
    for t in range(t0, 3):
        U, res, st = olat2.hmc_trajectory(U, prm, seed, t)
        assert st == 0
        got.append((res.dH, res.accepted, res.shift))
    assert np.array_equal(U, U_ref)
    assert got == ref[1:]


@pytest.mark.gpu
def test_library_chain_resumes(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("no CUDA device")
    from paper_0710_0066_gb300 import lqcd

    U0 = torch.from_numpy(syn.random_links(L, 0.3, SEED)).cuda()
    prm = lqcd.hmc_params(BETA, KAPPA, 0.5, 2, (lqcd.SW, lqcd.LF), [2, 2], 0, 0, 1, roll=1,
                          precision=lqcd.PREC_F32, tol=1e-11, use_graph=1, chrono=2)
    lat = lqcd.Lattice(L, L0_SLAB, -1)
    U, ref = U0.clone(), []
    for t in range(3):
        U, res = lat.hmc_trajectory(U, prm, SEED, t)
        ref.append((res.dH, res.accepted, res.shift))
    U_ref = U.cpu().numpy()
    U, res = lat.hmc_trajectory(U0.clone(), prm, SEED, 0)
    lat.close()
    ck = tmp_path / "chain.npz"
    np.savez(ck, U=U.cpu().numpy(), seed=np.uint64(SEED), next_traj=np.uint32(1))
    d = np.load(ck)
    U, seed, t0 = torch.from_numpy(d["U"]).cuda(), int(d["seed"]), int(d["next_traj"])
    lat2 = lqcd.Lattice(L, L0_SLAB, -1)
    got = []
    for t in range(t0, 3):
        U, res = lat2.hmc_trajectory(U, prm, seed, t)
        got.append((res.dH, res.accepted, res.shift))
    lat2.close()
    # the library's kernels reduce in a fixed order, so the resumed chain
    # agrees to rounding at most (asserted at 1e-12 of the O(1) links)
    assert float(np.abs(U.cpu().numpy() - U_ref).max()) <= 1e-12
    for (a, b) in zip(got, ref[1:]):
        assert abs(a[0] - b[0]) <= 1e-10 and a[1:] == b[1:]
