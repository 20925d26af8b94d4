"""Replica sharding on CPU with two gloo ranks.

Each rank runs the oracle's Lanczos recurrences on its share of the summed
orbitals (standing in for its GPU); the tridiagonals are all-gathered and
the self-energy and QP energies evaluated from the gathered set must equal
the single-process result."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import gw_inputs as gi
import oracle as O
from paper_2310_20103_gb300 import replicas as R


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = gi.make_workload("r", 4, 9, 24, [2, 3, 5], list(range(13)), 61, 3, k=12)
    lo, hi = R.shard_range(wl.n_m, rank, world)
    sub = gi.Workload(**{**wl.__dict__, "m_idx": wl.m_idx[lo:hi], "M": wl.M[:, lo:hi]})
    b = O.start_vectors(sub.eps, sub.n_v, O.coupling_vectors(sub.L, sub.M))
    a, be, b0, ke = O.lanczos(lambda X: O.apply_casida(sub.eps, sub.n_v, sub.L, X),
                              b.reshape(-1, sub.n_vc), sub.k)
    n_loc = hi - lo
    A, Bt, B0, KE = R.gather_coefficients(
        torch.from_numpy(a).reshape(wl.n_t, n_loc, -1),
        torch.from_numpy(be).reshape(wl.n_t, n_loc, -1),
        torch.from_numpy(b0).reshape(wl.n_t, n_loc),
        torch.from_numpy(ke).reshape(wl.n_t, n_loc), wl.n_m)
    tmax = R.max_over_ranks(float(rank + 1))
    if rank == 0:
        sig, poles, _ = O.sigma_lanczos(wl, coeffs=(A.numpy(), Bt.numpy(), B0.numpy(),
                                                    KE.numpy()))
        E, _ = O.solve_all_qp(wl, poles)
        np.savez(out_path, sig=sig, E=E, tmax=tmax)
    dist.destroy_process_group()


def test_shard_range_partitions():
    for n in (1, 7, 256):
        for world in (1, 2, 3, 8):
            parts = [R.shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            assert max(h - l for l, h in parts) - min(h - l for l, h in parts) <= 1


def test_targets_for_step_cover_without_overlap():
    seen = []
    for step in range(4):
        for rank in range(2):
            seen += R.targets_for_step(step, rank, 2, 2, 16)
    assert sorted(seen) == list(range(16))


def test_two_gloo_ranks_match_single_process(tmp_path):
    out = str(tmp_path / "r0.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = np.load(out)
    wl = gi.make_workload("r", 4, 9, 24, [2, 3, 5], list(range(13)), 61, 3, k=12)
    sig, poles, _ = O.sigma_lanczos(wl)
    E, _ = O.solve_all_qp(wl, poles)
    np.testing.assert_allclose(got["sig"], sig, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(got["E"], E, rtol=1e-12)
    assert float(got["tmax"]) == 2.0
