"""Multi-rank paths on the CPU (gloo, world size 2).

1. Slab-sharded nnTD sweep. X is split along mode 3 into one slab per rank and
   F3 by the same rows; F1, F2 and G are replicated. Per sweep (Alg. 1, step 1,
   with the multiplicative updates of the oracle):
     - modes 1, 2: each rank contracts its slab (X_s x_3 F3_s^T ...), the
       partial numerators are all-reduced; Den needs S3 = sum_s F3_s^T F3_s,
       also all-reduced;
     - mode 3: rows of the slab only, no exchange;
     - core: M = sum_s X_s x_1 F1^T x_2 F2^T x_3 F3_s^T and S3 all-reduced;
     - residual by the identity ||X||^2 - 2<M, G> + <G, G x_k S_k> with
       ||X||^2 all-reduced once.
   The gathered result must equal the unsharded oracle's sweep up to the
   summation order (1e-10 relative).
2. The timing helpers of the benchmark (barrier, max over ranks) on gloo.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as orc
from oracle.tensor_algebra import mode_product, unfold
from paper_1909_07570_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORLD = 2
DIMS, M_RANKS, ITERS = (11, 9, 14), (3, 4, 5), 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)


def _allreduce(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _core_den(G, S):
    D = G
    for k, Sk in enumerate(S):
        D = mode_product(D, Sk, k)
    return D


def _sharded_sweep(Xs, F12, F3s, G, x2, eps):
    F = [F12[0].copy(), F12[1].copy()]
    for n in (0, 1):
        Fl = [F[0], F[1], F3s]
        Z = Xs
        for k in range(3):
            if k != n:
                Z = mode_product(Z, Fl[k].T, k)
        num = _allreduce(unfold(Z, n) @ unfold(G, n).T)
        S = [F[0].T @ F[0], F[1].T @ F[1], _allreduce(F3s.T @ F3s)]
        W = G
        for k in range(3):
            if k != n:
                W = mode_product(W, S[k], k)
        den = F[n] @ (unfold(W, n) @ unfold(G, n).T)
        F[n] = orc.mu_step(F[n], num, den, eps)
    Z = mode_product(mode_product(Xs, F[0].T, 0), F[1].T, 1)
    num3 = unfold(Z, 2) @ unfold(G, 2).T
    W = mode_product(mode_product(G, F[0].T @ F[0], 0), F[1].T @ F[1], 1)
    den3 = F3s @ (unfold(W, 2) @ unfold(G, 2).T)
    F3s = orc.mu_step(F3s, num3, den3, eps)
    M = _allreduce(mode_product(Z, F3s.T, 2))
    S = [F[0].T @ F[0], F[1].T @ F[1], _allreduce(F3s.T @ F3s)]
    G = orc.mu_step(G, M, _core_den(G, S), eps)
    r2 = x2 - 2.0 * float(np.sum(M * G)) + float(np.sum(G * _core_den(G, S)))
    return F, F3s, G, np.sqrt(max(r2, 0.0) / x2)


def _slab_worker(rank, port, out_dir):
    _init(rank, port)
    try:
        X, _, F0, G0, _ = inputs.small_problem(DIMS, 3, M_RANKS, 3, seed=515)
        bounds = np.linspace(0, DIMS[2], WORLD + 1).astype(int)
        k0, k1 = bounds[rank], bounds[rank + 1]
        Xs = np.ascontiguousarray(X[:, :, k0:k1])
        F12 = [F0[0].copy(), F0[1].copy()]
        F3s = F0[2][k0:k1].copy()
        G = G0.copy()
        x2 = float(_allreduce(np.array([np.sum(Xs * Xs)]))[0])
        trace = []
        for _ in range(ITERS):
            F12, F3s, G, e = _sharded_sweep(Xs, F12, F3s, G, x2, orc.DEFAULT_EPS)
            trace.append(e)
        gathered = [None] * WORLD
        dist.all_gather_object(gathered, F3s)
        if rank == 0:
            np.savez(os.path.join(out_dir, "sharded.npz"), F1=F12[0], F2=F12[1],
                     F3=np.concatenate(gathered, axis=0), G=G, trace=np.array(trace))
    finally:
        dist.destroy_process_group()


def test_slab_sharded_sweep_matches_unsharded_oracle(tmp_path):
    port = _free_port()
    mp.spawn(_slab_worker, args=(port, str(tmp_path)), nprocs=WORLD, join=True)
    got = np.load(tmp_path / "sharded.npz")
    X, _, F0, G0, _ = inputs.small_problem(DIMS, 3, M_RANKS, 3, seed=515)
    F, G, trace = orc.ntd_fit(X, F0, G0, ITERS)
    for name, ref in (("F1", F[0]), ("F2", F[1]), ("F3", F[2]), ("G", G)):
        np.testing.assert_allclose(got[name], ref, rtol=1e-10, atol=1e-14, err_msg=name)
    np.testing.assert_allclose(got["trace"], trace, rtol=1e-10)


def _bench_worker(rank, port, out_dir):
    _init(rank, port)
    try:
        sys.path.insert(0, ROOT)
        import bench
        bench.barrier(WORLD)
        v = bench.max_over_ranks(1.5 + rank, WORLD)
        with open(os.path.join(out_dir, f"max{rank}.txt"), "w") as f:
            f.write(repr(v))
    finally:
        dist.destroy_process_group()


def test_bench_max_over_ranks_gloo(tmp_path):
    port = _free_port()
    mp.spawn(_bench_worker, args=(port, str(tmp_path)), nprocs=WORLD, join=True)
    for r in range(WORLD):
        assert float((tmp_path / f"max{r}.txt").read_text()) == pytest.approx(1.5 + WORLD - 1)
