"""The multirank study of Sec. 4.3 on the tensor of Ex. "equal": both
nnCANDELINC algorithms from many random starts at several assumed
multiranks, every fit on the GPU in batched launches (one thread block per
start):

  Alg. 1: nnTD (ntd_fit_small_batched), nnCPD of each fitted core
          (nncp_core_fit_batched), relative error of the lifted model;
  Alg. 2: nnCPD of X itself (nncp_core_fit_batched with X as the tensor),
          NMF of every CP factor (nmf_fit_batched), relative error of the
          lifted model.

The congruence against the planted factors (product of the cosines per
component, averaged over components under the best permutation, Sec. 4.1) is
a score of the results, computed on the host.
"""
from __future__ import annotations

import itertools

import numpy as np
import torch

from . import inputs, native


def mean_congruence(A, A_true):
    """Mean over components of prod_n cos(a_n, a_true_n), best permutation."""
    r = A_true[0].shape[1]
    C = np.ones((r, A[0].shape[1]))
    for a, t in zip(A, A_true):
        na = np.linalg.norm(a, axis=0)
        nt = np.linalg.norm(t, axis=0)
        with np.errstate(divide="ignore", invalid="ignore"):
            cos = (t.T @ a) / np.outer(nt, na)
        C = C * np.nan_to_num(cos)
    best = 0.0
    for perm in itertools.permutations(range(r)):
        best = max(best, float(np.mean(C[np.arange(r), perm])))
    return best


def batch_mean_congruence(A, A_true):
    """mean_congruence of many decompositions at once: A is a list over modes of
    (n, N_k, r) arrays, A_true a list over modes of (N_k, r) or (n, N_k, r)
    arrays. Returns n values (every permutation tried, as mean_congruence)."""
    n, r = A[0].shape[0], A[0].shape[2]
    C = np.ones((n, r, r))
    for a, t in zip(A, A_true):
        t = np.broadcast_to(t, (n,) + t.shape[-2:])
        na = np.linalg.norm(a, axis=1)                    # (n, r)
        nt = np.linalg.norm(t, axis=1)
        with np.errstate(divide="ignore", invalid="ignore"):
            cos = np.einsum("snq,snp->sqp", t, a) / (nt[:, :, None] * na[:, None, :])
        C = C * np.nan_to_num(cos)
    perms = np.array(list(itertools.permutations(range(r))))   # (P, r)
    vals = C[:, np.arange(r)[None, :], perms].mean(axis=2)     # (n, P)
    return vals.max(axis=1)


def run(multiranks=((3, 3, 3), (3, 4, 4), (4, 4, 4), (5, 5, 5)), starts=1000, iters=500,
        seed=2024, device="cuda"):
    """Returns {(alg, multirank): {"rel_err": array, "congruence": array}}."""
    dev = torch.device(device)
    A_true = inputs.example_equal_factors()
    dims, r = (4, 4, 4), 4
    Xh = np.einsum("iq,jq,kq->ijk", *A_true)
    X = torch.tensor(Xh, device=dev)
    out = {}
    def stack(arrs):  # one contiguous device tensor; row i is start i's array
        return torch.tensor(np.stack(arrs), device=dev)

    def congruences(Fs, Bs):
        A = [np.einsum("snm,smr->snr", f.cpu().numpy(), b.cpu().numpy()) for f, b in zip(Fs, Bs)]
        return batch_mean_congruence(A, A_true)

    for mi, m in enumerate(multiranks):
        inits = inputs.study_inits(dims, m, r, starts, seed + 101 * mi)
        # Alg. 1
        F = [stack([s["F"][k] for s in inits]) for k in range(3)]
        G = stack([s["G"] for s in inits])
        B = [stack([s["B"][k] for s in inits]) for k in range(3)]
        native.ntd_fit_small_batched([(X, [f[i] for f in F], G[i]) for i in range(starts)], iters)
        native.nncp_core_fit_batched([(G[i], [b[i] for b in B]) for i in range(starts)], iters)
        e1 = native.lifted_rel_err_batched(
            [(X, [f[i] for f in F], [b[i] for b in B]) for i in range(starts)]).cpu().numpy()
        out[("alg1", m)] = {"rel_err": e1, "congruence": congruences(F, B)}
        # Alg. 2
        A = [stack([s["A"][k] for s in inits]) for k in range(3)]
        F2 = [stack([s["F2"][k] for s in inits]) for k in range(3)]
        B2 = [stack([s["B2"][k] for s in inits]) for k in range(3)]
        native.nncp_core_fit_batched([(X, [a[i] for a in A]) for i in range(starts)], iters)
        native.nmf_fit_batched([(A[k][i], F2[k][i], B2[k][i]) for i in range(starts)
                                for k in range(3)], iters)
        e2 = native.lifted_rel_err_batched(
            [(X, [f[i] for f in F2], [b[i] for b in B2]) for i in range(starts)]).cpu().numpy()
        out[("alg2", m)] = {"rel_err": e2, "congruence": congruences(F2, B2)}
    return out


def run_paper_batch(problems=None, n_tensors=None, iters=None, dtype=torch.float64,
                    device="cuda", timings=None):
    """The batch experiment of Sec. 4.3: both algorithms on every tensor of
    inputs.paper_batch_problems (1000 planted 40^3 tensors, canonical multirank
    (3, 4, 5), rank 5, 5000 sweeps per stage in the paper), each stage one
    batched launch over all tensors. X (256 MB in FP32 at the paper's size)
    stays in global memory; each block keeps its factors and pass results in
    shared memory. Returns {"alg1" | "alg2": {"rel_err", "congruence"}} with
    the relative error of the lifted model and the congruence against the
    planted factors. With a dict `timings`, each batched GPU stage is timed
    with CUDA events on the current stream (milliseconds, stored by name)."""
    if problems is None:
        problems = inputs.paper_batch_problems(n_tensors)
    if iters is None:
        iters = inputs.PAPER_BATCH["iters"]
    dev = torch.device(device)
    n = len(problems)

    def stack(key, k=None):
        arrs = [p[key] if k is None else p[key][k] for p in problems]
        return torch.tensor(np.stack(arrs), dtype=dtype, device=dev)

    X = stack("X")

    A_true = [np.stack([p["A_true"][k] for p in problems]) for k in range(3)]

    def congruences(Fs, Bs):
        A = [np.einsum("snm,smr->snr", f.double().cpu().numpy(), b.double().cpu().numpy())
             for f, b in zip(Fs, Bs)]
        return batch_mean_congruence(A, A_true)

    def timed(name, fn):
        if timings is None:
            return fn()
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        timings[name] = e0.elapsed_time(e1)
        return r

    out = {}
    # Alg. 1: nnTD of every X, nnCPD of every core, lift.
    F = [stack("F", k) for k in range(3)]
    G = stack("G")
    B = [stack("B", k) for k in range(3)]
    j_ntd = [(X[i], [f[i] for f in F], G[i]) for i in range(n)]
    j_core = [(G[i], [b[i] for b in B]) for i in range(n)]
    j_err1 = [(X[i], [f[i] for f in F], [b[i] for b in B]) for i in range(n)]
    timed("alg1_ntd_ms", lambda: native.ntd_fit_small_batched(j_ntd, iters))
    timed("alg1_core_cp_ms", lambda: native.nncp_core_fit_batched(j_core, iters))
    e1 = timed("alg1_rel_err_ms", lambda: native.lifted_rel_err_batched(j_err1)).cpu().numpy()
    out["alg1"] = {"rel_err": e1, "congruence": congruences(F, B)}
    # Alg. 2: nnCPD of every X, NMF of every CP factor.
    A = [stack("A", k) for k in range(3)]
    F2 = [stack("F2", k) for k in range(3)]
    B2 = [stack("B2", k) for k in range(3)]
    j_cpx = [(X[i], [a[i] for a in A]) for i in range(n)]
    j_nmf = [(A[k][i], F2[k][i], B2[k][i]) for i in range(n) for k in range(3)]
    j_err2 = [(X[i], [f[i] for f in F2], [b[i] for b in B2]) for i in range(n)]
    timed("alg2_cp_ms", lambda: native.nncp_core_fit_batched(j_cpx, iters))
    timed("alg2_nmf_ms", lambda: native.nmf_fit_batched(j_nmf, iters))
    e2 = timed("alg2_rel_err_ms", lambda: native.lifted_rel_err_batched(j_err2)).cpu().numpy()
    out["alg2"] = {"rel_err": e2, "congruence": congruences(F2, B2)}
    return out


def summary(res):
    """Medians, quartiles and the share of starts with relative error < 1e-3."""
    rows = {}
    for (alg, m), v in res.items():
        e, c = v["rel_err"], v["congruence"]
        rows[f"{alg}_{'x'.join(map(str, m))}"] = {
            "rel_err_median": float(np.median(e)), "rel_err_q25": float(np.quantile(e, 0.25)),
            "rel_err_q75": float(np.quantile(e, 0.75)),
            "share_rel_err_below_1e-3": float(np.mean(e < 1e-3)),
            "congruence_mean": float(np.mean(c)), "congruence_std": float(np.std(c))}
    return rows


def summary_batch(res):
    """Per algorithm of the Sec. 4.3 batch: relative-error quartiles, the share
    of tensors below 1e-3, and the congruence mean and spread."""
    rows = {}
    for alg, v in res.items():
        e, c = v["rel_err"], v["congruence"]
        rows[alg] = {
            "rel_err_median": float(np.median(e)), "rel_err_q25": float(np.quantile(e, 0.25)),
            "rel_err_q75": float(np.quantile(e, 0.75)),
            "share_rel_err_below_1e-3": float(np.mean(e < 1e-3)),
            "congruence_mean": float(np.mean(c)), "congruence_std": float(np.std(c)),
            "share_congruence_above_0.99": float(np.mean(c > 0.99))}
    return rows
