"""Seeded synthetic inputs for nnCANDELINC, shared by the tests, the benchmark
and the oracle checks.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic. Both the CUDA path and the FP64 oracle receive the same
arrays from it (the data tensor X and the initial factors), so parity never
depends on two random generators agreeing.

The workloads stand in for the paper's synthetic experiments (Sec. 4.3: a
planted nonnegative CP with uniform factor entries); the paper's fluorescence
and copolymer data sets (Secs. 4.4, 4.5) are not available, so no real data is
used anywhere.

Recipe of a planted tensor:
  * factor entries A^(i)[n, q] i.i.d. from ``dist`` (uniform [0, 1) or
    exponential(1)); with ``zero_frac`` > 0 each entry is zeroed independently
    with that probability (sparse factors);
  * X0 = sum_q a^(1)_q o a^(2)_q o ... (outer products);
  * X = X0 + eta * E, with E i.i.d. uniform [0, 1) and eta chosen so that
    ||eta E||_F = noise * ||X0||_F.
Initial factors and cores are i.i.d. uniform on (0, 1]: strictly positive,
because a multiplicative update never moves an exact zero.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One synthetic nnCANDELINC problem: shapes, ranks, iteration counts."""

    name: str
    dims: tuple
    planted_rank: int
    m: tuple                 # Tucker multirank
    r: int                   # nnCP rank of the core
    iters: int               # nnTD sweeps
    cp_iters: int            # nnCP sweeps on the core
    dtype: str               # storage / arithmetic type of the plain path
    dist: str = "uniform"
    zero_frac: float = 0.0
    noise: float = 0.01
    seed: int = 1000
    refine_iters: int = 0    # FP32 refinement sweeps of the BF16 path
    extra: dict = field(default_factory=dict)


# The five workload shapes. Names state the content; sizes follow the task's
# synthetic configurations.
WORKLOADS = {
    "cp3_40x40x40_m5_fp64": Workload(
        "cp3_40x40x40_m5_fp64", (40, 40, 40), 3, (5, 5, 5), 3, 200, 200, "f64",
        noise=0.01, seed=1000),
    "cp10_256x256x256_m20_fp32": Workload(
        "cp10_256x256x256_m20_fp32", (256, 256, 256), 10, (20, 20, 20), 10, 500, 500, "f32",
        zero_frac=0.2, noise=0.02, seed=1001),
    "cp16_512x512x512_m32_bf16": Workload(
        "cp16_512x512x512_m32_bf16", (512, 512, 512), 16, (32, 32, 32), 16, 200, 200, "bf16",
        dist="exponential", noise=0.01, seed=1002, refine_iters=20),
    # The precision workload under the paper's protocol: 5000 iterations per
    # sub-solve without early stopping (Sec. 4.1); the last 200 nnTD sweeps
    # are FP32 refinement sweeps.
    "cp16_512x512x512_m32_bf16_5000": Workload(
        "cp16_512x512x512_m32_bf16_5000", (512, 512, 512), 16, (32, 32, 32), 16, 5000, 5000,
        "bf16", dist="exponential", noise=0.01, seed=1002, refine_iters=200),
    "cp12_128x128x128x64_m24_fp32": Workload(
        "cp12_128x128x128x64_m24_fp32", (128, 128, 128, 64), 12, (24, 24, 24, 16), 12, 300, 300,
        "f32", noise=0.01, seed=1004),
}


def planted_factors(dims, rank, rng, dist="uniform", zero_frac=0.0):
    """Factor matrices A^(i) (N_i x rank) of a planted nonnegative CP."""
    A = []
    for n in dims:
        if dist == "uniform":
            a = rng.random((n, rank))
        elif dist == "exponential":
            a = rng.exponential(1.0, (n, rank))
        else:
            raise ValueError(f"unknown distribution {dist!r}")
        if zero_frac > 0.0:
            a = a * (rng.random((n, rank)) >= zero_frac)
        A.append(a)
    return A


def _outer_sum(A):
    """sum_q a^(1)_q o ... o a^(d)_q, built mode by mode in float64."""
    d = len(A)
    letters = "abcdefgh"[:d]
    spec = ",".join(f"{c}z" for c in letters) + "->" + letters
    return np.ascontiguousarray(np.einsum(spec, *A, optimize=True))


def planted_tensor(dims, rank, seed, dist="uniform", zero_frac=0.0, noise=0.01):
    """X = X0 + eta E in float64, plus the planted factors (see module doc)."""
    rng = np.random.default_rng(seed)
    A = planted_factors(dims, rank, rng, dist, zero_frac)
    X = _outer_sum(A)
    if noise > 0.0:
        E = rng.random(X.shape)
        x0 = np.sqrt(np.sum(X * X))
        e = np.sqrt(np.sum(E * E))
        X += (noise * x0 / e) * E
    return X, A


def initial_tucker(dims, m, seed):
    """Initial F^(i) (N_i x m_i) and core G (m_1 x ... x m_d), i.i.d. U(0, 1]."""
    rng = np.random.default_rng(seed)
    F = [1.0 - rng.random((n, k)) for n, k in zip(dims, m)]
    G = 1.0 - rng.random(tuple(m))
    return F, G


def initial_cp(m, r, seed):
    """Initial B^(i) (m_i x r), i.i.d. U(0, 1]."""
    rng = np.random.default_rng(seed)
    return [1.0 - rng.random((k, r)) for k in m]


def make_problem(w: Workload):
    """X (float64), planted factors, initial (F, G) and initial B for ``w``."""
    X, A = planted_tensor(w.dims, w.planted_rank, w.seed, w.dist, w.zero_frac, w.noise)
    F0, G0 = initial_tucker(w.dims, w.m, w.seed + 7919)
    B0 = initial_cp(w.m, w.r, w.seed + 104729)
    return X, A, F0, G0, B0


def small_problem(dims, planted_rank, m, r, seed, dist="uniform", zero_frac=0.0, noise=0.01):
    """A planted problem of arbitrary shape, for tests."""
    w = Workload("custom", tuple(dims), planted_rank, tuple(m), r, 1, 1, "f64",
                 dist=dist, zero_frac=zero_frac, noise=noise, seed=seed)
    return make_problem(w)


# The batching workload: many planted tensors of uneven shapes (each mode
# length drawn from [32, 256]), planted rank r from [2, 8], multirank m = 2r,
# 1 % noise; each core then fitted at CP ranks 2..8 with 8 restarts. It stands
# in for the paper's many-small-tensor experiment (Sec. 4.3, 1000 planted
# tensors) at the batch sizes of the task's configuration.
BATCH = {"name": "batch64_uneven_32to256_m2r", "n_tensors": 64, "mode_range": (32, 256),
         "rank_range": (2, 8), "noise": 0.01, "seed": 1003, "iters": 500, "cp_iters": 500,
         "cp_ranks": tuple(range(2, 9)), "restarts": 8}


def batch_problems(n_tensors=None, seed=None):
    """The batching workload as a list of dicts {X (float64), dims, r, m, F0, G0}."""
    n = BATCH["n_tensors"] if n_tensors is None else n_tensors
    seed = BATCH["seed"] if seed is None else seed
    rng = np.random.default_rng(seed)
    lo, hi = BATCH["mode_range"]
    rlo, rhi = BATCH["rank_range"]
    out = []
    for b in range(n):
        dims = tuple(int(v) for v in rng.integers(lo, hi + 1, size=3))
        r = int(rng.integers(rlo, rhi + 1))
        m = (2 * r,) * 3
        X, _ = planted_tensor(dims, r, seed + 17 * (b + 1), noise=BATCH["noise"])
        F0, G0 = initial_tucker(dims, m, seed + 7919 + b)
        out.append({"X": X, "dims": dims, "r": r, "m": m, "F0": F0, "G0": G0})
    return out


def batch_core_inits(m, tensor_index, seed=None):
    """Initial B's of every (CP rank, restart) core fit of one batch tensor:
    a list of (rank, restart, [B^(n)])."""
    seed = BATCH["seed"] if seed is None else seed
    out = []
    for rk in BATCH["cp_ranks"]:
        for rs in range(BATCH["restarts"]):
            out.append((rk, rs, initial_cp(m, rk, seed + 104729 + 1009 * tensor_index
                                           + 31 * rk + rs)))
    return out


def example_equal_factors():
    """The factors A^(1), A^(2), A^(3) of Ex. "equal" (Sec. 3.1) as printed: X =
    I x_1 A^(1) x_2 A^(2) x_3 A^(3) is 4 x 4 x 4 with nonnegative rank 4 and
    nonnegative multirank (3, 4, 4); the tensor of the multirank study (Sec. 4.3)."""
    A1 = np.array([[1, 1, 0, 0], [1, 0, 1, 0], [0, 1, 0, 1], [0, 0, 1, 1]], dtype=np.float64)
    A2 = np.triu(np.ones((4, 4)))
    A3 = np.triu(np.ones((4, 4)))
    return [A1, A2, A3]


def study_inits(dims, m, r, starts, seed):
    """Random starts of the multirank study, i.i.d. U(0, 1]: per start the
    Tucker inits (F, G) and core CP init B of Alg. 1, and the CP init A and
    NMF inits (F, B) of Alg. 2."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(starts):
        out.append({
            "F": [1.0 - rng.random((n, k)) for n, k in zip(dims, m)],
            "G": 1.0 - rng.random(tuple(m)),
            "B": [1.0 - rng.random((k, r)) for k in m],
            "A": [1.0 - rng.random((n, r)) for n in dims],
            "F2": [1.0 - rng.random((n, k)) for n, k in zip(dims, m)],
            "B2": [1.0 - rng.random((k, r)) for k in m],
        })
    return out


# The batch experiment of Sec. 4.3: many tensors with a unique nnCPD whose
# factors are rank deficient, A^(i) = F^(i) B^(i) with F^(i) (N x kappa_i) and
# B^(i) (kappa_i x r) i.i.d. U[0, 1), X = I x_i A^(i) (no noise). A draw is
# kept only if the Kruskal ranks of the A^(i) add up to at least 2 r + 2
# (Kruskal's uniqueness condition; the paper's inequality sign is garbled).
# The paper's size: 1000 tensors of 40^3, kappa = (3, 4, 5), r = 5.
PAPER_BATCH = {"name": "paper_batch_1000x40cube_k345_r5", "n_tensors": 1000, "N": 40,
               "kappa": (3, 4, 5), "r": 5, "iters": 5000, "seed": 4300}


def kruskal_rank(A, tol=1e-9):
    """Largest k such that every k columns of A are linearly independent
    (input validation of the planted factors, by brute force over subsets)."""
    import itertools
    r = A.shape[1]
    for k in range(1, r + 1):
        for cols in itertools.combinations(range(r), k):
            if np.linalg.matrix_rank(A[:, cols], tol=tol * np.linalg.norm(A)) < k:
                return k - 1
    return r


def paper_batch_problems(n_tensors=None, N=None, seed=None):
    """The Sec. 4.3 batch: a list of dicts {X (float64), A_true, and per tensor
    the starts of both algorithms: F, G, B (Alg. 1) and A, F2, B2 (Alg. 2)},
    each U(0, 1], with the multirank m = kappa."""
    n = PAPER_BATCH["n_tensors"] if n_tensors is None else n_tensors
    N = PAPER_BATCH["N"] if N is None else N
    seed = PAPER_BATCH["seed"] if seed is None else seed
    kappa, r = PAPER_BATCH["kappa"], PAPER_BATCH["r"]
    dims = (N, N, N)
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        Fp = [rng.random((N, k)) for k in kappa]
        Bp = [rng.random((k, r)) for k in kappa]
        A = [f @ b for f, b in zip(Fp, Bp)]
        if sum(kruskal_rank(a) for a in A) < 2 * r + 2:
            continue
        X = _outer_sum(A)
        start = study_inits(dims, kappa, r, 1, int(rng.integers(1 << 31)))[0]
        start.update({"X": X, "A_true": A, "dims": dims, "m": kappa, "r": r})
        out.append(start)
    return out
