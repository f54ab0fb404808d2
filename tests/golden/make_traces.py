"""Writes the FP64 oracle traces that the full-length GPU parity tests compare
against (tests/test_gpu_fulllength.py).

Calls nothing but the oracle (``oracle/``) and the seeded input generator
(``paper_1909_07570_gb300.inputs``, which holds none of the method's
arithmetic). Every case runs the oracle on exactly the input the FP32 GPU path
receives: X rounded to float32 (and widened back to float64), the initial
factors as drawn. Each output file records the command that wrote it.

    python tests/golden/make_traces.py                 # every case
    python tests/golden/make_traces.py ntd_cp10_256cube_500 ...

Cases (the sweep counts of the synthetic workloads; the paper's protocol is a
fixed number of iterations without early stopping, Sec. 4.1):

  ntd_cp10_256cube_500      nnTD (Alg. 1, step 1) of the 256^3 rank-10 workload,
                            m = (20, 20, 20), 500 sweeps: per-sweep relative
                            error (FP64 identity) and the explicit final error;
                            then nnCPD of the fitted core (r = 10, 500 sweeps)
                            and the relative error of the lifted model
  ntd_cp16_512cube_200      nnTD of the 512^3 rank-16 workload, m = 32, 200
                            sweeps (the precision form's sweep count)
  ntd_cp16_512cube_5000     the same for the paper's 5000 sweeps, relative
                            error every sweep
  ntd4_cp12_128x128x128x64_300  nnTD of the 4-way workload, m = (24, 24, 24, 16),
                            300 sweeps
  pg_cp12_128x128x128x64_300    300 block projected-gradient steps on the lifted
                            loss of the same tensor (r = 12): loss after each
  batch64_subset            tensors 0 and 1 of the 64-tensor uneven batch: nnTD
                            (m = 2r, 500 sweeps), then core nnCPD at CP ranks 2,
                            5, 8 (restart 0, 500 sweeps) of the oracle's core
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1909_07570_gb300 import inputs  # noqa: E402


def as_fp32_input(X):
    """The tensor the FP32 GPU path computes on: X rounded to float32."""
    return np.asarray(X, dtype=np.float32).astype(np.float64)


def write(name, header, records):
    """records: list of (key, 1-D array). Format read by tests/_golden.py."""
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as fh:
        fh.write(f"# {name}: FP64 oracle output, written by\n")
        fh.write(f"#   python tests/golden/make_traces.py {name}\n")
        for ln in header:
            fh.write(f"# {ln}\n")
        for key, v in records:
            v = np.atleast_1d(np.asarray(v, dtype=np.float64))
            fh.write(f"vector {key} {v.size}\n")
            fh.write(" ".join(repr(float(x)) for x in v) + "\n")
    print(f"wrote {path}", flush=True)


def ntd_case(wname, sweeps, with_core=False):
    w = inputs.WORKLOADS[wname]
    X, _, F0, G0, B0 = inputs.make_problem(w)
    X = as_fp32_input(X)
    F, G, trace = oracle.ntd_fit(X, F0, G0, sweeps)
    recs = [("trace", trace), ("final_rel_err", oracle.rel_err_tucker(X, G, F))]
    head = [f"workload {wname}: dims {w.dims}, m {w.m}, {sweeps} sweeps, eps 1e-12",
            "trace: ||X - G x_k F^(k)|| / ||X|| after each sweep (residual identity, FP64)",
            "final_rel_err: the same error from the explicit reconstruction"]
    if with_core:
        B, ctr = oracle.nncp_fit(G, B0, w.cp_iters)
        A = oracle.lift(F, B)
        recs += [("core_trace", ctr), ("lifted_rel_err", oracle.rel_err_cp(X, A))]
        head += [f"core_trace: nnCPD of the fitted core, r = {w.r}, {w.cp_iters} sweeps",
                 "lifted_rel_err: ||X - I x_k F^(k) B^(k)|| / ||X|| (Eq. nnCANDELINC)"]
    return recs, head


def pg_case(wname, steps):
    w = inputs.WORKLOADS[wname]
    X, _, F0, _, B0 = inputs.make_problem(w)
    X = as_fp32_input(X)
    _, _, trace = oracle.lifted_pg_fit(X, F0, B0, steps)
    x2 = float(np.sum(X * X))
    return [("loss", trace), ("x_norm_sq", x2)], [
        f"workload {wname}: dims {w.dims}, m {w.m}, r {w.r}, {steps} projected-gradient steps",
        "loss: 1/2 ||X - I x_n F^(n) B^(n)||^2 after each step; x_norm_sq: ||X||^2"]


def batch_case():
    probs = inputs.batch_problems()
    B = inputs.BATCH
    recs, head = [], [f"batch {B['name']}: tensors 0 and 1, nnTD {B['iters']} sweeps, "
                      f"core nnCPD {B['cp_iters']} sweeps at ranks 2, 5, 8 (restart 0)"]
    for b in (0, 1):
        p = probs[b]
        X = as_fp32_input(p["X"])
        F, G, trace = oracle.ntd_fit(X, p["F0"], p["G0"], B["iters"])
        recs.append((f"t{b}_trace", trace))
        recs.append((f"t{b}_final_rel_err", oracle.rel_err_tucker(X, G, F)))
        inits = {(rk, rs): B0 for rk, rs, B0 in inputs.batch_core_inits(p["m"], b)}
        for rk in (2, 5, 8):
            _, ctr = oracle.nncp_fit(G, inits[(rk, 0)], B["cp_iters"])
            recs.append((f"t{b}_core_r{rk}_rel_err", ctr[-1]))
        head.append(f"tensor {b}: dims {p['dims']}, planted rank {p['r']}, m {p['m']}")
    return recs, head


CASES = {
    "ntd_cp10_256cube_500": lambda: ntd_case("cp10_256x256x256_m20_fp32", 500, with_core=True),
    "ntd_cp16_512cube_200": lambda: ntd_case("cp16_512x512x512_m32_bf16", 200),
    "ntd_cp16_512cube_5000": lambda: ntd_case("cp16_512x512x512_m32_bf16", 5000),
    "ntd4_cp12_128x128x128x64_300": lambda: ntd_case("cp12_128x128x128x64_m24_fp32", 300),
    "pg_cp12_128x128x128x64_300": lambda: pg_case("cp12_128x128x128x64_m24_fp32", 300),
    "batch64_subset": batch_case,
}


def main(names):
    for name in names or list(CASES):
        t0 = time.time()
        recs, head = CASES[name]()
        write(name, head, recs)
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
