"""Batching form on the GPU: ntd_fit_batched over tensors of uneven shapes
gives exactly the bits of one ntd_fit per problem (same kernels, same launch
shapes), agrees with the oracle, and reports per-job failures."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1909_07570_gb300 import inputs, native

pytestmark = pytest.mark.gpu


def _dev(p, dt):
    return (torch.tensor(p["X"], dtype=dt, device="cuda"),
            [torch.tensor(f, dtype=dt, device="cuda") for f in p["F0"]],
            torch.tensor(p["G0"], dtype=dt, device="cuda"))


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_batched_equals_single_fits_bitwise(precision):
    probs = inputs.batch_problems(n_tensors=6, seed=4242)
    probs = [dict(p, X=p["X"][:40, :36, :44].copy(order="C"), dims=(40, 36, 44),
                  F0=[p["F0"][0][:40], p["F0"][1][:36], p["F0"][2][:44]]) for p in probs]
    single = []
    for p in probs:
        X, F, G = _dev(p, torch.float32)
        err, tr = native.ntd_fit(X, F, G, 25, precision=precision)
        single.append((err, tr.cpu().numpy(), [f.cpu().numpy() for f in F], G.cpu().numpy()))
    batch = [_dev(p, torch.float32) for p in probs]
    errs, trs, sts = native.ntd_fit_batched(batch, 25, precision=precision, concurrency=4)
    assert sts == [0] * len(probs)
    for (X, F, G), e, tr, ref in zip(batch, errs, trs, single):
        assert e == ref[0]
        np.testing.assert_array_equal(tr.cpu().numpy(), ref[1])
        for a, b in zip(F, ref[2]):
            np.testing.assert_array_equal(a.cpu().numpy(), b)
        np.testing.assert_array_equal(G.cpu().numpy(), ref[3])


def test_batched_uneven_fp64_matches_oracle():
    probs = []
    for b, (dims, m) in enumerate([((13, 17, 11), (3, 4, 2)), ((29, 8, 21), (5, 2, 6)),
                                   ((7, 31, 16), (2, 6, 4))]):
        X, _, F0, G0, _ = inputs.small_problem(dims, 3, m, 2, seed=70 + b)
        probs.append({"X": X, "F0": F0, "G0": G0})
    batch = [_dev(p, torch.float64) for p in probs]
    errs, trs, sts = native.ntd_fit_batched(batch, 6, concurrency=3)
    for p, e, tr in zip(probs, errs, trs):
        Fo, Go, tro = orc.ntd_fit(p["X"], p["F0"], p["G0"], 6)
        np.testing.assert_allclose(tr.cpu().numpy(), tro, rtol=1e-9)
        assert abs(e - orc.rel_err_tucker(p["X"], Go, Fo)) < 1e-11


def test_batched_reports_the_failing_job():
    probs = inputs.batch_problems(n_tensors=3, seed=99)
    batch = [_dev(dict(p, X=p["X"][:20, :20, :20].copy(order="C"),
                       F0=[f[:20] for f in p["F0"]]), torch.float32) for p in probs]
    batch[1][0][0, 0, 0] = float("nan")
    with pytest.raises(native.NncError) as ei:
        native.ntd_fit_batched(batch, 3)
    assert ei.value.status == -3 and "job 1" in str(ei.value)


def _clone(ts):
    return [t.clone() for t in ts]


def test_autotuned_batched_fits_are_bit_identical_to_untuned():
    # The autotuner splits a fit's sweeps over trial launches at 32 .. 256
    # threads per block and runs the rest at the fastest; the results must be
    # the bits of one launch at 256 threads.
    rng = np.random.default_rng(5)
    cores, Bs = [], []
    for i in range(300):
        m = tuple(int(v) for v in rng.integers(2, 12, size=3))
        r = int(rng.integers(2, 9))
        cores.append(torch.tensor(rng.random(m), device="cuda"))
        Bs.append([torch.tensor(1.0 - rng.random((k, r)), device="cuda") for k in m])
    A = inputs.example_equal_factors()
    X = torch.tensor(np.einsum("iq,jq,kq->ijk", *A), device="cuda")
    inits = inputs.study_inits((4, 4, 4), (3, 4, 4), 4, 200, seed=9)
    big = inputs.paper_batch_problems(5, seed=77)
    runs = {}
    for on in (False, True):
        native.nnc_autotune_enable(on)
        B = [_clone(b) for b in Bs]
        e_cp = native.nncp_core_fit_batched([(cores[i], B[i]) for i in range(300)], 200)
        F = [[torch.tensor(f, device="cuda") for f in s["F"]] for s in inits]
        G = [torch.tensor(s["G"], device="cuda") for s in inits]
        e_ntd = native.ntd_fit_small_batched([(X, F[i], G[i]) for i in range(200)], 200)
        Xb = [torch.tensor(p["X"], device="cuda") for p in big]
        Fb = [[torch.tensor(f, device="cuda") for f in p["F"]] for p in big]
        Gb = [torch.tensor(p["G"], device="cuda") for p in big]
        e_l2 = native.ntd_fit_small_batched([(Xb[i], Fb[i], Gb[i]) for i in range(5)], 200)
        Ab = [[torch.tensor(a, device="cuda") for a in p["A"]] for p in big]
        e_cpx = native.nncp_core_fit_batched([(Xb[i], Ab[i]) for i in range(5)], 200)
        runs[on] = (e_cp, B, e_ntd, F, G, e_l2, Fb, Gb, e_cpx, Ab)
    native.nnc_autotune_enable(True)

    def flat(x):
        if isinstance(x, torch.Tensor):
            return [x.cpu().numpy()]
        return [a for y in x for a in flat(y)]

    for a, b in zip(flat(runs[False]), flat(runs[True])):
        np.testing.assert_array_equal(a, b)
