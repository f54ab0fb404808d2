"""The batched tiny-problem kernels against the oracle, and the multirank
study of Sec. 4.3 (Ex. "equal") end to end on a reduced number of starts."""
import numpy as np
import pytest
import torch

import oracle as orc
from _golden import load
from paper_1909_07570_gb300 import inputs, native, study

pytestmark = pytest.mark.gpu


def test_example_equal_factors_are_the_printed_ones():
    g = load("ex_equal.txt")
    for a, key in zip(inputs.example_equal_factors(), ("A1", "A2", "A3")):
        np.testing.assert_array_equal(a, g[key])


@pytest.mark.parametrize("m", [(3, 3, 3), (3, 4, 4), (5, 5, 5), (2, 6, 3)])
def test_ntd_small_batched_matches_oracle(m):
    A = inputs.example_equal_factors()
    X = np.einsum("iq,jq,kq->ijk", *A)
    inits = inputs.study_inits((4, 4, 4), m, 4, 5, seed=7)
    Xd = torch.tensor(X, device="cuda")
    F = [[torch.tensor(f, device="cuda") for f in s["F"]] for s in inits]
    G = [torch.tensor(s["G"], device="cuda") for s in inits]
    errs = native.ntd_fit_small_batched([(Xd, F[i], G[i]) for i in range(5)], 40).cpu().numpy()
    for i, s in enumerate(inits):
        Fo, Go, _ = orc.ntd_fit(X, s["F"], s["G"], 40)
        for a, b in zip(F[i], Fo):
            np.testing.assert_allclose(a.cpu().numpy(), b, rtol=1e-9, atol=1e-13)
        np.testing.assert_allclose(G[i].cpu().numpy(), Go, rtol=1e-9, atol=1e-13)
        assert errs[i] == pytest.approx(orc.rel_err_tucker(X, Go, Fo), rel=1e-9, abs=1e-13)


def test_nmf_and_lifted_batched_match_oracle():
    rng = np.random.default_rng(8)
    probs = [(rng.random((n, 4)), 1 - rng.random((n, k)), 1 - rng.random((k, 4)))
             for n, k in ((4, 3), (7, 5), (12, 4))]
    dev = [tuple(torch.tensor(x, device="cuda") for x in p) for p in probs]
    errs = native.nmf_fit_batched(dev, 60).cpu().numpy()
    for (A, F0, B0), (_, F, B), e in zip(probs, dev, errs):
        Fo, Bo, tro = orc.nmf_fit(A, F0, B0, 60)
        np.testing.assert_allclose(F.cpu().numpy(), Fo, rtol=1e-9, atol=1e-13)
        np.testing.assert_allclose(B.cpu().numpy(), Bo, rtol=1e-9, atol=1e-13)
        assert e == pytest.approx(tro[-1], rel=1e-9)
    X = rng.random((5, 6, 7))
    Fs = [1 - rng.random((n, k)) for n, k in zip(X.shape, (2, 3, 4))]
    Bs = [1 - rng.random((k, 3)) for k in (2, 3, 4)]
    e = native.lifted_rel_err_batched([(torch.tensor(X, device="cuda"),
                                        [torch.tensor(f, device="cuda") for f in Fs],
                                        [torch.tensor(b, device="cuda") for b in Bs])])
    assert e.item() == pytest.approx(orc.rel_err_cp(X, orc.lift(Fs, Bs)), rel=1e-12)


def test_multirank_study_runs_and_alg_pieces_agree_with_oracle():
    res = study.run(starts=40, iters=300, seed=11)
    assert len(res) == 8
    for v in res.values():
        assert np.isfinite(v["rel_err"]).all() and (v["rel_err"] >= 0).all()
        assert ((v["congruence"] >= -1e-12) & (v["congruence"] <= 1 + 1e-12)).all()
    # One start of each algorithm at the canonical multirank, recomputed by the oracle.
    A = inputs.example_equal_factors()
    X = np.einsum("iq,jq,kq->ijk", *A)
    s = inputs.study_inits((4, 4, 4), (4, 4, 4), 4, 40, 11 + 101 * 2)[0]
    Fo, Go, _ = orc.ntd_fit(X, s["F"], s["G"], 300)
    Bo, _ = orc.nncp_fit(Go, s["B"], 300)
    assert res[("alg1", (4, 4, 4))]["rel_err"][0] == pytest.approx(
        orc.rel_err_cp(X, orc.lift(Fo, Bo)), rel=1e-7, abs=1e-10)
    Ao, F2o, B2o, _, _ = orc.alg2_fit(X, s["A"], s["F2"], s["B2"], 300, 300)
    assert res[("alg2", (4, 4, 4))]["rel_err"][0] == pytest.approx(
        orc.rel_err_cp(X, orc.lift(F2o, B2o)), rel=1e-7, abs=1e-10)
    summ = study.summary(res)
    assert set(summ) == {f"{a}_{m}" for a in ("alg1", "alg2")
                         for m in ("3x3x3", "3x4x4", "4x4x4", "5x5x5")}


# ---------------------------------------------------------------------------
# Problems whose X does not fit in shared memory (X read from global memory,
# two passes per sweep) and the batch experiment of Sec. 4.3
# ---------------------------------------------------------------------------

L2_SHAPES = [((40, 40, 40), (3, 4, 5)), ((37, 29, 23), (5, 6, 7)), ((9, 50, 33), (2, 8, 3)),
             ((24, 20, 48), (12, 3, 9))]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_ntd_batched_x_in_global_memory_matches_oracle(dtype):
    probs = [inputs.small_problem(d, 3, m, 2, seed=31 + i, noise=0.02)
             for i, (d, m) in enumerate(L2_SHAPES)]
    Xd = [torch.tensor(p[0], dtype=dtype, device="cuda") for p in probs]
    F = [[torch.tensor(f, dtype=dtype, device="cuda") for f in p[2]] for p in probs]
    G = [torch.tensor(p[3], dtype=dtype, device="cuda") for p in probs]
    errs = native.ntd_fit_small_batched([(Xd[i], F[i], G[i]) for i in range(len(probs))],
                                        30).cpu().numpy()
    for i, p in enumerate(probs):
        Fo, Go, tro = orc.ntd_fit(p[0], p[2], p[3], 30)
        ref = orc.rel_err_tucker(p[0], Go, Fo)
        if dtype == torch.float64:
            for a, b in zip(F[i], Fo):
                np.testing.assert_allclose(a.cpu().numpy(), b, rtol=1e-9, atol=1e-14 * b.max())
            np.testing.assert_allclose(G[i].cpu().numpy(), Go, rtol=1e-9, atol=1e-14 * Go.max())
            assert errs[i] == pytest.approx(ref, rel=1e-9)
        else:
            assert abs(errs[i] - ref) <= 1e-5
        assert abs(ref - tro[-1]) <= 1e-10 * max(1.0, ref)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_nncp_batched_of_x_in_global_memory_matches_oracle(dtype):
    # nnCPD of X itself (Alg. 2, first step) through nncp_core_fit_batched with
    # tensors far larger than shared memory.
    cases = [((40, 40, 40), 5), ((37, 29, 23), 3), ((9, 50, 33), 12)]
    Xs, A0 = [], []
    for i, (d, r) in enumerate(cases):
        X, _ = inputs.planted_tensor(d, 4, 51 + i, noise=0.01)
        Xs.append(X)
        A0.append([1.0 - np.random.default_rng(61 + i).random((n, r)) for n in d])
    Xd = [torch.tensor(x, dtype=dtype, device="cuda") for x in Xs]
    A = [[torch.tensor(a, dtype=dtype, device="cuda") for a in a0] for a0 in A0]
    errs = native.nncp_core_fit_batched([(Xd[i], A[i]) for i in range(len(cases))],
                                        25).cpu().numpy()
    for i in range(len(cases)):
        Ao, tro = orc.nncp_fit(Xs[i], A0[i], 25)
        if dtype == torch.float64:
            for a, b in zip(A[i], Ao):
                np.testing.assert_allclose(a.cpu().numpy(), b, rtol=1e-9, atol=1e-14 * b.max())
            assert errs[i] == pytest.approx(tro[-1], rel=1e-9)
        else:
            assert abs(errs[i] - tro[-1]) <= 1e-5


def test_lifted_err_streams_a_large_x():
    X, _ = inputs.planted_tensor((40, 40, 40), 5, 71, noise=0.0)
    rng = np.random.default_rng(72)
    F = [rng.random((40, k)) for k in (3, 4, 5)]
    B = [rng.random((k, 5)) for k in (3, 4, 5)]
    e = native.lifted_rel_err_batched([(torch.tensor(X, device="cuda"),
                                        [torch.tensor(f, device="cuda") for f in F],
                                        [torch.tensor(b, device="cuda") for b in B])])
    assert float(e[0]) == pytest.approx(orc.rel_err_cp(X, orc.lift(F, B)), rel=1e-12)


def test_paper_batch_runs_and_matches_oracle_pipeline():
    # Six tensors of the Sec. 4.3 batch at 200 sweeps per stage; the first
    # tensor's whole pipeline (both algorithms) is replayed by the oracle.
    probs = inputs.paper_batch_problems(6)
    res = study.run_paper_batch(probs, iters=200)
    p = probs[0]
    Fo, Go, _ = orc.ntd_fit(p["X"], p["F"], p["G"], 200)
    Bo, _ = orc.nncp_fit(Go, p["B"], 200)
    e1 = orc.rel_err_cp(p["X"], orc.lift(Fo, Bo))
    assert res["alg1"]["rel_err"][0] == pytest.approx(e1, rel=1e-8, abs=1e-12)
    Ao, _ = orc.nncp_fit(p["X"], p["A"], 200)
    F2, B2 = [], []
    for k in range(3):
        f, b, _ = orc.nmf_fit(Ao[k], p["F2"][k], p["B2"][k], 200)
        F2.append(f)
        B2.append(b)
    e2 = orc.rel_err_cp(p["X"], orc.lift(F2, B2))
    assert res["alg2"]["rel_err"][0] == pytest.approx(e2, rel=1e-8, abs=1e-12)
    for alg in ("alg1", "alg2"):
        c = res[alg]["congruence"]
        assert np.all((c >= 0.0) & (c <= 1.0 + 1e-12))
        assert np.all(np.isfinite(res[alg]["rel_err"]))
