"""Host-side scoring of the Sec. 4.3 studies (no GPU): the congruence that
study.py computes for every decomposition agrees with the oracle's definition,
and the summaries report what they say."""
import numpy as np
import pytest

import oracle as orc
from paper_1909_07570_gb300 import study

RNG = np.random.default_rng(2027)


@pytest.mark.parametrize("r", [2, 4, 5])
def test_study_congruence_matches_the_oracle(r):
    for _ in range(5):
        A = [RNG.random((n, r)) for n in (7, 6, 5)]
        B = [RNG.random((n, r)) for n in (7, 6, 5)]
        assert study.mean_congruence(B, A) == pytest.approx(orc.mean_congruence(A, B), abs=1e-12)


def test_study_congruence_is_one_for_permuted_and_scaled_factors():
    A = [RNG.random((n, 5)) for n in (9, 8, 7)]
    perm = [3, 0, 4, 1, 2]
    B = [a[:, perm] * s for a, s in zip(A, (2.0, 0.5, 3.0))]
    assert study.mean_congruence(B, A) == pytest.approx(1.0, abs=1e-12)


def test_summaries():
    e = np.array([1e-4, 5e-4, 2e-3, 1e-2])
    c = np.array([0.995, 0.98, 0.999, 0.5])
    rows = study.summary_batch({"alg1": {"rel_err": e, "congruence": c}})["alg1"]
    assert rows["rel_err_median"] == pytest.approx(np.median(e))
    assert rows["share_rel_err_below_1e-3"] == pytest.approx(0.5)
    assert rows["share_congruence_above_0.99"] == pytest.approx(0.5)
    assert rows["congruence_mean"] == pytest.approx(np.mean(c))
    rows = study.summary({("alg2", (4, 4, 4)): {"rel_err": e, "congruence": c}})
    assert rows["alg2_4x4x4"]["share_rel_err_below_1e-3"] == pytest.approx(0.5)


def test_batch_congruence_matches_one_at_a_time():
    n, r = 7, 5
    A = [RNG.random((n, m, r)) for m in (9, 8, 7)]
    T = [RNG.random((n, m, r)) for m in (9, 8, 7)]
    got = study.batch_mean_congruence(A, T)
    for i in range(n):
        want = orc.mean_congruence([t[i] for t in T], [a[i] for a in A])
        assert got[i] == pytest.approx(want, abs=1e-12)
    T1 = [t[0] for t in T]  # one true decomposition for every fit (the multirank study)
    got1 = study.batch_mean_congruence(A, T1)
    for i in range(n):
        assert got1[i] == pytest.approx(study.mean_congruence([a[i] for a in A], T1), abs=1e-12)
