"""Failure detection without a GPU fault, and resuming a fit from saved factors.

* The tensor-core pass kernel bounds every mbarrier wait; the self-test runs
  that wait on a barrier nothing arrives on, with a limit of about a
  millisecond, and must get NNC_ERR_TIMEOUT back with the context intact.
* A fit of 2k sweeps and a fit of k sweeps resumed from its own output for k
  more agree (the MU state is just the factors and the core).
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1909_07570_gb300 import inputs, native

pytestmark = pytest.mark.gpu


def _dev(arrs, dtype):
    return [torch.tensor(a, dtype=dtype, device="cuda") for a in arrs]


def test_bounded_wait_gives_up_and_the_context_survives():
    assert native.nnc_wait_selftest(2_000_000) == -7
    assert native.nnc_wait_selftest(0) == -7
    # The context is still usable: a fit right after matches the oracle.
    X, _, F0, G0, _ = inputs.small_problem((12, 10, 8), 2, (3, 3, 3), 2, seed=3)
    F = _dev(F0, torch.float64)
    G = torch.tensor(G0, device="cuda")
    err, _ = native.ntd_fit(torch.tensor(X, device="cuda"), F, G, 5)
    Fo, Go, _ = orc.ntd_fit(X, F0, G0, 5)
    assert err == pytest.approx(orc.rel_err_tucker(X, Go, Fo), rel=1e-9)


@pytest.mark.parametrize("dtype,precision", [(torch.float64, "fp64"), (torch.float32, "fp32")])
def test_resumed_fit_matches_a_straight_fit(dtype, precision):
    X, _, F0, G0, _ = inputs.small_problem((40, 128, 36), 4, (5, 6, 7), 3, seed=17)
    Xd = torch.tensor(X, dtype=dtype, device="cuda")
    F1, G1 = _dev(F0, dtype), torch.tensor(G0, dtype=dtype, device="cuda")
    _, tr1 = native.ntd_fit(Xd, F1, G1, 40, precision=precision)
    F2, G2 = _dev(F0, dtype), torch.tensor(G0, dtype=dtype, device="cuda")
    _, tra = native.ntd_fit(Xd, F2, G2, 20, precision=precision)
    _, trb = native.ntd_fit(Xd, F2, G2, 20, precision=precision)  # resumed from F2, G2
    tol = 1e-11 if dtype == torch.float64 else 1e-5
    for a, b in zip(F1 + [G1], F2 + [G2]):
        np.testing.assert_allclose(b.double().cpu().numpy(), a.double().cpu().numpy(),
                                   rtol=tol, atol=tol * float(a.abs().max()))
    tr = np.concatenate([tra.cpu().numpy(), trb.cpu().numpy()])
    np.testing.assert_allclose(tr, tr1.cpu().numpy(), rtol=tol, atol=tol)
