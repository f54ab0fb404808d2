"""Per-fit statuses of the batched core nnCPD, the in-fit non-finite guard and
host-side allocation-failure injection. None of these faults the GPU: the bad
values are NaNs in the data or overflows in FP32 arithmetic, and the failing
allocation is refused on the host before the allocator is called.

* nncp_core_fit_batched writes one status per fit: a NaN in one job's core
  marks that job NONFINITE and leaves every other job's factors bitwise equal
  to a batch without the bad job; a bad descriptor marks its job INVALID_ARG
  and the rest still run (both kernels the batch may take).
* ntd_fit on a float32 tensor whose entries are near 1e30 overflows in FP32
  during the sweeps: the call returns NONFINITE and names the first bad sweep.
* nnc_debug_fail_alloc makes a chosen scratch allocation fail: the call
  returns ALLOC, and a fit right after matches the oracle.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as orc
from paper_1909_07570_gb300 import inputs, native

pytestmark = pytest.mark.gpu

NONFINITE, INVALID, ALLOC = -3, -1, -5


def _problems(seed, count, dims=None):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        if dims is None:
            d = 3 if i % 4 else 4
            m = tuple(int(v) for v in rng.integers(2, 13, size=d))
        else:
            m = dims
        r = int(rng.integers(2, 7))
        out.append((rng.random(m), inputs.initial_cp(m, r, seed + i)))
    return out


def _dev(problems, dtype=torch.float32):
    return [(torch.tensor(G, dtype=dtype, device="cuda"),
             [torch.tensor(b, dtype=dtype, device="cuda") for b in B]) for G, B in problems]


@pytest.mark.parametrize("dims,count", [(None, 11), ((30, 30, 30), 11), ((30, 30, 30), 20)])
def test_nan_core_marks_only_its_fit(dims, count):
    # dims None: small cores, the one-pass kernel; 30^3 cores (27,000 entries,
    # 3-way, r <= 16): the two-pass sweep, as one thread-block cluster per fit
    # (11 fits) or, when the clusters would not all fit on the GPU at once (20
    # fits), one block per fit.
    probs = _problems(11, count, dims)
    ref = _dev(probs)
    native.nncp_core_fit_batched(ref, 30)
    bad = _dev(probs)
    bad[4][0][(0,) * bad[4][0].dim()] = float("nan")
    st = torch.full((len(bad),), 99, dtype=torch.int32, device="cuda")
    errs = native.nncp_core_fit_batched(bad, 30, statuses=st)
    st = st.cpu().numpy()
    assert st[4] == NONFINITE
    assert (np.delete(st, 4) == 0).all()
    assert not np.isfinite(errs[4].item())
    for j in range(len(bad)):
        if j == 4:
            continue
        for a, b in zip(ref[j][1], bad[j][1]):
            assert torch.equal(a, b), j


def _raw_jobs(problems):
    jobs = (native.nncp_job * len(problems))()
    for i, (G, B) in enumerate(problems):
        jobs[i].G = G.data_ptr()
        jobs[i].d = G.dim()
        jobs[i].r = B[0].shape[1]
        for n in range(G.dim()):
            jobs[i].m[n] = G.shape[n]
            jobs[i].B[n] = B[n].data_ptr()
    return jobs


@pytest.mark.parametrize("dims", [None, (30, 30, 30)])
@pytest.mark.parametrize("entry", ["nncp_core_fit_batched", "nncp_core_fit_batched_noalloc"])
def test_bad_descriptor_marks_only_its_fit(entry, dims):
    if entry.endswith("noalloc") and dims is not None:
        pytest.skip("the no-alloc entry refuses batches for the two-pass kernel")
    probs = _problems(13, 7, dims)
    ref = _dev(probs)
    native.nncp_core_fit_batched(ref, 20)
    run = _dev(probs)
    jobs = _raw_jobs(run)
    jobs[2].r = 0  # invalid rank
    lib = native.load()
    opts = native.nnc_opts(20, 0, 1e-12)
    errs = torch.empty(len(run), dtype=torch.float64, device="cuda")
    st = torch.full((len(run),), 99, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # Without a status array a bad descriptor rejects the whole call.
    assert getattr(lib, entry)(len(run), jobs, native.NNC_FP32, ctypes.byref(opts),
                               ctypes.c_void_p(errs.data_ptr()), None, stream) == INVALID
    assert b"job 2" in lib.nnc_last_error_detail()
    rc = getattr(lib, entry)(len(run), jobs, native.NNC_FP32, ctypes.byref(opts),
                             ctypes.c_void_p(errs.data_ptr()), ctypes.c_void_p(st.data_ptr()),
                             stream)
    assert rc == 0
    st = st.cpu().numpy()
    assert st[2] == INVALID
    assert (np.delete(st, 2) == 0).all()
    for j in range(len(run)):
        if j != 2:
            for a, b in zip(ref[j][1], run[j][1]):
                assert torch.equal(a, b), j
    # The skipped job's factors are untouched: still the initial values.
    for b, b0 in zip(run[2][1], probs[2][1]):
        np.testing.assert_array_equal(b.cpu().numpy(), np.asarray(b0, dtype=np.float32))


def test_ntd_fit_overflow_in_fp32_is_reported():
    X, _, F0, G0, _ = inputs.small_problem((24, 20, 16), 3, (4, 4, 4), 2, seed=21)
    Xd = torch.tensor(X * 1e30, dtype=torch.float32, device="cuda")
    F = [torch.tensor(f, dtype=torch.float32, device="cuda") for f in F0]
    G = torch.tensor(G0, dtype=torch.float32, device="cuda")
    with pytest.raises(native.NncError) as ei:
        native.ntd_fit(Xd, F, G, 10)
    assert ei.value.status == NONFINITE
    assert "sweep" in str(ei.value)
    # The same data in FP64 is fine, and the context is intact.
    F = [torch.tensor(f, device="cuda") for f in F0]
    G = torch.tensor(G0, device="cuda")
    err, _ = native.ntd_fit(torch.tensor(X * 1e30, device="cuda"), F, G, 10)
    Fo, Go, _ = orc.ntd_fit(X, F0, G0, 10)
    assert err == pytest.approx(orc.rel_err_tucker(X, Go, Fo), rel=1e-9)


@pytest.mark.parametrize("nth", [1, 3, 7])
def test_injected_allocation_failure_then_a_clean_fit(nth):
    X, _, F0, G0, _ = inputs.small_problem((20, 128, 16), 3, (4, 5, 4), 2, seed=23)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    F = [torch.tensor(f, dtype=torch.float32, device="cuda") for f in F0]
    G = torch.tensor(G0, dtype=torch.float32, device="cuda")
    assert native.nnc_debug_fail_alloc(nth) == 0
    with pytest.raises(native.NncError) as ei:
        native.ntd_fit(Xd, F, G, 5)
    assert ei.value.status == ALLOC
    assert "injected" in str(ei.value)
    assert native.nnc_debug_fail_alloc(0) == 0  # fired once, then disarmed
    F = [torch.tensor(f, dtype=torch.float32, device="cuda") for f in F0]
    G = torch.tensor(G0, dtype=torch.float32, device="cuda")
    err, tr = native.ntd_fit(Xd, F, G, 5)
    Fo, Go, tro = orc.ntd_fit(X, F0, G0, 5)
    assert abs(err - orc.rel_err_tucker(X, Go, Fo)) <= 1e-5
    assert np.abs(tr.cpu().numpy() - tro).max() <= 1e-5
