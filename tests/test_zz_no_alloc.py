"""The allocation-free batched core nnCPD (nncp_core_fit_batched_noalloc).

Some callers cannot let a library allocate device memory: their runtime owns
every byte through its own pool, or they run a latency-critical loop where an
allocation may stall or fail. For them the library keeps the job table of the
batched core fit in a fixed array of its own device memory. This file checks,
through the C ABI, that two calls in a row of that entry point return what the
allocating entry point returns on the same problems, and that an oversized
batch is refused. It is collected last so that a stop at the first failure has
run every other test first; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1909_07570_gb300 import inputs, native

pytestmark = pytest.mark.gpu


def _problems(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        d = 3 if i % 4 else 4
        m = tuple(int(v) for v in rng.integers(2, 17, size=d))
        r = int(rng.integers(2, 9))
        G0 = rng.random(m)
        B0 = inputs.initial_cp(m, r, seed + i)
        out.append((G0, B0))
    return out


def _to_device(problems):
    return [(torch.tensor(G, dtype=torch.float32, device="cuda"),
             [torch.tensor(b, dtype=torch.float32, device="cuda") for b in B])
            for G, B in problems]


@pytest.mark.parametrize("call", [0, 1])
def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(call):
    # Two calls in a row with different batches: the second overwrites the
    # shared table the first one used.
    for seed, count in ((7, 45), (8, 23)):
        probs = _problems(seed + 100 * call, count)
        ref = _to_device(probs)
        new = _to_device(probs)
        e_ref = native.nncp_core_fit_batched(ref, 25)
        e_new = native.nncp_core_fit_batched_noalloc(new, 25)
        torch.cuda.synchronize()
        np.testing.assert_allclose(e_new.cpu().numpy(), e_ref.cpu().numpy(), rtol=1e-6, atol=0)
        for (_, Br), (_, Bn) in zip(ref, new):
            for a, b in zip(Br, Bn):
                np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=1e-6, atol=1e-9)


def test_noalloc_rejects_more_jobs_than_its_table():
    G = torch.rand(3, 3, 3, device="cuda")
    B = [torch.rand(3, 2, device="cuda") for _ in range(3)]
    with pytest.raises(native.NncError) as ei:
        native.nncp_core_fit_batched_noalloc([(G, B)] * 4097, 2)
    assert ei.value.status == -1
    assert "4096" in str(ei.value)


def test_noalloc_refuses_batches_for_the_two_pass_kernel():
    # A 40 x 40 x 40 tensor (64,000 entries) sends the allocating call to its
    # two-pass kernel; the no-alloc entry refuses the batch instead of running
    # another kernel, and says why.
    G = torch.rand(40, 40, 40, device="cuda")
    B = [torch.rand(40, 3, device="cuda") for _ in range(3)]
    with pytest.raises(native.NncError) as ei:
        native.nncp_core_fit_batched_noalloc([(G, B)], 5)
    assert ei.value.status == -6
    assert "two-pass" in str(ei.value)
    # The same batch runs through the allocating entry point.
    native.nncp_core_fit_batched([(G, B)], 5)


def test_noalloc_checks_options_and_clears_the_error_detail():
    G = torch.rand(4, 5, 3, device="cuda")
    B = [torch.rand(n, 2, device="cuda") for n in (4, 5, 3)]
    lib = native.load()
    jobs = (native.nncp_job * 1)()
    jobs[0].G, jobs[0].d, jobs[0].r = G.data_ptr(), 3, 2
    for n in range(3):
        jobs[0].m[n] = G.shape[n]
        jobs[0].B[n] = B[n].data_ptr()
    errs = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    bad = native.nnc_opts(3, 4, 1e-12)  # refine_iters > iters, as the allocating call rejects
    for entry in ("nncp_core_fit_batched", "nncp_core_fit_batched_noalloc"):
        assert getattr(lib, entry)(1, jobs, native.NNC_FP32, ctypes.byref(bad),
                                   ctypes.c_void_p(errs.data_ptr()), None, stream) == -1
    assert lib.nnc_last_error_detail() != b""
    good = native.nnc_opts(3, 0, 1e-12)
    assert lib.nncp_core_fit_batched_noalloc(1, jobs, native.NNC_FP32, ctypes.byref(good),
                                             ctypes.c_void_p(errs.data_ptr()),
                                             ctypes.c_void_p(st.data_ptr()), stream) == 0
    assert lib.nnc_last_error_detail() == b""
    assert int(st.item()) == 0
