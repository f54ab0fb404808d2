"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Both sides get the same seeded X and initial factors from
paper_1909_07570_gb300.inputs. Tolerances:
  * FP64 path: 1e-9 relative, elementwise (only the summation order differs);
  * FP32 path: 1e-4 relative elementwise after one sweep (FP32 rounding of
    sums over up to a few hundred terms, then one multiplicative update), and
    |rel_err_gpu - rel_err_oracle| <= 1e-5 on the relative-error trace.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1909_07570_gb300 import inputs, native

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _t(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _np(t):
    return t.detach().double().cpu().numpy()


def _run_ntd(X, F0, G0, iters, dtype, **kw):
    Xd = _t(X, dtype)
    F = [_t(f, dtype) for f in F0]
    G = _t(G0, dtype)
    err, tr = native.ntd_fit(Xd, F, G, iters, **kw)
    return err, (_np(tr) if tr is not None else None), [_np(f) for f in F], _np(G)


# ---------------------------------------------------------------------------
# nnTD
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,m", [((37, 29, 23), (5, 6, 7)), ((70, 45, 133), (9, 17, 20)),
                                    ((300, 9, 65), (33, 4, 64)), ((70, 66, 68), (64, 64, 64))])
def test_ntd_one_sweep_fp64_elementwise(dims, m):
    X, _, F0, G0, _ = inputs.small_problem(dims, 4, m, 3, seed=101)
    err, tr, F, G = _run_ntd(X, F0, G0, 1, torch.float64)
    Fo, Go, _ = orc.ntd_sweep(X, F0, G0)
    for a, b in zip(F, Fo):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-14 * np.abs(b).max())
    np.testing.assert_allclose(G, Go, rtol=1e-9, atol=1e-14 * np.abs(Go).max())
    assert abs(err - orc.rel_err_tucker(X, Go, Fo)) < 1e-11
    assert abs(tr[0] - err) < 1e-9


# N2 = 128 and 256 (with N3 % 4 == 0) take the tensor-core pass that also forms
# the mode-1 contraction per tile: m2 % 4 != 0, m3 % 4 != 0 and m = 32 included.
# The last two shapes run every factor update, H kernel and core kernel on the
# tensor cores (m <= 32, multiples of 4) with odd row counts (a last block of
# one row) and contraction lengths off multiples of 64 and of 8.
@pytest.mark.parametrize("dims,m", [((37, 29, 23), (5, 6, 7)), ((70, 45, 133), (9, 17, 20)),
                                    ((257, 130, 97), (32, 24, 16)), ((70, 66, 68), (64, 64, 64)),
                                    ((23, 256, 44), (5, 7, 6)), ((19, 128, 40), (4, 32, 32)),
                                    ((257, 130, 100), (32, 24, 16)), ((45, 67, 36), (12, 20, 8))])
def test_ntd_one_sweep_fp32_elementwise(dims, m):
    X, _, F0, G0, _ = inputs.small_problem(dims, 5, m, 3, seed=202, zero_frac=0.2, noise=0.02)
    err, tr, F, G = _run_ntd(X, F0, G0, 1, torch.float32)
    Fo, Go, _ = orc.ntd_sweep(X, F0, G0)
    for a, b in zip(F, Fo):
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6 * np.abs(b).max())
    np.testing.assert_allclose(G, Go, rtol=1e-4, atol=1e-6 * np.abs(Go).max())
    assert abs(err - orc.rel_err_tucker(X, Go, Fo)) < 1e-5


def test_ntd_trace_fp64_cp3_40cube_full():
    # The 40x40x40 FP64 workload at its full size and sweep count.
    w = inputs.WORKLOADS["cp3_40x40x40_m5_fp64"]
    X, _, F0, G0, _ = inputs.make_problem(w)
    err, tr, F, G = _run_ntd(X, F0, G0, w.iters, torch.float64)
    Fo, Go, tro = orc.ntd_fit(X, F0, G0, w.iters)
    np.testing.assert_allclose(tr, tro, rtol=1e-8)
    assert abs(err - orc.rel_err_tucker(X, Go, Fo)) < 1e-9
    assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])


def test_ntd_trace_fp32_parity_and_monotone():
    X, _, F0, G0, _ = inputs.small_problem((64, 80, 96), 6, (8, 10, 12), 4, seed=303,
                                           zero_frac=0.2, noise=0.02)
    err, tr, F, G = _run_ntd(X, F0, G0, 150, torch.float32)
    Fo, Go, tro = orc.ntd_fit(X, F0, G0, 150)
    assert np.max(np.abs(tr - tro)) <= 1e-5
    assert abs(err - orc.rel_err_tucker(X, Go, Fo)) <= 1e-5
    assert all((f >= 0).all() for f in F) and (G >= 0).all()


def test_ntd_full_size_cp10_256cube_fp32():
    # The 256^3 FP32 workload at full size, in the launch configuration the
    # benchmark times; the oracle runs the first 6 sweeps.
    w = inputs.WORKLOADS["cp10_256x256x256_m20_fp32"]
    X, _, F0, G0, _ = inputs.make_problem(w)
    err, tr, F, G = _run_ntd(X, F0, G0, 6, torch.float32)
    Fo, Go, tro = orc.ntd_fit(X, F0, G0, 6)
    assert np.max(np.abs(tr - tro)) <= 1e-5
    for a, b in zip(F, Fo):
        np.testing.assert_allclose(a, b, rtol=2e-3, atol=1e-5 * np.abs(b).max())


def test_ntd_degenerate_shapes():
    # A mode of length 1, a rank of 1, and zero sweeps.
    X, _, F0, G0, _ = inputs.small_problem((1, 7, 5), 2, (1, 2, 3), 2, seed=5)
    err, tr, F, G = _run_ntd(X, F0, G0, 3, torch.float64)
    Fo, Go, tro = orc.ntd_fit(X, F0, G0, 3)
    np.testing.assert_allclose(tr, tro, rtol=1e-9)
    err0, tr0, F1, G1 = _run_ntd(X, F0, G0, 0, torch.float64, trace=False)
    for a, b in zip(F1, F0):
        np.testing.assert_array_equal(a, b)
    assert abs(err0 - orc.rel_err_tucker(X, G0, F0)) < 1e-12


def test_ntd_rejects_bad_input():
    X, _, F0, G0, _ = inputs.small_problem((6, 5, 4), 2, (2, 2, 2), 2, seed=9)
    for bad, status in ((-1.0, -2), (float("nan"), -3)):
        Xb = X.copy()
        Xb[2, 1, 3] = bad
        with pytest.raises(native.NncError) as ei:
            _run_ntd(Xb, F0, G0, 2, torch.float32)
        assert ei.value.status == status
    F0b = [np.ones((6, 65)), F0[1], F0[2]]
    with pytest.raises(native.NncError) as ei:
        _run_ntd(X, F0b, np.ones((65, 2, 2)), 2, torch.float32)
    assert ei.value.status == -1


# ---------------------------------------------------------------------------
# 4-way nnTD (the d-way mode-product sweep)
# ---------------------------------------------------------------------------

# (70, 45, 9, 10) has m = 64 and 40 (split-K numerators over up to 64 x 8 x 8
# terms per entry, several 32-row tiles of F^(1)); the last case has a core of
# 32,000 doubles with slices of up to 4,000 entries per index of mode 4.
@pytest.mark.parametrize("dims,m", [((13, 11, 9, 10), (3, 4, 2, 5)), ((7, 1, 12, 9), (2, 1, 3, 4)),
                                    ((6, 40, 5, 33), (6, 9, 5, 8)),
                                    ((70, 45, 9, 10), (64, 40, 8, 8)),
                                    ((41, 43, 11, 5), (40, 40, 10, 2))])
def test_ntd4_one_sweep_fp64_elementwise(dims, m):
    X, _, F0, G0, _ = inputs.small_problem(dims, 3, m, 2, seed=111)
    err, tr, F, G = _run_ntd(X, F0, G0, 1, torch.float64)
    Fo, Go, _ = orc.ntd_sweep(X, F0, G0)
    for a, b in zip(F, Fo):
        np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-14 * np.abs(b).max())
    np.testing.assert_allclose(G, Go, rtol=1e-9, atol=1e-14 * np.abs(Go).max())
    assert abs(err - orc.rel_err_tucker(X, Go, Fo)) < 1e-11
    assert abs(tr[0] - err) < 1e-9


# (20, 8, 16, 36) takes the TF32x3 tensor-core passes (X viewed as 20 x 128 x 36);
# N4 = 13 is not a multiple of 4 and runs the SIMT passes; fp32_simt forces them.
# N3 = 128 and 256: whole 128-row tiles of the pass X x_4 F4^T per (i, j), and
# a mode-2 column product with a single row chunk.
@pytest.mark.parametrize("dims,m,precision", [((20, 8, 16, 36), (4, 3, 5, 6), "fp32"),
                                              ((6, 5, 128, 12), (3, 4, 5, 6), "fp32"),
                                              ((4, 3, 256, 8), (3, 2, 24, 4), "fp32"),
                                              ((17, 9, 11, 13), (5, 4, 3, 2), "fp32"),
                                              ((20, 8, 16, 36), (4, 3, 5, 6), "fp32_simt")])
def test_ntd4_fp32_sweep_and_trace(dims, m, precision):
    X, _, F0, G0, _ = inputs.small_problem(dims, 4, m, 2, seed=212, zero_frac=0.2, noise=0.02)
    err, tr, F, G = _run_ntd(X, F0, G0, 1, torch.float32, precision=precision)
    Fo, Go, _ = orc.ntd_sweep(X, F0, G0)
    for a, b in zip(F, Fo):
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-6 * np.abs(b).max())
    np.testing.assert_allclose(G, Go, rtol=1e-4, atol=1e-6 * np.abs(Go).max())
    err, tr, F, G = _run_ntd(X, F0, G0, 40, torch.float32, precision=precision)
    Fo, Go, tro = orc.ntd_fit(X, F0, G0, 40)
    assert np.max(np.abs(tr - tro)) <= 1e-5
    assert abs(err - orc.rel_err_tucker(X, Go, Fo)) <= 1e-5
    assert all((f >= 0).all() for f in F) and (G >= 0).all()


def test_ntd4_trace_fp64_monotone():
    X, _, F0, G0, _ = inputs.small_problem((12, 10, 14, 9), 3, (3, 3, 4, 3), 2, seed=313)
    err, tr, F, G = _run_ntd(X, F0, G0, 30, torch.float64)
    Fo, Go, tro = orc.ntd_fit(X, F0, G0, 30)
    np.testing.assert_allclose(tr, tro, rtol=1e-8)
    assert abs(err - orc.rel_err_tucker(X, Go, Fo)) < 1e-9
    assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])


def test_ntd4_full_size_cp12_128x128x128x64_fp32():
    # The 4-way workload at full size (TF32x3 passes over X viewed as
    # 128 x 16384 x 64); the oracle runs the same 3 sweeps.
    w = inputs.WORKLOADS["cp12_128x128x128x64_m24_fp32"]
    X, _, F0, G0, _ = inputs.make_problem(w)
    err, tr, F, G = _run_ntd(X, F0, G0, 3, torch.float32)
    Fo, Go, tro = orc.ntd_fit(X, F0, G0, 3)
    assert np.max(np.abs(tr - tro)) <= 1e-5
    assert abs(err - orc.rel_err_tucker(X, Go, Fo)) <= 1e-5
    for a, b in zip(F, Fo):
        np.testing.assert_allclose(a, b, rtol=2e-3, atol=1e-5 * np.abs(b).max())


def test_ntd4_limits():
    X, _, F0, G0, _ = inputs.small_problem((6, 5, 4, 8), 2, (2, 2, 2, 2), 2, seed=19)
    with pytest.raises(native.NncError) as ei:  # no BF16 form for d = 4
        _run_ntd(X, F0, G0, 2, torch.float32, precision="bf16")
    assert ei.value.status == -6
    Xb = X.copy()
    Xb[1, 2, 3, 4] = -1.0
    with pytest.raises(native.NncError) as ei:
        _run_ntd(Xb, F0, G0, 2, torch.float64)
    assert ei.value.status == -2
    # Zero sweeps leave F and G as given.
    err0, _, F1, G1 = _run_ntd(X, F0, G0, 0, torch.float64, trace=False)
    for a, b in zip(F1, F0):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(G1, G0)
    assert abs(err0 - orc.rel_err_tucker(X, G0, F0)) < 1e-12


# ---------------------------------------------------------------------------
# nnCP of the core, batched fits, lift, residual
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,r", [((5, 6, 7), 4), ((20, 20, 20), 10), ((3, 4, 2, 5), 3),
                                 ((32, 32, 32), 16),
                                 # one thread-block cluster per fit (16384 entries or more,
                                 # 3-way, r <= 16): the last CTAs' slabs short or empty,
                                 # ranks that are not multiples of 4, the threshold itself
                                 ((27, 31, 26), 5), ((40, 24, 33), 13), ((64, 16, 16), 8)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_nncp_core_fit(m, r, dtype):
    rng = np.random.default_rng(sum(m) + r)
    G0 = rng.random(m)
    B0 = inputs.initial_cp(m, r, 17)
    iters = 40
    G = _t(G0, dtype)
    B = [_t(b, dtype) for b in B0]
    err = native.nncp_core_fit(G, B, iters)
    Bo, tro = orc.nncp_fit(G0, B0, iters)
    if dtype == torch.float64:
        for a, b in zip(B, Bo):
            np.testing.assert_allclose(_np(a), b, rtol=1e-9, atol=1e-13)
        assert abs(err - tro[-1]) < 1e-11
    else:
        for a, b in zip(B, Bo):
            np.testing.assert_allclose(_np(a), b, rtol=2e-3, atol=1e-5 * np.abs(b).max())
        assert abs(err - tro[-1]) < 1e-5


@pytest.mark.parametrize("count", [3, 20])
def test_nncp_batched_large_cores(count):
    # Large 3-way cores: a few run one cluster each (3 x 8 CTAs), a batch whose
    # clusters would not all fit on the GPU at once one block each (20 x 8 CTAs
    # > the SM count); either way every fit matches the oracle, and a single
    # fit of a batch of three gives the batch's bits.
    rng = np.random.default_rng(40 + count)
    problems, ref = [], []
    for i in range(count):
        m = tuple(int(v) for v in rng.integers(26, 34, size=3))
        r = int(rng.integers(3, 17))
        G0 = rng.random(m)
        B0 = inputs.initial_cp(m, r, 300 + i)
        problems.append((_t(G0, torch.float32), [_t(b, torch.float32) for b in B0]))
        ref.append((G0, B0))
    errs = native.nncp_core_fit_batched(problems, 25).cpu().numpy()
    for i in range(0, count, 4 if count > 3 else 1):
        G0, B0 = ref[i]
        Bo, tro = orc.nncp_fit(G0, B0, 25)
        assert abs(errs[i] - tro[-1]) < 1e-5, i
        for a, b in zip(problems[i][1], Bo):
            np.testing.assert_allclose(_np(a), b, rtol=2e-3, atol=1e-5 * np.abs(b).max())
    if count == 3:
        G0, B0 = ref[1]
        G = _t(G0, torch.float32)
        B = [_t(b, torch.float32) for b in B0]
        e = native.nncp_core_fit(G, B, 25)
        assert e == errs[1]
        for a, b in zip(B, problems[1][1]):
            np.testing.assert_array_equal(_np(a), _np(b))


def test_nncp_batched_matches_single_fits():
    rng = np.random.default_rng(4)
    problems, singles = [], []
    for i in range(37):
        d = 3 if i % 5 else 4
        m = tuple(int(v) for v in rng.integers(2, 17, size=d))
        r = int(rng.integers(2, 9))
        G0 = rng.random(m)
        B0 = inputs.initial_cp(m, r, 100 + i)
        problems.append((_t(G0, torch.float32), [_t(b, torch.float32) for b in B0]))
        singles.append((_t(G0, torch.float32), [_t(b, torch.float32) for b in B0]))
    errs = native.nncp_core_fit_batched(problems, 30)
    for i, (G, B) in enumerate(singles):
        e = native.nncp_core_fit(G, B, 30)
        for a, b in zip(problems[i][1], B):
            np.testing.assert_array_equal(_np(a), _np(b))
        assert abs(float(errs[i]) - e) == 0.0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_lift_and_cp_residual(dtype):
    dims, m, r = (53, 41, 67), (7, 5, 9), 6
    rng = np.random.default_rng(8)
    F0 = [rng.random((n, k)) for n, k in zip(dims, m)]
    B0 = [rng.random((k, r)) for k in m]
    X, _ = inputs.planted_tensor(dims, 4, 11)
    A = native.candelinc_lift([_t(f, dtype) for f in F0], [_t(b, dtype) for b in B0])
    Ao = orc.lift(F0, B0)
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    for a, b in zip(A, Ao):
        np.testing.assert_allclose(_np(a), b, rtol=tol)
    rn, xn = native.recon_residual(_t(X, dtype), [_t(a, dtype) for a in Ao])
    ref = orc.rel_err_cp(X, Ao)
    assert abs(rn / xn - ref) <= (1e-12 if dtype == torch.float64 else 1e-6) * max(1.0, ref)
    assert abs(xn - orc.frobenius(X)) <= 1e-6 * xn


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_tucker_residual(dtype):
    dims, m = (45, 300, 259), (6, 7, 33)
    X, _, F0, G0, _ = inputs.small_problem(dims, 3, m, 2, seed=12)
    rn, xn = native.recon_residual(_t(X, dtype), [_t(f, dtype) for f in F0], _t(G0, dtype))
    ref = orc.rel_err_tucker(X, G0, F0)
    assert abs(rn / xn - ref) <= (1e-11 if dtype == torch.float64 else 1e-5) * ref


def test_alg1_end_to_end_fp64():
    # Alg. 1 on one small problem: nnTD, nnCP of the core, lift.
    X, _, F0, G0, B0 = inputs.small_problem((30, 26, 22), 3, (5, 5, 5), 3, seed=41)
    Xd = _t(X, torch.float64)
    F = [_t(f, torch.float64) for f in F0]
    G = _t(G0, torch.float64)
    native.ntd_fit(Xd, F, G, 50)
    B = [_t(b, torch.float64) for b in B0]
    native.nncp_core_fit(G, B, 60)
    A = native.candelinc_lift(F, B)
    rn, xn = native.recon_residual(Xd, A)
    Fo, Go, _ = orc.ntd_fit(X, F0, G0, 50)
    Bo, _ = orc.nncp_fit(Go, B0, 60)
    ref = orc.rel_err_cp(X, orc.lift(Fo, Bo))
    assert abs(rn / xn - ref) < 1e-9


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_residual_4way(dtype):
    dims, m, r = (17, 23, 9, 31), (4, 6, 3, 5), 5
    X, _, F0, G0, _ = inputs.small_problem(dims, 3, m, r, seed=23)
    rn, xn = native.recon_residual(_t(X, dtype), [_t(f, dtype) for f in F0], _t(G0, dtype))
    ref = orc.rel_err_tucker(X, G0, F0)
    assert abs(rn / xn - ref) <= (1e-11 if dtype == torch.float64 else 1e-5) * ref
    rng = np.random.default_rng(24)
    A = [rng.random((n, r)) for n in dims]
    rn, xn = native.recon_residual(_t(X, dtype), [_t(a, dtype) for a in A])
    ref = orc.rel_err_cp(X, A)
    assert abs(rn / xn - ref) <= (1e-12 if dtype == torch.float64 else 1e-6) * max(1.0, ref)
    assert abs(xn - orc.frobenius(X)) <= 1e-6 * xn
