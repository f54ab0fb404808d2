"""Parity of the mode-product kernels (the passes over X) with the oracle's
n-mode product, and of the BF16 + FP32-refinement nnTD path with the oracle.

SIMT kernels: FP64 to 1e-12 and FP32 to 1e-5 (relative to the largest entry).
Tensor-core kernels: X and F are rounded to BF16 on the host (round to nearest
even, as the device does) and the oracle multiplies the rounded values in FP64;
the device accumulates the same products in FP32, so the bound is the FP32
accumulation error, 1e-5 relative to the largest entry. The per-slice scales of
the BF16 copy are powers of two, which change no rounding.
BF16 path of ntd_fit: |rel_err - rel_err_oracle| <= 1e-3.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1909_07570_gb300 import inputs, native

pytestmark = pytest.mark.gpu


def _bf16_round(a):
    return torch.tensor(a, dtype=torch.float32).bfloat16().double().numpy()


def _close(got, ref, rtol):
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err <= rtol * scale, f"max err {err:.3e} vs scale {scale:.3e}"


@pytest.mark.parametrize("dims", [(37, 29, 23), (70, 45, 133), (5, 300, 2)])
@pytest.mark.parametrize("Q", [1, 7, 20, 64])
def test_mode_product_simt(dims, Q):
    rng = np.random.default_rng(sum(dims) + Q)
    X = rng.random(dims)
    for mode in range(3):
        F = rng.random((dims[mode], Q))
        ref = orc.mode_product(X, F.T, mode)
        for dt, prec, tol in ((torch.float64, "fp64", 1e-12), (torch.float32, "fp32_simt", 1e-5)):
            Y = native.mode_product(torch.tensor(X, dtype=dt, device="cuda"),
                                    torch.tensor(F, dtype=dt, device="cuda"), mode, precision=prec)
            _close(Y.double().cpu().numpy(), ref, tol)


@pytest.mark.parametrize("dims,Q", [((37, 29, 24), 5), ((200, 150, 132), 20), ((256, 256, 256), 32),
                                    ((70, 45, 600), 64), ((129, 3, 64), 17), ((300, 7, 36), 33)])
def test_mode_product_tf32x3_is_fp32_accurate(dims, Q):
    # Three TF32 products per term with FP32 accumulation: the error bound is the
    # FP32 one (about K 2^-24 relative to the sum of |terms|), like the SIMT path.
    rng = np.random.default_rng(23 + Q)
    X = rng.random(dims) * np.exp2(rng.integers(-6, 7, size=(dims[0], 1, 1)))
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    X32 = Xd.double().cpu().numpy()  # the float32 values both sides see
    for mode in (0, 2):
        F = rng.random((dims[mode], Q)).astype(np.float32).astype(np.float64)
        ref = orc.mode_product(X32, F.T, mode)
        Y = native.mode_product(Xd, torch.tensor(F, dtype=torch.float32, device="cuda"), mode,
                                precision="fp32")
        _close(Y.double().cpu().numpy(), ref, 1e-5)


@pytest.mark.parametrize("dims,Q", [((37, 29, 24), 5), ((200, 150, 132), 20), ((64, 128, 2048), 24),
                                    ((24, 128, 16), 16), ((9, 33, 8), 32), ((3, 1000, 4), 24),
                                    ((11, 7, 4), 1), ((5, 300, 2), 24), ((20, 40, 12), 33),
                                    ((2, 200, 20000), 24)])
def test_mode_product_middle_mode_tf32x3_is_fp32_accurate(dims, Q):
    # Mode 1 (the middle mode, strided in memory) with NNC_FP32: the column
    # product on mma.sync with TF32x3 operands, each 16-row chunk summed apart
    # and added with round-to-nearest; N3 % 4 != 0 or Q > 32 take the SIMT
    # kernel. Ragged column blocks (L N3 not a multiple of 256), ragged row
    # chunks (N2 % 16 != 0) and the split-J launches of narrow grids included;
    # (2, 200, 20000) runs unsplit over 200 rows (13 chunks through the ring).
    rng = np.random.default_rng(29 + Q + dims[1])
    X = rng.random(dims) * np.exp2(rng.integers(-6, 7, size=(dims[0], 1, 1)))
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    X32 = Xd.double().cpu().numpy()
    F = rng.random((dims[1], Q)).astype(np.float32).astype(np.float64)
    ref = orc.mode_product(X32, F.T, 1)
    Y = native.mode_product(Xd, torch.tensor(F, dtype=torch.float32, device="cuda"), 1,
                            precision="fp32")
    got = Y.double().cpu().numpy()
    _close(got, ref, 1e-5)
    # per slice too: the slices differ in magnitude by up to 2^12
    for i in range(dims[0]):
        _close(got[i], ref[i], 1e-5)


@pytest.mark.parametrize("dims,Q", [((37, 29, 23), 5), ((200, 150, 130), 20), ((256, 256, 256), 32),
                                    ((70, 45, 600), 64), ((129, 3, 64), 17)])
def test_mode_product_tensor_cores(dims, Q):
    rng = np.random.default_rng(11 + Q)
    # Slices of very different magnitude exercise the per-slice scales.
    X = rng.random(dims) * np.exp2(rng.integers(-6, 7, size=(dims[0], 1, 1)))
    Xb = _bf16_round(X)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    for mode in (0, 2):
        F = rng.random((dims[mode], Q))
        ref = orc.mode_product(Xb, _bf16_round(F).T, mode)
        Y = native.mode_product(Xd, torch.tensor(F, dtype=torch.float32, device="cuda"), mode,
                                precision="bf16")
        _close(Y.double().cpu().numpy(), ref, 1e-5)


def test_mode_product_tensor_cores_rejects_middle_mode():
    X = torch.rand(8, 8, 8, device="cuda")
    F = torch.rand(8, 4, device="cuda")
    with pytest.raises(native.NncError) as ei:
        native.mode_product(X, F, 1, precision="bf16")
    assert ei.value.status == -6


@pytest.mark.parametrize("dims,m,iters,refine", [((96, 80, 128), (8, 10, 12), 60, 10),
                                                 ((150, 64, 200), (16, 12, 20), 40, 0),
                                                 ((96, 128, 128), (8, 10, 12), 60, 10),
                                                 # every update, H and core kernel on the
                                                 # tensor cores, odd row counts, ragged
                                                 # contraction lengths
                                                 ((151, 72, 99), (12, 16, 28), 40, 5)])
def test_ntd_bf16_refine_parity(dims, m, iters, refine):
    X, _, F0, G0, _ = inputs.small_problem(dims, 6, m, 4, seed=606, dist="exponential")
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    F = [torch.tensor(f, dtype=torch.float32, device="cuda") for f in F0]
    G = torch.tensor(G0, dtype=torch.float32, device="cuda")
    err, tr = native.ntd_fit(Xd, F, G, iters, precision="bf16", refine_iters=refine)
    Fo, Go, tro = orc.ntd_fit(X, F0, G0, iters)
    tr = tr.cpu().numpy()
    assert np.max(np.abs(tr - tro)) <= 1e-3
    assert abs(err - orc.rel_err_tucker(X, Go, Fo)) <= 1e-3
    assert all((f >= 0).all() for f in F) and (G >= 0).all()


def test_ntd_bf16_full_size_cp16_512cube():
    # The 512^3 precision workload at full size in the benchmark's launch
    # configuration; the oracle runs its first 4 sweeps.
    w = inputs.WORKLOADS["cp16_512x512x512_m32_bf16"]
    X, _, F0, G0, _ = inputs.make_problem(w)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    F = [torch.tensor(f, dtype=torch.float32, device="cuda") for f in F0]
    G = torch.tensor(G0, dtype=torch.float32, device="cuda")
    _, tr = native.ntd_fit(Xd, F, G, 4, precision="bf16", refine_iters=0, rel_err=False)
    _, _, tro = orc.ntd_fit(X, F0, G0, 4)
    assert np.max(np.abs(tr.cpu().numpy() - tro)) <= 1e-3


@pytest.mark.parametrize("dims,m", [((64, 48, 80), (8, 6, 12)), ((40, 128, 36), (6, 9, 5))])
def test_ntd_fp32_tensor_cores_match_simt(dims, m):
    # NNC_FP32 (TF32x3 passes) and NNC_FP32_SIMT agree to FP32 rounding (N2 = 128:
    # the pass also forms the mode-1 contraction).
    X, _, F0, G0, _ = inputs.small_problem(dims, 5, m, 4, seed=808, noise=0.02)
    out = {}
    for prec in ("fp32", "fp32_simt"):
        Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
        F = [torch.tensor(f, dtype=torch.float32, device="cuda") for f in F0]
        G = torch.tensor(G0, dtype=torch.float32, device="cuda")
        err, tr = native.ntd_fit(Xd, F, G, 30, precision=prec)
        out[prec] = (err, tr.cpu().numpy())
    assert np.max(np.abs(out["fp32"][1] - out["fp32_simt"][1])) <= 5e-6
    _, _, tro = orc.ntd_fit(X, F0, G0, 30)
    assert np.max(np.abs(out["fp32"][1] - tro)) <= 1e-5


def test_pass_profiler_samples_and_changes_nothing():
    # The profiler times the passes of every 16th sweep through an instrumented
    # copy of the sweep graph; the fit it measures must come out bit-identical.
    X, _, F0, G0, _ = inputs.small_problem((64, 48, 80), 5, (8, 6, 12), 4, seed=909)
    runs = {}
    for on in (False, True):
        Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
        F = [torch.tensor(f, dtype=torch.float32, device="cuda") for f in F0]
        G = torch.tensor(G0, dtype=torch.float32, device="cuda")
        native.nnc_profile_enable(on)
        try:
            _, tr = native.ntd_fit(Xd, F, G, 40, precision="fp32")
            prof = {k: native.nnc_profile_read(k) for k in native.PASS_KINDS}
        finally:
            native.nnc_profile_enable(False)
        runs[on] = (tr.cpu().numpy(), [f.cpu().numpy() for f in F], G.cpu().numpy(), prof)
    assert np.array_equal(runs[False][0], runs[True][0])
    assert all(np.array_equal(a, b) for a, b in zip(runs[False][1], runs[True][1]))
    assert np.array_equal(runs[False][2], runs[True][2])
    prof = runs[True][3]
    assert prof[4][0] == 2 and prof[5][0] == 2  # sweeps 16 and 32 of 40
    assert prof[4][1] > 0 and prof[5][1] > 0
    assert all(prof[k][0] == 0 for k in (0, 1, 2, 3))
    assert all(v[0] == 0 for v in runs[False][3].values())
