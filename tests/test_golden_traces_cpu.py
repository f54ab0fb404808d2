"""The stored FP64 oracle traces (tests/golden/, written by
tests/golden/make_traces.py) against what the mathematics fixes, on the CPU:
every multiplicative-update trace is non-increasing, the final explicit error
equals the last identity entry, and the first sweeps of the 256^3 trace are
reproduced by the oracle as it stands."""
import os

import numpy as np
import pytest

import oracle as orc
from _golden import HERE, load
from paper_1909_07570_gb300 import inputs

NAMES = ["ntd_cp10_256cube_500", "ntd_cp16_512cube_200", "ntd_cp16_512cube_5000",
         "ntd4_cp12_128x128x128x64_300", "pg_cp12_128x128x128x64_300", "batch64_subset"]


def _load(name):
    if not os.path.exists(os.path.join(HERE, name + ".txt")):
        pytest.skip(f"{name} not written")
    return load(name + ".txt")


@pytest.mark.parametrize("name", NAMES)
def test_stored_traces_are_monotone(name):
    g = _load(name)
    for key, v in g.items():
        if key == "shape" or v.size < 2:
            continue
        assert np.all(np.diff(v) <= 1e-12 * v[:-1]), key


@pytest.mark.parametrize("name", ["ntd_cp10_256cube_500", "ntd_cp16_512cube_200",
                                  "ntd_cp16_512cube_5000", "ntd4_cp12_128x128x128x64_300"])
def test_final_explicit_error_equals_last_identity_entry(name):
    g = _load(name)
    assert abs(g["final_rel_err"][0] - g["trace"][-1]) <= 1e-9


def test_batch_subset_finals_equal_last_trace_entries():
    g = _load("batch64_subset")
    for b in (0, 1):
        assert abs(g[f"t{b}_final_rel_err"][0] - g[f"t{b}_trace"][-1]) <= 1e-9


def test_first_sweeps_reproduced_by_the_oracle():
    g = _load("ntd_cp10_256cube_500")
    w = inputs.WORKLOADS["cp10_256x256x256_m20_fp32"]
    X, _, F0, G0, _ = inputs.make_problem(w)
    X = np.asarray(X, dtype=np.float32).astype(np.float64)
    _, _, tr = orc.ntd_fit(X, F0, G0, 2)
    np.testing.assert_allclose(tr, g["trace"][:2], rtol=1e-12)
