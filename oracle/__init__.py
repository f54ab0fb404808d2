"""FP64 CPU oracle of nnCANDELINC (arXiv 1909.07570, Alg. 1).

TEST INFRASTRUCTURE, NOT THE PRODUCT. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import, call or run anything in this package. The CUDA library neither imports
it nor shares code with it; the only thing both sides take in is the seeded
synthetic input, which comes from ``paper_1909_07570_gb300.inputs``.

Every function is plain numpy in float64 and cites the definition, equation or
algorithm of the paper it follows. Parity pins: every function here is pinned by
a ``-m "not gpu"`` test in ``tests/test_oracle_pins.py`` (worked examples of the
paper, brute force, finite differences, fixed points, invariants).
"""
from .tensor_algebra import (  # noqa: F401
    cp_reconstruct,
    fold,
    frobenius,
    khatri_rao,
    mode_product,
    superdiagonal,
    tucker_reconstruct,
    unfold,
)
from .nncandelinc import (  # noqa: F401
    DEFAULT_EPS,
    alg2_fit,
    congruence_matrix,
    lift,
    POWER_ITERS,
    lifted_block_terms,
    lifted_loss,
    lifted_loss_grad,
    lifted_pg_fit,
    lifted_pg_step,
    mean_congruence,
    mu_step,
    nncp_fit,
    nncp_sweep,
    nncp_terms,
    ntd_core_terms,
    ntd_factor_terms,
    ntd_fit,
    nmf_fit,
    nmf_terms,
    ntd_sweep,
    power_iteration_lmax,
    rel_err_cp,
    rel_err_tucker,
    residual_sq_identity,
)
