"""nnCANDELINC on GB300: nonnegative Tucker compression, nonnegative CP of the
core and the lift A^(i) = F^(i) B^(i) (arXiv 1909.07570, Alg. 1), computed by
hand-written CUDA kernels for sm_103a behind a C ABI.

The native library is loaded on first use by :mod:`.native`; importing the
package itself needs no GPU.
"""
__all__ = ["inputs", "native"]
