"""Comparison helpers of the GPU parity tests.

Every check looks at each right-hand side twice: as a relative 2-norm error, and element
by element, as the largest absolute error over the largest entry of the expected vector.
A mistake confined to a few DOFs (the rows of one small boundary subdomain, one overlap
sum in the scatter) moves the 2-norm of a large vector very little but shows at once in
the element-wise figure."""
import numpy as np

# Bound for a preconditioner apply of the mixed form against the oracle's FP64 apply. The c64
# local factors come from the tensor-core LU, whose three-TF32 products carry a relative error
# of about 2.5 * 2^-21 (1.2e-6) each (FP32 multiply-adds: 2^-24); the solves carry that times
# the condition numbers of the local matrices (tens at the test sizes). Measured worst case
# 1.7e-5 element-wise (the per-step FP32 CUDA-core LU: 5.5e-6); 6e-5 leaves a margin of 3.5.
MIXED_APPLY_TOL = 6e-5
# Tensor-core local solves: the factors enter the MMA rounded to TF32 (unit roundoff 2^-12);
# measured worst case 1.8 units, bound 4 units.
TF32_SOLVE_TOL = 4 * 2.0 ** -12
# Load vector of the mixed form, which forms the quadrature moments in double-float arithmetic:
# each of the 27 products per moment carries about 3 * 2^-46 relative error, a moment about
# 2^-43, and an entry sums at most 6 tetrahedra x 3 bumps x 2 products of a moment with
# p_b . g_k: 36 * 2^-43 = 4.1e-12 of the largest such product, itself below max |f|.
LOAD_DF_TOL = 4.1e-12


def rel_errors(got, want):
    """(per-row relative 2-norm errors, per-row max |got - want| / max |want|) of [R, n]
    arrays (a 1-D vector is one row)."""
    g = np.atleast_2d(np.asarray(got))
    w = np.atleast_2d(np.asarray(want))
    assert g.shape == w.shape, (g.shape, w.shape)
    d = g - w
    wn = np.linalg.norm(w, axis=1)
    wi = np.abs(w).max(axis=1)
    norm = np.linalg.norm(d, axis=1) / np.where(wn > 0, wn, 1.0)
    elem = np.abs(d).max(axis=1) / np.where(wi > 0, wi, 1.0)
    return norm, elem


def assert_close(got, want, tol, elem_tol=None, what=""):
    """Both per-row figures of rel_errors at most tol (the element-wise one at most
    elem_tol, default tol); every value finite."""
    assert np.isfinite(np.asarray(got)).all(), f"{what}: non-finite values"
    norm, elem = rel_errors(got, want)
    et = tol if elem_tol is None else elem_tol
    print(f"{what}: max relative 2-norm error {norm.max():.3e} (bound {tol:.1e}), "
          f"max element-wise error / max|want| {elem.max():.3e} (bound {et:.1e})")
    assert norm.max() <= tol, (what, norm)
    assert elem.max() <= et, (what, elem)
    return norm, elem


def nopivot_growth(A):
    """max|U| / max|A| of the LU factorisation without pivoting of a dense matrix (right-looking
    elimination, written out): the quantity the library's growth monitor reports."""
    U = np.array(A, dtype=np.complex128)
    n = U.shape[0]
    for k in range(n - 1):
        l = U[k + 1:, k] / U[k, k]
        U[k + 1:, k + 1:] -= np.outer(l, U[k, k + 1:])
    return np.abs(np.triu(U)).max() / np.abs(A).max()
