"""Shared comparison rules of the GPU parity tests (test infrastructure).

Excitation energies are compared in Hartree (1e-6 Ha for the plain FP64 form,
1e-5 Ha for the mixed form).  Polarizabilities are compared element by
element:

    |alpha - alpha_ref| <= rtol * |alpha_ref| + rtol * FLOOR * max |alpha_ref|

with rtol = 1e-6 (plain) or 1e-5 (mixed) and FLOOR = 1e-3: an element a
thousand times smaller than the largest one is held to an absolute error of
rtol/1000 of the tensor's scale.  The floor exists because the Galerkin error
of alpha_vu = mu_v . (X_u + Y_u) is measured against the whole tensor: all
systems share one subspace, so the error is second order in the residuals,
but the rounding of the products (about 1e-5 relative for the BF16 hi+lo
tensor-core form) perturbs every element on the scale of the diagonal.
"""
import numpy as np

FLOOR = 1e-3


def alpha_excess(alpha, ref, rtol):
    """Largest |alpha - ref| / (rtol |ref| + rtol FLOOR max|ref|); <= 1 passes."""
    alpha, ref = np.asarray(alpha, dtype=float), np.asarray(ref, dtype=float)
    bound = rtol * np.abs(ref) + rtol * FLOOR * np.max(np.abs(ref))
    return float(np.max(np.abs(alpha - ref) / bound))


def alpha_report(alpha, ref):
    """(largest absolute error, largest per-element relative error)."""
    alpha, ref = np.asarray(alpha, dtype=float), np.asarray(ref, dtype=float)
    err = np.abs(alpha - ref)
    return float(err.max()), float(np.max(err / np.maximum(np.abs(ref), 1e-300)))
