"""Shared comparison rules of the GPU parity tests (test infrastructure).

Excitation energies are compared in Hartree (1e-6 Ha for the plain FP64 form,
1e-5 Ha for the mixed form).  Polarizabilities are compared element by
element:

    |alpha - alpha_ref| <= rtol * max(|alpha_ref|, FLOOR * max |alpha_ref|)

with rtol = 1e-6 (plain) or 1e-5 (mixed) and FLOOR = 0.05 (FP64 and FP32
products) or FLOOR_TC = 0.25 (BF16 hi+lo tensor-core products): every element
at least FLOOR of the largest one is held to rtol relative to itself, a
smaller one to rtol relative to FLOOR of the largest.  The bound never exceeds
rtol * max|alpha_ref| (a test relative to the whole tensor) and is tighter for
every element below the largest.  The floor exists because of the products'
own rounding: the Galerkin error of alpha_vu = mu_v . (X_u + Y_u) is second
order in the residuals (all systems share one subspace), but a relative
rounding of the products (about 1e-7 for FP32, 1e-5 for the BF16 hi+lo
tensor-core form) perturbs every element on the scale of the diagonal.  The
tensor-core products' rounding is as large as the mixed tolerance itself: on
a 21-dimensional problem an off-diagonal element 4.6 % of the largest came out
with a 2e-5 relative error (5e-7 absolute, 1e-6 of the tensor's scale).
"""
import numpy as np

FLOOR = 0.05
FLOOR_TC = 0.25


def alpha_excess(alpha, ref, rtol, floor=FLOOR):
    """Largest |alpha - ref| / (rtol max(|ref|, floor max|ref|)); <= 1 passes."""
    alpha, ref = np.asarray(alpha, dtype=float), np.asarray(ref, dtype=float)
    bound = rtol * np.maximum(np.abs(ref), floor * np.max(np.abs(ref)))
    return float(np.max(np.abs(alpha - ref) / bound))


def alpha_report(alpha, ref):
    """(largest absolute error, largest per-element relative error)."""
    alpha, ref = np.asarray(alpha, dtype=float), np.asarray(ref, dtype=float)
    err = np.abs(alpha - ref)
    return float(err.max()), float(np.max(err / np.maximum(np.abs(ref), 1e-300)))
