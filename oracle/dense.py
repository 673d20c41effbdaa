"""Plain-definition results on small inputs (oracle, FP64, CPU, LAPACK).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

  * tda:    the lowest eigenpairs of A (Eq. TDA), by ``numpy.linalg.eigh``.
  * casida: the lowest positive Omega of Eq. Casida.  With A-B positive
            definite, Omega^2 are the eigenvalues of the symmetric matrix
            (A-B)^(1/2) (A+B) (A-B)^(1/2); X+Y and X-Y follow from its
            eigenvectors, normalised so that X^T X - Y^T Y = 1.
  * polar:  alpha_vu(omega) of Eq. TDDFT_polar as the linear solve
            [(A B; B A) - omega diag(1,-1)] (X; Y) = (mu_u; mu_u),
            alpha_vu = mu_v^T X + mu_v^T Y (real orbitals, mu_vo = mu_ov).
"""
from __future__ import annotations

import numpy as np


def tda(A: np.ndarray, n_states: int):
    """Lowest ``n_states`` eigenpairs of A (Eq. TDA). Returns (Omega, X[n][ov])."""
    w, v = np.linalg.eigh(A)
    return w[:n_states], v[:, :n_states].T.copy()


def _sym_sqrt(M):
    w, q = np.linalg.eigh(M)
    if w[0] <= 0.0:
        raise np.linalg.LinAlgError("matrix is not positive definite (lambda_min=%g)" % w[0])
    return (q * np.sqrt(w)) @ q.T, (q / np.sqrt(w)) @ q.T


def casida(A: np.ndarray, B: np.ndarray, n_states: int):
    """Lowest positive excitation energies of Eq. Casida by the symmetric form.

    (A+B)(X+Y) = Omega (X-Y) and (A-B)(X-Y) = Omega (X+Y), so with
    S = (A-B)^(1/2): S (A+B) S z = Omega^2 z, X+Y = S z / sqrt(Omega),
    X-Y = sqrt(Omega) S^-1 z.  Returns (Omega, X, Y) with X^T X - Y^T Y = 1.
    """
    S, Sinv = _sym_sqrt(A - B)
    H = S @ (A + B) @ S
    w2, z = np.linalg.eigh(0.5 * (H + H.T))
    if w2[0] <= 0.0:
        raise np.linalg.LinAlgError("Casida problem has non-positive Omega^2 (%g)" % w2[0])
    om = np.sqrt(w2[:n_states])
    z = z[:, :n_states]
    U = (S @ z) / np.sqrt(om)
    W = (Sinv @ z) * np.sqrt(om)
    X = 0.5 * (U + W)
    Y = 0.5 * (U - W)
    return om, X.T.copy(), Y.T.copy()


def polar(A: np.ndarray, B: np.ndarray, mu: np.ndarray, omegas):
    """alpha[f][v][u] = (mu_v; mu_v)^T [(A B; B A) - w_f diag(1,-1)]^-1 (mu_u; mu_u)."""
    ov = A.shape[0]
    mu = np.atleast_2d(mu)
    nd = mu.shape[0]
    out = np.zeros((len(omegas), nd, nd))
    rhs = np.concatenate([mu.T, mu.T], axis=0)
    for f, w in enumerate(omegas):
        big = np.block([[A - w * np.eye(ov), B], [B, A + w * np.eye(ov)]])
        sol = np.linalg.solve(big, rhs)
        out[f] = rhs.T @ sol
    return out
