"""Response operators of ab initio TDDFT and of the ris model (oracle, FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definitions followed
  * Eq. hessian (Sec. 2.2.1): (A+B)_ia,jb = Delta_ia d_ij d_ab + 2 f^xc + 2(ia|jb)
    - c_x[(ib|ja) + (ij|ab)] and (A-B)_ia,jb = Delta d d + c_x[(ib|ja) - (ij|ab)],
    with Delta_ia = eps_a - eps_i.  f^xc is zero because the integrals are given,
    not generated (the ris model neglects it too, Sec. 2.2.2).
  * Eq. pqrs: (pq|rs) is a four-index Coulomb integral; with density fitting it
    is sum_P L^P_pq L^P_rs (Eq. pqrs_approx with the metric folded into L).
  * Coulomb prefactor: the printed Eq. hessian has 2(ia|jb) in A+B; the
    restricted-singlet convention has 2(ia|jb) in A and in B separately.  The
    prefactor is a parameter c_J of A and B:
        A = Delta + c_J (ia|jb) - a_x (ij|ab),    B = c_J (ia|jb) - a_x (ib|ja),
    so c_J = 1 is the equation as printed and c_J = 2 the singlet convention
    (default).  Both sides always take the same c_J.
  * Eq. TDDFT-ris_approx and Sec. 3.1-3.2: the ris operator uses its own
    minimal auxiliary factors; the Coulomb part uses all of them (s, p, d per
    atom), the exchange part only the s rows, and exchange integrals drop
    virtual orbitals with eps_a > eps_HOMO + t_cut and occupied orbitals with
    eps_i < eps_LUMO - t_cut (t_cut = 40 eV).  Coulomb is not truncated.

Two independent routes are given for every operator: a dense builder that
takes the four-index integral tensor over all orbitals and reads the Hessian
elements off it by orbital index (small sizes only), and a matrix-free
product over the three-index blocks (any size).  Tests pin each against the
other and against closed forms.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# Orbital-energy differences (Eq. hessian, first term)

def delta(eps_occ: np.ndarray, eps_vir: np.ndarray) -> np.ndarray:
    """Delta_ia = eps_a - eps_i, flattened with a fastest: index ia = i*n_vir + a."""
    return (eps_vir[None, :] - eps_occ[:, None]).reshape(-1)


# ----------------------------------------------------------------------------
# Dense route: four-index integrals by orbital index (small problems only)

def eri_from_factors(L_full: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum_P L^P_pq L^P_rs over all orbitals (Eq. pqrs with density fitting)."""
    n = L_full.shape[1]
    flat = L_full.reshape(L_full.shape[0], n * n)
    return (flat.T @ flat).reshape(n, n, n, n)


def dense_A_B(eps_occ, eps_vir, eri, a_x, c_J, eri_lr=None, b_x=0.0, F_full=None, w=None):
    """A and B of Eq. hessian read element by element from (pq|rs).

    Orbitals are ordered occupied first, so virtual a is orbital n_occ + a.
    Optional terms (variants of Eq. hessian for other functionals):
      * eri_lr, b_x: a second exchange integral set, as the long-range
        (erf-attenuated) exchange of a range-separated hybrid:
        A -= b_x (ij|ab)_LR, B -= b_x (ib|ja)_LR;
      * F_full [n_g][n_mo][n_mo], w [n_g]: a low-rank response kernel standing
        in for f^xc, (pq|f|rs) = sum_g w_g F^g_pq F^g_rs, entering A and B with
        the Coulomb prefactor: A += c_J (ia|f|jb), B += c_J (ia|f|jb).
    Without them f^xc = 0.
    """
    no, nv = eps_occ.size, eps_vir.size
    occ = np.arange(no)
    vir = no + np.arange(nv)
    ov = no * nv

    def blocks(e):
        # (ia|jb), (ij|ab), (ib|ja) as [ia][jb] matrices
        ia_jb = e[np.ix_(occ, vir, occ, vir)]
        ij_ab = e[np.ix_(occ, occ, vir, vir)].transpose(0, 2, 1, 3)
        ib_ja = e[np.ix_(occ, vir, occ, vir)].transpose(0, 3, 2, 1)
        return ia_jb.reshape(ov, ov), ij_ab.reshape(ov, ov), ib_ja.reshape(ov, ov)

    ia_jb, ij_ab, ib_ja = blocks(eri)
    A = c_J * ia_jb - a_x * ij_ab
    B = c_J * ia_jb - a_x * ib_ja
    if eri_lr is not None:
        _, ij_ab_lr, ib_ja_lr = blocks(eri_lr)
        A -= b_x * ij_ab_lr
        B -= b_x * ib_ja_lr
    if F_full is not None:
        n = F_full.shape[1]
        flat = F_full.reshape(F_full.shape[0], n * n)
        fker = (flat.T @ (np.asarray(w)[:, None] * flat)).reshape(n, n, n, n)
        f_ia_jb = blocks(fker)[0]
        A += c_J * f_ia_jb
        B += c_J * f_ia_jb
    A[np.diag_indices(ov)] += delta(eps_occ, eps_vir)
    return A, B


def dense_A_B_blocks(prob):
    """A and B of Eq. hessian (f^xc = 0) built densely from the three-index
    blocks, for problems too large for the four-index route of dense_A_B:
    (ia|jb) = sum_P L^P_ia L^P_jb, (ij|ab) = sum_P L^P_ij L^P_ab and
    (ib|ja) = sum_P L^P_ib L^P_ja, each as an [ia][jb] matrix (Eq. pqrs_approx)."""
    no, nv, na = prob.n_occ, prob.n_vir, prob.n_aux
    ov = no * nv
    Lov = prob.L_ov.reshape(na, ov)
    ia_jb = Lov.T @ Lov
    ij_ab = np.einsum("pij,pab->iajb", prob.L_oo, prob.L_vv, optimize=True).reshape(ov, ov)
    ib_ja = np.einsum("pib,pja->iajb", prob.L_ov, prob.L_ov, optimize=True).reshape(ov, ov)
    A = prob.coulomb_factor * ia_jb - prob.a_x * ij_ab
    B = prob.coulomb_factor * ia_jb - prob.a_x * ib_ja
    A[np.diag_indices(ov)] += delta(prob.eps_occ, prob.eps_vir)
    return A, B


def window(eps_occ, eps_vir, t_cut):
    """Exchange energy window of Sec. 3.1: keep occupied eps_i >= eps_LUMO - t_cut
    and virtual eps_a <= eps_HOMO + t_cut (the others are dropped)."""
    keep_o = eps_occ >= eps_vir[0] - t_cut
    keep_v = eps_vir <= eps_occ[-1] + t_cut
    return keep_o, keep_v


def dense_ris_A_B(prob, t_cut=None):
    """A and B of the ris model (Eq. TDDFT-ris_approx, rid structure of Sec. 3.2)
    from four-index integrals of its own factors, by orbital index.

    Coulomb-type integrals use every ris row; exchange-type integrals use the
    s rows listed in ``ris_K_index`` and only orbitals inside the window.
    """
    Lr = prob.extra["Lr_full"]
    eri_J = eri_from_factors(Lr)
    eri_K = eri_from_factors(Lr[prob.ris_K_index])
    t = prob.t_cut_ha if t_cut is None else t_cut
    ko, kv = window(prob.eps_occ, prob.eps_vir, t)
    no, nv = prob.n_occ, prob.n_vir
    mask_o = ko.astype(float)
    mask_v = kv.astype(float)
    # zero every exchange integral that touches a dropped orbital
    m = np.concatenate([mask_o, mask_v])
    eri_K = eri_K * m[:, None, None, None] * m[None, :, None, None] * m[None, None, :, None] * m[None, None, None, :]
    AJ, BJ = dense_A_B(prob.eps_occ, prob.eps_vir, eri_J, 0.0, prob.coulomb_factor)
    AK, BK = dense_A_B(prob.eps_occ, prob.eps_vir, eri_K, prob.a_x, 0.0)
    d = np.diag_indices(no * nv)
    AK[d] -= delta(prob.eps_occ, prob.eps_vir)
    return AJ + AK, BJ + BK


# ----------------------------------------------------------------------------
# Matrix-free route over the three-index blocks (Coulomb J, exchange K1, K2)

def _chunks(n, size):
    for p0 in range(0, n, size):
        yield p0, min(n, p0 + size)


def coulomb(L_ov, X, chunk=256, w=None):
    """J(X)_ia = sum_jb (ia|jb) X_jb = sum_P L^P_ia sum_jb L^P_jb X_jb.  X: [m][ov].
    With weights w [n_aux]: sum_P w_P L^P_ia sum_jb L^P_jb X_jb (the low-rank
    kernel term (ia|f|jb) of dense_A_B)."""
    n_aux = L_ov.shape[0]
    flat = L_ov.reshape(n_aux, -1)
    out = np.zeros_like(X)
    for p0, p1 in _chunks(n_aux, chunk):
        t = flat[p0:p1] @ X.T            # [P][m]
        if w is not None:
            t = np.asarray(w)[p0:p1, None] * t
        out += t.T @ flat[p0:p1]
    return out


def exchange_K1(L_oo, L_vv, X, chunk=64):
    """K1(X)_ib = sum_ja (ij|ab) X_ja = sum_P sum_j L^P_ij sum_a X_ja L^P_ab."""
    n_aux, no, _ = L_oo.shape
    nv = L_vv.shape[1]
    m = X.shape[0]
    X3 = X.reshape(m, no, nv)
    out = np.zeros((m, no, nv))
    for p0, p1 in _chunks(n_aux, chunk):
        # Z^P_(n,i,a) = sum_j L^P_ij X_(n,j,a)
        Z = np.einsum("pij,nja->npia", L_oo[p0:p1], X3, optimize=True)
        # sum over P and a of Z^P_(n,i,a) L^P_ab
        Zr = Z.transpose(0, 2, 1, 3).reshape(m * no, (p1 - p0) * nv)
        out += (Zr @ L_vv[p0:p1].reshape((p1 - p0) * nv, nv)).reshape(m, no, nv)
    return out.reshape(m, no * nv)


def exchange_K2(L_ov, X, chunk=64):
    """K2(X)_ia = sum_jb (ib|ja) X_jb = sum_P sum_j (sum_b L^P_ib X_jb) L^P_ja."""
    n_aux, no, nv = L_ov.shape
    m = X.shape[0]
    X3 = X.reshape(m, no, nv)
    out = np.zeros((m, no, nv))
    for p0, p1 in _chunks(n_aux, chunk):
        Lc = L_ov[p0:p1]
        Q = np.einsum("pib,njb->npij", Lc, X3, optimize=True)
        out += np.einsum("npij,pja->nia", Q, Lc, optimize=True)
    return out.reshape(m, no * nv)


class Operator:
    """Matrix-free A, A+B and A-B over density-fitted factors.

    ``Lx_oo``/``Lx_vv``/``Lx_ov`` are the exchange factor blocks (possibly
    window-restricted, zero outside the window), ``Lj_ov`` the Coulomb block.
    Optional variant terms (see dense_A_B): ``lr`` = (M_oo, M_ov, M_vv, b_x), a
    second exchange factor set with its own weight; ``kernel`` = (F_ov, w), the
    low-rank response kernel, added to the Coulomb term.
    """

    def __init__(self, eps_occ, eps_vir, Lj_ov, Lx_oo, Lx_ov, Lx_vv, a_x, c_J, lr=None, kernel=None):
        self.d = delta(eps_occ, eps_vir)
        self.Lj_ov, self.Lx_oo, self.Lx_ov, self.Lx_vv = Lj_ov, Lx_oo, Lx_ov, Lx_vv
        self.a_x, self.c_J = a_x, c_J
        self.lr, self.kernel = lr, kernel
        self.n_occ, self.n_vir = eps_occ.size, eps_vir.size

    def _parts(self, X, need_k2):
        """X, J and the exchange parts K1, K2 with their weight already applied
        (a_x K[L] + b_x K[M]), so the caller uses exchange weight 1."""
        X = np.atleast_2d(X)
        J = coulomb(self.Lj_ov, X)
        if self.kernel is not None:
            J = J + coulomb(self.kernel[0], X, w=self.kernel[1])
        K1 = self.a_x * exchange_K1(self.Lx_oo, self.Lx_vv, X) if self.a_x != 0.0 else np.zeros_like(X)
        K2 = self.a_x * exchange_K2(self.Lx_ov, X) if (need_k2 and self.a_x != 0.0) else np.zeros_like(X)
        if self.lr is not None and self.lr[3] != 0.0:
            M_oo, M_ov, M_vv, b_x = self.lr
            K1 = K1 + b_x * exchange_K1(M_oo, M_vv, X)
            if need_k2:
                K2 = K2 + b_x * exchange_K2(M_ov, X)
        return X, J, K1, K2

    def tda(self, X):
        """A X with A = Delta + c_J (ia|jb) - a_x (ij|ab)  (Eq. TDA uses A alone)."""
        X, J, K1, _ = self._parts(X, False)
        return tda_from_parts(self.d, X, J, K1, 1.0, self.c_J)

    def apb_amb(self, X):
        """((A+B) X, (A-B) X) from Eq. hessian (f^xc = 0 unless a kernel term is given)."""
        X, J, K1, K2 = self._parts(X, True)
        return pair_from_parts(self.d, X, J, K1, K2, 1.0, self.c_J)


def tda_from_parts(d, X, J, K1, a_x, c_J):
    """A X = Delta X + c_J J(X) - a_x K1(X)  (Eq. hessian, A alone)."""
    return d * X + c_J * J - a_x * K1


def pair_from_parts(d, X, J, K1, K2, a_x, c_J):
    """(A+B) X = Delta X + 2 c_J J - a_x (K1 + K2),  (A-B) X = Delta X + a_x (K2 - K1)
    (Eq. hessian with f^xc = 0).  J, K1, K2 may be sums of P-slices: every term is
    linear in the factors' outer products, so slices of P add up."""
    apb = d * X + 2.0 * c_J * J - a_x * (K1 + K2)
    amb = d * X + a_x * (K2 - K1)
    return apb, amb


def exact_operator(prob) -> Operator:
    """The ab initio (RI) operator from the exact factors, with the problem's
    optional second exchange set (``extra["exchange_lr"]``: M_oo, M_ov, M_vv,
    b_x) and low-rank kernel (``extra["kernel"]``: F_ov, w)."""
    ex = prob.extra or {}
    lr = ex.get("exchange_lr")
    ker = ex.get("kernel")
    return Operator(prob.eps_occ, prob.eps_vir, prob.L_ov, prob.L_oo, prob.L_ov, prob.L_vv,
                    prob.a_x, prob.coulomb_factor,
                    lr=(lr["M_oo"], lr["M_ov"], lr["M_vv"], lr["b_x"]) if lr else None,
                    kernel=(ker["F_ov"], ker["w"]) if ker else None)


def dense_exact_A_B(prob):
    """A and B of the exact operator from four-index tensors (small problems),
    with the problem's optional variant terms."""
    ex = prob.extra or {}
    lr = ex.get("exchange_lr")
    ker = ex.get("kernel")
    return dense_A_B(prob.eps_occ, prob.eps_vir, eri_from_factors(ex["L_full"]), prob.a_x,
                     prob.coulomb_factor,
                     eri_lr=eri_from_factors(lr["M_full"]) if lr else None, b_x=lr["b_x"] if lr else 0.0,
                     F_full=ker["F_full"] if ker else None, w=ker["w"] if ker else None)


def ris_operator(prob, t_cut=None, K_index=None) -> Operator:
    """The ris preconditioner operator T (Sec. 2.2.2, rid = (d, s) of Sec. 3.2).

    Coulomb from every ris row; exchange from the s rows only, with the
    occupied and virtual orbitals outside the t_cut window zeroed (Sec. 3.1).
    """
    t = prob.t_cut_ha if t_cut is None else t_cut
    ko, kv = window(prob.eps_occ, prob.eps_vir, t)
    idx = prob.ris_K_index if K_index is None else K_index
    Koo = prob.Lr_oo[idx] * ko[None, :, None] * ko[None, None, :]
    Kvv = prob.Lr_vv[idx] * kv[None, :, None] * kv[None, None, :]
    Kov = prob.Lr_ov[idx] * ko[None, :, None] * kv[None, None, :]
    return Operator(prob.eps_occ, prob.eps_vir, prob.Lr_ov, Koo, Kov, Kvv,
                    prob.a_x, prob.coulomb_factor)
