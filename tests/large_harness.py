"""Oracle products for workloads whose factors do not fit in host memory.

TEST INFRASTRUCTURE.  The large mixed workload (n_occ=150, n_vir=1350,
n_aux=6000, ris n_aux=1350) has 108 GB of FP64 factors over all orbitals, so
neither the tests nor the oracle ever hold them at once.  ``synth.chunked``
draws P-chunks of the factors in worker processes (and fills device tensors
with them); here each worker also evaluates the oracle's FP64 partial
products of given test vectors over its rows.  The Coulomb and exchange terms
of Eq. hessian are sums over P, so the parent adds the slices up
(``oracle.operators.pair_from_parts``).
"""
from __future__ import annotations

import numpy as np

from synth import chunked
from synth.chunked import CHUNK, load_ris  # noqa: F401  (re-exported for the tests)

VBLOCK = 16


def oracle_parts(oo, ov, vv, X):
    """The oracle's J, K1, K2 of the vectors X [m][ov] over one chunk of rows;
    vectors in blocks of VBLOCK keep a worker's intermediates near 2 GB."""
    from oracle import operators as O
    out = [np.zeros_like(X) for _ in range(3)]
    for v0 in range(0, X.shape[0], VBLOCK):
        Xb = X[v0:v0 + VBLOCK]
        out[0][v0:v0 + VBLOCK] = O.coulomb(ov, Xb)
        out[1][v0:v0 + VBLOCK] = O.exchange_K1(oo, vv, Xb)
        out[2][v0:v0 + VBLOCK] = O.exchange_K2(ov, Xb)
    return tuple(out)


def load_exact(name, meta, dev=None, X=None, workers=None):
    """Fill the device tensors dev = (L_oo, L_ov, L_vv) (FP32, [n_aux][p][q]) and/or
    return the oracle's summed (J, K1, K2) of the FP64 test vectors X [m][ov],
    in one pass over the rows."""
    hook = oracle_parts if X is not None else None
    res = chunked.load_exact(name, meta, dev, hook=hook, hook_args=(X,) if X is not None else (),
                             workers=workers)
    if X is None:
        return None
    J = K1 = K2 = None
    for _, _, (j, k1, k2) in res:
        J = j if J is None else J + j
        K1 = k1 if K1 is None else K1 + k1
        K2 = k2 if K2 is None else K2 + k2
    return J, K1, K2
