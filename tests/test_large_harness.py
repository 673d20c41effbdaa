"""The chunked loader of tests/large_harness.py on the small workload: the
factor blocks it writes and the oracle partial products it sums must equal
make_config's arrays and the oracle's whole-array products (Eq. hessian is a
sum over P, so the P-chunks add up to rounding)."""
import numpy as np
import pytest

from oracle import operators as O
from synth.generator import config_meta, make_config
from tests import large_harness as H


def test_chunked_loader_matches_whole_arrays():
    torch = pytest.importorskip("torch")
    name = "tda_small"
    p = make_config(name)
    meta = config_meta(name)
    no, nv, na = p.n_occ, p.n_vir, p.n_aux
    dev = (torch.zeros(na, no, no), torch.zeros(na, no, nv), torch.zeros(na, nv, nv))
    X = np.random.default_rng(5).standard_normal((2, p.n_ov))
    J, K1, K2 = H.load_exact(name, meta, dev, X, workers=2)
    for t, ref in zip(dev, (p.L_oo, p.L_ov, p.L_vv)):
        assert np.array_equal(t.numpy(), ref.astype(np.float32))
    d = O.delta(p.eps_occ, p.eps_vir)
    apb, amb = O.pair_from_parts(d, X, J, K1, K2, p.a_x, p.coulomb_factor)
    rp, rm = O.exact_operator(p).apb_amb(X)
    assert np.max(np.abs(apb - rp)) < 1e-12 * np.max(np.abs(rp))
    assert np.max(np.abs(amb - rm)) < 1e-12 * np.max(np.abs(rm))
    k = p.ris_K_index
    rdev = (torch.zeros(k.size, no, no), torch.zeros(p.n_ris, no, nv), torch.zeros(k.size, nv, nv))
    H.load_ris(name, meta, rdev, workers=2)
    assert np.array_equal(rdev[0].numpy(), p.Lr_oo[k].astype(np.float32))
    assert np.array_equal(rdev[1].numpy(), p.Lr_ov.astype(np.float32))
    assert np.array_equal(rdev[2].numpy(), p.Lr_vv[k].astype(np.float32))
