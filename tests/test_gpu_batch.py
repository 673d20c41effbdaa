"""Batched TDA solves (tddft_solve_tda_batch): many small problems advanced
together through grouped launches and a captured operator graph.

  * every problem of a batch of small molecules drawn like the batched
    workload (n_occ ~ U{8..16} here so that dense LAPACK is quick, n_vir =
    n_occ x U{4..8}, exact n_aux = 5 n_mo, ris n_aux = 9 ceil(n_occ/2),
    5-10 states, the coupling scaled by min(1, 12.5 / sqrt(n_occ n_vir)) as
    in the served and batched streams; rid and diag preconditioners mixed)
    converges, and its
    energies match the oracle's dense eigenvalues of A (Eq. TDA) within
    1e-5 Ha (the mixed tolerance: FP32 vectors and products);
  * a problem's results do not depend on what else is in the batch (every
    grouped product and reduction has a fixed order): solved alone and in the
    batch they agree to 1e-12;
  * the tile autotune timed its variants and the operator graph was replayed.
"""
import numpy as np
import pytest

from oracle import dense as D
from oracle import operators as O
from synth.generator import default_amplitude, make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2404_17133_gb300 import api as a
    return a


def _problems(n, seed=2405):
    g = np.random.Generator(np.random.Philox(key=np.array([seed, 7], dtype=np.uint64)))
    out = []
    for i in range(n):
        no = int(g.integers(8, 17))
        nv = no * int(g.integers(4, 9))
        ns = int(g.integers(5, 11))
        na = 5 * (no + nv)
        amp = default_amplitude(na) * min(1.0, 12.5 / np.sqrt(no * nv))
        p = make_problem(no, nv, na, 9 * ((no + 1) // 2), seeds=(5000 + 3 * i, 5001 + 3 * i, 5002 + 3 * i),
                         amplitude=amp)
        out.append((p, ns))
    return out


def _dense_tda(p, k):
    A, _ = O.dense_A_B_blocks(p)
    return D.tda(A, k)[0]


def test_batch_matches_dense(api):
    probs = _problems(12)
    solvers = [api.Solver.from_problem(p, precisions=2, dtype=api.F32) for p, _ in probs]
    try:
        opts = [api.default_opts(n_states=ns, precond=api.RID if i % 3 else api.DIAG, precision=api.MIXED)
                for i, (_, ns) in enumerate(probs)]
        st, res, info = api.solve_tda_batch(solvers, opts)
        assert st == api.OK, [r["stats"]["converged"] for r in res]
        print("\nbatch of %d: outer iterations %d, autotune %s -> variant %d, %d graph replays of %d nodes, "
              "%d launches, %.2f s" % (len(probs), info["outer_iterations"], info["autotune_ms"], info["variant"],
                                       info["graph_launches"], info["graph_nodes"], info["launches"],
                                       info["t_total_s"]))
        assert info["variant"] >= 0 and all(t > 0 for t in info["autotune_ms"])
        assert info["graph_launches"] >= 1
        worst = 0.0
        for (p, ns), r in zip(probs, res):
            ref = _dense_tda(p, ns)
            err = float(np.max(np.abs(r["omega"] - ref)))
            worst = max(worst, err)
            assert r["stats"]["converged"] == 1 and np.max(r["resid"]) < 1e-5
            assert err < 1e-5, (p.n_occ, p.n_vir, err)
        print("batch max |Omega - dense| = %.2e Ha" % worst)
    finally:
        for s in solvers:
            s.close()


def test_batch_result_independent_of_the_mix(api):
    probs = _problems(6, seed=77)
    solvers = [api.Solver.from_problem(p, precisions=2, dtype=api.F32) for p, _ in probs]
    try:
        opts = [api.default_opts(n_states=ns, precond=api.RID, precision=api.MIXED) for _, ns in probs]
        _, together, _ = api.solve_tda_batch(solvers, opts)
        for i in (0, 3):
            _, alone, _ = api.solve_tda_batch([solvers[i]], [opts[i]])
            assert np.max(np.abs(alone[0]["omega"] - together[i]["omega"])) <= 1e-12
        # the same context twice in one batch: its factors are only read
        _, twice, _ = api.solve_tda_batch([solvers[1], solvers[1]], [opts[1], opts[1]])
        assert np.max(np.abs(twice[0]["omega"] - twice[1]["omega"])) <= 1e-12
    finally:
        for s in solvers:
            s.close()


def test_batch_tile_variants_give_the_same_bits(api, monkeypatch):
    """Every grouped-GEMM tile variant (the autotune's choices) sums each
    element in the same K order, so forcing each one gives identical results."""
    probs = _problems(3, seed=91)
    solvers = [api.Solver.from_problem(p, precisions=2, dtype=api.F32) for p, _ in probs]
    try:
        opts = [api.default_opts(n_states=ns, precond=api.RID, precision=api.MIXED) for _, ns in probs]
        ref = None
        for v in range(5):
            monkeypatch.setenv("TDDFT_BATCH_VARIANT", str(v))
            _, res, info = api.solve_tda_batch(solvers, opts)
            assert info["variant"] == v
            om = np.concatenate([r["omega"] for r in res])
            if ref is None:
                ref = om
            assert np.array_equal(om, ref), v
    finally:
        for s in solvers:
            s.close()


def test_batch_arguments(api):
    p, ns = _problems(1)[0]
    s = api.Solver.from_problem(p, precisions=1)
    try:
        with pytest.raises(api.TddftError) as e:   # no MIXED copies
            api.solve_tda_batch([s], [api.default_opts(n_states=ns)])
        assert e.value.status == api.ERR_ARG
    finally:
        s.close()
