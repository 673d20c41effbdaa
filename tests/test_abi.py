"""C ABI checks that need no GPU: the library builds, loads, exports every entry
point that include/tddft.h declares, and the ctypes structures of the binding
have the C layout (sizes and field offsets compiled from the header by gcc)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tddft.h")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2404_17133_gb300 import api as a
    return a


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tddft_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tddft_create", "tddft_solve_tda", "tddft_solve_rpa", "tddft_solve_polar",
              "tddft_submit", "tddft_poll", "tddft_destroy", "tddft_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(api):
    lib = api.lib()
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert sorted(api.EXPORTED) == declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", api.LIBPATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (tddft_\w+)", out))
    assert set(declared_functions()) <= exported


def test_struct_layout_matches_header(api, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "tddft.h"
#define F(T, f) printf(#T "." #f " %zu\\n", offsetof(T, f));
int main(void) {
  printf("tddft_desc %zu\\ntddft_opts %zu\\ntddft_stats %zu\\ntddft_request %zu\\n",
         sizeof(tddft_desc), sizeof(tddft_opts), sizeof(tddft_stats), sizeof(tddft_request));
  F(tddft_desc, a_x) F(tddft_desc, precisions) F(tddft_desc, hbm_budget_gb)
  F(tddft_opts, tol) F(tddft_opts, max_iter) F(tddft_opts, outputs_on_device) F(tddft_opts, ris_fp8)
  F(tddft_stats, max_resid) F(tddft_stats, t_precond_s)
  F(tddft_request, omega) F(tddft_request, n_dip) F(tddft_request, alpha) F(tddft_request, stats)
  printf("tddft_serve_request %zu\\ntddft_server_state %zu\\n", sizeof(tddft_serve_request),
         sizeof(tddft_server_state));
  F(tddft_serve_request, desc) F(tddft_serve_request, ris_K_index) F(tddft_serve_request, kind)
  F(tddft_serve_request, req) F(tddft_serve_request, charged_bytes) F(tddft_serve_request, t_end_s)
  F(tddft_serve_request, error)
  F(tddft_server_state, active) F(tddft_server_state, completed) F(tddft_server_state, pool_high_bytes)
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True,
                                                               text=True).stdout.splitlines())
    assert int(vals["tddft_desc"]) == C.sizeof(api.Desc)
    assert int(vals["tddft_opts"]) == C.sizeof(api.Opts)
    assert int(vals["tddft_stats"]) == C.sizeof(api.Stats)
    assert int(vals["tddft_request"]) == C.sizeof(api.Request)
    assert int(vals["tddft_serve_request"]) == C.sizeof(api.ServeRequest)
    assert int(vals["tddft_server_state"]) == C.sizeof(api.ServerState)
    for key, v in vals.items():
        if "." in key:
            t, f = key.split(".")
            cls = {"tddft_desc": api.Desc, "tddft_opts": api.Opts, "tddft_stats": api.Stats,
                   "tddft_request": api.Request, "tddft_serve_request": api.ServeRequest,
                   "tddft_server_state": api.ServerState}[t]
            assert getattr(cls, f).offset == int(v), key


def test_defaults_follow_the_paper(api):
    """Sec. 3: threshold 1e-5; Sec. 3.1: inner 1e-2 / 20 iterations, guess 1e-3, t_cut 40 eV."""
    o = api.default_opts()
    assert o.tol == 1e-5 and o.inner_tol == 1e-2 and o.inner_max_iter == 20 and o.guess_tol == 1e-3
    assert o.precond == api.RID and o.n_extra_guess == -1
    d = api.Desc()
    api.lib().tddft_default_desc(C.byref(d))
    assert abs(d.t_cut_ha * 27.211386245988 - 40.0) < 1e-9
    assert d.a_x == 0.25 and d.coulomb_factor == 2.0


def test_null_arguments_are_rejected_without_gpu(api):
    """Argument checks run before any device work."""
    h = C.c_void_p()
    assert api.lib().tddft_create(None, None, None, None, None, None, None, None, None, None, 0, 0,
                                  None, C.byref(h)) == api.ERR_ARG
    assert b"null" in api.lib().tddft_last_error(None)
    assert api.lib().tddft_solve_tda(None, None, None, None, None, None) == api.ERR_ARG
    assert api.lib().tddft_poll(None, 1, 0) == api.ERR_ARG
    api.lib().tddft_destroy(None)
    assert api.lib().tddft_server_poll(None, 1, 0) == api.ERR_ARG
    assert api.lib().tddft_server_submit(None, None, None) == api.ERR_ARG
    api.lib().tddft_server_destroy(None)


def _desc(api, no, nv, na, nj, nk, precisions):
    d = api.Desc()
    api.lib().tddft_default_desc(C.byref(d))
    d.n_occ, d.n_vir, d.n_aux, d.n_aux_ris_J, d.n_aux_ris_K, d.precisions = no, nv, na, nj, nk, precisions
    return d


def test_admission_charge_counts_the_factor_copies(api):
    """The server's charge for the factor copies, against a plain count of the
    arrays tddft_create keeps: FP64 copies of L_oo, L_ov, L_vv and of the ris
    rows (PLAIN); FP32 copies plus two FP16 parts of the tensor-core copies with rows
    padded to a multiple of 8 elements (16-byte TMA strides) (MIXED: vv, ov^T per P, oo, ov, and
    the whole L_ov transposed for the Coulomb term), BF16 ris
    rows and their padded copies, FP8 copies of the ris exchange vv and ov^T rows padded to a
    multiple of 16 bytes with four floats per row (scales and norms)."""
    no, nv, na, nj, nk = 12, 70, 300, 54, 6
    ov = no * nv
    ris = nj * ov + nk * (no * no + nv * nv + ov)
    f64, _ = api.estimate_bytes(_desc(api, no, nv, na, nj, nk, 1), 0, api.default_opts())
    assert f64 == 8 * (na * (no * no + ov + nv * nv) + ris)
    pad = lambda n: -(-n // 8) * 8
    padded = nv * (pad(nv) + pad(no)) + no * (pad(no) + pad(nv))
    fmx, _ = api.estimate_bytes(_desc(api, no, nv, na, nj, nk, 2), 0, api.default_opts(precision=api.MIXED))
    pad16 = lambda n: -(-n // 16) * 16
    fp8 = nk * (nv * (pad16(nv) + pad16(no)) + 16)
    assert fmx == (4 * na * (no * no + ov + nv * nv) + 4 * na * padded + 4 * ov * pad(na) + 2 * ris
                   + 2 * nk * padded + fp8)
    both, _ = api.estimate_bytes(_desc(api, no, nv, na, nj, nk, 3), 0, api.default_opts())
    assert both == f64 + fmx


def test_admission_work_charge_grows_with_the_request(api):
    d = _desc(api, 20, 100, 600, 90, 10, 3)
    w = lambda kind, **kw: api.estimate_bytes(d, kind, api.default_opts(**kw), 3, 2)[1]
    assert w(0, n_states=5) < w(0, n_states=20)
    assert w(0, n_states=5, precond=api.DIAG) < w(0, n_states=5)
    assert w(0, n_states=5, max_subspace=40) < w(0, n_states=5)
    assert w(0, n_states=5, precision=api.MIXED) < w(0, n_states=5)
    with pytest.raises(api.TddftError):
        api.estimate_bytes(d, 3, api.default_opts())
