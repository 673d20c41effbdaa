"""Chunked drawing of workloads whose factors do not fit in host memory.

Like ``generator.py`` this module only draws numbers.  The large mixed workload
(n_occ=150, n_vir=1350, n_aux=6000, ris n_aux=1350) has 108 GB of FP64 factors
over all orbitals, so they are never built whole: worker processes (spawn)
draw P-chunks with the per-row streams of ``generator.factor_rows`` /
``generator.ris_rows`` and write them as FP32 into shared memory, from which
the parent copies them into device tensors.  A caller may pass ``hook``, a
module-level function called in the worker on every exact chunk as
``hook(L_oo, L_ov, L_vv, *hook_args)``; its results come back per chunk (the
tests use it to evaluate the oracle's partial products over the same rows).
"""
from __future__ import annotations

import os
from multiprocessing import get_context, shared_memory

import numpy as np

CHUNK = 40          # exact factor rows per task
RIS_CHUNK = 36      # ris rows per task: a multiple of 9, so every chunk starts on an s row


def _exact_task(args):
    name, p0, p1, shm_name, hook, hook_args = args
    from synth.generator import factor_rows
    oo, ov, vv = factor_rows(name, p0, p1)
    if shm_name is not None:
        shm = shared_memory.SharedMemory(name=shm_name)
        try:
            n = p1 - p0
            flat = np.ndarray((n * (oo[0].size + ov[0].size + vv[0].size),), dtype=np.float32, buffer=shm.buf)
            a, b = n * oo[0].size, n * (oo[0].size + ov[0].size)
            flat[:a] = oo.reshape(-1)
            flat[a:b] = ov.reshape(-1)
            flat[b:] = vv.reshape(-1)
            del flat
        finally:
            shm.close()
    out = hook(oo, ov, vv, *hook_args) if hook is not None else None
    return p0, p1, out


def _ris_task(args):
    name, r0, r1, shm_name = args
    from synth.generator import ris_rows
    roo, rov, rvv = ris_rows(name, r0, r1)
    k = [r - r0 for r in range(r0, r1) if r % 9 == 0]
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        n = r1 - r0
        flat = np.ndarray((n * rov[0].size + len(k) * (roo[0].size + rvv[0].size),), dtype=np.float32,
                          buffer=shm.buf)
        a = n * rov[0].size
        b = a + len(k) * roo[0].size
        flat[:a] = rov.reshape(-1)
        flat[a:b] = roo[k].reshape(-1)
        flat[b:] = rvv[k].reshape(-1)
        del flat
    finally:
        shm.close()
    return r0, r1, len(k)


def _pool(workers):
    # one BLAS thread per worker process (inherited by the spawned children)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    return get_context("spawn").Pool(workers)


def default_workers():
    return max(1, min(16, (os.cpu_count() or 2) - 1))


def load_exact(name, meta, dev=None, hook=None, hook_args=(), workers=None):
    """Fill the device tensors dev = (L_oo, L_ov, L_vv) (FP32, [n_aux][p][q]),
    or None to draw only for ``hook``.  Returns the hook's per-chunk results as
    a list of (p0, p1, result) in chunk order (empty without a hook)."""
    import torch
    workers = workers or default_workers()
    no, nv, na = meta["n_occ"], meta["n_vir"], meta["n_aux"]
    per = no * no + no * nv + nv * nv
    tasks = [(p0, min(na, p0 + CHUNK)) for p0 in range(0, na, CHUNK)]
    segs = [shared_memory.SharedMemory(create=True, size=CHUNK * per * 4) for _ in range(workers)] \
        if dev is not None else []
    results = []
    try:
        with _pool(workers) as pool:
            for w0 in range(0, len(tasks), workers):
                wave = tasks[w0:w0 + workers]
                args = [(name, p0, p1, segs[i].name if dev is not None else None, hook, tuple(hook_args))
                        for i, (p0, p1) in enumerate(wave)]
                for i, (p0, p1, out) in enumerate(pool.map(_exact_task, args)):
                    if dev is not None:
                        n = p1 - p0
                        host = torch.frombuffer(segs[i].buf, dtype=torch.float32, count=n * per)
                        a, b = n * no * no, n * (no * no + no * nv)
                        dev[0][p0:p1].copy_(host[:a].view(n, no, no))
                        dev[1][p0:p1].copy_(host[a:b].view(n, no, nv))
                        dev[2][p0:p1].copy_(host[b:].view(n, nv, nv))
                        del host
                    if hook is not None:
                        results.append((p0, p1, out))
        if dev is not None and dev[0].is_cuda:
            torch.cuda.synchronize()
    finally:
        for s in segs:
            s.close()
            s.unlink()
    return results


def load_ris(name, meta, dev, workers=None):
    """Fill dev = (Lr_oo [n_K][no][no], Lr_ov [n_ris][no][nv], Lr_vv [n_K][nv][nv]) (FP32):
    every ris row for the Coulomb block, the s rows (every 9th) for exchange."""
    import torch
    workers = workers or default_workers()
    no, nv, nr = meta["n_occ"], meta["n_vir"], meta["n_ris"]
    tasks = [(r0, min(nr, r0 + RIS_CHUNK)) for r0 in range(0, nr, RIS_CHUNK)]
    size = (RIS_CHUNK * no * nv + (RIS_CHUNK // 9 + 1) * (no * no + nv * nv)) * 4
    segs = [shared_memory.SharedMemory(create=True, size=size) for _ in range(workers)]
    try:
        with _pool(workers) as pool:
            for w0 in range(0, len(tasks), workers):
                wave = tasks[w0:w0 + workers]
                args = [(name, r0, r1, segs[i].name) for i, (r0, r1) in enumerate(wave)]
                for i, (r0, r1, nk) in enumerate(pool.map(_ris_task, args)):
                    n = r1 - r0
                    host = torch.frombuffer(segs[i].buf, dtype=torch.float32,
                                            count=n * no * nv + nk * (no * no + nv * nv))
                    a = n * no * nv
                    b = a + nk * no * no
                    k0 = (r0 + 8) // 9
                    dev[1][r0:r1].copy_(host[:a].view(n, no, nv))
                    dev[0][k0:k0 + nk].copy_(host[a:b].view(nk, no, no))
                    dev[2][k0:k0 + nk].copy_(host[b:].view(nk, nv, nv))
                    del host
        if dev[0].is_cuda:
            torch.cuda.synchronize()
    finally:
        for s in segs:
            s.close()
            s.unlink()
