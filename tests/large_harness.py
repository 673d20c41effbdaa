"""Chunked loading of workloads whose factors do not fit in host memory.

TEST INFRASTRUCTURE.  The large mixed workload (n_occ=150, n_vir=1350,
n_aux=6000, ris n_aux=1350) has 108 GB of FP64 factors over all orbitals, so
neither the tests nor the oracle ever hold them at once.  Worker processes
(spawn) draw P-chunks of the factors with the per-row generator of
``synth/generator.py``, write them as FP32 into shared memory for the parent
to copy to device tensors, and, when asked, return the oracle's FP64 partial
products of given test vectors over their rows -- the Coulomb and exchange
terms of Eq. hessian are sums over P, so the parent adds the slices up
(``oracle.operators.pair_from_parts``).
"""
from __future__ import annotations

import os
from multiprocessing import get_context, shared_memory

import numpy as np

CHUNK = 40
VBLOCK = 16


def _exact_task(args):
    name, p0, p1, shm_name, X = args
    from oracle import operators as O
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
    parts = None
    if X is not None:
        # vectors in blocks of VBLOCK keep a worker's intermediates near 2 GB
        out = [np.zeros_like(X) for _ in range(3)]
        for v0 in range(0, X.shape[0], VBLOCK):
            Xb = X[v0:v0 + VBLOCK]
            out[0][v0:v0 + VBLOCK] = O.coulomb(ov, Xb)
            out[1][v0:v0 + VBLOCK] = O.exchange_K1(oo, vv, Xb)
            out[2][v0:v0 + VBLOCK] = O.exchange_K2(ov, Xb)
        parts = tuple(out)
    return p0, p1, parts


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


def load_exact(name, meta, dev=None, X=None, workers=14):
    """Fill the device tensors dev = (L_oo, L_ov, L_vv) (FP32, [n_aux][p][q]) and/or
    return the oracle's summed (J, K1, K2) of the FP64 test vectors X [m][ov]."""
    import torch
    no, nv, na = meta["n_occ"], meta["n_vir"], meta["n_aux"]
    per = no * no + no * nv + nv * nv
    tasks = [(p0, min(na, p0 + CHUNK)) for p0 in range(0, na, CHUNK)]
    segs = [shared_memory.SharedMemory(create=True, size=CHUNK * per * 4) for _ in range(workers)] \
        if dev is not None else []
    J = K1 = K2 = None
    try:
        with _pool(workers) as pool:
            for w0 in range(0, len(tasks), workers):
                wave = tasks[w0:w0 + workers]
                args = [(name, p0, p1, segs[i].name if dev is not None else None, X)
                        for i, (p0, p1) in enumerate(wave)]
                for i, (p0, p1, parts) in enumerate(pool.map(_exact_task, args)):
                    if dev is not None:
                        n = p1 - p0
                        host = torch.frombuffer(segs[i].buf, dtype=torch.float32, count=n * per)
                        a, b = n * no * no, n * (no * no + no * nv)
                        dev[0][p0:p1].copy_(host[:a].view(n, no, no))
                        dev[1][p0:p1].copy_(host[a:b].view(n, no, nv))
                        dev[2][p0:p1].copy_(host[b:].view(n, nv, nv))
                        del host
                    if parts is not None:
                        J = parts[0] if J is None else J + parts[0]
                        K1 = parts[1] if K1 is None else K1 + parts[1]
                        K2 = parts[2] if K2 is None else K2 + parts[2]
        if dev is not None and dev[0].is_cuda:
            torch.cuda.synchronize()
    finally:
        for s in segs:
            s.close()
            s.unlink()
    return (J, K1, K2) if X is not None else None


def load_ris(name, meta, dev, workers=14):
    """Fill dev = (Lr_oo [n_K][no][no], Lr_ov [n_ris][no][nv], Lr_vv [n_K][nv][nv]) (FP32):
    every ris row for the Coulomb block, the s rows (every 9th) for exchange."""
    import torch
    no, nv, nr = meta["n_occ"], meta["n_vir"], meta["n_ris"]
    chunk = 36    # a multiple of 9, so every chunk starts on an s row
    tasks = [(r0, min(nr, r0 + chunk)) for r0 in range(0, nr, chunk)]
    size = (chunk * no * nv + (chunk // 9 + 1) * (no * no + nv * nv)) * 4
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
