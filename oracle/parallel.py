"""The oracle's assembly split over host processes, for meshes where one core
takes many minutes.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).  Assembly is a sum over
elements and facets (Eq. discreteElastoStatics, Eq. discreteLubrication), so
each worker sums ``Oracle.assemble_terms`` over one chunk of the elements and
facets and the parent adds the chunks and applies ``finish_assembly``.  No
arithmetic of the method lives here.  Workers are started with the ``spawn``
method, so a pool made after a CUDA context exists in the parent stays safe.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np
import scipy.sparse as sp

_O = None


def _init(oracle):
    global _O
    _O = oracle


def _chunk(args):
    elems, faces, U, P, with_jacobian = args
    o = _O
    neu = [(f, tb) for f, tb in zip(o.neu_faces, o.neu_traction) if int(f) in set(faces)]
    R, (r, c, v) = o.assemble_terms(U, P, elems, faces, neu, with_jacobian)
    J = None
    if with_jacobian:
        J = sp.coo_matrix((v, (r, c)), shape=(o.N, o.N)).tocsr()
        J.sum_duplicates()
    return R, J


def assemble(o, U=None, P=None, with_jacobian=True, workers=None, chunks_per_worker=4):
    """``o.assemble(U, P, with_jacobian)`` computed by a pool of processes."""
    U = o.U if U is None else U
    P = o.P if P is None else P
    workers = workers or os.cpu_count() or 1
    n = workers * chunks_per_worker
    elem_parts = np.array_split(np.arange(o.ne), n)
    face_parts = np.array_split(np.arange(o.nf), n)
    tasks = [(e.tolist(), f.tolist(), U, P, with_jacobian) for e, f in zip(elem_parts, face_parts)]
    ctx = mp.get_context("spawn")
    R = np.zeros(o.N)
    J = None
    with ctx.Pool(workers, initializer=_init, initargs=(o,)) as pool:
        for Rk, Jk in pool.imap_unordered(_chunk, tasks):
            R += Rk
            if Jk is not None:
                J = Jk if J is None else J + Jk
    return o.finish_assembly(R, J, U, P)
