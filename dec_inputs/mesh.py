"""Lattice and Delaunay meshes of the unit cube.

Node numbering follows the paper's spatial pre-sort (Sec. 2.2: nodes ordered
by z, then y, then x), which on a lattice is ``id = i + N*(j + N*k)`` for the
node at lattice index (i, j, k).  Keeping this order keeps every node's
neighbours within a band of about N*N ids, which is what lets a sparse
matrix-vector product gather its x values from nearby memory.

Tets are returned in a canonical form: vertex ids sorted ascending, then the
last two swapped where needed so that every tet is positively oriented, and
the tet list sorted lexicographically.  The same mesh therefore comes out no
matter how it was produced (single Delaunay call or blocks).
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def lattice_spacing(N: int) -> float:
    return 1.0 / (N - 1)


def _lattice_points(N: int) -> np.ndarray:
    g = np.arange(N, dtype=np.float64) / (N - 1)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")      # id = i + N*(j + N*k)
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def _signed_volume6(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    a = xyz[tets[:, 0]]
    u = xyz[tets[:, 1]] - a
    v = xyz[tets[:, 2]] - a
    w = xyz[tets[:, 3]] - a
    return np.einsum("ij,ij->i", u, np.cross(v, w))


def canonical_tets(tets: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    """Sort ids in each tet, orient positively (swap the last two), sort rows."""
    t = np.sort(np.asarray(tets, dtype=np.int64), axis=1)
    neg = _signed_volume6(xyz, t) < 0
    t[neg, 2], t[neg, 3] = t[neg, 3].copy(), t[neg, 2].copy()
    order = np.lexsort((t[:, 3], t[:, 2], t[:, 1], t[:, 0]))
    return np.ascontiguousarray(t[order].astype(np.int32))


def kuhn_lattice(N: int):
    """Unit cube, N^3 nodes, every lattice cell split into the 6 Kuhn tets
    that share the cell's main diagonal (0,0,0)->(1,1,1)."""
    xyz = _lattice_points(N)
    c = np.arange(N - 1)
    k, j, i = np.meshgrid(c, c, c, indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()

    def v(di, dj, dk):
        return (i + di) + N * ((j + dj) + N * (k + dk))

    v000, v111 = v(0, 0, 0), v(1, 1, 1)
    # the 6 monotone lattice paths from corner 000 to corner 111
    paths = [((1, 0, 0), (1, 1, 0)), ((1, 0, 0), (1, 0, 1)),
             ((0, 1, 0), (1, 1, 0)), ((0, 1, 0), (0, 1, 1)),
             ((0, 0, 1), (1, 0, 1)), ((0, 0, 1), (0, 1, 1))]
    tets = np.concatenate(
        [np.stack([v000, v(*p), v(*q), v111], axis=1) for p, q in paths])
    return xyz, canonical_tets(tets, xyz)


def jittered_lattice(N: int, rng: np.random.Generator, jitter: float = 0.2):
    """N^3 lattice of the unit cube with every node moved uniformly by up to
    +-jitter*h per coordinate; boundary nodes move only tangentially (a
    coordinate that sits on 0 or 1 stays there), so cube edges move only
    along the edge and corners stay fixed."""
    xyz = _lattice_points(N)
    h = lattice_spacing(N)
    d = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
    d[(xyz == 0.0) | (xyz == 1.0)] = 0.0
    return xyz + d


# --------------------------------------------------------------------------
# Delaunay tetrahedralisation by certified blocks.
#
# Qhull's cost grows faster than linearly on these lattice point sets, so the
# cube is split into blocks of lattice nodes.  Each block is triangulated
# together with a halo of neighbouring nodes; a tet is kept by the block that
# owns its smallest vertex id and only if its circumscribed ball provably
# contains no node outside the block+halo set (every excluded node lies in a
# known box, since nodes move at most jitter*h from their lattice site).  For
# points in general position the Delaunay tetrahedralisation is unique, so a
# certified tet of a sub-problem is a tet of the global one.
# --------------------------------------------------------------------------

def _circumspheres(P: np.ndarray, simp: np.ndarray):
    a = P[simp[:, 0]]
    A = np.stack([P[simp[:, 1]] - a, P[simp[:, 2]] - a, P[simp[:, 3]] - a], 1)
    rhs = 0.5 * np.einsum("ijk,ijk->ij", A, A)
    ok = np.abs(np.linalg.det(A)) > 0
    c = np.full((len(simp), 3), np.nan)
    if ok.any():
        c[ok] = np.linalg.solve(A[ok], rhs[ok][..., None])[..., 0]
    r = np.linalg.norm(c, axis=1)
    return c + a, r


def _block_task(args):
    (P, gid, lo, hi, core_lo, core_hi, N, h, jit) = args
    from scipy.spatial import Delaunay
    simp = Delaunay(P).simplices
    g = gid[simp]
    owner = g.min(axis=1)
    oi = owner % N
    oj = (owner // N) % N
    ok_ = owner // (N * N)
    own = ((oi >= core_lo[0]) & (oi < core_hi[0]) & (oj >= core_lo[1])
           & (oj < core_hi[1]) & (ok_ >= core_lo[2]) & (ok_ < core_hi[2]))
    simp, g = simp[own], g[own]
    c, r = _circumspheres(P, simp)
    good = np.isfinite(r)
    # distance from each centre to each box that may hold an excluded node
    for ax in range(3):
        boxes = []
        if lo[ax] > 0:
            boxes.append((0.0, (lo[ax] - 1) * h + jit))
        if hi[ax] < N:
            boxes.append((hi[ax] * h - jit, 1.0))
        for (b0, b1) in boxes:
            lo3 = np.zeros(3)
            hi3 = np.ones(3)
            lo3[ax], hi3[ax] = b0, b1
            d = np.maximum(np.maximum(lo3 - c, c - hi3), 0.0)
            dist = np.linalg.norm(d, axis=1)
            good &= dist > r * (1.0 + 1e-9) + 1e-13
    return g, int((~good).sum())


def delaunay_lattice(xyz: np.ndarray, N: int, jitter: float = 0.2,
                     block: int = 16, halo: int = 3, workers: int | None = None):
    """Delaunay tetrahedralisation of a jittered N^3 lattice (canonical tets)."""
    h = lattice_spacing(N)
    jit = jitter * h * (1.0 + 1e-12)
    nb = -(-N // block)

    def task(bi, bj, bk, H):
        core_lo = np.array([bi, bj, bk]) * block
        core_hi = np.minimum(core_lo + block, N)
        lo = np.maximum(core_lo - H, 0)
        hi = np.minimum(core_hi + H, N)
        ii = np.arange(lo[0], hi[0])
        jj = np.arange(lo[1], hi[1])
        kk = np.arange(lo[2], hi[2])
        K, J, I = np.meshgrid(kk, jj, ii, indexing="ij")
        gid = (I + N * (J + N * K)).ravel()
        return (xyz[gid], gid, lo, hi, core_lo, core_hi, N, h, jit)

    blocks = [(bi, bj, bk) for bk in range(nb) for bj in range(nb)
              for bi in range(nb)]
    if workers is None:
        workers = min(len(blocks), os.cpu_count() or 1)
    H = halo
    pending = blocks
    out = []
    while pending:
        args = [task(*b, H) for b in pending]
        if workers > 1 and len(args) > 1:
            with mp.get_context("spawn").Pool(workers) as pool:
                res = pool.map(_block_task, args, chunksize=1)
        else:
            res = [_block_task(a) for a in args]
        retry = []
        for b, (g, bad) in zip(pending, res):
            if bad:
                retry.append(b)
            else:
                out.append(g)
        pending = retry
        H += 2
        if pending and H > N:
            raise RuntimeError("Delaunay blocks could not be certified")
    tets = canonical_tets(np.concatenate(out), xyz)
    _check_tetrahedralisation(xyz, tets)
    return tets


def _check_tetrahedralisation(xyz: np.ndarray, tets: np.ndarray):
    """Unit volume, no inverted or flat tets, every face in one or two tets."""
    v6 = _signed_volume6(xyz, tets)
    if not (v6 > 0).all():
        raise RuntimeError("mesher produced a non-positive tet")
    vol = v6.sum() / 6.0
    if abs(vol - 1.0) > 1e-10:
        raise RuntimeError(f"tet volumes sum to {vol!r}, not 1")
    t = tets.astype(np.int64)
    faces = np.concatenate([t[:, [1, 2, 3]], t[:, [0, 2, 3]], t[:, [0, 1, 3]],
                            t[:, [0, 1, 2]]])
    faces.sort(axis=1)
    o = np.lexsort((faces[:, 2], faces[:, 1], faces[:, 0]))
    f = faces[o]
    same = (f[1:] == f[:-1]).all(axis=1)
    if (same[1:] & same[:-1]).any():
        raise RuntimeError("a face is shared by more than two tets")
