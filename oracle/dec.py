"""FP64 oracle of the DEC steady-conduction path (arXiv 2104.05999).

TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the benchmark's
CPU baseline, never by the product path.  Shares no code with the CUDA
library.

Section map
  Sec. 2.1 (cell complexes, d o d = 0, circumcentric dual, diagonal Hodge
           stars as dual/primal volume ratios)   -> edge_list, face_list,
           d0_matrix, d1_matrix, circumcentres, hodge_pieces, hodge_star1
  Sec. 2.1 (conductivity on dual 2-cells)        -> hodge_star1(k=...)
  Sec. 2.3 (Eq. 11-13: system, Dirichlet and Neumann treatment; a crack sets
           a dual face's conductivity to zero)  -> laplacian, crack_rho,
           edge_crack_state
  Sec. 2.3 (ParaSails sparse approximate inverse) -> fsai_factor (factored
           SPAI on the lower pattern, the reading this library takes)
  Sec. 2.3 / Sec. 3.1 (Krylov solve to rel. tolerance 1e-10) -> pcg
  Sec. 2.5 (effective conductivity = flux through a Dirichlet face) -> k_eff
  Sec. 3.1 (Eq. 14, volume-weighted RMS error over tets) -> rms_error
  Sec. 2.3 (Eq. 11-13, the tet-centred mixed system, flux block
           eliminated) and Sec. 3.1 (the 1e-8 Hodge limiter) -> tet_centred_solve
  Sec. 2.5, 3.3, 3.4 (crack growth: the max-flux face or a random face
           cracks at each step, k_eff after each) -> crackable_edges,
           crack_evolution

Readings of the paper this oracle takes (each also listed with the library):
  * unknowns live on nodes: L = d0^T *1 d0 (the primal Darcy form the paper
    extends), not the face/tet mixed system of Eq. 11;
  * *1 uses signed circumcentric dual areas (a piece whose circumcentre lies
    on the far side of a face counts negative), so that linear fields are
    reproduced exactly on any mesh, as Sec. 2.5 and Sec. 3.1 report;
  * the 1e-8 Hodge limiter of Sec. 3.1 is not applied: the node form divides
    only by primal edge lengths;
  * a per-tet conductivity becomes one value per dual face, the mean of k_T
    over the tets around the edge weighted by the unsigned areas of their
    parts of the face (signed weights would give negative conductances);
  * a crack disc that cuts any sub-triangle of an edge's dual face zeroes
    that edge's whole *1 entry;
  * the Krylov stopping rule is ||b - L x||_2 / ||b||_2 <= rtol with x0 = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = [
    "LOCAL_EDGES", "FACE_OF_SLOT", "DIRICHLET", "edge_list", "face_list",
    "d0_matrix", "d1_matrix", "tet_volumes", "circumcentre_tet",
    "circumcentre_tri", "hodge_pieces", "hodge_star1", "dual_volumes",
    "crack_rho", "edge_crack_state", "laplacian", "full_laplacian",
    "jacobi", "fsai_factor", "pcg", "k_eff", "rms_error", "solve_path",
    "crackable_edges", "crack_evolution", "degenerate_nodes",
    "tet_centred_solve", "tet_crack_evolution", "whitney_flux",
]

DIRICHLET = 1

# local vertex pairs of a tet's 6 edges; slot s of tet t is edge
# (tets[t, a], tets[t, b]) with (a, b) = LOCAL_EDGES[s]
LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
# for slot s = (a, b) the two remaining local vertices (c, d): the two faces
# of the tet that contain the edge are {a, b, c} and {a, b, d}
FACE_OF_SLOT = ((2, 3), (1, 3), (1, 2), (0, 3), (0, 2), (0, 1))


# ---------------------------------------------------------------------------
# Topology (Sec. 2.1): cells, incidence matrices d0, d1
# ---------------------------------------------------------------------------

def edge_list(tets: np.ndarray):
    """Unique edges (i < j), sorted lexicographically, and the tet->edge map.

    Returns ``E int32[ne, 2]`` and ``t2e int32[m, 6]`` with ``t2e[t, s]`` the
    edge id of local edge ``LOCAL_EDGES[s]`` of tet t.
    """
    t = np.asarray(tets, dtype=np.int64)
    pairs = np.stack([t[:, [a, b]] for (a, b) in LOCAL_EDGES], axis=1)
    pairs = np.sort(pairs, axis=2).reshape(-1, 2)
    E, inv = np.unique(pairs, axis=0, return_inverse=True)
    return E.astype(np.int32), inv.reshape(-1, 6).astype(np.int32)


def face_list(tets: np.ndarray) -> np.ndarray:
    """Unique triangular faces (i < j < k), sorted lexicographically."""
    t = np.asarray(tets, dtype=np.int64)
    tri = np.concatenate([t[:, [1, 2, 3]], t[:, [0, 2, 3]], t[:, [0, 1, 3]],
                          t[:, [0, 1, 2]]])
    tri.sort(axis=1)
    return np.unique(tri, axis=0).astype(np.int32)


def d0_matrix(E: np.ndarray, n: int) -> sp.csr_matrix:
    """Coboundary on 0-cochains: edge (i, j), i < j, oriented i -> j, so
    (d0 T)_e = T_j - T_i."""
    ne = len(E)
    rows = np.repeat(np.arange(ne), 2)
    cols = E.reshape(-1)
    vals = np.tile([-1.0, 1.0], ne)
    return sp.csr_matrix((vals, (rows, cols)), shape=(ne, n))


def d1_matrix(F: np.ndarray, E: np.ndarray, n: int) -> sp.csr_matrix:
    """Coboundary on 1-cochains for faces (a, b, c), a < b < c, oriented
    a -> b -> c: boundary = (a,b) + (b,c) - (a,c)."""
    key = E[:, 0].astype(np.int64) * n + E[:, 1]
    order = np.argsort(key)

    def eid(i, j):
        k = i.astype(np.int64) * n + j
        return order[np.searchsorted(key[order], k)]

    nf = len(F)
    a, b, c = F[:, 0], F[:, 1], F[:, 2]
    rows = np.repeat(np.arange(nf), 3)
    cols = np.stack([eid(a, b), eid(b, c), eid(a, c)], 1).reshape(-1)
    vals = np.tile([1.0, 1.0, -1.0], nf)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, len(E)))


# ---------------------------------------------------------------------------
# Geometry of the circumcentric dual (Sec. 2.1)
# ---------------------------------------------------------------------------

def tet_volumes(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    X = xyz[tets]
    u, v, w = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]
    return np.einsum("ij,ij->i", u, np.cross(v, w)) / 6.0


def circumcentre_tet(X: np.ndarray) -> np.ndarray:
    """Centre of the sphere through the 4 points X[t] (shape [m, 4, 3]):
    (x_k - x_0) . (c - x_0) = |x_k - x_0|^2 / 2 for k = 1, 2, 3."""
    A = X[:, 1:] - X[:, :1]
    rhs = 0.5 * np.einsum("tkj,tkj->tk", A, A)
    return X[:, 0] + np.linalg.solve(A, rhs[..., None])[..., 0]


def circumcentre_tri(X: np.ndarray) -> np.ndarray:
    """Centre of the circle through the 3 points X[t] (shape [m, 3, 3]) in
    their plane: c = x_0 + a u + b v with u = x_1 - x_0, v = x_2 - x_0 and
    [u.u u.v; u.v v.v] [a; b] = [u.u; v.v] / 2."""
    u = X[:, 1] - X[:, 0]
    v = X[:, 2] - X[:, 0]
    uu = np.einsum("ij,ij->i", u, u)
    uv = np.einsum("ij,ij->i", u, v)
    vv = np.einsum("ij,ij->i", v, v)
    det = uu * vv - uv * uv
    a = 0.5 * (uu * vv - vv * uv) / det
    b = 0.5 * (vv * uu - uu * uv) / det
    return X[:, 0] + a[:, None] * u + b[:, None] * v


def hodge_pieces(xyz: np.ndarray, tets: np.ndarray):
    """Signed circumcentric dual-face pieces of every (tet, edge).

    Within tet T, the dual face of edge e = (a, b) is the quadrilateral
    (m_e, c_F1, c_T, c_F2), with m_e the edge midpoint, c_Fi the circumcentres
    of the two faces F1 = {a,b,c}, F2 = {a,b,d} that contain e and c_T the
    tet circumcentre (Sec. 2.1, circumcentric dual).  All four points lie in
    the bisector plane of e, and c_T projects onto F at c_F, so each half
    (m_e, c_F, c_T) is a right triangle with area |m_e c_F| |c_F c_T| / 2.
    Its sign is the product of two signed heights: + when c_F lies on the
    same side of e as F's third vertex, times + when c_T lies on the same
    side of F as the tet's fourth vertex.

    Returns ``area f64[m, 6, 2]`` (the two signed sub-triangle areas of each
    slot) and the points ``(m_e [m,6,3], c_F [m,6,2,3], c_T [m,3])``.
    """
    X = xyz[np.asarray(tets, dtype=np.int64)]
    m = len(X)
    cT = circumcentre_tet(X)
    area = np.zeros((m, 6, 2))
    me = np.zeros((m, 6, 3))
    cF = np.zeros((m, 6, 2, 3))
    for s, (a, b) in enumerate(LOCAL_EDGES):
        xa, xb = X[:, a], X[:, b]
        me[:, s] = 0.5 * (xa + xb)
        for h, (c, d) in enumerate((FACE_OF_SLOT[s], FACE_OF_SLOT[s][::-1])):
            xc, xd = X[:, c], X[:, d]
            cf = circumcentre_tri(np.stack([xa, xb, xc], axis=1))
            cF[:, s, h] = cf
            # signed height of c_F above edge e inside face F
            u = cf - me[:, s]
            h1 = np.linalg.norm(u, axis=1) * np.sign(
                np.einsum("ij,ij->i", u, xc - me[:, s]))
            # signed height of c_T above face F inside the tet
            nF = np.cross(xb - xa, xc - xa)
            nF /= np.linalg.norm(nF, axis=1, keepdims=True)
            h2 = np.einsum("ij,ij->i", cT - cf, nF) * np.sign(
                np.einsum("ij,ij->i", xd - xa, nF))
            area[:, s, h] = 0.5 * h1 * h2
    return area, (me, cF, cT)


def hodge_star1(xyz, tets, E, t2e, k=None, cut=None):
    """Diagonal Hodge star on primal 1-cells (Sec. 2.1): *1[e] = |*e| / |e|,
    the signed circumcentric dual-face area over the edge length, times the
    conductivity of the dual face.

    Conductivity is one value per dual 2-cell (Sec. 2.1).  A per-tet field
    k_T is carried onto the dual face of e as the mean of k_T over the tets
    around e, weighted by the unsigned areas of their parts of that face:
        kappa_e = sum_T k_T |*e cap T| / sum_T |*e cap T|,
    (|*e cap T| summed over the two sub-triangles of the part), so constant k
    scales *1 and a cell-wise positive k keeps every conductance >= 0 where
    the geometric *1 is.  Edges marked in ``cut`` get *1 = 0 (a crack makes a
    dual face insulating, Sec. 2.5)."""
    area, _ = hodge_pieces(xyz, tets)
    piece = area.sum(axis=2)                       # [m, 6]
    dual_area = np.bincount(t2e.reshape(-1), weights=piece.reshape(-1),
                            minlength=len(E))
    length = np.linalg.norm(xyz[E[:, 1]] - xyz[E[:, 0]], axis=1)
    w = dual_area / length
    if k is not None:
        part = np.abs(area).sum(axis=2)            # unsigned part of *e in T
        num = np.bincount(t2e.reshape(-1),
                          weights=(part * np.asarray(k)[:, None]).reshape(-1),
                          minlength=len(E))
        den = np.bincount(t2e.reshape(-1), weights=part.reshape(-1),
                          minlength=len(E))
        kappa = np.divide(num, den, out=np.zeros_like(num), where=den > 0)
        w = kappa * w
    if cut is not None:
        w = np.where(cut, 0.0, w)
    return w


def dual_volumes(xyz, tets, E, t2e):
    """Volume of each node's circumcentric dual cell, as the sum of the
    pyramids with apex at the node over its dual-face pieces (height |e|/2,
    since each piece lies in the bisector plane of its edge)."""
    area, _ = hodge_pieces(xyz, tets)
    piece = area.sum(axis=2)
    t = np.asarray(tets)
    n = len(xyz)
    vol = np.zeros(n)
    for s, (a, b) in enumerate(LOCAL_EDGES):
        le = np.linalg.norm(xyz[t[:, b]] - xyz[t[:, a]], axis=1)
        pyr = piece[:, s] * le / 6.0               # (1/3) * base * (|e|/2)
        vol += np.bincount(t[:, a], weights=pyr, minlength=n)
        vol += np.bincount(t[:, b], weights=pyr, minlength=n)
    return vol


# ---------------------------------------------------------------------------
# Cracks: a penny disc that cuts a dual face insulates it (Sec. 2.5)
# ---------------------------------------------------------------------------

def crack_rho(P: np.ndarray, disc: np.ndarray) -> np.ndarray:
    """Distance, inside the disc's plane, from the disc centre to the part
    of each triangle that the plane cuts; +inf where the plane misses the
    triangle or contains it (coplanar pieces are not cut).

    ``P f64[q, 3, 3]`` triangles, ``disc`` = (cx, cy, cz, nx, ny, nz, r).
    The disc (closed) cuts triangle q iff crack_rho <= r.
    """
    c = disc[:3]
    nrm = disc[3:6]
    s = (P - c) @ nrm                               # [q, 3] signed heights
    q = len(P)
    # The plane meets the closed triangle in a segment (or a point) whose
    # ends are among: crossing points of edges whose end heights have
    # opposite signs, and vertices lying on the plane.  Unless the triangle
    # lies in the plane, there are at most two such points.
    cand = []
    for (i, j) in ((0, 1), (1, 2), (0, 2)):
        si, sj = s[:, i], s[:, j]
        cross = (si * sj) < 0
        t = np.where(cross, si / np.where(cross, si - sj, 1.0), 0.0)
        cand.append((cross, P[:, i] + t[:, None] * (P[:, j] - P[:, i])))
    for i in range(3):
        cand.append((s[:, i] == 0.0, P[:, i]))
    count = np.zeros(q, dtype=int)
    A = np.zeros((q, 3))
    B = np.zeros((q, 3))
    for ok, X in cand:
        A[ok & (count == 0)] = X[ok & (count == 0)]
        B[ok & (count == 1)] = X[ok & (count == 1)]
        count = count + ok
    B[count == 1] = A[count == 1]
    hit = (count >= 1) & (count <= 2)               # 3 = coplanar: not cut
    # distance from the disc centre to the segment AB
    d = B - A
    dd = np.einsum("ij,ij->i", d, d)
    tt = np.einsum("ij,ij->i", c - A, d) / np.where(dd > 0, dd, 1.0)
    tt = np.where(dd > 0, np.clip(tt, 0.0, 1.0), 0.0)
    rho = np.full(q, np.inf)
    rho[hit] = np.linalg.norm(c - (A + tt[:, None] * d), axis=1)[hit]
    return rho


def edge_crack_state(xyz, tets, E, t2e, discs, scales=None):
    """Per edge, the first crack state (index b into ``scales``) in which
    some disc, with radius scales[b] * r, cuts a sub-triangle of the edge's
    dual face; ``len(scales)`` (never) when none does.  ``scales=None``
    means the single state [1.0], so the result is 0 (cut) or 1 (intact).

    Brute force over every disc and every dual-face sub-triangle.
    """
    scales = np.array([1.0]) if scales is None else np.asarray(scales)
    B = len(scales)
    _, (me, cF, cT) = hodge_pieces(xyz, tets)
    m = len(tets)
    tri = np.empty((m, 6, 2, 3, 3))
    tri[:, :, :, 0] = me[:, :, None, :]
    tri[:, :, :, 1] = cF
    tri[:, :, :, 2] = cT[:, None, None, :]
    tri = tri.reshape(-1, 3, 3)
    first = np.full(len(tri), B, dtype=np.int64)
    for disc in np.asarray(discs):
        rho = crack_rho(tri, disc)
        # first state b with scales[b] * r >= rho (scales increase with b)
        for b in range(B):
            hit = (rho <= scales[b] * disc[6]) & (first > b)
            first[hit] = b
    per_slot = first.reshape(m, 6, 2).min(axis=2)
    out = np.full(len(E), B, dtype=np.int64)
    np.minimum.at(out, t2e.reshape(-1), per_slot.reshape(-1))
    return out


# ---------------------------------------------------------------------------
# System assembly (Sec. 2.3, Eq. 11-13), node form
# ---------------------------------------------------------------------------

def full_laplacian(n: int, E: np.ndarray, w: np.ndarray) -> sp.csr_matrix:
    """L = d0^T diag(w) d0 written out entry by entry: L_ij = L_ji = -w_e
    for every edge e = (i, j), L_ii = sum of w over the edges at i.  The
    structural pattern is the mesh graph plus the diagonal, and entries whose
    weight is zero stay in it as explicit zeros.  Columns are sorted."""
    i, j = E[:, 0].astype(np.int64), E[:, 1].astype(np.int64)
    diag = np.bincount(i, weights=w, minlength=n) + np.bincount(
        j, weights=w, minlength=n)
    rows = np.r_[i, j, np.arange(n)]
    cols = np.r_[j, i, np.arange(n)]
    vals = np.r_[-w, -w, diag]
    order = np.lexsort((cols, rows))
    indptr = np.r_[0, np.cumsum(np.bincount(rows, minlength=n))]
    return sp.csr_matrix((vals[order], cols[order].astype(np.int32),
                          indptr.astype(np.int32)), shape=(n, n))


def laplacian(n, E, w, tags, T0):
    """Node system with Dirichlet rows eliminated (Sec. 2.3, Eq. 12):
    the unknown is u = T - T0 on free nodes and 0 on Dirichlet nodes, so

      L_ij = -w_ij, L_ii = sum_j w_ij     on free (and zero-flux) rows,
      Dirichlet columns moved to the right-hand side:
      b_i  = sum_{j Dirichlet} w_ij T0_j,
      Dirichlet rows: identity, b_i = 0.

    Zero-flux boundaries need no change in the node form (Eq. 13 with
    f0 = 0).  A free row whose weights are all zero (a node isolated by
    cracks) becomes an identity row with b = 0.  The structural pattern is
    that of full_laplacian, explicit zeros included.

    Returns (L csr, b [n_sets, n], isolated bool[n]).
    """
    Lf = full_laplacian(n, E, w)
    dirich = np.asarray(tags) == DIRICHLET
    T0 = np.atleast_2d(T0)
    b = np.zeros((T0.shape[0], n))
    rows = np.repeat(np.arange(n), np.diff(Lf.indptr))
    cols = Lf.indices
    vals = Lf.data.copy()
    offd = rows != cols
    to_rhs = offd & ~dirich[rows] & dirich[cols]
    for s in range(T0.shape[0]):
        # b_i = - sum_{j in D} L_ij T0_j = sum_{j in D} w_ij T0_j
        b[s] = -np.bincount(rows[to_rhs], weights=vals[to_rhs] * T0[s][
            cols[to_rhs]], minlength=n)
    vals[to_rhs] = 0.0                              # Dirichlet columns
    drow = dirich[rows]
    vals[drow] = np.where(offd[drow], 0.0, 1.0)     # Dirichlet rows
    diag = vals[~offd]
    isolated = (diag == 0.0) & ~dirich
    iso_diag = ~offd & isolated[rows]
    vals[iso_diag] = 1.0
    b[:, isolated] = 0.0
    Lm = sp.csr_matrix((vals, Lf.indices.copy(), Lf.indptr.copy()),
                       shape=(n, n))
    return Lm, b, isolated


# ---------------------------------------------------------------------------
# Preconditioners (Sec. 2.3: sparse approximate inverse of the ParaSails
# family) and the Krylov solve
# ---------------------------------------------------------------------------

def jacobi(L: sp.csr_matrix) -> np.ndarray:
    """Inverse of the diagonal."""
    return 1.0 / L.diagonal()


def fsai_factor(L: sp.csr_matrix, shift_rel: float = 1e-12,
                pivot_rel: float = 1e-12) -> sp.csr_matrix:
    """Factored sparse approximate inverse G (lower triangular) with the
    pattern of lower(L), so that G^T G ~ L^-1.

    For each row i with pattern P_i = {j <= i : (i, j) in pattern(L)}:
    solve L[P_i, P_i] g = e_i, then G[i, P_i] = g / sqrt(g_i).  Then
    G L G^T has a unit diagonal.  A principal block whose Cholesky meets a
    pivot <= pivot_rel * max(diag) is treated as singular and solved again
    with shift_rel * max(diag) added to its diagonal.
    """
    n = L.shape[0]
    indptr, indices = L.indptr, L.indices
    rows, cols, vals = [], [], []
    for i in range(n):
        rc = indices[indptr[i]:indptr[i + 1]]
        P = rc[rc <= i]                             # sorted, ends with i
        A = L[P][:, P].toarray()
        g = _spd_solve_unit_last(A, shift_rel, pivot_rel)
        g = g / np.sqrt(g[-1])
        rows.append(np.full(len(P), i))
        cols.append(P)
        vals.append(g)
    return sp.csr_matrix((np.concatenate(vals),
                          (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def _spd_solve_unit_last(A, shift_rel, pivot_rel):
    k = len(A)
    e = np.zeros(k)
    e[-1] = 1.0
    scale = np.abs(np.diag(A)).max()
    try:
        C = np.linalg.cholesky(A)
        if np.diag(C).min() ** 2 <= pivot_rel * scale:
            raise np.linalg.LinAlgError
    except np.linalg.LinAlgError:
        A = A + shift_rel * scale * np.eye(k)
        C = np.linalg.cholesky(A)
    y = np.linalg.solve(C, e)
    return np.linalg.solve(C.T, y)


def pcg(L: sp.csr_matrix, b: np.ndarray, apply_M, rtol: float,
        max_iter: int = 100000):
    """Preconditioned conjugate gradients from x0 = 0 (Hestenes-Stiefel).

    Stops when the recursively updated residual satisfies
    ||r||_2 <= rtol ||b||_2 and the true residual ||b - L x||_2 does too
    (otherwise it carries on).  Returns (x, iterations, true rel. residual).
    """
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = apply_M(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < max_iter:
        q = L @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        if np.linalg.norm(r) <= rtol * bnorm:
            true = np.linalg.norm(b - L @ x) / bnorm
            if true <= rtol:
                return x, it, true
        z = apply_M(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, np.linalg.norm(b - L @ x) / bnorm


# ---------------------------------------------------------------------------
# Outputs (Sec. 2.5, Sec. 3.1)
# ---------------------------------------------------------------------------

def k_eff(xyz, E, w, T, tags):
    """Effective conductivity of the unit cube (Sec. 2.5): the heat flux
    through the Dirichlet face x = 0 with T0 = 1 there and 0 at x = 1.

      Q_in  = sum_{i in D, x_i = 0} sum_j w_ij (T_i - T_j)
      Q_out = sum_{i in D, x_i = 1} sum_j w_ij (T_j - T_i)
      energy = sum_e w_e (T_i - T_j)^2 = T^T L_full T

    Returns (Q_in, Q_out, energy); k_eff = Q_in for a unit temperature drop.
    """
    dirich = np.asarray(tags) == DIRICHLET
    i, j = E[:, 0], E[:, 1]
    flux = w * (T[i] - T[j])              # heat along edge i -> j
    n = len(xyz)
    out = np.bincount(i, weights=flux, minlength=n) - np.bincount(
        j, weights=flux, minlength=n)     # net outflow of every node
    x0 = dirich & (xyz[:, 0] == 0.0)
    x1 = dirich & (xyz[:, 0] == 1.0)
    return out[x0].sum(), -out[x1].sum(), np.sum(w * (T[i] - T[j]) ** 2)


def degenerate_nodes(n, E, w, tags):
    """Cracks can cut nodes off from the Dirichlet faces.  Returns
    (isolated, islands, island_nodes): free nodes with no conducting edge
    (identity rows, T = 0), and the components of two or more nodes of the
    graph of conducting edges (w > 0) that contain no Dirichlet node (their
    block of L is singular; its right-hand side is zero, so CG from x0 = 0
    leaves T = 0 there with a preconditioner that keeps the block apart)."""
    from scipy.sparse.csgraph import connected_components
    keep = np.asarray(w) > 0.0
    G = sp.coo_matrix((np.ones(int(keep.sum())), (E[keep, 0], E[keep, 1])),
                      shape=(n, n))
    _, lab = connected_components(G, directed=False)
    size = np.bincount(lab)
    dirich = np.zeros(len(size), dtype=bool)
    dirich[lab[np.asarray(tags) == DIRICHLET]] = True
    isolated = int(np.sum((size == 1) & ~dirich))
    island = (size >= 2) & ~dirich
    return isolated, int(island.sum()), int(size[island].sum())


# ---------------------------------------------------------------------------
# Crack evolution (Sec. 2.5, Sec. 3.3, Sec. 3.4)
# ---------------------------------------------------------------------------

def crackable_edges(w):
    """Edges whose dual face may crack.  The paper cracks the faces that lie
    between two cells (its non-boundary faces); in the node form every dual
    face separates the dual cells of the edge's two end points, so every
    edge that still carries conductance (w > 0) is a candidate."""
    return np.asarray(w) > 0.0


def crack_evolution(xyz, tets, tags, T0, k=None, rule="max_flux",
                    max_steps=100, order=None, precond="fsai", rtol=1e-13,
                    k_stop=1e-9):
    """A sequence of steady solutions with one more crack each (Sec. 2.5):

    * rule "max_flux" (Sec. 3.3, deterministic): crack the uncracked
      crackable edge whose dual face carries the largest flux |w_e (T_i -
      T_j)| in the current solution (the value of the flux 2-form on that
      face); the smallest edge id wins a tie;
    * rule "order" (Sec. 3.4, stochastic): crack order[s] at step s (the
      caller draws the random sequence).

    Cracking sets the edge's conductance to 0.  Each step re-solves from
    scratch and records k_eff; the loop ends after max_steps, when no
    candidate is left, or once k_eff <= k_stop * k_eff(uncracked) (the domain
    no longer conducts).  Returns dict(cracked, k_eff, k_eff0, T, w, E).
    """
    n = len(xyz)
    tags = np.asarray(tags)
    T0 = np.asarray(T0, dtype=np.float64).reshape(-1)
    E, t2e = edge_list(tets)
    w = hodge_star1(xyz, tets, E, t2e, k)
    cand = crackable_edges(w)
    dirich = tags == DIRICHLET

    def solve(wc):
        L, b, _ = laplacian(n, E, wc, tags, T0)
        if precond == "jacobi":
            dinv = jacobi(L)
            M = lambda r: dinv * r                 # noqa: E731
        else:
            G = fsai_factor(L)
            Gt = G.T.tocsr()
            M = lambda r: Gt @ (G @ r)             # noqa: E731
        u, _, _ = pcg(L, b[0], M, rtol)
        T = u + np.where(dirich, T0, 0.0)
        return T, k_eff(xyz, E, wc, T, tags)[0]

    wc = w.copy()
    T, k0 = solve(wc)
    cracked, keff = [], []
    for step in range(max_steps):
        if rule == "max_flux":
            live = np.flatnonzero(cand & (wc != 0.0))
            if len(live) == 0:
                break
            flux = np.abs(wc[live] * (T[E[live, 0]] - T[E[live, 1]]))
            e = int(live[np.argmax(flux)])        # first maximum: smallest id
        elif rule == "order":
            if order is None or step >= len(order):
                break
            e = int(order[step])
            if not (0 <= e < len(E)) or not cand[e] or wc[e] == 0.0:
                raise ValueError(f"order[{step}] = {e} is not an uncracked crackable edge")
        else:
            raise ValueError(f"unknown rule {rule}")
        wc[e] = 0.0
        cracked.append(e)
        T, q = solve(wc)
        keff.append(q)
        if q <= k_stop * k0:
            break
    return dict(cracked=np.array(cracked, dtype=np.int64), k_eff=np.array(keff),
                k_eff0=k0, T=T, w=wc, E=E)


# ---------------------------------------------------------------------------
# The paper's own tet-centred form (Sec. 2.3, Eq. 11-13), reduced
# ---------------------------------------------------------------------------

def tet_centred_solve(xyz, tets, tags, T0, kappa=1.0, limiter=1e-8,
                      cracked_faces=None, face_flux=None):
    """The mixed system of Eq. 11 (flux per face, potential per tet) with the
    flux block eliminated, as the paper's Schur-complement solve does: the
    flux block (1/kappa) *2 is diagonal, so the potentials alpha (one per tet,
    at its circumcentre) solve the two-point operator

      sum over faces f of w_f (alpha_T - alpha_T'),   w_f = kappa / *2_f,

    with *2_f = l_f / |f|: the signed circumcentric dual edge length over the
    face area.  Interior face: l_f = h_T + h_T', the signed distances of the
    two circumcentres to the face (both project onto the face circumcentre,
    so the dual edge is normal to it).  Boundary face: the incomplete dual
    edge h_T.  Dirichlet faces (all three nodes Dirichlet) contribute
    w_f (alpha_T - T0_f), T0_f the mean of their nodes' values; other
    boundary faces carry the flux ``face_flux[f]`` (Eq. 13: the Neumann data
    f0 integrated over the face, outward; None: 0).  A group of tets that
    cracks cut off from every Dirichlet face keeps alpha = 0 (its block is
    singular with zero right-hand side; one tet of it is anchored).  Sec. 3.1 limits Hodge
    entries from near-zero dual edges to 1e-8: *2_f = max(*2_f, limiter)
    (limiter=None: no limit).  Cracked faces get w_f = 0 (Sec. 2.5).

    Returns dict(alpha, q_in, q_out, faces, t2f, ell, area, w, limited):
    q_in the heat entering through the Dirichlet faces on x = 0, q_out the
    heat leaving through those on x = 1 (k_eff for the unit cube).
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    t = np.asarray(tets, dtype=np.int64)
    m = len(t)
    tags = np.asarray(tags)
    T0 = np.asarray(T0, dtype=np.float64).reshape(-1)
    opp = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))      # face opposite vertex v
    tri = np.stack([np.sort(t[:, list(o)], axis=1) for o in opp], axis=1)   # [m, 4, 3]
    faces, inv = np.unique(tri.reshape(-1, 3), axis=0, return_inverse=True)
    t2f = inv.reshape(m, 4)
    nf = len(faces)
    X = xyz[t]
    cT = circumcentre_tet(X)
    h = np.zeros((m, 4))
    for v, o in enumerate(opp):
        a, b, c = X[:, o[0]], X[:, o[1]], X[:, o[2]]
        nrm = np.cross(b - a, c - a)
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        outward = np.sign(np.einsum("ij,ij->i", a - X[:, v], nrm))
        h[:, v] = np.einsum("ij,ij->i", a - cT, nrm) * outward
    ell = np.bincount(t2f.reshape(-1), weights=h.reshape(-1), minlength=nf)
    count = np.bincount(t2f.reshape(-1), minlength=nf)
    P = xyz[faces]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    star = ell / area
    limited = 0
    if limiter is not None:
        limited = int(np.sum(star < limiter))
        star = np.maximum(star, limiter)
    w = kappa / star
    if cracked_faces is not None:
        w[np.asarray(cracked_faces, dtype=np.int64)] = 0.0
    # the tets of each face
    owner = np.full((nf, 2), -1, dtype=np.int64)
    slot = np.zeros(nf, dtype=np.int64)
    for T_, f in zip(np.repeat(np.arange(m), 4), t2f.reshape(-1)):
        owner[f, slot[f]] = T_
        slot[f] += 1
    inner = count == 2
    dface = (count == 1) & (tags[faces] == DIRICHLET).all(axis=1)
    T0f = T0[faces].mean(axis=1)
    i1, i2, wi = owner[inner, 0], owner[inner, 1], w[inner]
    rows = np.concatenate([i1, i2, i1, i2, owner[dface, 0]])
    cols = np.concatenate([i1, i2, i2, i1, owner[dface, 0]])
    vals = np.concatenate([wi, wi, -wi, -wi, w[dface]])
    # components of tets joined by conducting faces that touch no Dirichlet
    # face (cut off by cracks) have a singular block with zero right-hand
    # side; one anchored tet per component fixes their potential at 0
    from scipy.sparse.csgraph import connected_components
    cond = wi > 0.0
    Gc = sp.coo_matrix((np.ones(int(cond.sum())), (i1[cond], i2[cond])), shape=(m, m))
    _, lab = connected_components(Gc, directed=False)
    anchored = np.ones(lab.max() + 1, dtype=bool)
    anchored[lab[owner[dface & (w > 0.0), 0]]] = False
    first = np.full(lab.max() + 1, -1, dtype=np.int64)
    for T_ in range(m - 1, -1, -1):
        first[lab[T_]] = T_
    anchor = first[anchored]
    rows = np.concatenate([rows, anchor])
    cols = np.concatenate([cols, anchor])
    vals = np.concatenate([vals, np.ones(len(anchor))])
    S = sp.csr_matrix((vals, (rows, cols)), shape=(m, m))
    rhs = np.bincount(owner[dface, 0], weights=w[dface] * T0f[dface], minlength=m)
    if face_flux is not None:
        nface = (count == 1) & ~dface
        rhs -= np.bincount(owner[nface, 0], weights=np.asarray(face_flux)[nface],
                           minlength=m)
    import scipy.sparse.linalg as sla
    alpha = sla.spsolve(S.tocsc(), rhs)
    x_face = P[:, :, 0]
    on0 = dface & (x_face == 0.0).all(axis=1)
    on1 = dface & (x_face == 1.0).all(axis=1)
    q_in = np.sum(w[on0] * (T0f[on0] - alpha[owner[on0, 0]]))
    q_out = np.sum(w[on1] * (alpha[owner[on1, 0]] - T0f[on1]))
    bflux = np.zeros(nf)          # outward flux through each boundary face
    bflux[dface] = w[dface] * (alpha[owner[dface, 0]] - T0f[dface])
    if face_flux is not None:
        nface = (count == 1) & ~dface
        bflux[nface] = np.asarray(face_flux)[nface]
    return dict(alpha=alpha, q_in=q_in, q_out=q_out, faces=faces, t2f=t2f,
                ell=ell, area=area, w=w, limited=limited, S=S, cT=cT,
                owner=owner, interior=inner, dirichlet=dface, boundary_flux=bflux)


def whitney_flux(xyz, tets, out):
    """Flux vector at each tet's barycentre from its face fluxes (Whitney
    2-form interpolation, the paper's vector output at cell barycentres):
    v = sum_i phi_i (b - x_i) / (3 V), phi_i the outward flux through the
    face opposite vertex i.  Face fluxes come from a tet_centred_solve
    result: w_f (alpha_T - alpha_T') across interior faces and its
    ``boundary_flux`` (Dirichlet faces: w_f (alpha_T - T0_f); Neumann faces:
    the prescribed flux) through boundary faces.  Whitney 2-forms reproduce
    a constant flux field exactly."""
    t = np.asarray(tets, dtype=np.int64)
    X = xyz[t]
    V = tet_volumes(xyz, t)
    b = X.mean(axis=1)
    owner, w, alpha = out["owner"], out["w"], out["alpha"]
    t2f = out["t2f"]
    v = np.zeros((len(t), 3))
    for i in range(4):
        f = t2f[:, i]
        other = np.where(owner[f, 0] == np.arange(len(t)), owner[f, 1], owner[f, 0])
        phi = np.where(other >= 0, w[f] * (alpha - alpha[np.maximum(other, 0)]),
                       out["boundary_flux"][f])
        v += phi[:, None] * (b - X[:, i]) / (3.0 * V[:, None])
    return v


def tet_crack_evolution(xyz, tets, tags, T0, max_steps=100000, k_stop=1e-9,
                        limiter=1e-8, order=None):
    """Sec. 3.3 in the paper's own form: after each solve the interior face
    with the largest flux |w_f (alpha_T - alpha_T')| cracks (w_f = 0; the
    smallest face id wins a tie), or, with ``order`` (Sec. 3.4, a random
    sequence of interior faces drawn by the caller), face order[s] cracks at
    step s; until k_eff <= k_stop * k_eff(uncracked).
    Returns dict(cracked, k_eff, k_eff0, damage) with damage = cracked /
    interior faces (the paper's count-based damage parameter D_n)."""
    out = tet_centred_solve(xyz, tets, tags, T0, limiter=limiter)
    owner, inner = out["owner"], out["interior"]
    k0 = out["q_in"]
    cracked, keff = [], []
    is_cracked = np.zeros(len(out["faces"]), dtype=bool)
    for _ in range(max_steps):
        live = np.flatnonzero(inner & ~is_cracked)
        if len(live) == 0:
            break
        if order is not None:
            if len(cracked) >= len(order):
                break
            f = int(order[len(cracked)])
            if not inner[f] or is_cracked[f]:
                raise ValueError(f"order[{len(cracked)}] = {f} is not an uncracked interior face")
        else:
            a = out["alpha"]
            flux = np.abs(out["w"][live] * (a[owner[live, 0]] - a[owner[live, 1]]))
            f = int(live[np.argmax(flux)])
        is_cracked[f] = True
        cracked.append(f)
        out = tet_centred_solve(xyz, tets, tags, T0, limiter=limiter,
                                cracked_faces=np.flatnonzero(is_cracked))
        keff.append(out["q_in"])
        if out["q_in"] <= k_stop * k0:
            break
    return dict(cracked=np.array(cracked, dtype=np.int64), k_eff=np.array(keff),
                k_eff0=k0, damage=len(cracked) / max(1, int(inner.sum())),
                faces=out["faces"], owner=owner, interior=inner)


def rms_error(xyz, tets, T, T_exact):
    """Sec. 3.1, Eq. 14: sqrt(sum_tets (T_comp - T_exact)^2 V), with the tet
    value taken as the mean of its four nodal values."""
    V = tet_volumes(xyz, tets)
    err = (T - T_exact)[tets].mean(axis=1)
    return np.sqrt(np.sum(err ** 2 * V))


def solve_path(xyz, tets, tags, T0, k=None, discs=None, scales=None,
               precond="fsai", rtol=1e-13):
    """The whole path for one mesh: edges, *1 (with cracks), L and b,
    preconditioner, PCG per instance, k_eff per instance.

    Instances are the Dirichlet value sets of ``T0`` (shared *1), or, when
    ``scales`` is given, the crack states (shared T0[0]), or, when ``k`` is a
    stack of per-tet fields [F, m], the conductivity fields (Sec. 1: many
    material fields on one mesh; shared T0[0] and cracks).
    """
    n = len(xyz)
    E, t2e = edge_list(tets)
    T0 = np.atleast_2d(T0)
    first = None
    if discs is not None and len(discs):
        first = edge_crack_state(xyz, tets, E, t2e, discs, scales)
    if k is not None and np.ndim(k) == 2:
        if scales is not None:
            raise ValueError("conductivity fields and crack states at once")
        inst = []
        for kf in np.asarray(k):
            wf = hodge_star1(xyz, tets, E, t2e, kf)
            inst.append((wf if first is None else np.where(first == 0, 0.0, wf), T0[0]))
        w0 = hodge_star1(xyz, tets, E, t2e, np.asarray(k)[0])
        return _solve_instances(xyz, tets, tags, E, t2e, w0, first, inst, precond, rtol)
    w0 = hodge_star1(xyz, tets, E, t2e, k)
    if scales is not None:
        inst = [(np.where(first <= b, 0.0, w0), T0[0])
                for b in range(len(scales))]
    else:
        w = w0 if first is None else np.where(first == 0, 0.0, w0)
        inst = [(w, T0[s]) for s in range(T0.shape[0])]
    return _solve_instances(xyz, tets, tags, E, t2e, w0, first, inst, precond, rtol)


def _solve_instances(xyz, tets, tags, E, t2e, w0, first, inst, precond, rtol):
    """PCG and k_eff for each (*1, T0) instance of solve_path."""
    n = len(xyz)
    out = dict(E=E, t2e=t2e, w0=w0, first_cut=first, T=[], iters=[],
               relres=[], q_in=[], q_out=[], energy=[], w=[], L=[], b=[])
    dirich = np.asarray(tags) == DIRICHLET
    for w, t0 in inst:
        L, b, iso = laplacian(n, E, w, tags, t0)
        if precond == "jacobi":
            dinv = jacobi(L)
            M = lambda r, d=dinv: d * r            # noqa: E731
        else:
            G = fsai_factor(L)
            Gt = G.T.tocsr()
            M = lambda r, G=G, Gt=Gt: Gt @ (G @ r)  # noqa: E731
        u, it, rr = pcg(L, b[0], M, rtol)
        T = u + np.where(dirich, t0, 0.0)
        qi, qo, en = k_eff(xyz, E, w, T, tags)
        for key, val in (("T", T), ("iters", it), ("relres", rr),
                         ("q_in", qi), ("q_out", qo), ("energy", en),
                         ("w", w), ("L", L), ("b", b[0])):
            out[key].append(val)
    return out
