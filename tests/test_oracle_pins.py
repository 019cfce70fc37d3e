"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics (closed forms, invariants, library routines, brute force).

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a swapped index) fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from dec_inputs import make_workload, kuhn_lattice, node_tags

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                rows.setdefault(line[0], []).append(line[1:])
    return rows


def _single(P):
    T = np.array([[0, 1, 2, 3]])
    if O.tet_volumes(P, T)[0] < 0:
        T = np.array([[0, 1, 3, 2]])
    E, t2e = O.edge_list(T)
    return T, E, t2e


# ----------------------------------------------------------------- topology

def test_edge_list_brute_force():
    wl = make_workload("lognormal64", N=4)
    E, t2e = O.edge_list(wl.tets)
    edges = set()
    for t in wl.tets.tolist():
        for a, b in itertools.combinations(t, 2):
            edges.add((min(a, b), max(a, b)))
    assert [tuple(e) for e in E.tolist()] == sorted(edges)
    for t, row in zip(wl.tets.tolist(), t2e.tolist()):
        for s, (a, b) in enumerate(O.LOCAL_EDGES):
            assert tuple(E[row[s]]) == (min(t[a], t[b]), max(t[a], t[b]))


def test_kuhn9_counts_and_euler():
    g = {k: int(v[0][0]) for k, v in _golden("kuhn9_counts.txt").items()}
    xyz, tets = kuhn_lattice(9)
    E, _ = O.edge_list(tets)
    F = O.face_list(tets)
    assert (len(xyz), len(E), len(F), len(tets)) == (
        g["nodes"], g["edges"], g["faces"], g["tets"])
    assert len(xyz) - len(E) + len(F) - len(tets) == 1


@pytest.mark.parametrize("name,N", [("kuhn9", 5), ("lognormal64", 6)])
def test_d1_d0_is_zero_and_euler(name, N):
    wl = make_workload(name, N=N)
    E, _ = O.edge_list(wl.tets)
    F = O.face_list(wl.tets)
    D0 = O.d0_matrix(E, wl.n)
    D1 = O.d1_matrix(F, E, wl.n)
    assert abs(D1 @ D0).sum() == 0.0
    # every edge column of d1 is non-empty and has entries +-1 only
    assert set(np.unique(D1.data)) <= {-1.0, 1.0}
    assert wl.n - len(E) + len(F) - wl.m == 1


# ------------------------------------------------------------ Hodge star *1

def test_right_corner_tet_closed_form():
    g = _golden("right_corner_tet.txt")
    P = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    T, E, t2e = _single(P)
    w = O.hodge_star1(P, T, E, t2e)
    want = {(int(a), int(b)): float(v) for a, b, v in g["edge"]}
    for e, (i, j) in enumerate(E.tolist()):
        assert w[e] == pytest.approx(want[(i, j)], abs=1e-15)
    dv = O.dual_volumes(P, T, E, t2e)
    for i, v in g["dualvol"]:
        assert dv[int(i)] == pytest.approx(float(v), abs=1e-15)


def test_regular_tet_closed_form():
    # regular tet of edge a: by symmetry every *1 entry is equal and the four
    # dual cells split the volume a^3/(6 sqrt 2) equally; the pyramid relation
    # V/4 = (1/3)(a/2) * 3 * (a w) then gives w = a / (12 sqrt 2)
    rng = np.random.default_rng(7)
    a = 0.37
    P = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1.0]])
    P *= a / np.linalg.norm(P[0] - P[1])
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    P = P @ Q.T + rng.standard_normal(3)
    T, E, t2e = _single(P)
    w = O.hodge_star1(P, T, E, t2e)
    np.testing.assert_allclose(w, a / (12 * np.sqrt(2)), rtol=1e-13)
    V = a ** 3 / (6 * np.sqrt(2))
    np.testing.assert_allclose(O.dual_volumes(P, T, E, t2e), V / 4,
                               rtol=1e-12)


def test_kuhn_lattice_is_h_times_7_point_stencil():
    # on the cubic lattice every Kuhn tet has the cell centre as
    # circumcentre, the dual cells are the lattice cubes clipped to the
    # domain: *1 = h * (face fraction) on axis edges, 0 on diagonals
    N = 9
    h = 1.0 / (N - 1)
    xyz, tets = kuhn_lattice(N)
    E, t2e = O.edge_list(tets)
    w = O.hodge_star1(xyz, tets, E, t2e)
    d = xyz[E[:, 1]] - xyz[E[:, 0]]
    axis = (np.abs(d) > 1e-12).sum(axis=1) == 1
    assert axis.sum() == 1944
    np.testing.assert_allclose(w[~axis], 0.0, atol=1e-16)
    mid = 0.5 * (xyz[E[:, 0]] + xyz[E[:, 1]])
    frac = np.ones(len(E))
    for ax in range(3):
        onface = (np.abs(d[:, ax]) < 1e-12) & (
            (mid[:, ax] == 0.0) | (mid[:, ax] == 1.0))
        frac[onface] *= 0.5
    np.testing.assert_allclose(w[axis], h * frac[axis], rtol=1e-13)


def test_hodge_matches_voronoi_face_areas():
    # library routine: Qhull's Voronoi diagram gives the dual (Voronoi) face
    # of every interior edge of a Delaunay mesh; its area / edge length is *1
    from scipy.spatial import Voronoi
    wl = make_workload("lognormal64", N=7)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e)
    vor = Voronoi(wl.xyz)
    onb = ((wl.xyz == 0.0) | (wl.xyz == 1.0)).any(axis=1)
    index = {tuple(e): i for i, e in enumerate(E.tolist())}
    checked = 0
    for (p, q), rv in zip(vor.ridge_points, vor.ridge_vertices):
        if -1 in rv or onb[p] or onb[q]:
            continue
        V = vor.vertices[rv]
        c = V.mean(axis=0)
        av = sum(np.cross(V[i] - c, V[(i + 1) % len(V)] - c)
                 for i in range(len(V)))
        area = 0.5 * np.linalg.norm(av)
        e = index[(min(p, q), max(p, q))]
        ln = np.linalg.norm(wl.xyz[p] - wl.xyz[q])
        assert w[e] == pytest.approx(area / ln, rel=1e-10, abs=1e-15)
        checked += 1
    assert checked > 100


@pytest.mark.parametrize("name,N", [("kuhn9", 6), ("lognormal64", 8)])
def test_dual_volumes_tile_the_cube(name, N):
    wl = make_workload(name, N=N)
    E, t2e = O.edge_list(wl.tets)
    dv = O.dual_volumes(wl.xyz, wl.tets, E, t2e)
    assert dv.sum() == pytest.approx(1.0, abs=1e-13)
    # Dirichlet energy of each coordinate field, sum_e w_e (x_j - x_i)^2:
    # the dual cells close up inside the cube, so it reduces to the dual
    # area of the face x = 1 (resp. y = 1, z = 1), which is 1 for k = 1
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e)
    d = wl.xyz[E[:, 1]] - wl.xyz[E[:, 0]]
    M = np.einsum("e,ei,ej->ij", w, d, d)
    np.testing.assert_allclose(np.diag(M), 1.0, atol=1e-13)


def test_conductivity_is_one_value_per_dual_face():
    # Sec. 2.1: conductivity belongs to the dual 2-cell, so *1 with a
    # per-tet field is the geometric *1 times one kappa_e per edge, a
    # positive-weighted mean of the k_T around the edge
    wl = make_workload("lognormal64", N=6)
    E, t2e = O.edge_list(wl.tets)
    w0 = O.hodge_star1(wl.xyz, wl.tets, E, t2e)
    # constant k scales every entry
    wc = O.hodge_star1(wl.xyz, wl.tets, E, t2e, np.full(wl.m, 3.7))
    np.testing.assert_allclose(wc, 3.7 * w0, rtol=1e-15, atol=0)
    # kappa_e lies between the smallest and largest k_T around e, and a
    # conductance is never negative where the geometric *1 is not (the mesh
    # has pieces of both signs, so a signed weighting would break this)
    area, _ = O.hodge_pieces(wl.xyz, wl.tets)
    assert (area < 0).any()
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    kmin = np.full(len(E), np.inf)
    kmax = np.zeros(len(E))
    np.minimum.at(kmin, t2e.reshape(-1), np.repeat(wl.k, 6))
    np.maximum.at(kmax, t2e.reshape(-1), np.repeat(wl.k, 6))
    big = w0 > 1e-10 * w0.max()
    kap = w[big] / w0[big]
    assert (kap >= kmin[big] * (1 - 1e-12)).all()
    assert (kap <= kmax[big] * (1 + 1e-12)).all()
    assert (w0 >= 0).all() and (w >= 0).all()


def test_layered_conductivity_gives_the_series_solution():
    # two layers x < 1/2 (k1) and x > 1/2 (k2) between the Dirichlet faces:
    # the exact field is piecewise linear with k1 s1 = k2 s2 and the
    # effective conductivity is the series value 2 k1 k2 / (k1 + k2)
    k1, k2 = 1.0, 4.0
    wl = make_workload("kuhn9", N=5)                 # x = 1/2 is a node plane
    cx = wl.xyz[wl.tets, 0].mean(axis=1)
    k = np.where(cx < 0.5, k1, k2)
    out = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=k,
                       precond="jacobi", rtol=1e-14)
    Tm = k1 / (k1 + k2)
    x = wl.xyz[:, 0]
    exact = np.where(x <= 0.5, 1.0 - (1.0 - Tm) * 2.0 * x,
                     Tm * 2.0 * (1.0 - x))
    np.testing.assert_allclose(out["T"][0], exact, atol=1e-12)
    assert out["q_in"][0] == pytest.approx(2 * k1 * k2 / (k1 + k2), rel=1e-12)
    assert out["q_out"][0] == pytest.approx(2 * k1 * k2 / (k1 + k2), rel=1e-12)


# ------------------------------------------------------------------ cracks

def _rho_by_line_clipping(P, disc):
    """Independent route: intersect the disc plane with the triangle's plane
    into a line, clip the line to the triangle (2D half-planes), then take the
    distance from the centre to the clipped segment."""
    c, nrm = disc[:3], disc[3:6]
    u, v = P[1] - P[0], P[2] - P[0]
    nt = np.cross(u, v)
    dirv = np.cross(nrm, nt)
    if np.linalg.norm(dirv) < 1e-14 * np.linalg.norm(nt):
        return np.inf
    # a point on both planes: solve [nrm; nt; dirv] x = [nrm.c; nt.P0; 0]
    A = np.stack([nrm, nt, dirv])
    x0 = np.linalg.solve(A, [nrm @ c, nt @ P[0], dirv @ c])
    lo, hi = -np.inf, np.inf
    for i in range(3):
        a, b, o = P[i], P[(i + 1) % 3], P[(i + 2) % 3]
        ed = b - a
        inward = np.cross(nt, ed)
        if inward @ (o - a) < 0:
            inward = -inward
        f0 = inward @ (x0 - a)
        f1 = inward @ dirv
        if abs(f1) < 1e-300:
            if f0 < 0:
                return np.inf
            continue
        t = -f0 / f1
        if f1 > 0:
            lo = max(lo, t)
        else:
            hi = min(hi, t)
    if lo > hi:
        return np.inf
    A_, B_ = x0 + lo * dirv, x0 + hi * dirv
    d = B_ - A_
    tt = 0.0 if d @ d == 0 else np.clip((c - A_) @ d / (d @ d), 0, 1)
    return np.linalg.norm(c - (A_ + tt * d))


def test_crack_rho_against_line_clipping():
    rng = np.random.default_rng(11)
    P = rng.uniform(0, 1, size=(400, 3, 3))
    rho = np.zeros(400)
    ref = np.zeros(400)
    discs = []
    for q in range(400):
        nrm = rng.standard_normal(3)
        nrm /= np.linalg.norm(nrm)
        disc = np.r_[rng.uniform(0, 1, 3), nrm, 0.3]
        discs.append(disc)
        rho[q] = O.crack_rho(P[q:q + 1], disc)[0]
        ref[q] = _rho_by_line_clipping(P[q], disc)
    fin = np.isfinite(ref)
    assert fin.sum() > 100 and (~fin).sum() > 50
    assert (np.isfinite(rho) == fin).all()
    np.testing.assert_allclose(rho[fin], ref[fin], rtol=1e-9, atol=1e-12)


def test_crack_rho_special_cases():
    disc = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 1.0])      # plane z = 0
    tri = np.array([[[2.0, -1.0, -1.0], [2.0, 1.0, -1.0], [2.0, 0.0, 1.0]]])
    # plane meets the triangle on x = 2, y in [-0.5, 0.5]: distance 2
    assert O.crack_rho(tri, disc)[0] == pytest.approx(2.0)
    flat = np.array([[[0.1, 0, 0], [0.2, 0, 0], [0.1, 0.2, 0.0]]])
    assert O.crack_rho(flat, disc)[0] == np.inf                 # coplanar
    above = tri + np.array([0, 0, 1.5])
    assert O.crack_rho(above, disc)[0] == np.inf                # missed
    touch = np.array([[[0.5, 0, 0], [0.5, 1, 1], [0.5, -1, 1.0]]])
    assert O.crack_rho(touch, disc)[0] == pytest.approx(0.5)    # one vertex


def test_crack_states_are_nested_and_k_eff_falls():
    wl = make_workload("growth96", N=8, n_discs=6, n_scales=5)
    out = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       discs=wl.discs, scales=wl.scales, precond="fsai",
                       rtol=1e-12)
    first = out["first_cut"]
    assert first.min() >= 0 and first.max() <= len(wl.scales)
    cut_counts = [(first <= b).sum() for b in range(len(wl.scales))]
    assert cut_counts == sorted(cut_counts) and cut_counts[-1] > 0
    q = np.array(out["q_in"])
    assert (np.diff(q) <= 1e-12).all() and q[-1] < q[0] < 1.0 + 1e-10


# -------------------------------------------------------- system and solve

def test_laplacian_symmetric_zero_row_sums_psd():
    wl = make_workload("lognormal64", N=5)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    L = O.full_laplacian(wl.n, E, w)
    assert abs(L - L.T).sum() == 0.0
    rs = np.asarray(L.sum(axis=1)).ravel()
    assert np.abs(rs).max() <= 1e-14 * np.abs(L.diagonal()).max()
    ev = np.linalg.eigvalsh(L.toarray())
    assert ev.min() > -1e-12 and abs(ev[0]) < 1e-12
    # structural pattern = mesh graph + diagonal
    assert L.nnz == 2 * len(E) + wl.n
    # the entry-by-entry form equals the product d0^T diag(w) d0
    D0 = O.d0_matrix(E, wl.n)
    P = (D0.T @ sp.diags(w) @ D0).toarray()
    np.testing.assert_allclose(L.toarray(), P, rtol=0, atol=1e-15)


def test_pcg_matches_dense_solve_with_dirichlet_partition():
    wl = make_workload("lognormal64", N=5)       # 125 nodes
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    Lf = O.full_laplacian(wl.n, E, w).toarray()
    D = wl.tags == 1
    F = ~D
    T0 = wl.T0[0]
    T = T0.copy()
    T[F] = np.linalg.solve(Lf[np.ix_(F, F)], -Lf[np.ix_(F, D)] @ T0[D])
    for pre in ("jacobi", "fsai"):
        out = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                           precond=pre, rtol=1e-13)
        np.testing.assert_allclose(out["T"][0], T, rtol=0, atol=1e-11)
        assert out["relres"][0] <= 1e-13


def test_fsai_full_pattern_is_inverse_cholesky():
    # with a full lower pattern the factored approximate inverse is exact:
    # G^T G = A^-1 and G A G^T = I
    rng = np.random.default_rng(3)
    X = rng.standard_normal((9, 9))
    A = X @ X.T + 9 * np.eye(9)
    G = O.fsai_factor(sp.csr_matrix(A)).toarray()
    assert np.allclose(np.triu(G, 1), 0.0)
    np.testing.assert_allclose(G @ A @ G.T, np.eye(9), atol=1e-12)
    np.testing.assert_allclose(G.T @ G, np.linalg.inv(A), atol=1e-12)


def test_fsai_sparse_pattern_unit_diagonal():
    wl = make_workload("lognormal64", N=6)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    L, b, _ = O.laplacian(wl.n, E, w, wl.tags, wl.T0)
    G = O.fsai_factor(L)
    lowpat = sp.tril(L, format="csr")
    assert (G.indptr == lowpat.indptr).all()
    assert (G.indices == lowpat.indices).all()
    np.testing.assert_allclose((G @ L @ G.T).diagonal(), 1.0, rtol=1e-12)


@pytest.mark.parametrize("name,N", [("kuhn9", None), ("lognormal64", 9)])
def test_linear_field_is_exact_and_k_eff_is_one(name, N):
    # Sec. 2.5 / 3.1: for constant conductivity the computed field is the
    # linear solution and k_eff equals the prescribed conductivity
    wl = make_workload(name, N=N)
    out = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=None,
                       precond=wl.precond, rtol=1e-13)
    T = out["T"][0]
    exact = 1.0 - wl.xyz[:, 0]
    np.testing.assert_allclose(T, exact, atol=1e-11)
    assert O.rms_error(wl.xyz, wl.tets, T, exact) < 1e-11
    for key in ("q_in", "q_out", "energy"):
        assert out[key][0] == pytest.approx(1.0, abs=1e-11)


def test_k_eff_flux_balance_and_dirichlet_bound():
    wl = make_workload("lognormal64", N=8)
    out = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       precond="fsai", rtol=1e-13)
    qi, qo, en = out["q_in"][0], out["q_out"][0], out["energy"][0]
    assert qi == pytest.approx(qo, rel=1e-10)
    assert qi == pytest.approx(en, rel=1e-10)
    # Dirichlet principle with the trial field 1 - x
    E, w = out["E"], out["w"][0]
    dx = wl.xyz[E[:, 1], 0] - wl.xyz[E[:, 0], 0]
    assert qi <= np.sum(w * dx ** 2) * (1 + 1e-12)
    # zero-flux boundary: no heat leaves through y, z faces
    T = out["T"][0]
    Lf = O.full_laplacian(wl.n, E, w)
    net = Lf @ T
    free = wl.tags != 1
    assert np.abs(net[free]).max() < 1e-11


def test_isolated_node_becomes_identity_row():
    wl = make_workload("lognormal64", N=5)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e)
    free = np.flatnonzero(wl.tags == 0)[3]
    w[(E[:, 0] == free) | (E[:, 1] == free)] = 0.0
    L, b, iso = O.laplacian(wl.n, E, w, wl.tags, wl.T0)
    assert iso[free] and iso.sum() == 1
    assert L[free, free] == 1.0 and b[0, free] == 0.0
    assert node_tags(wl.xyz)[free] == 0


# ----------------------------------------------------- crack evolution

def _dense_T(wl, E, w):
    """Dirichlet solve by dense elimination (independent of PCG)."""
    Lf = O.full_laplacian(wl.n, E, w).toarray()
    D = wl.tags == 1
    F = ~D
    T = wl.T0[0].copy()
    A = Lf[np.ix_(F, F)]
    rhs = -Lf[np.ix_(F, D)] @ T[D]
    # rows of nodes cut off from everything are zero: keep their T at 0
    iso = np.abs(A).sum(axis=1) == 0.0
    A[iso, iso] = 1.0
    T[F] = np.linalg.solve(A, rhs)
    return T


def _x_faces_connected(wl, E, w):
    from scipy.sparse.csgraph import connected_components
    keep = w > 0.0
    G = sp.coo_matrix((np.ones(keep.sum()), (E[keep, 0], E[keep, 1])),
                      shape=(wl.n, wl.n))
    _, lab = connected_components(G, directed=False)
    x = wl.xyz[:, 0]
    return bool(np.intersect1d(lab[x == 0.0], lab[x == 1.0]).size)


def test_max_flux_crack_is_the_largest_face_flux():
    # Sec. 3.3: the face carrying the largest flux cracks first; flux of the
    # dual face of e = |w_e (T_i - T_j)|, here from a dense solve and a loop
    wl = make_workload("lognormal64", N=5)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    T = _dense_T(wl, E, w)
    best, best_e = -1.0, -1
    for e in range(len(E)):
        if w[e] > 0.0:
            f = abs(w[e] * (T[E[e, 0]] - T[E[e, 1]]))
            if f > best:
                best, best_e = f, e
    out = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                            max_steps=1)
    assert out["cracked"].tolist() == [best_e]
    w1 = w.copy()
    w1[best_e] = 0.0
    T1 = _dense_T(wl, E, w1)
    q = O.k_eff(wl.xyz, E, w1, T1, wl.tags)[0]
    assert out["k_eff"][0] == pytest.approx(q, rel=1e-10)


def test_crack_growth_is_monotone_and_ends_at_separation():
    # removing conductance never raises k_eff (Rayleigh monotonicity); the
    # loop ends exactly when the cracks separate x = 0 from x = 1
    wl = make_workload("lognormal64", N=5)
    out = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                            max_steps=2000)
    k = out["k_eff"]
    assert (np.diff(k) <= 1e-12 * out["k_eff0"]).all()
    assert k[-1] <= 1e-9 * out["k_eff0"] < k[-2]
    E, w = out["E"], out["w"]
    assert not _x_faces_connected(wl, E, w)
    w_prev = w.copy()
    w_prev[out["cracked"][-1]] = O.hodge_star1(
        wl.xyz, wl.tets, E, O.edge_list(wl.tets)[1], wl.k)[out["cracked"][-1]]
    assert _x_faces_connected(wl, E, w_prev)


def test_kuhn_separation_needs_the_min_cut():
    # on the Kuhn lattice the conducting edges form the cubic grid (the
    # diagonals carry *1 = 0), whose smallest x = 0 / x = 1 cut has N^2 edges
    # (N^2 disjoint straight paths, Menger): no rule separates it sooner
    N = 4
    wl = make_workload("kuhn9", N=N)
    out = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=None,
                            precond="jacobi", max_steps=500)
    assert len(out["cracked"]) >= N * N
    assert not _x_faces_connected(wl, out["E"], out["w"])


def test_ordered_cracks_equal_cutting_them_at_once():
    # Sec. 3.4: the stochastic rule cracks a given random sequence; the end
    # state equals a solve with all those conductances set to 0
    wl = make_workload("lognormal64", N=5)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    rng = np.random.default_rng(7)
    order = rng.permutation(np.flatnonzero(O.crackable_edges(w)))[:12]
    out = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                            rule="order", order=order, max_steps=12)
    assert out["cracked"].tolist() == order.tolist()
    w12 = w.copy()
    w12[order] = 0.0
    T = _dense_T(wl, E, w12)
    assert out["k_eff"][-1] == pytest.approx(O.k_eff(wl.xyz, E, w12, T, wl.tags)[0],
                                             rel=1e-10)
    with pytest.raises(ValueError):
        O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                          rule="order", order=[order[0], order[0]], max_steps=2)


def test_degenerate_nodes_counts_isolated_nodes_and_islands():
    # a 3 x 3 x 3 Kuhn lattice with hand-made cuts: zeroing every edge of the
    # centre node isolates it; zeroing every edge leaving the pair {centre,
    # its +y neighbour} except the one between them makes an island of 2
    wl = make_workload("kuhn9", N=3)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e)
    w = np.where(w > 1e-12, w, 0.0)                 # drop the ~1e-17 diagonals
    c = 1 + 3 * (1 + 3 * 1)                         # node (1, 1, 1)
    wi = w.copy()
    wi[(E[:, 0] == c) | (E[:, 1] == c)] = 0.0
    assert O.degenerate_nodes(wl.n, E, wi, wl.tags) == (1, 0, 0)
    d = 1 + 3 * (2 + 3 * 1)                         # node (1, 2, 1), on y = 1
    pair = {c, d}
    touch = np.isin(E[:, 0], list(pair)) | np.isin(E[:, 1], list(pair))
    inside = np.isin(E[:, 0], list(pair)) & np.isin(E[:, 1], list(pair))
    wp = w.copy()
    wp[touch & ~inside] = 0.0
    assert wp[inside].max() > 0.0
    assert O.degenerate_nodes(wl.n, E, wp, wl.tags) == (0, 1, 2)
    assert O.degenerate_nodes(wl.n, E, w, wl.tags) == (0, 0, 0)


def test_conductivity_fields_as_instances():
    # Sec. 1: many material fields on one mesh.  Scaling every conductivity
    # by c scales L and b by c: T is unchanged and k_eff scales by c; each
    # field obeys the Dirichlet-principle bound with the trial field 1 - x
    wl = make_workload("lognormal64", N=5)
    c = np.array([1.0, 2.5, 0.4])
    fields = c[:, None] * wl.k[None, :]
    out = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=fields, precond="fsai",
                       rtol=1e-13)
    q = np.array(out["q_in"])
    np.testing.assert_allclose(q / q[0], c, rtol=1e-11)
    for f in range(3):
        np.testing.assert_allclose(out["T"][f], out["T"][0], rtol=0, atol=1e-11)
        E, w = out["E"], out["w"][f]
        dx = wl.xyz[E[:, 1], 0] - wl.xyz[E[:, 0], 0]
        assert q[f] <= np.sum(w * dx ** 2) * (1 + 1e-12)
    single = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=fields[1],
                          precond="fsai", rtol=1e-13)
    assert single["q_in"][0] == pytest.approx(q[1], rel=1e-12)
    with pytest.raises(ValueError):
        O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=fields, scales=[1.0, 2.0])


# -------------------------------------------- the paper's tet-centred form

def test_tet_form_is_exact_for_a_linear_field_without_the_limiter():
    # Sec. 3.1: when no Hodge entry is limited the method is exact for the
    # linear solution: alpha_T = 1 - x(c_T) at every circumcentre, k_eff = 1
    wl = make_workload("lognormal64", N=6)
    out = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0], limiter=1e-8)
    assert out["limited"] == 0
    np.testing.assert_allclose(out["alpha"], 1.0 - out["cT"][:, 0], atol=1e-11)
    assert out["q_in"] == pytest.approx(1.0, abs=1e-11)
    assert out["q_out"] == pytest.approx(1.0, abs=1e-11)
    S = out["S"]
    assert abs(S - S.T).sum() == 0.0


def test_tet_form_limiter_on_the_kuhn_lattice():
    # the 6 Kuhn tets of a cube share one circumcentre (the cube centre), so
    # the 6 faces inside each cube have dual edges of length 0: 6 (N-1)^3
    # limited entries; the limiter then leaves a small, non-zero error
    # (Sec. 3.1: the limiter is visible as non-machine-zero error)
    N = 4
    wl = make_workload("kuhn9", N=N)
    out = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0], limiter=1e-8)
    assert out["limited"] == 6 * (N - 1) ** 3
    err = np.abs(out["alpha"] - (1.0 - out["cT"][:, 0])).max()
    assert 1e-10 < err < 1e-5
    assert out["q_in"] == pytest.approx(1.0, abs=1e-5)


def test_tet_form_max_flux_cracking_ends_at_separation():
    # Sec. 3.3 in the tet form: k_eff never rises as faces crack, and the
    # loop ends exactly when no chain of uncracked interior faces links a
    # tet on x = 0 to a tet on x = 1
    from scipy.sparse.csgraph import connected_components
    wl = make_workload("lognormal64", N=5)
    out = O.tet_crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0])
    k = out["k_eff"]
    assert (np.diff(k) <= 1e-12 * out["k_eff0"]).all()
    assert k[-1] <= 1e-9 * out["k_eff0"] < k[-2]
    m = len(wl.tets)
    owner, inner = out["owner"], out["interior"]

    def linked(cracked):
        keep = inner.copy()
        keep[cracked] = False
        G = sp.coo_matrix((np.ones(keep.sum()), (owner[keep, 0], owner[keep, 1])),
                          shape=(m, m))
        _, lab = connected_components(G, directed=False)
        x = wl.xyz[:, 0]
        on = lambda v: np.flatnonzero((x[wl.tets] == v).sum(axis=1) == 3)  # noqa: E731
        return bool(np.intersect1d(lab[on(0.0)], lab[on(1.0)]).size)
    assert not linked(out["cracked"])
    assert linked(out["cracked"][:-1])


def test_tet_form_cut_off_tets_keep_zero_potential():
    # cracking the four faces of an interior tet cuts it off: its block is
    # singular with zero right-hand side and its potential stays 0; the rest
    # of the solution is finite and the cube still conducts
    wl = make_workload("lognormal64", N=5)
    base = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0])
    inner = base["interior"]
    t2f = base["t2f"]
    T = int(np.flatnonzero(inner[t2f].all(axis=1))[0])   # a tet with 4 interior faces
    out = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0], cracked_faces=t2f[T])
    assert out["alpha"][T] == 0.0
    assert np.isfinite(out["alpha"]).all()
    assert 0.0 < out["q_in"] <= base["q_in"] * (1 + 1e-12)


def test_tet_form_random_cracking_separates_near_the_papers_damage():
    # Sec. 3.4 reports that random face cracking makes the cube
    # non-conductive at a damage of about 0.55 (its 44,879-face mesh, 100
    # paths); a random path on a small mesh lands in the same range
    wl = make_workload("lognormal64", N=6)
    base = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0])
    order = np.random.default_rng(100).permutation(np.flatnonzero(base["interior"]))
    out = O.tet_crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], order=order)
    assert 0.4 < out["damage"] < 0.75


def test_tet_form_neumann_flux_and_whitney_output():
    # Eq. 13: with x = 1 a Neumann face carrying the outflow of the linear
    # field (unit flux density, i.e. |f| through each face), the linear
    # field is still the solution; Whitney 2-forms turn its face fluxes back
    # into the constant flux vector (1, 0, 0) at every barycentre
    wl = make_workload("lognormal64", N=6)
    tags = wl.tags.copy()
    tags[wl.xyz[:, 0] == 1.0] = 2                      # x = 1 becomes zero-flux...
    base = O.tet_centred_solve(wl.xyz, wl.tets, tags, wl.T0[0])
    P = wl.xyz[base["faces"]]
    on1 = (P[:, :, 0] == 1.0).all(axis=1)
    flux = np.where(on1, base["area"], 0.0)            # ...with unit outflow density
    out = O.tet_centred_solve(wl.xyz, wl.tets, tags, wl.T0[0], face_flux=flux)
    np.testing.assert_allclose(out["alpha"], 1.0 - out["cT"][:, 0], atol=1e-11)
    assert out["q_in"] == pytest.approx(1.0, abs=1e-11)
    v = O.whitney_flux(wl.xyz, wl.tets, out)
    np.testing.assert_allclose(v, np.tile([1.0, 0.0, 0.0], (len(wl.tets), 1)), atol=1e-10)
    # without the prescribed outflow the x = 1 face is insulated: no flux
    assert abs(base["q_in"]) < 1e-10


# ------------------------------------------- crack states and kappa_e, by hand

def test_crack_state_of_one_tet_by_hand():
    # hand-derived first crack states (tests/golden/right_corner_tet_crack.txt):
    # the edge takes the smallest rho over its two sub-triangles (Sec. 2.5: a
    # crack through any part of the dual face insulates it), states are the
    # first radius factor that reaches rho
    g = _golden("right_corner_tet_crack.txt")
    disc = np.array([float(v) for v in g["disc"][0]])
    scales = np.array([float(v) for v in g["scales"][0]])
    P = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    T, E, t2e = _single(P)
    first = O.edge_crack_state(P, T, E, t2e, disc[None, :], scales)
    index = {tuple(e): i for i, e in enumerate(E.tolist())}
    assert len(g["edge"]) == len(E)
    for i, j, _rho, b in g["edge"]:
        assert first[index[(int(i), int(j))]] == int(b), (i, j)
    # single state: 0 = cut, 1 = intact
    one = O.edge_crack_state(P, T, E, t2e, disc[None, :])
    for i, j, _rho, b in g["edge"]:
        assert one[index[(int(i), int(j))]] == (0 if int(b) == 0 else 1)


def _kuhn_axis_disc_rho(N, x0, yc, zc):
    """Closed-form crack distances on the Kuhn lattice for a disc in the
    plane x = x0 (generic: not on a lattice or half-lattice plane) centred at
    (x0, yc, zc).  The circumcentric dual of the Kuhn lattice is the cubic
    dual lattice (every Kuhn tet has its cell's centre as circumcentre):
      * an axis edge's dual face is the square of side h in its bisector
        plane, centred on the edge midpoint, clipped to the cube;
      * a face diagonal's dual face has zero area: the segments from its
        face's centre to the centres of the one or two cells on either side;
      * a body diagonal's dual is the cell centre alone, which no disc cuts
        (a point lies in the plane or misses it).
    The plane x = x0 meets: y-edges and z-edges at lattice index
    i* = round(x0 / h) (their squares span x0), and the diagonals of the
    cell faces x = i* h (their dual segments cross x0 at the face centre);
    nothing else.  Returns {(node a, node b): rho}."""
    h = 1.0 / (N - 1)
    i = int(round(x0 / h))
    assert abs(x0 - i * h) < 0.5 * h and abs(abs(x0 - i * h) - 0.5 * h) > 1e-6

    def nid(a, b, c):
        return a + N * (b + N * c)

    def gap(v, lo, hi):
        lo, hi = max(lo, 0.0), min(hi, 1.0)
        return max(lo - v, 0.0, v - hi)

    rho = {}
    for j in range(N - 1):              # y-edges (i, j, k) -> (i, j+1, k)
        for k in range(N):
            rho[(nid(i, j, k), nid(i, j + 1, k))] = np.hypot(
                (j + 0.5) * h - yc, gap(zc, (k - 0.5) * h, (k + 0.5) * h))
    for j in range(N):                  # z-edges (i, j, k) -> (i, j, k+1)
        for k in range(N - 1):
            rho[(nid(i, j, k), nid(i, j, k + 1))] = np.hypot(
                gap(yc, (j - 0.5) * h, (j + 0.5) * h), (k + 0.5) * h - zc)
    for j in range(N - 1):              # diagonals (i,j,k) -> (i,j+1,k+1)
        for k in range(N - 1):
            rho[(nid(i, j, k), nid(i, j + 1, k + 1))] = np.hypot(
                (j + 0.5) * h - yc, (k + 0.5) * h - zc)
    return rho


def test_crack_states_on_the_kuhn_lattice_closed_form():
    # two discs normal to x and to z (the second as the first with the axes
    # permuted), several radius factors: first state per edge = min over
    # discs of the first factor that reaches the closed-form rho
    N = 6
    xyz, tets = kuhn_lattice(N)
    E, t2e = O.edge_list(tets)
    scales = np.array([0.3, 0.55, 0.8, 1.0])
    discs = np.array([[0.37, 0.52, 0.44, 1.0, 0.0, 0.0, 0.31],
                      [0.29, 0.63, 0.61, 0.0, 0.0, 1.0, 0.26]])
    index = {tuple(e): q for q, e in enumerate(E.tolist())}
    expect = np.full(len(E), len(scales))
    margins = []
    # disc 0: plane x = 0.37
    rho0 = _kuhn_axis_disc_rho(N, 0.37, 0.52, 0.44)
    # disc 1: plane z = 0.61; relabel axes (x, y, z) -> (z, x, y), i.e. solve
    # the problem for coordinates (z, x, y) and map node ids back
    rho1p = _kuhn_axis_disc_rho(N, 0.61, 0.29, 0.63)

    def unperm(a):            # id in permuted labels (z, x, y) -> real id
        zz, xx, yy = a % N, (a // N) % N, a // (N * N)
        return xx + N * (yy + N * zz)

    rho1 = {tuple(sorted((unperm(a), unperm(b)))): r for (a, b), r in rho1p.items()}
    for rho, r in ((rho0, 0.31), (rho1, 0.26)):
        for (a, b), d in rho.items():
            q = index[(min(a, b), max(a, b))]
            hit = np.flatnonzero(scales * r >= d)
            margins.append(np.min(np.abs(scales * r - d)))
            if hit.size:
                expect[q] = min(expect[q], hit[0])
    assert min(margins) > 1e-9            # no ties with the thresholds
    first = O.edge_crack_state(xyz, tets, E, t2e, discs, scales)
    assert (expect < len(scales)).sum() > 20
    assert len(set(expect.tolist())) == len(scales) + 1   # every state occurs
    np.testing.assert_array_equal(first, expect)


def test_conductivity_weights_by_hand():
    # Sec. 2.1 (conductivity on the dual 2-cell), values derived by hand in
    # tests/golden/two_tet_conductivity.txt: an unweighted mean of k_T, or
    # weights by signed part area (parallel conductances), give other values
    g = _golden("two_tet_conductivity.txt")
    k = np.array([float(v) for v in g["k"][0]])
    P = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]])
    T = np.array([[0, 1, 2, 3], [1, 2, 3, 4]])
    for t in range(2):
        if O.tet_volumes(P, T[t:t + 1])[0] < 0:
            T[t, 2], T[t, 3] = T[t, 3], T[t, 2]
    E, t2e = O.edge_list(T)
    w = O.hodge_star1(P, T, E, t2e, k)
    index = {tuple(e): i for i, e in enumerate(E.tolist())}
    assert len(g["edge"]) == len(E)
    for i, j, v in g["edge"]:
        assert w[index[(int(i), int(j))]] == pytest.approx(float(v), rel=1e-13)
    # k = 1 gives the purely geometric star: 1/4, 1/12 and 1/24
    w1 = O.hodge_star1(P, T, E, t2e)
    assert w1[index[(1, 2)]] == pytest.approx(1.0 / 24.0, rel=1e-13)
    assert w1[index[(1, 4)]] == pytest.approx(1.0 / 12.0, rel=1e-13)


def test_rms_error_closed_forms():
    # Sec. 3.1, Eq. 14: sqrt(sum_T e_T^2 V_T), e_T the mean of the 4 nodal
    # errors.  A constant error c gives |c| on the unit cube; an error of 1
    # at one interior Kuhn node (24 tets of volume h^3/6 around it, e_T =
    # 1/4) gives sqrt(4 h^3 / 16) = h^1.5 / 2
    N = 5
    h = 1.0 / (N - 1)
    xyz, tets = kuhn_lattice(N)
    base = np.zeros(len(xyz))
    assert O.rms_error(xyz, tets, base + 0.3, base) == pytest.approx(0.3, rel=1e-13)
    node = 2 + N * (2 + N * 2)
    e = base.copy()
    e[node] = 1.0
    assert (tets == node).any(axis=1).sum() == 24
    assert O.rms_error(xyz, tets, e, base) == pytest.approx(h ** 1.5 / 2, rel=1e-13)
