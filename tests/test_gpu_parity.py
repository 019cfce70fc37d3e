"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (tolerances stated per test):
  integer structure (edges, tet->edge map, CSR, crack states away from the
  threshold band): bit-exact;
  *1 and the values of L and b: 1e-12 relative to the largest entry;
  FP64 and mixed-precision temperatures: 1e-8 relative L2;
  k_eff (flux through x = 0): 1e-8 relative.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from dec_inputs import make_workload

pytestmark = pytest.mark.gpu

T_RTOL = 1e-8
K_RTOL = 1e-8
W_RTOL = 1e-12


@pytest.fixture(scope="module")
def abi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2104_05999_gb300 import _build, abi as _abi
    _build.build()
    _abi.load()
    return _abi


@pytest.fixture
def ctx(abi):
    c = abi.Context(device=0)
    yield c
    c.close()


def _oracle_structure(wl):
    E, t2e = O.edge_list(wl.tets)
    L = O.full_laplacian(wl.n, E, np.ones(len(E)))
    return E, t2e, L


CASES = [("kuhn9", None), ("lognormal64", 12), ("lognormal64", 17)]


@pytest.mark.parametrize("name,N", CASES)
def test_edges_and_csr_structure_bit_exact(ctx, name, N):
    wl = make_workload(name, N=N)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    E, t2e = ctx.dec_get_edges()
    Eo, t2eo, Lo = _oracle_structure(wl)
    assert np.array_equal(E, Eo)
    assert np.array_equal(t2e, t2eo)
    rowptr, col, _, _ = ctx.dec_get_csr(values=False)
    assert np.array_equal(rowptr, Lo.indptr)
    assert np.array_equal(col, Lo.indices)


@pytest.mark.parametrize("name,N", CASES)
def test_hodge_star_matches_oracle(ctx, name, N):
    wl = make_workload(name, N=N)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    ctx.dec_hodge_assemble(wl.k)
    w, fc = ctx.dec_get_hodge()
    Eo, t2eo, _ = _oracle_structure(wl)
    wo = O.hodge_star1(wl.xyz, wl.tets, Eo, t2eo, wl.k)
    scale = np.abs(wo).max()
    np.testing.assert_allclose(w, wo, rtol=0, atol=W_RTOL * scale)
    assert (fc == 1).all()          # no discs: never cut


@pytest.mark.parametrize("precond", ["jacobi", "fsai"])
def test_laplacian_values_rhs_and_preconditioner(ctx, abi, precond):
    wl = make_workload("lognormal64", N=11)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    ctx.dec_hodge_assemble(wl.k)
    pc = abi.DEC_PRECOND_FSAI if precond == "fsai" else abi.DEC_PRECOND_JACOBI
    ctx.dec_laplacian_build(wl.T0, pc)
    rowptr, col, val, b = ctx.dec_get_csr(0)
    Eo, t2eo = O.edge_list(wl.tets)
    wo = O.hodge_star1(wl.xyz, wl.tets, Eo, t2eo, wl.k)
    Lo, bo, _ = O.laplacian(wl.n, Eo, wo, wl.tags, wl.T0)
    assert np.array_equal(rowptr, Lo.indptr) and np.array_equal(col, Lo.indices)
    np.testing.assert_allclose(val, Lo.data, rtol=0,
                               atol=W_RTOL * np.abs(Lo.data).max())
    np.testing.assert_allclose(b, bo[0], rtol=0, atol=W_RTOL * np.abs(bo).max())
    g = ctx.dec_get_precond()
    if precond == "jacobi":
        d = np.zeros_like(val)
        diagpos = [rowptr[i] + np.searchsorted(col[rowptr[i]:rowptr[i + 1]], i)
                   for i in range(wl.n)]
        d[diagpos] = 1.0 / Lo.diagonal()
        np.testing.assert_allclose(g, d, rtol=1e-13)
    else:
        G = O.fsai_factor(Lo)
        # library layout: lower/diag entries hold G[row, col], upper G[col, row]
        rows = np.repeat(np.arange(wl.n), np.diff(rowptr))
        want = np.where(col <= rows, np.asarray(G[rows, col]).ravel(),
                        np.asarray(G[col, rows]).ravel())
        np.testing.assert_allclose(g, want, rtol=1e-10, atol=1e-12)


def _run(abi, ctx, wl, precond, mode, rtol, discs=None, scales=None, T0=None):
    from paper_2104_05999_gb300 import run_path
    return run_path(ctx, wl.xyz, wl.tets, wl.tags,
                    wl.T0 if T0 is None else T0, k=wl.k,
                    discs=discs, scales=scales, precond=precond, mode=mode,
                    rtol=rtol, max_iter=50000)


def test_kuhn9_jacobi_fp64_is_exact(abi, ctx):
    # the configuration with a closed-form answer: T = 1 - x, k_eff = 1
    wl = make_workload("kuhn9")
    res = _run(abi, ctx, wl, "jacobi", "fp64", 1e-12)
    exact = 1.0 - wl.xyz[:, 0]
    assert res.relres[0] <= 1e-12
    np.testing.assert_allclose(res.T[0], exact, atol=1e-10)
    for q in (res.q_in[0], res.q_out[0], res.energy[0]):
        assert q == pytest.approx(1.0, rel=K_RTOL)


@pytest.mark.parametrize("precond,mode", [("jacobi", "fp64"), ("fsai", "fp64"),
                                          ("fsai", "mixed"), ("jacobi", "mixed"),
                                          ("fsai", "mixed_phased"),
                                          ("jacobi", "mixed_phased")])
@pytest.mark.parametrize("N", [9, 16])
def test_lognormal_solve_matches_oracle(abi, ctx, precond, mode, N):
    wl = make_workload("lognormal64", N=N)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       precond="fsai", rtol=1e-13)
    res = _run(abi, ctx, wl, precond, mode, 1e-10)
    assert res.relres[0] <= 1e-10
    Tr = ref["T"][0]
    assert np.linalg.norm(res.T[0] - Tr) / np.linalg.norm(Tr) <= T_RTOL
    assert abs(res.q_in[0] - ref["q_in"][0]) <= K_RTOL * abs(ref["q_in"][0])
    # flux balance on the solved field
    assert res.q_out[0] == pytest.approx(res.q_in[0], rel=1e-7)


def test_several_dirichlet_sets(abi, ctx):
    wl = make_workload("hetero192", N=10, n_discs=0, n_sets=3)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       precond="fsai", rtol=1e-13)
    res = _run(abi, ctx, wl, "fsai", "mixed", 1e-10)
    for s in range(3):
        Tr = ref["T"][s]
        assert np.linalg.norm(res.T[s] - Tr) / np.linalg.norm(Tr) <= T_RTOL
        assert abs(res.energy[s] - ref["energy"][s]) <= K_RTOL * ref["energy"][s]


def _crack_band(wl, E, t2e, discs, scales, gpu_first, ref_first):
    """Edges whose crack state differs must have a sub-triangle whose cut
    distance sits within 1e-12 h of a state threshold (FP64 ties)."""
    bad = np.flatnonzero(gpu_first != ref_first)
    if len(bad) == 0:
        return 0
    _, (me, cF, cT) = O.hodge_pieces(wl.xyz, wl.tets)
    h = 1.0 / (wl.N - 1)
    sc = np.array([1.0]) if scales is None else scales
    for e in bad:
        tri = []
        for t, s in zip(*np.nonzero(t2e == e)):
            for hh in range(2):
                tri.append(np.stack([me[t, s], cF[t, s, hh], cT[t]]))
        tri = np.array(tri)
        close = False
        for d in discs:
            rho = O.crack_rho(tri, d)
            if np.any(np.abs(rho[:, None] - sc[None, :] * d[6]) <= 1e-12 * h):
                close = True
        assert close, f"edge {e}: crack state differs away from a tie"
    return len(bad)


def test_cracked_mesh_states_and_solution(abi, ctx):
    wl = make_workload("cracked128", N=14)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       discs=wl.discs, precond="fsai", rtol=1e-13)
    res = _run(abi, ctx, wl, "fsai", "mixed", 1e-10, discs=wl.discs)
    w, fc = ctx.dec_get_hodge()
    E, t2e = ctx.dec_get_edges()
    ref_first = np.minimum(ref["first_cut"], 1)
    assert (ref_first == 0).sum() > 0          # the discs do cut something
    _crack_band(wl, E, t2e, wl.discs, None, fc.astype(np.int64), ref_first)
    Tr = ref["T"][0]
    assert np.linalg.norm(res.T[0] - Tr) / np.linalg.norm(Tr) <= T_RTOL
    assert abs(res.q_in[0] - ref["q_in"][0]) <= K_RTOL * abs(ref["q_in"][0])


def test_crack_growth_states(abi, ctx):
    wl = make_workload("growth96", N=10, n_discs=8, n_scales=6)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       discs=wl.discs, scales=wl.scales, precond="fsai",
                       rtol=1e-13)
    res = _run(abi, ctx, wl, "fsai", "mixed", 1e-10, discs=wl.discs,
               scales=wl.scales)
    _, fc = ctx.dec_get_hodge()
    E, t2e = ctx.dec_get_edges()
    _crack_band(wl, E, t2e, wl.discs, wl.scales, fc.astype(np.int64),
                ref["first_cut"])
    q = res.q_in
    np.testing.assert_allclose(q, ref["q_in"], rtol=K_RTOL)
    assert (np.diff(q) <= 1e-9).all()           # cracks only grow


def test_full_size_lognormal64_structure_and_properties(abi, ctx):
    """64^3 jittered Delaunay, the benchmarked workload: integer structure
    bit-exact, *1 on every edge, FSAI rows on a sample, and the solution
    checked through properties that hold at any size."""
    wl = make_workload("lognormal64")
    res = _run(abi, ctx, wl, "fsai", "fp64", 1e-10)
    E, t2e = ctx.dec_get_edges()
    Eo, t2eo = O.edge_list(wl.tets)
    assert np.array_equal(E, Eo) and np.array_equal(t2e, t2eo)
    w, _ = ctx.dec_get_hodge()
    wo = O.hodge_star1(wl.xyz, wl.tets, Eo, t2eo, wl.k)
    np.testing.assert_allclose(w, wo, rtol=0, atol=W_RTOL * np.abs(wo).max())
    Lo, bo, _ = O.laplacian(wl.n, Eo, wo, wl.tags, wl.T0)
    rowptr, col, val, b = ctx.dec_get_csr(0)
    assert np.array_equal(rowptr, Lo.indptr) and np.array_equal(col, Lo.indices)
    # FSAI rows on a sample, computed one by one by the oracle
    g = ctx.dec_get_precond()
    rng = np.random.default_rng(0)
    for i in rng.choice(wl.n, 200, replace=False):
        P = col[rowptr[i]:rowptr[i + 1]]
        P = P[P <= i]
        A = Lo[P][:, P].toarray()
        gi = np.linalg.solve(A, np.eye(len(P))[-1])
        gi /= np.sqrt(gi[-1])
        np.testing.assert_allclose(g[rowptr[i]:rowptr[i] + len(P)], gi,
                                   rtol=1e-10, atol=1e-12)
    # the GPU solution satisfies the oracle's system to the requested residual
    dirich = wl.tags == 1
    u = res.T[0] - np.where(dirich, wl.T0[0], 0.0)
    rel = np.linalg.norm(bo[0] - Lo @ u) / np.linalg.norm(bo[0])
    assert rel <= 1.05e-10
    q_in, q_out, en = O.k_eff(wl.xyz, Eo, wo, res.T[0], wl.tags)
    assert res.q_in[0] == pytest.approx(q_in, rel=K_RTOL)
    assert q_in == pytest.approx(q_out, rel=1e-6)
    assert q_in == pytest.approx(en, rel=1e-6)


def test_errors_are_reported_not_raised_on_gpu(abi, ctx):
    wl = make_workload("kuhn9")
    with pytest.raises(abi.DecError) as e:
        ctx.dec_hodge_assemble(None)
    assert e.value.status == abi.DEC_ERR_STATE
    bad = wl.tets.copy()
    bad[0, 0] = wl.n + 5
    with pytest.raises(abi.DecError) as e:
        ctx.dec_mesh_upload(wl.xyz, bad, wl.tags)
    assert e.value.status == abi.DEC_ERR_MESH
    inv = wl.tets.copy()
    inv[0, [2, 3]] = inv[0, [3, 2]]
    with pytest.raises(abi.DecError) as e:
        ctx.dec_mesh_upload(wl.xyz, inv, wl.tags)
    assert e.value.status == abi.DEC_ERR_MESH
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    with pytest.raises(abi.DecError) as e:
        ctx.dec_hodge_assemble(-np.ones(wl.m))
    assert e.value.status == abi.DEC_ERR_ARG
    ctx.dec_hodge_assemble(None)
    ctx.dec_laplacian_build(wl.T0, abi.DEC_PRECOND_JACOBI)
    st, iters, relres = ctx.dec_solve(1e-12, 2, abi.DEC_MODE_FP64,
                                      raise_on_error=False)
    assert st == abi.DEC_NOT_CONVERGED and iters[0] == 2


def test_device_resident_inputs(abi, ctx):
    import torch
    from paper_2104_05999_gb300 import run_path
    wl = make_workload("lognormal64", N=9)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(a).to(dev)  # noqa: E731
    torch.cuda.synchronize()
    res = run_path(ctx, t(wl.xyz), t(wl.tets), t(wl.tags), t(wl.T0), k=t(wl.k),
                   precond="fsai", mode="fp64", rtol=1e-10)
    host = _run(abi, ctx, wl, "fsai", "fp64", 1e-10)
    assert np.array_equal(res.T, host.T)        # deterministic reductions
    assert res.q_in[0] == host.q_in[0]


# ------------------------------------------------------------ batched solve

def test_batched_crack_states_match_oracle(abi, ctx):
    """All crack states of a growing disc population in one batched launch
    (one FSAI factor per state, per-instance masks)."""
    wl = make_workload("growth96", N=10, n_discs=8, n_scales=6)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       discs=wl.discs, scales=wl.scales, precond="fsai",
                       rtol=1e-13)
    res = _run(abi, ctx, wl, "fsai_shared", "batched", 1e-10, discs=wl.discs,
               scales=wl.scales)
    assert (res.relres <= 1e-10).all() and (res.iters > 0).all()
    _, fc = ctx.dec_get_hodge()
    E, t2e = ctx.dec_get_edges()
    _crack_band(wl, E, t2e, wl.discs, wl.scales, fc.astype(np.int64),
                ref["first_cut"])
    for s in range(len(wl.scales)):
        Tr = ref["T"][s]
        assert np.linalg.norm(res.T[s] - Tr) / np.linalg.norm(Tr) <= T_RTOL
    np.testing.assert_allclose(res.q_in, ref["q_in"], rtol=K_RTOL)
    # right-hand sides of the batched set-up equal the oracle's per state
    for s in (0, len(wl.scales) - 1):
        _, _, _, b = ctx.dec_get_csr(s)
        np.testing.assert_allclose(b, ref["b"][s], rtol=0,
                                   atol=W_RTOL * np.abs(ref["b"][s]).max())


def test_batched_dirichlet_sets_match_oracle(abi, ctx):
    wl = make_workload("hetero192", N=9, n_sets=5)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       discs=wl.discs, precond="fsai", rtol=1e-13)
    res = _run(abi, ctx, wl, "fsai_shared", "batched", 1e-10, discs=wl.discs)
    for s in range(5):
        Tr = ref["T"][s]
        assert np.linalg.norm(res.T[s] - Tr) / np.linalg.norm(Tr) <= T_RTOL
        assert abs(res.energy[s] - ref["energy"][s]) <= K_RTOL * ref["energy"][s]


def test_batched_64_states_widest_stride(abi, ctx):
    # 64 instances: one row per 64 threads, the largest instance stride
    wl = make_workload("growth96", N=8, n_discs=5, n_scales=64)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       discs=wl.discs, scales=wl.scales, precond="jacobi",
                       rtol=1e-13)
    res = _run(abi, ctx, wl, "fsai_shared", "batched", 1e-10, discs=wl.discs,
               scales=wl.scales)
    np.testing.assert_allclose(res.q_in, ref["q_in"], rtol=K_RTOL)
    assert (np.diff(res.q_in) <= 1e-9).all()


def test_batched_mode_needs_shared_factor(abi, ctx):
    wl = make_workload("growth96", N=6, n_discs=3, n_scales=3)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    ctx.dec_hodge_assemble(wl.k, wl.discs, wl.scales)
    ctx.dec_laplacian_build(wl.T0, abi.DEC_PRECOND_FSAI)
    st, _, _ = ctx.dec_solve(1e-10, 1000, abi.DEC_MODE_MIXED_BATCHED,
                             raise_on_error=False)
    assert st == abi.DEC_ERR_STATE


def test_batched_autotuner_is_cached_and_does_not_change_results(abi, ctx):
    wl = make_workload("growth96", N=8, n_discs=5, n_scales=40)
    with pytest.raises(abi.DecError):
        ctx.dec_get_batch_variant()                # no batched solve yet
    res1 = _run(abi, ctx, wl, "fsai_shared", "batched", 1e-10, discs=wl.discs,
                scales=wl.scales)
    v1 = ctx.dec_get_batch_variant()
    assert v1 in (2, 4, 12, 114, 106)            # staged variants: Dirichlet sets only
    T2 = np.zeros_like(res1.T)
    _, it2, _ = ctx.dec_solve(1e-10, 50000, abi.DEC_MODE_MIXED_BATCHED, T2)
    assert ctx.dec_get_batch_variant() == v1     # tuned once per mesh and stride
    assert np.array_equal(res1.T, T2)
    assert np.array_equal(res1.iters, it2)


def test_batched_variants_are_bit_identical(abi, ctx):
    """Every launch variant of the batched kernel adds a row's entries in
    the same order: forced one by one on 8 Dirichlet sets (where the staged
    variants apply), they give identical temperatures and iterations, and
    those match the oracle."""
    from paper_2104_05999_gb300 import run
    wl = make_workload("hetero192", N=13)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k, discs=wl.discs,
                       precond="fsai", rtol=1e-13)
    base = None
    for v in (2, 4, 12, 114, 106, 1004, 2004, 2002, 2512):
        ctx.dec_set_batch_variant(v)
        res = run.run_path(ctx, wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k, discs=wl.discs,
                           mode="batched", rtol=1e-10)
        assert ctx.dec_get_batch_variant() == v
        if base is None:
            base = res
            for b in range(len(wl.T0)):
                Tr = ref["T"][b]
                assert np.linalg.norm(res.T[b] - Tr) <= T_RTOL * np.linalg.norm(Tr)
        else:
            assert np.array_equal(res.T, base.T), v
            assert np.array_equal(res.iters, base.iters), v
    ctx.dec_set_batch_variant(0)
    with pytest.raises(abi.DecError):
        ctx.dec_set_batch_variant(7)
    # a staged variant does not fit crack states
    wg = make_workload("growth96", N=6, n_discs=3, n_scales=3)
    ctx.dec_set_batch_variant(2004)
    ctx.dec_mesh_upload(wg.xyz, wg.tets, wg.tags)
    ctx.dec_hodge_assemble(wg.k, wg.discs, wg.scales)
    ctx.dec_laplacian_build(wg.T0, abi.DEC_PRECOND_FSAI_SHARED)
    st, _, _ = ctx.dec_solve(1e-10, 1000, abi.DEC_MODE_MIXED_BATCHED, raise_on_error=False)
    assert st == abi.DEC_ERR_ARG


@pytest.mark.parametrize("mode", ["fp64", "mixed_phased"])
def test_sell_shapes_are_bit_identical(abi, ctx, mode):
    """The single-instance SELL kernels' launch shapes (register round trips
    of 4, 8 or 12 entries at 4 or 8 blocks per SM for L; staged or chunked
    FSAI halves) add every row's entries in the same order: forced one by
    one they give identical temperatures and iterations, and the
    autotuner's pick is one of them."""
    from paper_2104_05999_gb300 import run
    wl = make_workload("lognormal64", N=20)
    prec = 0 if mode == "fp64" else 1
    res0 = run.run_path(ctx, wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k, mode=mode, rtol=1e-10)
    tuned = ctx.dec_get_sell_variant(prec)
    assert tuned[0] in (408, 808, 412, 804) and tuned[1] in (14, 8)
    for l_shape in (408, 808, 412, 804):
        for g_shape in (14, 8):
            ctx.dec_set_sell_variant(l_shape, g_shape)
            res = run.run_path(ctx, wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k, mode=mode,
                               rtol=1e-10)
            assert ctx.dec_get_sell_variant(prec) == (l_shape, g_shape)
            assert np.array_equal(res.T, res0.T), (l_shape, g_shape)
            assert np.array_equal(res.iters, res0.iters), (l_shape, g_shape)
    ctx.dec_set_sell_variant(0, 0)
    with pytest.raises(abi.DecError):
        ctx.dec_set_sell_variant(407, 14)
