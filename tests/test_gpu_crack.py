"""Crack growth on the GPU (dec_crack_evolve, Sec. 2.5, 3.3, 3.4) against
the FP64 oracle's crack_evolution.

Bars: the cracked edge ids are bit-exact, except where two candidates' face
fluxes lie within 1e-8 relative of each other in the oracle's solution (a
tie that FP64 solutions differing at the 1e-10 level may break either way;
the comparison stops there); k_eff after every step within 1e-8 of the
uncracked k_eff (k_eff falls to ~0 at separation, so the bar is absolute
in units of k_eff(uncracked)).

The library updates only the rows a crack changes and starts each solve
from the previous solution; the oracle rebuilds and solves from zero at
every step, as does the library with DEC_CRACK_REBUILD.
"""
import numpy as np
import pytest

import oracle as O
from dec_inputs import make_workload

pytestmark = pytest.mark.gpu

K_TOL = 1e-8
TIE = 1e-8


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


def _setup(abi, ctx, wl, precond):
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    ctx.dec_hodge_assemble(wl.k)
    ctx.dec_laplacian_build(wl.T0[:1], abi.DEC_PRECOND_FSAI if precond == "fsai"
                            else abi.DEC_PRECOND_JACOBI)


def _flux_tie(wl, E, w_state, T, a, b):
    fa = abs(w_state[a] * (T[E[a, 0]] - T[E[a, 1]]))
    fb = abs(w_state[b] * (T[E[b, 0]] - T[E[b, 1]]))
    return abs(fa - fb) <= TIE * max(fa, fb)


# the Kuhn lattice is symmetric: its face fluxes tie exactly from the first
# step on, so only the lognormal mesh is held to a long common prefix
@pytest.mark.parametrize("name,N,precond,prefix", [("lognormal64", 5, "fsai", 20),
                                                    ("kuhn9", 4, "jacobi", 0)])
def test_max_flux_growth_matches_oracle(abi, ctx, name, N, precond, prefix):
    wl = make_workload(name, N=N)
    ref = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                            precond=precond, max_steps=2000, rtol=1e-13)
    _setup(abi, ctx, wl, precond)
    st, cracked, keff = ctx.dec_crack_evolve(abi.DEC_CRACK_MAX_FLUX, 2000,
                                             rtol=1e-12)
    E = ref["E"]
    k0 = ref["k_eff0"]
    n_ref = len(ref["cracked"])
    # walk both sequences; at a divergence it must be a flux tie
    w0 = O.hodge_star1(wl.xyz, wl.tets, E, O.edge_list(wl.tets)[1], wl.k)
    same = 0
    for s in range(min(n_ref, len(cracked))):
        if cracked[s] != ref["cracked"][s]:
            ws = w0.copy()
            ws[ref["cracked"][:s]] = 0.0
            # the oracle's solution before step s
            if s == 0:
                T = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                                      precond=precond, max_steps=0)["T"]
            else:
                T = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                                      precond=precond, rule="order",
                                      order=ref["cracked"][:s], max_steps=s)["T"]
            assert _flux_tie(wl, E, ws, T, int(cracked[s]), int(ref["cracked"][s])), s
            break
        assert abs(keff[s] - ref["k_eff"][s]) <= K_TOL * k0, (s, keff[s], ref["k_eff"][s])
        same += 1
    if same == n_ref:
        # no tie met: the whole sequence, and where it ended, agree
        assert len(cracked) == n_ref
    assert same >= min(n_ref, prefix)
    # either way the GPU run ends with the domain separated
    assert keff[-1] <= 1e-9 * k0
    if name == "kuhn9":
        assert len(cracked) >= N * N     # the min cut of the cubic grid


def _walk_max_flux(wl, ref, cracked, keff, precond):
    """Number of leading steps where the GPU's max-flux picks and k_eff
    agree with the oracle; a divergence must be a flux tie."""
    E = ref["E"]
    k0 = ref["k_eff0"]
    w0 = O.hodge_star1(wl.xyz, wl.tets, E, O.edge_list(wl.tets)[1], wl.k)
    same = 0
    for s in range(min(len(ref["cracked"]), len(cracked))):
        if cracked[s] != ref["cracked"][s]:
            ws = w0.copy()
            ws[ref["cracked"][:s]] = 0.0
            T = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                                  precond=precond, rule="order",
                                  order=ref["cracked"][:s], max_steps=s)["T"]
            assert _flux_tie(wl, E, ws, T, int(cracked[s]), int(ref["cracked"][s])), s
            break
        assert abs(keff[s] - ref["k_eff"][s]) <= K_TOL * k0, (s, keff[s], ref["k_eff"][s])
        same += 1
    return same


@pytest.mark.parametrize("rebuild", [False, True])
def test_max_flux_growth_at_N10(abi, ctx, rebuild):
    # 100 steps on the 10^3 jittered Delaunay cube (1000 nodes)
    wl = make_workload("lognormal64", N=10)
    ref = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                            precond="fsai", max_steps=100, rtol=1e-13)
    _setup(abi, ctx, wl, "fsai")
    rule = abi.DEC_CRACK_MAX_FLUX | (abi.DEC_CRACK_REBUILD if rebuild else 0)
    st, cracked, keff = ctx.dec_crack_evolve(rule, 100, rtol=1e-12)
    assert len(cracked) == 100
    assert _walk_max_flux(wl, ref, cracked, keff, "fsai") >= 40


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_ordered_growth_at_N12(abi, ctx, mode):
    wl = make_workload("lognormal64", N=12)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    order = np.random.default_rng(5).permutation(np.flatnonzero(O.crackable_edges(w)))[:60]
    ref = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                            rule="order", order=order, max_steps=60, rtol=1e-13)
    _setup(abi, ctx, wl, "fsai")
    md = abi.DEC_MODE_FP64 if mode == "fp64" else abi.DEC_MODE_MIXED
    st, cracked, keff = ctx.dec_crack_evolve(abi.DEC_CRACK_ORDER, 60, order=order,
                                             rtol=1e-12 if mode == "fp64" else 1e-11,
                                             mode=md)
    assert cracked.tolist() == order.tolist()
    np.testing.assert_allclose(keff, ref["k_eff"], rtol=0, atol=K_TOL * ref["k_eff0"])


@pytest.mark.parametrize("precond", ["fsai", "jacobi"])
def test_row_updates_equal_a_rebuild(abi, ctx, precond):
    # the same cracks with row updates + warm starts and with full rebuilds
    # + cold starts: the same k_eff per step (to the solver tolerance), and
    # the warm starts need fewer CG iterations
    wl = make_workload("lognormal64", N=10)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    order = np.random.default_rng(9).permutation(np.flatnonzero(O.crackable_edges(w)))[:80]
    res = {}
    for rebuild in (False, True):
        _setup(abi, ctx, wl, precond)
        rule = abi.DEC_CRACK_ORDER | (abi.DEC_CRACK_REBUILD if rebuild else 0)
        _, cracked, keff = ctx.dec_crack_evolve(rule, 80, order=order, rtol=1e-12)
        res[rebuild] = (keff, ctx.dec_get_crack_iterations())
        # the row updates leave L and the preconditioner as a rebuild makes them
        _, _, val, b = ctx.dec_get_csr(0)
        g = ctx.dec_get_precond()
        res[("sys", rebuild)] = (val, b, g)
    np.testing.assert_allclose(res[False][0], res[True][0], rtol=0,
                               atol=1e-9 * res[True][0][0])
    assert res[False][1] < res[True][1]
    v0, b0, g0 = res[("sys", False)]
    v1, b1, g1 = res[("sys", True)]
    assert np.array_equal(v0, v1) and np.array_equal(b0, b1)
    np.testing.assert_allclose(g0, g1, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_ordered_growth_matches_oracle(abi, ctx, mode):
    wl = make_workload("lognormal64", N=6)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    order = np.random.default_rng(11).permutation(np.flatnonzero(O.crackable_edges(w)))[:30]
    ref = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                            rule="order", order=order, max_steps=30, rtol=1e-13)
    _setup(abi, ctx, wl, "fsai")
    md = abi.DEC_MODE_FP64 if mode == "fp64" else abi.DEC_MODE_MIXED
    st, cracked, keff = ctx.dec_crack_evolve(abi.DEC_CRACK_ORDER, 30, order=order,
                                             rtol=1e-12 if mode == "fp64" else 1e-11,
                                             mode=md)
    assert cracked.tolist() == order.tolist()
    np.testing.assert_allclose(keff, ref["k_eff"], rtol=0, atol=K_TOL * ref["k_eff0"])
    # the cracks stay in the context: its *1 state and k_eff are the last step's
    _, fc = ctx.dec_get_hodge()
    assert set(np.flatnonzero(fc == 0).tolist()) == set(order.tolist())
    q_in, _, _ = ctx.dec_k_eff()
    assert q_in[0] == keff[-1]


def test_ordered_growth_rejects_an_edge_that_is_already_cut(abi, ctx):
    wl = make_workload("lognormal64", N=5)
    _setup(abi, ctx, wl, "fsai")
    E, _ = ctx.dec_get_edges()
    w, _ = ctx.dec_get_hodge()
    a, b = np.flatnonzero(w > 0.0)[:2]
    order = np.array([a, b, a], dtype=np.int32)
    st, cracked, keff = ctx.dec_crack_evolve(abi.DEC_CRACK_ORDER, 3, order=order,
                                             raise_on_error=False)
    assert st == abi.DEC_ERR_ARG
    assert cracked.tolist() == [a, b]
    st, _, _ = ctx.dec_crack_evolve(abi.DEC_CRACK_ORDER, 1, order=np.array([len(E)]),
                                    raise_on_error=False)
    assert st == abi.DEC_ERR_ARG


# ------------------------------------------------- Monte-Carlo paths

def _orders(wl, P, S, seed):
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    cand = np.flatnonzero(O.crackable_edges(w))
    return np.stack([np.random.default_rng(seed + b).permutation(cand)[:S]
                     for b in range(P)]).astype(np.int32)


def test_monte_carlo_paths_match_oracle(abi, ctx):
    # Sec. 3.4: several random crack orders solved as one batch; every
    # path's k_eff after every step against the oracle's ordered cracking
    wl = make_workload("lognormal64", N=8)
    P, S = 6, 40
    orders = _orders(wl, P, S, 100)
    _setup(abi, ctx, wl, "fsai")
    st, keffs, steps = ctx.dec_crack_paths(orders, rtol=1e-11)
    assert (steps == S).all()
    for b in range(P):
        ref = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                                rule="order", order=orders[b], max_steps=S, rtol=1e-13)
        np.testing.assert_allclose(keffs[b], ref["k_eff"], rtol=0,
                                   atol=K_TOL * ref["k_eff0"])
    # the context keeps the paths as instances: dec_k_eff gives the last states
    q_in, _, _ = ctx.dec_k_eff()
    np.testing.assert_allclose(q_in, [k[-1] for k in keffs], rtol=1e-12)


def test_monte_carlo_paths_run_to_separation(abi, ctx):
    # each path stops at the step that separates the cube; the step count
    # per path equals the oracle's
    wl = make_workload("lognormal64", N=5)
    E, t2e = O.edge_list(wl.tets)
    w = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    ncand = int(O.crackable_edges(w).sum())
    P = 4
    orders = _orders(wl, P, ncand, 7)
    _setup(abi, ctx, wl, "fsai")
    st, keffs, steps = ctx.dec_crack_paths(orders, rtol=1e-11)
    for b in range(P):
        ref = O.crack_evolution(wl.xyz, wl.tets, wl.tags, wl.T0[0], k=wl.k,
                                rule="order", order=orders[b], max_steps=ncand,
                                rtol=1e-13)
        assert steps[b] == len(ref["k_eff"]) < ncand
        assert keffs[b][-1] <= 1e-9 * ref["k_eff0"]
        np.testing.assert_allclose(keffs[b][:-1], ref["k_eff"][:-1], rtol=0,
                                   atol=K_TOL * ref["k_eff0"])


def test_monte_carlo_paths_reject_a_repeated_edge(abi, ctx):
    wl = make_workload("lognormal64", N=5)
    orders = _orders(wl, 3, 5, 1)
    orders[1, 3] = orders[1, 1]                  # cracked twice in path 1
    _setup(abi, ctx, wl, "fsai")
    st, keffs, steps = ctx.dec_crack_paths(orders, raise_on_error=False)
    assert st == abi.DEC_ERR_ARG
    assert steps.tolist() == [3, 3, 3]
