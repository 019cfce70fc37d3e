"""Crack growth on the GPU (dec_crack_evolve, Sec. 2.5, 3.3, 3.4) against
the FP64 oracle's crack_evolution.

Bars: the cracked edge ids are bit-exact, except where two candidates' face
fluxes lie within 1e-8 relative of each other in the oracle's solution (a
tie that FP64 solutions differing at the 1e-10 level may break either way;
the comparison stops there); k_eff after every step within 1e-8 of the
uncracked k_eff (k_eff falls to ~0 at separation, so the bar is absolute
in units of k_eff(uncracked)).
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
