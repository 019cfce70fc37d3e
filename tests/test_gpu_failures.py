"""Failure paths of the CUDA library, reached without any GPU fault.

* DEC_ERR_TIMEOUT: the persistent solves wait at grid barriers that poll a
  bounded number of times.  dec_set_barrier_test shortens the bound and
  withholds one block, so the other blocks' wait runs out: the call must
  return DEC_ERR_TIMEOUT (no hang, no fault) and the context must still give
  the oracle's answer once the switch is off.
* DEC_ERR_BREAKDOWN: a valid but strongly obtuse tet has a node whose
  circumcentric dual volume is negative (Sec. 2.1, signed dual pieces), so
  the free node's Laplacian row is negative and CG meets p.Lp < 0 at once.
"""
import numpy as np
import pytest

import oracle as O
from dec_inputs import make_workload

pytestmark = pytest.mark.gpu

SPIN = 4096          # polls of 32-256 ns: about a millisecond per wait


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
    ctx.dec_hodge_assemble(wl.k, wl.discs, wl.scales)
    ctx.dec_laplacian_build(wl.T0, precond)


def test_persistent_mixed_solve_times_out_and_recovers(abi, ctx):
    wl = make_workload("lognormal64", N=10)
    _setup(abi, ctx, wl, abi.DEC_PRECOND_FSAI)
    ctx.dec_set_barrier_test(SPIN, 1)
    st, _, _ = ctx.dec_solve(1e-10, 5000, abi.DEC_MODE_MIXED, raise_on_error=False)
    assert st == abi.DEC_ERR_TIMEOUT
    ctx.dec_set_barrier_test(0, 0)
    T = np.zeros((1, wl.n))
    st, it, rr = ctx.dec_solve(1e-10, 5000, abi.DEC_MODE_MIXED, T)
    assert st == abi.DEC_OK and rr[0] <= 1e-10
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       precond="fsai", rtol=1e-13)
    assert np.linalg.norm(T[0] - ref["T"][0]) <= 1e-8 * np.linalg.norm(ref["T"][0])
    q_in, _, _ = ctx.dec_k_eff()
    assert q_in[0] == pytest.approx(ref["q_in"][0], rel=1e-8)


def test_batched_solve_times_out_and_recovers(abi, ctx):
    wl = make_workload("growth96", N=8, n_discs=5, n_scales=6)
    _setup(abi, ctx, wl, abi.DEC_PRECOND_FSAI_SHARED)
    ctx.dec_set_barrier_test(SPIN, 1)
    for _ in range(2):     # first call: autotuner launches; second: tuned
        st, _, _ = ctx.dec_solve(1e-10, 5000, abi.DEC_MODE_MIXED_BATCHED,
                                 raise_on_error=False)
        assert st == abi.DEC_ERR_TIMEOUT
    ctx.dec_set_barrier_test(0, 0)
    T = np.zeros((len(wl.scales), wl.n))
    st, it, rr = ctx.dec_solve(1e-10, 5000, abi.DEC_MODE_MIXED_BATCHED, T)
    assert st == abi.DEC_OK and (rr <= 1e-10).all()
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k, discs=wl.discs,
                       scales=wl.scales, precond="fsai", rtol=1e-13)
    q_in, _, _ = ctx.dec_k_eff()
    np.testing.assert_allclose(q_in, ref["q_in"], rtol=1e-8)


def test_short_spin_limit_alone_changes_nothing(abi, ctx):
    # every block present: a generous but finite poll limit must not fire
    wl = make_workload("lognormal64", N=9)
    _setup(abi, ctx, wl, abi.DEC_PRECOND_FSAI)
    T0 = np.zeros((1, wl.n))
    ctx.dec_solve(1e-10, 5000, abi.DEC_MODE_MIXED, T0)
    ctx.dec_set_barrier_test(1 << 22, 0)
    T1 = np.zeros((1, wl.n))
    ctx.dec_solve(1e-10, 5000, abi.DEC_MODE_MIXED, T1)
    ctx.dec_set_barrier_test(0, 0)
    assert np.array_equal(T0, T1)


def test_barrier_test_arguments(abi, ctx):
    for bad in ((-1, 0), (1 << 32, 0), (10, 2)):
        with pytest.raises(abi.DecError) as e:
            ctx.dec_set_barrier_test(*bad)
        assert e.value.status == abi.DEC_ERR_ARG


OBTUSE = np.array([[0.92, 0.36, 0.79], [0.09, 0.82, 0.16],
                   [0.23, 0.08, 0.92], [0.17, 0.31, 0.67]])


def test_negative_dual_volume_gives_breakdown(abi, ctx):
    tets = np.array([[0, 1, 3, 2]], dtype=np.int32)      # positively oriented
    assert O.tet_volumes(OBTUSE, tets)[0] > 0
    tags = np.array([1, 1, 1, 0], dtype=np.uint8)       # node 3 free
    T0 = np.array([[1.0, 0.0, 0.0, 0.0]])
    E, t2e = O.edge_list(tets)
    w = O.hodge_star1(OBTUSE, tets, E, t2e)
    L, b, _ = O.laplacian(4, E, w, tags, T0)
    assert L[3, 3] < 0 and b[0, 3] != 0                  # indefinite 1x1 system
    ctx.dec_mesh_upload(np.ascontiguousarray(OBTUSE), tets, tags)
    ctx.dec_hodge_assemble(None)
    ctx.dec_laplacian_build(T0, abi.DEC_PRECOND_JACOBI)
    st, _, _ = ctx.dec_solve(1e-10, 100, abi.DEC_MODE_FP64, raise_on_error=False)
    assert st == abi.DEC_ERR_BREAKDOWN
    # the context stays usable: a valid mesh solves afterwards
    wl = make_workload("kuhn9", N=5)
    _setup(abi, ctx, wl, abi.DEC_PRECOND_JACOBI)
    T = np.zeros((1, wl.n))
    ctx.dec_solve(1e-12, 1000, abi.DEC_MODE_FP64, T)
    np.testing.assert_allclose(T[0], 1.0 - wl.xyz[:, 0], atol=1e-10)
