"""The FP32 geometry of well-shaped tets (DEC_GEOM_MIXED, the circumcentric
Hodge star of Sec. 2.1 computed in FP32 where L^3 <= 16 |6V|) against the
FP64 oracle, beside the FP64 geometry.

Bars, per result: FP64 geometry as in the parity tests (*1 to 1e-12 of the
largest weight); FP32 geometry *1 to 2e-6 of the largest weight on every
edge and 1e-6 relative L2 (a CPU emulation of the same formulas in FP32 on
these meshes gives 1.8e-7 and 8.6e-8); crack states identical to the FP64
geometry's, bit for bit (the FP32 circumcentre is only a filter with an
error bound); k_eff within 1e-6 of the oracle (against 1e-8 with FP64
geometry)."""
import numpy as np
import pytest

import oracle as O
from dec_inputs import make_workload

pytestmark = pytest.mark.gpu

W64_ATOL = 1e-12      # of the largest |*1|, FP64 geometry
W32_ATOL = 2e-6       # of the largest |*1|, FP32 geometry
W32_L2 = 1e-6
K32_RTOL = 1e-6


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


@pytest.mark.parametrize("name,N,cracked", [("lognormal64", 24, False),
                                            ("hetero192", 20, True),
                                            ("kuhn9", None, False)])
def test_mixed_geometry_hodge_star(abi, ctx, name, N, cracked):
    wl = make_workload(name, N=N)
    discs = wl.discs if cracked else None
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    E, t2e = O.edge_list(wl.tets)
    wo = O.hodge_star1(wl.xyz, wl.tets, E, t2e, wl.k)
    scale = np.abs(wo).max()
    ctx.dec_set_geom_precision(abi.DEC_GEOM_FP64)
    ctx.dec_hodge_assemble(wl.k, discs)
    w64, fc64 = ctx.dec_get_hodge()
    assert ctx.dec_get_geom_fp64_tets() == wl.m
    ctx.dec_set_geom_precision(abi.DEC_GEOM_MIXED)
    ctx.dec_hodge_assemble(wl.k, discs)
    w32, fc32 = ctx.dec_get_hodge()
    n64 = ctx.dec_get_geom_fp64_tets()
    # dec_get_hodge reports the uncracked *1 and, separately, the crack states
    if cracked:
        assert (fc64 == 0).sum() > 0
        assert np.array_equal(fc32, fc64)
    err64 = np.abs(w64 - wo).max() / scale
    err32 = np.abs(w32 - wo).max() / scale
    l2 = np.linalg.norm(w32 - wo) / np.linalg.norm(wo)
    print(f"{name}: FP64 tets {n64} of {wl.m}; *1 error (of max) FP64 {err64:.2e}, "
          f"FP32 {err32:.2e}, FP32 L2 {l2:.2e}")
    assert err64 <= W64_ATOL
    assert err32 <= W32_ATOL and l2 <= W32_L2
    if name == "kuhn9":
        assert n64 == 0                       # every Kuhn tet is well shaped
    else:
        assert 0 < n64 < 0.1 * wl.m           # slivers stay in FP64


def test_mixed_geometry_k_eff(abi, ctx):
    from paper_2104_05999_gb300 import run
    wl = make_workload("hetero192", N=14)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k, discs=wl.discs,
                       precond="fsai", rtol=1e-13)
    ctx.dec_set_geom_precision(abi.DEC_GEOM_MIXED)
    res = run.run_path(ctx, wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k, discs=wl.discs,
                       mode="batched", rtol=1e-10, want_T=False)
    rel = np.abs(res.q_in - ref["q_in"]) / np.abs(ref["q_in"]).max()
    print("k_eff relative error per set, FP32 geometry:", rel)
    assert rel.max() <= K32_RTOL
