"""Several conductivity fields on one mesh (Sec. 1: many material fields
share a mesh; Sec. 2.1: conductivity lives on the dual 2-cells), solved as
instances: per-instance FP64 PCG and the batched mixed solve, against the
FP64 oracle (T within 1e-8 relative L2, k_eff within 1e-8)."""
import numpy as np
import pytest

import oracle as O
from dec_inputs import make_fields, make_workload

pytestmark = pytest.mark.gpu

T_RTOL = 1e-8
K_RTOL = 1e-8


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


def test_field_stars_equal_single_field_assembly_bit_for_bit(abi, ctx):
    wl = make_workload("lognormal64", N=9)
    k = make_fields(wl, 5, sigma=1.2)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    ctx.dec_hodge_assemble_fields(k, wl.discs)
    ctx.dec_laplacian_build(wl.T0, abi.DEC_PRECOND_FSAI)
    with abi.Context(device=0) as one:
        one.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
        for f in range(5):
            one.dec_hodge_assemble(np.ascontiguousarray(k[f]), wl.discs)
            one.dec_laplacian_build(wl.T0, abi.DEC_PRECOND_FSAI)
            _, _, v1, b1 = one.dec_get_csr(0)
            _, _, vf, bf = ctx.dec_get_csr(f)
            assert np.array_equal(v1, vf) and np.array_equal(b1, bf)


@pytest.mark.parametrize("mode,precond", [("fp64", "fsai"), ("mixed", "fsai"),
                                          ("batched", "fsai_shared")])
def test_fields_match_oracle(abi, ctx, mode, precond):
    from paper_2104_05999_gb300 import run_path
    wl = make_workload("hetero192", N=10, n_sets=1)
    k = make_fields(wl, 6, sigma=1.5)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=k, discs=wl.discs,
                       precond="fsai", rtol=1e-13)
    res = run_path(ctx, wl.xyz, wl.tets, wl.tags, wl.T0, k=k, discs=wl.discs,
                   precond=precond, mode=mode, rtol=1e-10, max_iter=50000)
    assert len(res.q_in) == 6 and (res.relres <= 1e-10).all()
    for f in range(6):
        Tr = ref["T"][f]
        assert np.linalg.norm(res.T[f] - Tr) / np.linalg.norm(Tr) <= T_RTOL
    np.testing.assert_allclose(res.q_in, ref["q_in"], rtol=K_RTOL)
    np.testing.assert_allclose(res.energy, ref["energy"], rtol=K_RTOL)


def test_batched_fields_widest_stride(abi, ctx):
    # 40 fields: stride 64, 16 threads per row
    from paper_2104_05999_gb300 import run_path
    wl = make_workload("lognormal64", N=8)
    k = make_fields(wl, 40, sigma=1.0)
    ref = O.solve_path(wl.xyz, wl.tets, wl.tags, wl.T0, k=k, precond="fsai",
                       rtol=1e-13)
    res = run_path(ctx, wl.xyz, wl.tets, wl.tags, wl.T0, k=k, mode="batched",
                   rtol=1e-10, max_iter=50000)
    np.testing.assert_allclose(res.q_in, ref["q_in"], rtol=K_RTOL)


def test_fields_argument_checks(abi, ctx):
    wl = make_workload("lognormal64", N=6)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    bad = make_fields(wl, 2)
    bad[1, 3] = -1.0
    with pytest.raises(abi.DecError) as e:
        ctx.dec_hodge_assemble_fields(bad)
    assert e.value.status == abi.DEC_ERR_ARG
    with pytest.raises(abi.DecError) as e:
        ctx.dec_hodge_assemble_fields(make_fields(wl, 65))
    assert e.value.status == abi.DEC_ERR_LIMIT
    ctx.dec_hodge_assemble_fields(make_fields(wl, 3))
    with pytest.raises(abi.DecError) as e:      # fields and several T0 sets
        ctx.dec_laplacian_build(np.repeat(wl.T0, 2, axis=0), abi.DEC_PRECOND_FSAI)
    assert e.value.status == abi.DEC_ERR_ARG
