"""The paper's own tet-centred form on the GPU (dec_tet_solve: Sec. 2.3,
Eq. 11-13 with the flux block eliminated; Sec. 3.1 limiter; Eq. 13 Neumann
flux; Whitney flux vectors) against the oracle's tet_centred_solve and
whitney_flux.  Bars: faces and the tet->face map bit-exact; potentials within
1e-8 relative L2 (the oracle solves directly, the GPU by FP64 PCG with FSAI
to 1e-11: the true residual of these small cracked systems levels off near
1e-12 in FP64); k_eff within 1e-8."""
import numpy as np
import pytest

import oracle as O
from dec_inputs import make_workload

pytestmark = pytest.mark.gpu


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


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name,N", [("lognormal64", 7), ("kuhn9", 5)])
def test_faces_match_oracle(ctx, name, N):
    wl = make_workload(name, N=N)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    faces, t2f = ctx.dec_tet_get_faces()
    ref = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0])
    assert np.array_equal(faces, ref["faces"])
    assert np.array_equal(t2f, ref["t2f"])


def test_linear_field_is_exact_without_the_limiter(ctx):
    # Sec. 3.1: where nothing is limited the form reproduces T = 1 - x at
    # every circumcentre and k_eff = 1
    wl = make_workload("lognormal64", N=7)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    res = ctx.dec_tet_solve(wl.T0[0], limiter=1e-8, rtol=1e-11)
    ref = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0], limiter=1e-8)
    assert res["limited"] == ref["limited"] == 0
    np.testing.assert_allclose(res["alpha"], 1.0 - ref["cT"][:, 0], atol=1e-10)
    assert res["q_in"] == pytest.approx(1.0, rel=1e-9)
    assert res["q_out"] == pytest.approx(1.0, rel=1e-9)


def test_kuhn_limiter_matches_oracle(ctx):
    # the Kuhn lattice has 6 (N-1)^3 zero-length dual edges: the limiter
    # acts on all of them, on both sides alike.  The six tets of each cube
    # are then joined by w = 1/1e-8 against w ~ h elsewhere, so b - A x
    # carries rounding of about 1e8 * 1e-16 per row: in FP64 the relative
    # residual cannot go much below 1e-7 (the oracle's direct solution has
    # 1.8e-7 at N = 5, and a plain FP64 Jacobi CG levels off at 5.6e-7,
    # 1.2e-7 from it), so this case solves to 1e-6 and compares to 1e-6.
    N = 5
    wl = make_workload("kuhn9", N=N)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    res = ctx.dec_tet_solve(wl.T0[0], limiter=1e-8, rtol=1e-6)
    ref = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0], limiter=1e-8)
    assert res["limited"] == ref["limited"] == 6 * (N - 1) ** 3
    assert res["relres"] <= 1e-6
    assert _rel(res["alpha"], ref["alpha"]) <= 1e-6
    assert res["q_in"] == pytest.approx(ref["q_in"], rel=1e-6)


def test_cracked_faces_and_cut_off_tets(ctx):
    wl = make_workload("lognormal64", N=8)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    base = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0])
    inner = np.flatnonzero(base["interior"])
    t2f = base["t2f"]
    T = int(np.flatnonzero(base["interior"][t2f].all(axis=1))[0])
    cracked = np.unique(np.r_[np.random.default_rng(3).choice(inner, 300, replace=False), t2f[T]])
    ref = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0], cracked_faces=cracked)
    res = ctx.dec_tet_solve(wl.T0[0], cracked_faces=cracked, rtol=1e-11)
    assert res["alpha"][T] == 0.0 and ref["alpha"][T] == 0.0
    assert _rel(res["alpha"], ref["alpha"]) <= 1e-8
    assert res["q_in"] == pytest.approx(ref["q_in"], rel=1e-8)
    assert res["q_out"] == pytest.approx(ref["q_out"], rel=1e-8)
    assert res["q_in"] < base["q_in"]


def test_neumann_flux_and_whitney_vectors(ctx):
    # Eq. 13: x = 1 becomes a flux boundary carrying the linear field's
    # outflow; the solution stays linear and the Whitney vectors are (1, 0, 0)
    wl = make_workload("lognormal64", N=6)
    tags = wl.tags.copy()
    tags[wl.xyz[:, 0] == 1.0] = 2
    ctx.dec_mesh_upload(wl.xyz, wl.tets, tags)
    base = O.tet_centred_solve(wl.xyz, wl.tets, tags, wl.T0[0])
    P = wl.xyz[base["faces"]]
    flux = np.where((P[:, :, 0] == 1.0).all(axis=1), base["area"], 0.0)
    ref = O.tet_centred_solve(wl.xyz, wl.tets, tags, wl.T0[0], face_flux=flux)
    res = ctx.dec_tet_solve(wl.T0[0], face_flux=flux, rtol=1e-11)
    assert _rel(res["alpha"], ref["alpha"]) <= 1e-8
    np.testing.assert_allclose(res["alpha"], 1.0 - ref["cT"][:, 0], atol=1e-9)
    v = ctx.dec_tet_whitney()
    np.testing.assert_allclose(v, O.whitney_flux(wl.xyz, wl.tets, ref), atol=1e-8)
    np.testing.assert_allclose(v, np.tile([1.0, 0.0, 0.0], (len(wl.tets), 1)), atol=1e-8)


def test_whitney_with_cracks_matches_oracle(ctx):
    wl = make_workload("lognormal64", N=7)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    base = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0])
    cracked = np.random.default_rng(4).choice(np.flatnonzero(base["interior"]), 200,
                                              replace=False)
    ref = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0], cracked_faces=cracked,
                              kappa=2.5)
    res = ctx.dec_tet_solve(wl.T0[0], kappa=2.5, cracked_faces=cracked, rtol=1e-11)
    assert _rel(res["alpha"], ref["alpha"]) <= 1e-8
    vref = O.whitney_flux(wl.xyz, wl.tets, ref)
    v = ctx.dec_tet_whitney()
    assert np.linalg.norm(v - vref) <= 1e-8 * np.linalg.norm(vref)


def test_tet_solve_arguments(abi, ctx):
    wl = make_workload("lognormal64", N=5)
    with pytest.raises(abi.DecError) as e:
        ctx.dec_tet_whitney()
    assert e.value.status in (abi.DEC_ERR_STATE, abi.DEC_ERR_ARG)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    with pytest.raises(abi.DecError) as e:
        ctx.dec_tet_solve(wl.T0[0], cracked_faces=np.array([10 ** 8]))
    assert e.value.status == abi.DEC_ERR_ARG
    with pytest.raises(abi.DecError) as e:
        ctx.dec_tet_solve(wl.T0[0], kappa=-1.0)
    assert e.value.status == abi.DEC_ERR_ARG


def test_device_inputs_match_host_inputs(ctx):
    # T0, cracked faces and face fluxes may be CUDA tensors, as for the
    # other entry points; the result equals the host-array call bit for bit
    import torch
    wl = make_workload("lognormal64", N=6)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    faces, _ = ctx.dec_tet_get_faces()
    cracked = np.arange(0, len(faces), 7, dtype=np.int32)
    host = ctx.dec_tet_solve(wl.T0[0], cracked_faces=cracked, rtol=1e-11)
    dev = torch.device("cuda", 0)
    res = ctx.dec_tet_solve(torch.from_numpy(wl.T0[0].copy()).to(dev),
                            cracked_faces=torch.from_numpy(cracked).to(dev), rtol=1e-11)
    assert np.array_equal(res["alpha"], host["alpha"])
    assert res["q_in"] == host["q_in"]


def test_cut_off_pair_keeps_zero_potential(ctx):
    # two neighbouring tets cut off from the rest by cracks on their other
    # six faces: a singular 2x2 block with zero right-hand side (the FSAI
    # factor meets a zero pivot there and takes the shifted factorisation);
    # both potentials stay 0, as the oracle's anchored solve gives, and the
    # rest matches the oracle
    wl = make_workload("lognormal64", N=8)
    ctx.dec_mesh_upload(wl.xyz, wl.tets, wl.tags)
    base = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0])
    t2f, owner = base["t2f"], base["owner"]
    inner = base["interior"]
    T1 = next(t for t in range(len(wl.tets)) if inner[t2f[t]].all()
              and all(inner[t2f[o]].all() for o in owner[t2f[t]].ravel() if o != t))
    f = t2f[T1][0]
    T2 = int(owner[f][0] if owner[f][1] == T1 else owner[f][1])
    cracked = np.setdiff1d(np.r_[t2f[T1], t2f[T2]], [f]).astype(np.int32)
    ref = O.tet_centred_solve(wl.xyz, wl.tets, wl.tags, wl.T0[0], cracked_faces=cracked)
    res = ctx.dec_tet_solve(wl.T0[0], cracked_faces=cracked, rtol=1e-11)
    assert ref["alpha"][T1] == 0.0 and ref["alpha"][T2] == 0.0
    assert res["alpha"][T1] == 0.0 and res["alpha"][T2] == 0.0
    assert _rel(res["alpha"], ref["alpha"]) <= 1e-8
