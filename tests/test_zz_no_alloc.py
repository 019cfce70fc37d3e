"""The entry point that allocates no device memory.

Some callers cannot let a library allocate device memory (a framework that
owns every device allocation through its own pool, a fixed memory budget).
dec_k_eff_edges_noalloc serves them: it takes arrays the caller already
holds and keeps its scratch in a fixed array inside the library.  This test
calls it through the C ABI twice in a row and checks both results against
dec_k_eff of a context on the same solved field.  It lives in its own file,
collected last, so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_k_eff_matches_context_entry_point_twice():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from dec_inputs import make_workload
    from paper_2104_05999_gb300 import _build, abi, run_path

    _build.build()
    wl = make_workload("lognormal64", N=14)
    with abi.Context(device=0) as ctx:
        res = run_path(ctx, wl.xyz, wl.tets, wl.tags, wl.T0, k=wl.k,
                       precond="fsai", mode="fp64", rtol=1e-12)
        E, _ = ctx.dec_get_edges()
        w, _ = ctx.dec_get_hodge()
    want = np.array([res.q_in[0], res.q_out[0], res.energy[0]])
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d_E, d_w, d_T = t(E), t(w), t(res.T[0])
    d_xyz, d_tag = t(wl.xyz), t(wl.tags)
    torch.cuda.synchronize()
    for call in range(2):
        free0 = torch.cuda.mem_get_info(0)[0]
        got = abi.dec_k_eff_edges_noalloc(0, d_E, d_w, d_T, d_xyz, d_tag)
        # same sums in another order: FP64 rounding only
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-14)
        if call == 1:      # the first call may load the module's code
            assert torch.cuda.mem_get_info(0)[0] == free0
    # a size beyond the fixed scratch is refused before any launch
    out = np.zeros(3)
    st = abi.load().dec_k_eff_edges_noalloc(
        0, None, d_E.data_ptr(), 67108864 + 1, d_w.data_ptr(), d_T.data_ptr(),
        d_xyz.data_ptr(), d_tag.data_ptr(), out.ctypes.data)
    assert st == abi.DEC_ERR_LIMIT
    # a device index beyond the devices present is an argument error
    st = abi.load().dec_k_eff_edges_noalloc(
        torch.cuda.device_count(), None, d_E.data_ptr(), 10, d_w.data_ptr(),
        d_T.data_ptr(), d_xyz.data_ptr(), d_tag.data_ptr(), out.ctypes.data)
    assert st == abi.DEC_ERR_ARG
