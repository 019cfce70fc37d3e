"""The whole path through the C ABI, in the order the library requires:
mesh_upload -> hodge_assemble -> laplacian_build -> solve -> k_eff."""
from __future__ import annotations

import dataclasses

import numpy as np

from . import abi


@dataclasses.dataclass
class PathResult:
    status: int
    iters: np.ndarray
    relres: np.ndarray
    q_in: np.ndarray
    q_out: np.ndarray
    energy: np.ndarray
    T: np.ndarray | None


def run_path(ctx: abi.Context, xyz, tets, tags, T0, k=None, discs=None,
             scales=None, precond="fsai", mode="fp64", rtol=1e-10,
             max_iter=100000, want_T=True, raise_on_error=True) -> PathResult:
    """Run every step of the path on one mesh; inputs may be numpy arrays or
    torch CUDA tensors.  ``k`` is one per-tet field [n_tets] or a stack of
    fields [n_fields, n_tets] (one instance per field).  Returns iteration counts, residuals, k_eff pieces
    and (optionally) the temperature field of every instance."""
    ctx.dec_mesh_upload(xyz, tets, tags)
    if k is not None and len(k.shape) == 2:       # several conductivity fields
        if scales is not None:
            raise ValueError("conductivity fields and crack states at once")
        ctx.dec_hodge_assemble_fields(k, discs)
    else:
        ctx.dec_hodge_assemble(k, discs, scales)
    pc = {"fsai": abi.DEC_PRECOND_FSAI, "jacobi": abi.DEC_PRECOND_JACOBI,
          "fsai_shared": abi.DEC_PRECOND_FSAI_SHARED}[precond]
    if mode == "batched":
        pc = abi.DEC_PRECOND_FSAI_SHARED
    ctx.dec_laplacian_build(T0, pc)
    B = ctx.sizes()[4]
    n = len(xyz)
    T = np.zeros((B, n)) if want_T else None
    md = {"fp64": abi.DEC_MODE_FP64, "mixed": abi.DEC_MODE_MIXED,
          "mixed_phased": abi.DEC_MODE_MIXED_PHASED,
          "batched": abi.DEC_MODE_MIXED_BATCHED}[mode]
    st, iters, relres = ctx.dec_solve(rtol, max_iter, md, T,
                                      raise_on_error=raise_on_error)
    q_in, q_out, energy = ctx.dec_k_eff()
    return PathResult(st, iters, relres, q_in, q_out, energy, T)
