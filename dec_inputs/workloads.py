"""Named workloads: a mesh plus the fields one solve needs.

The five production workloads are the unit-cube problems of the paper's
study (Sec. 2.5, Sec. 3.1-3.4) at the sizes this library is measured on:

  kuhn9        9^3 Kuhn lattice, k = 1, Jacobi PCG to 1e-12 (exact T = 1 - x)
  lognormal64  64^3 jittered Delaunay, k = exp(N(0,1)) per tet
  cracked128   128^3 jittered Delaunay, k = 1, 2000 penny discs
  growth96     96^3 jittered Delaunay, 1500 discs, 64 radius scales
  hetero192    192^3 jittered Delaunay, k = exp(1.5 N(0,1)), 5000 discs,
               8 Dirichlet value sets

Each is seeded with ``1000 + index``; every random draw comes from its own
child stream of that seed (jitter, conductivity, discs, Dirichlet values), so
a workload's inputs do not depend on what else was generated.  Smaller
variants keep the same recipe at another lattice size (``N=...``).

Meshes are cached on disk (``DEC_INPUT_CACHE`` or ``~/.cache/dec_inputs``)
because the Delaunay step dominates input generation.
"""
from __future__ import annotations

import dataclasses
import hashlib
import os

import numpy as np

from .fields import (conductivity_fields, crack_scales, dirichlet_values,
                     lognormal_conductivity, node_tags, penny_discs)
from .mesh import delaunay_lattice, jittered_lattice, kuhn_lattice


@dataclasses.dataclass
class Workload:
    name: str
    N: int
    xyz: np.ndarray            # f64[n, 3]
    tets: np.ndarray           # i32[m, 4], positively oriented
    tags: np.ndarray           # u8[n]: 0 free, 1 Dirichlet, 2 zero flux
    T0: np.ndarray             # f64[n_sets, n] Dirichlet values
    k: np.ndarray | None       # f64[m] per-tet conductivity, None = 1
    discs: np.ndarray | None   # f64[nd, 7] penny discs, None = no cracks
    scales: np.ndarray | None  # f64[B] disc radius scales, None = [1]
    rtol: float                # relative residual the solve stops at
    precond: str               # "jacobi" | "fsai"
    mode: str                  # "fp64" | "mixed" | "batched"

    @property
    def n(self) -> int:
        return len(self.xyz)

    @property
    def m(self) -> int:
        return len(self.tets)

    @property
    def batch(self) -> int:
        if self.scales is not None:
            return len(self.scales)
        return self.T0.shape[0]


# name -> (index, default N, kind, sigma, n_discs, (rmin, rmax), n_scales,
#          n_dirichlet_sets, rtol, precond, mode)
WORKLOADS = {
    "kuhn9":       (0, 9,   "kuhn",     0.0, 0,    None,          0,  1, 1e-12, "jacobi", "fp64"),
    "lognormal64": (1, 64,  "delaunay", 1.0, 0,    None,          0,  1, 1e-10, "fsai",   "fp64"),
    "cracked128":  (2, 128, "delaunay", 0.0, 2000, (0.02, 0.06),  0,  1, 1e-10, "fsai",   "mixed"),
    "growth96":    (3, 96,  "delaunay", 0.0, 1500, (0.02, 0.05),  64, 1, 1e-10, "fsai",   "batched"),
    "hetero192":   (4, 192, "delaunay", 1.5, 5000, (0.02, 0.06),  0,  8, 1e-10, "fsai",   "batched"),
}


def _cache_dir() -> str:
    d = os.environ.get("DEC_INPUT_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "dec_inputs")
    os.makedirs(d, exist_ok=True)
    return d


def _delaunay_mesh(N: int, seed: int, jitter: float, rng_jit):
    xyz = jittered_lattice(N, rng_jit, jitter)
    tag = hashlib.sha1(xyz.tobytes()).hexdigest()[:16]
    path = os.path.join(_cache_dir(), f"delaunay_N{N}_s{seed}_{tag}.npz")
    if os.path.exists(path):
        try:
            with np.load(path) as z:
                return xyz, z["tets"]
        except Exception:
            pass
    tets = delaunay_lattice(xyz, N, jitter)
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, tets=tets)
    os.replace(tmp, path)
    return xyz, tets


def make_workload(name: str, N: int | None = None, n_discs: int | None = None,
                  n_scales: int | None = None, n_sets: int | None = None,
                  jitter: float = 0.2) -> Workload:
    """Build a named workload, optionally at another lattice size N.

    When N is smaller than the default, disc radii are scaled by
    N_default / N and the disc count by (N / N_default)^3 unless given, so
    that about the same share of dual faces is cut.
    """
    (idx, N0, kind, sigma, nd0, rr, nsc, nset, rtol, precond,
     mode) = WORKLOADS[name]
    N = N0 if N is None else int(N)
    seed = 1000 + idx
    ss = np.random.SeedSequence(seed).spawn(4)
    rng_jit, rng_k, rng_disc, rng_T0 = (np.random.default_rng(s) for s in ss)
    if kind == "kuhn":
        xyz, tets = kuhn_lattice(N)
    else:
        xyz, tets = _delaunay_mesh(N, seed, jitter, rng_jit)
    tags = node_tags(xyz)
    T0 = dirichlet_values(xyz, tags, nset if n_sets is None else n_sets,
                          rng_T0)
    k = lognormal_conductivity(len(tets), sigma, rng_k) if sigma > 0 else None
    discs = None
    if nd0:
        f = N0 / N
        nd = n_discs if n_discs is not None else max(
            1, int(round(nd0 / f ** 3)))
        discs = penny_discs(nd, rr[0] * f, rr[1] * f, rng_disc)
    scales = None
    if nsc:
        scales = crack_scales(nsc if n_scales is None else n_scales)
    return Workload(name=name if N == N0 else f"{name}@{N}", N=N, xyz=xyz,
                    tets=tets, tags=tags, T0=T0, k=k, discs=discs,
                    scales=scales, rtol=rtol, precond=precond, mode=mode)


def make_fields(wl: Workload, n_fields: int, sigma: float = 1.0) -> np.ndarray:
    """``n_fields`` lognormal conductivity fields on the mesh of ``wl``
    (many material fields on one mesh), drawn from their own child stream of
    the workload's seed, so the workload's other inputs are unchanged."""
    idx = WORKLOADS[wl.name.split("@")[0]][0]
    rng = np.random.default_rng(np.random.SeedSequence(1000 + idx).spawn(5)[4])
    return conductivity_fields(wl.m, n_fields, sigma, rng)
