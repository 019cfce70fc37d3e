"""Boundary tags, Dirichlet values, conductivity fields and penny discs.

The paper's test problem (Sec. 2.5) is a unit cube with temperatures 1 and 0
prescribed on two opposite faces and zero flux on the other four.  Here the
Dirichlet faces are x = 0 (T0 = 1) and x = 1 (T0 = 0).  Nodes on cube edges
and corners that lie on an x face count as Dirichlet; every other boundary
node is a zero-flux (Neumann) node.

Cracks (Sec. 2.5: a crack turns a face's conductivity to zero) are supplied as
penny-shaped discs, each row ``cx, cy, cz, nx, ny, nz, r`` with a unit normal.
"""
from __future__ import annotations

import numpy as np

FREE, DIRICHLET, NEUMANN = 0, 1, 2


def node_tags(xyz: np.ndarray) -> np.ndarray:
    x = xyz[:, 0]
    onb = ((xyz == 0.0) | (xyz == 1.0)).any(axis=1)
    tag = np.where(onb, NEUMANN, FREE).astype(np.uint8)
    tag[(x == 0.0) | (x == 1.0)] = DIRICHLET
    return tag


def dirichlet_values(xyz: np.ndarray, tags: np.ndarray, n_sets: int = 1,
                     rng: np.random.Generator | None = None) -> np.ndarray:
    """``[n_sets, n]`` Dirichlet values.  Set 0 is the paper's problem:
    T0 = 1 on x = 0, 0 on x = 1.  Further sets draw T0 ~ U[0, 1] per Dirichlet
    node.  Entries at non-Dirichlet nodes are 0 and unused."""
    n = len(xyz)
    T0 = np.zeros((n_sets, n), dtype=np.float64)
    d = tags == DIRICHLET
    T0[0, d & (xyz[:, 0] == 0.0)] = 1.0
    for s in range(1, n_sets):
        T0[s, d] = rng.uniform(0.0, 1.0, size=int(d.sum()))
    return T0


def lognormal_conductivity(m: int, sigma: float,
                           rng: np.random.Generator) -> np.ndarray:
    """Per-tet conductivity k = exp(sigma * N(0, 1))."""
    return np.exp(sigma * rng.standard_normal(m))


def conductivity_fields(m: int, n_fields: int, sigma: float,
                        rng: np.random.Generator) -> np.ndarray:
    """``n_fields`` independent per-tet lognormal fields, ``f64[n_fields, m]``
    (field f, tet t: exp(sigma * N(0, 1)))."""
    return np.exp(sigma * rng.standard_normal((n_fields, m)))


def penny_discs(nd: int, rmin: float, rmax: float,
                rng: np.random.Generator) -> np.ndarray:
    """nd discs: centre U[0,1]^3, normal uniform on the sphere (normalised
    Gaussian), radius U[rmin, rmax].  Returns ``f64[nd, 7]``."""
    c = rng.uniform(0.0, 1.0, size=(nd, 3))
    nrm = rng.standard_normal((nd, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r = rng.uniform(rmin, rmax, size=nd)
    return np.ascontiguousarray(np.concatenate([c, nrm, r[:, None]], axis=1))


def crack_scales(B: int, s0: float = 0.2, s1: float = 1.0) -> np.ndarray:
    """Radius scale of each crack state of a growing population:
    linear from s0 to s1 over B states."""
    if B == 1:
        return np.array([s1])
    return s0 + (s1 - s0) * np.arange(B, dtype=np.float64) / (B - 1)
