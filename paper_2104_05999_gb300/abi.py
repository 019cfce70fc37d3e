"""ctypes binding of the C ABI in ``include/dec.h`` (libdec_gb300.so).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays may be numpy arrays (host memory) or torch CUDA tensors
(device memory of the context's GPU); they must be C-contiguous and of the
dtype the C declaration names.  Every call raises ``DecError`` on a non-OK
status.  Loading fails loudly when the compiled library is missing: there is
no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import lib_path

DEC_OK = 0
DEC_ERR_ARG = 1
DEC_ERR_MESH = 2
DEC_ERR_CUDA = 3
DEC_ERR_BREAKDOWN = 4
DEC_NOT_CONVERGED = 5
DEC_ERR_TIMEOUT = 6
DEC_ERR_STATE = 7
DEC_ERR_LIMIT = 8
STATUS_NAMES = {
    0: "DEC_OK", 1: "DEC_ERR_ARG", 2: "DEC_ERR_MESH", 3: "DEC_ERR_CUDA",
    4: "DEC_ERR_BREAKDOWN", 5: "DEC_NOT_CONVERGED", 6: "DEC_ERR_TIMEOUT",
    7: "DEC_ERR_STATE", 8: "DEC_ERR_LIMIT"}

DEC_NODE_FREE, DEC_NODE_DIRICHLET, DEC_NODE_NEUMANN = 0, 1, 2
DEC_PRECOND_JACOBI, DEC_PRECOND_FSAI, DEC_PRECOND_FSAI_SHARED = 0, 1, 2
DEC_MODE_FP64, DEC_MODE_MIXED, DEC_MODE_MIXED_PHASED, DEC_MODE_MIXED_BATCHED = 0, 1, 2, 3
DEC_KERNEL_SPMV_F64, DEC_KERNEL_SPMV_F32 = 0, 1
DEC_KERNEL_FSAI_F64, DEC_KERNEL_FSAI_BF16 = 2, 3
DEC_CRACK_MAX_FLUX, DEC_CRACK_ORDER, DEC_CRACK_REBUILD = 0, 1, 16
DEC_GEOM_FP64, DEC_GEOM_MIXED = 0, 1

_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_D = C.c_double

# name -> (argtypes); all return dec_status (int)
SIGNATURES = {
    "dec_create": [C.POINTER(_P), C.c_int, _P],
    "dec_destroy": [_P],
    "dec_mesh_upload": [_P, _P, _I64, _P, _I64, _P],
    "dec_hodge_assemble": [_P, _P, _P, _I64, _P, _I32],
    "dec_hodge_assemble_fields": [_P, _P, _I32, _P, _I64],
    "dec_laplacian_build": [_P, _P, _I32, _I32],
    "dec_solve": [_P, _D, _I32, _I32, _P, _P, _P],
    "dec_k_eff": [_P, _P, _P, _P],
    "dec_crack_evolve": [_P, _I32, _I32, _P, _D, _I32, _I32, _D, _P, _P, _P],
    "dec_get_batch_variant": [_P, _P],
    "dec_get_batch_kernel_ms": [_P, _P],
    "dec_get_batch_phase_ms": [_P, _P],
    "dec_get_crack_iterations": [_P, _P],
    "dec_crack_paths": [_P, _I32, _I32, _P, _D, _I32, _D, _P, _P],
    "dec_tet_solve": [_P, _P, _D, _D, _P, _I64, _P, _D, _I32, _P, _P, _P, _P, _P],
    "dec_tet_get_faces": [_P, _P, _P, _P],
    "dec_tet_whitney": [_P, _P],
    "dec_get_sizes": [_P, _P, _P, _P, _P, _P],
    "dec_get_edges": [_P, _P, _P],
    "dec_get_hodge": [_P, _P, _P],
    "dec_get_csr": [_P, _I32, _P, _P, _P, _P],
    "dec_get_precond": [_P, _P],
    "dec_time_kernel": [_P, _I32, _I32, _I64, _P],
    "dec_get_launch_count": [_P, _P],
    "dec_set_barrier_test": [_P, _I64, _I32],
    "dec_set_geom_precision": [_P, _I32],
    "dec_set_batch_variant": [_P, _I32],
    "dec_set_sell_variant": [_P, _I32, _I32],
    "dec_get_sell_variant": [_P, _I32, _P, _P],
    "dec_get_geom_fp64_tets": [_P, _P],
    "dec_k_eff_edges_noalloc": [C.c_int, _P, _P, _I64, _P, _P, _P, _P, _P],
}

_lib = None


def load(path: str | None = None):
    """Load the compiled library (once).  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library {path} is not built; run "
            "paper_2104_05999_gb300._build.build() first")
    lib = C.CDLL(path)
    for name, argt in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = argt
        fn.restype = C.c_int
    lib.dec_last_error.argtypes = [_P]
    lib.dec_last_error.restype = C.c_char_p
    _lib = lib
    return lib


class DecError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.message = message
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


def _host_or_tensor(a, dtype):
    """A torch tensor as it is; anything else as a C-contiguous numpy array
    of ``dtype`` (keep the result alive while its address is in use)."""
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a, dtype):
    """Address of a contiguous numpy array / torch tensor of ``dtype``."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
        return a.ctypes.data
    # torch tensor (host or device)
    import torch
    tdt = {np.float64: torch.float64, np.int32: torch.int32,
           np.uint8: torch.uint8}[np.dtype(dtype).type]
    if a.dtype != tdt or not a.is_contiguous():
        raise TypeError(f"expected a contiguous {tdt} tensor")
    return a.data_ptr()


class Context:
    """One dec_ctx: owns the device buffers of one mesh and its solves."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self.lib = load()
        h = _P()
        st = self.lib.dec_create(C.byref(h), int(device), stream)
        if st != DEC_OK:
            raise DecError(st, self.lib.dec_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st != DEC_OK:
            raise DecError(st, self.lib.dec_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.dec_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- entry points -------------------------------------------------
    def dec_mesh_upload(self, xyz, tets, node_tag):
        n = len(xyz)
        m = len(tets)
        return self._check(self.lib.dec_mesh_upload(
            self.h, _ptr(xyz, np.float64), n, _ptr(tets, np.int32), m,
            _ptr(node_tag, np.uint8)))

    def dec_hodge_assemble(self, k=None, discs=None, scales=None):
        nd = 0 if discs is None else len(discs)
        ns = 0 if scales is None else len(scales)
        return self._check(self.lib.dec_hodge_assemble(
            self.h, _ptr(k, np.float64), _ptr(discs, np.float64), nd,
            _ptr(scales, np.float64), ns))

    def dec_hodge_assemble_fields(self, k, discs=None):
        """k: [n_fields, n_tets] conductivity fields (one *1 per field)."""
        nd = 0 if discs is None else len(discs)
        return self._check(self.lib.dec_hodge_assemble_fields(
            self.h, _ptr(k, np.float64), int(k.shape[0]), _ptr(discs, np.float64), nd))

    def dec_laplacian_build(self, T0, precond=DEC_PRECOND_FSAI):
        n_sets = 1 if T0.ndim == 1 else T0.shape[0]
        return self._check(self.lib.dec_laplacian_build(
            self.h, _ptr(T0, np.float64), n_sets, int(precond)))

    def dec_solve(self, rtol, max_iter=100000, mode=DEC_MODE_FP64, T_out=None,
                  raise_on_error=True):
        """Returns (status, iters[B], relres[B])."""
        B = self.sizes()[4]
        iters = np.zeros(B, dtype=np.int32)
        relres = np.zeros(B, dtype=np.float64)
        st = self.lib.dec_solve(self.h, float(rtol), int(max_iter), int(mode),
                                _ptr(T_out, np.float64), iters.ctypes.data,
                                relres.ctypes.data)
        if raise_on_error:
            self._check(st)
        return st, iters, relres

    def dec_k_eff(self):
        B = self.sizes()[4]
        q_in = np.zeros(B)
        q_out = np.zeros(B)
        energy = np.zeros(B)
        self._check(self.lib.dec_k_eff(self.h, q_in.ctypes.data,
                                       q_out.ctypes.data, energy.ctypes.data))
        return q_in, q_out, energy

    def dec_crack_evolve(self, rule, max_steps, order=None, rtol=1e-10,
                         max_iter=100000, mode=DEC_MODE_FP64, k_stop=1e-9,
                         raise_on_error=True):
        """Crack growth from the current state; returns (status, cracked
        edge per step, k_eff per step), trimmed to the steps done."""
        cracked = np.zeros(max(max_steps, 1), dtype=np.int32)
        keff = np.zeros(max(max_steps, 1))
        steps = C.c_int32(0)
        keep = None
        optr = None
        if order is not None:
            keep = _host_or_tensor(order, np.int32)
            optr = _ptr(keep, np.int32)
        st = self.lib.dec_crack_evolve(self.h, int(rule), int(max_steps), optr,
                                       float(rtol), int(max_iter), int(mode),
                                       float(k_stop), cracked.ctypes.data,
                                       keff.ctypes.data, C.byref(steps))
        if raise_on_error:
            self._check(st)
        k = steps.value
        return st, cracked[:k].copy(), keff[:k].copy()

    def dec_crack_paths(self, orders, rtol=1e-10, max_iter=100000, k_stop=1e-9,
                        raise_on_error=True):
        """Stochastic cracking of several paths at once; ``orders`` is
        [n_paths, max_steps].  Returns (status, k_eff per path trimmed to
        its steps, steps per path)."""
        orders = _host_or_tensor(orders, np.int32)
        P, S = orders.shape
        keff = np.zeros((P, max(S, 1)))
        steps = np.zeros(P, dtype=np.int32)
        st = self.lib.dec_crack_paths(self.h, int(P), int(S), _ptr(orders, np.int32),
                                      float(rtol), int(max_iter), float(k_stop),
                                      keff.ctypes.data, steps.ctypes.data)
        if raise_on_error:
            self._check(st)
        return st, [keff[b, :steps[b]].copy() for b in range(P)], steps

    def dec_tet_solve(self, T0, kappa=1.0, limiter=1e-8, cracked_faces=None,
                      face_flux=None, rtol=1e-12, max_iter=100000, raise_on_error=True):
        """The paper's tet-centred form; returns dict(status, alpha, q_in,
        q_out, iters, relres, limited)."""
        n, m = self.sizes()[:2]
        alpha = np.zeros(m)
        q2 = np.zeros(2)
        it = C.c_int32()
        rr = C.c_double()
        nl = C.c_int64()
        T0 = _host_or_tensor(T0, np.float64)
        cf = _host_or_tensor(cracked_faces, np.int32)
        ff = _host_or_tensor(face_flux, np.float64)
        st = self.lib.dec_tet_solve(
            self.h, _ptr(T0, np.float64), float(kappa), float(limiter), _ptr(cf, np.int32),
            0 if cf is None else len(cf), _ptr(ff, np.float64),
            float(rtol), int(max_iter), alpha.ctypes.data, q2.ctypes.data, C.byref(it),
            C.byref(rr), C.byref(nl))
        if raise_on_error:
            self._check(st)
        return dict(status=st, alpha=alpha, q_in=q2[0], q_out=q2[1], iters=it.value,
                    relres=rr.value, limited=nl.value)

    def dec_tet_get_faces(self):
        m = self.sizes()[1]
        nf = C.c_int64()
        self._check(self.lib.dec_tet_get_faces(self.h, C.byref(nf), None, None))
        faces = np.zeros((nf.value, 3), dtype=np.int32)
        t2f = np.zeros((m, 4), dtype=np.int32)
        self._check(self.lib.dec_tet_get_faces(self.h, C.byref(nf), faces.ctypes.data,
                                               t2f.ctypes.data))
        return faces, t2f

    def dec_tet_whitney(self):
        m = self.sizes()[1]
        v = np.zeros((m, 3))
        self._check(self.lib.dec_tet_whitney(self.h, v.ctypes.data))
        return v

    # ---- getters --------------------------------------------------------
    def dec_get_batch_variant(self):
        """Gather entries per round trip the autotuner picked for the last
        batched solve (0: register gathers)."""
        v = C.c_int32()
        self._check(self.lib.dec_get_batch_variant(self.h, C.byref(v)))
        return v.value

    def dec_set_geom_precision(self, precision):
        """DEC_GEOM_FP64 or DEC_GEOM_MIXED for the next Hodge assemblies."""
        self._check(self.lib.dec_set_geom_precision(self.h, int(precision)))

    def dec_get_geom_fp64_tets(self):
        """Tets the last Hodge assembly computed in FP64."""
        v = C.c_int64()
        self._check(self.lib.dec_get_geom_fp64_tets(self.h, C.byref(v)))
        return v.value

    def dec_set_batch_variant(self, variant=0):
        """Force a batched launch variant (a dec_get_batch_variant code; 0:
        autotune)."""
        self._check(self.lib.dec_set_batch_variant(self.h, int(variant)))

    def dec_set_sell_variant(self, l_shape=0, g_shape=0):
        """Force the single-instance SELL launch shapes (0: autotune)."""
        self._check(self.lib.dec_set_sell_variant(self.h, int(l_shape), int(g_shape)))

    def dec_get_sell_variant(self, precision):
        """(L shape, FSAI shape) codes in use for precision 0 (FP64) or 1."""
        a, b = C.c_int32(), C.c_int32()
        self._check(self.lib.dec_get_sell_variant(self.h, int(precision), C.byref(a),
                                                  C.byref(b)))
        return a.value, b.value

    def dec_get_crack_iterations(self):
        """CG iterations summed over the steps of the last crack growth."""
        v = C.c_int64()
        self._check(self.lib.dec_get_crack_iterations(self.h, C.byref(v)))
        return v.value

    def dec_get_batch_phase_ms(self):
        """ms per FP32 iteration of the last batched solve's five phases
        (SpMM, x/r update, FSAI lower, FSAI upper, p update)."""
        v = np.zeros(5)
        self._check(self.lib.dec_get_batch_phase_ms(self.h, v.ctypes.data))
        return v

    def dec_get_batch_kernel_ms(self):
        """Device time (ms) of the last batched solve's persistent launch."""
        v = C.c_double()
        self._check(self.lib.dec_get_batch_kernel_ms(self.h, C.byref(v)))
        return v.value

    def sizes(self):
        v = [C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()]
        b = C.c_int32()
        self._check(self.lib.dec_get_sizes(self.h, *[C.byref(x) for x in v],
                                           C.byref(b)))
        return tuple(x.value for x in v) + (b.value,)

    def dec_get_edges(self):
        n, m, ne, nnz, B = self.sizes()
        E = np.zeros((ne, 2), dtype=np.int32)
        t2e = np.zeros((m, 6), dtype=np.int32)
        self._check(self.lib.dec_get_edges(self.h, E.ctypes.data, t2e.ctypes.data))
        return E, t2e

    def dec_get_hodge(self):
        n, m, ne, nnz, B = self.sizes()
        w = np.zeros(ne)
        fc = np.zeros(ne, dtype=np.uint8)
        self._check(self.lib.dec_get_hodge(self.h, w.ctypes.data, fc.ctypes.data))
        return w, fc

    def dec_get_csr(self, inst=0, values=True):
        n, m, ne, nnz, B = self.sizes()
        rowptr = np.zeros(n + 1, dtype=np.int32)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz) if values else None
        b = np.zeros(n) if values else None
        self._check(self.lib.dec_get_csr(
            self.h, int(inst), rowptr.ctypes.data, col.ctypes.data,
            None if val is None else val.ctypes.data,
            None if b is None else b.ctypes.data))
        return rowptr, col, val, b

    def dec_get_precond(self):
        nnz = self.sizes()[3]
        g = np.zeros(nnz)
        self._check(self.lib.dec_get_precond(self.h, g.ctypes.data))
        return g

    def dec_get_launch_count(self):
        c = C.c_int64()
        self._check(self.lib.dec_get_launch_count(self.h, C.byref(c)))
        return c.value

    def dec_set_barrier_test(self, spin_limit=0, withhold_block=0):
        """Testing aid: shorter barrier waits and a withheld block in the
        persistent solves (see dec.h); (0, 0) restores normal operation."""
        return self._check(self.lib.dec_set_barrier_test(
            self.h, int(spin_limit), int(withhold_block)))

    def dec_time_kernel(self, kernel, reps=20, flush_bytes=512 << 20):
        """Mean duration (ms) of one launch of a solver kernel, cold L2."""
        ms = C.c_double()
        self._check(self.lib.dec_time_kernel(self.h, int(kernel), int(reps),
                                             int(flush_bytes), C.byref(ms)))
        return ms.value


def dec_k_eff_edges_noalloc(device, E, w, T, xyz, node_tag, stream=None):
    """q_in, q_out, energy of one temperature field from device arrays,
    through the entry point that allocates no device memory (see dec.h)."""
    lib = load()
    out = np.zeros(3)
    st = lib.dec_k_eff_edges_noalloc(
        int(device), stream, _ptr(E, np.int32), int(E.shape[0]),
        _ptr(w, np.float64), _ptr(T, np.float64), _ptr(xyz, np.float64),
        _ptr(node_tag, np.uint8), out.ctypes.data)
    if st != DEC_OK:
        raise DecError(st, "dec_k_eff_edges_noalloc failed")
    return out
