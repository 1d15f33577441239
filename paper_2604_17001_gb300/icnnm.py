"""Thin ctypes binding of libicnnm.so (include/icnnm.h). Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.

Buffers may be numpy arrays (host memory) or torch CUDA tensors (device memory,
passed by pointer). There is no CPU fallback: if the library is missing, loading
fails loudly.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libicnnm.so")

OK, EINVAL, ENOMEM, EAGAIN, ENOTFOUND, ECUDA, ETIMEOUT, ECANCELED, EUNSUPPORTED, ENOCONV = range(10)
FP32, BF16, BF16X3 = 0, 1, 2


class icnnm_shape(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("dims", C.c_int64 * 3), ("kdims", C.c_int64 * 3)]


class icnnm_params(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("theta0", C.c_double), ("rho", C.c_double),
                ("theta_max", C.c_double), ("max_iters", C.c_int32), ("tol", C.c_double),
                ("check_every", C.c_int32), ("prec", C.c_int32)]


class icnnm_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("residual", C.c_double), ("objective", C.c_double),
                ("theta", C.c_double), ("seconds", C.c_double), ("latency", C.c_double)]

    def as_dict(self):
        return dict(iters=self.iters, residual=self.residual, objective=self.objective,
                    theta=self.theta, seconds=self.seconds, latency=self.latency)


class icnnm_tile_config(C.Structure):
    _fields_ = [("adj_tap_width", C.c_int32), ("fwd_channel_width", C.c_int32), ("fwd_u_stages", C.c_int32)]


class icnnm_tile_result(C.Structure):
    _fields_ = [("cfg", icnnm_tile_config), ("adj_tap_width", C.c_int32), ("fwd_channel_width", C.c_int32),
                ("fwd_u_stages", C.c_int32), ("ms_per_iter", C.c_double)]


TILE_TABLE = os.path.join(HERE, "tile_table.json")


class ICNNMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"icnnm status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libicnnm.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build the CUDA library first (paper_2604_17001_gb300.build)")
    lib = C.CDLL(path)
    P, I32, I64, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    sig = {
        "icnnm_params_default": ([C.POINTER(icnnm_params)], I32),
        "icnnm_create": ([C.POINTER(P), C.c_int, C.c_size_t, P], I32),
        "icnnm_destroy": ([P], None),
        "icnnm_strerror": ([I32], C.c_char_p),
        "icnnm_last_error": ([P], C.c_char_p),
        "icnnm_learn_V": ([P, C.POINTER(I64), I32, C.POINTER(icnnm_shape), C.POINTER(P), P, P], I32),
        "icnnm_solve": ([P, C.POINTER(icnnm_shape), P, P, P, C.POINTER(icnnm_params), P,
                         C.POINTER(icnnm_stats)], I32),
        "icnnm_solve_batch": ([P, I32, C.POINTER(icnnm_shape), C.POINTER(P), C.POINTER(P), P,
                               C.POINTER(icnnm_params), C.POINTER(P), C.POINTER(icnnm_stats)], I32),
        "icnnm_submit": ([P, C.POINTER(icnnm_shape), P, P, P, C.POINTER(icnnm_params), C.POINTER(U64)], I32),
        "icnnm_poll": ([P, U64, P, C.POINTER(icnnm_stats)], I32),
        "icnnm_wait": ([P, U64, I64, P, C.POINTER(icnnm_stats)], I32),
        "icnnm_cancel": ([P, U64], I32),
        "icnnm_profile_enable": ([P, I32], I32),
        "icnnm_profile_read": ([P, I32, C.POINTER(D), C.POINTER(I64)], I32),
        "icnnm_profile_voxels": ([P, I32, C.POINTER(I64)], I32),
        "icnnm_job_bytes": ([P, C.POINTER(icnnm_shape), I32, C.POINTER(C.c_size_t)], I32),
        "icnnm_set_tile_config": ([P, C.POINTER(I64), C.POINTER(icnnm_tile_config)], I32),
        "icnnm_set_deterministic": ([P, I32], I32),
        "icnnm_autotune": ([P, P, I32, C.POINTER(icnnm_shape), I32, C.POINTER(icnnm_tile_config),
                            C.POINTER(icnnm_tile_result), I32, C.POINTER(I32)], I32),
        "icnnm_check_bounded_wait": ([P, I64], I32),
        "icnnm_cnnm_solve": ([P, C.POINTER(icnnm_shape), P, P, C.POINTER(icnnm_params), P,
                              C.POINTER(icnnm_stats)], I32),
        "icnnm_solve_fft": ([P, C.POINTER(icnnm_shape), P, P, P, C.POINTER(icnnm_params), P,
                             C.POINTER(icnnm_stats)], I32),
        "icnnm_spectral_diagnostics": ([P, C.POINTER(icnnm_shape), P, P, D, P, C.POINTER(I32), C.POINTER(D),
                                        C.POINTER(D)], I32),
        "icnnm_learn_V_noalloc": ([C.POINTER(I64), I32, C.POINTER(icnnm_shape), C.POINTER(P), P, P, P], I32),
        "icnnm_noalloc_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(x):
    """Address of a numpy array (host) or a torch tensor (its device or host storage)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def make_shape(dims, kdims) -> icnnm_shape:
    """dims = (H, W, T) or (H, W); kdims = (k1, k2, k3) or (k1, k2)."""
    s = icnnm_shape()
    s.ndim = 3 if len(dims) == 3 else 2
    d = list(dims) + [1] * (3 - len(dims))
    kd = list(kdims) + [1] * (3 - len(kdims))
    for i in range(3):
        s.dims[i] = int(d[i])
        s.kdims[i] = int(kd[i])
    return s


def params(**kw) -> icnnm_params:
    p = icnnm_params()
    load().icnnm_params_default(C.byref(p))
    for k, v in kw.items():
        if k == "lam":
            k = "lambda_"
        if k == "prec" and isinstance(v, str):
            v = {"fp32": FP32, "bf16": BF16, "bf16x3": BF16X3}[v]
        setattr(p, k, v)
    return p


def icnnm_learn_V_noalloc(refs, kdims, V_out=None, eig_out=None, stream=None):
    """Allocation-free learn_V: ``refs`` are torch CUDA tensors (device memory), the
    outputs default to host numpy arrays. Returns (V, eig) like Context.icnnm_learn_V."""
    lib = load()
    kd = list(kdims) + [1] * (3 - len(kdims))
    k = int(np.prod(kd))
    b = len(refs)
    shapes = (icnnm_shape * b)()
    ptrs = (C.c_void_p * b)()
    for i, r in enumerate(refs):
        shp = tuple(r.shape)
        dims = (shp[1], shp[2], shp[0]) if len(shp) == 3 else (shp[0], shp[1])
        shapes[i] = make_shape(dims, kdims)
        ptrs[i] = _ptr(r)
    own = V_out is None
    if own:
        V_out = np.zeros((k, k), dtype=np.float64)
        if eig_out is None:
            eig_out = np.zeros(k, dtype=np.float64)
    st = lib.icnnm_learn_V_noalloc((C.c_int64 * 3)(*kd), b, shapes, ptrs, _ptr(V_out), _ptr(eig_out),
                                   C.c_void_p(stream) if stream else None)
    if st != OK:
        raise ICNNMError(st, lib.icnnm_noalloc_last_error().decode())
    if own:
        return V_out.T.copy(), eig_out
    return V_out, eig_out


class Context:
    """An icnnm_ctx on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, stream=None, tile_table=TILE_TABLE):
        """tile_table: JSON file of tile configurations per kernel size (written by the
        autotuner; the package's table by default, None for the built-in defaults)."""
        self.lib = load()
        self.h = C.c_void_p()
        st = self.lib.icnnm_create(C.byref(self.h), device, hbm_budget_bytes,
                                   C.c_void_p(stream) if stream else None)
        if st != OK:
            raise ICNNMError(st, self.lib.icnnm_strerror(st).decode())
        if tile_table and os.path.exists(tile_table):
            import json
            for ent in json.load(open(tile_table)).get("entries", []):
                self.icnnm_set_tile_config(ent["kdims"], ent["adj_tap_width"], ent["fwd_channel_width"],
                                           ent["fwd_u_stages"])

    def close(self):
        if self.h:
            self.lib.icnnm_destroy(self.h)
            self.h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        if st != OK:
            msg = self.lib.icnnm_last_error(self.h).decode() or self.lib.icnnm_strerror(st).decode()
            raise ICNNMError(st, msg)

    # -- learn V ------------------------------------------------------------------
    def icnnm_learn_V(self, refs, kdims, V_out=None, eig_out=None):
        """refs: list of float32 tensors (numpy (T,H,W) / (H,W) or torch CUDA). Returns
        (V, eig) with V a (k, k) float64 array whose column i is eigenvector i."""
        kd = list(kdims) + [1] * (3 - len(kdims))
        k = int(np.prod(kd))
        b = len(refs)
        shapes = (icnnm_shape * b)()
        ptrs = (C.c_void_p * b)()
        for i, r in enumerate(refs):
            shp = tuple(r.shape)
            dims = (shp[1], shp[2], shp[0]) if len(shp) == 3 else (shp[0], shp[1])
            shapes[i] = make_shape(dims, kdims)
            ptrs[i] = _ptr(r)
        own = V_out is None
        if own:
            V_out = np.zeros((k, k), dtype=np.float64)      # stored column-major: row i = column i
            eig_out = np.zeros(k, dtype=np.float64) if eig_out is None else eig_out
        kdv = (C.c_int64 * 3)(*kd)
        self._check(self.lib.icnnm_learn_V(self.h, kdv, b, shapes, ptrs, _ptr(V_out), _ptr(eig_out)))
        if own:
            return V_out.T.copy(), eig_out
        return V_out, eig_out

    def icnnm_cnnm_solve(self, M, mask, kdims, dims=None, L_out=None, **kw):
        """CNNM (no V): M (float32) and mask (uint8) as for icnnm_solve; FP32, fixed
        iteration count. Returns (L, stats dict)."""
        shp = tuple(M.shape)
        if dims is None:
            dims = (shp[1], shp[2], shp[0]) if len(shp) == 3 else (shp[0], shp[1])
        s = make_shape(dims, kdims)
        kw.setdefault("prec", "fp32")
        p = params(**kw)
        if L_out is None:
            L_out = np.zeros(shp, dtype=np.float32) if isinstance(M, np.ndarray) else M.new_zeros(shp)
        st = icnnm_stats()
        self._check(self.lib.icnnm_cnnm_solve(self.h, C.byref(s), _ptr(M), _ptr(mask), C.byref(p), _ptr(L_out),
                                              C.byref(st)))
        return L_out, st.as_dict()

    def icnnm_spectral_diagnostics(self, L0, V, kdims, rank_tol=1e-6, dims=None):
        """Relative convolution eigenvalues sigma (in V's column order), r_K, alpha_K and
        mu_K of L0 ((T, H, W) / (H, W) float32 array or tensor) with respect to V (a
        (k, k) array whose column i is eigenvector i). Returns a dict."""
        shp = tuple(L0.shape)
        if dims is None:
            dims = (shp[1], shp[2], shp[0]) if len(shp) == 3 else (shp[0], shp[1])
        s = make_shape(dims, kdims)
        k = int(np.prod(kdims))
        sigma = np.zeros(k, dtype=np.float64)
        r = C.c_int32(0)
        a, mu = C.c_double(0.0), C.c_double(0.0)
        Vc = self._v_colmajor(V)
        self._check(self.lib.icnnm_spectral_diagnostics(self.h, C.byref(s), _ptr(L0), _ptr(Vc), float(rank_tol),
                                                        _ptr(sigma), C.byref(r), C.byref(a), C.byref(mu)))
        return dict(sigma=sigma, r_K=int(r.value), alpha_K=float(a.value), mu_K=float(mu.value))

    # -- solves -----------------------------------------------------------------
    @staticmethod
    def _v_colmajor(V):
        """(k, k) array whose column i is eigenvector i -> column-major buffer."""
        if isinstance(V, np.ndarray):
            return np.ascontiguousarray(V.T, dtype=np.float64)
        return V.t().contiguous().double()

    def icnnm_solve(self, M, mask, V, kdims, dims=None, L_out=None, **kw):
        """Solve one problem. M (float32) and mask (uint8) are (T, H, W) or (H, W) arrays
        or tensors. Returns (L, stats dict)."""
        shp = tuple(M.shape)
        if dims is None:
            dims = (shp[1], shp[2], shp[0]) if len(shp) == 3 else (shp[0], shp[1])
        s = make_shape(dims, kdims)
        p = params(**kw)
        Vc = self._v_colmajor(V)
        if L_out is None:
            L_out = np.zeros(shp, dtype=np.float32) if isinstance(M, np.ndarray) else M.new_zeros(shp)
        st = icnnm_stats()
        self._check(self.lib.icnnm_solve(self.h, C.byref(s), _ptr(M), _ptr(mask), _ptr(Vc), C.byref(p),
                                         _ptr(L_out), C.byref(st)))
        return L_out, st.as_dict()

    def icnnm_solve_fft(self, M, mask, V, kdims, dims=None, L_out=None, **kw):
        """As icnnm_solve, computed in the frequency domain (power-of-two dims; FP32
        complex spectra whatever ``prec`` says). Returns (L, stats dict)."""
        shp = tuple(M.shape)
        if dims is None:
            dims = (shp[1], shp[2], shp[0]) if len(shp) == 3 else (shp[0], shp[1])
        s = make_shape(dims, kdims)
        p = params(**kw)
        Vc = self._v_colmajor(V)
        if L_out is None:
            L_out = np.zeros(shp, dtype=np.float32) if isinstance(M, np.ndarray) else M.new_zeros(shp)
        st = icnnm_stats()
        self._check(self.lib.icnnm_solve_fft(self.h, C.byref(s), _ptr(M), _ptr(mask), _ptr(Vc), C.byref(p),
                                             _ptr(L_out), C.byref(st)))
        return L_out, st.as_dict()

    def icnnm_solve_batch(self, Ms, masks, V, kdims, L_outs=None, **kw):
        n = len(Ms)
        shapes = (icnnm_shape * n)()
        pM, pK, pL = (C.c_void_p * n)(), (C.c_void_p * n)(), (C.c_void_p * n)()
        if L_outs is None:
            L_outs = [np.zeros(m.shape, dtype=np.float32) if isinstance(m, np.ndarray) else m.new_zeros(m.shape)
                      for m in Ms]
        for i, M in enumerate(Ms):
            shp = tuple(M.shape)
            dims = (shp[1], shp[2], shp[0]) if len(shp) == 3 else (shp[0], shp[1])
            shapes[i] = make_shape(dims, kdims)
            pM[i], pK[i], pL[i] = _ptr(M), _ptr(masks[i]), _ptr(L_outs[i])
        p = params(**kw)
        Vc = self._v_colmajor(V)
        st = (icnnm_stats * n)()
        self._check(self.lib.icnnm_solve_batch(self.h, n, shapes, pM, pK, _ptr(Vc), C.byref(p), pL, st))
        return L_outs, [x.as_dict() for x in st]

    # -- serving ----------------------------------------------------------------
    def icnnm_submit(self, M, mask, V, kdims, **kw) -> int:
        shp = tuple(M.shape)
        dims = (shp[1], shp[2], shp[0]) if len(shp) == 3 else (shp[0], shp[1])
        s = make_shape(dims, kdims)
        p = params(**kw)
        Vc = self._v_colmajor(V)
        jid = C.c_uint64()
        self._check(self.lib.icnnm_submit(self.h, C.byref(s), _ptr(M), _ptr(mask), _ptr(Vc), C.byref(p),
                                          C.byref(jid)))
        return jid.value

    def icnnm_poll(self, job_id: int, L_out=None):
        """Returns (status, stats dict or None); status EAGAIN while not done."""
        st = icnnm_stats()
        r = self.lib.icnnm_poll(self.h, job_id, _ptr(L_out), C.byref(st))
        if r == EAGAIN:
            return r, None
        self._check(r)
        return r, st.as_dict()

    def icnnm_wait(self, job_id: int, L_out=None, timeout_ms: int = -1):
        st = icnnm_stats()
        r = self.lib.icnnm_wait(self.h, job_id, timeout_ms, _ptr(L_out), C.byref(st))
        if r == EAGAIN:
            return r, None
        self._check(r)
        return r, st.as_dict()

    def icnnm_cancel(self, job_id: int):
        self._check(self.lib.icnnm_cancel(self.h, job_id))

    def icnnm_set_deterministic(self, on: bool):
        self._check(self.lib.icnnm_set_deterministic(self.h, 1 if on else 0))

    def icnnm_set_tile_config(self, kdims, adj_tap_width=0, fwd_channel_width=0, fwd_u_stages=0):
        kd = list(kdims) + [1] * (3 - len(kdims))
        cfg = icnnm_tile_config(int(adj_tap_width), int(fwd_channel_width), int(fwd_u_stages))
        self._check(self.lib.icnnm_set_tile_config(self.h, (C.c_int64 * 3)(*kd), C.byref(cfg)))

    def icnnm_autotune(self, dims_list, kdims, V, iters=10):
        """Time every distinct tile geometry on synthetic jobs of the given dims (all
        stepped together) and adopt the fastest. Returns (best dict, list of results)."""
        n = len(dims_list)
        shapes = (icnnm_shape * n)()
        for i, d in enumerate(dims_list):
            shapes[i] = make_shape(d, kdims)
        best = icnnm_tile_config()
        res = (icnnm_tile_result * 16)()
        nres = C.c_int32()
        Vc = self._v_colmajor(V)
        self._check(self.lib.icnnm_autotune(self.h, _ptr(Vc), n, shapes, int(iters), C.byref(best), res, 16,
                                            C.byref(nres)))
        out = [dict(adj_tap_width=r.adj_tap_width, fwd_channel_width=r.fwd_channel_width,
                    fwd_u_stages=r.fwd_u_stages, ms_per_iter=r.ms_per_iter) for r in res[:nres.value]]
        return dict(adj_tap_width=best.adj_tap_width, fwd_channel_width=best.fwd_channel_width,
                    fwd_u_stages=best.fwd_u_stages), out

    def icnnm_job_bytes(self, dims, kdims, prec="bf16") -> int:
        s = make_shape(dims, kdims)
        n = C.c_size_t()
        self._check(self.lib.icnnm_job_bytes(self.h, C.byref(s), {"fp32": FP32, "bf16": BF16, "bf16x3": BF16X3}.get(prec, prec),
                                             C.byref(n)))
        return n.value

    def icnnm_check_bounded_wait(self, limit_ns: int) -> int:
        """Status of the bounded-wait check (ETIMEOUT when the wait gave up as it should)."""
        return self.lib.icnnm_check_bounded_wait(self.h, int(limit_ns))
