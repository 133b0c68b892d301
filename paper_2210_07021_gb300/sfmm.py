"""Python binding of the sFMM C ABI (include/sfmm.h).

Argument marshalling only: every step of the solve runs in libsfmm.so's CUDA
kernels.  Tensors are torch CUDA tensors (PyTorch supplies device memory and
streams); host entry points take numpy arrays.  There is no CPU fallback: if
the library is missing or no GPU is present, the calls raise.
"""
import ctypes
import os

import numpy as np

from . import build as _build

SFMM_OK, SFMM_EINVAL, SFMM_ENOMEM, SFMM_ECUDA, SFMM_ETIMEOUT, SFMM_EDEGENERATE = range(6)
SFMM_FP64, SFMM_MIXED, SFMM_MIXED_DF, SFMM_FP32 = 0, 1, 2, 3
(ARR_SRC_KEYS, ARR_SRC_PERM, ARR_NODE_PREFIX, ARR_NODE_LEVEL, ARR_NODE_RANGE, ARR_NODE_CHILD0, ARR_NODE_PARENT,
 ARR_NODE_GEOM, ARR_MULTIPOLE, ARR_LOCAL, ARR_M2L, ARR_P2P, ARR_TGT_KEYS, ARR_NODE_TRANGE,
 ARR_SRC_OFFSETS, ARR_TGT_OFFSETS) = range(16)

EXPORTS = ["sfmm_default_options", "sfmm_plan", "sfmm_potential", "sfmm_deflection", "sfmm_deflection_host",
           "sfmm_adjoint", "sfmm_shear", "sfmm_deflection_batch",
           "sfmm_destroy", "sfmm_last_error", "sfmm_order", "sfmm_get_stats", "sfmm_set_timing",
           "sfmm_debug_copy", "sfmm_keys", "sfmm_sort_keys_static", "sfmm_peak_rate", "sfmm_set_wait_limit",
           "sfmm_graph_capture", "sfmm_graph_launch", "sfmm_graph_info", "sfmm_graph_release"]
STATIC_SORT_MAX_N = 1 << 18


class Options(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("c_s", ctypes.c_double), ("c_t", ctypes.c_double),
                ("precision", ctypes.c_int), ("zero_mean", ctypes.c_int), ("q_f32", ctypes.c_int),
                ("n_max", ctypes.c_int64), ("m_max", ctypes.c_int64), ("stream", ctypes.c_void_p),
                ("m2l_tensor_cores", ctypes.c_int), ("sigma", ctypes.c_double), ("wait_limit", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64), ("depth", ctypes.c_int64),
                ("n_m2l", ctypes.c_int64), ("n_p2p", ctypes.c_int64), ("p2p_interactions", ctypes.c_int64),
                ("launches", ctypes.c_int64),
                ("ms", ctypes.c_double * 8), ("near_ms", ctypes.c_double)]


class GraphStats(ctypes.Structure):
    _fields_ = [("n_shells", ctypes.c_int64), ("kernel_nodes", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("overflows", ctypes.c_int64), ("recaptures", ctypes.c_int64), ("n_nodes", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64), ("n_m2l", ctypes.c_int64), ("n_p2p", ctypes.c_int64)]


class SfmmError(RuntimeError):
    pass


_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libsfmm.so (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise SfmmError(f"{_build.LIB} is missing; build it with paper_2210_07021_gb300/build.py")
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    vp, i64, ci, cd_ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.sfmm_default_options.argtypes = [ctypes.POINTER(Options)]
    L.sfmm_default_options.restype = ci
    L.sfmm_plan.argtypes = [ctypes.POINTER(vp), ci, ci, cd_, ctypes.POINTER(Options)]
    L.sfmm_plan.restype = ci
    L.sfmm_potential.argtypes = [vp, vp, vp, i64, vp, i64, vp]
    L.sfmm_potential.restype = ci
    L.sfmm_deflection.argtypes = [vp, vp, vp, i64, vp, i64, vp, vp]
    L.sfmm_deflection.restype = ci
    L.sfmm_deflection_host.argtypes = [vp, vp, vp, i64, vp, i64, vp, vp]
    L.sfmm_deflection_host.restype = ci
    L.sfmm_adjoint.argtypes = [vp, vp, vp, i64, vp, i64, vp, vp, vp, vp]
    L.sfmm_adjoint.restype = ci
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.sfmm_deflection_batch.argtypes = [vp, ci, pp, pp, ctypes.POINTER(i64), pp, ctypes.POINTER(i64), pp, pp, ci]
    L.sfmm_deflection_batch.restype = ci
    L.sfmm_shear.argtypes = [vp, vp, vp, i64, vp, i64, vp, vp, vp, vp]
    L.sfmm_shear.restype = ci
    L.sfmm_destroy.argtypes = [vp]
    L.sfmm_destroy.restype = None
    L.sfmm_last_error.argtypes = [vp]
    L.sfmm_last_error.restype = ctypes.c_char_p
    L.sfmm_order.argtypes = [vp]
    L.sfmm_order.restype = ci
    L.sfmm_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    L.sfmm_get_stats.restype = ci
    L.sfmm_set_timing.argtypes = [vp, ci]
    L.sfmm_set_timing.restype = ci
    L.sfmm_debug_copy.argtypes = [vp, ci, vp, i64, ctypes.POINTER(i64)]
    L.sfmm_debug_copy.restype = ci
    L.sfmm_keys.argtypes = [vp, i64, vp, vp]
    L.sfmm_keys.restype = ci
    L.sfmm_sort_keys_static.argtypes = [vp, i64, vp, vp, vp]
    L.sfmm_sort_keys_static.restype = ci
    L.sfmm_set_wait_limit.argtypes = [vp, ci]
    L.sfmm_set_wait_limit.restype = ci
    L.sfmm_peak_rate.argtypes = [ci, ctypes.POINTER(ctypes.c_double), vp]
    L.sfmm_peak_rate.restype = ci
    L.sfmm_graph_capture.argtypes = [vp, ci, pp, pp, ctypes.POINTER(i64), pp, ctypes.POINTER(i64), pp, pp, cd_]
    L.sfmm_graph_capture.restype = ci
    L.sfmm_graph_launch.argtypes = [vp]
    L.sfmm_graph_launch.restype = ci
    L.sfmm_graph_info.argtypes = [vp, ctypes.POINTER(GraphStats)]
    L.sfmm_graph_info.restype = ci
    L.sfmm_graph_release.argtypes = [vp]
    L.sfmm_graph_release.restype = ci
    _lib = L
    return L


def _check(st, plan=None):
    if st != SFMM_OK:
        msg = load().sfmm_last_error(plan).decode(errors="replace")
        raise SfmmError(f"sfmm status {st}: {msg}")


def _dptr(t, dtype, shape_last=None, name="tensor"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise SfmmError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise SfmmError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise SfmmError(f"{name} must be contiguous")
    if shape_last is not None and (t.dim() != 2 or t.shape[1] != shape_last):
        raise SfmmError(f"{name} must have shape [n, {shape_last}]")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """An sFMM plan (sfmm_plan): tree depth, order p (or a tolerance) and options."""

    def __init__(self, max_depth=29, p=0, tol=1e-10, leaf_size=32, c_s=2.0, c_t=0.5, precision=SFMM_FP64,
                 zero_mean=False, q_f32=False, n_max=0, m_max=0, stream=None, m2l_tensor_cores=True, sigma=0.0,
                 wait_limit=0):
        L = load()
        o = Options()
        L.sfmm_default_options(ctypes.byref(o))
        o.leaf_size, o.c_s, o.c_t = leaf_size, c_s, c_t
        o.precision, o.zero_mean, o.q_f32 = precision, int(bool(zero_mean)), int(bool(q_f32))
        o.n_max, o.m_max = n_max, m_max
        o.m2l_tensor_cores = int(bool(m2l_tensor_cores))
        o.sigma = float(sigma)
        o.wait_limit = int(wait_limit)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = None
        o.stream = stream
        self._opt = o
        h = ctypes.c_void_p()
        _check(L.sfmm_plan(ctypes.byref(h), max_depth, p, tol, ctypes.byref(o)))
        self._h = h
        self.q_f32 = bool(q_f32)

    def close(self):
        if getattr(self, "_h", None):
            load().sfmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def order(self):
        return load().sfmm_order(self._h)

    def set_wait_limit(self, polls=0):
        """Polls after which the bounded device waits give up (0 = default; a test hook)."""
        _check(load().sfmm_set_wait_limit(self._h, int(polls)), self._h)

    def set_timing(self, on=True):
        """0/False off, 1/True per-phase device times, 2 also the near-field pair count."""
        _check(load().sfmm_set_timing(self._h, int(on)), self._h)

    def stats(self):
        s = Stats()
        _check(load().sfmm_get_stats(self._h, ctypes.byref(s)), self._h)
        d = {k: getattr(s, k) for k, _ in Stats._fields_ if k != "ms"}
        d["ms"] = list(s.ms)
        return d

    def _qdtype(self):
        import torch
        return torch.float32 if self.q_f32 else torch.float64

    def potential(self, src, q, tgt, psi=None):
        """psi [M] at the targets (device tensors in, device tensor out)."""
        import torch
        M = tgt.shape[0]
        if psi is None:
            psi = torch.empty(M, dtype=torch.float64, device=tgt.device)
        st = load().sfmm_potential(self._h, _dptr(src, torch.float64, 3, "src"), _dptr(q, self._qdtype(), None, "q"),
                                   src.shape[0], _dptr(tgt, torch.float64, 3, "tgt"), M,
                                   _dptr(psi, torch.float64, None, "psi"))
        _check(st, self._h)
        return psi

    def deflection(self, src, q, tgt, with_psi=True, psi=None, alpha=None):
        """(psi [M] or None, alpha [M, 2]) at the targets (device tensors)."""
        import torch
        M = tgt.shape[0]
        if alpha is None:
            alpha = torch.empty((M, 2), dtype=torch.float64, device=tgt.device)
        if with_psi and psi is None:
            psi = torch.empty(M, dtype=torch.float64, device=tgt.device)
        st = load().sfmm_deflection(self._h, _dptr(src, torch.float64, 3, "src"), _dptr(q, self._qdtype(), None, "q"),
                                    src.shape[0], _dptr(tgt, torch.float64, 3, "tgt"), M,
                                    _dptr(psi, torch.float64, None, "psi") if with_psi else None,
                                    _dptr(alpha, torch.float64, 2, "alpha"))
        _check(st, self._h)
        return (psi if with_psi else None), alpha

    def deflection_batch(self, shells, with_psi=True, lanes=4):
        """Solve independent shells [(src, q, tgt), ...] (device tensors) on
        `lanes` concurrent internal solvers; returns [(psi or None, alpha), ...]."""
        import torch
        n = len(shells)
        outs = []
        V = ctypes.c_void_p * max(n, 1)
        I = ctypes.c_int64 * max(n, 1)
        a_src, a_q, a_tgt, a_psi, a_alpha = V(), V(), V(), V(), V()
        a_n, a_m = I(), I()
        for i, (src, q, tgt) in enumerate(shells):
            M = tgt.shape[0]
            alpha = torch.empty((M, 2), dtype=torch.float64, device=tgt.device)
            psi = torch.empty(M, dtype=torch.float64, device=tgt.device) if with_psi else None
            a_src[i] = _dptr(src, torch.float64, 3, "src")
            a_q[i] = _dptr(q, self._qdtype(), None, "q")
            a_tgt[i] = _dptr(tgt, torch.float64, 3, "tgt")
            a_psi[i] = _dptr(psi, torch.float64, None, "psi") if with_psi else None
            a_alpha[i] = _dptr(alpha, torch.float64, 2, "alpha")
            a_n[i], a_m[i] = src.shape[0], M
            outs.append((psi, alpha))
        st = load().sfmm_deflection_batch(self._h, n, a_src, a_q, a_n, a_tgt, a_m, a_psi if with_psi else None,
                                          a_alpha, lanes)
        _check(st, self._h)
        return outs

    def graph_capture(self, shells, with_psi=True, slack=0.25):
        """Bind this plan to shells [(src, q, tgt), ...] (device tensors, kept
        referenced by the plan) and record their solves into one CUDA graph
        (sfmm_graph_capture; the returned outputs already hold one solve).
        Returns [(psi or None, alpha), ...]: the buffers every graph_launch()
        rewrites.  Update the shells' tensors in place between launches."""
        import torch
        n = len(shells)
        V = ctypes.c_void_p * max(n, 1)
        I = ctypes.c_int64 * max(n, 1)
        a_src, a_q, a_tgt, a_psi, a_alpha = V(), V(), V(), V(), V()
        a_n, a_m = I(), I()
        outs = []
        for i, (src, q, tgt) in enumerate(shells):
            M = tgt.shape[0]
            alpha = torch.empty((M, 2), dtype=torch.float64, device=tgt.device)
            psi = torch.empty(M, dtype=torch.float64, device=tgt.device) if with_psi else None
            a_src[i] = _dptr(src, torch.float64, 3, "src")
            a_q[i] = _dptr(q, self._qdtype(), None, "q")
            a_tgt[i] = _dptr(tgt, torch.float64, 3, "tgt")
            a_psi[i] = _dptr(psi, torch.float64, None, "psi") if with_psi else None
            a_alpha[i] = _dptr(alpha, torch.float64, 2, "alpha")
            a_n[i], a_m[i] = src.shape[0], M
            outs.append((psi, alpha))
        self._graph_refs = None
        st = load().sfmm_graph_capture(self._h, n, a_src, a_q, a_n, a_tgt, a_m, a_psi if with_psi else None,
                                       a_alpha, float(slack))
        _check(st, self._h)
        self._graph_refs = (list(shells), outs)
        return outs

    def graph_launch(self):
        """Replay the recorded graph (sfmm_graph_launch); synchronous."""
        _check(load().sfmm_graph_launch(self._h), self._h)

    def graph_info(self):
        g = GraphStats()
        _check(load().sfmm_graph_info(self._h, ctypes.byref(g)), self._h)
        return {k: getattr(g, k) for k, _ in GraphStats._fields_}

    def graph_release(self):
        _check(load().sfmm_graph_release(self._h), self._h)
        self._graph_refs = None

    def shear(self, src, q, tgt, with_psi=False, with_alpha=False, with_mu=False):
        """(gamma [M, 2], psi or None, alpha or None, mu or None) at the targets:
        the shear, the potential, the deflection and the magnification
        mu = 1/((1 - tr H/2)^2 - |gamma|^2) (FP64 path; see sfmm_shear)."""
        import torch
        M = tgt.shape[0]
        gamma = torch.empty((M, 2), dtype=torch.float64, device=tgt.device)
        psi = torch.empty(M, dtype=torch.float64, device=tgt.device) if with_psi else None
        alpha = torch.empty((M, 2), dtype=torch.float64, device=tgt.device) if with_alpha else None
        mu = torch.empty(M, dtype=torch.float64, device=tgt.device) if with_mu else None
        st = load().sfmm_shear(self._h, _dptr(src, torch.float64, 3, "src"), _dptr(q, self._qdtype(), None, "q"),
                               src.shape[0], _dptr(tgt, torch.float64, 3, "tgt"), M,
                               _dptr(psi, torch.float64, None, "psi"), _dptr(alpha, torch.float64, 2, "alpha"),
                               _dptr(gamma, torch.float64, 2, "gamma"), _dptr(mu, torch.float64, None, "mu"))
        _check(st, self._h)
        return gamma, psi, alpha, mu

    def adjoint(self, src, q, tgt, g_psi=None, g_alpha=None, want_q=True, want_src=True):
        """(dL/dq [N] or None, dL/dy [N, 3] or None) for a loss of this plan's
        deflection outputs, given dL/dpsi [M] and/or dL/dalpha [M, 2] (device
        tensors; FP64 adjoint sFMM, see sfmm_adjoint)."""
        import torch
        N = src.shape[0]
        gq = torch.empty(N, dtype=torch.float64, device=src.device) if want_q else None
        gs = torch.empty((N, 3), dtype=torch.float64, device=src.device) if want_src else None
        st = load().sfmm_adjoint(self._h, _dptr(src, torch.float64, 3, "src"), _dptr(q, self._qdtype(), None, "q"),
                                 N, _dptr(tgt, torch.float64, 3, "tgt"), tgt.shape[0],
                                 _dptr(g_psi, torch.float64, None, "g_psi"), _dptr(g_alpha, torch.float64, 2, "g_alpha"),
                                 _dptr(gq, torch.float64, None, "grad_q"), _dptr(gs, torch.float64, 3, "grad_src"))
        _check(st, self._h)
        return gq, gs

    def deflection_host(self, src, q, tgt, with_psi=True, psi=None, alpha=None):
        """Host-array variant (numpy in, numpy out); copies happen inside the call."""
        src = np.ascontiguousarray(src, dtype=np.float64)
        tgt = np.ascontiguousarray(tgt, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float32 if self.q_f32 else np.float64)
        M = tgt.shape[0]
        if alpha is None:
            alpha = np.empty((M, 2))
        if with_psi and psi is None:
            psi = np.empty(M)
        vp = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
        st = load().sfmm_deflection_host(self._h, vp(src), vp(q), src.shape[0], vp(tgt), M,
                                         vp(psi) if with_psi else None, vp(alpha))
        _check(st, self._h)
        return (psi if with_psi else None), alpha

    def debug(self, which, dtype, cols=None):
        """Copy an internal array of the last solve to a numpy array."""
        L = load()
        need = ctypes.c_int64()
        _check(L.sfmm_debug_copy(self._h, which, None, 0, ctypes.byref(need)), self._h)
        itemsize = np.dtype(dtype).itemsize
        a = np.empty(need.value // itemsize, dtype=dtype)
        if a.size:
            _check(L.sfmm_debug_copy(self._h, which, ctypes.c_void_p(a.ctypes.data), need.value, None), self._h)
        if cols:
            a = a.reshape(-1, cols)
        return a


def keys(xyz):
    """Order-29 nested keys of a [n, 3] float64 CUDA tensor (uint64 as int64)."""
    import torch
    n = xyz.shape[0]
    out = torch.empty(n, dtype=torch.int64, device=xyz.device)
    st = load().sfmm_keys(_dptr(xyz, torch.float64, 3, "xyz"), n, ctypes.c_void_p(out.data_ptr()),
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _check(st)
    return out


def sort_keys_static(xyz, keys=None, perm=None):
    """Keys and stable sort without any device allocation inside the library
    (sfmm_sort_keys_static): returns (keys as int64 view of uint64, perm int32)."""
    import torch
    n = xyz.shape[0]
    if keys is None:
        keys = torch.empty(n, dtype=torch.int64, device=xyz.device)
    if perm is None:
        perm = torch.empty(n, dtype=torch.int32, device=xyz.device)
    st = load().sfmm_sort_keys_static(_dptr(xyz, torch.float64, 3, "xyz"), n, ctypes.c_void_p(keys.data_ptr()),
                                      ctypes.c_void_p(perm.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _check(st)
    return keys, perm


PEAK_FP32, PEAK_FP32X2, PEAK_FP64, PEAK_MUFU = range(4)


def peak_rate(which):
    """Measured FP32 / packed FP32x2 / FP64 FMA rate (flop/s) or MUFU rate
    (rcp + lg2 operations/s) of the current GPU (sfmm_peak_rate)."""
    import torch
    v = ctypes.c_double()
    _check(load().sfmm_peak_rate(which, ctypes.byref(v), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return v.value
