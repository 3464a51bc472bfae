"""Thin Python binding of libbem.so (include/bem.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch only provides device
memory and the stream.  There is no CPU fallback: if the library is missing or
fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbem.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "bem.h")

FP64, MIXED, DF = 0, 1, 2
CONDUCTOR, FLOATING, DIELECTRIC, SHEET = 0, 1, 2, 3
_KIND = {"conductor": CONDUCTOR, "floating": FLOATING, "dielectric": DIELECTRIC, "sheet": SHEET}

ERRORS = {0: "BEM_OK", -1: "BEM_ERR_ARG", -2: "BEM_ERR_CUDA", -3: "BEM_ERR_DEGENERATE",
          -4: "BEM_ERR_NOT_CONVERGED", -5: "BEM_ERR_TIMEOUT", -6: "BEM_ERR_NOMEM",
          -7: "BEM_ERR_CAPACITY"}


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class bem_region(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("floating_id", ctypes.c_int32), ("V0", ctypes.c_double),
                ("eps_plus", ctypes.c_double), ("eps_minus", ctypes.c_double)]


class bem_mesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("np", ctypes.c_int64),
                ("X", ctypes.POINTER(ctypes.c_double)), ("tri", ctypes.POINTER(ctypes.c_int32)),
                ("region", ctypes.POINTER(ctypes.c_int32)), ("nregions", ctypes.c_int32),
                ("regions", ctypes.POINTER(bem_region))]


class bem_params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("far_order", ctypes.c_int32),
                ("gmres_restart", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("max_points", ctypes.c_int64),
                ("timing", ctypes.c_int32), ("residual", ctypes.c_int32),
                ("far32_variant", ctypes.c_int32), ("adjoint_checkpoint", ctypes.c_int32),
                ("adjoint_lines", ctypes.c_int64), ("trace_cluster", ctypes.c_int32)]


RESIDUAL_DF, RESIDUAL_FP64, RESIDUAL_DF_UPDATE = 0, 1, 2


class bem_trace_params(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("r_max", ctypes.c_double), ("c", ctypes.c_double),
                ("E0", ctypes.c_double), ("d", ctypes.c_double), ("e_floor", ctypes.c_double),
                ("max_steps", ctypes.c_int64)]


class bem_counters(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("far_launches", ctypes.c_int64 * 3),
                ("pairs", ctypes.c_int64 * 3), ("near_pairs", ctypes.c_int64 * 3),
                ("far_ms", ctypes.c_double * 3), ("matvecs", ctypes.c_int64 * 3),
                ("gmres_iters", ctypes.c_int64), ("far32_variant", ctypes.c_int64),
                ("phi_pairs", ctypes.c_int64 * 3), ("chunks32p", ctypes.c_int64),
                ("fast_chunks32p", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


class bem_tuning(ctypes.Structure):
    _fields_ = [("far32_variant", ctypes.c_int32), ("far32_slots", ctypes.c_int32),
                ("source", ctypes.c_int32), ("bucket", ctypes.c_int32), ("n_candidates", ctypes.c_int32),
                ("cand_variant", ctypes.c_int32 * 12), ("cand_slots", ctypes.c_int32 * 12),
                ("cand_ms", ctypes.c_float * 12)]

    def as_dict(self):
        n = self.n_candidates
        return {"far32_variant": self.far32_variant, "far32_slots": self.far32_slots,
                "source": ["fixed", "timed", "table"][self.source], "bucket": self.bucket,
                "candidates": [{"variant": self.cand_variant[k], "slots": self.cand_slots[k],
                                "ms": self.cand_ms[k]} for k in range(n)]}


class bem_p1_params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("far_order", ctypes.c_int32), ("sing_order", ctypes.c_int32),
                ("near_radial", ctypes.c_int32), ("near_angular", ctypes.c_int32),
                ("gmres_restart", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("far32_variant", ctypes.c_int32),
                ("max_points", ctypes.c_int64), ("timing", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class bem_batch_counters(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int64), ("nrhs", ctypes.c_int64),
                ("far_launches", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("rhs_pairs", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("arnoldi_steps", ctypes.c_int64),
                ("lines", ctypes.c_int64), ("far_timed", ctypes.c_int64), ("far_ms", ctypes.c_double),
                ("eval_pairs", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_vp = ctypes.c_void_p
_i32, _i64, _dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_pvp = ctypes.POINTER(_vp)
_SIGS = {
    "bem_default_params": (None, [ctypes.POINTER(bem_params)]),
    "bem_create": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(bem_mesh), ctypes.POINTER(bem_params), _vp]),
    "bem_destroy": (_i32, [_vp]),
    "bem_last_error": (ctypes.c_char_p, [_vp]),
    "bem_sizes": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                         ctypes.POINTER(_i64)]),
    "bem_sync": (_i32, [_vp]),
    "bem_get_counters": (_i32, [_vp, ctypes.POINTER(bem_counters)]),
    "bem_reset_counters": (_i32, [_vp]),
    "bem_assemble_rows": (_i32, [_vp, _i64, _i64, _i32, _vp, _i64]),
    "bem_matvec": (_i32, [_vp, _i32, _i32, _vp, _vp]),
    "bem_rhs": (_i32, [_vp, _i32, _vp, _vp]),
    "bem_solve": (_i32, [_vp, _i32, _i32, _vp, _vp, _dbl, ctypes.POINTER(_i32), ctypes.POINTER(_dbl)]),
    "bem_eval_field": (_i32, [_vp, _i32, _vp, _i64, _vp, _vp, _vp]),
    "bem_eval_field_static": (_i32, [_vp, _i32, _vp, _i64, _vp, _vp, _vp]),
    "bem_surface_field": (_i32, [_vp, _i32, _vp, _vp]),
    "bem_default_trace_params": (None, [ctypes.POINTER(bem_trace_params)]),
    "bem_matvec_transpose": (_i32, [_vp, _i32, _vp, _vp]),
    "bem_adjoint": (_i32, [_vp, _i32, _vp, _i64, _vp, ctypes.POINTER(bem_trace_params), _vp, _vp,
                           _vp, _vp, _vp]),
    "bem_trace_lines": (_i32, [_vp, _i32, _vp, _i64, _vp, ctypes.POINTER(bem_trace_params), _vp,
                               _vp, _vp, _vp]),
    "bem_measure_peaks": (_i32, [ctypes.POINTER(_dbl)] * 3),
    "bem_p1_default_params": (None, [ctypes.POINTER(bem_p1_params)]),
    "bem_p1_create": (_i32, [ctypes.POINTER(_vp), _i64, _vp, _i64, _i64, _vp, _vp, _i32,
                             ctypes.POINTER(bem_region), ctypes.POINTER(bem_p1_params), _vp]),
    "bem_get_tuning": (_i32, [_vp, ctypes.POINTER(bem_tuning)]),
    "bem_clear_tuning_table": (None, []),
    "bem_batch_create": (_i32, [_pvp, _pvp, _i32, _i32, _i32]),
    "bem_batch_destroy": (_i32, [_vp]),
    "bem_batch_last_error": (ctypes.c_char_p, [_vp]),
    "bem_batch_get_counters": (_i32, [_vp, ctypes.POINTER(bem_batch_counters)]),
    "bem_batch_reset_counters": (_i32, [_vp]),
    "bem_batch_matvec": (_i32, [_vp, _pvp, _pvp]),
    "bem_batch_solve": (_i32, [_vp, _i32, _pvp, _pvp, _dbl, ctypes.POINTER(_i32),
                               ctypes.POINTER(_dbl)]),
    "bem_batch_eval_field": (_i32, [_vp, _i32, _pvp, ctypes.POINTER(_i64), _pvp, _pvp, _pvp]),
    "bem_batch_trace": (_i32, [_vp, _i32, _pvp, ctypes.POINTER(_i64), _pvp,
                               ctypes.POINTER(bem_trace_params), _pvp, _pvp, _pvp]),
}
_lib = None


def header_symbols(path: str = HEADER):
    """Names of the functions declared in include/bem.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bem_[a-z_0-9]+)\s*\(", txt)))


def lib():
    """Load libbem.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libbem.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, ctx=None):
    if rc != 0:
        msg = lib().bem_last_error(ctx)
        raise BemError(rc, msg.decode() if msg else "")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def default_params(**kw) -> bem_params:
    p = bem_params()
    lib().bem_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Context:
    """One mesh on the current CUDA device (bem_create / bem_destroy)."""

    def __init__(self, mesh, stream=None, **params):
        import torch
        self._torch = torch
        L = lib()
        self.X = np.ascontiguousarray(mesh.X, dtype=np.float64)
        self.tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        self.region = np.ascontiguousarray(mesh.region, dtype=np.int32)
        regs = (bem_region * len(mesh.regions))()
        for k, r in enumerate(mesh.regions):
            regs[k].kind = _KIND[r["kind"]]
            regs[k].floating_id = int(r.get("floating_id", 0))
            regs[k].V0 = float(r.get("V0", 0.0))
            regs[k].eps_plus = float(r.get("eps_plus", 1.0))
            regs[k].eps_minus = float(r.get("eps_minus", 1.0))
        self._regs = regs
        m = bem_mesh(len(self.X), len(self.tri), self.X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     self.tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                     self.region.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(mesh.regions),
                     regs)
        self.params = default_params(**params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = L.bem_create(ctypes.byref(h), ctypes.byref(m), ctypes.byref(self.params),
                          ctypes.c_void_p(self.stream.cuda_stream))
        _check(rc, None)
        self.h = h
        a, b, c, d = (ctypes.c_int64() for _ in range(4))
        _check(L.bem_sizes(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), h)
        self.np, self.nunk, self.nfloat, self.near_pairs = a.value, b.value, c.value, d.value
        self.nregions = len(mesh.regions)

    def close(self):
        if getattr(self, "h", None):
            lib().bem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, dtype=None):
        t = self._torch
        x = a if isinstance(a, t.Tensor) else t.as_tensor(np.asarray(a))
        return x.to(device="cuda", dtype=dtype or t.float64).contiguous()

    def sync(self):
        _check(lib().bem_sync(self.h), self.h)

    def counters(self) -> dict:
        c = bem_counters()
        _check(lib().bem_get_counters(self.h, ctypes.byref(c)), self.h)
        return c.as_dict()

    def reset_counters(self):
        _check(lib().bem_reset_counters(self.h), self.h)

    def tuning(self) -> dict:
        t = bem_tuning()
        _check(lib().bem_get_tuning(self.h, ctypes.byref(t)), self.h)
        return t.as_dict()

    def rhs(self, V0=None, nrhs=1):
        t = self._torch
        b = t.empty((nrhs, self.nunk), dtype=t.float64, device="cuda")
        v = None if V0 is None else self._dev(V0)
        _check(lib().bem_rhs(self.h, nrhs, _ptr(v), _ptr(b)), self.h)
        return b

    def matvec(self, x, precision=FP64, out=None):
        t = self._torch
        x = self._dev(x)
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        y = out if out is not None else t.empty_like(x)
        _check(lib().bem_matvec(self.h, precision, nrhs, _ptr(x), _ptr(y)), self.h)
        return y

    def solve(self, precision=FP64, V0=None, tol=1e-8, nrhs=1, out=None):
        t = self._torch
        v = None if V0 is None else self._dev(V0)
        u = out if out is not None else t.empty((nrhs, self.nunk), dtype=t.float64, device="cuda")
        it = ctypes.c_int32()
        rel = (ctypes.c_double * nrhs)()
        rc = lib().bem_solve(self.h, precision, nrhs, _ptr(v), _ptr(u), tol, ctypes.byref(it), rel)
        _check(rc, self.h)
        return u, it.value, list(rel)

    def eval_field(self, u, pts, precision=FP64, want_phi=True, want_E=True, phi=None, E=None):
        t = self._torch
        u = self._dev(u)
        pts = self._dev(pts)
        M = pts.shape[0]
        if want_phi and phi is None:
            phi = t.empty(M, dtype=t.float64, device="cuda")
        if want_E and E is None:
            E = t.empty((M, 3), dtype=t.float64, device="cuda")
        _check(lib().bem_eval_field(self.h, precision, _ptr(u), M, _ptr(pts),
                                    _ptr(phi if want_phi else None), _ptr(E if want_E else None)),
               self.h)
        return phi, E

    def eval_field_static(self, u, pts, precision=FP64, phi=None, E=None):
        """bem_eval_field_static: same result as eval_field; the call itself
        allocates nothing on the library side (scratch is a fixed static array).
        phi and E may be passed in preallocated."""
        t = self._torch
        u = self._dev(u)
        pts = self._dev(pts)
        M = pts.shape[0]
        phi = t.empty(M, dtype=t.float64, device="cuda") if phi is None else phi
        E = t.empty((M, 3), dtype=t.float64, device="cuda") if E is None else E
        _check(lib().bem_eval_field_static(self.h, precision, _ptr(u), M, _ptr(pts), _ptr(phi),
                                           _ptr(E)), self.h)
        return phi, E

    def trace_lines(self, u, seeds, precision=FP64, **tp):
        """bem_trace_lines: K, status, nsteps, xend per seed (device tensors)."""
        t = self._torch
        p = bem_trace_params()
        lib().bem_default_trace_params(ctypes.byref(p))
        for k, v in tp.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        u = self._dev(u)
        seeds = self._dev(seeds)
        L = seeds.shape[0]
        K = t.empty(L, dtype=t.float64, device="cuda")
        st = t.empty(L, dtype=t.int32, device="cuda")
        ns = t.empty(L, dtype=t.int32, device="cuda")
        xe = t.empty((L, 3), dtype=t.float64, device="cuda")
        _check(lib().bem_trace_lines(self.h, precision, _ptr(u), L, _ptr(seeds), ctypes.byref(p),
                                     _ptr(K), _ptr(st), _ptr(ns), _ptr(xe)), self.h)
        return K, st, ns, xe

    def _trace_params(self, tp):
        p = bem_trace_params()
        lib().bem_default_trace_params(ctypes.byref(p))
        for k, v in tp.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        return p

    def matvec_transpose(self, x, precision=FP64):
        t = self._torch
        x = self._dev(x)
        y = t.empty_like(x)
        _check(lib().bem_matvec_transpose(self.h, precision, _ptr(x), _ptr(y)), self.h)
        return y

    def adjoint(self, u, seeds, dL_dK, precision=FP64, **tp):
        """bem_adjoint: (K, dJ/dX [nv,3], dJ/dV0 [nregions], dJ/deps [nregions,2])
        for J = sum_l dL_dK[l] K_l."""
        t = self._torch
        p = self._trace_params(tp)
        u = self._dev(u)
        seeds = self._dev(seeds)
        w = self._dev(dL_dK)
        L = seeds.shape[0]
        K = t.empty(L, dtype=t.float64, device="cuda")
        gX = t.empty((len(self.X), 3), dtype=t.float64, device="cuda")
        gV0 = t.empty(self.nregions, dtype=t.float64, device="cuda")
        geps = t.empty((self.nregions, 2), dtype=t.float64, device="cuda")
        _check(lib().bem_adjoint(self.h, precision, _ptr(u), L, _ptr(seeds), ctypes.byref(p), _ptr(w),
                                 _ptr(K), _ptr(gX), _ptr(gV0), _ptr(geps)), self.h)
        return K, gX, gV0, geps

    def surface_field(self, u, precision=FP64):
        t = self._torch
        u = self._dev(u)
        E = t.empty((self.np, 3), dtype=t.float64, device="cuda")
        _check(lib().bem_surface_field(self.h, precision, _ptr(u), _ptr(E)), self.h)
        return E

    def assemble_rows(self, row0=0, row1=None, precision=FP64):
        t = self._torch
        row1 = self.nunk if row1 is None else row1
        A = t.empty((row1 - row0, self.nunk), dtype=t.float64, device="cuda")
        _check(lib().bem_assemble_rows(self.h, row0, row1, precision, _ptr(A), self.nunk), self.h)
        return A


def clear_tuning_table():
    """bem_clear_tuning_table: the next context of every size bucket times its candidates."""
    lib().bem_clear_tuning_table()


def measure_peaks() -> dict:
    """bem_measure_peaks on the current device: FP32 (paired and scalar) and FP64
    multiply-add rates in TFLOP/s."""
    a, b, c = _dbl(), _dbl(), _dbl()
    _check(lib().bem_measure_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), None)
    return {"fp32_tflops": a.value, "fp64_tflops": b.value, "fp32_scalar_tflops": c.value}


def _regions(regions):
    regs = (bem_region * len(regions))()
    for k, r in enumerate(regions):
        regs[k].kind = _KIND[r["kind"]]
        regs[k].floating_id = int(r.get("floating_id", 0))
        regs[k].V0 = float(r.get("V0", 0.0))
        regs[k].eps_plus = float(r.get("eps_plus", 1.0))
        regs[k].eps_minus = float(r.get("eps_minus", 1.0))
    return regs


class P1Context(Context):
    """Curved six-node triangles with the mapped linear basis, collocation at the
    vertices (bem_p1_create).  nodes [nn, 3] (the first nv the corners), tri6 [N, 6],
    body [N] region index per triangle, regions as for flat meshes (conductor, floating
    and dielectric kinds).  Products, solves, dense rows and fields as Context."""

    def __init__(self, nodes, tri6, nv, body, regions, stream=None, **params):
        import torch
        self._torch = torch
        L = lib()
        self.nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        self.tri6 = np.ascontiguousarray(tri6, dtype=np.int32)
        self.body = np.ascontiguousarray(body, dtype=np.int32)
        self._regs = _regions(regions)
        p = bem_p1_params()
        L.bem_p1_default_params(ctypes.byref(p))
        for k, v in params.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        self.p1params = p
        self.params = default_params()
        self.params.eta, self.params.far_order = p.eta, p.far_order
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = L.bem_p1_create(ctypes.byref(h), len(self.nodes), self.nodes.ctypes.data_as(ctypes.c_void_p),
                             int(nv), len(self.tri6), self.tri6.ctypes.data_as(ctypes.c_void_p),
                             self.body.ctypes.data_as(ctypes.c_void_p), len(regions), self._regs,
                             ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream))
        _check(rc, None)
        self.h = h
        a, b, c, d = (ctypes.c_int64() for _ in range(4))
        _check(L.bem_sizes(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), h)
        self.np, self.nunk, self.nfloat, self.near_pairs = a.value, b.value, c.value, d.value
        self.nv = int(nv)
        self.nregions = len(regions)
        self.X = self.nodes[: self.nv]


def _ptr_array(tensors):
    """Host array of device pointers (None -> NULL entries)."""
    return (_vp * len(tensors))(*[None if t is None else t.data_ptr() for t in tensors])


class Batch:
    """bem_batch: several Contexts (one device, one stream, one far_order in 2..4,
    one gmres_restart) with nrhs right-hand sides each, served by one persistent
    regular-pair launch, a CUDA-graph Arnoldi iteration and one persistent tracer
    launch.  The contexts are kept alive by this object."""

    def __init__(self, contexts, nrhs=1, timing=False):
        import torch
        self._torch = torch
        self.contexts = list(contexts)
        self.nrhs = int(nrhs)
        arr = (_vp * len(self.contexts))(*[c.h.value for c in self.contexts])
        h = _vp()
        rc = lib().bem_batch_create(ctypes.byref(h), arr, len(self.contexts), self.nrhs,
                                    1 if timing else 0)
        if rc != 0:
            raise BemError(rc, "bem_batch_create: contexts must share device, stream, far_order "
                               "(2..4) and gmres_restart; 1 <= nrhs <= 4")
        self.h = h

    def _check(self, rc):
        if rc != 0:
            msg = lib().bem_batch_last_error(self.h)
            raise BemError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            lib().bem_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def counters(self) -> dict:
        c = bem_batch_counters()
        self._check(lib().bem_batch_get_counters(self.h, ctypes.byref(c)))
        return c.as_dict()

    def reset_counters(self):
        self._check(lib().bem_batch_reset_counters(self.h))

    def _vecs(self, xs):
        t = self._torch
        out = []
        for c, x in zip(self.contexts, xs):
            x = x if isinstance(x, t.Tensor) else t.as_tensor(np.asarray(x))
            out.append(x.to(device="cuda", dtype=t.float64).reshape(self.nrhs, c.nunk).contiguous())
        return out

    def matvec(self, xs):
        """y_i = A_i x_i (mixed form) for every instance; xs: per instance [nrhs][nunk_i]."""
        t = self._torch
        xs = self._vecs(xs)
        ys = [t.empty_like(x) for x in xs]
        self._check(lib().bem_batch_matvec(self.h, _ptr_array(xs), _ptr_array(ys)))
        return ys

    def solve(self, V0=None, tol=1e-8, precision=MIXED, check=True):
        """u_i [nrhs][nunk_i] per instance, Arnoldi iterations and relative residuals
        [n][nrhs].  V0: per instance [nrhs][nregions_i] conductor potentials, or None."""
        t = self._torch
        n, nr = len(self.contexts), self.nrhs
        v = None
        if V0 is not None:
            v = [(x if isinstance(x, t.Tensor) else t.as_tensor(np.asarray(x))).to(
                device="cuda", dtype=t.float64).reshape(nr, c.nregions).contiguous()
                 for c, x in zip(self.contexts, V0)]
        us = [t.empty((nr, c.nunk), dtype=t.float64, device="cuda") for c in self.contexts]
        it = (_i32 * (n * nr))()
        rel = (_dbl * (n * nr))()
        rc = lib().bem_batch_solve(self.h, precision, None if v is None else _ptr_array(v),
                                   _ptr_array(us), tol, it, rel)
        if check or rc not in (0, -4):
            self._check(rc)
        return us, np.array(it[:]).reshape(n, nr), np.array(rel[:]).reshape(n, nr)

    def eval_field(self, us, pts, precision=MIXED):
        """bem_batch_eval_field: lists of (phi, E) per instance for its points."""
        t = self._torch
        us = [u.to(device="cuda", dtype=t.float64).reshape(-1).contiguous() for u in us]
        ps = [(p if isinstance(p, t.Tensor) else t.as_tensor(np.asarray(p))).to(
            device="cuda", dtype=t.float64).reshape(-1, 3).contiguous() for p in pts]
        M = (_i64 * len(ps))(*[len(p) for p in ps])
        phi = [t.empty(len(p), dtype=t.float64, device="cuda") for p in ps]
        E = [t.empty((len(p), 3), dtype=t.float64, device="cuda") for p in ps]
        self._check(lib().bem_batch_eval_field(self.h, precision, _ptr_array(us), M, _ptr_array(ps),
                                               _ptr_array(phi), _ptr_array(E)))
        return phi, E

    def trace(self, us, seeds, precision=MIXED, **tp):
        """Lines of every instance in one launch: lists of K, status, nsteps (device)."""
        t = self._torch
        p = bem_trace_params()
        lib().bem_default_trace_params(ctypes.byref(p))
        for k, val in tp.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, val)
        us = [u.to(device="cuda", dtype=t.float64).reshape(-1).contiguous() for u in us]
        sd = [(s if isinstance(s, t.Tensor) else t.as_tensor(np.asarray(s))).to(
            device="cuda", dtype=t.float64).reshape(-1, 3).contiguous() for s in seeds]
        L = (_i64 * len(sd))(*[len(s) for s in sd])
        K = [t.empty(len(s), dtype=t.float64, device="cuda") for s in sd]
        st = [t.empty(len(s), dtype=t.int32, device="cuda") for s in sd]
        ns = [t.empty(len(s), dtype=t.int32, device="cuda") for s in sd]
        self._check(lib().bem_batch_trace(self.h, precision, _ptr_array(us), L, _ptr_array(sd),
                                          ctypes.byref(p), _ptr_array(K), _ptr_array(st),
                                          _ptr_array(ns)))
        return K, st, ns
