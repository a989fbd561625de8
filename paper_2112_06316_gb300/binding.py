"""ctypes binding of the C ABI in ``include/ifgf.h`` (argument marshalling only).

Every numerical step runs in ``libifgf.so``; this module converts Python /
torch arguments to pointers and sizes, checks the returned status and raises
``IFGFError`` with ``ifgf_last_error()``'s message.  There is no fallback: if
the shared library is missing the import of a plan fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libifgf.so")
MAXD = 20

IFGF_OK = 0
STATUS = {0: "IFGF_OK", -1: "IFGF_EINVAL", -2: "IFGF_ENOMEM", -3: "IFGF_ECUDA", -4: "IFGF_ENOTCONVERGED",
          -5: "IFGF_EUNSUPPORTED", -6: "IFGF_EINTERNAL"}
FP64 = 0
MIXED = 1
# ifgf_layer: the operator's kernel (combined field, double layer alone, single layer alone)
LAYER_COMBINED = 0
LAYER_DOUBLE = 1
LAYER_SINGLE = 2


class IFGFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class CParams(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_double), ("eta", ctypes.c_double),
        ("Ps", ctypes.c_int), ("Pang", ctypes.c_int), ("nC0", ctypes.c_int), ("nS0", ctypes.c_int),
        ("levels", ctypes.c_int), ("leaf_target", ctypes.c_double),
        ("cone_rule", ctypes.c_int), ("factor_mode", ctypes.c_int),
        ("identity_coef", ctypes.c_double),
        ("root_center", ctypes.c_double * 3), ("root_side", ctypes.c_double),
        ("cone_band", ctypes.c_double),
        ("far_field", ctypes.c_int), ("layer", ctypes.c_int), ("leaf_max", ctypes.c_int),
    ]


class CInfo(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64), ("D", ctypes.c_int),
        ("root_center", ctypes.c_double * 3), ("root_side", ctypes.c_double),
        ("nbox", ctypes.c_int * (MAXD + 1)), ("ns", ctypes.c_int * (MAXD + 1)),
        ("nC", ctypes.c_int * (MAXD + 1)), ("split", ctypes.c_int * (MAXD + 1)),
        ("nrc", ctypes.c_int64 * (MAXD + 1)),
        ("cousin_evals", ctypes.c_int64 * (MAXD + 1)),
        ("prop_evals", ctypes.c_int64 * (MAXD + 1)),
        ("leaf_evals", ctypes.c_int64), ("near_pairs", ctypes.c_int64),
        ("correction_nnz", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
        ("near_block_chunks", ctypes.c_int64),
    ]


# (name, restype, argtypes) of every exported entry point
_VP = ctypes.c_void_p
_SIGS = [
    ("ifgf_params_default", None, [ctypes.POINTER(CParams), ctypes.c_double]),
    ("ifgf_supported_orders", ctypes.c_char_p, []),
    ("ifgf_last_error", ctypes.c_char_p, []),
    ("ifgf_plan_create", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.POINTER(CParams), _VP,
                                        ctypes.POINTER(_VP)]),
    ("ifgf_plan_dry_run", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.POINTER(CParams),
                                         ctypes.POINTER(CInfo)]),
    ("ifgf_plan_set_correction", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64]),
    ("ifgf_apply", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    ("ifgf_apply_adjoint", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    ("ifgf_apply_vjp", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_int, _VP]),
    ("ifgf_apply_noalloc", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    ("ifgf_plan_workspace_bytes", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    ("ifgf_apply_ws", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int64, _VP]),
    ("ifgf_apply_vjp_ws", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int, _VP]),
    ("ifgf_rp_correction", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                                          ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    ("ifgf_rp_correction_gpu", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.c_int32, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_double, _VP,
                                              ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    ("ifgf_free", None, [_VP]),
    ("ifgf_field", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    ("ifgf_far_field", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    ("ifgf_far_field_ifgf", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    ("ifgf_plan_create_with_targets", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.c_int64,
                                                     ctypes.POINTER(CParams), _VP, ctypes.POINTER(_VP)]),
    ("ifgf_field_ifgf", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    ("ifgf_gmres", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), _VP, _VP]),
    ("ifgf_plan_info", ctypes.c_int, [_VP, ctypes.POINTER(CInfo)]),
    ("ifgf_plan_check", ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_int64)]),
    ("ifgf_plan_set_profiling", ctypes.c_int, [_VP, ctypes.c_int]),
    ("ifgf_plan_stage_times", ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    ("ifgf_plan_destroy", None, [_VP]),
    ("ifgf_plan_set_rhs_block", ctypes.c_int, [_VP, ctypes.c_int]),
    ("ifgf_plan_set_tc_fill", ctypes.c_int, [_VP, ctypes.c_double]),
    ("ifgf_plan_set_tc_engine", ctypes.c_int, [_VP, ctypes.c_int]),
    ("ifgf_group_create", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(_VP)]),
    ("ifgf_group_set_streams", ctypes.c_int, [_VP, ctypes.c_int]),
    ("ifgf_group_apply", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP]),
    ("ifgf_group_captures", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    ("ifgf_plan_set_interp_engine", ctypes.c_int, [_VP, ctypes.c_int]),
    ("ifgf_group_destroy", None, [_VP]),
]
STAGES = ["gather", "leaf", "prop", "near", "cousin", "scatter", "correction", "prop_tc", "cousin_sum", "prop_cs"]

_lib = None


def lib():
    """Load ``libifgf.so`` (built by ``paper_2112_06316_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2112_06316_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return [s[0] for s in _SIGS]


def check(status: int):
    if status != IFGF_OK:
        raise IFGFError(status, lib().ifgf_last_error().decode())


@dataclass
class Params:
    """Python mirror of ``ifgf_params`` (defaults of ``ifgf_params_default``)."""

    k: float
    eta: float | None = None
    Ps: int = 3
    Pang: int = 5
    nC0: int = 2
    nS0: int = 1
    levels: int = 0
    leaf_target: float = 64.0
    cone_rule: int = 0
    factor_mode: int = 0
    identity_coef: float = 0.5
    root_center: tuple = (0.0, 0.0, 0.0)
    root_side: float = 0.0
    cone_band: float = 1e-4
    far_field: int = 0
    layer: int = 0  # LAYER_COMBINED, LAYER_DOUBLE or LAYER_SINGLE
    leaf_max: int = 0  # > 0: adaptive octree, boxes of at most leaf_max points are leaves

    def to_c(self) -> CParams:
        p = CParams()
        lib().ifgf_params_default(ctypes.byref(p), ctypes.c_double(self.k))
        p.eta = self.k if self.eta is None else self.eta
        p.Ps, p.Pang, p.nC0, p.nS0, p.levels = self.Ps, self.Pang, self.nC0, self.nS0, self.levels
        p.leaf_target = self.leaf_target
        p.cone_rule, p.factor_mode = self.cone_rule, self.factor_mode
        p.identity_coef = self.identity_coef
        for a in range(3):
            p.root_center[a] = self.root_center[a]
        p.root_side = self.root_side
        p.cone_band = self.cone_band
        p.far_field = self.far_field
        p.layer = self.layer
        p.leaf_max = self.leaf_max
        return p


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _stream_ptr(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _info_dict(ci) -> dict:
    D = ci.D
    return {
        "N": ci.N, "D": D, "root_center": tuple(ci.root_center), "root_side": ci.root_side,
        "nbox": [ci.nbox[i] for i in range(D + 1)], "ns": [ci.ns[i] for i in range(D + 1)],
        "nC": [ci.nC[i] for i in range(D + 1)], "split": [ci.split[i] for i in range(D + 1)],
        "nrc": [ci.nrc[i] for i in range(D + 1)],
        "cousin_evals": [ci.cousin_evals[i] for i in range(D + 1)],
        "prop_evals": [ci.prop_evals[i] for i in range(D + 1)],
        "leaf_evals": ci.leaf_evals, "near_pairs": ci.near_pairs,
        "correction_nnz": ci.correction_nnz, "device_bytes": ci.device_bytes,
        "near_block_chunks": ci.near_block_chunks,
    }


def dry_run(points, normals, weights, params: Params) -> dict:
    """Host-only plan statistics (``ifgf_plan_dry_run``); needs no GPU."""
    x = _host(points, np.float64)
    n = _host(normals, np.float64)
    w = _host(weights, np.float64)
    ci = CInfo()
    cp = params.to_c()
    check(lib().ifgf_plan_dry_run(x.ctypes.data, n.ctypes.data, w.ctypes.data, ctypes.c_int64(x.shape[0]),
                                  ctypes.byref(cp), ctypes.byref(ci)))
    return _info_dict(ci)


class Plan:
    """An ``ifgf_plan``: octree, cone structure and device geometry for one surface.

    With ``targets`` ((M, 3) off-surface points) the plan is built by
    ``ifgf_plan_create_with_targets``: the targets join the octree as points of weight 0 and
    ``field_ifgf`` gives the potential there; the plan's own applies act on all
    ``n_sources + n_targets`` points (``N``)."""

    def __init__(self, points, normals, weights, params: Params, stream=None, targets=None):
        x = _host(points, np.float64)
        n = _host(normals, np.float64)
        w = _host(weights, np.float64)
        if x.ndim != 2 or x.shape[1] != 3 or n.shape != x.shape or w.shape != (x.shape[0],):
            raise ValueError("points/normals must be (N, 3) and weights (N,)")
        self.params = params
        self.n_sources = int(x.shape[0])
        cp = params.to_c()
        h = _VP()
        if targets is None:
            self.n_targets = 0
            check(lib().ifgf_plan_create(x.ctypes.data, n.ctypes.data, w.ctypes.data, ctypes.c_int64(self.n_sources),
                                         ctypes.byref(cp), _VP(_stream_ptr(stream)), ctypes.byref(h)))
        else:
            t = _host(targets, np.float64).reshape(-1, 3)
            self.n_targets = int(t.shape[0])
            check(lib().ifgf_plan_create_with_targets(x.ctypes.data, n.ctypes.data, w.ctypes.data,
                                                      ctypes.c_int64(self.n_sources), t.ctypes.data,
                                                      ctypes.c_int64(self.n_targets), ctypes.byref(cp),
                                                      _VP(_stream_ptr(stream)), ctypes.byref(h)))
        self.N = self.n_sources + self.n_targets
        self._h = h

    @classmethod
    def with_targets(cls, points, normals, weights, targets, params: Params, stream=None) -> "Plan":
        """``Plan(points, normals, weights, params, stream, targets=targets)``."""
        return cls(points, normals, weights, params, stream=stream, targets=targets)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ifgf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        ci = CInfo()
        check(lib().ifgf_plan_info(self._h, ctypes.byref(ci)))
        return _info_dict(ci)

    def set_correction(self, rowptr, col, val):
        """CSR correction over the caller's point order; val complex (nnz,)."""
        rp = _host(rowptr, np.int64)
        cl = _host(col, np.int32)
        v = _host(np.asarray(val, dtype=np.complex128).view(np.float64), np.float64)
        nnz = int(rp[-1]) if rp.size else 0
        check(lib().ifgf_plan_set_correction(self._h, rp.ctypes.data, cl.ctypes.data, v.ctypes.data,
                                             ctypes.c_int64(nnz)))

    def apply_ptr(self, sigma_ptr: int, y_ptr: int, nrhs: int, prec: int, stream=None):
        """Raw-pointer apply: sigma/y device buffers of N x nrhs complex."""
        check(lib().ifgf_apply(self._h, _VP(sigma_ptr), _VP(y_ptr), ctypes.c_int(nrhs), ctypes.c_int(prec),
                               _VP(_stream_ptr(stream))))

    def adjoint(self, g, out=None, stream=None):
        """out = A^H g for a CUDA tensor g of shape (nrhs, N) or (N,); dtype selects the precision."""
        import torch

        if not (isinstance(g, torch.Tensor) and g.is_cuda):
            raise TypeError("g must be a CUDA torch tensor")
        prec = FP64 if g.dtype == torch.complex128 else MIXED if g.dtype == torch.complex64 else None
        if prec is None:
            raise TypeError("g must be complex64 or complex128")
        squeeze = g.dim() == 1
        gg = (g.reshape(1, -1) if squeeze else g).contiguous()
        if gg.shape[-1] != self.N:
            raise ValueError(f"g must have N={self.N} columns")
        y = torch.empty_like(gg) if out is None else out
        check(lib().ifgf_apply_adjoint(self._h, _VP(gg.data_ptr()), _VP(y.data_ptr()), ctypes.c_int(gg.shape[0]),
                                       ctypes.c_int(prec), _VP(_stream_ptr(stream))))
        return y.reshape(-1) if squeeze else y

    def vjp(self, sigma, g, stream=None, with_dk: bool = True):
        """(A^H g, Re <g, dA/dk sigma>) for CUDA tensors sigma, g of shape (nrhs, N) or (N,); with
        with_dk False the k-derivative is skipped (0.0 is returned in its place)."""
        import torch

        if sigma.dtype != g.dtype or sigma.shape != g.shape:
            raise ValueError("sigma and g must have the same shape and dtype")
        prec = FP64 if sigma.dtype == torch.complex128 else MIXED if sigma.dtype == torch.complex64 else None
        if prec is None:
            raise TypeError("complex64 or complex128 expected")
        squeeze = sigma.dim() == 1
        s_ = (sigma.reshape(1, -1) if squeeze else sigma).contiguous()
        g_ = (g.reshape(1, -1) if squeeze else g).contiguous()
        out = torch.empty_like(s_)
        dk = ctypes.c_double(0.0)
        check(lib().ifgf_apply_vjp(self._h, _VP(s_.data_ptr()), _VP(g_.data_ptr()), _VP(out.data_ptr()),
                                   ctypes.c_int(s_.shape[0]), ctypes.byref(dk) if with_dk else None,
                                   ctypes.c_int(prec), _VP(_stream_ptr(stream))))
        return (out.reshape(-1) if squeeze else out), float(dk.value)

    def workspace_bytes(self, nrhs: int, prec: int) -> int:
        """Bytes of the apply workspace for nrhs right-hand sides in one precision."""
        n = ctypes.c_int64()
        check(lib().ifgf_plan_workspace_bytes(self._h, ctypes.c_int(nrhs), ctypes.c_int(prec), ctypes.byref(n)))
        return int(n.value)

    def apply_with_state(self, sigma, stream=None):
        """(y, state): y = A sigma computed on a fresh workspace tensor `state` that holds the
        forward state afterwards (for vjp_from_state)."""
        import torch

        prec = FP64 if sigma.dtype == torch.complex128 else MIXED if sigma.dtype == torch.complex64 else None
        if prec is None or not sigma.is_cuda:
            raise TypeError("sigma must be a complex64 or complex128 CUDA tensor")
        squeeze = sigma.dim() == 1
        s_ = (sigma.reshape(1, -1) if squeeze else sigma).contiguous()
        if s_.shape[-1] != self.N:
            raise ValueError(f"sigma must have N={self.N} columns")
        nb = self.workspace_bytes(int(s_.shape[0]), prec)
        state = torch.empty(max(nb, 1) + 256, dtype=torch.uint8, device=s_.device)
        off = (-state.data_ptr()) % 256  # 256-byte aligned view
        ws = state[off:off + max(nb, 1)]
        y = torch.empty_like(s_)
        check(lib().ifgf_apply_ws(self._h, _VP(s_.data_ptr()), _VP(y.data_ptr()), ctypes.c_int(s_.shape[0]),
                                  ctypes.c_int(prec), _VP(ws.data_ptr()), ctypes.c_int64(nb), _VP(_stream_ptr(stream))))
        return (y.reshape(-1) if squeeze else y), ws

    def vjp_from_state(self, state, g, stream=None, with_dk: bool = True):
        """(A^H g, Re <g, dA/dk sigma>) from the forward state of apply_with_state(sigma); with
        with_dk False the k-derivative is skipped (0.0 is returned in its place)."""
        import torch

        prec = FP64 if g.dtype == torch.complex128 else MIXED if g.dtype == torch.complex64 else None
        if prec is None:
            raise TypeError("complex64 or complex128 expected")
        squeeze = g.dim() == 1
        g_ = (g.reshape(1, -1) if squeeze else g).contiguous()
        out = torch.empty_like(g_)
        dk = ctypes.c_double(0.0)
        check(lib().ifgf_apply_vjp_ws(self._h, _VP(state.data_ptr()), ctypes.c_int64(state.numel()),
                                      _VP(g_.data_ptr()), _VP(out.data_ptr()), ctypes.c_int(g_.shape[0]),
                                      ctypes.byref(dk) if with_dk else None, ctypes.c_int(prec),
                                      _VP(_stream_ptr(stream))))
        return (out.reshape(-1) if squeeze else out), float(dk.value)

    def apply_noalloc_ptr(self, sigma_ptr: int, y_ptr: int, nrhs: int, prec: int, stream=None):
        """Raw-pointer ``ifgf_apply_noalloc`` (workspace in the library's fixed device array)."""
        check(lib().ifgf_apply_noalloc(self._h, _VP(sigma_ptr), _VP(y_ptr), ctypes.c_int(nrhs), ctypes.c_int(prec),
                                       _VP(_stream_ptr(stream))))

    def apply(self, sigma, out=None, stream=None):
        """y = A sigma for a CUDA torch tensor sigma of shape (nrhs, N) or (N,).

        complex128 selects the FP64 path, complex64 the mixed path.
        """
        import torch

        if not (isinstance(sigma, torch.Tensor) and sigma.is_cuda):
            raise TypeError("sigma must be a CUDA torch tensor")
        if sigma.dtype == torch.complex128:
            prec = FP64
        elif sigma.dtype == torch.complex64:
            prec = MIXED
        else:
            raise TypeError("sigma must be complex64 (mixed) or complex128 (FP64)")
        squeeze = sigma.dim() == 1
        s = sigma.reshape(1, -1) if squeeze else sigma
        if s.shape[-1] != self.N:
            raise ValueError(f"sigma must have N={self.N} columns")
        s = s.contiguous()
        if out is not None and (out.shape != sigma.shape or out.dtype != sigma.dtype or not out.is_contiguous()):
            raise ValueError("out must match sigma's shape/dtype and be contiguous")
        y = torch.empty_like(s) if out is None else out.view(s.shape)
        self.apply_ptr(s.data_ptr(), y.data_ptr(), int(s.shape[0]), prec, stream)
        return y.reshape(-1) if squeeze else y

    def _eval_off_surface(self, fn, sigma, targets, out, stream):
        import torch

        if not (isinstance(sigma, torch.Tensor) and sigma.is_cuda):
            raise TypeError("sigma must be a CUDA torch tensor")
        prec = FP64 if sigma.dtype == torch.complex128 else MIXED if sigma.dtype == torch.complex64 else None
        if prec is None:
            raise TypeError("sigma must be complex64 (mixed) or complex128 (FP64)")
        squeeze = sigma.dim() == 1
        s = (sigma.reshape(1, -1) if squeeze else sigma).contiguous()
        if s.shape[-1] != self.N:
            raise ValueError(f"sigma must have N={self.N} columns")
        t = torch.as_tensor(targets, dtype=torch.float64, device=sigma.device).reshape(-1, 3).contiguous()
        M = int(t.shape[0])
        y = torch.empty((s.shape[0], M), dtype=s.dtype, device=s.device) if out is None else out
        if y.shape != (s.shape[0], M) or y.dtype != s.dtype or not y.is_contiguous():
            raise ValueError("out must be a contiguous (nrhs, M) tensor of sigma's dtype")
        check(fn(self._h, _VP(s.data_ptr()), _VP(t.data_ptr()), ctypes.c_int64(M), _VP(y.data_ptr()),
                 ctypes.c_int(s.shape[0]), ctypes.c_int(prec), _VP(_stream_ptr(stream))))
        return y.reshape(-1) if squeeze else y

    def field(self, sigma, targets, out=None, stream=None):
        """Combined-layer potential (``ifgf_field``) at targets (M, 3) for sigma of shape (nrhs, N) or (N,)."""
        return self._eval_off_surface(lib().ifgf_field, sigma, targets, out, stream)

    def far_field(self, sigma, directions, out=None, stream=None):
        """Far-field pattern (``ifgf_far_field``) at unit directions (M, 3)."""
        return self._eval_off_surface(lib().ifgf_far_field, sigma, directions, out, stream)

    def field_ifgf(self, sigma, out=None, stream=None):
        """Potential at the targets of a plan made by ``Plan.with_targets`` (``ifgf_field_ifgf``) for
        surface densities sigma of shape (nrhs, n_sources) or (n_sources,)."""
        import torch

        if not (isinstance(sigma, torch.Tensor) and sigma.is_cuda):
            raise TypeError("sigma must be a CUDA torch tensor")
        prec = FP64 if sigma.dtype == torch.complex128 else MIXED if sigma.dtype == torch.complex64 else None
        if prec is None:
            raise TypeError("sigma must be complex64 (mixed) or complex128 (FP64)")
        nt = self.n_targets
        if not nt:
            raise ValueError("the plan has no targets (build it with Plan.with_targets)")
        squeeze = sigma.dim() == 1
        s = (sigma.reshape(1, -1) if squeeze else sigma).contiguous()
        if s.shape[-1] != self.n_sources:
            raise ValueError(f"sigma must have n_sources={self.n_sources} columns")
        y = torch.empty((s.shape[0], nt), dtype=s.dtype, device=s.device) if out is None else out
        if y.shape != (s.shape[0], nt) or y.dtype != s.dtype or not y.is_contiguous():
            raise ValueError("out must be a contiguous (nrhs, n_targets) tensor of sigma's dtype")
        check(lib().ifgf_field_ifgf(self._h, _VP(s.data_ptr()), _VP(y.data_ptr()), ctypes.c_int(s.shape[0]),
                                    ctypes.c_int(prec), _VP(_stream_ptr(stream))))
        return y.reshape(-1) if squeeze else y

    def far_field_ifgf(self, sigma, directions, out=None, stream=None):
        """Far-field pattern from the IFGF level-3 interpolants (``ifgf_far_field_ifgf``); the
        plan must have been created with ``Params(far_field=1)``."""
        return self._eval_off_surface(lib().ifgf_far_field_ifgf, sigma, directions, out, stream)

    def gmres(self, rhs, x0=None, restart: int = 50, maxit: int = 200, tol: float = 1e-6,
              precision: int = FP64, stream=None):
        """Solve A x = rhs (complex128 CUDA vector of length N) with ``ifgf_gmres``.

        Returns (x, converged, iterations, relative-residual history)."""
        import torch

        if not (isinstance(rhs, torch.Tensor) and rhs.is_cuda and rhs.dtype == torch.complex128):
            raise TypeError("rhs must be a complex128 CUDA tensor")
        b = rhs.reshape(-1).contiguous()
        if b.numel() != self.N:
            raise ValueError("rhs must have N entries")
        x = torch.zeros_like(b) if x0 is None else x0.reshape(-1).to(torch.complex128).clone().contiguous()
        it = ctypes.c_int(0)
        hist = np.zeros(maxit + 1)
        st = lib().ifgf_gmres(self._h, _VP(b.data_ptr()), _VP(x.data_ptr()), ctypes.c_int(restart), ctypes.c_int(maxit),
                              ctypes.c_double(tol), ctypes.c_int(precision), ctypes.byref(it), _VP(hist.ctypes.data),
                              _VP(_stream_ptr(stream)))
        if st not in (IFGF_OK, -4):
            check(st)
        return x, st == IFGF_OK, int(it.value), hist[: it.value + 1]

    def set_profiling(self, enable: bool = True):
        check(lib().ifgf_plan_set_profiling(self._h, ctypes.c_int(int(enable))))

    def stage_times(self):
        """[(stage, level, ms)] of the last apply made with profiling on."""
        cap = 80
        kind = (ctypes.c_int * cap)()
        level = (ctypes.c_int * cap)()
        ms = (ctypes.c_double * cap)()
        n = lib().ifgf_plan_stage_times(self._h, cap, kind, level, ms)
        if n < 0:
            check(n)
        return [(STAGES[kind[i]], level[i], ms[i]) for i in range(n)]

    def set_tc_fill(self, min_fill: float):
        check(lib().ifgf_plan_set_tc_fill(self._h, ctypes.c_double(min_fill)))

    def set_tc_engine(self, engine: int):
        """1 = tcgen05 (tensor memory), 0 = warp-level mma.sync."""
        check(lib().ifgf_plan_set_tc_engine(self._h, ctypes.c_int(engine)))

    def set_interp_engine(self, engine: int):
        """1 = cone-stationary CUDA-core interpolation kernels (default), 0 = point-stationary."""
        check(lib().ifgf_plan_set_interp_engine(self._h, ctypes.c_int(engine)))

    def set_rhs_block(self, rhs_block: int):
        check(lib().ifgf_plan_set_rhs_block(self._h, ctypes.c_int(rhs_block)))

    def missed_lookups(self, stream=None) -> int:
        m = ctypes.c_int64()
        check(lib().ifgf_plan_check(self._h, _VP(_stream_ptr(stream)), ctypes.byref(m)))
        return int(m.value)


def rp_correction(points, normals, weights, patch_node, m: int, k: float, eta: float | None = None,
                  delta: float = 0.0, n_beta: int = 48, d_grade: float = 5.0, device: bool = False, stream=None):
    """Rectangular-polar correction as numpy CSR (rowptr int64 (N+1,), col int32 (nnz,), val
    complex128 (nnz,)) over the caller's point order, ready for ``Plan.set_correction``:
    ``ifgf_rp_correction`` (host only) or, with ``device``, ``ifgf_rp_correction_gpu`` (the
    quadrature on the current GPU)."""
    x = _host(points, np.float64)
    n = _host(normals, np.float64)
    w = _host(weights, np.float64)
    pn = _host(patch_node, np.int32)
    N = int(x.shape[0])
    if x.shape != (N, 3) or n.shape != (N, 3) or w.shape != (N,) or pn.shape != (N,):
        raise ValueError("points/normals (N, 3), weights and patch_node (N,) expected")
    rp, cl, vl = _VP(), _VP(), _VP()
    args = (x.ctypes.data, n.ctypes.data, w.ctypes.data, ctypes.c_int64(N), pn.ctypes.data, ctypes.c_int32(m),
            ctypes.c_double(k), ctypes.c_double(k if eta is None else eta), ctypes.c_double(delta),
            ctypes.c_int32(n_beta), ctypes.c_double(d_grade))
    if device:
        check(lib().ifgf_rp_correction_gpu(*args, _VP(_stream_ptr(stream)), ctypes.byref(rp), ctypes.byref(cl),
                                           ctypes.byref(vl)))
    else:
        check(lib().ifgf_rp_correction(*args, ctypes.byref(rp), ctypes.byref(cl), ctypes.byref(vl)))
    try:
        rowptr = np.ctypeslib.as_array(ctypes.cast(rp, ctypes.POINTER(ctypes.c_int64)), shape=(N + 1,)).copy()
        nnz = int(rowptr[-1])
        col = np.ctypeslib.as_array(ctypes.cast(cl, ctypes.POINTER(ctypes.c_int32)), shape=(max(nnz, 1),))[:nnz].copy()
        val = np.ctypeslib.as_array(ctypes.cast(vl, ctypes.POINTER(ctypes.c_double)),
                                    shape=(max(2 * nnz, 2),))[:2 * nnz].copy().view(np.complex128)
    finally:
        for ptr in (rp, cl, vl):
            lib().ifgf_free(ptr)
    return rowptr, col, val


class IFGFOperator(Plan):
    """The operator A of Eq. CombLayIE for one surface and wavenumber: a ``Plan`` built from
    (points, normals, weights, k, params).  ``params`` supplies every setting but k (defaults
    of ``Params`` when omitted); ``apply``, ``adjoint``, ``vjp``, ``gmres``, ``field`` and
    ``far_field`` are the plan's."""

    def __init__(self, points, normals, weights, k: float, params: Params | None = None, stream=None):
        import dataclasses

        prm = Params(k=float(k)) if params is None else dataclasses.replace(params, k=float(k))
        super().__init__(points, normals, weights, prm, stream)


def supported_orders():
    return [tuple(int(v) for v in s.split("x")) for s in lib().ifgf_supported_orders().decode().split(",")]


class Group:
    """``ifgf_group``: one CUDA-graph apply over several plans (each with its own rhs)."""

    def __init__(self, plans, nstreams: int = 4):
        self.plans = list(plans)
        arr = (_VP * len(self.plans))(*[p.handle for p in self.plans])
        h = _VP()
        check(lib().ifgf_group_create(arr, ctypes.c_int(len(self.plans)), ctypes.byref(h)))
        self._h = h
        self.set_streams(nstreams)

    def set_streams(self, nstreams: int):
        check(lib().ifgf_group_set_streams(self._h, ctypes.c_int(nstreams)))
        self.nstreams = nstreams

    def apply(self, sigmas, outs, stream=None):
        """outs[i] = A_i sigmas[i]; tensors of shape (nrhs_i, N_i), one complex dtype for all."""
        import torch

        dt = sigmas[0].dtype
        prec = FP64 if dt == torch.complex128 else MIXED
        n = len(self.plans)
        sp = (_VP * n)(*[s.data_ptr() for s in sigmas])
        yp = (_VP * n)(*[y.data_ptr() for y in outs])
        nr = (ctypes.c_int * n)(*[int(s.shape[0]) if s.dim() == 2 else 1 for s in sigmas])
        check(lib().ifgf_group_apply(self._h, sp, yp, nr, ctypes.c_int(prec), _VP(_stream_ptr(stream))))
        return outs

    def captures(self) -> int:
        """Number of CUDA graphs this group has captured (replays add nothing)."""
        n = ctypes.c_int64()
        check(lib().ifgf_group_captures(self._h, ctypes.byref(n)))
        return int(n.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ifgf_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
