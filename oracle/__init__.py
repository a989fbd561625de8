"""FP64 CPU oracle for the IFGF-accelerated CFIE apply (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs use this package.  It shares no code with
``paper_2112_06316_gb300`` (the CUDA library) and never imports it.

* ``direct`` / ``direct_adjoint``: the plain O(N^2) combined-field sum of
  Eq. field1 (kernel of Eq. GreenFunction / Eq. double_layer, identity term of
  Eq. CombLayIE) and its conjugate transpose, on all rows or a row subset.
* ``ifgf``: the IFGF apply of Section 3.4 in FP64, stage by stage (``oracle.c``).
* ``ifgf_far_field``: the far-field pattern from the IFGF level-3 interpolants
  (the s -> 0 limit of the factorisation), FP64.
* ``field`` / ``far_field``: the combined-layer potential of Eq. CombinedLayer at
  off-surface targets and its far-field pattern (Eq. FarField), plain numpy sums.
* ``mie``: closed-form sound-soft sphere solutions (module ``oracle.mie``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "rp.c")]
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
MAXD = 20


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc (FP64, OpenMP) into ``oracle/_build``."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", *_SRCS, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_double), ("eta", ctypes.c_double),
        ("Ps", ctypes.c_int), ("Pang", ctypes.c_int), ("nC0", ctypes.c_int), ("nS0", ctypes.c_int),
        ("levels", ctypes.c_int), ("leaf_target", ctypes.c_double),
        ("cone_rule", ctypes.c_int), ("factor_mode", ctypes.c_int),
        ("identity_coef", ctypes.c_double),
        ("root_center", ctypes.c_double * 3), ("root_side", ctypes.c_double),
        ("far_field", ctypes.c_int), ("layer", ctypes.c_int), ("leaf_max", ctypes.c_int),
    ]


class OracleInfo(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int),
        ("root_center", ctypes.c_double * 3), ("root_side", ctypes.c_double),
        ("nbox", ctypes.c_int * (MAXD + 1)), ("ns", ctypes.c_int * (MAXD + 1)),
        ("nC", ctypes.c_int * (MAXD + 1)), ("split", ctypes.c_int * (MAXD + 1)),
        ("nrc", ctypes.c_int64 * (MAXD + 1)),
        ("cousin_evals", ctypes.c_int64 * (MAXD + 1)),
        ("prop_evals", ctypes.c_int64 * (MAXD + 1)),
        ("leaf_evals", ctypes.c_int64), ("near_pairs", ctypes.c_int64),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.oracle_direct_rows.restype = ctypes.c_int
        _lib.oracle_direct_adjoint_rows.restype = ctypes.c_int
        _lib.oracle_direct_rows_layer.restype = ctypes.c_int
        _lib.oracle_direct_adjoint_rows_layer.restype = ctypes.c_int
        _lib.oracle_ifgf.restype = ctypes.c_int
        _lib.oracle_ifgf_far_field.restype = ctypes.c_int
        _lib.oracle_cheb_interp_1d.restype = ctypes.c_double
        _lib.oracle_cheb_interp_1d.argtypes = [ctypes.c_int, dp, ctypes.c_double]
        _lib.oracle_num_threads.restype = ctypes.c_int
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


@dataclass
class IFGFParams:
    """Parameters of the IFGF apply (same meaning as the library's ifgf_params)."""

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
    identity_coef: float = 0.0
    root_center: tuple = (0.0, 0.0, 0.0)
    root_side: float = 0.0
    far_field: int = 0
    layer: int = 0  # 0 combined field, 1 double layer, 2 single layer
    leaf_max: int = 0  # > 0: adaptive octree (boxes of at most leaf_max points are leaves)

    def to_c(self) -> OracleParams:
        p = OracleParams()
        p.k = self.k
        p.eta = self.k if self.eta is None else self.eta
        p.Ps, p.Pang, p.nC0, p.nS0, p.levels = self.Ps, self.Pang, self.nC0, self.nS0, self.levels
        p.leaf_target = self.leaf_target
        p.cone_rule, p.factor_mode = self.cone_rule, self.factor_mode
        p.identity_coef = self.identity_coef
        for a in range(3):
            p.root_center[a] = self.root_center[a]
        p.root_side = self.root_side
        p.far_field = self.far_field
        p.layer = self.layer
        p.leaf_max = self.leaf_max
        return p


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _geom(points, normals, weights):
    x = np.ascontiguousarray(points, dtype=np.float64)
    n = np.ascontiguousarray(normals, dtype=np.float64)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    return x, n, w


def _dens(sigma, N):
    s = np.asarray(sigma)
    if s.ndim == 1:
        s = s[None, :]
    if s.shape[1] != N:
        raise ValueError("density must be (nrhs, N)")
    return np.ascontiguousarray(s, dtype=np.complex128)


def direct(points, normals, weights, k, eta, sigma, cI=0.0, rows=None, layer=0) -> np.ndarray:
    """y_l = cI sigma_l + sum_{m != l} K(x_l, x_m) w_m sigma_m for l in rows (all if None), with K the
    combined field dPhi/dnu(y) - i eta Phi (layer 0), the double layer dPhi/dnu(y) (1) or the single
    layer Phi (2).

    sigma: (nrhs, N) complex; returns (nrhs, len(rows)) complex128.
    """
    x, n, w = _geom(points, normals, weights)
    N = x.shape[0]
    s = _dens(sigma, N)
    nrhs = s.shape[0]
    if rows is None:
        r = None
        nrows = N
    else:
        r = np.ascontiguousarray(rows, dtype=np.int64)
        nrows = r.shape[0]
    out = np.zeros((nrhs, nrows), dtype=np.complex128)
    cI = complex(cI)
    rc = lib().oracle_direct_rows_layer(
        ctypes.c_int(layer), ctypes.c_int64(N), _dptr(x), _dptr(n), _dptr(w), ctypes.c_double(k), ctypes.c_double(eta),
        ctypes.c_double(cI.real), ctypes.c_double(cI.imag), ctypes.c_int(nrhs),
        s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_int64(nrows),
        None if r is None else r.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise RuntimeError(f"oracle_direct_rows failed ({rc})")
    return out


def direct_adjoint(points, normals, weights, k, eta, g, cI=0.0, rows=None, layer=0) -> np.ndarray:
    """(A^H g)_m = conj(cI) g_m + w_m sum_{l != m} conj(K(x_l, x_m)) g_l for m in rows (K of `layer`)."""
    x, n, w = _geom(points, normals, weights)
    N = x.shape[0]
    s = _dens(g, N)
    nrhs = s.shape[0]
    if rows is None:
        r = None
        nrows = N
    else:
        r = np.ascontiguousarray(rows, dtype=np.int64)
        nrows = r.shape[0]
    out = np.zeros((nrhs, nrows), dtype=np.complex128)
    cI = complex(cI)
    rc = lib().oracle_direct_adjoint_rows_layer(
        ctypes.c_int(layer), ctypes.c_int64(N), _dptr(x), _dptr(n), _dptr(w), ctypes.c_double(k), ctypes.c_double(eta),
        ctypes.c_double(cI.real), ctypes.c_double(cI.imag), ctypes.c_int(nrhs),
        s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_int64(nrows),
        None if r is None else r.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise RuntimeError(f"oracle_direct_adjoint_rows failed ({rc})")
    return out


def ifgf(points, normals, weights, params: IFGFParams, sigma):
    """Algorithm 1 in FP64.  Returns (y (nrhs, N) complex128, info dict)."""
    x, n, w = _geom(points, normals, weights)
    N = x.shape[0]
    s = _dens(sigma, N)
    nrhs = s.shape[0]
    out = np.zeros((nrhs, N), dtype=np.complex128)
    info = OracleInfo()
    p = params.to_c()
    rc = lib().oracle_ifgf(ctypes.byref(p), ctypes.c_int64(N), _dptr(x), _dptr(n), _dptr(w), ctypes.c_int(nrhs),
                           s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(info))
    if rc != 0:
        raise RuntimeError(f"oracle_ifgf failed ({rc})")
    return out, _info_dict(info)


def ifgf_far_field(points, normals, weights, params: IFGFParams, sigma, xhat):
    """Far-field pattern (Eq. FarField) from the IFGF level-3 interpolants in FP64: the leaf
    expansions and propagation of Section 3.4, then for every direction the s -> 0 limit
    sum_B e^{-ik xhat.y_B} / (4 pi) Interp(F_B)(0, theta, phi) over the level-3 boxes (the
    plan keeps every is = 0 segment of level 3).  xhat: (M, 3) unit directions.  Returns
    ((nrhs, M) complex128, info dict)."""
    x, n, w = _geom(points, normals, weights)
    N = x.shape[0]
    s = _dens(sigma, N)
    nrhs = s.shape[0]
    xh = np.ascontiguousarray(xhat, dtype=np.float64).reshape(-1, 3)
    M = xh.shape[0]
    out = np.zeros((nrhs, M), dtype=np.complex128)
    info = OracleInfo()
    p = params.to_c()
    rc = lib().oracle_ifgf_far_field(ctypes.byref(p), ctypes.c_int64(N), _dptr(x), _dptr(n), _dptr(w),
                                     ctypes.c_int(nrhs), s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     ctypes.c_int64(M), _dptr(xh),
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(info))
    if rc != 0:
        raise RuntimeError(f"oracle_ifgf_far_field failed ({rc})")
    return out, _info_dict(info)


def _info_dict(info) -> dict:
    D = info.D
    d = {
        "D": D,
        "root_center": tuple(info.root_center),
        "root_side": info.root_side,
        "nbox": [info.nbox[i] for i in range(D + 1)],
        "ns": [info.ns[i] for i in range(D + 1)],
        "nC": [info.nC[i] for i in range(D + 1)],
        "split": [info.split[i] for i in range(D + 1)],
        "nrc": [info.nrc[i] for i in range(D + 1)],
        "cousin_evals": [info.cousin_evals[i] for i in range(D + 1)],
        "prop_evals": [info.prop_evals[i] for i in range(D + 1)],
        "leaf_evals": info.leaf_evals,
        "near_pairs": info.near_pairs,
    }
    return d


def auto_levels(points, leaf_target=64.0) -> int:
    x = np.ascontiguousarray(points, dtype=np.float64)
    return int(lib().oracle_auto_levels(ctypes.c_int64(x.shape[0]), _dptr(x), ctypes.c_double(leaf_target)))


def kernel(k, eta, x, y, ny) -> complex:
    o = np.zeros(2)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, ny)]
    lib().oracle_kernel(ctypes.c_double(k), ctypes.c_double(eta), _dptr(a[0]), _dptr(a[1]), _dptr(a[2]), _dptr(o))
    return complex(o[0], o[1])


def layer_kernels(k, x, y, ny):
    """(Phi(x, y), dPhi/dnu(y)) of Eq. GreenFunction and Eq. double_layer."""
    o = np.zeros(4)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, ny)]
    lib().oracle_layer_kernels(ctypes.c_double(k), _dptr(a[0]), _dptr(a[1]), _dptr(a[2]), _dptr(o))
    return complex(o[0], o[1]), complex(o[2], o[3])


def wfactors(k, eta, x, y0, h, y, ny, split: bool, literal: bool = False):
    """Analytic factors (W_C,) or (W2, W13) at x for source y of the box (y0, h)."""
    o = np.zeros(4)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y0, y, ny)]
    lib().oracle_wfactors(ctypes.c_double(k), ctypes.c_double(eta), _dptr(a[0]), _dptr(a[1]), ctypes.c_double(h),
                          _dptr(a[2]), _dptr(a[3]), ctypes.c_int(int(split)), ctypes.c_int(int(literal)), _dptr(o))
    return (complex(o[0], o[1]), complex(o[2], o[3])) if split else (complex(o[0], o[1]),)


def cheb_interp_1d(values, t) -> float:
    v = np.ascontiguousarray(values, dtype=np.float64)
    return float(lib().oracle_cheb_interp_1d(ctypes.c_int(v.shape[0]), _dptr(v), ctypes.c_double(t)))


def cube_sphere_patches(n: int, m: int):
    """Patch id, node index and node -> point map of the cube-sphere ordering of
    ``workloads.cube_sphere(n, m)`` (faces, then 'ij' meshgrid of face parameters)."""
    P = n // m
    idx = np.arange(6 * n * n)
    f = idx // (n * n)
    loc = idx % (n * n)
    iu, iv = loc // n, loc % n
    q = f * P * P + (iu // m) * P + (iv // m)
    nd = (iu % m) * m + (iv % m)
    node_of = np.empty(6 * P * P * m * m, dtype=np.int32)
    node_of[q * m * m + nd] = idx
    return q.astype(np.int32), nd.astype(np.int32), node_of


def rp_correction_sphere(points, normals, weights, n: int, m: int, radius: float, k: float, eta: float,
                         delta: float | None = None, Nbeta: int = 48, dgrade: float = 5.0):
    """Rectangular-polar correction C (rows = targets) for a cube-sphere surface.

    Returns (rowptr int64 (N+1,), col int32 (nnz,), val complex128 (nnz,)).  delta defaults
    to the nominal sub-patch side pi R / (2P)."""
    x, nu, w = _geom(points, normals, weights)
    N = x.shape[0]
    P = n // m
    q, nd, node_of = cube_sphere_patches(n, m)
    if delta is None:
        delta = math.pi * radius / (2 * P)
    lo, hi = x.min(0), x.max(0)
    L = float((hi - lo).max() * (1 + 2.0 ** -30))
    rp = ctypes.POINTER(ctypes.c_int64)()
    cp = ctypes.POINTER(ctypes.c_int32)()
    vp = ctypes.POINTER(ctypes.c_double)()
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    rc = lib().oracle_rp_correction(ctypes.c_int64(N), _dptr(x), _dptr(nu), _dptr(w), ip(q), ip(nd), ip(node_of),
                                    ctypes.c_double(radius), ctypes.c_int(P), ctypes.c_int(m), ctypes.c_double(k),
                                    ctypes.c_double(eta), ctypes.c_double(delta), ctypes.c_int(Nbeta),
                                    ctypes.c_double(dgrade), ctypes.c_double(1e-14 * L), ctypes.byref(rp),
                                    ctypes.byref(cp), ctypes.byref(vp))
    if rc != 0:
        raise RuntimeError(f"oracle_rp_correction failed ({rc})")
    rowptr = np.ctypeslib.as_array(rp, shape=(N + 1,)).copy()
    nnz = int(rowptr[-1])
    col = np.ctypeslib.as_array(cp, shape=(max(nnz, 1),))[:nnz].copy()
    val = np.ctypeslib.as_array(vp, shape=(max(2 * nnz, 2),))[:2 * nnz].copy().view(np.complex128)
    for ptr in (rp, cp, vp):
        lib().oracle_rp_free(ctypes.cast(ptr, ctypes.c_void_p))
    return rowptr, col, val


def csr_apply(rowptr, col, val, sigma) -> np.ndarray:
    """Plain sparse product (C sigma)_l = sum_{j in row l} val_j sigma_{col_j}, per rhs."""
    s = np.asarray(sigma, dtype=np.complex128)
    if s.ndim == 1:
        s = s[None, :]
    rp = np.asarray(rowptr, dtype=np.int64)
    cl = np.asarray(col, dtype=np.int64)
    v = np.asarray(val, dtype=np.complex128)
    out = np.zeros((s.shape[0], rp.shape[0] - 1), dtype=np.complex128)
    for l in range(rp.shape[0] - 1):
        j0, j1 = rp[l], rp[l + 1]
        out[:, l] = s[:, cl[j0:j1]] @ v[j0:j1]
    return out


def _root_side(x) -> float:
    lo, hi = x.min(0), x.max(0)
    return float((hi - lo).max() * (1 + 2.0 ** -30))


def field(points, normals, weights, k, eta, sigma, targets, layer=0) -> np.ndarray:
    """Combined-layer potential of Eq. CombinedLayer at arbitrary targets x, discretised with
    the surface quadrature (the off-surface counterpart of Eq. field1):

        u(x) = sum_m [dPhi(x, y_m)/dnu(y_m) - i eta Phi(x, y_m)] w_m sigma_m
        (layer 1: the dPhi/dnu term alone; layer 2: Phi alone),
        Phi = e^{ikr} / (4 pi r)                      (Eq. GreenFunction)
        dPhi/dnu(y) = e^{ikr} (1 - ikr) <x - y, nu(y)> / (4 pi r^3)   (Eq. double_layer)

    Every source is summed (targets are not surface points); a pair closer than 1e-14 times
    the root-box side contributes 0, the rule of the on-surface sum.  sigma: (nrhs, N);
    targets: (M, 3); returns (nrhs, M) complex128."""
    x, nu, w = _geom(points, normals, weights)
    N = x.shape[0]
    s = _dens(sigma, N)
    t = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
    tol = 1e-14 * _root_side(x)
    ws = s * w[None, :]
    out = np.zeros((s.shape[0], t.shape[0]), dtype=np.complex128)
    chunk = max(1, 4_000_000 // N)  # targets per block of pairs (bounds the temporaries)
    for j0 in range(0, t.shape[0], chunk):
        d = t[j0:j0 + chunk, None, :] - x[None, :, :]          # x - y, (c, N, 3)
        r = np.sqrt(np.einsum("cni,cni->cn", d, d))
        dn = np.einsum("cni,ni->cn", d, nu)                     # <x - y, nu(y)>
        keep = r >= tol
        rr = np.where(keep, r, 1.0)
        e = np.exp(1j * k * rr) / (4.0 * math.pi * rr)
        dl = e * (1.0 - 1j * k * rr) * dn / rr ** 2
        K = e if layer == 2 else dl if layer == 1 else dl - 1j * eta * e
        K = np.where(keep, K, 0.0)
        out[:, j0:j0 + chunk] = ws @ K.T
    return out


def far_field(points, normals, weights, k, eta, sigma, xhat, layer=0) -> np.ndarray:
    """Far-field pattern of Eq. FarField with the surface quadrature:

        u_inf(xhat) = (1 / 4 pi) sum_m [-i k <xhat, nu_m> - i eta] e^{-i k <xhat, y_m>} w_m sigma_m

    (d/dnu(y) of e^{-ik xhat.y} is -ik xhat.nu(y); layer 1 keeps that term alone, layer 2 replaces the
    bracket by 1).  sigma: (nrhs, N); xhat: (M, 3) directions,
    used as given; returns (nrhs, M) complex128."""
    x, nu, w = _geom(points, normals, weights)
    N = x.shape[0]
    s = _dens(sigma, N)
    xh = np.ascontiguousarray(xhat, dtype=np.float64).reshape(-1, 3)
    ws = s * w[None, :]
    out = np.zeros((s.shape[0], xh.shape[0]), dtype=np.complex128)
    chunk = max(1, 4_000_000 // N)  # directions per block of terms (bounds the temporaries)
    for j0 in range(0, xh.shape[0], chunk):
        d = xh[j0:j0 + chunk]
        c = 1.0 if layer == 2 else -1j * k * (d @ nu.T) - (0.0 if layer == 1 else 1j * eta)
        K = c * np.exp(-1j * k * (d @ x.T)) / (4.0 * math.pi)  # (c, N)
        out[:, j0:j0 + chunk] = ws @ K.T
    return out
