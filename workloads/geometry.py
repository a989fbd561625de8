"""Seeded synthetic surfaces and densities (inputs only, no IFGF arithmetic).

Surfaces follow the paper's discretisation recipe (Section 4): the surface is a
union of logical-quadrilateral patches (Eq. param_def), each carrying a tensor
grid of Chebyshev-Gauss (Fejer first-rule) nodes (Eq. FejersNodes) with the
Fejer weights of Eq. FejersWeights; the quadrature area weight of a node is
``w_i * w_j * J`` (Eq. ReguIntOpQuadrature), J the surface Jacobian.

Cube-sphere grids are equiangular: a face parameter ``u in (-1, 1)`` maps to
``X = tan(pi u / 4)``, the face point ``(X, Y, 1)`` (permuted per face) is
projected on the unit sphere.  A face of ``n x n`` points is split in
``(n/m)^2`` sub-patches of ``m x m`` Fejer nodes each.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Surface:
    """A discretised closed surface.

    points, normals: (N, 3) float64; normals are outward unit vectors.
    weights: (N,) float64 quadrature area weights (sum ~ surface area).
    patch: (N,) int32 patch id; uv: (N, 2) float64 patch parameters.
    """

    name: str
    points: np.ndarray
    normals: np.ndarray
    weights: np.ndarray
    patch: np.ndarray
    uv: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.points.shape[0])

    def diameter(self) -> float:
        ext = self.points.max(0) - self.points.min(0)
        return float(ext.max())


def fejer_nodes(m: int) -> np.ndarray:
    """Chebyshev-Gauss nodes cos(pi (2i+1) / (2m)), i = 0..m-1 (Eq. FejersNodes)."""
    i = np.arange(m)
    return np.cos(np.pi * (2 * i + 1) / (2 * m))


def fejer_weights(m: int) -> np.ndarray:
    """Fejer first-rule weights on (-1, 1) (Eq. FejersWeights)."""
    j = np.arange(m)
    acc = np.zeros(m)
    for ell in range(1, m // 2 + 1):
        acc += np.cos(ell * np.pi * (2 * j + 1) / m) / (4.0 * ell * ell - 1.0)
    return (2.0 / m) * (1.0 - 2.0 * acc)


def _face_params(n: int, m: int):
    """Face parameters u (length n) and 1-D weights, for n/m sub-patches of m nodes."""
    if n % m:
        raise ValueError("n must be a multiple of m")
    P = n // m
    t = fejer_nodes(m)
    wt = fejer_weights(m)
    u = np.empty(n)
    w = np.empty(n)
    sub = np.empty(n, dtype=np.int64)
    for p in range(P):
        u[p * m:(p + 1) * m] = -1.0 + (2 * p + 1 + t) / P
        w[p * m:(p + 1) * m] = wt / P
        sub[p * m:(p + 1) * m] = p
    return u, w, sub, P


_FACES = [(0, 1.0), (0, -1.0), (1, 1.0), (1, -1.0), (2, 1.0), (2, -1.0)]


def _face_frame(ax: int, sg: float):
    """Unit vectors (e_X, e_Y, e_n) of a cube face: face point = X e_X + Y e_Y + e_n."""
    e = np.eye(3)
    o1, o2 = (ax + 1) % 3, (ax + 2) % 3
    return e[o1], e[o2] * sg, e[ax] * sg


def _cube_directions(n: int, m: int):
    """Unit directions q(u, v), their u/v derivatives and the 2-D parameter weights."""
    u, w1, sub, P = _face_params(n, m)
    U, V = np.meshgrid(u, u, indexing="ij")
    WU, WV = np.meshgrid(w1, w1, indexing="ij")
    SU, SV = np.meshgrid(sub, sub, indexing="ij")
    X = np.tan(np.pi * U / 4)
    Y = np.tan(np.pi * V / 4)
    dX = (np.pi / 4) * (1 + X * X)
    dY = (np.pi / 4) * (1 + Y * Y)
    qs, qu, qv, ws, pid, uvs = [], [], [], [], [], []
    for f, (ax, sg) in enumerate(_FACES):
        eX, eY, en = _face_frame(ax, sg)
        p = X[..., None] * eX + Y[..., None] * eY + en
        rho = np.sqrt(1 + X * X + Y * Y)[..., None]
        q = p / rho
        pu = dX[..., None] * eX
        pv = dY[..., None] * eY
        # d(p/|p|) = (I - q q^T) dp / |p|
        du = (pu - q * np.sum(q * pu, -1, keepdims=True)) / rho
        dv = (pv - q * np.sum(q * pv, -1, keepdims=True)) / rho
        qs.append(q.reshape(-1, 3))
        qu.append(du.reshape(-1, 3))
        qv.append(dv.reshape(-1, 3))
        ws.append((WU * WV).reshape(-1))
        pid.append((f * P * P + SU * P + SV).reshape(-1))
        uvs.append(np.stack([U, V], -1).reshape(-1, 2))
    return (np.concatenate(qs), np.concatenate(qu), np.concatenate(qv),
            np.concatenate(ws), np.concatenate(pid).astype(np.int32), np.concatenate(uvs))


def _finish(name, x, xu, xv, wpar, pid, uv, meta):
    nrm = np.cross(xu, xv)
    J = np.linalg.norm(nrm, axis=1)
    nrm = nrm / J[:, None]
    # orient outward (all bodies here are star-shaped about the origin)
    sgn = np.sign(np.sum(nrm * x, axis=1))
    nrm = nrm * sgn[:, None]
    return Surface(name, np.ascontiguousarray(x), np.ascontiguousarray(nrm),
                   np.ascontiguousarray(wpar * J), pid, uv, meta)


def patch_node_index(s: Surface) -> np.ndarray:
    """For every point, q * m^2 + i * m + j: the point is node (i, j) of patch q, where i and j
    index the Chebyshev-Gauss nodes of Eq. FejersNodes (cos(pi (2i+1) / (2m))) along the patch's
    own u and v parameters.  For the cube-sphere family (sphere, ellipsoid, star body)."""
    n, m = int(s.meta["n"]), int(s.meta["m"])
    P = n // m
    t = fejer_nodes(m)
    pid = s.patch.astype(np.int64)
    su, sv = (pid // P) % P, pid % P
    ul = P * (s.uv[:, 0] + 1.0) - (2 * su + 1)  # local patch parameters in (-1, 1)
    vl = P * (s.uv[:, 1] + 1.0) - (2 * sv + 1)
    i = np.argmin(np.abs(ul[:, None] - t[None, :]), axis=1)
    j = np.argmin(np.abs(vl[:, None] - t[None, :]), axis=1)
    return (pid * m * m + i * m + j).astype(np.int32)


def cube_sphere(n: int, m: int | None = None, radius: float = 1.0) -> Surface:
    """Sphere of the given radius: 6 faces x n x n points, m x m Fejer sub-patches.

    Normals are exact (x / |x|); the area weight is w_i w_j times the
    equiangular Jacobian (pi/4)^2 (1+X^2)(1+Y^2) / (1+X^2+Y^2)^(3/2) / P^2.
    """
    m = n if m is None else m
    q, qu, qv, w, pid, uv = _cube_directions(n, m)
    s = _finish("sphere", radius * q, radius * qu, radius * qv, w, pid, uv,
                {"n": n, "m": m, "radius": radius})
    s.normals = np.ascontiguousarray(q)  # exact normals
    return s


def ellipsoid(n: int, m: int, axes) -> Surface:
    """Ellipsoid x = diag(axes) q(u, v) on the cube-sphere direction grid."""
    A = np.asarray(axes, dtype=np.float64)
    q, qu, qv, w, pid, uv = _cube_directions(n, m)
    return _finish("ellipsoid", q * A, qu * A, qv * A, w, pid, uv,
                   {"n": n, "m": m, "axes": A.tolist()})


def _real_ylm(l: int, mm: int, theta, phi):
    """Real orthonormal spherical harmonic Y_lm(theta, phi)."""
    from scipy.special import lpmv

    am = abs(mm)
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    # lpmv includes the Condon-Shortley phase; it cancels in |Y|^2 and is irrelevant here
    P = lpmv(am, l, np.cos(theta))
    if mm == 0:
        return norm * P
    if mm > 0:
        return math.sqrt(2) * norm * P * np.cos(am * phi)
    return math.sqrt(2) * norm * P * np.sin(am * phi)


def star_body(n: int, m: int, seed: int, lmax: int = 6, amp: float = 0.2) -> Surface:
    """Smooth star-shaped body r(q) = 1 + amp * sum_{l=1..lmax} a_lm Y_lm(q).

    a_lm ~ N(0, 1/l^2) from ``numpy.random.default_rng(seed)``; redrawn with the
    next draw while min r < 0.3.  Normals and Jacobians use central differences
    of the analytic map in (u, v) (step 1e-5).
    """
    rng = np.random.default_rng(seed)
    while True:
        coeffs = [(l, mm, rng.normal(0.0, 1.0 / l)) for l in range(1, lmax + 1) for mm in range(-l, l + 1)]
        qq, _, _, _, _, _ = _cube_directions(8, 8)
        rr = _star_radius(qq, coeffs, amp)
        if rr.min() >= 0.3:
            break
    u, w1, sub, P = _face_params(n, m)
    U, V = np.meshgrid(u, u, indexing="ij")
    WU, WV = np.meshgrid(w1, w1, indexing="ij")
    SU, SV = np.meshgrid(sub, sub, indexing="ij")
    h = 1e-5
    xs, xus, xvs, ws, pid, uvs = [], [], [], [], [], []
    for f, (ax, sg) in enumerate(_FACES):
        eX, eY, en = _face_frame(ax, sg)

        def xmap(UU, VV):
            X = np.tan(np.pi * UU / 4)
            Y = np.tan(np.pi * VV / 4)
            p = X[..., None] * eX + Y[..., None] * eY + en
            q = p / np.linalg.norm(p, axis=-1, keepdims=True)
            return q * _star_radius(q.reshape(-1, 3), coeffs, amp).reshape(q.shape[:-1])[..., None]

        x = xmap(U, V)
        xu = (xmap(U + h, V) - xmap(U - h, V)) / (2 * h)
        xv = (xmap(U, V + h) - xmap(U, V - h)) / (2 * h)
        xs.append(x.reshape(-1, 3))
        xus.append(xu.reshape(-1, 3))
        xvs.append(xv.reshape(-1, 3))
        ws.append((WU * WV).reshape(-1))
        pid.append((f * P * P + SU * P + SV).reshape(-1))
        uvs.append(np.stack([U, V], -1).reshape(-1, 2))
    return _finish("star", np.concatenate(xs), np.concatenate(xus), np.concatenate(xvs),
                   np.concatenate(ws), np.concatenate(pid).astype(np.int32), np.concatenate(uvs),
                   {"n": n, "m": m, "seed": seed, "lmax": lmax, "amp": amp})


def _star_radius(q, coeffs, amp):
    theta = np.arccos(np.clip(q[:, 2], -1.0, 1.0))
    phi = np.arctan2(q[:, 1], q[:, 0])
    r = np.ones(q.shape[0])
    for l, mm, a in coeffs:
        r += amp * a * _real_ylm(l, mm, theta, phi)
    return r


def sphere_workload(n: int, m: int, wavelengths_diameter: float, radius: float = 1.0):
    """Sphere with 6 n^2 points whose diameter is the given number of wavelengths.

    Returns (surface, k).  k = 2 pi / lambda with lambda = 2 radius / wavelengths.
    """
    s = cube_sphere(n, m, radius)
    lam = 2.0 * radius / wavelengths_diameter
    return s, 2.0 * math.pi / lam


def two_spheres(n_big: int = 16, n_small: int = 24, radius_small: float = 0.15, offset: float = 1.6,
                m: int = 8) -> Surface:
    """A non-uniform point set: the unit cube-sphere (6 n_big^2 points) and a cube-sphere of radius
    radius_small centred at (offset, 0, 0) with 6 n_small^2 points.  With the defaults (1,536 and
    3,456 points) the small sphere's point density is 20x the large one's, in one corner of the
    root box.  Patch ids of the small sphere follow the large sphere's."""
    a, b = cube_sphere(n_big, m), cube_sphere(n_small, m)
    c = np.array([offset, 0.0, 0.0])
    return Surface("two_spheres", np.concatenate([a.points, radius_small * b.points + c]),
                   np.concatenate([a.normals, b.normals]),
                   np.concatenate([a.weights, radius_small ** 2 * b.weights]),
                   np.concatenate([a.patch, b.patch + int(a.patch.max()) + 1]).astype(np.int32),
                   np.concatenate([a.uv, b.uv]), dict(n_big=n_big, n_small=n_small, m=m))


def random_density(N: int, nrhs: int, seed: int) -> np.ndarray:
    """Complex128 density, shape (nrhs, N) (one row per right-hand side).

    Real and imaginary parts are i.i.d. N(0, 1) from default_rng(seed).
    """
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((nrhs, N))
    im = rng.standard_normal((nrhs, N))
    return re + 1j * im


def scatterer_batch(seed: int = 3, count: int = 24, n_min: int = 64, n_max: int = 256, d_min: float = 2.0,
                    d_max: float = 24.0):
    """Uneven batch of scatterers: spheres (even index) and ellipsoids with axis ratios
    from U[1, 3] (odd index); diameters D_i ~ U[d_min, d_max] wavelengths; points
    N_i ~ 20k + 380k (D_i^2 - 4) / 572 rounded to 6 n^2 with n a multiple of 8 in
    [n_min, n_max].  Returns a list of (surface, k) with k = 2 pi D_i / diameter."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dw = rng.uniform(d_min, d_max)
        nt = 20000 + 380000 * (dw * dw - 4) / 572
        n = int(np.clip(round(math.sqrt(max(nt, 1) / 6) / 8) * 8, n_min, n_max))
        if i % 2 == 0:
            s = cube_sphere(n, 8)
        else:
            s = ellipsoid(n, 8, (1.0, rng.uniform(1, 3), rng.uniform(1, 3)))
        out.append((s, 2 * math.pi * dw / s.diameter()))
    return out
