"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This package holds no arithmetic of the IFGF method: it only produces surface
discretisations (points, outward unit normals, quadrature area weights) and
seeded complex densities.  See ``workloads.geometry``.
"""
from .geometry import (  # noqa: F401
    fejer_nodes,
    fejer_weights,
    cube_sphere,
    ellipsoid,
    patch_node_index,
    star_body,
    sphere_workload,
    two_spheres,
    random_density,
    scatterer_batch,
    Surface,
)
