"""Seeded synthetic inputs: triangulated solids and target sets.

This package is the only code that the FP64 oracle and the CUDA library have
in common.  It produces plain arrays (vertices, triangles, a sigma per
triangle, targets) and holds none of the level-set method's arithmetic: no
kernel, no quadrature rule, no pseudonormal, no Newton step.  The few vector
operations it does (a triangle's area for the sigma rule of a workload, a face
normal to place a target at a signed offset from the surface) exist only to
build inputs.

Random numbers come from numpy's Philox counter-based generator, seeded per
workload.  The paper's own inputs (CAD meshes from GiD/FreeCAD, Sec. 5) are
not available; these generators stand in for them with the same kinds of
structure: flat faces with sharp edges (cube), strong grading and jitter
(torus), multiscale features (bumped icosphere), and many small meshes of
varied size (ellipsoids).
"""
from .meshes import (  # noqa: F401
    Mesh,
    QuadMesh,
    quadratic_from_flat,
    quadratic_icosphere,
    quadratic_torus,
    cube,
    torus,
    icosphere,
    bumped_icosphere,
    ellipsoid,
    sigma_half_sqrt2area,
    targets_uniform,
    targets_near_surface,
    rng,
)
from .workloads import (  # noqa: F401
    cube_c1,
    torus_c2,
    icosphere_c3,
    ellipsoid_batch_c4,
    serve_stream_c5,
)
