"""GB300-native (sm_103a) formation of Galerkin mass matrices of trimmed
bi-variate B-spline patches by row-wise weighted quadrature with sum
factorisation (Marussig, "Fast formation and assembly of isogeometric Galerkin
matrices for trimmed patches"), with hybrid Gauss and discontinuous weighted
quadrature for cut basis functions, the L2 projection built on the matrix, its
extended B-spline form, and its adjoint with respect to a density spline in the
coefficient.

The compute path is the C-ABI library libtrimwq.so (include/trimwq.h); this
package only builds it and marshals arguments to it.

Typical use (device tensors are torch CUDA tensors; `spec` is a patch
description: degree, knot vectors, trimming curve, geometry, coefficient,
method -- see api.make_patch_desc)::

    P = Patch(spec)                          # all patch tables on the GPU
    rp, col, val = P.form_mass("fp64")       # CSR of M (also "fp32", "fp32x2")
    u, iters, rel = P.l2_project(f, (rp, col, val))
    # extended B-splines: stable coefficients on cut functions
    xcsr = P.form_mass_extended((rp, col, val))
    u, iters, rel = P.l2_project_extended(f, xcsr)
    # many patches in one persistent launch
    B = Batch([P1, P2, ...], [P1.alloc_csr(), P2.alloc_csr(), ...], "fp64")
    B.run()
    # gradient of a projection loss with respect to the density coefficients
    L = projection_loss(d, spec, f, g, extended=True); L.backward()
"""
from .api import Batch, Patch, ProjectionLoss, TWError, launch_count, load, projection_loss  # noqa: F401
