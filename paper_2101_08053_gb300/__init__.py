"""GB300-native (sm_103a) formation of Galerkin mass matrices of trimmed
bi-variate B-spline patches by row-wise weighted quadrature with sum
factorisation (Marussig, "Fast formation and assembly of isogeometric Galerkin
matrices for trimmed patches"), with hybrid Gauss and discontinuous weighted
quadrature for cut basis functions, the L2 projection built on the matrix, and its adjoint with respect to a
density spline in the coefficient.

The compute path is the C-ABI library libtrimwq.so (include/trimwq.h); this
package only builds it and marshals arguments to it.
"""
from .api import Batch, Patch, ProjectionLoss, TWError, launch_count, load, projection_loss  # noqa: F401
