// mpm_mg.cu -- block preconditioner for the Newton system (Sec. 3.4 solves
// it with a Schur-complement block preconditioner; here the sub-solves are
// geometric multigrid on the structured background grid instead of AMG).
//
//   J = [A  B1]      M^{-1} = [A^-1  -A^-1 B1 S^-1]      S ~ C + C_stab - B2 diag(A)^-1 B1
//       [B2 C ]               [0          S^-1     ]
//
// applied as  z_p = S^-1 v_p,  z_u = A^-1 (v_u - B1 z_p), with A^-1 and S^-1
// each one multigrid V-cycle.  The hierarchies are built from the unscaled
// physical blocks (Galerkin coarse operators then weigh every node by its
// physical stiffness / mass); the Krylov solver sees the preconditioner of its
// symmetrically scaled system as D^-1 M^-1 D^-1.  Dirichlet and inactive DOFs
// are masked out of the finest restriction, prolongation and Galerkin
// product.  S is assembled on the sparsity of J (the fill of
// B2 diag(A)^-1 B1 outside it is lumped onto the diagonal, which keeps the
// row sums of S).
//
// Multigrid: vertex-centred factor-2 coarsening of the node lattice, bilinear
// (trilinear) prolongation P, Galerkin coarse operators P^T A P stored as
// dense 5^d-point block stencils (the Galerkin product of a stencil of radius
// <= 3 with bilinear P has radius <= 2 and stays at 2), damped block-Jacobi
// smoothing, and an exact solve on the coarsest grid (a dense inverse formed
// at set-up by LU with partial pivoting).  Every kernel is a gather with a
// fixed summation order (deterministic, no atomics).
#include <math.h>

#include <utility>

#include "mpm_internal.cuh"

// The implementation body (kernels and host sequencing) is written once in
// terms of `real` and compiled for FP64 (the FP64 path and the inspection
// calls) and for FP32 (the mixed-precision path).
namespace upmpm {

#define MG_REAL double
#define MG_NS mg64
#include "mpm_mg_impl.cuh"
#undef MG_NS
#undef MG_REAL

#define MG_REAL float
#define MG_NS mg32
#include "mpm_mg_impl.cuh"
#undef MG_NS
#undef MG_REAL

}  // namespace upmpm
