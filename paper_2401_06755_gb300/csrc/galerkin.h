// Galerkin coarse operators for a coefficient field (galerkin.cu).
#pragma once

#include "internal.h"

namespace nn4 {

struct PlanImpl;

// Coefficients of a general symmetric 27-point operator on a level: 27 arrays of the level's
// size and pitch, array d = (dx+1) + 3 (dy+1) + 9 (dz+1) holding A[i, i + (dx, dy, dz)] at node i
// (zero where the neighbour lies outside the grid or either node is a Dirichlet node; 1 on the
// diagonal of Dirichlet nodes).
constexpr int kA27 = 27;

// Level 0 -> 1: A_1 = P^T A_0 P with A_0 the operator of Eq. k-T for the FP64 coefficient field k
// (pitch gf.pitch) and constant-coefficient spacing hf.  `ct` selects the arithmetic (NN4_F64 or
// NN4_F32); `out` is a 27-array block of that type with pitch gc.pitch.
int launch_galerkin_from_k(nn4_dtype ct, const double* k, const LevelGeom& gf, const double hf[3], void* out,
                           const LevelGeom& gc, cudaStream_t s);
// Level l -> l+1 from the 27-array block of level l (type ct, pitch gf.pitch).
int launch_galerkin_next(nn4_dtype ct, const void* af, const LevelGeom& gf, void* out, const LevelGeom& gc,
                         cudaStream_t s);
// Elementwise conversion of a 27-array block from type ct to type dt (same pitch).
int launch_convert27(nn4_dtype ct, const void* src, nn4_dtype dt, void* dst, const LevelGeom& g, cudaStream_t s);

// Sets the 13 lower arrays of a 27-array block of type ct (NN4_F64 or NN4_F32) from the upper
// ones (A[i, i+D] := A[i+D, i]), making the stored operator exactly symmetric.
int launch_symmetrize27(nn4_dtype ct, void* a27, const LevelGeom& g, cudaStream_t s);

// Residual / Jacobi passes with a symmetric 27-array operator (OP_RESIDUAL, OP_JACOBI); only the
// upper arrays 13..26 are read.  x and b must be 16-byte aligned with pitch * element size a
// multiple of 16 bytes (TMA tiles).
int launch_pass27(nn4_dtype dt, int op, const PassArgs& a, const void* x, const void* a27, cudaStream_t s);

// Builds the coefficient hierarchy of plan P (levels >= 1) and returns the coarsest operator as
// a dense row-major matrix over all coarsest nodes in `dense` (defined in plan.cu).
int build_galerkin_hierarchy(PlanImpl* P, std::vector<double>& dense);

}  // namespace nn4
