// Quadratic element mappings of curved elements (host side, FP64).
//
// The paper maps each element from its reference element, x = M(x~), and
// evaluates the Jacobian J_ij = dM_i / dx~_j, its determinant and inverse
// analytically (Sec. 2, Eqs. "mapping_function", "mapping_jacobian",
// "inverse_mapping_jacobian").  Curved elements use the second-order Lagrange
// map M(x~) = sum_k X_k N_k(x~) on the nodes
//   { reference points with every coordinate in {-1, 0, 1} },
// lexicographic with x~ fastest: tri 6, quad 9, tet 10, pri 18, hex 27 nodes.
// N_k spans the type's quadratic space: total degree <= 2 on simplices, degree
// <= 2 per coordinate on quadrilaterals / hexahedra, their product on prisms.
#pragma once

#include <vector>

namespace sdrt {

// Number of mapping nodes of a shape.
int map_nnodes(int shape);
// Reference coordinates of the mapping nodes (nnodes x nd).
std::vector<double> map_nodes(int shape);
// Shape functions N[k] and gradients dN[k * nd + d] = dN_k / dx~_d at the
// reference point x (nd coordinates).
void map_shape(int shape, const double* x, double* N, double* dN);

}  // namespace sdrt
