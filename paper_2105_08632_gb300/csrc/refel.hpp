// Reference elements, point sets and FP64 SDRT operators (host side).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace sdrt {

enum Shape { TRI = 0, QUAD = 1, TET = 2, PRI = 3, HEX = 4 };

// One element type with its FP64 operators (paper App. A / App. B).
struct RefElement {
    int shape = 0, p = 0, nd = 0, nfaces = 0;
    int nsol = 0, nfe = 0, nfi = 0, nfiu = 0;
    std::vector<double> xs;        // nsol x nd   solution points
    std::vector<double> xfe;       // nfe x nd    external flux points
    std::vector<double> nfe_ref;   // nfe x nd    outward unit reference normals
    std::vector<int> fe_face;      // nfe         face of each external point
    std::vector<double> face_nrm;  // nfaces x nd outward unit reference normals
    std::vector<double> xfiu;      // nfiu x nd   unique internal flux points
    std::vector<int> fi_point;     // nfi         unique point of each internal DOF
    std::vector<int> fi_axis;      // nfi         reference axis of each internal DOF
    // Operators, row-major FP64.
    std::vector<double> M0;        // nfe  x nsol
    std::vector<double> M12;       // nfiu x nsol
    std::vector<double> M13;       // nsol x nfi
    std::vector<double> M14;       // nsol x nfe
    std::vector<double> M15;       // nd*nsol x nfi   (rows: axis outer)
    std::vector<double> M16;       // nd*nsol x nfe
    double cond_hint = 0;          // max |entry| of the inverse flux Vandermonde
    // Element quadrature exact for polynomials of degree 10 (ensemble
    // averages of the Taylor-Green diagnostics): Gauss-Legendre tensor rule
    // with 7 points per direction, collapsed (Duffy) onto simplices.
    std::vector<double> xq;        // nq x nd  points
    std::vector<double> wq;        // nq       weights (sum = reference volume)
    std::vector<double> Mq;        // nq x nsol solution nodal basis at the points
};

// Builds the element; throws std::runtime_error on failure.
RefElement build_ref_element(int shape, int p);

int shape_ndim(int shape);
int shape_nverts(int shape);
int shape_nfaces(int shape);
// Reference vertices (nverts x nd) and face vertex lists.
const std::vector<double>& ref_vertices(int shape);
const std::vector<std::vector<int>>& face_vertices(int shape);

// Gauss-Legendre nodes on [-1, 1], ascending.
std::vector<double> gauss_legendre(int n);
// Gauss-Legendre weights of those nodes.
std::vector<double> gauss_legendre_weights(const std::vector<double>& x);

// Quadrature rule on the reference element of `shape` with n Gauss-Legendre
// points per direction (tensor rule; collapsed onto simplices): points (nq x nd)
// and weights.
void element_quadrature(int shape, int n, std::vector<double>& X, std::vector<double>& W);

}  // namespace sdrt
