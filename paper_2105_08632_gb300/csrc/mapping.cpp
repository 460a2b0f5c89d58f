// Quadratic element mappings (see mapping.hpp).  The shape functions are
// written in closed form:
//   simplices  barycentric coordinates l: vertex node l_i (2 l_i - 1), edge
//              node between vertices i and j 4 l_i l_j;
//   quadrilaterals / hexahedra  products of the 1D quadratic Lagrange
//              polynomials on {-1, 0, 1};
//   prisms     triangle basis in (x~, y~) times the 1D basis in z~.
#include "mapping.hpp"

#include <stdexcept>

#include "refel.hpp"

namespace sdrt {

namespace {

// 1D quadratic Lagrange polynomial of node a in {-1, 0, 1} and its derivative.
double lag(int a, double t) { return a < 0 ? 0.5 * t * (t - 1) : a == 0 ? 1 - t * t : 0.5 * t * (t + 1); }
double dlag(int a, double t) { return a < 0 ? t - 0.5 : a == 0 ? -2 * t : t + 0.5; }

// Barycentric coordinates (nd + 1) of a reference simplex point and their
// constant gradients: l_0 = -(1 + sum x) / 2 on the tetrahedron, -(x + y) / 2
// on the triangle; l_i = (x_{i-1} + 1) / 2.
void bary(int nd, const double* x, double* l, double* dl) {
    double s = 0;
    for (int d = 0; d < nd; ++d) s += x[d];
    l[0] = nd == 2 ? -0.5 * s : -0.5 * (1 + s);
    for (int i = 0; i <= nd; ++i)
        for (int d = 0; d < nd; ++d) dl[i * nd + d] = i == 0 ? -0.5 : (i - 1 == d ? 0.5 : 0.0);
    for (int i = 1; i <= nd; ++i) l[i] = 0.5 * (x[i - 1] + 1);
}

// P2 simplex basis function of the node with coordinates xn: value and gradient.
void p2(int nd, const double* xn, const double* x, double& N, double* dN) {
    double ln[4], dln[12], l[4], dl[12];
    bary(nd, xn, ln, dln);
    bary(nd, x, l, dl);
    int idx[2], n = 0;
    for (int i = 0; i <= nd; ++i)
        if (ln[i] > 0.25) idx[n++] = i;           // 1 index: vertex node; 2: edge midpoint
    if (n == 1) {
        const int i = idx[0];
        N = l[i] * (2 * l[i] - 1);
        for (int d = 0; d < nd; ++d) dN[d] = (4 * l[i] - 1) * dl[i * nd + d];
    } else {
        const int i = idx[0], j = idx[1];
        N = 4 * l[i] * l[j];
        for (int d = 0; d < nd; ++d) dN[d] = 4 * (dl[i * nd + d] * l[j] + l[i] * dl[j * nd + d]);
    }
}

}  // namespace

std::vector<double> map_nodes(int shape) {
    const int nd = shape_ndim(shape);
    std::vector<double> out;
    const int n = nd == 2 ? 9 : 27;
    for (int c = 0; c < n; ++c) {
        double x[3] = {double(c % 3 - 1), double((c / 3) % 3 - 1), double(c / 9 - 1)};
        bool in = true;
        if (shape == TRI || shape == PRI) in = x[0] + x[1] <= 0;
        if (shape == TET) in = x[0] + x[1] + x[2] <= -1;
        if (in)
            for (int d = 0; d < nd; ++d) out.push_back(x[d]);
    }
    return out;
}

int map_nnodes(int shape) { return (int)map_nodes(shape).size() / shape_ndim(shape); }

void map_shape(int shape, const double* x, double* N, double* dN) {
    const int nd = shape_ndim(shape);
    const std::vector<double> X = map_nodes(shape);
    const int nn = (int)X.size() / nd;
    for (int k = 0; k < nn; ++k) {
        const double* xn = &X[(size_t)k * nd];
        double* g = dN + (size_t)k * nd;
        switch (shape) {
            case TRI:
            case TET: p2(nd, xn, x, N[k], g); break;
            case QUAD:
            case HEX: {
                double v = 1;
                for (int d = 0; d < nd; ++d) v *= lag((int)xn[d], x[d]);
                N[k] = v;
                for (int d = 0; d < nd; ++d) {
                    double t = dlag((int)xn[d], x[d]);
                    for (int o = 0; o < nd; ++o)
                        if (o != d) t *= lag((int)xn[o], x[o]);
                    g[d] = t;
                }
                break;
            }
            case PRI: {
                double Nt, dNt[2];
                p2(2, xn, x, Nt, dNt);
                const int a = (int)xn[2];
                N[k] = Nt * lag(a, x[2]);
                g[0] = dNt[0] * lag(a, x[2]);
                g[1] = dNt[1] * lag(a, x[2]);
                g[2] = Nt * dlag(a, x[2]);
                break;
            }
            default: throw std::runtime_error("bad shape");
        }
    }
}

}  // namespace sdrt
