// Reference elements, point sets and FP64 SDRT operators (host side).
//
// Point sets follow paper App. A: Gauss-Legendre (GL) points on tensor-product
// elements and on quadrilateral faces; on simplices the paper's Williams-Shunn
// points (coordinates not printed in the paper) are replaced by a symmetric,
// derivable family: the barycentric lattice of degree q warped by the
// (q+1)-point GL rule, lambda_a = (1 + m v_{i_a} - sum_{b != a} v_{i_b}) / (m + 1)
// (m = 2 triangle, 3 tetrahedron), which is invariant under every vertex
// permutation, so glued faces see coincident points in any orientation.
//
// Operators (paper Sec. 2.1 Vandermonde relations, App. B matrix form) are
// built from a Legendre-product modal basis: solution space P_p / Q_p /
// P_p(x,y) x P_p(z); Raviart-Thomas space (App. A) spanned by
//   simplex:  e_c L_a(x) (|a| <= p)  and  x * L_a(x) (|a| = p),
//   tensor:   e_c L_a(x) with a_c <= p+1, a_d <= p otherwise,
//   prism:    e_c L_a (c < 2, a0+a1 <= p, a2 <= p), (x,y,0) L_a (a0+a1 = p, a2 <= p),
//             e_2 L_a (a0+a1 <= p, a2 <= p+1),
// where L_a(x) = prod_d P_{a_d}(x_d) (Legendre polynomials).  x * L_a spans
// x * Pbar_p modulo P_p^ND because the top-degree part of L_a is a multiple of x^a.
#include "refel.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <stdexcept>

namespace sdrt {

namespace {

const std::vector<double> kVerts[5] = {
    {-1, -1, 1, -1, -1, 1},
    {-1, -1, 1, -1, 1, 1, -1, 1},
    {-1, -1, -1, 1, -1, -1, -1, 1, -1, -1, -1, 1},
    {-1, -1, -1, 1, -1, -1, -1, 1, -1, -1, -1, 1, 1, -1, 1, -1, 1, 1},
    {-1, -1, -1, 1, -1, -1, 1, 1, -1, -1, 1, -1, -1, -1, 1, 1, -1, 1, 1, 1, 1, -1, 1, 1},
};
const std::vector<std::vector<int>> kFaces[5] = {
    {{0, 1}, {1, 2}, {2, 0}},
    {{0, 1}, {1, 2}, {3, 2}, {0, 3}},
    {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}},
    {{0, 1, 2}, {0, 1, 4, 3}, {1, 2, 5, 4}, {0, 2, 5, 3}, {3, 4, 5}},
    {{0, 1, 2, 3}, {0, 1, 5, 4}, {1, 2, 6, 5}, {3, 2, 6, 7}, {0, 3, 7, 4}, {4, 5, 6, 7}},
};
// Outward reference normals (unnormalised).
const std::vector<std::vector<double>> kFaceNrm[5] = {
    {{0, -1}, {1, 1}, {-1, 0}},
    {{0, -1}, {1, 0}, {0, 1}, {-1, 0}},
    {{0, 0, -1}, {0, -1, 0}, {1, 1, 1}, {-1, 0, 0}},
    {{0, 0, -1}, {0, -1, 0}, {1, 1, 0}, {-1, 0, 0}, {0, 0, 1}},
    {{0, 0, -1}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, 0, 1}},
};

// Legendre polynomial P_n(x) and derivative by the three-term recurrence.
void legendre(int n, double x, double* P, double* dP) {
    P[0] = 1.0;
    dP[0] = 0.0;
    if (n >= 1) {
        P[1] = x;
        dP[1] = 1.0;
    }
    for (int k = 1; k < n; ++k) {
        P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
        dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k];
    }
}

// Barycentric coordinates of the warped simplex lattice of degree q (m = 2 or 3).
std::vector<std::vector<double>> warped_lattice(int dim, int q) {
    std::vector<double> g = gauss_legendre(q + 1);
    std::vector<double> v(q + 1);
    for (int i = 0; i <= q; ++i) v[i] = 0.5 * (g[i] + 1.0);
    std::vector<std::vector<double>> out;
    if (dim == 2) {
        for (int b = 0; b <= q; ++b)
            for (int a = 0; a + b <= q; ++a) {
                int c = q - a - b;
                double l1 = (1 + 2 * v[a] - v[b] - v[c]) / 3;
                double l2 = (1 + 2 * v[b] - v[a] - v[c]) / 3;
                double l0 = (1 + 2 * v[c] - v[a] - v[b]) / 3;
                out.push_back({l0, l1, l2});
            }
    } else {
        for (int c = 0; c <= q; ++c)
            for (int b = 0; b + c <= q; ++b)
                for (int a = 0; a + b + c <= q; ++a) {
                    int d = q - a - b - c;
                    int idx[4] = {d, a, b, c};
                    double sum = v[d] + v[a] + v[b] + v[c];
                    std::vector<double> lam(4);
                    for (int k = 0; k < 4; ++k) lam[k] = (1 + 4 * v[idx[k]] - sum) / 4;
                    out.push_back(lam);
                }
    }
    return out;
}

void push_bary(std::vector<double>& X, const std::vector<double>& lam, const double* V, const int* vid,
               int nv, int nd) {
    for (int d = 0; d < nd; ++d) {
        double s = 0;
        for (int k = 0; k < nv; ++k) s += lam[k] * V[vid[k] * nd + d];
        X.push_back(s);
    }
}

// Dense LU inverse with partial pivoting; throws if singular.
std::vector<double> invert(std::vector<double> A, int n) {
    std::vector<double> inv(n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = std::fabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(A[i * n + k]) > best) {
                best = std::fabs(A[i * n + k]);
                piv = i;
            }
        if (best < 1e-300) throw std::runtime_error("singular Vandermonde matrix");
        if (piv != k)
            for (int j = 0; j < n; ++j) {
                std::swap(A[k * n + j], A[piv * n + j]);
                std::swap(inv[k * n + j], inv[piv * n + j]);
            }
        double d = 1.0 / A[k * n + k];
        for (int j = 0; j < n; ++j) {
            A[k * n + j] *= d;
            inv[k * n + j] *= d;
        }
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            double f = A[i * n + k];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[i * n + j] -= f * A[k * n + j];
                inv[i * n + j] -= f * inv[k * n + j];
            }
        }
    }
    return inv;
}

struct Mode {
    int kind;   // 0: e_comp * L_a ; 1: (x_0..x_{nx-1}) * L_a
    int comp;   // component (kind 0) or nx (kind 1)
    int a[3];
};

std::vector<std::array<int, 3>> sol_multi(int shape, int p) {
    std::vector<std::array<int, 3>> out;
    int nd = shape_ndim(shape);
    for (int k = 0; k <= (nd == 3 ? p : 0); ++k)
        for (int j = 0; j <= p; ++j)
            for (int i = 0; i <= p; ++i) {
                bool ok;
                if (shape == TRI) ok = i + j <= p;
                else if (shape == TET) ok = i + j + k <= p;
                else if (shape == PRI) ok = i + j <= p;
                else ok = true;
                if (ok) out.push_back({i, j, k});
            }
    return out;
}

std::vector<Mode> rt_modes(int shape, int p) {
    std::vector<Mode> m;
    int nd = shape_ndim(shape);
    auto loop3 = [&](int mi, int mj, int mk, auto pred, auto emit) {
        for (int k = 0; k <= (nd == 3 ? mk : 0); ++k)
            for (int j = 0; j <= mj; ++j)
                for (int i = 0; i <= mi; ++i)
                    if (pred(i, j, k)) emit(i, j, k);
    };
    if (shape == TRI || shape == TET) {
        for (int c = 0; c < nd; ++c)
            loop3(p, p, p, [&](int i, int j, int k) { return i + j + k <= p; },
                  [&](int i, int j, int k) { m.push_back({0, c, {i, j, k}}); });
        loop3(p, p, p, [&](int i, int j, int k) { return i + j + k == p; },
              [&](int i, int j, int k) { m.push_back({1, nd, {i, j, k}}); });
    } else if (shape == QUAD || shape == HEX) {
        for (int c = 0; c < nd; ++c)
            loop3(c == 0 ? p + 1 : p, c == 1 ? p + 1 : p, c == 2 ? p + 1 : p,
                  [](int, int, int) { return true; },
                  [&](int i, int j, int k) { m.push_back({0, c, {i, j, k}}); });
    } else {  // prism
        for (int c = 0; c < 2; ++c)
            loop3(p, p, p, [&](int i, int j, int) { return i + j <= p; },
                  [&](int i, int j, int k) { m.push_back({0, c, {i, j, k}}); });
        loop3(p, p, p, [&](int i, int j, int) { return i + j == p; },
              [&](int i, int j, int k) { m.push_back({1, 2, {i, j, k}}); });
        loop3(p, p, p + 1, [&](int i, int j, int) { return i + j <= p; },
              [&](int i, int j, int k) { m.push_back({0, 2, {i, j, k}}); });
    }
    return m;
}

// Values of L_a and of its partial derivatives at one point.
struct LegTab {
    double P[3][16], dP[3][16];
    void set(const double* x, int nd, int n) {
        for (int d = 0; d < 3; ++d) {
            double xd = d < nd ? x[d] : 0.0;
            legendre(n, xd, P[d], dP[d]);
        }
    }
    double L(const int* a, int nd) const {
        double v = 1;
        for (int d = 0; d < nd; ++d) v *= P[d][a[d]];
        return v;
    }
    double dL(const int* a, int nd, int dd) const {
        double v = 1;
        for (int d = 0; d < nd; ++d) v *= (d == dd ? dP[d][a[d]] : P[d][a[d]]);
        return v;
    }
};

}  // namespace

int shape_ndim(int s) { return (s == TRI || s == QUAD) ? 2 : 3; }
int shape_nverts(int s) { return (int)kVerts[s].size() / shape_ndim(s); }
int shape_nfaces(int s) { return (int)kFaces[s].size(); }
const std::vector<double>& ref_vertices(int s) { return kVerts[s]; }
const std::vector<std::vector<int>>& face_vertices(int s) { return kFaces[s]; }

std::vector<double> gauss_legendre(int n) {
    std::vector<double> x(n);
    std::vector<double> P(n + 2), dP(n + 2);
    for (int i = 0; i < n; ++i) {
        double r = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            legendre(n, r, P.data(), dP.data());
            double dr = P[n] / dP[n];
            r -= dr;
            if (std::fabs(dr) < 1e-16) break;
        }
        x[i] = r;
    }
    std::sort(x.begin(), x.end());
    return x;
}

std::vector<double> gauss_legendre_weights(const std::vector<double>& x) {
    const int n = (int)x.size();
    std::vector<double> w(n), P(n + 2), dP(n + 2);
    for (int i = 0; i < n; ++i) {
        legendre(n, x[i], P.data(), dP.data());
        w[i] = 2.0 / ((1.0 - x[i] * x[i]) * dP[n] * dP[n]);
    }
    return w;
}

void element_quadrature(int shape, int n, std::vector<double>& X, std::vector<double>& W) {
    const std::vector<double> g = gauss_legendre(n), w = gauss_legendre_weights(g);
    X.clear();
    W.clear();
    // Triangle x_i >= -1, x + y <= 0: x = (1 + a)(1 - b)/2 - 1, y = b, factor (1 - b)/2.
    auto tri = [&](std::vector<double>& Xt, std::vector<double>& Wt) {
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                Xt.push_back((1 + g[i]) * (1 - g[j]) / 2 - 1);
                Xt.push_back(g[j]);
                Wt.push_back(w[i] * w[j] * (1 - g[j]) / 2);
            }
    };
    if (shape == QUAD || shape == HEX) {
        const int nz = shape == HEX ? n : 1;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    X.push_back(g[i]);
                    X.push_back(g[j]);
                    if (shape == HEX) X.push_back(g[k]);
                    W.push_back(w[i] * w[j] * (shape == HEX ? w[k] : 1.0));
                }
    } else if (shape == TRI) {
        tri(X, W);
    } else if (shape == PRI) {
        std::vector<double> Xt, Wt;
        tri(Xt, Wt);
        for (int k = 0; k < n; ++k)
            for (size_t m = 0; m < Wt.size(); ++m) {
                X.insert(X.end(), {Xt[2 * m], Xt[2 * m + 1], g[k]});
                W.push_back(Wt[m] * w[k]);
            }
    } else {
        // Tetrahedron x_i >= -1, x + y + z <= -1: z = c, y = (1 + b)(1 - c)/2 - 1,
        // x = (1 + a)(-y - c)/2 - 1, factor (1 - c)/2 (-y - c)/2.
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    const double z = g[k];
                    const double y = (1 + g[j]) * (1 - z) / 2 - 1;
                    const double x = (1 + g[i]) * (-y - z) / 2 - 1;
                    X.insert(X.end(), {x, y, z});
                    W.push_back(w[i] * w[j] * w[k] * (1 - z) / 2 * (-y - z) / 2);
                }
    }
}

RefElement build_ref_element(int shape, int p) {
    if (shape < 0 || shape > 4) throw std::runtime_error("unknown element shape");
    if (p < 1 || p > 8) throw std::runtime_error("degree out of range");
    RefElement R;
    R.shape = shape;
    R.p = p;
    const int nd = shape_ndim(shape);
    R.nd = nd;
    R.nfaces = shape_nfaces(shape);
    const double* V = kVerts[shape].data();
    std::vector<double> g = gauss_legendre(p + 1);
    std::vector<double> gi = gauss_legendre(p);

    // Solution points.
    auto tri_set = [&](int q, std::vector<double>& X) {
        int vid[3] = {0, 1, 2};
        for (auto& lam : warped_lattice(2, q)) push_bary(X, lam, kVerts[TRI].data(), vid, 3, 2);
    };
    if (shape == TRI) {
        tri_set(p, R.xs);
    } else if (shape == TET) {
        int vid[4] = {0, 1, 2, 3};
        for (auto& lam : warped_lattice(3, p)) push_bary(R.xs, lam, V, vid, 4, 3);
    } else if (shape == QUAD) {
        for (int j = 0; j <= p; ++j)
            for (int i = 0; i <= p; ++i) R.xs.insert(R.xs.end(), {g[i], g[j]});
    } else if (shape == HEX) {
        for (int k = 0; k <= p; ++k)
            for (int j = 0; j <= p; ++j)
                for (int i = 0; i <= p; ++i) R.xs.insert(R.xs.end(), {g[i], g[j], g[k]});
    } else {
        std::vector<double> t;
        tri_set(p, t);
        for (int k = 0; k <= p; ++k)
            for (size_t m = 0; m < t.size() / 2; ++m) R.xs.insert(R.xs.end(), {t[2 * m], t[2 * m + 1], g[k]});
    }
    R.nsol = (int)R.xs.size() / nd;

    // External flux points, face by face.
    for (int f = 0; f < R.nfaces; ++f) {
        const auto& fv = kFaces[shape][f];
        std::vector<double> n = kFaceNrm[shape][f];
        double nn = 0;
        for (double c : n) nn += c * c;
        nn = std::sqrt(nn);
        for (double& c : n) c /= nn;
        R.face_nrm.insert(R.face_nrm.end(), n.begin(), n.end());
        size_t before = R.xfe.size();
        if (nd == 2) {
            const double* A = V + fv[0] * 2;
            const double* B = V + fv[1] * 2;
            for (int i = 0; i <= p; ++i) {
                double s = 0.5 * (1 + g[i]);
                R.xfe.insert(R.xfe.end(), {A[0] + (B[0] - A[0]) * s, A[1] + (B[1] - A[1]) * s});
            }
        } else if (fv.size() == 3) {
            int vid[3] = {fv[0], fv[1], fv[2]};
            for (auto& lam : warped_lattice(2, p)) push_bary(R.xfe, lam, V, vid, 3, 3);
        } else if (shape == HEX) {
            int fixed = 0;
            for (int d = 0; d < 3; ++d)
                if (n[d] != 0) fixed = d;
            int f0 = fixed == 0 ? 1 : 0;
            int f1 = fixed == 2 ? 1 : 2;
            for (int j = 0; j <= p; ++j)
                for (int i = 0; i <= p; ++i) {
                    double x[3];
                    x[fixed] = n[fixed] > 0 ? 1.0 : -1.0;
                    x[f0] = g[i];
                    x[f1] = g[j];
                    R.xfe.insert(R.xfe.end(), {x[0], x[1], x[2]});
                }
        } else {  // prism quadrilateral face: bottom edge fv[0] -> fv[1] fastest, z outer
            const double* A = V + fv[0] * 3;
            const double* B = V + fv[1] * 3;
            for (int j = 0; j <= p; ++j)
                for (int i = 0; i <= p; ++i) {
                    double s = 0.5 * (1 + g[i]);
                    R.xfe.insert(R.xfe.end(), {A[0] + (B[0] - A[0]) * s, A[1] + (B[1] - A[1]) * s, g[j]});
                }
        }
        size_t cnt = (R.xfe.size() - before) / nd;
        for (size_t i = 0; i < cnt; ++i) {
            R.fe_face.push_back(f);
            R.nfe_ref.insert(R.nfe_ref.end(), n.begin(), n.end());
        }
    }
    R.nfe = (int)R.fe_face.size();

    // Internal flux points and DOFs.
    if (shape == TRI || shape == TET) {
        if (shape == TRI) tri_set(p - 1, R.xfiu);
        else {
            int vid[4] = {0, 1, 2, 3};
            for (auto& lam : warped_lattice(3, p - 1)) push_bary(R.xfiu, lam, V, vid, 4, 3);
        }
        int nu = (int)R.xfiu.size() / nd;
        for (int d = 0; d < nd; ++d)
            for (int k = 0; k < nu; ++k) {
                R.fi_point.push_back(k);
                R.fi_axis.push_back(d);
            }
    } else if (shape == QUAD || shape == HEX) {
        for (int d = 0; d < nd; ++d) {
            int n0 = d == 0 ? p : p + 1, n1 = d == 1 ? p : p + 1, n2 = nd == 3 ? (d == 2 ? p : p + 1) : 1;
            for (int k = 0; k < n2; ++k)
                for (int j = 0; j < n1; ++j)
                    for (int i = 0; i < n0; ++i) {
                        int idx = (int)R.xfiu.size() / nd;
                        R.xfiu.push_back(d == 0 ? gi[i] : g[i]);
                        R.xfiu.push_back(d == 1 ? gi[j] : g[j]);
                        if (nd == 3) R.xfiu.push_back(d == 2 ? gi[k] : g[k]);
                        R.fi_point.push_back(idx);
                        R.fi_axis.push_back(d);
                    }
        }
    } else {  // prism
        std::vector<double> t1, t2;
        tri_set(p - 1, t1);
        tri_set(p, t2);
        for (int k = 0; k <= p; ++k)
            for (size_t m = 0; m < t1.size() / 2; ++m) R.xfiu.insert(R.xfiu.end(), {t1[2 * m], t1[2 * m + 1], g[k]});
        int n1 = (int)R.xfiu.size() / 3;
        for (int k = 0; k < p; ++k)
            for (size_t m = 0; m < t2.size() / 2; ++m) R.xfiu.insert(R.xfiu.end(), {t2[2 * m], t2[2 * m + 1], gi[k]});
        int n2 = (int)R.xfiu.size() / 3 - n1;
        for (int d = 0; d < 2; ++d)
            for (int k = 0; k < n1; ++k) {
                R.fi_point.push_back(k);
                R.fi_axis.push_back(d);
            }
        for (int k = 0; k < n2; ++k) {
            R.fi_point.push_back(n1 + k);
            R.fi_axis.push_back(2);
        }
    }
    R.nfiu = (int)R.xfiu.size() / nd;
    R.nfi = (int)R.fi_point.size();

    // Solution nodal basis: L(X) = Psi(X) Vs^{-1}.
    const int maxn = p + 3;
    auto smulti = sol_multi(shape, p);
    if ((int)smulti.size() != R.nsol) throw std::runtime_error("solution space / point count mismatch");
    LegTab T;
    std::vector<double> Vs(R.nsol * R.nsol);
    for (int r = 0; r < R.nsol; ++r) {
        T.set(&R.xs[r * nd], nd, maxn);
        for (int m = 0; m < R.nsol; ++m) Vs[r * R.nsol + m] = T.L(smulti[m].data(), nd);
    }
    std::vector<double> Vs_inv = invert(Vs, R.nsol);
    auto interp = [&](const std::vector<double>& X, int npts, std::vector<double>& out) {
        out.assign((size_t)npts * R.nsol, 0.0);
        std::vector<double> psi(R.nsol);
        for (int i = 0; i < npts; ++i) {
            T.set(&X[i * nd], nd, maxn);
            for (int m = 0; m < R.nsol; ++m) psi[m] = T.L(smulti[m].data(), nd);
            for (int r = 0; r < R.nsol; ++r) {
                double s = 0;
                for (int m = 0; m < R.nsol; ++m) s += psi[m] * Vs_inv[m * R.nsol + r];
                out[(size_t)i * R.nsol + r] = s;
            }
        }
    };
    interp(R.xfe, R.nfe, R.M0);
    interp(R.xfiu, R.nfiu, R.M12);
    element_quadrature(shape, 7, R.xq, R.wq);
    interp(R.xq, (int)R.wq.size(), R.Mq);

    // Flux nodal basis: Vf[sigma][m] = psi^f_m(x_sigma) . n_sigma, flux DOFs = ext then internal.
    auto modes = rt_modes(shape, p);
    const int nf = R.nfe + R.nfi;
    if ((int)modes.size() != nf) throw std::runtime_error("RT space / flux DOF count mismatch");
    auto mode_val = [&](const Mode& md, const double* x, const double* dir) {
        double Lv = T.L(md.a, nd);
        if (md.kind == 0) return Lv * dir[md.comp];
        double s = 0;
        for (int d = 0; d < md.comp; ++d) s += x[d] * dir[d];
        return s * Lv;
    };
    auto mode_div = [&](const Mode& md, const double* x) {
        if (md.kind == 0) return T.dL(md.a, nd, md.comp);
        double s = md.comp * T.L(md.a, nd);
        for (int d = 0; d < md.comp; ++d) s += x[d] * T.dL(md.a, nd, d);
        return s;
    };
    std::vector<double> Vf((size_t)nf * nf);
    for (int s = 0; s < nf; ++s) {
        double x[3] = {0, 0, 0}, dir[3] = {0, 0, 0};
        if (s < R.nfe) {
            for (int d = 0; d < nd; ++d) {
                x[d] = R.xfe[s * nd + d];
                dir[d] = R.nfe_ref[s * nd + d];
            }
        } else {
            int nu = s - R.nfe;
            for (int d = 0; d < nd; ++d) x[d] = R.xfiu[R.fi_point[nu] * nd + d];
            dir[R.fi_axis[nu]] = 1.0;
        }
        T.set(x, nd, maxn);
        for (int m = 0; m < nf; ++m) Vf[(size_t)s * nf + m] = mode_val(modes[m], x, dir);
    }
    std::vector<double> Cf = invert(Vf, nf);   // l^f_nu = sum_m Cf[m][nu] psi^f_m
    for (double c : Cf) R.cond_hint = std::max(R.cond_hint, std::fabs(c));
    std::vector<double> D((size_t)R.nsol * nf, 0.0);
    std::vector<double> dv(nf);
    for (int r = 0; r < R.nsol; ++r) {
        T.set(&R.xs[r * nd], nd, maxn);
        for (int m = 0; m < nf; ++m) dv[m] = mode_div(modes[m], &R.xs[r * nd]);
        for (int nu = 0; nu < nf; ++nu) {
            double s = 0;
            for (int m = 0; m < nf; ++m) s += dv[m] * Cf[(size_t)m * nf + nu];
            D[(size_t)r * nf + nu] = s;
        }
    }
    R.M14.resize((size_t)R.nsol * R.nfe);
    R.M13.resize((size_t)R.nsol * R.nfi);
    for (int r = 0; r < R.nsol; ++r) {
        for (int j = 0; j < R.nfe; ++j) R.M14[(size_t)r * R.nfe + j] = D[(size_t)r * nf + j];
        for (int j = 0; j < R.nfi; ++j) R.M13[(size_t)r * R.nfi + j] = D[(size_t)r * nf + R.nfe + j];
    }
    R.M16.assign((size_t)nd * R.nsol * R.nfe, 0.0);
    R.M15.assign((size_t)nd * R.nsol * R.nfi, 0.0);
    for (int d = 0; d < nd; ++d)
        for (int r = 0; r < R.nsol; ++r) {
            for (int j = 0; j < R.nfe; ++j)
                R.M16[((size_t)d * R.nsol + r) * R.nfe + j] = R.nfe_ref[j * nd + d] * R.M14[(size_t)r * R.nfe + j];
            for (int j = 0; j < R.nfi; ++j)
                R.M15[((size_t)d * R.nsol + r) * R.nfi + j] =
                    (R.fi_axis[j] == d ? 1.0 : 0.0) * R.M13[(size_t)r * R.nfi + j];
        }
    return R;
}

}  // namespace sdrt
