// Build-time generator of the operator-specialised SDRT kernels.
//
// For every (element shape, degree) listed below it builds the reference
// element with the library's own FP64 operator code (refel.cpp: point sets of
// paper App. A, operators M0, M12, M13, M14 of App. B) and writes one CUDA
// translation unit that instantiates the fused stage kernel of gen_stage.cuh
// with those operators baked in as FP32 immediates:
//   * interpolation rows [M0; M12] and divergence columns [M14 | M13] keep only
//     their structural non-zeros (entries below 1e-11 of the matrix's largest
//     are the rounding of exact zeros: on tensor-product elements each flux
//     point depends on one line of solution points; the entries are dropped
//     only when the gap to the smallest kept entry exceeds 1e6, otherwise
//     only exact zeros are; both sizes are printed in each file);
//   * the flux points are split into groups (external points face by face,
//     then the unique internal points) whose point states and DOF fluxes fit a
//     shared-memory budget; the kernel interpolates, evaluates the fluxes and
//     accumulates the divergence group by group.
// Also writes gen_table.cpp, which maps (shape, degree) to the launchers.
//
// Usage: opgen <output directory>
#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <fstream>
#include <sstream>
#include <stdexcept>
#include <string>
#include <vector>

#include "refel.hpp"

using namespace sdrt;

namespace {

struct Key {
    int shape, p;
    const char* name;
};

// The specialised element types: the shapes and degrees of the batched
// mixed-element workloads (hexahedra and prisms up to degree 3 / 4,
// tetrahedra up to 4).  Degree-4 hexahedra (125 solution points) stay on the
// generic kernels: their register and shared-memory footprint does not fit
// this scheme.
const Key kKeys[] = {{HEX, 1, "hex1"}, {HEX, 2, "hex2"}, {HEX, 3, "hex3"}, {PRI, 1, "pri1"}, {PRI, 2, "pri2"},
                     {PRI, 3, "pri3"}, {PRI, 4, "pri4"}, {TET, 1, "tet1"}, {TET, 2, "tet2"}, {TET, 3, "tet3"},
                     {TET, 4, "tet4"}};

// Row units (point states + DOF fluxes) of one group.
constexpr int kBudget = 64;
constexpr double kZeroRel = 1e-11;

std::string flt(double x) {
    char b[64];
    std::snprintf(b, sizeof b, "%.9ef", (double)(float)x);
    return b;
}

struct Sparse {
    // entries (row, col, value) of a dense row-major matrix above the threshold
    std::vector<std::vector<std::pair<int, double>>> rows;
    double dropped_max = 0, kept_min = 1e300;
};

Sparse sparsify_at(const std::vector<double>& A, int nr, int nc, double thr) {
    double mx = 0;
    for (double a : A) mx = std::max(mx, std::fabs(a));
    Sparse S;
    S.rows.resize(nr);
    for (int r = 0; r < nr; ++r)
        for (int c = 0; c < nc; ++c) {
            const double a = A[(size_t)r * nc + c];
            const double rel = std::fabs(a) / mx;
            if (rel > thr) {
                S.rows[r].push_back({c, a});
                S.kept_min = std::min(S.kept_min, rel);
            } else {
                S.dropped_max = std::max(S.dropped_max, rel);
            }
        }
    return S;
}

// Structural zeros dropped when they are separated from the kept entries by
// more than six orders of magnitude; otherwise (the simplices' dense
// operators, whose small entries are genuine) only exact zeros are dropped.
Sparse sparsify(const std::vector<double>& A, int nr, int nc) {
    Sparse S = sparsify_at(A, nr, nc, kZeroRel);
    if (S.dropped_max > 0 && S.kept_min / S.dropped_max < 1e6) S = sparsify_at(A, nr, nc, 0.0);
    return S;
}

struct Point {
    bool ext;
    int id;                    // external point sigma or unique internal point k
    int face;                  // external: its face
    std::vector<int> dofs;     // internal: DOF indices nu
    std::vector<int> axes;     // internal: their reference axes
};

void generate(const Key& key, const std::string& dir, std::ostringstream& table) {
    const RefElement R = build_ref_element(key.shape, key.p);
    const int NS = R.nsol, NFE = R.nfe, NFIU = R.nfiu, NFI = R.nfi;
    // [M0; M12] (NFE + NFIU) x NS and [M14 | M13] NS x (NFE + NFI).
    std::vector<double> Ai((size_t)(NFE + NFIU) * NS), Ad((size_t)NS * (NFE + NFI));
    for (int r = 0; r < NFE; ++r)
        for (int c = 0; c < NS; ++c) Ai[(size_t)r * NS + c] = R.M0[(size_t)r * NS + c];
    for (int r = 0; r < NFIU; ++r)
        for (int c = 0; c < NS; ++c) Ai[(size_t)(NFE + r) * NS + c] = R.M12[(size_t)r * NS + c];
    for (int r = 0; r < NS; ++r) {
        for (int c = 0; c < NFE; ++c) Ad[(size_t)r * (NFE + NFI) + c] = R.M14[(size_t)r * NFE + c];
        for (int c = 0; c < NFI; ++c) Ad[(size_t)r * (NFE + NFI) + NFE + c] = R.M13[(size_t)r * NFI + c];
    }
    const Sparse SI = sparsify(Ai, NFE + NFIU, NS);
    // columns of the divergence: transpose of the sparse rows
    const Sparse SDr = sparsify(Ad, NS, NFE + NFI);
    std::vector<std::vector<std::pair<int, double>>> dcol(NFE + NFI);
    for (int r = 0; r < NS; ++r)
        for (auto& e : SDr.rows[r]) dcol[e.first].push_back({r, e.second});

    // Points and groups.
    std::vector<Point> pts;
    for (int s = 0; s < NFE; ++s) pts.push_back({true, s, R.fe_face[s], {}, {}});
    for (int k = 0; k < NFIU; ++k) {
        Point P{false, k, -1, {}, {}};
        for (int nu = 0; nu < NFI; ++nu)
            if (R.fi_point[nu] == k) {
                P.dofs.push_back(nu);
                P.axes.push_back(R.fi_axis[nu]);
            }
        if (P.dofs.empty() || P.dofs.size() > 3) throw std::runtime_error("internal point without 1..3 DOFs");
        pts.push_back(P);
    }
    // Threads per (element, variable) column: large element types split the
    // rows of every operator application over SPLIT threads (more warps per
    // SM at the same shared memory per element).
    const int SPLIT = NS > 20 ? 2 : 1;
    int budget = SPLIT > 1 ? kBudget : (NS <= 10 ? kBudget / 2 : kBudget * 3 / 4);
    if (SPLIT > 1) {
        // Shared memory of the stage kernel (gen_stage.cuh Smem, 5 variables,
        // 32 elements) for group rows <= b; shrink the groups (not below 48
        // rows) where that lets three CTAs share an SM.
        const int CS = (NS + 3) / 4 % 2 ? (NS + 3) / 4 * 4 : (NS + 3) / 4 * 4 + 4;
        auto smem = [&](int b) {
            const int us = 5 * 32 * CS, main = us + b * 160 + (10 + 4 * R.nfaces) * 32 + NFE * 32;
            int crec = std::min(NFE, std::max(1, b - 1)) * 5;
            if (crec % 2 == 0) ++crec;
            return 4 * std::max(main, us + 32 * crec);
        };
        const int three = 228 * 1024 / 3 - 1024;
        if (smem(kBudget) > three)
            for (int b = kBudget - 1; b >= 48; --b)
                if (smem(b) <= three) {
                    budget = b;
                    break;
                }
    }
    std::vector<std::vector<int>> groups(1);
    int units = 0;
    for (int i = 0; i < (int)pts.size(); ++i) {
        const int u = 1 + (pts[i].ext ? 1 : (int)pts[i].dofs.size());
        if (units + u > budget && !groups.back().empty()) {
            groups.emplace_back();
            units = 0;
        }
        groups.back().push_back(i);
        units += u;
    }
    int GR = 0;                    // largest group: point rows + DOF rows
    for (auto& g : groups) {
        int nf = 0;
        for (int i : g) nf += pts[i].ext ? 1 : (int)pts[i].dofs.size();
        GR = std::max(GR, (int)g.size() + nf);
    }
    long nnzI = 0, nnzD = 0;
    for (auto& r : SI.rows) nnzI += (long)r.size();
    for (auto& c : dcol) nnzD += (long)c.size();
    const int NSH = (NS + SPLIT - 1) / SPLIT;      // divergence rows per part

    // x[j * ldx] = sum_c A[row_j][c] u[c] for the rows (row_j, j) listed; u is
    // the thread's solution column, contiguous and 16-byte aligned in shared
    // memory, read as float4 blocks of the columns used
    auto emit_rows = [&](std::ostringstream& o, const std::vector<std::pair<int, int>>& rows) {
        std::vector<int> used(NS, 0);
        for (auto& rj : rows)
            for (auto& e : SI.rows[rj.first]) used[e.first] = 1;
        for (int b = 0; 4 * b < NS; ++b) {
            bool any = false;
            for (int c = 4 * b; c < std::min(NS, 4 * b + 4); ++c) any = any || used[c];
            if (!any) continue;
            o << "        const float4 b" << b << " = reinterpret_cast<const float4*>(u)[" << b << "];\n";
            const char* comp[4] = {"x", "y", "z", "w"};
            for (int c = 4 * b; c < std::min(NS, 4 * b + 4); ++c)
                if (used[c]) o << "        const float u" << c << " = b" << b << "." << comp[c - 4 * b] << ";\n";
        }
        for (auto& rj : rows) {
            auto& rr = SI.rows[rj.first];
            std::string e = "0.0f";
            for (size_t q = 0; q < rr.size(); ++q) {
                const std::string term = "u" + std::to_string(rr[q].first);
                e = q == 0 ? flt(rr[q].second) + " * " + term
                           : "fmaf(" + flt(rr[q].second) + ", " + term + ", " + e + ")";
            }
            o << "        x[" << rj.second << " * ldx] = " << e << ";\n";
        }
    };

    std::ostringstream o;
    const std::string N = key.name;
    std::string T = N;
    T[0] = (char)std::toupper(T[0]);
    o << "// Generated by csrc/gen/opgen.cpp from the library's FP64 operators: do not edit.\n"
      << "// " << N << ": nsol " << NS << ", nfe " << NFE << ", nfiu " << NFIU << ", nfi " << NFI << "; non-zeros "
      << "[M0; M12] " << nnzI << " of " << (long)(NFE + NFIU) * NS << ", [M14 | M13] " << nnzD << " of "
      << (long)NS * (NFE + NFI) << "\n"
      << "// relative size of the largest dropped / smallest kept entry: interpolation " << SI.dropped_max << " / "
      << SI.kept_min << ", divergence " << SDr.dropped_max << " / " << SDr.kept_min << "\n"
      << "#include \"gen_stage.cuh\"\n\nnamespace sdrt {\nnamespace gen {\nnamespace {\n\n";
    // point descriptors: (ext sigma | -(k+1), face, first FS row, ndof | axes << 2)
    o << "__constant__ int4 c_desc[" << pts.size() << "] = {";
    std::vector<int> goff;
    int off = 0;
    for (auto& g : groups) {
        goff.push_back(off);
        int fs = 0;
        for (int i : g) {
            const Point& P = pts[i];
            if (P.ext) {
                o << "{" << P.id << "," << P.face << "," << fs << ",1},";
                fs += 1;
            } else {
                int w = (int)P.dofs.size();
                for (size_t q = 0; q < P.axes.size(); ++q) w |= P.axes[q] << (2 + 2 * q);
                o << "{" << -(P.id + 1) << ",-1," << fs << "," << w << "},";
                fs += (int)P.dofs.size();
            }
            ++off;
        }
    }
    o << "};\n\n";
    o << "struct " << T << " {\n"
      << "    static constexpr int NS = " << NS << ", NFE = " << NFE << ", NFIU = " << NFIU << ", NFI = " << NFI
      << ", NF = " << R.nfaces << ", NG = " << groups.size() << ", GR = " << GR << ", SPLIT = " << SPLIT
      << ", NSH = " << NSH << ";\n"
      << "    template <int G> struct Grp;\n"
      << "    static __device__ __forceinline__ int4 desc(int i) { return c_desc[i]; }\n";
    // ext: external-point rows of chunk c (ECH rows), part h, from the state
    // in shared memory; x indexed from the chunk's first row
    const int ECH = std::min(NFE, std::max(1, GR - 1)), NECH = (NFE + ECH - 1) / ECH;
    o << "    static constexpr int ECH = " << ECH << ", NECH = " << NECH << ";\n";
    o << "    static __device__ __forceinline__ void ext(int c, int h, const float* __restrict__ u, "
         "float* __restrict__ x, const int ldx) {\n";
    bool first = true;
    for (int c = 0; c < NECH; ++c) {
        const int c0 = c * ECH, c1 = std::min(NFE, c0 + ECH);
        for (int h = 0; h < SPLIT; ++h) {
            const int r0 = c0 + h * (c1 - c0) / SPLIT, r1 = c0 + (h + 1) * (c1 - c0) / SPLIT;
            std::vector<std::pair<int, int>> rows;
            for (int r = r0; r < r1; ++r) rows.push_back({r, r - c0});
            o << "      " << (first ? "" : "} else ") << "if (c == " << c << " && h == " << h << ") {\n";
            first = false;
            emit_rows(o, rows);
        }
    }
    o << "      }\n    }\n};\n\n";
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        auto& g = groups[gi];
        int nf = 0;
        for (int i : g) nf += pts[i].ext ? 1 : (int)pts[i].dofs.size();
        o << "template <> struct " << T << "::Grp<" << gi << "> {\n"
          << "    static constexpr int NP = " << g.size() << ", NDOF = " << nf << ", OFF = " << goff[gi] << ";\n"
          << "    static __device__ __forceinline__ void interp(int h, const float* __restrict__ u, "
             "float* __restrict__ x, const int ldx) {\n";
        const int np = (int)g.size();
        for (int h = 0; h < SPLIT; ++h) {
            std::vector<std::pair<int, int>> rows;
            for (int j = h * np / SPLIT; j < (h + 1) * np / SPLIT; ++j) {
                const Point& P = pts[g[j]];
                rows.push_back({P.ext ? P.id : NFE + P.id, j});
            }
            o << "      " << (h ? "} else " : "") << (h + 1 < SPLIT ? "if (h == " + std::to_string(h) + ") " : "")
              << "{\n";
            emit_rows(o, rows);
        }
        o << "      }\n    }\n"
          << "    static __device__ __forceinline__ void div(int h, const float* __restrict__ f, const int ldf, "
             "float (&r)[" << NSH << "]) {\n";
        for (int h = 0; h < SPLIT; ++h) {
            const int q0 = h * NSH, q1 = std::min(NS, (h + 1) * NSH);
            o << "      " << (h ? "} else " : "") << (h + 1 < SPLIT ? "if (h == " + std::to_string(h) + ") " : "")
              << "{\n";
            int fs = 0;
            for (int i : g) {
                const Point& P = pts[i];
                std::vector<int> cols;
                if (P.ext) cols.push_back(P.id);
                else
                    for (int nu : P.dofs) cols.push_back(NFE + nu);
                for (int col : cols) {
                    bool any = false;
                    for (auto& e : dcol[col]) any = any || (e.first >= q0 && e.first < q1);
                    if (any) {
                        o << "        { const float t = f[" << fs << " * ldf];";
                        for (auto& e : dcol[col])
                            if (e.first >= q0 && e.first < q1)
                                o << " r[" << e.first - q0 << "] = fmaf(" << flt(e.second) << ", t, r[" << e.first - q0
                                  << "]);";
                        o << " }\n";
                    }
                    ++fs;
                }
            }
        }
        o << "      }\n    }\n};\n\n";
    }
    o << "}  // namespace\n}  // namespace gen\n\n"
      << "int launch_gen_" << N << "(int kind, const GenArgs& a, int V, int sys, int rie, int nsm, cudaStream_t st) {\n"
      << "    return gen::launch_gen<gen::" << T << ">(kind, a, V, sys, rie, nsm, st);\n}\n\n"
      << "}  // namespace sdrt\n";
    std::ofstream f(dir + "/gen_" + N + ".cu");
    f << o.str();
    if (!f) throw std::runtime_error("cannot write " + dir + "/gen_" + N + ".cu");
    table << "    if (shape == " << key.shape << " && p == " << key.p << ") return launch_gen_" << N << ";\n";
}

}  // namespace

int main(int argc, char** argv) {
    if (argc != 2) {
        std::fprintf(stderr, "usage: opgen <output directory>\n");
        return 2;
    }
    const std::string dir = argv[1];
    try {
        std::ostringstream table, decl;
        for (const Key& k : kKeys) {
            generate(k, dir, table);
            decl << "int launch_gen_" << k.name
                 << "(int kind, const GenArgs& a, int V, int sys, int rie, int nsm, cudaStream_t st);\n";
        }
        std::ofstream f(dir + "/gen_table.cpp");
        f << "// Generated by csrc/gen/opgen.cpp: do not edit.\n#include \"gen_api.hpp\"\n\nnamespace sdrt {\n\n"
          << decl.str() << "\nGenLauncher gen_launcher(int shape, int p) {\n"
          << table.str() << "    return nullptr;\n}\n\n}  // namespace sdrt\n";
        if (!f) throw std::runtime_error("cannot write gen_table.cpp");
    } catch (const std::exception& e) {
        std::fprintf(stderr, "opgen: %s\n", e.what());
        return 1;
    }
    return 0;
}
