// Host-side plan construction for the GB300 finite-element library.
//
//  * Quadrature (Sec. 3.1 assumes exact rules): collapsed product of
//    Gauss-Jacobi rules; the 1-D nodes are found by Newton's method with
//    deflation on the three-term recurrence of the Jacobi polynomials and the
//    weights from the classical Christoffel formula.
//  * Reference basis (Appendix A): equispaced Lagrange nodes, product form
//    phi_a = prod_i prod_{j<a_i} (p lambda_i - j)/(j+1), evaluated together
//    with its gradient by forward-mode dual arithmetic (value, gradient).
//  * Dof map: canonical numbering by mesh entity (vertices, edges, faces,
//    cell interiors), each entity ranked by its sorted vertex ids and each
//    node inside an entity by its multiplicities.
//  * CSR pattern, the (row, cell)-sorted incidence stream and the column
//    slots used by the segmented assembly (Sec. 3.3).
//  * Contraction operands: the tabulated products of Algorithm 1 arranged as
//    the shared B operand of one GEMM per tile of cells, rounded once to the
//    storage format (List 1, u_s) and laid out as 128-byte-swizzled K-major
//    tiles for the tensor cores.
#include "fe_host.h"
#include "fe_internal.h"

#include <algorithm>
#include <climits>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <thread>

#include "../../include/fe_gb300.h"

namespace fe {
namespace host {

unsigned hardware_threads() {
    unsigned n = std::thread::hardware_concurrency();
    return n == 0 ? 1u : std::min(n, 64u);
}

template <class F>
static void parallel_for(int64_t n, F &&f) {
    unsigned nt = hardware_threads();
    if (n < 4096 || nt == 1) {
        f(0, n);
        return;
    }
    std::vector<std::thread> th;
    int64_t chunk = (n + nt - 1) / nt;
    for (unsigned t = 0; t < nt; ++t) {
        int64_t b = t * chunk, e = std::min(n, b + chunk);
        if (b >= e) break;
        th.emplace_back([&f, b, e] { f(b, e); });
    }
    for (auto &x : th) x.join();
}

// --------------------------------------------------------------------------
// Quadrature
// --------------------------------------------------------------------------
// P_n^{(alpha,0)}(x) and its derivative by the three-term recurrence.
static void jacobi_eval(int n, double a, double x, double &p, double &dp) {
    const double b = 0.0;
    double p0 = 1.0, p1 = 0.5 * ((a - b) + (a + b + 2.0) * x);
    if (n == 0) { p = 1.0; dp = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double s = 2.0 * k + a + b;
        double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
        double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
        double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
        double p2 = (c2 * p1 - c3 * p0) / c1;
        p0 = p1;
        p1 = p2;
    }
    p = p1;
    // (2n+a+b)(1-x^2) P_n' = n[(a-b) - (2n+a+b) x] P_n + 2(n+a)(n+b) P_{n-1}
    double s = 2.0 * n + a + b;
    dp = (n * ((a - b) - s * x) * p1 + 2.0 * (n + a) * (n + b) * p0) / (s * (1.0 - x * x));
}

bool gauss_jacobi(int m, int alpha, std::vector<double> &t, std::vector<double> &w) {
    if (m < 1 || m > 64 || alpha < 0 || alpha > 2) return false;
    const double a = alpha;
    std::vector<double> x(m);
    for (int i = 0; i < m; ++i) {
        // Chebyshev-like start, refined by deflated Newton.
        double z = -std::cos(M_PI * (i + 0.75) / (m + 0.5));
        if (i > 0 && z <= x[i - 1]) z = x[i - 1] + 1e-3 * (1.0 - x[i - 1]);
        for (int it = 0; it < 200; ++it) {
            double p, dp;
            jacobi_eval(m, a, z, p, dp);
            double defl = 0.0;
            for (int j = 0; j < i; ++j) defl += 1.0 / (z - x[j]);
            double delta = p / (dp - p * defl);
            z -= delta;
            if (std::fabs(delta) <= 1e-17 * std::max(1.0, std::fabs(z))) break;
        }
        x[i] = z;
    }
    std::sort(x.begin(), x.end());
    t.resize(m);
    w.resize(m);
    for (int i = 0; i < m; ++i) {
        double p, dp;
        jacobi_eval(m, a, x[i], p, dp);
        // w = 2^{a+1} / ((1 - x^2) P_m'(x)^2) for beta = 0; mapped to [0,1] by / 2^{a+1}
        double wx = std::ldexp(1.0, alpha + 1) / ((1.0 - x[i] * x[i]) * dp * dp);
        t[i] = 0.5 * (1.0 + x[i]);
        w[i] = wx / std::ldexp(1.0, alpha + 1);
    }
    return true;
}

bool collapsed_rule(int d, int m, std::vector<double> &pts, std::vector<double> &wts) {
    std::vector<double> ta, wa, tb, wb, tc, wc;
    if (!gauss_jacobi(m, 0, ta, wa) || !gauss_jacobi(m, 1, tb, wb)) return false;
    pts.clear();
    wts.clear();
    if (d == 2) {
        for (int ib = 0; ib < m; ++ib)
            for (int ia = 0; ia < m; ++ia) {
                pts.push_back(ta[ia] * (1.0 - tb[ib]));
                pts.push_back(tb[ib]);
                wts.push_back(wa[ia] * wb[ib]);
            }
        return true;
    }
    if (!gauss_jacobi(m, 2, tc, wc)) return false;
    for (int ic = 0; ic < m; ++ic)
        for (int ib = 0; ib < m; ++ib)
            for (int ia = 0; ia < m; ++ia) {
                pts.push_back(ta[ia] * (1.0 - tb[ib]) * (1.0 - tc[ic]));
                pts.push_back(tb[ib] * (1.0 - tc[ic]));
                pts.push_back(tc[ic]);
                wts.push_back(wa[ia] * wb[ib] * wc[ic]);
            }
    return true;
}

bool tensor_rule(int d, int m, std::vector<double> &pts, std::vector<double> &wts) {
    std::vector<double> t, w;
    if (!gauss_jacobi(m, 0, t, w)) return false;
    int n = 1;
    for (int i = 0; i < d; ++i) n *= m;
    pts.assign((size_t)n * d, 0.0);
    wts.assign(n, 0.0);
    for (int q = 0; q < n; ++q) {
        int r = q;
        double wq = 1.0;
        for (int i = 0; i < d; ++i) {   // x index fastest
            const int ii = r % m;
            r /= m;
            pts[(size_t)q * d + i] = t[ii];
            wq *= w[ii];
        }
        wts[q] = wq;
    }
    return true;
}

// --------------------------------------------------------------------------
// Reference basis
// --------------------------------------------------------------------------
int n_phi_box(int d, int p) {
    int n = 1;
    for (int i = 0; i < d; ++i) n *= (p + 1);
    return n;
}

int n_phi(int d, int p) {
    int64_t n = 1;
    for (int i = 1; i <= d; ++i) n = n * (p + i) / i;
    return (int)n;
}

std::vector<int> lattice_nodes(int d, int p) {
    std::vector<std::vector<int>> all;
    std::vector<int> a(d + 1, 0);
    // enumerate all multi-indices with |a| = p
    std::function<void(int, int)> rec = [&](int i, int left) {
        if (i == d) {
            a[d] = left;
            all.push_back(a);
            return;
        }
        for (int v = 0; v <= left; ++v) {
            a[i] = v;
            rec(i + 1, left - v);
        }
    };
    rec(0, p);
    auto key_less = [d](const std::vector<int> &x, const std::vector<int> &y) {
        std::vector<int> sx, sy;
        for (int i = 0; i <= d; ++i) {
            if (x[i] > 0) sx.push_back(i);
            if (y[i] > 0) sy.push_back(i);
        }
        if (sx.size() != sy.size()) return sx.size() < sy.size();
        if (sx != sy) return sx < sy;
        return x > y;  // descending lexicographic
    };
    std::sort(all.begin(), all.end(), key_less);
    std::vector<int> out;
    for (auto &v : all) out.insert(out.end(), v.begin(), v.end());
    return out;
}

namespace {
struct Dual {
    double v;
    double g[3];
};
}  // namespace

void tabulate(int d, int p, const double *pts, int n_q, std::vector<double> &phi, std::vector<double> &dphi) {
    const int nph = n_phi(d, p);
    std::vector<int> nodes = lattice_nodes(d, p);
    phi.assign((size_t)nph * n_q, 0.0);
    dphi.assign((size_t)d * nph * n_q, 0.0);
    for (int q = 0; q < n_q; ++q) {
        // barycentric coordinates as duals in the reference coordinates X
        Dual lam[4];
        double s = 0.0;
        for (int i = 0; i < d; ++i) s += pts[q * d + i];
        lam[0].v = 1.0 - s;
        for (int k = 0; k < 3; ++k) lam[0].g[k] = (k < d) ? -1.0 : 0.0;
        for (int i = 1; i <= d; ++i) {
            lam[i].v = pts[q * d + i - 1];
            for (int k = 0; k < 3; ++k) lam[i].g[k] = (k == i - 1) ? 1.0 : 0.0;
        }
        for (int n = 0; n < nph; ++n) {
            Dual acc{1.0, {0.0, 0.0, 0.0}};
            for (int i = 0; i <= d; ++i) {
                int ai = nodes[n * (d + 1) + i];
                for (int j = 0; j < ai; ++j) {
                    double inv = 1.0 / (j + 1);
                    Dual f{(p * lam[i].v - j) * inv, {p * lam[i].g[0] * inv, p * lam[i].g[1] * inv, p * lam[i].g[2] * inv}};
                    Dual r;
                    r.v = acc.v * f.v;
                    for (int k = 0; k < 3; ++k) r.g[k] = acc.v * f.g[k] + f.v * acc.g[k];
                    acc = r;
                }
            }
            phi[(size_t)n * n_q + q] = acc.v;
            for (int k = 0; k < d; ++k) dphi[((size_t)k * nph + n) * n_q + q] = acc.g[k];
        }
    }
}

// Q_p basis of boxed cells: phi_a(X) = prod_i l_{a_i}(X_i), each 1-D factor
// l_j(t) = prod_{m != j} (p t - m)/(j - m) evaluated as a dual number (value
// and derivative), the product over the directions formed with the gradient.
void tabulate_box(int d, int p, const double *pts, int n_q, std::vector<double> &phi, std::vector<double> &dphi) {
    const int nph = n_phi_box(d, p);
    phi.assign((size_t)nph * n_q, 0.0);
    dphi.assign((size_t)d * nph * n_q, 0.0);
    std::vector<double> lv((size_t)d * (p + 1)), ld((size_t)d * (p + 1));
    for (int q = 0; q < n_q; ++q) {
        for (int i = 0; i < d; ++i) {
            const double t = pts[q * d + i];
            for (int j = 0; j <= p; ++j) {
                double v = 1.0, g = 0.0;   // dual number (v, g) of the running product
                for (int m = 0; m <= p; ++m) {
                    if (m == j) continue;
                    const double inv = 1.0 / (double)(j - m);
                    const double fv = (p * t - m) * inv, fg = p * inv;
                    g = g * fv + v * fg;
                    v = v * fv;
                }
                lv[(size_t)i * (p + 1) + j] = v;
                ld[(size_t)i * (p + 1) + j] = g;
            }
        }
        for (int k = 0; k < nph; ++k) {
            int a[3] = {0, 0, 0}, r = k;
            for (int i = 0; i < d; ++i) {
                a[i] = r % (p + 1);
                r /= (p + 1);
            }
            double v = 1.0;
            double g[3] = {1.0, 1.0, 1.0};
            for (int i = 0; i < d; ++i) {
                const double fv = lv[(size_t)i * (p + 1) + a[i]], fd = ld[(size_t)i * (p + 1) + a[i]];
                for (int s2 = 0; s2 < d; ++s2) g[s2] *= (s2 == i) ? fd : fv;
                v *= fv;
            }
            phi[(size_t)k * n_q + q] = v;
            for (int s2 = 0; s2 < d; ++s2) dphi[((size_t)s2 * nph + k) * n_q + q] = g[s2];
        }
    }
}

// --------------------------------------------------------------------------
// Canonical dof map by mesh entities
// --------------------------------------------------------------------------
namespace {
// Lexicographic ranks of compositions of p into s positive parts.
struct CompositionRanks {
    int p, s;
    std::vector<int> rank;  // indexed by base-(p+1) code of the tuple
    int count = 0;
    CompositionRanks(int p_, int s_) : p(p_), s(s_) {
        int sz = 1;
        for (int i = 0; i < s; ++i) sz *= (p + 1);
        rank.assign(sz, -1);
        std::vector<int> t(s);
        std::function<void(int, int)> rec = [&](int i, int left) {
            if (i == s - 1) {
                if (left >= 1) {
                    t[i] = left;
                    rank[code(t.data())] = count++;
                }
                return;
            }
            for (int v = 1; v <= left - (s - 1 - i); ++v) {
                t[i] = v;
                rec(i + 1, left - v);
            }
        };
        if (s >= 1 && p >= s) rec(0, p);
    }
    int code(const int *t) const {
        int c = 0;
        for (int i = 0; i < s; ++i) c = c * (p + 1) + t[i];
        return c;
    }
};
}  // namespace

static std::string build_dofmap(int d, int p, int64_t n_vertices, int64_t n_cells, const int32_t *cells,
                                std::vector<int32_t> &cell_dofs, int64_t &n_dofs) {
    const int nv = d + 1;
    const int nph = n_phi(d, p);
    std::vector<int> nodes = lattice_nodes(d, p);
    cell_dofs.assign((size_t)n_cells * nph, -1);
    // Unique entities of sizes 2..d+1 as sorted vertex tuples.
    std::vector<std::vector<std::array<int32_t, 4>>> ent(5);
    for (int s = 2; s <= nv; ++s) {
        auto &E = ent[s];
        // subsets of size s of the local vertices
        std::vector<std::vector<int>> subsets;
        for (int mask = 0; mask < (1 << nv); ++mask)
            if (__builtin_popcount(mask) == s) {
                std::vector<int> sub;
                for (int i = 0; i < nv; ++i)
                    if (mask & (1 << i)) sub.push_back(i);
                subsets.push_back(sub);
            }
        E.reserve((size_t)n_cells * subsets.size());
        for (int64_t c = 0; c < n_cells; ++c)
            for (auto &sub : subsets) {
                std::array<int32_t, 4> t{-1, -1, -1, -1};
                for (int i = 0; i < s; ++i) t[i] = cells[c * nv + sub[i]];
                std::sort(t.begin(), t.begin() + s);
                E.push_back(t);
            }
        std::sort(E.begin(), E.end());
        E.erase(std::unique(E.begin(), E.end()), E.end());
    }
    std::vector<CompositionRanks> ranks;
    for (int s = 0; s <= 4; ++s) ranks.emplace_back(p, s);
    // offsets of each entity size class
    int64_t off[6];
    off[2] = n_vertices;
    for (int s = 2; s <= nv; ++s) off[s + 1] = off[s] + (int64_t)ent[s].size() * ranks[s].count;
    n_dofs = off[nv + 1];
    if (n_dofs > INT32_MAX) return "too many degrees of freedom for int32 indices";
    for (int64_t c = 0; c < n_cells; ++c) {
        for (int n = 0; n < nph; ++n) {
            const int *a = &nodes[n * nv];
            std::array<std::pair<int32_t, int>, 4> sup;
            int s = 0;
            for (int i = 0; i < nv; ++i)
                if (a[i] > 0) sup[s++] = {cells[c * nv + i], a[i]};
            if (s == 1) {
                cell_dofs[c * nph + n] = sup[0].first;
                continue;
            }
            std::sort(sup.begin(), sup.begin() + s);
            std::array<int32_t, 4> t{-1, -1, -1, -1};
            int mult[4];
            for (int i = 0; i < s; ++i) {
                t[i] = sup[i].first;
                mult[i] = sup[i].second;
            }
            auto &E = ent[s];
            auto it = std::lower_bound(E.begin(), E.end(), t);
            int64_t er = it - E.begin();
            int r = ranks[s].rank[ranks[s].code(mult)];
            cell_dofs[c * nph + n] = (int32_t)(off[s] + er * ranks[s].count + r);
        }
    }
    return "";
}

// Boxed cells.  Node k (lattice a) weighs each cell vertex v with
// w_v = prod_i (bit_i(v) ? a_i : p - a_i) (its Q1 coordinates times p^d); its
// support is the set of vertices with w_v > 0, i.e. the vertex, edge, face or
// cell interior it lies on.  Entities of each support size are ranked by their
// sorted global vertex ids; inside an entity the nodes are ranked by their
// weights listed in that sorted-id order (lexicographic).  dof = vertex id for
// vertex nodes, else offset(size) + entity rank * nodes per entity + node rank,
// the sizes in increasing order: the same numbering as keys sorted by (support
// size, vertex ids, weights), computed entity by entity.
static std::string build_dofmap_box(int d, int p, int64_t n_vertices, int64_t n_cells, const int32_t *cells,
                                    std::vector<int32_t> &cell_dofs, int64_t &n_dofs) {
    const int nv = 1 << d;
    const int nph = n_phi_box(d, p);
    std::vector<std::array<int, 8>> W(nph);
    std::vector<int> supmask(nph, 0);
    for (int k = 0; k < nph; ++k) {
        int a[3] = {0, 0, 0}, r = k;
        for (int i = 0; i < d; ++i) {
            a[i] = r % (p + 1);
            r /= (p + 1);
        }
        for (int v = 0; v < nv; ++v) {
            int w = 1;
            for (int i = 0; i < d; ++i) w *= ((v >> i) & 1) ? a[i] : p - a[i];
            W[k][v] = w;
            if (w > 0) supmask[k] |= 1 << v;
        }
    }
    // the distinct supports (local vertex masks) of size >= 2 and the nodes on each
    std::map<int, std::vector<int>> on_support;
    for (int k = 0; k < nph; ++k)
        if (__builtin_popcount(supmask[k]) >= 2) on_support[supmask[k]].push_back(k);
    // unique global entities per support size, as sorted vertex tuples
    std::map<int, std::vector<std::array<int32_t, 8>>> ent;
    for (auto &kv : on_support) {
        const int mask = kv.first, s = __builtin_popcount(mask);
        auto &E = ent[s];
        for (int64_t c = 0; c < n_cells; ++c) {
            std::array<int32_t, 8> t;
            t.fill(-1);
            int n = 0;
            for (int v = 0; v < nv; ++v)
                if (mask & (1 << v)) t[n++] = cells[c * nv + v];
            std::sort(t.begin(), t.begin() + s);
            E.push_back(t);
        }
    }
    int per_size[9] = {0};
    for (auto &kv : on_support) per_size[__builtin_popcount(kv.first)] = (int)kv.second.size();
    int64_t off[10];
    off[2] = n_vertices;
    for (int s = 2; s <= 8; ++s) {
        auto it = ent.find(s);
        if (it != ent.end()) {
            std::sort(it->second.begin(), it->second.end());
            it->second.erase(std::unique(it->second.begin(), it->second.end()), it->second.end());
        }
        const int64_t cnt = (it == ent.end()) ? 0 : (int64_t)it->second.size() * per_size[s];
        off[s + 1] = off[s] + cnt;
    }
    n_dofs = off[9];
    if (n_dofs > INT32_MAX) return "too many degrees of freedom for int32 indices";
    cell_dofs.assign((size_t)n_cells * nph, -1);
    std::vector<std::pair<std::array<int, 8>, int>> tuples;
    for (int64_t c = 0; c < n_cells; ++c) {
        for (int k = 0; k < nph; ++k)
            if (__builtin_popcount(supmask[k]) == 1)
                cell_dofs[c * nph + k] = cells[c * nv + __builtin_ctz(supmask[k])];
        for (auto &kv : on_support) {
            const int mask = kv.first, s = __builtin_popcount(mask);
            // local vertices of the support in increasing global id
            std::array<std::pair<int32_t, int>, 8> gv;
            int n = 0;
            for (int v = 0; v < nv; ++v)
                if (mask & (1 << v)) gv[n++] = {cells[c * nv + v], v};
            std::sort(gv.begin(), gv.begin() + s);
            std::array<int32_t, 8> t;
            t.fill(-1);
            for (int i = 0; i < s; ++i) t[i] = gv[i].first;
            const auto &E = ent[s];
            const int64_t er = std::lower_bound(E.begin(), E.end(), t) - E.begin();
            tuples.clear();
            for (int k : kv.second) {
                std::array<int, 8> wt;
                wt.fill(0);
                for (int i = 0; i < s; ++i) wt[i] = W[k][gv[i].second];
                tuples.push_back({wt, k});
            }
            std::sort(tuples.begin(), tuples.end());
            for (size_t r = 0; r < tuples.size(); ++r)
                cell_dofs[c * nph + tuples[r].second] = (int32_t)(off[s] + er * per_size[s] + (int64_t)r);
        }
    }
    return "";
}

std::string build_pattern(int d, int p, int64_t n_vertices, int64_t n_cells, const int32_t *cells, Pattern &P,
                          bool with_streams, bool boxed, int64_t slice_cells) {
    if (d != 2 && d != 3) return "cell dimension must be 2 or 3";
    const int nv = boxed ? (1 << d) : d + 1;
    for (int64_t i = 0; i < n_cells * nv; ++i)
        if (cells[i] < 0 || cells[i] >= n_vertices) return "cell vertex index out of range";
    for (int64_t c = 0; c < n_cells; ++c)
        for (int i = 0; i < nv; ++i)
            for (int j = i + 1; j < nv; ++j)
                if (cells[c * nv + i] == cells[c * nv + j]) return "cell with a repeated vertex";
    P.d = d;
    P.p = p;
    P.n_phi = boxed ? n_phi_box(d, p) : n_phi(d, p);
    P.n_vertices = n_vertices;
    P.n_cells = n_cells;
    const int nph = P.n_phi;
    std::string err = boxed ? build_dofmap_box(d, p, n_vertices, n_cells, cells, P.cell_dofs, P.n_dofs)
                            : build_dofmap(d, p, n_vertices, n_cells, cells, P.cell_dofs, P.n_dofs);
    if (!err.empty()) return err;
    const int64_t nd = P.n_dofs;
    // incidence dof -> (c, k) with c ascending (counting sort, stable)
    std::vector<int64_t> iptr(nd + 1, 0);
    for (int64_t i = 0; i < n_cells * nph; ++i) iptr[P.cell_dofs[i] + 1]++;
    for (int64_t i = 0; i < nd; ++i) iptr[i + 1] += iptr[i];
    std::vector<int32_t> ielem((size_t)n_cells * nph);
    {
        std::vector<int64_t> fill(iptr.begin(), iptr.end() - 1);
        for (int64_t c = 0; c < n_cells; ++c)
            for (int k = 0; k < nph; ++k) ielem[fill[P.cell_dofs[c * nph + k]]++] = (int32_t)(c * nph + k);
    }
    if ((int64_t)n_cells * nph > INT32_MAX) return "too many element rows for int32 indices";
    // rows: sorted unique union of the dofs of the incident cells
    std::vector<int64_t> rlen(nd, 0);
    unsigned nt = hardware_threads();
    std::vector<std::vector<int32_t>> parts(nt);
    std::vector<int64_t> part_begin(nt + 1, nd);
    {
        int64_t chunk = (nd + nt - 1) / nt;
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t) {
            int64_t b = std::min<int64_t>(nd, t * chunk), e = std::min<int64_t>(nd, b + chunk);
            part_begin[t] = b;
            th.emplace_back([&, t, b, e] {
                std::vector<int32_t> buf;
                auto &out = parts[t];
                for (int64_t i = b; i < e; ++i) {
                    buf.clear();
                    for (int64_t j = iptr[i]; j < iptr[i + 1]; ++j) {
                        int64_t c = ielem[j] / nph;
                        buf.insert(buf.end(), &P.cell_dofs[c * nph], &P.cell_dofs[c * nph] + nph);
                    }
                    std::sort(buf.begin(), buf.end());
                    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
                    rlen[i] = (int64_t)buf.size();
                    out.insert(out.end(), buf.begin(), buf.end());
                }
            });
        }
        for (auto &x : th) x.join();
    }
    P.row_ptr.assign(nd + 1, 0);
    for (int64_t i = 0; i < nd; ++i) P.row_ptr[i + 1] = P.row_ptr[i] + rlen[i];
    P.nnz = P.row_ptr[nd];
    P.col_idx.resize(P.nnz);
    int64_t maxr = 0;
    for (int64_t i = 0; i < nd; ++i) maxr = std::max(maxr, rlen[i]);
    P.max_row = (int)maxr;
    {
        int64_t pos = 0;
        for (unsigned t = 0; t < nt; ++t) {
            std::copy(parts[t].begin(), parts[t].end(), P.col_idx.begin() + pos);
            pos += (int64_t)parts[t].size();
            std::vector<int32_t>().swap(parts[t]);
        }
    }
    if (!with_streams) return "";
    if (maxr > 65535) return "row longer than 65535 entries: slot stream would overflow";
    P.inc_ptr = iptr;
    P.inc_elem = ielem;
    P.inc_slot.resize((size_t)n_cells * nph * nph);
    parallel_for(nd, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i) {
            const int32_t *cb = P.col_idx.data() + P.row_ptr[i];
            const int32_t *ce = P.col_idx.data() + P.row_ptr[i + 1];
            for (int64_t j = iptr[i]; j < iptr[i + 1]; ++j) {
                int64_t c = ielem[j] / nph;
                for (int l = 0; l < nph; ++l) {
                    const int32_t *it = std::lower_bound(cb, ce, P.cell_dofs[c * nph + l]);
                    P.inc_slot[(size_t)j * nph + l] = (uint16_t)(it - cb);
                }
            }
        }
    });
    // contribution lists of every CSR entry (segments of the sorted element entries)
    {
        int64_t max_inc = 0;
        for (int64_t i = 0; i < nd; ++i) max_inc = std::max(max_inc, iptr[i + 1] - iptr[i]);
        if (max_inc > 256 || nph > 256) return "more than 256 incidences per row or local dofs: code stream would overflow";
        P.contrib_cnt.assign(P.nnz, 0);
        P.contrib_base.assign(nd + 1, 0);
        for (int64_t i = 0; i < nd; ++i) P.contrib_base[i + 1] = P.contrib_base[i] + (iptr[i + 1] - iptr[i]) * nph;
        P.contrib_code.resize((size_t)n_cells * nph * nph);
        std::atomic<int> overflow{0};
        parallel_for(nd, [&](int64_t b, int64_t e) {
            std::vector<int> fillpos;
            for (int64_t i = b; i < e; ++i) {
                const int64_t r0 = P.row_ptr[i];
                const int len = (int)(P.row_ptr[i + 1] - r0);
                const int ninc = (int)(iptr[i + 1] - iptr[i]);
                // counts per slot, then offsets, then codes in incidence (= cell) order
                bool row_over = false;
                for (int t = 0; t < ninc; ++t)
                    for (int l = 0; l < nph; ++l) {
                        const int sl = P.inc_slot[(size_t)(iptr[i] + t) * nph + l];
                        if (P.contrib_cnt[r0 + sl] == 255) row_over = true;
                        else P.contrib_cnt[r0 + sl]++;
                    }
                if (row_over) {   // the codes would not fit the counts: reported below
                    overflow = 1;
                    continue;
                }
                fillpos.assign(len + 1, 0);
                for (int j = 0; j < len; ++j) fillpos[j + 1] = fillpos[j] + P.contrib_cnt[r0 + j];
                uint16_t *codes = P.contrib_code.data() + P.contrib_base[i];
                for (int t = 0; t < ninc; ++t)
                    for (int l = 0; l < nph; ++l) {
                        const int sl = P.inc_slot[(size_t)(iptr[i] + t) * nph + l];
                        codes[fillpos[sl]++] = (uint16_t)(t | (l << 8));
                    }
            }
        });
        if (overflow) return "a CSR entry has more than 255 contributions";
        // assembly chunks, and the codes re-counted from each chunk's first incidence;
        // with slicing a chunk also ends where the completion slice of its rows
        // (the slice of the row's last incident cell) changes
        auto row_slice = [&](int64_t i) -> int64_t {
            return (slice_cells > 0 && iptr[i + 1] > iptr[i]) ? (int64_t)(ielem[iptr[i + 1] - 1] / nph) / slice_cells : 0;
        };
        P.chunk_row.assign(1, 0);
        int64_t ent = 0, inc = 0, cur_slice = row_slice(0);
        for (int64_t i = 0; i < nd; ++i) {
            const int64_t ei = P.contrib_base[i + 1] - P.contrib_base[i], ii = iptr[i + 1] - iptr[i];
            const int64_t sl = row_slice(i);
            if (i > P.chunk_row.back() &&
                (ent + ei > kAsmChunkEntries || inc + ii > kAsmChunkIncidences || sl != cur_slice)) {
                P.chunk_row.push_back((int32_t)i);
                ent = inc = 0;
            }
            cur_slice = sl;
            ent += ei;
            inc += ii;
        }
        P.chunk_row.push_back((int32_t)nd);
        const int64_t n_chunks = (int64_t)P.chunk_row.size() - 1;
        P.chunk_slice.clear();
        P.slice_span = 0;
        if (slice_cells > 0) {
            P.chunk_slice.resize(n_chunks);
            for (int64_t k = 0; k < n_chunks; ++k) P.chunk_slice[k] = (int32_t)row_slice(P.chunk_row[k]);
            for (int64_t i = 0; i < nd; ++i)
                if (iptr[i + 1] > iptr[i]) {
                    const int64_t lo = (int64_t)(ielem[iptr[i]] / nph) / slice_cells;
                    P.slice_span = std::max<int>(P.slice_span, (int)(row_slice(i) - lo + 1));
                }
        }
        P.chunk_desc.resize((size_t)(n_chunks + 1) * 4);
        for (int64_t k = 0; k <= n_chunks; ++k) {
            const int64_t r = P.chunk_row[k];
            P.chunk_desc[k * 4 + 0] = r;
            P.chunk_desc[k * 4 + 1] = P.contrib_base[r];
            P.chunk_desc[k * 4 + 2] = iptr[r];
            P.chunk_desc[k * 4 + 3] = P.row_ptr[r];
        }
        P.contrib_dest.assign(P.contrib_code.size(), 0);
        parallel_for(n_chunks, [&](int64_t b, int64_t e) {
            for (int64_t k = b; k < e; ++k) {
                const int64_t e0 = iptr[P.chunk_row[k]];
                const int64_t c0 = P.contrib_base[P.chunk_row[k]];
                for (int64_t i = P.chunk_row[k]; i < P.chunk_row[k + 1]; ++i) {
                    const unsigned shift = (unsigned)(iptr[i] - e0);
                    for (int64_t j = P.contrib_base[i]; j < P.contrib_base[i + 1]; ++j) {
                        const unsigned code = P.contrib_code[j] + shift;
                        P.contrib_code[j] = (uint16_t)code;
                        P.contrib_dest[c0 + (int64_t)(code & 0xFFu) * nph + (code >> 8)] = (uint16_t)(j - c0);
                    }
                }
            }
        });
    }
    // vertex incidence for the adjoint's vertex scatter
    P.vinc_ptr.assign(n_vertices + 1, 0);
    for (int64_t i = 0; i < n_cells * nv; ++i) P.vinc_ptr[cells[i] + 1]++;
    for (int64_t i = 0; i < n_vertices; ++i) P.vinc_ptr[i + 1] += P.vinc_ptr[i];
    P.vinc.resize((size_t)n_cells * nv);
    {
        std::vector<int64_t> fill(P.vinc_ptr.begin(), P.vinc_ptr.end() - 1);
        for (int64_t c = 0; c < n_cells; ++c)
            for (int j = 0; j < nv; ++j) P.vinc[fill[cells[c * nv + j]]++] = (int32_t)(c * nv + j);
    }
    return "";
}

// --------------------------------------------------------------------------
// Storage formats and operand images
// --------------------------------------------------------------------------
double round_to_format(double x, int mbits, int emin, double maxfinite) {
    if (x == 0.0 || !std::isfinite(x)) return x;
    int e;
    std::frexp(x, &e);
    int E = e - 1;
    if (E < emin) E = emin;
    double ulp = std::ldexp(1.0, E - mbits);
    double r = std::nearbyint(x / ulp) * ulp;
    if (std::fabs(r) > maxfinite) r = std::copysign(maxfinite, x);
    return r;
}

Format format_of(int prec) {
    switch (prec) {
        case FE_PREC_BF16: return {2, 7, -126, 3.3895313892515355e38, 1};
        case FE_PREC_FP16: return {2, 10, -14, 65504.0, 15};
        case FE_PREC_TF32:
        case FE_PREC_TF32X3: return {4, 10, -126, 3.4028234663852886e38, 1};
        case FE_PREC_E4M3: return {1, 3, -6, 448.0, 8};
        default: return {8, 52, -1022, 1.7976931348623157e308, 1};
    }
}

uint32_t encode(int prec, double r) {
    if (prec == FE_PREC_BF16 || prec == FE_PREC_TF32 || prec == FE_PREC_TF32X3) {
        float f = (float)r;  // exact: r is representable
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return prec == FE_PREC_BF16 ? (u >> 16) : u;
    }
    uint32_t sign = std::signbit(r) ? 1u : 0u;
    double a = std::fabs(r);
    if (prec == FE_PREC_FP16) {
        if (a == 0.0) return sign << 15;
        int e;
        std::frexp(a, &e);
        int E = e - 1;
        if (E < -14) return (sign << 15) | (uint32_t)std::lrint(a * std::ldexp(1.0, 24));
        uint32_t mant = (uint32_t)std::lrint((a * std::ldexp(1.0, -E) - 1.0) * 1024.0);
        return (sign << 15) | ((uint32_t)(E + 15) << 10) | mant;
    }
    // e4m3
    if (a == 0.0) return sign << 7;
    int e;
    std::frexp(a, &e);
    int E = e - 1;
    if (E < -6) return (sign << 7) | (uint32_t)std::lrint(a * std::ldexp(1.0, 9));
    uint32_t mant = (uint32_t)std::lrint((a * std::ldexp(1.0, -E) - 1.0) * 8.0);
    return (sign << 7) | ((uint32_t)(E + 7) << 3) | mant;
}

int row_block_rows(int n_phi_) { return std::max(1, 240 / n_phi_); }

bool row_block_default(int n_phi_) {
    const int n_sym = n_phi_ * (n_phi_ + 1) / 2;
    if (n_sym <= 256) return false;
    const int R = row_block_rows(n_phi_);
    return (n_phi_ + R - 1) / R <= 2 * ((n_sym + 255) / 256);
}

std::vector<int> np_candidates(int n_phi_) {
    const int n_sym = n_phi_ * (n_phi_ + 1) / 2;
    std::vector<int> out;
    if (n_sym <= 256) {
        out.push_back((n_sym + 15) / 16 * 16);
        return out;
    }
    out.push_back(-row_block_rows(n_phi_));
    // wide passes: as many rows as fill both 256-column TMEM halves (one
    // accumulator, each coefficient chunk feeding two MMAs)
    const int wide_rows = 512 / n_phi_;
    if (wide_rows > row_block_rows(n_phi_) && wide_rows * n_phi_ > 256) out.push_back(-wide_rows);
    // half as many rows per pass: a smaller staging area leaves room for a
    // deeper operand ring
    if (row_block_rows(n_phi_) >= 2) out.push_back(-(row_block_rows(n_phi_) / 2));
    const int passes = (n_sym + 255) / 256;
    out.push_back(256);
    // the narrowest multiple of 16 with the same number of passes
    int np = ((n_sym + passes - 1) / passes + 15) / 16 * 16;
    if (np != 256) out.push_back(np);
    // one more pass with narrower tiles
    int np2 = ((n_sym + passes) / (passes + 1) + 15) / 16 * 16;
    if (np2 >= 64 && np2 != np && np2 != 256) out.push_back(np2);
    return out;
}

std::vector<int> stage_columns(int n_phi_, bool v4, int *conflicts) {
    const int n_sym = n_phi_ * (n_phi_ + 1) / 2;
    std::vector<int> col(n_sym);
    for (int i = 0; i < n_sym; ++i) col[i] = i;
    if (conflicts) *conflicts = -1;
    if (n_sym > 256) return col;
    const int ncol = (n_sym + 15) / 16 * 16;
    // pair index of (k, l), k <= l, in row order
    auto pair_of = [&](int k, int l) {
        if (k > l) std::swap(k, l);
        return k * n_phi_ - k * (k - 1) / 2 + (l - k);
    };
    // groups of each pair (one or two output positions)
    const int npos = n_phi_ * n_phi_;
    const int ngroups = v4 ? ((npos + 127) / 128) * 4 : (npos + 31) / 32;
    std::vector<std::vector<int>> members(ngroups);
    std::vector<std::array<int, 2>> groups_of(n_sym, {-1, -1});
    for (int pos = 0; pos < npos; ++pos) {
        const int g = v4 ? (pos / 128) * 4 + (pos & 3) : pos / 32;
        const int pr = pair_of(pos / n_phi_, pos % n_phi_);
        bool seen = false;
        for (int m : members[g]) seen = seen || (m == pr);
        if (!seen) members[g].push_back(pr);
        if (groups_of[pr][0] < 0) groups_of[pr][0] = g;
        else if (groups_of[pr][0] != g) groups_of[pr][1] = g;
    }
    std::vector<int> cap(32);
    for (int r = 0; r < 32; ++r) cap[r] = (ncol - r + 31) / 32;
    std::vector<int> best_colour(n_sym, 0);
    int best = INT32_MAX;
    uint64_t rng = 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        rng ^= rng << 13;
        rng ^= rng >> 7;
        rng ^= rng << 17;
        return rng;
    };
    std::vector<int> order(n_sym), colour(n_sym), left(32);
    std::vector<std::array<int, 32>> used(ngroups);
    for (int attempt = 0; attempt < 400 && best > 0; ++attempt) {
        for (int i = 0; i < n_sym; ++i) order[i] = i;
        // pairs in two groups first, random order within
        for (int i = n_sym - 1; i > 0; --i) std::swap(order[i], order[next() % (uint64_t)(i + 1)]);
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return (groups_of[a][1] >= 0) > (groups_of[b][1] >= 0); });
        for (auto &u : used) u.fill(0);
        left = cap;
        for (int pr : order) {
            int pick = -1, pick_cost = INT32_MAX, pick_left = -1;
            const int r0 = (int)(next() & 31);
            for (int t = 0; t < 32; ++t) {
                const int r = (r0 + t) & 31;
                if (left[r] == 0) continue;
                int cost = 0;
                for (int g : groups_of[pr])
                    if (g >= 0) cost += used[g][r];
                if (cost < pick_cost || (cost == pick_cost && left[r] > pick_left)) {
                    pick = r;
                    pick_cost = cost;
                    pick_left = left[r];
                }
            }
            colour[pr] = pick;
            --left[pick];
            for (int g : groups_of[pr])
                if (g >= 0) ++used[g][pick];
        }
        int excess = 0;
        for (int g = 0; g < ngroups; ++g)
            for (int r = 0; r < 32; ++r) excess += std::max(0, used[g][r] - 1);
        if (excess < best) {
            best = excess;
            best_colour = colour;
        }
    }
    // the pairs of colour r take columns r, r + 32, r + 64, ... in pair order
    std::vector<int> next_slot(32);
    for (int r = 0; r < 32; ++r) next_slot[r] = r;
    for (int pr = 0; pr < n_sym; ++pr) {
        col[pr] = next_slot[best_colour[pr]];
        next_slot[best_colour[pr]] += 32;
    }
    if (conflicts) *conflicts = best;
    return col;
}

void build_operand(int prec, int form, int d, int n_phi_, int n_q, const std::vector<double> &phi,
                   const std::vector<double> &dphi, OperandImage &img, int np_pass,
                   const std::vector<int> &col_of_sym) {
    const Format F = format_of(prec);
    const int eb = F.elem_bytes;
    const int KCE = 128 / eb;
    const bool stiff = (form == FE_FORM_STIFFNESS);
    const int n_pairs = stiff ? d * (d + 1) / 2 : 1;
    const int K_true = n_q * n_pairs;
    const int n_sym = n_phi_ * (n_phi_ + 1) / 2;
    std::vector<std::pair<int, int>> pairs;
    for (int s = 0; s < d; ++s)
        for (int t = s; t < d; ++t) pairs.push_back({s, t});
    std::vector<std::pair<int, int>> sym;
    for (int k = 0; k < n_phi_; ++k)
        for (int l = k; l < n_phi_; ++l) sym.push_back({k, l});
    auto B = [&](int s, int k, int q) { return dphi[((size_t)s * n_phi_ + k) * n_q + q]; };
    // P[K][col] in FP64: the product of two tabulated factors (Sec. 3.1, triple products)
    std::vector<double> Pv((size_t)K_true * n_sym);
    double maxabs = 0.0;
    for (int q = 0; q < n_q; ++q)
        for (int j = 0; j < n_pairs; ++j) {
            int K = q * n_pairs + j;
            for (int c = 0; c < n_sym; ++c) {
                int k = sym[c].first, l = sym[c].second;
                double v;
                if (stiff) {
                    int s = pairs[j].first, t = pairs[j].second;
                    v = B(s, k, q) * B(t, l, q);
                    if (s != t) v += B(t, k, q) * B(s, l, q);
                } else {
                    v = phi[(size_t)k * n_q + q] * phi[(size_t)l * n_q + q];
                }
                Pv[(size_t)K * n_sym + c] = v;
                maxabs = std::max(maxabs, std::fabs(v));
            }
        }
    int eP = 0;
    if (prec == FE_PREC_FP16 || prec == FE_PREC_E4M3) {
        int e;
        std::frexp(maxabs, &e);
        eP = F.target_exp - e;
    }
    img.p_inv_scale = std::ldexp(1.0, -eP);
    img.n_blk = (prec == FE_PREC_TF32X3) ? 3 : 1;
    img.n_pairs = n_pairs;
    // K blocks (quadrature window qw of KW points, pair j, split block blk),
    // numbered h = (qw n_pairs + j) n_blk + blk; a 128-byte chunk holds
    // KCE / KW consecutive blocks (two 64-point blocks for e4m3, so that a
    // builder thread needs only a 64-point window, one block otherwise)
    const int KW = tc_window_points(prec);
    const int WPC = KCE / KW;
    img.n_qw = (n_q + KW - 1) / KW;
    const int n_blocks = img.n_qw * n_pairs * img.n_blk;
    img.n_kchunks = (n_blocks + WPC - 1) / WPC;
    img.n_cols = n_sym;
    if (np_pass == 0 && row_block_default(n_phi_)) np_pass = -row_block_rows(n_phi_);
    if (np_pass < 0) {
        const int R = std::min(-np_pass, n_phi_);
        img.rows_per_pass = R;
        img.NP = (R * n_phi_ + 15) / 16 * 16;
        img.n_pass = (n_phi_ + R - 1) / R;
        img.n_cols = img.n_pass * img.NP;
    } else if (np_pass >= 16 && np_pass <= 256 && np_pass % 16 == 0) {
        img.NP = np_pass;
        img.n_pass = (n_sym + np_pass - 1) / np_pass;
    } else if (n_sym <= 256) {
        img.NP = (n_sym + 15) / 16 * 16;
        img.n_pass = 1;
    } else {
        img.NP = 256;
        img.n_pass = (n_sym + 255) / 256;
    }
    // rounded values (and TF32 tails)
    std::vector<double> hi(Pv.size()), lo;
    for (size_t i = 0; i < Pv.size(); ++i) hi[i] = round_to_format(std::ldexp(Pv[i], eP), F.mbits, F.emin, F.maxfinite);
    if (img.n_blk == 3) {
        lo.resize(Pv.size());
        for (size_t i = 0; i < Pv.size(); ++i) lo[i] = round_to_format(std::ldexp(Pv[i], eP) - hi[i], F.mbits, F.emin, F.maxfinite);
    }
    (void)K_true;
    // pair at each operand column (-1: padding)
    std::vector<int> pair_at((size_t)img.n_pass * img.NP, -1);
    if (img.rows_per_pass > 0) {
        // pass n: rows k = n R .. n R + R - 1, column (k - n R) n_phi + l
        const int R = img.rows_per_pass;
        for (int n = 0; n < img.n_pass; ++n)
            for (int r = 0; r < R * n_phi_; ++r) {
                const int k = n * R + r / n_phi_, l = r % n_phi_;
                if (k >= n_phi_) continue;
                const int a = std::min(k, l), b = std::max(k, l);
                pair_at[(size_t)n * img.NP + r] = a * n_phi_ - a * (a - 1) / 2 + (b - a);
            }
    } else {
        for (int c = 0; c < n_sym; ++c) {
            const int colc = col_of_sym.empty() ? c : col_of_sym[c];
            if (colc >= 0 && colc < (int)pair_at.size()) pair_at[colc] = c;
        }
        if (!col_of_sym.empty()) img.n_cols = std::min<int>((int)pair_at.size(), (n_sym + 15) / 16 * 16);
    }
    const size_t block = (size_t)img.NP * 128;
    img.bytes.assign(block * img.n_kchunks * img.n_pass, 0);
    for (int n = 0; n < img.n_pass; ++n)
        for (int ch = 0; ch < img.n_kchunks; ++ch) {
            uint8_t *base = img.bytes.data() + ((size_t)n * img.n_kchunks + ch) * block;
            for (int r = 0; r < img.NP; ++r) {
                const int col = n * img.NP + r;
                const int pr = pair_at[col];
                for (int e = 0; e < KCE; ++e) {
                    const int h = ch * WPC + e / KW;   // K block of this byte range
                    const int qw = h / (n_pairs * img.n_blk);
                    const int j = (h / img.n_blk) % n_pairs;
                    const int blk = h % img.n_blk;
                    const int q = qw * KW + e % KW;
                    double v = 0.0;
                    if (pr >= 0 && h < n_blocks && q < n_q) {
                        const std::vector<double> &src = (blk == 1) ? lo : hi;  // C_hi P_hi, C_hi P_lo, C_lo P_hi
                        v = src[(size_t)(q * n_pairs + j) * n_sym + pr];
                    }
                    uint32_t bits = encode(prec, v);
                    int byte = e * eb;
                    size_t off = (size_t)(r >> 3) * 1024 + (r & 7) * 128 + ((((byte >> 4) ^ (r & 7)) & 7) << 4) + (byte & 15);
                    std::memcpy(base + off, &bits, eb);  // little-endian low bytes
                }
            }
        }
}

}  // namespace host
}  // namespace fe
