// Host-side construction of the adaptive mesh and its device tables.
//
// Sec. 3.1 of the paper: the box is first covered by coarse uniform cubes and
// cells are halved where resolution is needed; each cell carries the tensor
// product of 1D Lagrange polynomials through the Gauss-Lobatto points, and
// "bridged" functions make the discrete space continuous across cells.  On a
// 2:1-balanced octree this is the conforming Q_p space: a node of a fine leaf
// that lies on the face or edge of a coarser neighbour without being one of
// that neighbour's nodes is a hanging node, whose value is the coarse
// neighbour's polynomial evaluated there.  The mesh is static during a run
// (Sec. 4), so everything here runs once, on the host, before upload.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <unordered_set>

#include "afem_internal.h"

namespace afem {

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
int cuda_error(cudaError_t e, const char* what) {
    return set_error(AFEM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
const char* last_error_cstr() { return g_last_error.c_str(); }

// ---------------------------------------------------------- 1D GLL basis
// Nodes on [-1,1]: the endpoints and the roots of P_p'.  The interior roots
// are found by Newton's method on P_p', with P_p'' from Legendre's equation
// (1 - x^2) P'' = 2 x P' - p (p+1) P, started from the Chebyshev extrema.
static void legendre_and_deriv(int p, double x, double& P, double& dP) {
    double p0 = 1.0, p1 = x;
    if (p == 0) { P = 1.0; dP = 0.0; return; }
    for (int k = 2; k <= p; ++k) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
    }
    P = p1;
    // P_p' = p (x P_p - P_{p-1}) / (x^2 - 1), valid away from +-1.
    dP = p * (x * p1 - p0) / (x * x - 1.0);
}

Basis1D make_basis(int p) {
    Basis1D b;
    b.p = p;
    double x[kMaxP1];
    x[0] = -1.0;
    x[p] = 1.0;
    for (int j = 1; j < p; ++j) {
        double t = -std::cos(M_PI * j / p);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre_and_deriv(p, t, P, dP);
            double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
            double step = dP / d2P;
            t -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        x[j] = t;
    }
    for (int j = 0; j <= p; ++j) {
        double P, dP;
        legendre_and_deriv(p, x[j], P, dP);
        if (j == 0 || j == p) {  // P_p(+-1) = (+-1)^p
            P = (j == 0 && (p % 2)) ? -1.0 : 1.0;
        }
        b.xi[j] = 0.5 * (x[j] + 1.0);
        b.w[j] = 0.5 * 2.0 / (p * (p + 1.0) * P * P);
    }
    b.xi[0] = 0.0;
    b.xi[p] = 1.0;
    // Lagrange derivative matrix D[q][j] = L_j'(xi_q) by barycentric weights.
    double lam[kMaxP1], D[kMaxP1][kMaxP1];
    for (int j = 0; j <= p; ++j) {
        double prod = 1.0;
        for (int m = 0; m <= p; ++m)
            if (m != j) prod *= (b.xi[j] - b.xi[m]);
        lam[j] = 1.0 / prod;
    }
    for (int q = 0; q <= p; ++q) {
        double diag = 0.0;
        for (int j = 0; j <= p; ++j) {
            if (j == q) continue;
            D[q][j] = (lam[j] / lam[q]) / (b.xi[q] - b.xi[j]);
            diag -= D[q][j];
        }
        D[q][q] = diag;
    }
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p; ++j) {
            double s = 0.0;
            for (int q = 0; q <= p; ++q) s += b.w[q] * D[q][i] * D[q][j];
            b.K[i][j] = s;
            b.S[i][j] = 0.5 * (b.w[i] * D[i][j] - b.w[j] * D[j][i]);
        }
    return b;
}

double lagrange_value(const Basis1D& b, int j, double t) {
    double v = 1.0;
    for (int m = 0; m <= b.p; ++m)
        if (m != j) v *= (t - b.xi[m]) / (b.xi[j] - b.xi[m]);
    return v;
}

// L_j'(t) by the product rule on the Lagrange product form.
static double lagrange_deriv(const Basis1D& b, int j, double t) {
    double d = 0.0;
    for (int k = 0; k <= b.p; ++k) {
        if (k == j) continue;
        double term = 1.0 / (b.xi[j] - b.xi[k]);
        for (int m = 0; m <= b.p; ++m)
            if (m != j && m != k) term *= (t - b.xi[m]) / (b.xi[j] - b.xi[m]);
        d += term;
    }
    return d;
}

// n-point Gauss-Legendre rule on [0, 1] (roots of P_n by Newton's method).
static void gauss_legendre01(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double P = 0.0, dP = 1.0;
        for (int it = 0; it < 100; ++it) {
            legendre_and_deriv(n, t, P, dP);
            const double step = P / dP;
            t -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        legendre_and_deriv(n, t, P, dP);
        x[n - 1 - i] = 0.5 * (t + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dP * dP);   // 2 / ((1 - t^2) P'^2), halved for [0, 1]
    }
}

// ------------------------------------------------------------ octree
namespace {

constexpr int kFracBits = 40;    // fractional bits of integer point coordinates
constexpr int kCoordBits = 20;   // bits per axis of a leaf index at its level

struct Leaf {
    int32_t l;
    int64_t i, j, k;
};

inline uint64_t leaf_key(int l, int64_t i, int64_t j, int64_t k) {
    return (uint64_t(l) << 60) | (uint64_t(i) << 40) | (uint64_t(j) << 20) | uint64_t(k);
}

struct Key3 {
    int64_t x, y, z;
    bool operator==(const Key3& o) const { return x == o.x && y == o.y && z == o.z; }
};
struct Key3Hash {
    size_t operator()(const Key3& k) const {
        uint64_t h = uint64_t(k.x) * 0x9E3779B97F4A7C15ull;
        h ^= uint64_t(k.y) + 0x7F4A7C159E3779B9ull + (h << 6) + (h >> 2);
        h ^= uint64_t(k.z) + 0x94D049BB133111EBull + (h << 6) + (h >> 2);
        return size_t(h ^ (h >> 31));
    }
};

uint64_t spread3(uint64_t v) {  // 21 bits -> every third bit
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
}

}  // namespace

// eta_K^2 of Kelly's indicator on the Coulomb potential of the nuclei (Sec. 3.1):
// (h_K / 24) sum over the faces F of int_F [d_n V_h]^2, V_h the cellwise GLL
// interpolant of V = -sum Z_a / |r - R_a|, [d_n V_h] the jump of its normal
// derivative to the leaf across each (sub)face (a coarser or equal leaf covers
// the whole face, four finer leaves a quarter each), integrated by the
// (p+1) x (p+1) Gauss-Legendre rule of the (sub)face; no term on the box
// surface; +inf for a leaf whose closed box contains a nucleus.
static const double kelly_c3 = 3.0 * std::log(2.0 + std::sqrt(3.0)) - M_PI / 2.0;

template <typename FindLeaf>
static double kelly_eta2(const afem_mesh_desc& d, const Basis1D& B, const Leaf& c, FindLeaf& find_leaf) {
    const int p = B.p, p1 = p + 1;
    const double h0 = (d.hi - d.lo) / d.n_coarse;
    auto geom = [&](const Leaf& f, double& h, double* c0) {
        h = h0 / double(int64_t(1) << f.l);
        c0[0] = d.lo + double(f.i) * h;
        c0[1] = d.lo + double(f.j) * h;
        c0[2] = d.lo + double(f.k) * h;
    };
    double h, c0[3];
    geom(c, h, c0);
    for (int n = 0; n < d.n_nuclei; ++n) {
        bool in = true;
        for (int ax = 0; ax < 3; ++ax)
            if (d.nuc_pos[n][ax] < c0[ax] || d.nuc_pos[n][ax] > c0[ax] + h) in = false;
        if (in) return HUGE_VAL;
    }
    // nodal values V[c][b][a] of a leaf
    auto values = [&](const Leaf& f, double* V) {
        double hf, cf[3];
        geom(f, hf, cf);
        for (int cz = 0; cz < p1; ++cz)
            for (int cy = 0; cy < p1; ++cy)
                for (int cx = 0; cx < p1; ++cx) {
                    const double x = cf[0] + hf * B.xi[cx], y = cf[1] + hf * B.xi[cy], z = cf[2] + hf * B.xi[cz];
                    double v = 0.0;
                    for (int n = 0; n < d.n_nuclei; ++n) {
                        const double dx = x - d.nuc_pos[n][0], dy = y - d.nuc_pos[n][1], dz = z - d.nuc_pos[n][2];
                        const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
                        // a node on a nucleus: the mean of 1/|r| over a cube of the node's GLL volume
                        v -= r > 1e-10 ? d.nuc_charge[n] / r
                                       : d.nuc_charge[n] * kelly_c3 / (hf * std::cbrt(B.w[cx] * B.w[cy] * B.w[cz]));
                    }
                    V[(cz * p1 + cy) * p1 + cx] = v;
                }
    };
    // d/dx_ax of a leaf's interpolant at point X
    auto dn = [&](const Leaf& f, const double* V, const double* X, int ax) {
        double hf, cf[3];
        geom(f, hf, cf);
        double L[3][kMaxP1];
        for (int q = 0; q < 3; ++q) {
            const double t = (X[q] - cf[q]) / hf;
            for (int a = 0; a < p1; ++a) L[q][a] = q == ax ? lagrange_deriv(B, a, t) / hf : lagrange_value(B, a, t);
        }
        double r = 0.0;
        for (int cz = 0; cz < p1; ++cz)
            for (int cy = 0; cy < p1; ++cy)
                for (int cx = 0; cx < p1; ++cx) r += V[(cz * p1 + cy) * p1 + cx] * L[0][cx] * L[1][cy] * L[2][cz];
        return r;
    };
    double gx[kMaxP1], gw[kMaxP1];
    gauss_legendre01(p1, gx, gw);
    double Vc[kMaxP1 * kMaxP1 * kMaxP1], Vn[kMaxP1 * kMaxP1 * kMaxP1];
    values(c, Vc);
    const int64_t nmax = int64_t(d.n_coarse) << c.l;
    double tot = 0.0;
    // int over the square face (corner fc, side hs, normal ax at x_ax = xf) of the jump to leaf f
    auto face = [&](const Leaf& f, const double* Vf, const double* fc, double hs, int ax, double xf) {
        const int o0 = ax == 0 ? 1 : 0, o1 = ax == 2 ? 1 : 2;
        double acc = 0.0;
        for (int a = 0; a < p1; ++a)
            for (int b = 0; b < p1; ++b) {
                double X[3];
                X[ax] = xf;
                X[o0] = fc[o0] + hs * gx[a];
                X[o1] = fc[o1] + hs * gx[b];
                const double J = dn(c, Vc, X, ax) - dn(f, Vf, X, ax);
                acc += gw[a] * gw[b] * hs * hs * J * J;
            }
        return acc;
    };
    for (int ax = 0; ax < 3; ++ax)
        for (int side = 0; side < 2; ++side) {
            int64_t nb[3] = {c.i, c.j, c.k};
            nb[ax] += side ? 1 : -1;
            if (nb[ax] < 0 || nb[ax] >= nmax) continue;
            Leaf f;
            const double xf = c0[ax] + side * h;
            if (find_leaf(c.l, nb[0], nb[1], nb[2], f)) {
                values(f, Vn);
                tot += face(f, Vn, c0, h, ax, xf);
            } else {
                const int o0 = ax == 0 ? 1 : 0, o1 = ax == 2 ? 1 : 2;
                for (int u = 0; u < 2; ++u)
                    for (int v = 0; v < 2; ++v) {
                        int64_t ch[3] = {2 * nb[0], 2 * nb[1], 2 * nb[2]};
                        ch[ax] += side ? 0 : 1;
                        ch[o0] += u;
                        ch[o1] += v;
                        const Leaf fine{c.l + 1, ch[0], ch[1], ch[2]};
                        double cs[3] = {c0[0], c0[1], c0[2]};
                        cs[o0] += u * 0.5 * h;
                        cs[o1] += v * 0.5 * h;
                        values(fine, Vn);
                        tot += face(fine, Vn, cs, 0.5 * h, ax, xf);
                    }
            }
        }
    return h / 24.0 * tot;
}

static int build_host_mesh_leaves(const afem_mesh_desc& d, const std::vector<Leaf>* given, HostMesh& M);

int build_host_mesh(const afem_mesh_desc& d, HostMesh& M) { return build_host_mesh_leaves(d, nullptr, M); }

int build_host_mesh_cells(const afem_mesh_desc& d, const std::vector<int32_t>& lev, const std::vector<int32_t>& ci,
                          const std::vector<int32_t>& cj, const std::vector<int32_t>& ck, HostMesh& M) {
    std::vector<Leaf> given(lev.size());
    for (size_t q = 0; q < lev.size(); ++q) given[q] = {lev[q], ci[q], cj[q], ck[q]};
    return build_host_mesh_leaves(d, &given, M);
}

// Builds the mesh from `given` leaves (balanced here) when non-null, else
// from the refinement rule of the description.
static int build_host_mesh_leaves(const afem_mesh_desc& d, const std::vector<Leaf>* given, HostMesh& M) {
    const int p = d.degree;
    const int p1 = p + 1;
    const int nn = p1 * p1 * p1;
    const int nc = d.n_coarse;
    M.p = p;
    M.lo = d.lo;
    M.hi = d.hi;
    M.n_coarse = nc;
    M.h0 = (d.hi - d.lo) / nc;
    const double h0 = M.h0;
    const Basis1D B = make_basis(p);

    std::vector<Leaf> leaves;
    std::unordered_set<uint64_t> leafset;
    auto rebuild_set = [&]() {
        leafset.clear();
        leafset.reserve(leaves.size() * 2);
        for (const Leaf& c : leaves) leafset.insert(leaf_key(c.l, c.i, c.j, c.k));
    };
    // Leaf containing the level-l cell (i,j,k): that cell or one of its ancestors.
    auto find_leaf = [&](int l, int64_t i, int64_t j, int64_t k, Leaf& out) -> bool {
        for (int l2 = l; l2 >= 0; --l2) {
            const int s = l - l2;
            if (leafset.count(leaf_key(l2, i >> s, j >> s, k >> s))) {
                out = {l2, i >> s, j >> s, k >> s};
                return true;
            }
        }
        return false;
    };
    auto split_into = [](const Leaf& c, std::vector<Leaf>& next) {
        for (int s = 0; s < 8; ++s)
            next.push_back({c.l + 1, 2 * c.i + (s & 1), 2 * c.j + ((s >> 1) & 1), 2 * c.k + ((s >> 2) & 1)});
    };
    // 2:1 balance across faces, edges and vertices
    auto balance = [&]() -> int {
        rebuild_set();
        for (;;) {
            std::unordered_set<uint64_t> split;
            for (const Leaf& c : leaves) {
                if (c.l < 2) continue;
                const int64_t n = int64_t(nc) << c.l;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (!dx && !dy && !dz) continue;
                            const int64_t a = c.i + dx, b = c.j + dy, e = c.k + dz;
                            if (a < 0 || b < 0 || e < 0 || a >= n || b >= n || e >= n) continue;
                            Leaf f;
                            if (find_leaf(c.l, a, b, e, f) && f.l < c.l - 1)
                                split.insert(leaf_key(f.l, f.i, f.j, f.k));
                        }
            }
            if (split.empty()) return AFEM_OK;
            std::vector<Leaf> next;
            next.reserve(leaves.size() + 8 * split.size());
            for (const Leaf& c : leaves) {
                if (split.count(leaf_key(c.l, c.i, c.j, c.k))) split_into(c, next);
                else next.push_back(c);
            }
            leaves.swap(next);
            if (leaves.size() > (size_t(1) << 26)) return set_error(AFEM_EMESH, "mesh: more than 2^26 leaves");
            rebuild_set();
        }
    };
    int brc;
    if (given) {
        // ---- explicit leaves (a coarsened copy of another mesh's octree)
        leaves = *given;
        if ((brc = balance())) return brc;
    } else if (d.refine_mode == AFEM_REFINE_KELLY) {
        // ---- Kelly's indicator on the Coulomb potential of the nuclei (Sec. 3.1)
        for (int i = 0; i < nc; ++i)
            for (int j = 0; j < nc; ++j)
                for (int k = 0; k < nc; ++k) leaves.push_back({0, i, j, k});
        rebuild_set();
        for (;;) {
            std::vector<Leaf> next;
            next.reserve(leaves.size() * 2);
            bool any = false;
            for (const Leaf& c : leaves) {
                if (c.l < d.kelly_max_level && kelly_eta2(d, B, c, find_leaf) > d.kelly_threshold * d.kelly_threshold) {
                    split_into(c, next);
                    any = true;
                } else {
                    next.push_back(c);
                }
            }
            if (!any) break;
            leaves.swap(next);
            if (leaves.size() > (size_t(1) << 26)) return set_error(AFEM_EMESH, "mesh: more than 2^26 leaves");
            if ((brc = balance())) return brc;
        }
    } else {
        // ---- the geometric rule toward the nuclei
        leaves.reserve(size_t(nc) * nc * nc);
        for (int i = 0; i < nc; ++i)
            for (int j = 0; j < nc; ++j)
                for (int k = 0; k < nc; ++k) leaves.push_back({0, i, j, k});
        for (;;) {
            bool any = false;
            std::vector<Leaf> next;
            next.reserve(leaves.size() * 2);
            for (const Leaf& c : leaves) {
                const double h = h0 / double(int64_t(1) << c.l);
                const double a[3] = {d.lo + double(c.i) * h, d.lo + double(c.j) * h, d.lo + double(c.k) * h};
                bool split = false;
                for (int n = 0; n < d.n_nuclei && !split; ++n) {
                    if (c.l >= d.nuc_levels[n]) continue;
                    double d2 = 0.0;
                    for (int ax = 0; ax < 3; ++ax) {
                        const double R = d.nuc_pos[n][ax];
                        const double b = a[ax] + h;
                        if (R < a[ax]) {
                            const double t = a[ax] - R;
                            d2 += t * t;
                        } else if (R > b) {
                            const double t = R - b;
                            d2 += t * t;
                        }
                    }
                    const double ch = d.refine_c * h;
                    split = d2 <= ch * ch;
                }
                if (split) {
                    any = true;
                    split_into(c, next);
                } else {
                    next.push_back(c);
                }
            }
            leaves.swap(next);
            if (!any) break;
            if (leaves.size() > (size_t(1) << 26))
                return set_error(AFEM_EMESH, "mesh: more than 2^26 leaves");
        }
        if ((brc = balance())) return brc;
    }
    int Lf = 0;
    for (const Leaf& c : leaves) Lf = std::max(Lf, int(c.l));
    M.max_level = Lf;
    if ((int64_t(nc) << Lf) >= (int64_t(1) << kCoordBits))
        return set_error(AFEM_EMESH, "mesh: n_coarse * 2^levels exceeds 2^20");

    // ---- Morton (Z-order) traversal of the leaves
    std::vector<std::pair<uint64_t, size_t>> order(leaves.size());
    for (size_t q = 0; q < leaves.size(); ++q) {
        const Leaf& c = leaves[q];
        const int s = Lf - c.l;
        order[q] = {spread3(uint64_t(c.i) << s) | (spread3(uint64_t(c.j) << s) << 1) |
                        (spread3(uint64_t(c.k) << s) << 2),
                    q};
    }
    std::sort(order.begin(), order.end());
    const size_t ncell = leaves.size();
    {
        std::vector<Leaf> sorted(ncell);
        for (size_t q = 0; q < ncell; ++q) sorted[q] = leaves[order[q].second];
        leaves.swap(sorted);
    }
    std::unordered_map<uint64_t, int64_t> cell_of;
    cell_of.reserve(ncell * 2);
    for (size_t q = 0; q < ncell; ++q)
        cell_of[leaf_key(leaves[q].l, leaves[q].i, leaves[q].j, leaves[q].k)] = int64_t(q);

    // ---- support points: integer coordinates in units of h_finest / 2^kFracBits
    std::unordered_map<Key3, int64_t, Key3Hash> point_of;
    point_of.reserve(ncell * nn);
    std::vector<Key3> pkey;
    std::vector<int64_t> cellpt(ncell * nn);
    std::vector<double> mf;   // assembled GLL weight per support point
    for (size_t q = 0; q < ncell; ++q) {
        const Leaf& c = leaves[q];
        const int64_t S = int64_t(1) << (Lf - c.l + kFracBits);
        int64_t off[kMaxP1];
        for (int a = 0; a < p1; ++a) off[a] = std::llround(B.xi[a] * double(S));
        const double h = h0 / double(int64_t(1) << c.l);
        const double h3 = h * h * h;
        for (int cz = 0; cz < p1; ++cz)
            for (int cy = 0; cy < p1; ++cy)
                for (int cx = 0; cx < p1; ++cx) {
                    const Key3 key{c.i * S + off[cx], c.j * S + off[cy], c.k * S + off[cz]};
                    auto it = point_of.find(key);
                    int64_t id;
                    if (it == point_of.end()) {
                        id = int64_t(pkey.size());
                        point_of.emplace(key, id);
                        pkey.push_back(key);
                        mf.push_back(0.0);
                    } else {
                        id = it->second;
                    }
                    cellpt[q * nn + cx + p1 * (cy + p1 * cz)] = id;
                    mf[id] += h3 * B.w[cx] * B.w[cy] * B.w[cz];
                }
    }
    const int64_t npts = int64_t(pkey.size());

    // ---- hanging nodes: nodes of a leaf inside the closure of a coarser
    // face/edge/vertex neighbour that are not nodes of that neighbour.
    std::vector<int64_t> hang_src_ptr(npts + 1, 0);
    std::vector<std::vector<std::pair<int64_t, double>>> hang_rows;   // per hanging point
    std::vector<int64_t> hang_row_of(npts, -1);
    for (size_t q = 0; q < ncell; ++q) {
        const Leaf& c = leaves[q];
        if (c.l == 0) continue;
        const int64_t n = int64_t(nc) << c.l;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz) continue;
                    const int64_t a = c.i + dx, b = c.j + dy, e = c.k + dz;
                    if (a < 0 || b < 0 || e < 0 || a >= n || b >= n || e >= n) continue;
                    Leaf f;
                    if (!find_leaf(c.l, a, b, e, f) || f.l != c.l - 1) continue;
                    const int64_t qc = cell_of.at(leaf_key(f.l, f.i, f.j, f.k));
                    // offsets of this leaf inside the coarse neighbour, in fine cells
                    const int64_t del[3] = {c.i - 2 * f.i, c.j - 2 * f.j, c.k - 2 * f.k};
                    for (int cz = 0; cz < p1; ++cz)
                        for (int cy = 0; cy < p1; ++cy)
                            for (int cx = 0; cx < p1; ++cx) {
                                const int loc[3] = {cx, cy, cz};
                                double t[3];
                                bool inside = true, is_node = true;
                                for (int ax = 0; ax < 3; ++ax) {
                                    t[ax] = (double(del[ax]) + B.xi[loc[ax]]) * 0.5;
                                    if (t[ax] < -1e-12 || t[ax] > 1.0 + 1e-12) inside = false;
                                    double best = 1.0;
                                    for (int m = 0; m < p1; ++m)
                                        best = std::min(best, std::fabs(t[ax] - B.xi[m]));
                                    if (best > 1e-9) is_node = false;
                                }
                                if (!inside || is_node) continue;
                                const int64_t pt = cellpt[q * nn + cx + p1 * (cy + p1 * cz)];
                                if (hang_row_of[pt] >= 0) continue;
                                hang_row_of[pt] = int64_t(hang_rows.size());
                                std::vector<std::pair<int64_t, double>> row;
                                double Lx[kMaxP1], Ly[kMaxP1], Lz[kMaxP1];
                                for (int m = 0; m < p1; ++m) {
                                    Lx[m] = lagrange_value(B, m, t[0]);
                                    Ly[m] = lagrange_value(B, m, t[1]);
                                    Lz[m] = lagrange_value(B, m, t[2]);
                                }
                                for (int mz = 0; mz < p1; ++mz)
                                    for (int my = 0; my < p1; ++my)
                                        for (int mx = 0; mx < p1; ++mx) {
                                            const double wgt = Lx[mx] * Ly[my] * Lz[mz];
                                            if (wgt == 0.0) continue;
                                            row.push_back({cellpt[qc * nn + mx + p1 * (my + p1 * mz)], wgt});
                                        }
                                hang_rows.push_back(std::move(row));
                            }
                }
    }
    (void)hang_src_ptr;

    // ---- numbering: interior masters, then surface masters, each in first-touch order
    const int64_t top = (int64_t(nc) << Lf) << kFracBits;
    std::vector<int64_t> master_id(npts, -1), hang_id(npts, -1);
    int64_t nint = 0, nmaster = 0, nhang = 0;
    auto on_surface = [&](const Key3& k) {
        return k.x == 0 || k.y == 0 || k.z == 0 || k.x == top || k.y == top || k.z == top;
    };
    for (int64_t pt = 0; pt < npts; ++pt)
        if (hang_row_of[pt] < 0 && !on_surface(pkey[pt])) master_id[pt] = nint++;
    nmaster = nint;
    for (int64_t pt = 0; pt < npts; ++pt)
        if (hang_row_of[pt] < 0 && on_surface(pkey[pt])) master_id[pt] = nmaster++;
    for (int64_t pt = 0; pt < npts; ++pt)
        if (hang_row_of[pt] >= 0) hang_id[pt] = nhang++;
    if (nmaster >= (int64_t(1) << 31) || nhang >= (int64_t(1) << 30))
        return set_error(AFEM_EMESH, "mesh: index range exceeds int32");

    M.n_master = nmaster;
    M.n_interior = nint;
    M.n_hanging = nhang;
    M.lev.resize(ncell);
    M.ci.resize(ncell);
    M.cj.resize(ncell);
    M.ck.resize(ncell);
    M.corner.resize(ncell * 3);
    M.h.resize(ncell);
    M.cell_node.resize(ncell * nn);
    for (size_t q = 0; q < ncell; ++q) {
        const Leaf& c = leaves[q];
        M.lev[q] = c.l;
        M.ci[q] = int32_t(c.i);
        M.cj[q] = int32_t(c.j);
        M.ck[q] = int32_t(c.k);
        const double h = h0 / double(int64_t(1) << c.l);
        M.h[q] = h;
        M.corner[3 * q + 0] = d.lo + double(c.i) * h;
        M.corner[3 * q + 1] = d.lo + double(c.j) * h;
        M.corner[3 * q + 2] = d.lo + double(c.k) * h;
        for (int n = 0; n < nn; ++n) {
            const int64_t pt = cellpt[q * nn + n];
            M.cell_node[q * nn + n] =
                master_id[pt] >= 0 ? int32_t(master_id[pt]) : int32_t(-hang_id[pt] - 1);
        }
    }
    const double unit = h0 / double(int64_t(1) << Lf) / double(int64_t(1) << kFracBits);
    auto coord = [&](const Key3& k, double* x) {
        x[0] = d.lo + double(k.x) * unit;
        x[1] = d.lo + double(k.y) * unit;
        x[2] = d.lo + double(k.z) * unit;
    };
    M.master_xyz.assign(nmaster * 3, 0.0);
    M.hang_xyz.assign(nhang * 3, 0.0);
    M.ml.assign(nmaster, 0.0);
    M.mf_master.assign(nmaster, 0.0);
    M.mf_hang.assign(nhang, 0.0);
    std::vector<double>& mf_master = M.mf_master;
    std::vector<double>& mf_hang = M.mf_hang;
    for (int64_t pt = 0; pt < npts; ++pt) {
        if (master_id[pt] >= 0) {
            coord(pkey[pt], &M.master_xyz[3 * master_id[pt]]);
            M.ml[master_id[pt]] += mf[pt];
            mf_master[master_id[pt]] = mf[pt];
        } else {
            coord(pkey[pt], &M.hang_xyz[3 * hang_id[pt]]);
            mf_hang[hang_id[pt]] = mf[pt];
        }
    }
    M.hang_ptr.assign(nhang + 1, 0);
    M.hang_master.clear();
    M.hang_w.clear();
    {
        std::vector<int64_t> pt_of_hang(nhang);
        for (int64_t pt = 0; pt < npts; ++pt)
            if (hang_id[pt] >= 0) pt_of_hang[hang_id[pt]] = pt;
        for (int64_t hh = 0; hh < nhang; ++hh) {
            const auto& row = hang_rows[hang_row_of[pt_of_hang[hh]]];
            for (const auto& e : row) {
                const int64_t m = master_id[e.first];
                if (m < 0)
                    return set_error(AFEM_EMESH,
                                     "mesh: hanging point constrained by another hanging point");
                M.hang_master.push_back(int32_t(m));
                M.hang_w.push_back(e.second);
                M.ml[m] += e.second * mf_hang[hh];
            }
            M.hang_ptr[hh + 1] = int32_t(M.hang_master.size());
        }
    }

    // ---- nuclear potential V = -sum_a Z_a / |x - R_a| at masters and hanging points.
    // A support point on a nucleus takes -Z c3 / s with s = m_f^(1/3) and
    // c3 = 3 ln(2 + sqrt 3) - pi/2, the mean of 1/|r| over a unit cube.
    const double c3 = 3.0 * std::log(2.0 + std::sqrt(3.0)) - M_PI / 2.0;
    auto potential = [&](const double* x, double mfx) {
        double v = 0.0;
        for (int n = 0; n < d.n_nuclei; ++n) {
            const double rx = x[0] - d.nuc_pos[n][0], ry = x[1] - d.nuc_pos[n][1],
                         rz = x[2] - d.nuc_pos[n][2];
            const double r = std::sqrt(rx * rx + ry * ry + rz * rz);
            if (r < 1e-10)
                v -= d.nuc_charge[n] * c3 / std::cbrt(mfx);
            else
                v -= d.nuc_charge[n] / r;
        }
        return v;
    };
    M.v_master.resize(nmaster);
    M.v_hang.resize(nhang);
    for (int64_t m = 0; m < nmaster; ++m) M.v_master[m] = potential(&M.master_xyz[3 * m], mf_master[m]);
    for (int64_t hh = 0; hh < nhang; ++hh) M.v_hang[hh] = potential(&M.hang_xyz[3 * hh], mf_hang[hh]);
    // ---- nuclear force on an electron, -grad V = -sum_a Z_a (x - R_a) / |x - R_a|^3
    // (the Ehrenfest acceleration's potential part); 0 at a support point on a
    // nucleus, where the cube-averaged value vanishes by symmetry.
    auto force = [&](const double* x, double* f) {
        f[0] = f[1] = f[2] = 0.0;
        for (int n = 0; n < d.n_nuclei; ++n) {
            const double r3[3] = {x[0] - d.nuc_pos[n][0], x[1] - d.nuc_pos[n][1], x[2] - d.nuc_pos[n][2]};
            const double r = std::sqrt(r3[0] * r3[0] + r3[1] * r3[1] + r3[2] * r3[2]);
            if (r < 1e-10) continue;
            const double c = d.nuc_charge[n] / (r * r * r);
            for (int k = 0; k < 3; ++k) f[k] -= c * r3[k];
        }
    };
    M.f_master.resize(3 * size_t(nmaster));
    M.f_hang.resize(3 * size_t(nhang));
    for (int64_t m = 0; m < nmaster; ++m) force(&M.master_xyz[3 * m], &M.f_master[3 * m]);
    for (int64_t hh = 0; hh < nhang; ++hh) force(&M.hang_xyz[3 * hh], &M.f_hang[3 * hh]);

    // ---- diagonal of the constrained stiffness A = C^T (sum_K P_K^T A_K P_K) C:
    // per cell, each master k has local coefficients c_k (1 at its own node,
    // the constraint weights at hanging nodes), and adds c_k^T A_K c_k.
    M.stiff_diag.assign(nmaster, 0.0);
    {
        std::vector<std::pair<int32_t, std::pair<int, double>>> loc;   // (master, (node, coef))
        for (size_t q = 0; q < ncell; ++q) {
            loc.clear();
            for (int n = 0; n < nn; ++n) {
                const int32_t id = M.cell_node[q * nn + n];
                if (id >= 0) {
                    loc.push_back({id, {n, 1.0}});
                } else {
                    const int32_t hh = -id - 1;
                    for (int32_t e = M.hang_ptr[hh]; e < M.hang_ptr[hh + 1]; ++e)
                        loc.push_back({M.hang_master[e], {n, M.hang_w[e]}});
                }
            }
            std::sort(loc.begin(), loc.end(),
                      [](const auto& a, const auto& b) { return a.first < b.first; });
            const double h = M.h[q];
            auto Aloc = [&](int i, int j) {
                const int ia = i % p1, ib = (i / p1) % p1, ic = i / (p1 * p1);
                const int ja = j % p1, jb = (j / p1) % p1, jc = j / (p1 * p1);
                double v = 0.0;
                if (ib == jb && ic == jc) v += B.K[ia][ja] * B.w[ib] * B.w[ic];
                if (ia == ja && ic == jc) v += B.w[ia] * B.K[ib][jb] * B.w[ic];
                if (ia == ja && ib == jb) v += B.w[ia] * B.w[ib] * B.K[ic][jc];
                return h * v;
            };
            for (size_t s0 = 0; s0 < loc.size();) {
                size_t s1 = s0;
                while (s1 < loc.size() && loc[s1].first == loc[s0].first) ++s1;
                double acc = 0.0;
                for (size_t a = s0; a < s1; ++a)
                    for (size_t b = s0; b < s1; ++b)
                        acc += loc[a].second.second * loc[b].second.second *
                               Aloc(loc[a].second.first, loc[b].second.first);
                M.stiff_diag[loc[s0].first] += acc;
                s0 = s1;
            }
        }
    }
    return AFEM_OK;
}

// ------------------------------------------------------------ upload
template <typename T>
static int upload(T*& dst, const T* src, size_t n) {
    dst = nullptr;
    if (n == 0) return AFEM_OK;
    cudaError_t e = cudaMalloc(&dst, n * sizeof(T));
    if (e != cudaSuccess) return set_error(AFEM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    AFEM_CUDA_TRY(cudaMemcpy(dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return AFEM_OK;
}

int upload_mesh(afem_mesh* m) {
    const HostMesh& H = m->host;
    DeviceMesh& D = m->dev;
    const int nn = (H.p + 1) * (H.p + 1) * (H.p + 1);
    D.p = H.p;
    D.ncell = int64_t(H.lev.size());
    D.n_master = H.n_master;
    D.n_interior = H.n_interior;
    D.n_hanging = H.n_hanging;
    D.nnz = int64_t(H.hang_master.size());
    std::vector<double4> geom(D.ncell);
    for (int64_t q = 0; q < D.ncell; ++q)
        geom[q] = make_double4(H.corner[3 * q], H.corner[3 * q + 1], H.corner[3 * q + 2], H.h[q]);
    std::vector<double> ml_inv(H.n_master);
    for (int64_t k = 0; k < H.n_master; ++k) ml_inv[k] = 1.0 / H.ml[k];
    int rc;
    if ((rc = upload(D.cell_node, H.cell_node.data(), H.cell_node.size()))) return rc;
    if ((rc = upload(D.cell_geom, geom.data(), geom.size()))) return rc;
    if ((rc = upload(D.hang_ptr, H.hang_ptr.data(), H.hang_ptr.size()))) return rc;
    if ((rc = upload(D.hang_master, H.hang_master.data(), H.hang_master.size()))) return rc;
    if ((rc = upload(D.hang_w, H.hang_w.data(), H.hang_w.size()))) return rc;
    if ((rc = upload(D.ml, H.ml.data(), H.ml.size()))) return rc;
    if ((rc = upload(D.ml_inv, ml_inv.data(), ml_inv.size()))) return rc;
    if ((rc = upload(D.v_master, H.v_master.data(), H.v_master.size()))) return rc;
    if ((rc = upload(D.v_hang, H.v_hang.data(), H.v_hang.size()))) return rc;
    if ((rc = upload(D.f_master, H.f_master.data(), H.f_master.size()))) return rc;
    if ((rc = upload(D.f_hang, H.f_hang.data(), H.f_hang.size()))) return rc;
    {
        std::vector<double> dinv(H.n_master, 0.0);
        for (int64_t k = 0; k < H.n_interior; ++k) dinv[k] = 1.0 / H.stiff_diag[k];
        if ((rc = upload(D.stiff_dinv, dinv.data(), dinv.size()))) return rc;
    }
    {
        std::vector<double> mxyz(H.master_xyz);
        if ((rc = upload(D.master_xyz, mxyz.data(), mxyz.size()))) return rc;
        if ((rc = upload(D.hang_xyz, H.hang_xyz.data(), H.hang_xyz.size()))) return rc;
        if ((rc = upload(D.mf_master, H.mf_master.data(), H.mf_master.size()))) return rc;
        if ((rc = upload(D.mf_hang, H.mf_hang.data(), H.mf_hang.size()))) return rc;
    }
    {
        auto to_f = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
        std::vector<float4> g32(D.ncell);
        for (int64_t q = 0; q < D.ncell; ++q)
            g32[q] = make_float4(float(H.corner[3 * q]), float(H.corner[3 * q + 1]), float(H.corner[3 * q + 2]),
                                 float(H.h[q]));
        std::vector<float> dinv32(H.n_master, 0.0f);
        for (int64_t k = 0; k < H.n_interior; ++k) dinv32[k] = float(1.0 / H.stiff_diag[k]);
        if ((rc = upload(D.cell_geom32, g32.data(), g32.size()))) return rc;
        auto hw = to_f(H.hang_w), vm = to_f(H.v_master), vh = to_f(H.v_hang);
        if ((rc = upload(D.hang_w32, hw.data(), hw.size()))) return rc;
        if ((rc = upload(D.v_master32, vm.data(), vm.size()))) return rc;
        if ((rc = upload(D.v_hang32, vh.data(), vh.size()))) return rc;
        if ((rc = upload(D.stiff_dinv32, dinv32.data(), dinv32.size()))) return rc;
        // the potential at every cell node in cell order: the FP32 cell pass reads it
        // coalesced instead of gathering it through the node map
        std::vector<float> vc(size_t(D.ncell) * nn);
        for (size_t o = 0; o < vc.size(); ++o) {
            const int32_t idx = H.cell_node[o];
            vc[o] = float(idx >= 0 ? H.v_master[idx] : H.v_hang[-idx - 1]);
        }
        if ((rc = upload(D.v_cell32, vc.data(), vc.size()))) return rc;
        std::vector<float> mli32(H.n_master);
        for (int64_t k = 0; k < H.n_master; ++k) mli32[k] = float(1.0 / H.ml[k]);
        if ((rc = upload(D.ml_inv32, mli32.data(), mli32.size()))) return rc;
    }
    return AFEM_OK;
}

void free_device_mesh(DeviceMesh& D) {
    // workspaces live on the mesh object; see afem_mesh_destroy
    cudaFree(D.cell_node);
    cudaFree(D.cell_geom);
    cudaFree(D.hang_ptr);
    cudaFree(D.hang_master);
    cudaFree(D.hang_w);
    cudaFree(D.ml);
    cudaFree(D.ml_inv);
    cudaFree(D.v_master);
    cudaFree(D.v_hang);
    cudaFree(D.f_master);
    cudaFree(D.f_hang);
    cudaFree(D.stiff_dinv);
    cudaFree(D.master_xyz);
    cudaFree(D.hang_xyz);
    cudaFree(D.mf_master);
    cudaFree(D.mf_hang);
    cudaFree(D.cell_geom32);
    cudaFree(D.hang_w32);
    cudaFree(D.v_master32);
    cudaFree(D.v_hang32);
    cudaFree(D.v_cell32);
    cudaFree(D.ml_inv32);
    cudaFree(D.stiff_dinv32);
    D = DeviceMesh{};
}

}  // namespace afem
