// Host-side construction of the linear octree, its nodes, and the geometric tables.
//
//  * top-down refinement by region predicates, octants outside the box dropped
//    (Sec. "Octree based Mesh Generation": refine an octant while a user function says so);
//  * 2:1 balance across faces, edges and vertices (same section);
//  * meshing: independent nodes, hanging nodes with 2 (edge) or 4 (face) parents -- the
//    interpolation operators I1d and I2d = I1d x I1d of Algorithm 3;
//  * triangle tables, background triangles B_T of every element (Algorithm 1), a (y, z) grid
//    for ray casting, the Nitsche surface quadrature (Eq. weakbc and its remark on h_b), and
//    the strong-boundary / In-only node rows (Algorithm 1, Fig. IBM).
//
// Leaves are kept sorted by the Morton code of their anchor; the leaf containing a point is
// the last leaf whose code does not exceed the point's code (binary search).  Arithmetic that
// decides geometry (region tests, box / AABB overlaps, triangle normals and centroids, h_b) is
// compiled with floating-point contraction disabled so that it is reproducible bit for bit.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "imga_internal.h"

#ifdef _OPENMP
#include <omp.h>
#include <parallel/algorithm>
#endif

namespace imga {

namespace {

inline uint32_t octsize(int l) { return 1u << (kMaxDepth - l); }

inline bool inside_box(const Mesh& m, int64_t x, int64_t y, int64_t z) {
    return x >= 0 && y >= 0 && z >= 0 && x < m.hiI[0] && y < m.hiI[1] && z < m.hiI[2];
}

void phys_box(const Mesh& m, const uint32_t a[3], uint32_t s, double b0[3], double b1[3]) {
    for (int k = 0; k < 3; ++k) {
        b0[k] = m.lo[k] + (double)a[k] * m.scale;
        b1[k] = m.lo[k] + (double)(a[k] + s) * m.scale;
    }
}

bool region_meets(const imga_region& r, const double b0[3], const double b1[3]) {
    const double* p = r.par;
    switch (r.kind) {
        case 0: {  // spherical band: nearest and farthest distance of the box to the centre
            double near2 = 0.0, far2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                double below = b0[k] - p[k], above = p[k] - b1[k];
                double dn = std::max(0.0, std::max(below, above));
                near2 = near2 + dn * dn;
                double df = std::max(std::fabs(b0[k] - p[k]), std::fabs(b1[k] - p[k]));
                far2 = far2 + df * df;
            }
            double outer = p[3] + p[4], inner = p[3] - p[4];
            if (!(near2 <= outer * outer)) return false;
            return inner <= 0.0 || far2 >= inner * inner;
        }
        case 1:
            for (int k = 0; k < 3; ++k)
                if (!(b0[k] <= p[3 + k] && b1[k] >= p[k])) return false;
            return true;
        default: {  // cone along +x tested at the box centre, inflated by half the diagonal
            double cx = 0.5 * (b0[0] + b1[0]), cy = 0.5 * (b0[1] + b1[1]), cz = 0.5 * (b0[2] + b1[2]);
            double half_diag = 0.8660254037844386 * (b1[0] - b0[0]);
            double s = cx - p[0];
            if (s < -half_diag || s > p[3] + half_diag) return false;
            double ry = cy - p[1], rz = cz - p[2];
            double rad = std::sqrt(ry * ry + rz * rz);
            return rad <= p[4] + std::max(s, 0.0) * p[5] + half_diag;
        }
    }
}

int wanted_level(const Mesh& m, const uint32_t a[3], int l) {
    double b0[3], b1[3];
    phys_box(m, a, octsize(l), b0, b1);
    int t = m.base_level;
    for (const imga_region& r : m.regions)
        if (r.level > t && region_meets(r, b0, b1)) t = r.level;
    return t;
}

struct Oct { uint32_t a[3]; int l; };

}  // namespace

// Leaf lookup: keys are 60-bit Morton codes of 20-bit anchors.  The table of the top kLutBits
// bits (an octant of level kLutBits / 3) narrows the binary search to the leaves under that
// octant.  A coarser leaf spans several such octants and leaves their ranges empty: the answer
// is then the leaf just before the range, as the plain search over all keys would find.
constexpr int kLutBits = 21, kLutShift = 3 * kMaxDepth - kLutBits;

int64_t find_leaf(const Mesh& m, int64_t x, int64_t y, int64_t z) {
    if (!inside_box(m, x, y, z)) return -1;
    uint64_t k = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
    auto first = m.key.begin(), last = m.key.end();
    if (m.key_lut_n == m.key.size() && !m.key_lut.empty()) {
        const uint64_t p = k >> kLutShift;
        first = m.key.begin() + m.key_lut[p];
        last = m.key.begin() + m.key_lut[p + 1];
    }
    auto it = std::upper_bound(first, last, k);
    if (it == m.key.begin()) return -1;
    int64_t e = (int64_t)(it - m.key.begin()) - 1;
    uint32_t s = octsize(m.lev[e]);
    const uint32_t* a = &m.anc[3 * e];
    if ((uint64_t)x - a[0] < s && (uint64_t)y - a[1] < s && (uint64_t)z - a[2] < s) return e;
    return -1;
}

static void set_leaves(Mesh& m, const std::vector<Oct>& L) {
    size_t n = L.size();
    m.anc.resize(3 * n);
    m.lev.resize(n);
    m.key.resize(n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        for (int k = 0; k < 3; ++k) m.anc[3 * i + k] = L[i].a[k];
        m.lev[i] = (uint8_t)L[i].l;
        m.key[i] = morton3(L[i].a[0], L[i].a[1], L[i].a[2]);
    }
    // prefix table: key_lut[p] = lower bound of p << kLutShift
    const size_t np = (size_t)1 << kLutBits;
    m.key_lut.assign(np + 1, (int32_t)n);
    size_t i = 0;
    for (size_t p = 0; p <= np; ++p) {
        while (i < n && (m.key[i] >> kLutShift) < p) ++i;
        m.key_lut[p] = (int32_t)i;
    }
    m.key_lut_n = n;
}

// depth-first refinement of the subtree rooted at o, children in Morton order: leaves come out sorted
static void refine_subtree(const Mesh& m, Oct root, std::vector<Oct>& leaves) {
    std::vector<Oct> stack;
    stack.push_back(root);
    while (!stack.empty()) {
        Oct o = stack.back();
        stack.pop_back();
        if (o.l < wanted_level(m, o.a, o.l)) {
            uint32_t h = octsize(o.l) >> 1;
            for (int c = 7; c >= 0; --c) {   // pushed in reverse so child 0 is processed first
                Oct ch{{o.a[0] + ((c & 1) ? h : 0), o.a[1] + ((c & 2) ? h : 0), o.a[2] + ((c & 4) ? h : 0)}, o.l + 1};
                if (inside_box(m, ch.a[0], ch.a[1], ch.a[2])) stack.push_back(ch);
            }
        } else {
            leaves.push_back(o);
        }
    }
}

bool build_octree(Mesh& m, std::string& err) {
    // top-down refinement.  The octants of the first kSplitLevel levels are visited depth first;
    // each octant of level kSplitLevel that still needs refining is a subtree refined on its own
    // thread.  Concatenating leaves and subtrees in visiting order gives the same Morton-ordered
    // list as one depth-first pass.
    constexpr int kSplitLevel = 4;
    std::vector<Oct> items;          // leaves above kSplitLevel, and the subtree roots at it
    std::vector<char> is_root;
    {
        std::vector<Oct> stack;
        stack.push_back({{0, 0, 0}, 0});
        while (!stack.empty()) {
            Oct o = stack.back();
            stack.pop_back();
            if (o.l < wanted_level(m, o.a, o.l)) {
                if (o.l == kSplitLevel) { items.push_back(o); is_root.push_back(1); continue; }
                uint32_t h = octsize(o.l) >> 1;
                for (int c = 7; c >= 0; --c) {
                    Oct ch{{o.a[0] + ((c & 1) ? h : 0), o.a[1] + ((c & 2) ? h : 0), o.a[2] + ((c & 4) ? h : 0)}, o.l + 1};
                    if (inside_box(m, ch.a[0], ch.a[1], ch.a[2])) stack.push_back(ch);
                }
            } else {
                items.push_back(o);
                is_root.push_back(0);
            }
        }
    }
    std::vector<std::vector<Oct>> sub(items.size());
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < (int64_t)items.size(); ++i)
        if (is_root[i]) refine_subtree(m, items[i], sub[i]);
    std::vector<Oct> leaves;
    {
        size_t total = 0;
        for (size_t i = 0; i < items.size(); ++i) total += is_root[i] ? sub[i].size() : 1;
        leaves.reserve(total);
        for (size_t i = 0; i < items.size(); ++i) {
            if (is_root[i]) leaves.insert(leaves.end(), sub[i].begin(), sub[i].end());
            else leaves.push_back(items[i]);
            std::vector<Oct>().swap(sub[i]);
        }
    }
    set_leaves(m, leaves);
    // 2:1 balance: a leaf of level l forces every leaf it touches to level >= l - 1.  The fine
    // leaf finds the coarse one by probing just outside each face, edge and vertex.  The first
    // pass probes from every leaf.  After a pass, a violation needs a fine side that the pass
    // created, or one that found a violation in it and was not split: a pair of untouched leaves
    // was balanced before, and a new child G of a split leaf B is too coarse only for a leaf
    // that was already more than one level finer than B.  So later passes probe from those
    // leaves only.  Every split is forced, so the result is the coarsest balanced refinement
    // whatever the order.
    static const int nb[26][3] = {{-1,-1,-1},{0,-1,-1},{1,-1,-1},{-1,0,-1},{0,0,-1},{1,0,-1},{-1,1,-1},{0,1,-1},{1,1,-1},
                                  {-1,-1,0},{0,-1,0},{1,-1,0},{-1,0,0},{1,0,0},{-1,1,0},{0,1,0},{1,1,0},
                                  {-1,-1,1},{0,-1,1},{1,-1,1},{-1,0,1},{0,0,1},{1,0,1},{-1,1,1},{0,1,1},{1,1,1}};
    std::vector<int64_t> probe;
    bool probe_all = true;
    for (int pass = 0; pass < 64; ++pass) {
        const int64_t n = m.n_elem();
        const int64_t n_probe = probe_all ? n : (int64_t)probe.size();
        std::vector<uint8_t> split(n, 0), found(n, 0);
        int any = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(| : any)
        for (int64_t i = 0; i < n_probe; ++i) {
            const int64_t e = probe_all ? i : probe[i];
            int l = m.lev[e];
            if (l < 2) continue;
            int64_t s = octsize(l);
            const uint32_t* a = &m.anc[3 * e];
            // the grandparent octant (edge 4s) has been refined, so every leaf inside it has level
            // >= l - 1: only probes that leave it can find a leaf two levels coarser
            int64_t g0[3];
            for (int k = 0; k < 3; ++k) g0[k] = (int64_t)a[k] & ~(4 * s - 1);
            for (int d = 0; d < 26; ++d) {
                int64_t q[3];
                bool out = false;
                for (int k = 0; k < 3; ++k) {
                    q[k] = nb[d][k] < 0 ? (int64_t)a[k] - 1 : nb[d][k] > 0 ? (int64_t)a[k] + s : (int64_t)a[k];
                    out = out || q[k] < g0[k] || q[k] >= g0[k] + 4 * s;
                }
                if (!out) continue;
                int64_t o = find_leaf(m, q[0], q[1], q[2]);
                if (o >= 0 && m.lev[o] < l - 1) {
                    __atomic_store_n(&split[o], (uint8_t)1, __ATOMIC_RELAXED);
                    found[e] = 1;
                    any = 1;
                }
            }
        }
        if (!any) break;
        std::vector<Oct> next;
        std::vector<int64_t> next_probe;
        next.reserve(n + 8 * std::count(split.begin(), split.end(), 1));
        for (int64_t e = 0; e < n; ++e) {
            const uint32_t* a = &m.anc[3 * e];
            int l = m.lev[e];
            if (!split[e]) {
                if (found[e]) next_probe.push_back((int64_t)next.size());
                next.push_back({{a[0], a[1], a[2]}, l});
                continue;
            }
            uint32_t h = octsize(l) >> 1;
            for (int c = 0; c < 8; ++c) {
                Oct ch{{a[0] + ((c & 1) ? h : 0), a[1] + ((c & 2) ? h : 0), a[2] + ((c & 4) ? h : 0)}, l + 1};
                if (inside_box(m, ch.a[0], ch.a[1], ch.a[2])) {
                    next_probe.push_back((int64_t)next.size());
                    next.push_back(ch);
                }
            }
        }
        set_leaves(m, next);
        probe.swap(next_probe);
        probe_all = false;
        if (pass == 63) { err = "2:1 balance did not converge"; return false; }
    }
    for (int64_t e = 0; e < m.n_elem(); ++e)
        if (m.lev[e] > kMaxLevel - 1) { err = "leaf level beyond the supported maximum"; return false; }
    return true;
}

bool build_nodes(Mesh& m, std::string& err) {
    const int64_t ne = m.n_elem();
    // every leaf corner, deduplicated by Morton code of its coordinates
    std::vector<uint64_t> ck(8 * ne);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e) {
        uint32_t s = octsize(m.lev[e]);
        const uint32_t* a = &m.anc[3 * e];
        for (int c = 0; c < 8; ++c)
            ck[8 * e + c] = morton3(a[0] + ((c & 1) ? s : 0), a[1] + ((c & 2) ? s : 0), a[2] + ((c & 4) ? s : 0));
    }
    // unique corner codes: neighbouring leaves in Morton order share most corners, so each chunk
    // of leaves is sorted and deduplicated on its own first (in cache, in parallel); the global
    // sort then sees a few keys per node instead of up to eight
    std::vector<uint64_t> uk;
    {
        constexpr int64_t kChunk = 1 << 14;                         // leaves per chunk
        const int64_t nchunk = (ne + kChunk - 1) / kChunk;
        std::vector<std::vector<uint64_t>> part(nchunk);
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t c = 0; c < nchunk; ++c) {
            const int64_t a = 8 * c * kChunk, b = std::min<int64_t>(8 * ne, 8 * (c + 1) * kChunk);
            std::vector<uint64_t>& v = part[c];
            v.assign(ck.begin() + a, ck.begin() + b);
            std::sort(v.begin(), v.end());
            v.erase(std::unique(v.begin(), v.end()), v.end());
        }
        size_t total = 0;
        for (const auto& v : part) total += v.size();
        uk.reserve(total);
        for (auto& v : part) { uk.insert(uk.end(), v.begin(), v.end()); std::vector<uint64_t>().swap(v); }
    }
#ifdef _OPENMP
    __gnu_parallel::sort(uk.begin(), uk.end());
#else
    std::sort(uk.begin(), uk.end());
#endif
    uk.erase(std::unique(uk.begin(), uk.end()), uk.end());
    const int64_t nu = (int64_t)uk.size();
    // coordinates of each unique corner, read back from its Morton code
    std::vector<uint32_t> ux(3 * nu);
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < nu; ++u)
        for (int k = 0; k < 3; ++k) ux[3 * u + k] = compact1by2(uk[u] >> k);
    // hanging test: P is hanging when a leaf touching P does not have P as a corner
    std::vector<int8_t> np(nu, 0);
    std::vector<uint32_t> par(12 * nu);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(| : bad)
    for (int64_t u = 0; u < nu; ++u) {
        const uint32_t* P = &ux[3 * u];
        for (int nbh = 0; nbh < 8 && np[u] == 0; ++nbh) {
            int64_t q[3] = {(int64_t)P[0] - (nbh & 1), (int64_t)P[1] - ((nbh >> 1) & 1), (int64_t)P[2] - ((nbh >> 2) & 1)};
            int64_t o = find_leaf(m, q[0], q[1], q[2]);
            if (o < 0) continue;
            uint32_t s = octsize(m.lev[o]);
            const uint32_t* a = &m.anc[3 * o];
            int mid[3], nmid = 0;
            for (int k = 0; k < 3; ++k) {
                if (P[k] == a[k] || P[k] == a[k] + s) mid[k] = 0;
                else if (P[k] == a[k] + s / 2) { mid[k] = 1; ++nmid; }
                else { bad = 1; mid[k] = 0; }
            }
            if (nmid == 0) continue;
            if (nmid > 2) { bad = 1; continue; }
            np[u] = (int8_t)(1 << nmid);
            for (int p = 0; p < np[u]; ++p) {
                int bit = 0;
                for (int k = 0; k < 3; ++k) {
                    if (mid[k]) { par[12 * u + 3 * p + k] = a[k] + (((p >> bit) & 1) ? s : 0); ++bit; }
                    else par[12 * u + 3 * p + k] = P[k];
                }
            }
        }
    }
    if (bad) { err = "mesh is not 2:1 balanced (hanging node off an edge/face midpoint)"; return false; }
    // independent nodes (Morton order) and hanging nodes (Morton order)
    std::vector<int64_t> slot(nu);
    int64_t nn = 0, nh = 0;
    for (int64_t u = 0; u < nu; ++u) slot[u] = np[u] ? -(++nh) : nn++;
    m.nijk.resize(3 * nn);
    m.hpar.assign(4 * nh, -1);
    m.hnp.resize(nh);
    std::vector<uint64_t> nkey(nn);
    for (int64_t u = 0; u < nu; ++u)
        if (slot[u] >= 0) {
            for (int k = 0; k < 3; ++k) m.nijk[3 * slot[u] + k] = ux[3 * u + k];
            nkey[slot[u]] = uk[u];
        }
    for (int64_t u = 0; u < nu; ++u) {
        if (slot[u] >= 0) continue;
        int64_t h = -slot[u] - 1;
        m.hnp[h] = np[u];
        for (int p = 0; p < np[u]; ++p) {
            const uint32_t* Q = &par[12 * u + 3 * p];
            uint64_t pk = morton3(Q[0], Q[1], Q[2]);
            auto it = std::lower_bound(nkey.begin(), nkey.end(), pk);
            if (it == nkey.end() || *it != pk) { err = "parent of a hanging node is not an independent node"; return false; }
            m.hpar[4 * h + p] = (int32_t)(it - nkey.begin());
        }
    }
    m.conn.resize(8 * ne);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < 8 * ne; ++i) {
        int64_t u = std::lower_bound(uk.begin(), uk.end(), ck[i]) - uk.begin();
        m.conn[i] = slot[u] >= 0 ? (int32_t)slot[u] : (int32_t)(nn + (-slot[u] - 1));
    }
    return true;
}

bool build_triangles(Mesh& m, const double* t, int64_t n, std::string& err) {
    TriHost& T = m.tri;
    T.n = n;
    T.v.assign(t, t + 9 * n);
    T.nrm.resize(3 * n);
    T.cen.resize(3 * n);
    T.bmin.resize(3 * n);
    T.bmax.resize(3 * n);
    T.area.resize(n);
    for (int64_t i = 0; i < n; ++i) {
        const double* v = &T.v[9 * i];
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) { e1[k] = v[3 + k] - v[k]; e2[k] = v[6 + k] - v[k]; }
        double cx = e1[1] * e2[2] - e1[2] * e2[1];
        double cy = e1[2] * e2[0] - e1[0] * e2[2];
        double cz = e1[0] * e2[1] - e1[1] * e2[0];
        double len = std::sqrt(cx * cx + cy * cy + cz * cz);
        if (!(len > 0.0)) { err = "degenerate triangle " + std::to_string(i); return false; }
        T.nrm[3 * i] = cx / len;
        T.nrm[3 * i + 1] = cy / len;
        T.nrm[3 * i + 2] = cz / len;
        T.area[i] = 0.5 * len;
        for (int k = 0; k < 3; ++k) {
            T.cen[3 * i + k] = (v[k] + v[3 + k] + v[6 + k]) / 3.0;
            T.bmin[3 * i + k] = std::min(std::min(v[k], v[3 + k]), v[6 + k]);
            T.bmax[3 * i + k] = std::max(std::max(v[k], v[3 + k]), v[6 + k]);
        }
    }
    return true;
}

// Background triangles: for every triangle, descend the octree from the root through the
// octants its bounding box meets, down to the leaves; B_T(e) = triangles whose box meets the
// closed box of e widened on every side by kBtPad times its edge.  Stored as CSR sorted by
// element, then triangle.
//
// The widening keeps the normal test of Algorithm 6 sound where a face of the body lies on a
// plane of the grid, as axis-aligned faces at round coordinates do.  Whether such a face's
// triangles meet the exact closed box of the element beside it is then a matter of rounding or
// of the surface's noise.  A point of that element in front of the face, but behind the planes
// of neighbouring triangles that reach into the element, would be called In when the face is
// left out.  A larger B_T is never less safe: an added triangle either agrees with the others
// or makes the test undecided, and the point goes to the exact ray.  Octants are widened by the
// same fraction of their own edge, which covers the widened boxes of the leaves inside them.
constexpr double kBtPad = 1e-2;

void build_background(Mesh& m) {
    const int64_t nt = m.tri.n, ne = m.n_elem();
    std::vector<std::vector<std::pair<int32_t, int32_t>>> local;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            local.resize(omp_get_num_threads());
#else
            local.resize(1);
#endif
        }
#ifdef _OPENMP
        auto& mine = local[omp_get_thread_num()];
#else
        auto& mine = local[0];
#endif
        std::vector<Oct> st;
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nt; ++t) {
            const double* lo = &m.tri.bmin[3 * t];
            const double* hi = &m.tri.bmax[3 * t];
            st.clear();
            st.push_back({{0, 0, 0}, 0});
            while (!st.empty()) {
                Oct o = st.back();
                st.pop_back();
                double b0[3], b1[3];
                uint32_t s = octsize(o.l);
                phys_box(m, o.a, s, b0, b1);
                const double pad_o = kBtPad * ((double)s * m.scale);
                bool meet = true;
                for (int k = 0; k < 3; ++k)
                    if (!(lo[k] <= b1[k] + pad_o && hi[k] >= b0[k] - pad_o)) meet = false;
                if (!meet) continue;
                int64_t e = find_leaf(m, o.a[0], o.a[1], o.a[2]);
                if (e >= 0 && m.lev[e] <= o.l) {
                    // the octant lies inside leaf e: test the leaf's own widened box
                    double c0[3], c1[3];
                    const uint32_t se = octsize(m.lev[e]);
                    phys_box(m, &m.anc[3 * e], se, c0, c1);
                    const double pad = kBtPad * ((double)se * m.scale);
                    bool hit = true;
                    for (int k = 0; k < 3; ++k)
                        if (!(lo[k] <= c1[k] + pad && hi[k] >= c0[k] - pad)) hit = false;
                    if (hit) mine.push_back({(int32_t)e, (int32_t)t});
                    continue;
                }
                uint32_t h = s >> 1;
                for (int c = 0; c < 8; ++c) {
                    Oct ch{{o.a[0] + ((c & 1) ? h : 0), o.a[1] + ((c & 2) ? h : 0), o.a[2] + ((c & 4) ? h : 0)}, o.l + 1};
                    if (inside_box(m, ch.a[0], ch.a[1], ch.a[2])) st.push_back(ch);
                }
            }
        }
    }
    std::vector<std::pair<int32_t, int32_t>> all;
    for (auto& v : local) all.insert(all.end(), v.begin(), v.end());
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    m.bt_off.assign(ne + 1, 0);
    m.bt_idx.resize(all.size());
    for (size_t i = 0; i < all.size(); ++i) { m.bt_off[all[i].first + 1]++; m.bt_idx[i] = all[i].second; }
    for (int64_t e = 0; e < ne; ++e) m.bt_off[e + 1] += m.bt_off[e];
}

// Ray grid: triangles binned by their (y, z) bounding boxes widened by a margin far above
// rounding, so that a ray cast along +x can only hit -- or graze -- triangles listed in the
// cell of its origin.
void build_ray_grid(Mesh& m) {
    RayGridHost& g = m.grid;
    const int64_t nt = m.tri.n;
    g.ny = g.nz = 0;
    g.off.assign(1, 0);
    g.idx.clear();
    if (nt == 0) return;
    double ylo = 1e300, yhi = -1e300, zlo = 1e300, zhi = -1e300, ext = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
        ylo = std::min(ylo, m.tri.bmin[3 * t + 1]); yhi = std::max(yhi, m.tri.bmax[3 * t + 1]);
        zlo = std::min(zlo, m.tri.bmin[3 * t + 2]); zhi = std::max(zhi, m.tri.bmax[3 * t + 2]);
    }
    for (int k = 0; k < 3; ++k) ext = std::max(ext, std::fabs(m.lo[k]) + std::fabs(m.hi[k]));
    ext = std::max(ext, std::max(std::fabs(ylo), std::max(std::fabs(yhi), std::max(std::fabs(zlo), std::fabs(zhi)))));
    const double margin = 1e-9 * ext;
    int n1 = (int)std::min(2048.0, std::max(1.0, std::sqrt((double)nt) * 1.5));
    g.ny = g.nz = n1;
    g.y0 = ylo - 2 * margin;
    g.z0 = zlo - 2 * margin;
    g.dy = (yhi - ylo + 4 * margin) / n1;
    g.dz = (zhi - zlo + 4 * margin) / n1;
    auto cell = [&](double v, double v0, double dv, int n) {
        int c = (int)std::floor((v - v0) / dv);
        return std::min(std::max(c, 0), n - 1);
    };
    std::vector<int32_t> cnt(n1 * n1 + 1, 0);
    std::vector<int> r(4 * nt);
    for (int64_t t = 0; t < nt; ++t) {
        r[4 * t] = cell(m.tri.bmin[3 * t + 1] - margin, g.y0, g.dy, n1);
        r[4 * t + 1] = cell(m.tri.bmax[3 * t + 1] + margin, g.y0, g.dy, n1);
        r[4 * t + 2] = cell(m.tri.bmin[3 * t + 2] - margin, g.z0, g.dz, n1);
        r[4 * t + 3] = cell(m.tri.bmax[3 * t + 2] + margin, g.z0, g.dz, n1);
        for (int a = r[4 * t]; a <= r[4 * t + 1]; ++a)
            for (int b = r[4 * t + 2]; b <= r[4 * t + 3]; ++b) cnt[a * n1 + b + 1]++;
    }
    for (int i = 0; i < n1 * n1; ++i) cnt[i + 1] += cnt[i];
    g.off = cnt;
    g.idx.resize(cnt[n1 * n1]);
    std::vector<int32_t> pos(cnt.begin(), cnt.end() - 1);
    for (int64_t t = 0; t < nt; ++t)
        for (int a = r[4 * t]; a <= r[4 * t + 1]; ++a)
            for (int b = r[4 * t + 2]; b <= r[4 * t + 3]; ++b) g.idx[pos[a * n1 + b]++] = (int32_t)t;
}

// Nitsche surface quadrature: 3 points per triangle (barycentric 2/3, 1/6, 1/6 and
// permutations, weight area/3), each owned by the leaf that contains it, fluid-outward normal
// n = -n_t, h_b = largest |(x_a - c_t).n_t| over the owner's Out corners, at least 0.01 h.
// Points in In elements are dropped.
void build_surface_points(Mesh& m) {
    static const double B[3][3] = {{2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0},
                                   {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0}};
    m.sq.clear();
    const TriHost& T = m.tri;
    for (int64_t t = 0; t < T.n; ++t) {
        const double* v = &T.v[9 * t];
        const double* nt = &T.nrm[3 * t];
        const double* ct = &T.cen[3 * t];
        for (int q = 0; q < 3; ++q) {
            double x[3];
            int64_t I[3];
            bool ok = true;
            for (int k = 0; k < 3; ++k) {
                x[k] = (B[q][0] * v[k] + B[q][1] * v[3 + k]) + B[q][2] * v[6 + k];
                double f = std::floor((x[k] - m.lo[k]) / m.scale);
                if (!(f >= 0.0 && f < (double)m.hiI[k])) { ok = false; break; }
                I[k] = (int64_t)f;
            }
            if (!ok) continue;
            int64_t e = find_leaf(m, I[0], I[1], I[2]);
            if (e < 0 || m.marker[e] == 1) continue;
            uint32_t s = octsize(m.lev[e]);
            double h = (double)s * m.scale;
            double hb = 0.0;
            for (int c = 0; c < 8; ++c) {
                if ((m.cflags[e] >> c) & 1) continue;
                double xa[3];
                for (int k = 0; k < 3; ++k) xa[k] = m.lo[k] + (double)(m.anc[3 * e + k] + (((c >> k) & 1) ? s : 0)) * m.scale;
                double dist = std::fabs((xa[0] - ct[0]) * nt[0] + (xa[1] - ct[1]) * nt[1] + (xa[2] - ct[2]) * nt[2]);
                if (dist > hb) hb = dist;
            }
            if (hb < 0.01 * h) hb = 0.01 * h;
            double rec[10] = {x[0], x[1], x[2], -nt[0], -nt[1], -nt[2], T.area[t] / 3.0, hb, (double)e, (double)t};
            m.sq.insert(m.sq.end(), rec, rec + 10);
        }
    }
}

// Strong rows: bits 0-2 velocity and bit 3 pressure prescribed on the box (u_inf on every face
// but the outlet x = hi; p = 0 on the outlet); bit 4: node touched by no active element.
void build_bc_flags(Mesh& m) {
    const int64_t nn = m.n_nodes(), ne = m.n_elem();
    m.bcflag.assign(nn, 0);
    std::vector<uint8_t> active(nn, 0);
    for (int64_t e = 0; e < ne; ++e) {
        if (m.marker[e] == 1) continue;
        for (int c = 0; c < 8; ++c) {
            int32_t id = m.conn[8 * e + c];
            if (id < nn) active[id] = 1;
            else {
                int64_t h = id - nn;
                for (int p = 0; p < m.hnp[h]; ++p) active[m.hpar[4 * h + p]] = 1;
            }
        }
    }
    for (int64_t n = 0; n < nn; ++n) {
        const uint32_t* X = &m.nijk[3 * n];
        uint8_t f = 0;
        bool outlet = (int64_t)X[0] == m.hiI[0];
        bool other = X[0] == 0 || X[1] == 0 || X[2] == 0 || (int64_t)X[1] == m.hiI[1] || (int64_t)X[2] == m.hiI[2];
        if (other) f |= 7;
        if (outlet) f |= 8;
        if (!active[n]) f |= 16;
        m.bcflag[n] = f;
    }
}

// Block pattern of the Jacobian assembled in 4 x 4 blocks, K = sum_e M_e^T k_e M_e (Algorithms 2
// and 4): block (i, j) is present when nodes i and j both enter one element through M_e -- as
// corners, or as parents of a hanging corner (Algorithm 3).  Every element counts, In elements
// too (their blocks stay zero), so the pattern depends on the octree alone and holds whatever the
// body does; every node is in some element, so every diagonal block is present.
void build_bsr_pattern(Mesh& m) {
    const int64_t ne = m.n_elem(), nn = m.n_nodes();
    // the distinct nodes that element e reaches through M_e (at most 8 x 4)
    auto nodes_of = [&](int64_t e, int32_t* out) {
        int k = 0;
        for (int c = 0; c < 8; ++c) {
            const int32_t id = m.conn[8 * e + c];
            if (id < nn) { out[k++] = id; continue; }
            const int64_t h = id - nn;
            for (int p = 0; p < m.hnp[h]; ++p) out[k++] = m.hpar[4 * h + p];
        }
        std::sort(out, out + k);
        return (int)(std::unique(out, out + k) - out);
    };
    // node -> elements
    std::vector<int64_t> off(nn + 1, 0);
    for (int64_t e = 0; e < ne; ++e) {
        int32_t buf[32];
        const int k = nodes_of(e, buf);
        for (int i = 0; i < k; ++i) ++off[buf[i] + 1];
    }
    for (int64_t i = 0; i < nn; ++i) off[i + 1] += off[i];
    std::vector<int32_t> elems(off[nn]);
    {
        std::vector<int64_t> pos(off.begin(), off.end() - 1);
        for (int64_t e = 0; e < ne; ++e) {
            int32_t buf[32];
            const int k = nodes_of(e, buf);
            for (int i = 0; i < k; ++i) elems[pos[buf[i]]++] = (int32_t)e;
        }
    }
    // row i = sorted union of the node sets of its elements; counted, then written
    auto row = [&](int64_t i, std::vector<int32_t>& tmp) {
        tmp.clear();
        for (int64_t q = off[i]; q < off[i + 1]; ++q) {
            int32_t buf[32];
            const int k = nodes_of(elems[q], buf);
            tmp.insert(tmp.end(), buf, buf + k);
        }
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    };
    m.bsr_ptr.assign(nn + 1, 0);
#pragma omp parallel
    {
        std::vector<int32_t> tmp;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t i = 0; i < nn; ++i) {
            row(i, tmp);
            m.bsr_ptr[i + 1] = (int64_t)tmp.size();
        }
    }
    for (int64_t i = 0; i < nn; ++i) m.bsr_ptr[i + 1] += m.bsr_ptr[i];
    m.bsr_idx.resize(m.bsr_ptr[nn]);
#pragma omp parallel
    {
        std::vector<int32_t> tmp;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t i = 0; i < nn; ++i) {
            row(i, tmp);
            std::copy(tmp.begin(), tmp.end(), m.bsr_idx.begin() + m.bsr_ptr[i]);
        }
    }
}

}  // namespace imga
