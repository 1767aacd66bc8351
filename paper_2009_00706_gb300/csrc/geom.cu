// Device geometry: in/out classification (Algorithm 6), element markers (Algorithm 5) and the
// adaptive sub-cell quadrature of Intercepted elements (Sec. "Adaptive Quadrature", Fig. GP).
//
// Compiled with -fmad=false: every decision (sign of (P - c_t).n_t, Moller-Trumbore barycentrics)
// is evaluated as a fixed sequence of IEEE float64 operations, so flags are reproducible bit for
// bit and independent of the launch configuration.
//
// Work decomposition
//  * markers: one thread per element.  An element that no triangle box meets cannot be crossed
//    by the surface, so one ray from its centre decides all its points; otherwise its 8 corners
//    are tested against its background triangles B_T(e), falling back to a ray when the normal
//    test is not unanimous.
//  * rays along +x only visit the triangles binned in the (y, z) grid cell of their origin (the
//    bins are widened far beyond rounding, so no hit or graze is missed); a ray that grazes an
//    edge or vertex is re-cast along +y, then +z, over all triangles.
//  * sub-cell quadrature: one thread per Intercepted element walks the sub-cell tree depth first
//    in Morton child order (count pass, prefix sum, write pass), so every element's point list
//    comes out in a fixed order.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>

#include "imga_internal.h"

namespace imga {

namespace {

constexpr double kGauss = 0.57735026918962576451;   // 1/sqrt(3)
constexpr double kGraze = 1e-12;

struct GeomView {
    const uint64_t* key;
    const uint32_t* anc;
    const uint8_t* lev;
    int64_t n_elem;
    double lo[3], scale;
    int64_t hiI[3];
    const double* tv;
    const double* tn;
    const double* tc;
    int64_t n_tri;
    const int32_t* bt_off;
    const int32_t* bt_idx;
    const int32_t* rg_off;
    const int32_t* rg_idx;
    int rg_ny, rg_nz;
    double rg_y0, rg_z0, rg_dy, rg_dz;
    const int8_t* marker;   // element markers (read by the classification of arbitrary points)
};

__device__ __forceinline__ uint64_t dpart1by2(uint64_t v) {
    v &= 0x1fffff;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ int64_t d_find_leaf(const GeomView& g, int64_t x, int64_t y, int64_t z) {
    if (x < 0 || y < 0 || z < 0 || x >= g.hiI[0] || y >= g.hiI[1] || z >= g.hiI[2]) return -1;
    uint64_t k = dpart1by2(x) | (dpart1by2(y) << 1) | (dpart1by2(z) << 2);
    int64_t lo = 0, hi = g.n_elem;   // first index with key > k
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (g.key[mid] <= k) lo = mid + 1; else hi = mid;
    }
    int64_t e = lo - 1;
    if (e < 0) return -1;
    uint32_t s = 1u << (kMaxDepth - g.lev[e]);
    const uint32_t* a = g.anc + 3 * e;
    if ((uint64_t)(x - a[0]) < s && (uint64_t)(y - a[1]) < s && (uint64_t)(z - a[2]) < s) return e;
    return -1;
}

// Moller-Trumbore against triangle t along axis `dir`; returns 1 hit, 0 miss, sets *graze
__device__ __forceinline__ int mt_hit(const GeomView& g, int64_t t, const double P[3], int dir, bool* graze) {
    double d[3] = {0.0, 0.0, 0.0};
    d[dir] = 1.0;
    const double* v = g.tv + 9 * t;
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) { e1[k] = v[3 + k] - v[k]; e2[k] = v[6 + k] - v[k]; }
    double pv[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
    double det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    double tv[3] = {P[0] - v[0], P[1] - v[1], P[2] - v[2]};
    double u = (tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2]) * inv;
    if (u < -kGraze || u > 1.0 + kGraze) return 0;
    double qv[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2], tv[0] * e1[1] - tv[1] * e1[0]};
    double w = (d[0] * qv[0] + d[1] * qv[1] + d[2] * qv[2]) * inv;
    if (w < -kGraze || u + w > 1.0 + kGraze) return 0;
    double tt = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * inv;
    if (tt <= 0.0) return 0;
    if (u < kGraze || w < kGraze || u + w > 1.0 - kGraze) *graze = true;
    return 1;
}

__device__ int ray_parity(const GeomView& g, const double P[3], int dir, bool* graze) {
    *graze = false;
    int count = 0;
    if (dir == 0) {
        int a = (int)floor((P[1] - g.rg_y0) / g.rg_dy);
        int b = (int)floor((P[2] - g.rg_z0) / g.rg_dz);
        if (g.rg_ny == 0 || a < 0 || b < 0 || a >= g.rg_ny || b >= g.rg_nz) return 0;
        int c = a * g.rg_nz + b;
        for (int32_t i = g.rg_off[c]; i < g.rg_off[c + 1]; ++i) count += mt_hit(g, g.rg_idx[i], P, 0, graze);
    } else {
        for (int64_t t = 0; t < g.n_tri; ++t) count += mt_hit(g, t, P, dir, graze);
    }
    return count & 1;
}

__device__ int ray_classify(const GeomView& g, const double P[3], unsigned long long* nrays) {
    atomicAdd(nrays, 1ull);
    int par[3];
    for (int dir = 0; dir < 3; ++dir) {
        bool gz;
        par[dir] = ray_parity(g, P, dir, &gz);
        if (!gz) return par[dir];
    }
    return (par[0] + par[1] + par[2]) >= 2 ? 1 : 0;
}

// normal test: 0 Out, 1 In, -1 undecided (Algorithm 6 with outward normals)
__device__ int normal_test(const GeomView& g, int64_t e, const double P[3], double tol) {
    int32_t b = g.bt_off[e], end = g.bt_off[e + 1];
    if (b == end) return -1;
    int npos = 0, nneg = 0;
    for (int32_t i = b; i < end; ++i) {
        const double* c = g.tc + 3 * g.bt_idx[i];
        const double* n = g.tn + 3 * g.bt_idx[i];
        double dx = P[0] - c[0], dy = P[1] - c[1], dz = P[2] - c[2];
        double s = dx * n[0] + dy * n[1] + dz * n[2];
        if (s > tol) ++npos;
        else if (s < -tol) ++nneg;
    }
    if (npos == end - b) return 0;
    if (nneg == end - b) return 1;
    return -1;
}

__device__ int is_in(const GeomView& g, int64_t e, const double P[3], unsigned long long* nrays) {
    double h = (double)(1u << (kMaxDepth - g.lev[e])) * g.scale;
    int r = normal_test(g, e, P, 1e-12 * h);
    if (r >= 0) return r;
    return ray_classify(g, P, nrays);
}

__global__ void markers_kernel(GeomView g, int8_t* marker, uint8_t* cflags, unsigned long long* nrays) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= g.n_elem) return;
    uint32_t s = 1u << (kMaxDepth - g.lev[e]);
    const uint32_t* a = g.anc + 3 * e;
    int flags = 0;
    if (g.bt_off[e] == g.bt_off[e + 1]) {
        double C[3];
        for (int k = 0; k < 3; ++k) C[k] = g.lo[k] + (double)(a[k] + s / 2) * g.scale;
        flags = ray_classify(g, C, nrays) ? 0xff : 0;
    } else {
        for (int c = 0; c < 8; ++c) {
            double P[3];
            for (int k = 0; k < 3; ++k) P[k] = g.lo[k] + (double)(a[k] + (((c >> k) & 1) ? s : 0)) * g.scale;
            if (is_in(g, e, P, nrays)) flags |= 1 << c;
        }
    }
    cflags[e] = (uint8_t)flags;
    marker[e] = (int8_t)(flags == 0xff ? 1 : flags == 0 ? 0 : 2);
}

// ------------------------------------------------------------------------------------------
// Warp-cooperative ray parity: the whole warp casts one point's ray (P uniform across the warp);
// lanes stride over the candidate triangles, the hit count is a warp sum and a graze anywhere is
// a graze of the ray.  Same result as ray_parity / ray_classify (the parity of an integer sum).
// ------------------------------------------------------------------------------------------
__device__ int warp_ray_parity(const GeomView& g, const double P[3], int dir, bool* graze) {
    const int lane = threadIdx.x & 31;
    int count = 0;
    bool gz = false;
    if (dir == 0) {
        const int a = (int)floor((P[1] - g.rg_y0) / g.rg_dy);
        const int b = (int)floor((P[2] - g.rg_z0) / g.rg_dz);
        if (g.rg_ny != 0 && a >= 0 && b >= 0 && a < g.rg_ny && b < g.rg_nz) {
            const int c = a * g.rg_nz + b;
            for (int32_t i = g.rg_off[c] + lane; i < g.rg_off[c + 1]; i += 32) count += mt_hit(g, g.rg_idx[i], P, 0, &gz);
        }
    } else {
        for (int64_t t = lane; t < g.n_tri; t += 32) count += mt_hit(g, t, P, dir, &gz);
    }
    const unsigned total = __reduce_add_sync(0xffffffffu, (unsigned)count);
    *graze = __any_sync(0xffffffffu, gz) != 0;
    return (int)(total & 1u);
}

__device__ int warp_ray_classify(const GeomView& g, const double P[3], unsigned long long* nrays) {
    if (nrays && (threadIdx.x & 31) == 0) atomicAdd(nrays, 1ull);
    int par[3];
    for (int dir = 0; dir < 3; ++dir) {
        bool gz;
        par[dir] = warp_ray_parity(g, P, dir, &gz);
        if (!gz) return par[dir];
    }
    return (par[0] + par[1] + par[2]) >= 2 ? 1 : 0;
}

// Lanes whose normal test was undecided (r < 0 and `want`) get the ray verdict, one point at a time
// for the whole warp.
__device__ void warp_resolve(const GeomView& g, bool want, const double P[3], int& r, unsigned long long* nrays) {
    unsigned need = __ballot_sync(0xffffffffu, want && r < 0);
    while (need) {
        const int src = __ffs(need) - 1;
        double Q[3];
        for (int k = 0; k < 3; ++k) Q[k] = __shfl_sync(0xffffffffu, P[k], src);
        const int v = warp_ray_classify(g, Q, nrays);
        if ((int)(threadIdx.x & 31) == src) r = v;
        need &= need - 1;
    }
}

struct Cell { uint8_t l; uint32_t i[3]; };

// Depth-first sub-cell walk of one Intercepted element (Fig. GP), a warp per element: lanes 0-7
// classify the 8 Gauss points of the cell on top of the stack (undecided ones by warp-cooperative
// rays); all In -> dropped, all Out -> kept, mixed -> split into 8 children (pushed by lanes 0-7 so
// child 0 is visited first) until lmax, where the Out points are kept.  Kept points are compacted
// in Gauss-point order.  pts == nullptr counts only.
constexpr int kWalkWarps = 4;
__device__ int64_t cut_walk_warp(const GeomView& g, int64_t e, int lmax, double* pts, float* ptsf,
                                 unsigned long long* nrays, Cell* st) {
    const int lane = threadIdx.x & 31, gp = lane & 7;
    const uint32_t* a = g.anc + 3 * e;
    const double h = (double)(1u << (kMaxDepth - g.lev[e])) * g.scale, hh = 0.5 * h;
    double x0[3];
    for (int k = 0; k < 3; ++k) x0[k] = g.lo[k] + (double)a[k] * g.scale;
    if (lane == 0) st[0] = Cell{0, {0, 0, 0}};
    __syncwarp();
    int sp = 1;
    int64_t n = 0;
    while (sp > 0) {
        const Cell c = st[--sp];
        __syncwarp();
        double xi[3], P[3];
        for (int k = 0; k < 3; ++k) {
            const double num = (double)(2 * c.i[k] + 1) + (((gp >> k) & 1) ? kGauss : -kGauss);
            xi[k] = num / (double)(1u << c.l) - 1.0;
            P[k] = x0[k] + (xi[k] + 1.0) * hh;
        }
        int r = lane < 8 ? normal_test(g, e, P, 1e-12 * h) : 0;
        warp_resolve(g, lane < 8, P, r, nrays);
        const unsigned in = __ballot_sync(0xffffffffu, lane < 8 && r == 1) & 0xffu;
        if (in == 0xffu) continue;
        if (in != 0u && c.l < lmax) {
            if (lane < 8)
                st[sp + 7 - lane] = Cell{(uint8_t)(c.l + 1), {2 * c.i[0] + (lane & 1), 2 * c.i[1] + ((lane >> 1) & 1),
                                                            2 * c.i[2] + ((lane >> 2) & 1)}};
            __syncwarp();
            sp += 8;
            continue;
        }
        const unsigned out = ~in & 0xffu;
        if (pts && lane < 8 && ((out >> lane) & 1u)) {
            const int64_t q = n + __popc(out & ((1u << lane) - 1u));
            const double w = 1.0 / (double)(1u << (3 * c.l));
            double* o = pts + 4 * q;
            o[0] = xi[0]; o[1] = xi[1]; o[2] = xi[2]; o[3] = w;
            float* of = ptsf + 4 * q;
            of[0] = (float)xi[0]; of[1] = (float)xi[1]; of[2] = (float)xi[2]; of[3] = (float)w;
        }
        n += __popc(out);
    }
    return n;
}

__global__ void __launch_bounds__(32 * kWalkWarps) cut_count_warp(GeomView g, const int32_t* cut_list, int64_t n_cut,
                                                                  int lmax, int64_t* count, unsigned long long* nrays) {
    __shared__ Cell st[kWalkWarps][8 * 6];
    const int w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kWalkWarps + w;
    if (i >= n_cut) return;
    const int64_t c = cut_walk_warp(g, cut_list[i], lmax, nullptr, nullptr, nrays, st[w]);
    if ((threadIdx.x & 31) == 0) count[i] = c;
}

__global__ void __launch_bounds__(32 * kWalkWarps) cut_write_warp(GeomView g, const int32_t* cut_list, int64_t n_cut,
                                                                  int lmax, const int64_t* off, double* pts, float* ptsf,
                                                                  unsigned long long* nrays) {
    __shared__ Cell st[kWalkWarps][8 * 6];
    const int w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kWalkWarps + w;
    if (i >= n_cut) return;
    cut_walk_warp(g, cut_list[i], lmax, pts + 4 * off[i], ptsf + 4 * off[i], nrays, st[w]);
}

// imga_classify with a lane per point and warp-cooperative rays for the undecided ones.  A point
// in an element whose box meets no triangle takes the element's stored marker: no triangle crosses
// the element, so all its points share the verdict that Algorithm 5 reached for it.  Points in
// elements with background triangles get the normal test of Algorithm 6, then a ray if it is
// undecided.  ray_only sends every point in the box to ray parity (the conventional test the
// paper compares against).  cnt[4] (may be null) accumulates, one atomic per warp and counter,
// the points settled by the marker, given the normal test, decided by it, and sent to a ray.
__global__ void classify_warp(GeomView g, const double* pts, int64_t n, uint8_t* flags, int ray_only,
                              unsigned long long* cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    double P[3] = {0.0, 0.0, 0.0};
    int r = 0;
    bool want = false, by_marker = false, tested = false;
    int64_t e = -1;
    if (valid) {
        for (int k = 0; k < 3; ++k) P[k] = pts[3 * i + k];
        bool inside = true;
        int64_t I[3];
        for (int k = 0; k < 3; ++k) {
            const double f = floor((P[k] - g.lo[k]) / g.scale);
            if (!(f >= 0.0 && f < (double)g.hiI[k])) inside = false;
            else I[k] = (int64_t)f;
        }
        if (inside) e = d_find_leaf(g, I[0], I[1], I[2]);
        if (e >= 0) {
            if (ray_only) {
                r = -1;
                want = true;
            } else if (g.bt_off[e] == g.bt_off[e + 1]) {
                r = g.marker[e] == 1 ? 1 : 0;
                by_marker = true;
            } else {
                const double h = (double)(1u << (kMaxDepth - g.lev[e])) * g.scale;
                r = normal_test(g, e, P, 1e-12 * h);
                tested = true;
                want = true;
            }
        }
    }
    if (cnt) {
        const unsigned full = 0xffffffffu;
        const unsigned bm = __ballot_sync(full, by_marker), bt = __ballot_sync(full, tested),
                       bd = __ballot_sync(full, tested && r >= 0), br = __ballot_sync(full, want && r < 0);
        if ((threadIdx.x & 31) == 0) {
            if (bm) atomicAdd(cnt + 0, (unsigned long long)__popc(bm));
            if (bt) atomicAdd(cnt + 1, (unsigned long long)__popc(bt));
            if (bd) atomicAdd(cnt + 2, (unsigned long long)__popc(bd));
            if (br) atomicAdd(cnt + 3, (unsigned long long)__popc(br));
        }
    }
    warp_resolve(g, want, P, r, nullptr);
    if (valid) flags[i] = (uint8_t)(e < 0 ? 0 : r);
}

GeomView view(const Mesh& m) {
    GeomView g;
    g.key = m.d.key;
    g.anc = m.d.anc;
    g.lev = m.d.lev;
    g.n_elem = m.n_elem();
    for (int k = 0; k < 3; ++k) { g.lo[k] = m.lo[k]; g.hiI[k] = m.hiI[k]; }
    g.scale = m.scale;
    g.tv = m.d.tv;
    g.tn = m.d.tn;
    g.tc = m.d.tc;
    g.n_tri = m.tri.n;
    g.bt_off = m.d.bt_off;
    g.bt_idx = m.d.bt_idx;
    g.rg_off = m.d.rg_off;
    g.rg_idx = m.d.rg_idx;
    g.rg_ny = m.grid.ny;
    g.rg_nz = m.grid.nz;
    g.rg_y0 = m.grid.y0;
    g.rg_z0 = m.grid.z0;
    g.rg_dy = m.grid.dy;
    g.rg_dz = m.grid.dz;
    g.marker = m.d.marker;
    return g;
}

template <class T>
bool upload(T** dst, const std::vector<T>& src, std::string& err, size_t min_elems = 1) {
    size_t n = std::max(src.size(), min_elems);
    if (cudaMalloc((void**)dst, n * sizeof(T)) != cudaSuccess) { err = "cudaMalloc failed"; return false; }
    if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        err = "cudaMemcpy failed";
        return false;
    }
    return true;
}

bool check(cudaError_t e, std::string& err, const char* what) {
    if (e == cudaSuccess) return true;
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
}

}  // namespace

bool device_upload_geometry(Mesh& m, std::string& err) {
    DeviceMesh& d = m.d;
    d.n_elem = m.n_elem();
    d.n_nodes = m.n_nodes();
    d.n_hang = m.n_hang();
    d.n_tri = m.tri.n;
    std::vector<int32_t> hp(m.hpar);
    if (!upload(&d.key, m.key, err) || !upload(&d.anc, m.anc, err) || !upload(&d.lev, m.lev, err) ||
        !upload(&d.conn, m.conn, err) || !upload(&d.hpar, hp, err) || !upload(&d.tv, m.tri.v, err) ||
        !upload(&d.tn, m.tri.nrm, err) || !upload(&d.tc, m.tri.cen, err) || !upload(&d.bt_off, m.bt_off, err) ||
        !upload(&d.bt_idx, m.bt_idx, err) || !upload(&d.rg_off, m.grid.off, err) || !upload(&d.rg_idx, m.grid.idx, err))
        return false;
    if (!check(cudaMalloc((void**)&d.marker, std::max<int64_t>(1, d.n_elem)), err, "cudaMalloc")) return false;
    if (!check(cudaMalloc((void**)&d.cflags, std::max<int64_t>(1, d.n_elem)), err, "cudaMalloc")) return false;
    if (!check(cudaMalloc((void**)&d.counters, kCounters * sizeof(unsigned long long)), err, "cudaMalloc")) return false;
    return check(cudaMemset(d.counters, 0, kCounters * sizeof(unsigned long long)), err, "cudaMemset");
}

// rays cast while building (markers, sub-cell quadrature): counters[kBuildRays]
static int64_t read_rays(const Mesh& m) {
    unsigned long long n = 0;
    cudaMemcpy(&n, m.d.counters + kBuildRays, sizeof(n), cudaMemcpyDeviceToHost);
    return (int64_t)n;
}

bool device_markers(Mesh& m, std::string& err) {
    const int64_t ne = m.n_elem();
    unsigned long long* nrays = m.d.counters + kBuildRays;
    cudaMemset(nrays, 0, sizeof(unsigned long long));
    GeomView g = view(m);
    if (ne > 0) markers_kernel<<<(unsigned)((ne + 127) / 128), 128>>>(g, m.d.marker, m.d.cflags, nrays);
    if (!check(cudaDeviceSynchronize(), err, "markers kernel")) return false;
    m.marker.resize(ne);
    m.cflags.resize(ne);
    if (!check(cudaMemcpy(m.marker.data(), m.d.marker, ne, cudaMemcpyDeviceToHost), err, "copy markers")) return false;
    if (!check(cudaMemcpy(m.cflags.data(), m.d.cflags, ne, cudaMemcpyDeviceToHost), err, "copy flags")) return false;
    m.n_rays = read_rays(m);
    m.out_list.clear();
    m.cut_list.clear();
    m.n_in = 0;
    for (int64_t e = 0; e < ne; ++e) {
        if (m.marker[e] == 0) m.out_list.push_back((int32_t)e);
        else if (m.marker[e] == 2) m.cut_list.push_back((int32_t)e);
        else ++m.n_in;
    }
    return true;
}

bool device_cut_quadrature(Mesh& m, std::string& err) {
    const int64_t nc = (int64_t)m.cut_list.size();
    GeomView g = view(m);
    if (!upload(&m.d.out_list, m.out_list, err) || !upload(&m.d.cut_list, m.cut_list, err)) return false;
    {
        std::vector<int32_t> oc(8 * m.out_list.size());
        std::vector<uint8_t> ol(m.out_list.size());
        for (size_t i = 0; i < m.out_list.size(); ++i) {
            for (int c = 0; c < 8; ++c) oc[8 * i + c] = m.conn[8 * (size_t)m.out_list[i] + c];
            ol[i] = m.lev[m.out_list[i]];
        }
        if (!upload(&m.d.out_conn, oc, err) || !upload(&m.d.out_lev, ol, err)) return false;
    }
    int64_t* cnt = nullptr;
    if (!check(cudaMalloc((void**)&cnt, (nc + 1) * sizeof(int64_t)), err, "cudaMalloc")) return false;
    unsigned long long* nrays = m.d.counters + kBuildRays;
    cudaMemset(nrays, 0, sizeof(unsigned long long));
    if (nc > 0) cut_count_warp<<<(unsigned)((nc + kWalkWarps - 1) / kWalkWarps), 32 * kWalkWarps>>>(g, m.d.cut_list, nc, m.lmax, cnt, nrays);
    if (!check(cudaDeviceSynchronize(), err, "cut count kernel")) { cudaFree(cnt); return false; }
    std::vector<int64_t> c(nc);
    if (nc) cudaMemcpy(c.data(), cnt, nc * sizeof(int64_t), cudaMemcpyDeviceToHost);
    m.cut_off.assign(nc + 1, 0);
    for (int64_t i = 0; i < nc; ++i) m.cut_off[i + 1] = m.cut_off[i] + c[i];
    const int64_t np = m.cut_off[nc];
    cudaFree(cnt);
    if (!upload(&m.d.cut_off, m.cut_off, err)) return false;
    if (!check(cudaMalloc((void**)&m.d.cut_pts, std::max<int64_t>(1, np) * 4 * sizeof(double)), err, "cudaMalloc")) return false;
    if (!check(cudaMalloc((void**)&m.d.cut_pts_f, std::max<int64_t>(1, np) * 4 * sizeof(float)), err, "cudaMalloc")) return false;
    if (nc > 0)
        cut_write_warp<<<(unsigned)((nc + kWalkWarps - 1) / kWalkWarps), 32 * kWalkWarps>>>(
            g, m.d.cut_list, nc, m.lmax, m.d.cut_off, m.d.cut_pts, m.d.cut_pts_f, nrays);
    if (!check(cudaDeviceSynchronize(), err, "cut write kernel")) return false;
    m.n_rays += read_rays(m) / 2;   // the write pass repeats the count pass's casts
    m.cut_pts.resize(4 * np);
    if (np) cudaMemcpy(m.cut_pts.data(), m.d.cut_pts, 4 * np * sizeof(double), cudaMemcpyDeviceToHost);
    m.cut_off_elem.assign(m.n_elem() + 1, 0);
    for (int64_t i = 0; i < nc; ++i) m.cut_off_elem[m.cut_list[i] + 1] = c[i];
    for (int64_t e = 0; e < m.n_elem(); ++e) m.cut_off_elem[e + 1] += m.cut_off_elem[e];
    return true;
}

// Deterministic scatter (o2n of Algorithm 2 in a fixed order).  The element kernels write their
// 8 x 4 contributions to slots: volume slots, one per Out element (out_list order) then one per
// Intercepted element (cut_list order), in the element precision; surface slots in float64, one per
// element of the dense surface bucket (sq_list order) then one per point of the sparse bucket.  The
// incidence list holds, for every independent node, the (slot, corner, weight) entries that reach it
// through M_e: weight 1 for a corner that is the node, 1/2 or 1/4 for a hanging corner whose parent
// it is; entries ordered by slot, so the node sums in the same order on every call.
// Entry encoding (32 bits): bits 0-2 corner, bits 3-4 weight (0: 1, 1: 1/2, 2: 1/4), bits 5-31
// global slot (volume slots first; at most 2^27 slots).
bool build_incidence(Mesh& m, const std::vector<int32_t>& sq_el, const std::vector<int32_t>& dense, std::string& err) {
    const int64_t nn = m.n_nodes(), nv = (int64_t)(m.out_list.size() + m.cut_list.size());
    const int64_t ns = m.n_sq_elem + m.n_sq_sparse;
    m.n_vslots = nv;
    m.n_sslots = ns;
    if (nv + ns >= ((int64_t)1 << 27)) { err = "too many element slots for the incidence list (2^27)"; return false; }
    auto elem_of = [&](int64_t s) -> int64_t {
        if (s < (int64_t)m.out_list.size()) return m.out_list[s];
        if (s < nv) return m.cut_list[s - (int64_t)m.out_list.size()];
        if (s < nv + m.n_sq_elem) return dense[s - nv];
        return sq_el[s - nv - m.n_sq_elem];
    };
    std::vector<int64_t> ptr(nn + 1, 0);
    auto visit = [&](auto&& fn) {
        for (int64_t s = 0; s < nv + ns; ++s) {
            const int64_t e = elem_of(s);
            for (int c = 0; c < 8; ++c) {
                const int32_t id = m.conn[8 * e + c];
                if (id < nn) { fn(id, (uint32_t)(s << 5) | (uint32_t)c); continue; }
                const int64_t h = id - nn;
                const int np = m.hnp[h];
                const uint32_t wc = np == 4 ? 2u : 1u;
                for (int q = 0; q < np; ++q) fn(m.hpar[4 * h + q], (uint32_t)(s << 5) | (wc << 3) | (uint32_t)c);
            }
        }
    };
    visit([&](int64_t node, uint32_t) { ptr[node + 1] += 1; });
    for (int64_t i = 0; i < nn; ++i) ptr[i + 1] += ptr[i];
    std::vector<uint32_t> inc(std::max<int64_t>(1, ptr[nn]));
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    visit([&](int64_t node, uint32_t code) { inc[fill[node]++] = code; });
    // stored as a fixed head of kIncHead entries per node (sentinel-padded: one aligned 32-byte load,
    // no offset to fetch first) and the rest of each list in CSR form; the list order is kept
    std::vector<uint32_t> head((size_t)std::max<int64_t>(1, nn) * kIncHead, kIncNone);
    std::vector<int64_t> optr(nn + 1, 0);
    for (int64_t i = 0; i < nn; ++i) optr[i + 1] = optr[i] + std::max<int64_t>(0, ptr[i + 1] - ptr[i] - kIncHead);
    std::vector<uint32_t> oinc(std::max<int64_t>(1, optr[nn]));
    for (int64_t i = 0; i < nn; ++i)
        for (int64_t q = ptr[i], k = 0; q < ptr[i + 1]; ++q, ++k) {
            if (k < kIncHead) head[(size_t)i * kIncHead + k] = inc[q];
            else oinc[optr[i] + k - kIncHead] = inc[q];
        }
    const size_t slot_bytes = (size_t)std::max<int64_t>(1, nv) * 32 * sizeof(double);
    if (!upload(&m.d.inc_head, head, err) || !upload(&m.d.inc_ptr, optr, err) || !upload(&m.d.inc, oinc, err)) return false;
    if (!check(cudaMalloc((void**)&m.d.sv, slot_bytes), err, "cudaMalloc") ||
        !check(cudaMalloc((void**)&m.d.ss, (size_t)std::max<int64_t>(1, ns) * 32 * sizeof(double)), err, "cudaMalloc"))
        return false;
    return true;
}

// surface points (sorted by owning element, reference coordinates) and boundary flags
bool device_upload_quadrature(Mesh& m, std::string& err) {
    const int64_t ns = (int64_t)m.sq.size() / 10;
    std::vector<int64_t> order(ns);
    for (int64_t i = 0; i < ns; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return m.sq[10 * a + 8] < m.sq[10 * b + 8]; });
    // two buckets: points of elements hosting fewer than kNitscheDenseMin points first (one thread per
    // point), then the runs of the other elements (one warp per element)
    {
        std::vector<int64_t> sparse, dense;
        for (int64_t j = 0; j < ns;) {
            int64_t k = j;
            while (k < ns && m.sq[10 * order[k] + 8] == m.sq[10 * order[j] + 8]) ++k;
            auto& dst = (k - j) >= kNitscheDenseMin ? dense : sparse;
            dst.insert(dst.end(), order.begin() + j, order.begin() + k);
            j = k;
        }
        m.n_sq_sparse = (int64_t)sparse.size();
        sparse.insert(sparse.end(), dense.begin(), dense.end());
        order.swap(sparse);
    }
    std::vector<int32_t> el(ns), src(ns);
    std::vector<double> xr(3 * ns), nr(3 * ns), w(ns), tb(ns);
    for (int64_t j = 0; j < ns; ++j) {
        const double* r = &m.sq[10 * order[j]];
        src[j] = (int32_t)order[j];
        int64_t e = (int64_t)r[8];
        el[j] = (int32_t)e;
        double h = (double)(1u << (kMaxDepth - m.lev[e])) * m.scale;
        for (int k = 0; k < 3; ++k) {
            double x0 = m.lo[k] + (double)m.anc[3 * e + k] * m.scale;
            xr[3 * j + k] = (r[k] - x0) / (0.5 * h) - 1.0;
            nr[3 * j + k] = r[3 + k];
        }
        w[j] = r[6];
        tb[j] = 1.0 / r[7];
    }
    // runs of points per host element in the dense bucket
    std::vector<int32_t> sl;
    std::vector<int64_t> so;
    for (int64_t j = m.n_sq_sparse; j < ns; ++j)
        if (j == m.n_sq_sparse || el[j] != el[j - 1]) { sl.push_back(el[j]); so.push_back(j); }
    so.push_back(ns);
    m.n_sq_elem = (int64_t)sl.size();
    m.sq_off_h = so;
    m.sq_hosts.assign(el.begin(), el.end());
    std::sort(m.sq_hosts.begin(), m.sq_hosts.end());
    m.sq_hosts.erase(std::unique(m.sq_hosts.begin(), m.sq_hosts.end()), m.sq_hosts.end());
    // float64 penalty matrices, one per run of points of one element in device order (dense elements:
    // their slot; sparse elements: the slot of their first point)
    std::vector<int64_t> pq, pslot;
    std::vector<double> pen;
    m.pen_elem.clear();
    for (int64_t j = 0; j < ns;) {
        int64_t k = j;
        while (k < ns && el[k] == el[j]) ++k;
        m.pen_elem.push_back(el[j]);
        pq.push_back(j);
        pslot.push_back(j >= m.n_sq_sparse ? (int64_t)(std::lower_bound(so.begin(), so.end() - 1, j) - so.begin())
                                           : m.n_sq_elem + j);
        double P[36] = {0.0};
        for (int64_t q = j; q < k; ++q) {
            double fm[3], fp[3], phi[8];
            for (int a = 0; a < 3; ++a) { fm[a] = 0.5 * (1.0 - xr[3 * q + a]); fp[a] = 0.5 * (1.0 + xr[3 * q + a]); }
            for (int c = 0; c < 8; ++c) phi[c] = ((c & 1) ? fp[0] : fm[0]) * ((c & 2) ? fp[1] : fm[1]) * ((c & 4) ? fp[2] : fm[2]);
            const double wq = w[q] * tb[q];
            int t = 0;
            for (int a = 0; a < 8; ++a)
                for (int b = a; b < 8; ++b, ++t) P[t] += wq * phi[a] * phi[b];
        }
        pen.insert(pen.end(), P, P + 36);
        j = k;
    }
    pq.push_back(ns);
    if (!upload(&m.d.sq_elem, el, err) || !upload(&m.d.sq_x, xr, err) || !upload(&m.d.sq_n, nr, err) ||
        !upload(&m.d.sq_w, w, err) || !upload(&m.d.sq_taub, tb, err) || !upload(&m.d.sq_list, sl, err) ||
        !upload(&m.d.sq_off, so, err) || !upload(&m.d.sq_src, src, err) || !upload(&m.d.sq_hosts, m.sq_hosts, err) ||
        !upload(&m.d.pen_elem, m.pen_elem, err) || !upload(&m.d.pen_q, pq, err) || !upload(&m.d.pen_slot, pslot, err) ||
        !upload(&m.d.pen, pen, err) ||
        !upload(&m.d.bcflag, m.bcflag, err))
        return false;
    if (!build_incidence(m, el, sl, err)) return false;
    const size_t next = (size_t)(m.n_nodes() + m.n_hang());
    if (!check(cudaMalloc((void**)&m.d.slot, std::max<int64_t>(1, m.n_elem()) * sizeof(int32_t)), err, "cudaMalloc")) return false;
    if (!check(cudaMalloc((void**)&m.d.nd_f, std::max<size_t>(1, 24 * next) * sizeof(float)), err, "cudaMalloc") ||
        !check(cudaMalloc((void**)&m.d.nd_d, std::max<size_t>(1, 24 * next) * sizeof(double)), err, "cudaMalloc"))
        return false;
    return true;
}

// the arrays a batched mesh (several problems merged) needs for residual / J v / Jacobians
bool device_upload_batch(Mesh& m, std::string& err) {
    DeviceMesh& d = m.d;
    d.n_elem = m.n_elem();
    d.n_nodes = m.n_nodes();
    d.n_hang = m.n_hang();
    d.n_tri = 0;
    std::vector<int32_t> hp(m.hpar);
    std::vector<int32_t> oc(8 * m.out_list.size());
    std::vector<uint8_t> ol(m.out_list.size());
    std::vector<uint16_t> op(m.out_list.size());
    for (size_t i = 0; i < m.out_list.size(); ++i) {
        for (int c = 0; c < 8; ++c) oc[8 * i + c] = m.conn[8 * (size_t)m.out_list[i] + c];
        ol[i] = m.lev[m.out_list[i]];
        op[i] = m.eprob[m.out_list[i]];
    }
    std::vector<float> ptsf(m.cut_pts.begin(), m.cut_pts.end());
    std::vector<float> muf(m.pmu.begin(), m.pmu.end());
    if (!upload(&d.lev, m.lev, err) || !upload(&d.conn, m.conn, err) || !upload(&d.hpar, hp, err) ||
        !upload(&d.marker, m.marker, err) || !upload(&d.cflags, m.cflags, err) || !upload(&d.out_list, m.out_list, err) ||
        !upload(&d.out_conn, oc, err) || !upload(&d.out_lev, ol, err) || !upload(&d.out_prob, op, err) ||
        !upload(&d.cut_list, m.cut_list, err) || !upload(&d.cut_off, m.cut_off, err) ||
        !upload(&d.cut_pts, m.cut_pts, err) || !upload(&d.cut_pts_f, ptsf, err) || !upload(&d.eprob, m.eprob, err) ||
        !upload(&d.pmu, m.pmu, err) || !upload(&d.pmuf, muf, err))
        return false;
    return device_upload_quadrature(m, err);
}

// the arrays a part of a partitioned mesh needs for residual / J v (its own elements and nodes)
bool device_upload_part(Mesh& m, std::string& err) {
    DeviceMesh& d = m.d;
    d.n_elem = m.n_elem();
    d.n_nodes = m.n_nodes();
    d.n_hang = m.n_hang();
    d.n_tri = 0;
    std::vector<int32_t> oc(8 * m.out_list.size());
    std::vector<uint8_t> ol(m.out_list.size());
    for (size_t i = 0; i < m.out_list.size(); ++i) {
        for (int c = 0; c < 8; ++c) oc[8 * i + c] = m.conn[8 * (size_t)m.out_list[i] + c];
        ol[i] = m.lev[m.out_list[i]];
    }
    std::vector<float> ptsf(m.cut_pts.begin(), m.cut_pts.end());
    if (!upload(&d.lev, m.lev, err) || !upload(&d.conn, m.conn, err) || !upload(&d.hpar, m.hpar, err) ||
        !upload(&d.marker, m.marker, err) || !upload(&d.cflags, m.cflags, err) || !upload(&d.out_list, m.out_list, err) ||
        !upload(&d.out_conn, oc, err) || !upload(&d.out_lev, ol, err) || !upload(&d.cut_list, m.cut_list, err) ||
        !upload(&d.cut_off, m.cut_off, err) || !upload(&d.cut_pts, m.cut_pts, err) || !upload(&d.cut_pts_f, ptsf, err))
        return false;
    return device_upload_quadrature(m, err);
}

int device_classify(const Mesh& m, const double* pts, int64_t n, uint8_t* flags, void* stream) {
    if (n <= 0) return 0;
    GeomView g = view(m);
    classify_warp<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(g, pts, n, flags, m.classify_ray_only ? 1 : 0,
                                                                                 m.d.counters);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

void device_free(Mesh& m) {
    DeviceMesh& d = m.d;
    void* ptrs[] = {d.key, d.anc, d.lev, d.conn, d.hpar, d.tv, d.tn, d.tc, d.bt_off, d.bt_idx, d.rg_off, d.rg_idx,
                    d.marker, d.cflags, d.out_list, d.out_conn, d.out_lev, d.out_prob, d.eprob, d.pmu, d.pmuf, d.cut_list, d.cut_off, d.cut_pts, d.cut_pts_f, d.cut_order, d.sq_elem, d.sq_x,
                    d.sq_n, d.sq_w, d.sq_taub, d.sq_src, d.sq_hosts, d.pen_elem, d.pen_q, d.pen_slot, d.pen, d.inc_head, d.inc_ptr, d.inc, d.sv, d.ss, d.sq_list, d.sq_off, d.bcflag, d.bcmask_user, d.bcval_user, m.scratch, d.nd_f, d.nd_d, d.slot,
                    d.counters, d.fq_items, d.fq_cnt};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    d = DeviceMesh();
    m.scratch = nullptr;
}

}  // namespace imga
