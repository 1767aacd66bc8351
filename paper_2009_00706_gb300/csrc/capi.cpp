// C ABI of the imga library: argument checks, mesh life cycle, dispatch to the device stages.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "imga_internal.h"

struct imga_mesh_s {
    imga::Mesh m;
};
struct imga_partition_s {
    imga::Partition* P = nullptr;
    const imga::Mesh* mesh = nullptr;
};
struct imga_mlp_s {
    imga::Mlp* M = nullptr;
    int nin = 0, nout = 0, device = 0;
};

namespace imga {
thread_local std::string g_last_error;
void set_error(const std::string& s) { g_last_error = s; }
}  // namespace imga

using imga::set_error;

namespace {

double ms_since(std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
}

imga_status fail(imga_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

imga_status cuda_status(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return IMGA_OK;
    return fail(IMGA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool physics_ok(const imga_physics* p) {
    return p && p->rho > 0.0 && p->mu >= 0.0 && p->dt > 0.0 && p->time_scheme >= 0 && p->time_scheme <= 2 &&
           std::isfinite(p->rho) && std::isfinite(p->mu) && std::isfinite(p->dt) && p->C_b >= 0.0 && p->C_I >= 0.0;
}

}  // namespace

static imga_status build_mesh_impl(const double* tri, int64_t n_tri, const imga_mesh_params* P, int device,
                                   imga_mesh* out, imga_mesh_s*& hold) {
    if (!out || !P) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n_tri < 0 || (n_tri > 0 && !tri)) return fail(IMGA_ERR_INVALID_ARG, "bad triangle array");
    if (P->base_level < 0 || P->base_level > imga::kMaxLevel - 2) return fail(IMGA_ERR_INVALID_ARG, "base_level out of range");
    if (P->quad_max_split < 0 || P->quad_max_split > 4) return fail(IMGA_ERR_INVALID_ARG, "quad_max_split out of range (0..4)");
    if (P->n_regions < 0 || (P->n_regions > 0 && !P->regions)) return fail(IMGA_ERR_INVALID_ARG, "bad region array");
    for (int r = 0; r < P->n_regions; ++r)
        if (P->regions[r].level < 0 || P->regions[r].level > imga::kMaxLevel - 2 || P->regions[r].kind < 0 ||
            P->regions[r].kind > 2)
            return fail(IMGA_ERR_INVALID_ARG, "region level or kind out of range");
    const bool host_only = device < 0;
    if (!host_only && cudaSetDevice(device) != cudaSuccess) return cuda_status("cudaSetDevice");
    imga_mesh_s* h = new (std::nothrow) imga_mesh_s();
    if (!h) return fail(IMGA_ERR_OOM, "host allocation failed");
    hold = h;
    imga::Mesh& m = h->m;
    m.device = device;
    if (!host_only) cudaDeviceGetAttribute(&m.n_sm, cudaDevAttrMultiProcessorCount, device);
    double L = 0.0;
    for (int k = 0; k < 3; ++k) {
        m.lo[k] = P->lo[k];
        m.hi[k] = P->hi[k];
        if (!(P->hi[k] > P->lo[k])) { delete h; hold = nullptr; return fail(IMGA_ERR_INVALID_ARG, "empty box"); }
        L = std::max(L, P->hi[k] - P->lo[k]);
    }
    m.scale = L / (double)(1u << imga::kMaxDepth);
    m.base_level = P->base_level;
    m.lmax = P->quad_max_split;
    m.regions.assign(P->regions, P->regions + P->n_regions);
    for (int k = 0; k < 3; ++k) {
        double f = (P->hi[k] - P->lo[k]) / m.scale;
        m.hiI[k] = (int64_t)std::llround(f);
        int64_t cell = 1ll << (imga::kMaxDepth - P->base_level);
        if (std::fabs(f - (double)m.hiI[k]) > 1e-6 || m.hiI[k] % cell != 0) {
            delete h; hold = nullptr;
            return fail(IMGA_ERR_INVALID_ARG, "box edge " + std::to_string(k) + " is not a whole number of base-level cells");
        }
    }
    std::string err;
    auto t0 = std::chrono::steady_clock::now();
    if (!imga::build_octree(m, err) || !imga::build_nodes(m, err)) { delete h; hold = nullptr; return fail(IMGA_ERR_INVALID_ARG, err); }
    m.setup_ms[0] = ms_since(t0);
    t0 = std::chrono::steady_clock::now();
    if (!imga::build_triangles(m, tri, n_tri, err)) { delete h; hold = nullptr; return fail(IMGA_ERR_SURFACE, err); }
    imga::build_background(m);
    imga::build_ray_grid(m);
    m.setup_ms[1] = ms_since(t0);
    if (host_only) {
        m.host_only = true;
        *out = h;
        return IMGA_OK;
    }
    t0 = std::chrono::steady_clock::now();
    if (!imga::device_upload_geometry(m, err) || !imga::device_markers(m, err) || !imga::device_cut_quadrature(m, err)) {
        imga::device_free(m);
        delete h; hold = nullptr;
        return fail(IMGA_ERR_CUDA, err);
    }
    m.setup_ms[2] = ms_since(t0);
    t0 = std::chrono::steady_clock::now();
    imga::build_surface_points(m);
    imga::build_bc_flags(m);
    if (!imga::device_upload_quadrature(m, err)) { imga::device_free(m); delete h; hold = nullptr; return fail(IMGA_ERR_CUDA, err); }
    if (cudaDeviceSynchronize() != cudaSuccess) { imga::device_free(m); delete h; hold = nullptr; return cuda_status("build"); }
    m.setup_ms[3] = ms_since(t0);
    *out = h;
    return IMGA_OK;
}

static imga_status build_batch_impl(const imga_problem* probs, int n, int device, imga_mesh* out,
                                   std::vector<imga_mesh>& parts, imga_mesh_s*& hold) {
    if (!out || !probs || n < 1 || n > 65535) return fail(IMGA_ERR_INVALID_ARG, "bad problem list");
    *out = nullptr;
    if (device < 0) return fail(IMGA_ERR_INVALID_ARG, "batched meshes need a device");
    parts.assign(n, nullptr);
    std::vector<double> mu(n);
    auto cleanup = [&]() { for (imga_mesh& q : parts) { imga_destroy_mesh(q); q = nullptr; } };
    for (int p = 0; p < n; ++p) {
        if (!(probs[p].mu >= 0.0)) { cleanup(); return fail(IMGA_ERR_INVALID_ARG, "bad problem viscosity"); }
        imga_status st = imga_build_mesh(probs[p].tri_xyz_host, probs[p].n_tri, &probs[p].params, device, &parts[p]);
        if (st != IMGA_OK) { std::string e = imga::g_last_error; cleanup(); return fail(st, "problem " + std::to_string(p) + ": " + e); }
        mu[p] = probs[p].mu;
    }
    imga_mesh_s* h = new (std::nothrow) imga_mesh_s();
    if (!h) { cleanup(); return fail(IMGA_ERR_OOM, "host allocation failed"); }
    hold = h;
    imga::Mesh& m = h->m;
    m.device = device;
    m.batched = true;
    m.n_sm = parts[0]->m.n_sm;
    std::vector<const imga::Mesh*> pm;
    for (imga_mesh q : parts) pm.push_back(&q->m);
    std::string err;
    bool ok = imga::merge_meshes(m, pm, mu, err);
    for (int k = 0; k < 4; ++k)
        for (imga_mesh q : parts) m.setup_ms[k] += q->m.setup_ms[k];
    cleanup();
    if (!ok || cudaDeviceSynchronize() != cudaSuccess) { imga::device_free(m); delete h; hold = nullptr; return fail(IMGA_ERR_CUDA, err.empty() ? "batch upload" : err); }
    *out = h;
    return IMGA_OK;
}

// An exception (a host allocation failing inside the builders) must not cross the C ABI: free
// what was built so far and report it.
static imga_status abandon(imga_mesh_s*& hold, imga_mesh* out, const std::exception& e) {
    if (hold) {
        if (hold->m.device >= 0) imga::device_free(hold->m);
        delete hold;
        hold = nullptr;
    }
    if (out) *out = nullptr;
    if (dynamic_cast<const std::bad_alloc*>(&e)) return fail(IMGA_ERR_OOM, "host allocation failed while building the mesh");
    return fail(IMGA_ERR_INVALID_ARG, std::string("mesh build failed: ") + e.what());
}

extern "C" {

const char* imga_last_error(void) { return imga::g_last_error.c_str(); }

imga_status imga_build_mesh(const double* tri, int64_t n_tri, const imga_mesh_params* P, int device, imga_mesh* out) {
    imga_mesh_s* hold = nullptr;
    try {
        return build_mesh_impl(tri, n_tri, P, device, out, hold);
    } catch (const std::exception& e) {
        return abandon(hold, out, e);
    }
}

imga_status imga_build_mesh_batch(const imga_problem* probs, int n, int device, imga_mesh* out) {
    std::vector<imga_mesh> parts;
    imga_mesh_s* hold = nullptr;
    try {
        return build_batch_impl(probs, n, device, out, parts, hold);
    } catch (const std::exception& e) {
        for (imga_mesh& q : parts) { imga_destroy_mesh(q); q = nullptr; }
        return abandon(hold, out, e);
    }
}

imga_status imga_mesh_problems(imga_mesh h, int* n_problems, int64_t* elem_off, int64_t* node_off) {
    if (!h) return fail(IMGA_ERR_INVALID_ARG, "null mesh");
    const imga::Mesh& m = h->m;
    const int np = m.batched ? (int)m.prob_elem_off.size() : 1;
    if (n_problems) *n_problems = np;
    for (int p = 0; p <= np; ++p) {
        if (elem_off) elem_off[p] = !m.batched ? (p ? m.n_elem() : 0) : (p < np ? m.prob_elem_off[p] : m.n_elem());
        if (node_off) node_off[p] = !m.batched ? (p ? m.n_nodes() : 0) : (p < np ? m.prob_node_off[p] : m.n_nodes());
    }
    return IMGA_OK;
}

void imga_destroy_mesh(imga_mesh h) {
    if (!h) return;
    if (h->m.host_only) { delete h; return; }
    imga::profile_reset(h->m);
    imga::solver_free(h->m);
    imga::multilevel_free(h->m);
    if (h->m.force_part) cudaFree(h->m.force_part);
    imga::graphs_free(h->m);
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->m.device);
    imga::device_free(h->m);
    cudaSetDevice(cur);
    delete h;
}

imga_status imga_mesh_get_info(imga_mesh h, imga_mesh_info* info) {
    if (!h || !info) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    const imga::Mesh& m = h->m;
    std::memset(info, 0, sizeof(*info));
    info->n_elem = m.n_elem();
    info->n_nodes = m.n_nodes();
    info->n_hanging = m.n_hang();
    info->n_out = (int64_t)m.out_list.size();
    info->n_cut = (int64_t)m.cut_list.size();
    info->n_in = m.n_in;
    info->n_cut_points = m.cut_off.empty() ? 0 : m.cut_off.back();
    info->n_surface_points = (int64_t)m.sq.size() / 10;
    info->n_tri = m.tri.n;
    info->n_bt = (int64_t)m.bt_idx.size();
    info->n_rays = m.n_rays;
    for (int k = 0; k < 3; ++k) info->hi_int[k] = m.hiI[k];
    info->scale = m.scale;
    for (int k = 0; k < 4; ++k) info->setup_ms[k] = m.setup_ms[k];
    return IMGA_OK;
}

imga_status imga_mesh_export(imga_mesh h, uint32_t* anchors, uint8_t* levels, int32_t* conn, uint32_t* node_ijk,
                             int32_t* hang_parents, int8_t* hang_np) {
    if (!h) return fail(IMGA_ERR_INVALID_ARG, "null mesh");
    const imga::Mesh& m = h->m;
    if (anchors) std::memcpy(anchors, m.anc.data(), m.anc.size() * sizeof(uint32_t));
    if (levels) std::memcpy(levels, m.lev.data(), m.lev.size());
    if (conn) std::memcpy(conn, m.conn.data(), m.conn.size() * sizeof(int32_t));
    if (node_ijk) std::memcpy(node_ijk, m.nijk.data(), m.nijk.size() * sizeof(uint32_t));
    if (hang_parents) std::memcpy(hang_parents, m.hpar.data(), m.hpar.size() * sizeof(int32_t));
    if (hang_np) std::memcpy(hang_np, m.hnp.data(), m.hnp.size());
    return IMGA_OK;
}

imga_status imga_export_markers(imga_mesh h, int8_t* marker, uint8_t* cflags) {
    if (!h) return fail(IMGA_ERR_INVALID_ARG, "null mesh");
    if (marker) std::memcpy(marker, h->m.marker.data(), h->m.marker.size());
    if (cflags) std::memcpy(cflags, h->m.cflags.data(), h->m.cflags.size());
    return IMGA_OK;
}

imga_status imga_export_cut_points(imga_mesh h, int64_t* offsets, double* points) {
    if (!h) return fail(IMGA_ERR_INVALID_ARG, "null mesh");
    const imga::Mesh& m = h->m;
    if (offsets) std::memcpy(offsets, m.cut_off_elem.data(), m.cut_off_elem.size() * sizeof(int64_t));
    if (points) {
        // cut_pts is in cut-list order, which is element order
        std::memcpy(points, m.cut_pts.data(), m.cut_pts.size() * sizeof(double));
    }
    return IMGA_OK;
}

imga_status imga_export_background(imga_mesh h, int32_t* offsets, int32_t* tri_ids) {
    if (!h) return fail(IMGA_ERR_INVALID_ARG, "null mesh");
    if (offsets) std::memcpy(offsets, h->m.bt_off.data(), h->m.bt_off.size() * sizeof(int32_t));
    if (tri_ids) std::memcpy(tri_ids, h->m.bt_idx.data(), h->m.bt_idx.size() * sizeof(int32_t));
    return IMGA_OK;
}

imga_status imga_export_surface_points(imga_mesh h, double* out) {
    if (!h || !out) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    std::memcpy(out, h->m.sq.data(), h->m.sq.size() * sizeof(double));
    return IMGA_OK;
}

imga_status imga_classify(imga_mesh h, const double* pts, int64_t n, uint8_t* flags, void* stream) {
    if (!h || n < 0 || (n > 0 && (!pts || !flags))) return fail(IMGA_ERR_INVALID_ARG, "bad argument");
    if (h->m.host_only) return fail(IMGA_ERR_INVALID_ARG, "mesh was built host-only (device < 0)");
    if (h->m.batched) return fail(IMGA_ERR_INVALID_ARG, "classify a point against one of the problems' own meshes");
    if (imga::device_classify(h->m, pts, n, flags, stream)) return cuda_status("classify");
    return IMGA_OK;
}

imga_status imga_node_coords(imga_mesh h, double* xyz, void* stream) {
    if (!h || !xyz) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    const imga::Mesh& m = h->m;
    const int64_t nn = m.n_nodes();
    std::vector<double> c;
    try {
        c.resize(3 * nn);
    } catch (const std::bad_alloc&) {
        return fail(IMGA_ERR_OOM, "node coordinates: host allocation failed");
    }
    for (int64_t i = 0; i < nn; ++i)
        for (int k = 0; k < 3; ++k) c[3 * i + k] = m.lo[k] + (double)m.nijk[3 * i + k] * m.scale;
    if (m.host_only) {
        std::copy(c.begin(), c.end(), xyz);
        return IMGA_OK;
    }
    if (nn == 0) return IMGA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(xyz, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);     // the host buffer must outlive the copy
    if (e != cudaSuccess) return fail(IMGA_ERR_CUDA, std::string("node coordinates: ") + cudaGetErrorString(e));
    return IMGA_OK;
}

imga_status imga_bsr_pattern(imga_mesh h, int64_t* n_blocks, int64_t* indptr, int32_t* indices) {
    if (!h || !n_blocks) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    imga::Mesh& m = h->m;
    if (m.bsr_ptr.size() != (size_t)m.n_nodes() + 1) {
        try {
            imga::build_bsr_pattern(m);
        } catch (const std::bad_alloc&) {
            m.bsr_ptr.clear();
            m.bsr_idx.clear();
            return fail(IMGA_ERR_OOM, "block pattern: host allocation failed");
        }
    }
    *n_blocks = (int64_t)m.bsr_idx.size();
    if (indptr) std::copy(m.bsr_ptr.begin(), m.bsr_ptr.end(), indptr);
    if (indices) std::copy(m.bsr_idx.begin(), m.bsr_idx.end(), indices);
    return IMGA_OK;
}

imga_status imga_classify_counts(imga_mesh h, int64_t* counts, int reset) {
    if (!h || !counts) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    if (h->m.host_only || h->m.batched || !h->m.d.counters)
        return fail(IMGA_ERR_INVALID_ARG, "mesh has no classification counts (host-only or batched)");
    int cur = 0;
    cudaGetDevice(&cur);
    unsigned long long c[imga::kClassifyCounts] = {};
    cudaError_t e = cudaSetDevice(h->m.device);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c, h->m.d.counters, sizeof(c), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset) e = cudaMemset(h->m.d.counters, 0, sizeof(c));
    if (e == cudaSuccess && reset) e = cudaDeviceSynchronize();
    cudaSetDevice(cur);
    if (e != cudaSuccess) return fail(IMGA_ERR_CUDA, std::string("classify counts: ") + cudaGetErrorString(e));
    for (int k = 0; k < imga::kClassifyCounts; ++k) counts[k] = (int64_t)c[k];
    return IMGA_OK;
}

static imga_status apply(imga_mesh h, const double* u, const double* up, const double* up2, const double* f,
                         const imga_physics* ph, int precision, const double* v, double* out, void* stream) {
    if (!h || !u || !up || !out) return fail(IMGA_ERR_INVALID_ARG, "null vector");
    if (h->m.host_only) return fail(IMGA_ERR_INVALID_ARG, "mesh was built host-only (device < 0)");
    if (!physics_ok(ph)) return fail(IMGA_ERR_INVALID_ARG, "bad physics parameters");
    if (ph->time_scheme == 2 && !up2) return fail(IMGA_ERR_INVALID_ARG, "BDF2 needs u_prev2");
    if (precision != 0 && precision != 1) return fail(IMGA_ERR_INVALID_ARG, "precision must be 0 (FP64) or 1 (mixed)");
    for (const void* p : {(const void*)u, (const void*)up, (const void*)up2, (const void*)f, (const void*)v, (const void*)out})
        if (p && ((uintptr_t)p & 15)) return fail(IMGA_ERR_INVALID_ARG, "node vectors must be 16-byte aligned");
    if (imga::vms_apply(h->m, u, up, up2, f, *ph, precision, v, out, stream)) return cuda_status("residual/jvp launch");
    return IMGA_OK;
}

imga_status imga_residual(imga_mesh h, const double* u, const double* up, const double* up2, const double* f,
                          const imga_physics* ph, int precision, double* R, void* stream) {
    return apply(h, u, up, up2, f, ph, precision, nullptr, R, stream);
}

imga_status imga_jvp(imga_mesh h, const double* u, const double* up, const double* up2, const double* f,
                     const imga_physics* ph, int precision, const double* v, double* Jv, void* stream) {
    if (!v) return fail(IMGA_ERR_INVALID_ARG, "null direction");
    return apply(h, u, up, up2, f, ph, precision, v, Jv, stream);
}

imga_status imga_element_jacobians(imga_mesh h, const double* u, const double* up, const double* up2, const double* f,
                                   const imga_physics* ph, int precision, const int32_t* elems, int64_t n, double* K,
                                   void* stream) {
    if (!h || !u || !up || n < 0 || (n > 0 && (!elems || !K))) return fail(IMGA_ERR_INVALID_ARG, "bad argument");
    if (h->m.host_only) return fail(IMGA_ERR_INVALID_ARG, "mesh was built host-only (device < 0)");
    if (!physics_ok(ph)) return fail(IMGA_ERR_INVALID_ARG, "bad physics parameters");
    if (ph->time_scheme == 2 && !up2) return fail(IMGA_ERR_INVALID_ARG, "BDF2 needs u_prev2");
    if (precision != 0 && precision != 1) return fail(IMGA_ERR_INVALID_ARG, "precision must be 0 (FP64) or 1 (mixed)");
    if (imga::element_jacobians(h->m, u, up, up2, f, *ph, precision, elems, n, K, stream)) return cuda_status("element_jacobians");
    return IMGA_OK;
}

static imga_status state_ok(imga_mesh h, const double* u, const double* up, const double* up2, const imga_physics* ph,
                            int precision) {
    if (!h || !u || !up) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    if (h->m.host_only) return fail(IMGA_ERR_INVALID_ARG, "mesh was built host-only (device < 0)");
    if (!physics_ok(ph)) return fail(IMGA_ERR_INVALID_ARG, "bad physics parameters");
    if (ph->time_scheme == 2 && !up2) return fail(IMGA_ERR_INVALID_ARG, "BDF2 needs u_prev2");
    if (precision != 0 && precision != 1) return fail(IMGA_ERR_INVALID_ARG, "precision must be 0 (FP64) or 1 (mixed)");
    return IMGA_OK;
}

imga_status imga_bsr_assemble(imga_mesh h, const double* u, const double* up, const double* up2, const double* f,
                              const imga_physics* ph, int precision, double* vals, void* stream) {
    imga_status st = state_ok(h, u, up, up2, ph, precision);
    if (st != IMGA_OK) return st;
    if (!vals) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    std::string err;
    const int64_t* bp;
    const int32_t* bi;
    double* ks;
    try {
        if (imga::bsr_device_pattern(h->m, &bp, &bi, &ks, err)) return fail(IMGA_ERR_OOM, err);
    } catch (const std::bad_alloc&) {
        return fail(IMGA_ERR_OOM, "block pattern: host allocation failed");
    }
    if (imga::bsr_assemble(h->m, u, up, up2, f, *ph, precision, bp, bi, vals, ks, stream)) return cuda_status("bsr_assemble");
    return IMGA_OK;
}

imga_status imga_bsr_spmv(imga_mesh h, const double* vals, const double* x, double* y, void* stream) {
    if (!h || !vals || !x || !y) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    if (h->m.host_only) return fail(IMGA_ERR_INVALID_ARG, "mesh was built host-only (device < 0)");
    std::string err;
    if (imga::bsr_spmv(h->m, vals, x, y, stream, err)) return fail(err.empty() ? IMGA_ERR_CUDA : IMGA_ERR_INVALID_ARG, err.empty() ? "bsr_spmv launch failed" : err);
    return IMGA_OK;
}

imga_status imga_multilevel_setup(imga_mesh h, const double* u, const double* up, const double* up2, const double* f,
                                  const imga_physics* ph, int precision, int agg, int coarse_max, int sweeps, double omega,
                                  void* stream) {
    imga_status st = state_ok(h, u, up, up2, ph, precision);
    if (st != IMGA_OK) return st;
    if (agg < 2 || coarse_max < 1 || coarse_max > 24 || sweeps < 1 || !(omega > 0.0))
        return fail(IMGA_ERR_INVALID_ARG, "multilevel: agg >= 2, 1 <= coarse_max <= 24, sweeps >= 1, omega > 0");
    std::string err;
    try {
        if (imga::multilevel_prepare(h->m, agg, coarse_max, err)) return fail(IMGA_ERR_OOM, err);
    } catch (const std::bad_alloc&) {
        return fail(IMGA_ERR_OOM, "multilevel: host allocation failed");
    }
    if (imga::multilevel_setup(h->m, u, up, up2, f, *ph, precision, sweeps, omega, stream, err)) return fail(IMGA_ERR_CUDA, err);
    return IMGA_OK;
}

imga_status imga_multilevel_apply(imga_mesh h, const double* r, double* z, void* stream) {
    if (!h || !r || !z) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    if (!h->m.mlev) return fail(IMGA_ERR_INVALID_ARG, "multilevel: call imga_multilevel_setup first");
    if (imga::multilevel_apply(h->m, r, z, stream)) return cuda_status("multilevel_apply");
    return IMGA_OK;
}

imga_status imga_multilevel_info(imga_mesh h, int* n_levels, int64_t* rows, int* singular) {
    if (!h || !n_levels) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    *n_levels = imga::multilevel_info(h->m, rows, singular);
    return IMGA_OK;
}

imga_status imga_surface_force(imga_mesh h, const double* u, const double* up, const imga_physics* ph, double* F,
                               void* stream) {
    imga_status st = state_ok(h, u, up, up, ph, 0);
    if (st != IMGA_OK) return st;
    if (!F) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    imga::Mesh& m = h->m;
    if (!m.force_part && cudaMalloc((void**)&m.force_part, imga::kForcePartials * sizeof(double)) != cudaSuccess)
        return fail(IMGA_ERR_OOM, "cudaMalloc failed");
    if (imga::surface_force(m, u, up, *ph, F, m.force_part, stream)) return cuda_status("surface_force");
    return IMGA_OK;
}

imga_status imga_time_steps(imga_mesh h, double* u, double* u_prev, const double* f, const imga_physics* ph,
                            const imga_solver_opts* o, int n_steps, double* force_hist, int* newton_hist,
                            int* krylov_hist, void* stream) {
    if (!h || !u || !u_prev || !ph || !o || n_steps < 0) return fail(IMGA_ERR_INVALID_ARG, "bad argument");
    imga_status st = state_ok(h, u, u_prev, u_prev, ph, o->precision);
    if (st != IMGA_OK) return st;
    imga::Mesh& m = h->m;
    const size_t bytes = (size_t)m.n_nodes() * 4 * sizeof(double);
    cudaStream_t s = (cudaStream_t)stream;
    double *up2 = nullptr, *un = nullptr, *F = nullptr;
    if (cudaMalloc((void**)&up2, std::max<size_t>(bytes, 8)) != cudaSuccess ||
        cudaMalloc((void**)&un, std::max<size_t>(bytes, 8)) != cudaSuccess || cudaMalloc((void**)&F, 3 * sizeof(double)) != cudaSuccess) {
        cudaFree(up2); cudaFree(un);
        return fail(IMGA_ERR_OOM, "cudaMalloc failed");
    }
    if (!m.force_part && cudaMalloc((void**)&m.force_part, imga::kForcePartials * sizeof(double)) != cudaSuccess) {
        cudaFree(up2); cudaFree(un); cudaFree(F);
        return fail(IMGA_ERR_OOM, "cudaMalloc failed");
    }
    imga_status rc = IMGA_OK;
    for (int k = 0; k < n_steps && rc == IMGA_OK; ++k) {
        // BDF2 starts with one backward-Euler step (no second previous level yet)
        imga_physics p = *ph;
        if (p.time_scheme == 2 && k == 0) p.time_scheme = 0;
        cudaMemcpyAsync(un, u, bytes, cudaMemcpyDeviceToDevice, s);   // the new level starts from u^n
        imga_solver_stats stats;
        rc = imga_newton_step(h, un, u, p.time_scheme == 2 ? up2 : nullptr, f, &p, o, &stats, stream);
        if (rc != IMGA_OK && rc != IMGA_ERR_NOT_CONVERGED) break;
        if (newton_hist) newton_hist[k] = stats.newton_its;
        if (krylov_hist) krylov_hist[k] = stats.krylov_its;
        const imga_status conv = rc;
        rc = IMGA_OK;
        cudaMemcpyAsync(up2, u, bytes, cudaMemcpyDeviceToDevice, s);   // shift the levels
        cudaMemcpyAsync(u_prev, u, bytes, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(u, un, bytes, cudaMemcpyDeviceToDevice, s);
        if (force_hist) {
            if (imga::surface_force(m, u, u_prev, p, F, m.force_part, s)) { rc = cuda_status("surface_force"); break; }
            cudaMemcpyAsync(force_hist + 3 * k, F, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
        }
        if (conv == IMGA_ERR_NOT_CONVERGED) rc = fail(IMGA_ERR_NOT_CONVERGED, "a time step's Newton solve did not converge");
    }
    cudaStreamSynchronize(s);
    cudaFree(up2); cudaFree(un); cudaFree(F);
    return rc;
}

imga_status imga_partition_build(imga_mesh h, int k, double ts_over_tv, imga_partition* out) {
    if (!h || !out) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (h->m.batched) return fail(IMGA_ERR_INVALID_ARG, "batched meshes are not partitioned");
    if (h->m.user_bc) return fail(IMGA_ERR_INVALID_ARG, "partitions take the default strong rows (no imga_set_dirichlet)");
    if (!(ts_over_tv >= 0.0)) return fail(IMGA_ERR_INVALID_ARG, "ts_over_tv must be >= 0");
    std::string err;
    imga::Partition* P = nullptr;
    try {
        if (imga::partition_build(h->m, k, ts_over_tv, &P, err)) return fail(err.rfind("partition: 1", 0) == 0 ? IMGA_ERR_INVALID_ARG : IMGA_ERR_OOM, err);
    } catch (const std::bad_alloc&) {
        return fail(IMGA_ERR_OOM, "partition: host allocation failed");
    }
    imga_partition_s* ps = new imga_partition_s();
    ps->P = P;
    ps->mesh = &h->m;
    *out = ps;
    return IMGA_OK;
}

void imga_partition_destroy(imga_partition p) {
    if (!p) return;
    imga::partition_free(p->P);
    delete p;
}

imga_status imga_partition_info(imga_partition p, int* k, int64_t* elem_off, double* weight, int64_t* n_owned,
                                int64_t* n_ghost) {
    if (!p || !k) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    imga::partition_info(p->P, elem_off, weight, n_owned, n_ghost);
    *k = imga::partition_count(p->P);
    return IMGA_OK;
}

imga_status imga_partition_nodes(imga_partition p, int part, int64_t* nodes, int32_t* ghost_owner) {
    if (!p || part < 0 || part >= imga::partition_count(p->P)) return fail(IMGA_ERR_INVALID_ARG, "bad argument");
    imga::partition_nodes(p->P, part, nodes, ghost_owner);
    return IMGA_OK;
}

static imga_status partition_apply(imga_partition p, const double* u, const double* up, const double* up2, const double* f,
                                   const imga_physics* ph, int precision, const double* v, double* out, void* stream) {
    if (!p || !out) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    if (!u || !up) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    if (p->mesh->host_only) return fail(IMGA_ERR_INVALID_ARG, "partition of a host-only mesh has no device parts");
    if (!physics_ok(ph)) return fail(IMGA_ERR_INVALID_ARG, "bad physics parameters");
    if (ph->time_scheme == 2 && !up2) return fail(IMGA_ERR_INVALID_ARG, "BDF2 needs u_prev2");
    if (precision != 0 && precision != 1) return fail(IMGA_ERR_INVALID_ARG, "precision must be 0 (FP64) or 1 (mixed)");
    if (ph->g_points) return fail(IMGA_ERR_INVALID_ARG, "partitions take the uniform body velocity (g_points = NULL)");
    if (imga::partition_apply(p->P, u, up, up2, f, *ph, precision, v, out, stream)) return cuda_status("partition");
    return IMGA_OK;
}

imga_status imga_partition_residual(imga_partition p, const double* u, const double* up, const double* up2,
                                    const double* f, const imga_physics* ph, int precision, double* R, void* stream) {
    return partition_apply(p, u, up, up2, f, ph, precision, nullptr, R, stream);
}

imga_status imga_partition_jvp(imga_partition p, const double* u, const double* up, const double* up2, const double* f,
                               const imga_physics* ph, int precision, const double* v, double* Jv, void* stream) {
    if (!v) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    return partition_apply(p, u, up, up2, f, ph, precision, v, Jv, stream);
}

imga_status imga_peak_flops(int device, int kind, double* tflops) {
    if (!tflops || kind < 0 || kind > 2) return fail(IMGA_ERR_INVALID_ARG, "kind must be 0, 1 or 2 and tflops non-null");
    std::string err;
    if (imga::peak_flops(device, kind, tflops, err)) return fail(IMGA_ERR_CUDA, err);
    return IMGA_OK;
}

imga_status imga_newton_step(imga_mesh h, double* u, const double* up, const double* up2, const double* f,
                             const imga_physics* ph, const imga_solver_opts* o, imga_solver_stats* stats, void* stream) {
    if (!h || !u || !up || !o || !stats) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    if (h->m.host_only) return fail(IMGA_ERR_INVALID_ARG, "mesh was built host-only (device < 0)");
    if (!physics_ok(ph)) return fail(IMGA_ERR_INVALID_ARG, "bad physics parameters");
    if (ph->time_scheme == 2 && !up2) return fail(IMGA_ERR_INVALID_ARG, "BDF2 needs u_prev2");
    if (o->gmres_m < 1 || o->gmres_m > 63 || o->max_newton < 0 || o->max_krylov < 1 || !(o->rtol >= 0.0) ||
        !(o->krylov_rtol > 0.0) || (o->precision != 0 && o->precision != 1) || o->precond < 0 || o->precond > 4 ||
        (o->linear_solver != 0 && o->linear_solver != 1) || o->ml_agg < 0 || o->ml_agg == 1 || o->ml_coarse_max < 0 ||
        o->ml_coarse_max > 24 || o->ml_sweeps < 0 || o->ml_omega < 0.0 ||
        (o->precond == 2 && !o->learned))
        return fail(IMGA_ERR_INVALID_ARG, "bad solver options");
    imga_solver_opts oo = *o;
    if (oo.precond == 2) oo.learned = ((const imga_mlp_s*)o->learned)->M;
    std::string err;
    int rc = imga::newton_solve(h->m, u, up, up2, f, *ph, oo, stats, stream, err);
    if (rc == 3) return fail(IMGA_ERR_OOM, err);
    if (rc == 2) return fail(IMGA_ERR_NUMERIC, err);
    if (rc) return fail(IMGA_ERR_CUDA, err);
    if (cudaGetLastError() != cudaSuccess) return cuda_status("newton_step");
    if (!stats->converged) return fail(IMGA_ERR_NOT_CONVERGED, "Newton did not reach the tolerance");
    return IMGA_OK;
}

imga_status imga_mlp_create(int n_in, int width, int n_out, uint64_t seed, int device, imga_mlp* out) {
    if (!out || n_in < 1 || width < 1 || n_out < 1 || width > 4096 || n_in > 1 << 16 || n_out > 1 << 16)
        return fail(IMGA_ERR_INVALID_ARG, "bad MLP shape");
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return cuda_status("cudaSetDevice");
    imga_mlp_s* h = new imga_mlp_s();
    std::string err;
    if (imga::mlp_create(n_in, width, n_out, seed, &h->M, err)) { delete h; return fail(IMGA_ERR_OOM, err); }
    h->nin = n_in;
    h->nout = n_out;
    h->device = device;
    *out = h;
    return IMGA_OK;
}

void imga_mlp_destroy(imga_mlp h) {
    if (!h) return;
    imga::mlp_destroy(h->M);
    delete h;
}

imga_status imga_mlp_shape(imga_mlp h, int64_t* n_params, int* n_in_pad) {
    if (!h) return fail(IMGA_ERR_INVALID_ARG, "null MLP");
    if (n_params) *n_params = imga::mlp_nparam(h->M);
    if (n_in_pad) *n_in_pad = imga::mlp_nin_pad(h->M);
    return IMGA_OK;
}

imga_status imga_mlp_params(imga_mlp h, float* host, int set) {
    if (!h || !host) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    if (imga::mlp_params(h->M, host, set)) return cuda_status("mlp_params");
    return IMGA_OK;
}

imga_status imga_mlp_forward(imga_mlp h, const float* X, int64_t ldx, int64_t n, float* Y, void* stream) {
    if (!h || n < 0 || (n > 0 && (!X || !Y)) || ldx < h->nin) return fail(IMGA_ERR_INVALID_ARG, "bad argument");
    if (imga::mlp_forward(h->M, X, ldx, n, Y, (cudaStream_t)stream)) return cuda_status("mlp_forward");
    return IMGA_OK;
}

imga_status imga_mlp_gradient(imga_mlp h, const float* X, int64_t ldx, const float* T, int64_t n, double* loss,
                              float* grad_host, void* stream) {
    if (!h || n < 1 || !X || !T || !loss || ldx < h->nin) return fail(IMGA_ERR_INVALID_ARG, "bad argument");
    if (imga::mlp_gradient(h->M, X, ldx, T, n, loss, (cudaStream_t)stream)) return cuda_status("mlp_gradient");
    if (grad_host && imga::mlp_grads(h->M, grad_host)) return cuda_status("mlp_gradient copy");
    return IMGA_OK;
}

imga_status imga_mlp_train(imga_mlp h, const float* X, int64_t ldx, const float* T, int64_t n, int epochs, int batch,
                           float lr, double* loss_hist, void* stream) {
    if (!h || n < 1 || !X || !T || epochs < 0 || batch < 1 || ldx < h->nin || !(lr > 0.f))
        return fail(IMGA_ERR_INVALID_ARG, "bad argument");
    if (imga::mlp_train(h->M, X, ldx, T, n, epochs, batch, lr, loss_hist, (cudaStream_t)stream)) return cuda_status("mlp_train");
    return IMGA_OK;
}

imga_status imga_precond_dataset(imga_mesh h, const double* u, const double* up, const double* up2, const double* f,
                                 const imga_physics* ph, int precision, const int32_t* elems, int64_t n, int ldx,
                                 float* X, float* T, float* scale, void* stream) {
    if (!h || !u || !up || n < 0 || (n > 0 && (!elems || !X || !scale)) || ldx < 1027)
        return fail(IMGA_ERR_INVALID_ARG, "bad argument");
    if (h->m.host_only) return fail(IMGA_ERR_INVALID_ARG, "mesh was built host-only (device < 0)");
    if (!physics_ok(ph) || (ph->time_scheme == 2 && !up2)) return fail(IMGA_ERR_INVALID_ARG, "bad physics parameters");
    if (n == 0) return IMGA_OK;
    double* K = nullptr;
    if (cudaMalloc((void**)&K, (size_t)n * 1024 * sizeof(double)) != cudaSuccess) return fail(IMGA_ERR_OOM, "cudaMalloc failed");
    int rc = imga::precond_dataset(h->m, u, up, up2, f, *ph, precision, elems, n, ldx, X, T, scale, K, (cudaStream_t)stream);
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(K);
    if (rc) return cuda_status("precond_dataset");
    return IMGA_OK;
}

imga_status imga_gemm_bf16(int M, int N, int K, const float* A, const float* B, float* C, void* stream) {
    if (M < 0 || N < 0 || K < 0 || (M * N > 0 && (!A || !B || !C))) return fail(IMGA_ERR_INVALID_ARG, "bad argument");
    if (imga::gemm_bf16_test(M, N, K, A, B, C, (cudaStream_t)stream)) return cuda_status("gemm_bf16");
    return IMGA_OK;
}

imga_status imga_set_option(imga_mesh h, int option, int64_t value) {
    if (!h) return fail(IMGA_ERR_INVALID_ARG, "null mesh");
    if (h->m.host_only) return fail(IMGA_ERR_INVALID_ARG, "mesh was built host-only (device < 0)");
    switch (option) {
        case IMGA_OPT_GRAPHS:
            if (!value) imga::graphs_free(h->m);
            h->m.use_graphs = value != 0;
            return IMGA_OK;
        case IMGA_OPT_AUTOTUNE:
            for (int p = 0; p < 2; ++p)
                for (int j = 0; j < 2; ++j) {
                    h->m.tune_pending[p][j] = value != 0;
                    if (!value) { h->m.cut_tune[p][j] = imga::Mesh::CutTune(); h->m.out_bps[p][j] = 0; }
                }
            imga::graphs_free(h->m);
            return IMGA_OK;
        case IMGA_OPT_CLASSIFY_RAYS:
            if (h->m.batched) return fail(IMGA_ERR_INVALID_ARG, "batched meshes do not classify points");
            h->m.classify_ray_only = value != 0;
            return IMGA_OK;
        case IMGA_OPT_DETERMINISTIC:
            h->m.deterministic = value != 0;
            imga::graphs_free(h->m);   // captured launches carry the scatter
            return IMGA_OK;
        case IMGA_OPT_FUSED: {
            if (value && !h->m.d.fq_cnt) {
                std::string err;
                if (imga::fused_prepare(h->m, err)) return fail(IMGA_ERR_CUDA, err);
            }
            h->m.fused = value != 0;
            imga::graphs_free(h->m);   // captured launches carry the kernels
            return IMGA_OK;
        }
        case IMGA_OPT_CONCURRENT:
            h->m.concurrent = value != 0;
            imga::graphs_free(h->m);
            return IMGA_OK;
        case IMGA_OPT_FUSED_SPLIT:
            if (value < 1 || value > 4) return fail(IMGA_ERR_INVALID_ARG, "IMGA_OPT_FUSED_SPLIT takes 1 .. 4");
            h->m.fused_heavy_warps = (int)value;
            imga::graphs_free(h->m);
            return IMGA_OK;
        default:
            return fail(IMGA_ERR_INVALID_ARG, "unknown option");
    }
}

imga_status imga_fused_info(imga_mesh h, int64_t* counts) {
    if (!h || !counts) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    counts[0] = h->m.fused ? 1 : 0;
    for (int k = 0; k < 3; ++k) counts[1 + k] = h->m.fq_counts[k];
    counts[4] = (int64_t)h->m.out_list.size();
    counts[5] = h->m.fused_heavy_warps;
    return IMGA_OK;
}

imga_status imga_tuning_interior(imga_mesh h, int32_t* bps, float* ms) {
    if (!h || !bps) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    for (int p = 0; p < 2; ++p)
        for (int j = 0; j < 2; ++j) {
            bps[2 * p + j] = h->m.out_bps[p][j];
            if (ms)
                for (int c = 0; c < 5; ++c) ms[10 * p + 5 * j + c] = h->m.out_tune_ms[p][j][c];
        }
    return IMGA_OK;
}

imga_status imga_tuning(imga_mesh h, int32_t* shape, float* ms) {
    if (!h || !shape) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    for (int p = 0; p < 2; ++p)
        for (int j = 0; j < 2; ++j) {
            shape[4 * p + 2 * j] = h->m.cut_tune[p][j].wpb;
            shape[4 * p + 2 * j + 1] = h->m.cut_tune[p][j].lpt;
            if (ms)
                for (int c = 0; c < 6; ++c) ms[12 * p + 6 * j + c] = h->m.cut_tune_ms[p][j][c];
        }
    return IMGA_OK;
}

imga_status imga_profile(imga_mesh h, int enable) {
    if (!h) return fail(IMGA_ERR_INVALID_ARG, "null mesh");
    if (enable) imga::profile_reset(h->m);
    h->m.profiling = enable != 0;
    return IMGA_OK;
}

imga_status imga_profile_read(imga_mesh h, double* ms, int64_t* launches) {
    if (!h) return fail(IMGA_ERR_INVALID_ARG, "null mesh");
    if (imga::profile_collect(h->m)) return cuda_status("profile_read");
    for (int k = 0; k < imga::kProfKinds; ++k) {
        if (ms) ms[k] = h->m.prof_ms[k];
        if (launches) launches[k] = h->m.prof_n[k];
    }
    return IMGA_OK;
}

imga_status imga_jvp_noalloc(imga_mesh h, const double* u, const double* up, const double* up2, const double* f,
                             const imga_physics* ph, int precision, const double* v, double* Jv, void* stream) {
    if (!h || !u || !up || !v || !Jv) return fail(IMGA_ERR_INVALID_ARG, "null argument");
    if (h->m.host_only) return fail(IMGA_ERR_INVALID_ARG, "mesh was built host-only (device < 0)");
    if (!physics_ok(ph)) return fail(IMGA_ERR_INVALID_ARG, "bad physics parameters");
    if (ph->time_scheme == 2 && !up2) return fail(IMGA_ERR_INVALID_ARG, "BDF2 needs u_prev2");
    if (precision != 0 && precision != 1) return fail(IMGA_ERR_INVALID_ARG, "precision must be 0 (FP64) or 1 (mixed)");
    for (const void* p : {(const void*)u, (const void*)up, (const void*)up2, (const void*)f, (const void*)v, (const void*)Jv})
        if (p && ((uintptr_t)p & 15)) return fail(IMGA_ERR_INVALID_ARG, "node vectors must be 16-byte aligned");
    std::string err;
    if (imga::vms_jvp_noalloc(h->m, u, up, up2, f, *ph, precision, v, Jv, stream, err))
        return fail(IMGA_ERR_INVALID_ARG, "imga_jvp_noalloc: " + err);
    return cuda_status("jvp_noalloc launch");
}

imga_status imga_selftest_conversions(int device, int64_t n, uint64_t seed, int64_t* mismatches) {
    if (n < 0 || !mismatches) return fail(IMGA_ERR_INVALID_ARG, "n must be >= 0 and mismatches non-null");
    if (cudaSetDevice(device) != cudaSuccess) return cuda_status("cudaSetDevice");
    std::string err;
    if (imga::conversion_selftest(n, seed, mismatches, err)) return fail(IMGA_ERR_CUDA, "conversion self-check: " + err);
    return cuda_status("conversion self-check");
}

imga_status imga_set_dirichlet(imga_mesh h, const uint8_t* mask, const double* val, void* stream) {
    if (!h) return fail(IMGA_ERR_INVALID_ARG, "null mesh");
    if (h->m.host_only) return fail(IMGA_ERR_INVALID_ARG, "mesh was built host-only (device < 0)");
    imga::Mesh& m = h->m;
    imga::graphs_free(m);   // graphs bake the boundary rows in
    if (!mask && !val) { m.user_bc = false; return IMGA_OK; }
    if (!mask || !val) return fail(IMGA_ERR_INVALID_ARG, "mask and values go together");
    const int64_t nn = m.n_nodes();
    if (!m.d.bcmask_user) {
        if (cudaMalloc((void**)&m.d.bcmask_user, std::max<int64_t>(1, nn)) != cudaSuccess ||
            cudaMalloc((void**)&m.d.bcval_user, std::max<int64_t>(1, nn) * 4 * sizeof(double)) != cudaSuccess)
            return fail(IMGA_ERR_OOM, "cudaMalloc failed");
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemcpyAsync(m.d.bcmask_user, mask, nn, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m.d.bcval_user, val, nn * 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    m.user_bc = true;
    return cuda_status("set_dirichlet");
}

}  // extern "C"
