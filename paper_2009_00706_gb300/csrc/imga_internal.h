// Internal data structures of the imga library (host side + device pointers).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/imga.h"

namespace imga {

constexpr int kMaxDepth = 20;     // integer coordinates on [0, 2^20] per root edge
constexpr int kMaxLevel = 15;     // deepest leaf level the mesh accepts (+1 internal)
// DeviceMesh::counters: points imga_classify settled by the stored marker, gave the normal test,
// decided by it, sent to ray parity; then the rays cast while building the mesh
constexpr int kClassifyCounts = 4, kBuildRays = 4, kCounters = 5;

// Morton code: bit b of x, y, z -> bits 3b, 3b+1, 3b+2
inline uint64_t part1by2(uint64_t v) {
    v &= 0x1fffff;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}
inline uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return part1by2(x) | (part1by2(y) << 1) | (part1by2(z) << 2);
}
// inverse of part1by2: bits 3b -> bit b (21 bits)
inline uint32_t compact1by2(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (uint32_t)v;
}

// Triangle tables (structure of arrays, float64), shared by the host and the device copies.
struct TriHost {
    int64_t n = 0;
    std::vector<double> v;      // [n][9]
    std::vector<double> nrm;    // [n][3] unit normal, out of the body
    std::vector<double> cen;    // [n][3]
    std::vector<double> bmin, bmax;  // [n][3]
    std::vector<double> area;   // [n]
};

// uniform grid over the (y, z) projection of the triangles, for rays cast along +x
struct RayGridHost {
    int ny = 0, nz = 0;
    double y0 = 0, z0 = 0, dy = 1, dz = 1;
    std::vector<int32_t> off;   // [ny*nz + 1]
    std::vector<int32_t> idx;
};

// device mirror of everything the kernels read
struct DeviceMesh {
    int64_t n_elem = 0, n_nodes = 0, n_hang = 0, n_tri = 0;
    uint64_t* key = nullptr;      // [n_elem] Morton key of each anchor (sorted)
    uint32_t* anc = nullptr;      // [n_elem][3]
    uint8_t* lev = nullptr;       // [n_elem]
    int32_t* conn = nullptr;      // [n_elem][8]
    int32_t* hpar = nullptr;      // [n_hang][4]
    // triangles
    double* tv = nullptr;         // [n_tri][9]
    double* tn = nullptr;         // [n_tri][3]
    double* tc = nullptr;         // [n_tri][3]
    int32_t* bt_off = nullptr;    // [n_elem + 1]
    int32_t* bt_idx = nullptr;
    int32_t* rg_off = nullptr;    // ray grid
    int32_t* rg_idx = nullptr;
    // classification results
    int8_t* marker = nullptr;     // [n_elem]
    uint8_t* cflags = nullptr;    // [n_elem]
    // quadrature
    int32_t* out_list = nullptr;  // Out elements
    int32_t* out_conn = nullptr;  // [n_out][8] their corner -> node (or n_nodes + hanging) indices
    uint8_t* out_lev = nullptr;   // [n_out] their levels
    uint16_t* out_prob = nullptr; // [n_out] their problem (batched meshes), else null
    uint16_t* eprob = nullptr;    // [n_elem] problem of every element (batched meshes), else null
    double* pmu = nullptr;        // [n_prob] viscosity of every problem (batched meshes)
    float* pmuf = nullptr;
    int32_t* cut_list = nullptr;  // Intercepted elements
    int64_t* cut_off = nullptr;   // [n_cut + 1] into cut_pts
    double* cut_pts = nullptr;    // [n][4] (xi0, xi1, xi2, reference weight)
    float* cut_pts_f = nullptr;   // [n][4] float copy
    int32_t* sq_elem = nullptr;   // surface points, sorted by element
    double* sq_x = nullptr;       // [n][3] reference coordinates in the element
    double* sq_n = nullptr;       // [n][3]
    double* sq_w = nullptr;
    double* sq_taub = nullptr;    // 1 / h_b
    int32_t* sq_src = nullptr;    // position of every surface point in the export order (imga_physics.g_points)
    int32_t* cut_order = nullptr;   // Intercepted list positions by decreasing point count (autotuner)
    int32_t* sq_hosts = nullptr;  // every element hosting a surface point (increasing)
    // float64 Nitsche penalty per surface-hosting element (in device point order): element, point range
    // [pen_q[i], pen_q[i+1]), destination slot, and the packed upper triangle of sum_q (w_q/h_b) phi_a phi_b
    int32_t* pen_elem = nullptr;
    int64_t* pen_q = nullptr;
    int64_t* pen_slot = nullptr;
    double* pen = nullptr;
    // deterministic scatter: node -> (slot, corner, weight) incidence and the element-contribution slots
    uint32_t* inc_head = nullptr; // [n_nodes][kIncHead] first entries of each node's list (kIncNone pads)
    int64_t* inc_ptr = nullptr;   // [n_nodes + 1] the rest of each list (CSR)
    uint32_t* inc = nullptr;      // bits 0-2 corner, 3-4 weight code, 5-31 global slot
    void* sv = nullptr;           // volume slots [n_vslots][8][4] of the element precision (sized for float64)
    double* ss = nullptr;         // surface slots [n_sslots][8][4] float64
    int32_t* sq_list = nullptr;   // elements hosting at least kNitscheDenseMin surface points
    int64_t* sq_off = nullptr;    // [n_sq_elem + 1] their point ranges in the sorted arrays
    // fused launch: work items (bits 30-31 kind, 0-29 index) and the claim counters [2]
    uint32_t* fq_items = nullptr;
    unsigned long long* fq_cnt = nullptr;
    // per-call node workspace (node_prep): value, tangent and force data of every independent and
    // hanging node, one float and one double copy
    float* nd_f = nullptr;        // [3][n_nodes + n_hang][8]
    double* nd_d = nullptr;
    int32_t* slot = nullptr;      // [n_elem] position of an element in a requested list, or -1
    // [kCounters]: the kClassifyCounts point counts of imga_classify, then the rays cast while building
    unsigned long long* counters = nullptr;
    // boundary rows
    uint8_t* bcflag = nullptr;    // [n_nodes] bits 0-3 box Dirichlet, bit 4 In-only node
    uint8_t* bcmask_user = nullptr;
    double* bcval_user = nullptr;
};

// node incidence lists of the deterministic scatter: fixed head length and its padding code
constexpr int kIncHead = 8;
constexpr uint32_t kIncNone = 0xFFFFFFFFu;

// elements hosting at least this many surface points take the warp-per-element surface kernel
constexpr int kNitscheDenseMin = 8;
// timed kernel classes: Out, Intercepted, surface, strong rows / node sums, node preparation, fused launch
constexpr int kProfKinds = 6;

struct GraphKey {
    const double *u, *up, *up2, *f, *v;
    double* out;
    int precision;
    int user_bc;
    imga_physics ph;
};

struct Mesh {
    int device = 0;
    double lo[3], hi[3], scale = 1.0;
    int64_t hiI[3];
    int base_level = 0, lmax = 3;
    std::vector<imga_region> regions;
    // octree
    std::vector<uint64_t> key;
    // key_lut[p] = first leaf whose key has the top kLutBits bits >= p (p = 0 .. 2^kLutBits);
    // valid while key_lut_n == key.size()
    std::vector<int32_t> key_lut;
    size_t key_lut_n = 0;
    std::vector<uint32_t> anc;    // [n][3]
    std::vector<uint8_t> lev;
    // nodes
    std::vector<uint32_t> nijk;   // [n_nodes][3]
    std::vector<int32_t> conn;    // [n_elem][8]
    std::vector<int32_t> hpar;    // [n_hang][4]
    std::vector<int8_t> hnp;
    // geometry
    TriHost tri;
    std::vector<int32_t> bt_off, bt_idx;
    RayGridHost grid;
    std::vector<int8_t> marker;
    std::vector<uint8_t> cflags;
    std::vector<int32_t> out_list, cut_list;
    std::vector<int64_t> cut_off_elem;   // [n_elem + 1] for export
    std::vector<double> cut_pts;         // [n][4] in cut_list order
    std::vector<int64_t> cut_off;        // [n_cut + 1]
    std::vector<double> sq;              // [n][10] surface points (export layout)
    int64_t n_sq_sparse = 0;             // surface points of elements hosting < kNitscheDenseMin (stored first)
    int64_t n_sq_elem = 0;               // elements hosting >= kNitscheDenseMin surface points
    std::vector<int32_t> sq_hosts;       // every element hosting a surface point (increasing)
    std::vector<int32_t> pen_elem;       // surface-hosting elements in device point order (nitsche_penalty)
    std::vector<int64_t> sq_off_h;       // host copy of DeviceMesh::sq_off
    int64_t n_vslots = 0, n_sslots = 0;  // deterministic scatter: volume slots (active elements), surface slots
    bool deterministic = true;           // IMGA_OPT_DETERMINISTIC: slots + ordered node sums (1) or atomics (0)
    std::vector<uint8_t> bcflag;
    // block pattern of the assembled Jacobian (imga_bsr_pattern), built on first use
    std::vector<int64_t> bsr_ptr;        // [n_nodes + 1]
    std::vector<int32_t> bsr_idx;        // [n_blocks] block columns, increasing within a row
    int64_t n_in = 0, n_rays = 0;
    // batched meshes: element -> problem, per-problem viscosity and element/node offsets
    std::vector<uint16_t> eprob;
    std::vector<double> pmu;
    std::vector<int64_t> prob_elem_off, prob_node_off;
    double setup_ms[4] = {0, 0, 0, 0};
    bool user_bc = false;
    bool host_only = false;
    bool batched = false;
    bool classify_ray_only = false;      // imga_classify: ray parity for every point (IMGA_OPT_CLASSIFY_RAYS)
    // CUDA-graph execution of residual / J v (imga_set_option): cached executable graphs keyed by the
    // call's pointers and parameters, and two side streams + fork/join events for parallel branches
    bool use_graphs = false;
    // Intercepted-element bucket: warps per block and element order (0 Morton, 1 longest first),
    // per [float64 0 / mixed 1][residual 0 / J v 1]; set by the autotuner
    struct CutTune { int wpb = 4, lpt = 0; };
    CutTune cut_tune[2][2];
    float cut_tune_ms[2][2][6] = {};   // candidate times of the last tuning (ms per launch)
    bool tune_pending[2][2] = {{false, false}, {false, false}};
    // Out-element bucket: resident blocks per SM of the persistent interior kernel (0: the occupancy
    // limit), per [float64 / mixed][residual / J v], and the candidate times of the last tuning
    int out_bps[2][2] = {{0, 0}, {0, 0}};
    float out_tune_ms[2][2][5] = {};
    bool concurrent = true;              // IMGA_OPT_CONCURRENT: Intercepted / surface kernels on side streams
    // one persistent launch over the Out and Intercepted buckets (IMGA_OPT_FUSED): its queue holds the
    // Intercepted elements by decreasing point count (Eq. Wpart's volume cost)
    bool fused = false;
    int fused_heavy_warps = 4;           // warps per block that start on the Intercepted elements (1 .. 4)
    int64_t fq_n = 0;                    // items in fq_items
    int64_t fq_counts[3] = {0, 0, 0};    // queued Intercepted elements, dense surface elements, sparse surface points
    std::vector<std::pair<GraphKey, void*>> graphs;
    void* side[3] = {nullptr, nullptr, nullptr};   // two branch streams + the private capture stream
    void* fork_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // fork, 2 joins, caller->graph, graph->caller
    int n_sm = 1;                        // streaming multiprocessors of the device
    DeviceMesh d;
    void* scratch = nullptr;             // device workspace for the kernels
    void* solver_work = nullptr;         // Krylov workspace (solver.cu)
    void* mlev = nullptr;                // assembled matrix and multilevel hierarchy (bsr.cu)
    double* force_part = nullptr;        // workspace of imga_surface_force
    // per-kernel profiling (CUDA events, one pair per launch, resolved at read time)
    bool profiling = false;
    struct ProfEv { void *a, *b; int launches; };   // event pair around `launches` kernels
    std::vector<ProfEv> prof_ev[kProfKinds];
    double prof_ms[kProfKinds] = {};
    int64_t prof_n[kProfKinds] = {};
    size_t scratch_bytes = 0;

    int64_t n_elem() const { return (int64_t)lev.size(); }
    int64_t n_nodes() const { return (int64_t)nijk.size() / 3; }
    int64_t n_hang() const { return (int64_t)hnp.size(); }
};

// host builders (mesh_host.cpp)
bool build_octree(Mesh& m, std::string& err);
bool build_nodes(Mesh& m, std::string& err);
bool build_triangles(Mesh& m, const double* tri, int64_t n, std::string& err);
void build_background(Mesh& m);
void build_ray_grid(Mesh& m);
void build_surface_points(Mesh& m);
void build_bc_flags(Mesh& m);
int64_t find_leaf(const Mesh& m, int64_t x, int64_t y, int64_t z);
void build_bsr_pattern(Mesh& m);

// device stages (geom.cu)
bool build_incidence(Mesh& m, const std::vector<int32_t>& sq_el, const std::vector<int32_t>& dense, std::string& err);
bool device_upload_geometry(Mesh& m, std::string& err);
bool device_markers(Mesh& m, std::string& err);
bool device_cut_quadrature(Mesh& m, std::string& err);
bool device_upload_quadrature(Mesh& m, std::string& err);
bool device_upload_batch(Mesh& m, std::string& err);
bool device_upload_part(Mesh& m, std::string& err);
int device_classify(const Mesh& m, const double* pts, int64_t n, uint8_t* flags, void* stream);
void device_free(Mesh& m);

// residual / Jv (vms.cu)
int conversion_selftest(int64_t n, uint64_t seed, int64_t* mismatches, std::string& err);
int vms_apply_skip(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                   const imga_physics& ph, int precision, const double* v, double* out, void* stream, const int* skip);
void vms_prepare();
int vms_apply(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
              const imga_physics& ph, int precision, const double* v, double* out, void* stream);

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // fixed scratch of imga_jvp_noalloc
constexpr int kMaxDevices = 64;
int vms_jvp_noalloc(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                    const imga_physics& ph, int precision, const double* v, double* out, void* stream,
                    std::string& err);

int surface_force(const Mesh& m, const double* u, const double* up, const imga_physics& ph, double* F, double* part,
                  void* stream);
constexpr int kForcePartials = 256 * 3;   // doubles of workspace for surface_force

void profile_reset(Mesh& m);
int profile_collect(Mesh& m);
int fused_prepare(Mesh& m, std::string& err);
void graphs_free(Mesh& m);

// element Jacobians and block-Jacobi (jac.cu)
int element_jacobians(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                      const imga_physics& ph, int precision, const int32_t* elems, int64_t n, double* K, void* stream);
int block_jacobi_setup(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                       const imga_physics& ph, int precision, double* D, double* Dinv, void* stream);
int block_jacobi_apply(const Mesh& m, const double* Dinv, const double* x, double* y, void* stream);
int bsr_assemble(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                 const imga_physics& ph, int precision, const int64_t* bptr, const int32_t* bidx, double* val,
                 double* Ks, void* stream);

// learned block preconditioner (mlp.cu)
struct Mlp;
int mlp_create(int nin, int width, int nout, uint64_t seed, Mlp** out, std::string& err);
void mlp_destroy(Mlp* M);
int64_t mlp_nparam(const Mlp* M);
int mlp_nin_pad(const Mlp* M);
int mlp_params(Mlp* M, float* host, int set);
int mlp_grads(Mlp* M, float* host);
int mlp_forward(Mlp* M, const float* X, int64_t ldx, int64_t n, float* Y, cudaStream_t s);
int mlp_gradient(Mlp* M, const float* X, int64_t ldx, const float* T, int64_t n, double* loss, cudaStream_t s);
int mlp_train(Mlp* M, const float* X, int64_t ldx, const float* T, int64_t n, int epochs, int batch, float lr,
              double* loss_hist, cudaStream_t s);
int precond_dataset(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                    const imga_physics& ph, int precision, const int32_t* elems, int64_t n, int ldx, float* X,
                    float* T, float* scale, double* Kbuf, cudaStream_t s);
int precond_correction(const Mesh& m, const imga_physics& ph, const int32_t* elems, int64_t n, const float* C,
                       const float* scale, float omega, const double* v, double* zc, double* z, cudaStream_t s);
int gemm_bf16_test(int M, int N, int K, const float* A, const float* B, float* C, cudaStream_t s);

// assembled matrix and multilevel preconditioner (bsr.cu)
int multilevel_prepare(Mesh& m, int agg, int coarse_max, std::string& err);
int multilevel_setup(Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                     const imga_physics& ph, int precision, int nu, double omega, void* stream, std::string& err);
int multilevel_apply(Mesh& m, const double* r, double* z, void* stream);
int multilevel_info(Mesh& m, int64_t* rows, int* singular);
void multilevel_free(Mesh& m);
int bsr_spmv(Mesh& m, const double* val, const double* x, double* y, void* stream, std::string& err);
int bsr_device_pattern(Mesh& m, const int64_t** ptr, const int32_t** idx, double** ks, std::string& err);
double* multilevel_matrix(Mesh& m);

// Newton-GMRES (solver.cu)
int newton_solve(Mesh& m, double* u, const double* up, const double* up2, const double* f, const imga_physics& ph,
                 const imga_solver_opts& o, imga_solver_stats* stats, void* stream, std::string& err);
void solver_free(Mesh& m);

bool merge_meshes(Mesh& m, const std::vector<const Mesh*>& parts, const std::vector<double>& mu, std::string& err);

// weighted SFC partition into k parts with halo exchange (partition.cu)
struct Partition;
int partition_build(const Mesh& m, int k, double ts_over_tv, Partition** out, std::string& err);
int partition_apply(Partition* P, const double* u, const double* up, const double* up2, const double* f,
                    const imga_physics& ph, int precision, const double* v, double* out, void* stream);
int partition_info(const Partition* P, int64_t* elem_off, double* weight, int64_t* n_owned, int64_t* n_ghost);
int partition_nodes(const Partition* P, int p, int64_t* nodes, int32_t* ghost_owner);
int partition_count(const Partition* P);
void partition_free(Partition* P);

// arithmetic-pipe microbenchmark (peak.cu)
int peak_flops(int device, int kind, double* tflops, std::string& err);

void set_error(const std::string& s);

}  // namespace imga
