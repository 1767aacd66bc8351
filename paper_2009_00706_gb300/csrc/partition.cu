// Weighted space-filling-curve partition of one mesh into k parts with ghost layers and explicit halo
// exchange (Sec. "Partitioning" and Eq. (Wpart); the ghost layers of Sec. "Octree based Mesh
// Generation"), run as k parts on one GPU.
//
// Eq. (Wpart) weighs element e by its quadrature work relative to an Out element:
//     W(e) = n_Vgp(e) / n_Tgp + (T_s / T_v) n_Sgp(e) / n_Tgp,   n_Tgp = 8 for Q1,
// n_Vgp the volume points evaluated (8 for Out, the kept sub-cell points for Intercepted, none for In)
// and n_Sgp its surface points.  The Morton order of the elements is cut into k contiguous ranges of
// equal total weight.
//
// Part p owns the nodes it is the lowest-numbered part to touch (through M_e: corners and the parents
// of hanging corners) and keeps the others it touches as ghosts.  Its sub-mesh numbers the owned nodes
// first, then the ghosts, both in global order.  One residual or J v runs as the data flow of a
// multi-GPU step, every transfer through explicit buffers:
//   1. every part copies its owned rows of the inputs from the global vectors;
//   2. halo gather: the owners pack the rows their neighbours hold as ghosts into send buffers, the
//      buffers move (a device copy here, a send / receive between GPUs), the receivers unpack them
//      into their ghost rows;
//   3. every part runs the element kernels on its own elements (strong rows on owned nodes only);
//   4. halo reduce-add: every part packs its ghost rows of the output, the buffers move, the owners add
//      them to their rows in part order, skipping the prescribed components;
//   5. every part writes its owned rows to the global output.
// On a mesh built host-only the partition and the halo lists are built without a GPU (unit weights:
// the markers and sub-cell points are computed on the device).

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "imga_internal.h"

namespace imga {

namespace {

// dst[i] = src[idx[i]] (rows of 4 doubles)
__global__ void rows_gather(int64_t n, const int64_t* __restrict__ idx, const double* __restrict__ src,
                            double* __restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * n) return;
    dst[t] = src[4 * idx[t >> 2] + (t & 3)];
}

// dst[idx[i]] = src[i]
__global__ void rows_scatter(int64_t n, const int64_t* __restrict__ idx, const double* __restrict__ src,
                             double* __restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * n) return;
    dst[4 * idx[t >> 2] + (t & 3)] = src[t];
}

// dst[idx[i]] += src[i] for the components the node does not prescribe (mask bits of flag)
__global__ void rows_add_free(int64_t n, const int64_t* __restrict__ idx, const double* __restrict__ src,
                              const uint8_t* __restrict__ flag, double* __restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * n) return;
    const int64_t r = idx[t >> 2];
    const int k = (int)(t & 3);
    uint8_t mask = (uint8_t)(flag[r] & 15);
    if (flag[r] & 16) mask = 15;
    if (!((mask >> k) & 1)) dst[4 * r + k] += src[t];
}

inline unsigned nblocks(int64_t threads) { return (unsigned)std::max<int64_t>(1, (threads + 255) / 256); }

}  // namespace

struct Part {
    int64_t e0 = 0, e1 = 0;             // global element range
    double weight = 0.0;
    std::vector<int64_t> nodes;         // local -> global node (owned first, then ghosts)
    int64_t n_owned = 0;
    std::vector<int> ghost_owner;       // [n ghosts]
    Mesh* mesh = nullptr;               // sub-mesh (device meshes only)
    // device: local -> global rows, local vectors u, up, up2, f, v, out
    int64_t* d_nodes = nullptr;
    double* d_vec[6] = {};
    // halo: for every other part q, the positions in this part's local numbering of the rows it
    // sends to q (owned rows q holds as ghosts) and receives from q (its ghosts owned by q)
    std::vector<std::vector<int64_t>> send_idx, recv_idx;
    std::vector<int64_t*> d_send, d_recv;
    std::vector<double*> d_sbuf, d_rbuf;   // send / receive buffers, 5 vectors x rows x 4
};

struct Partition {
    int k = 0;
    bool device = false;
    const Mesh* global = nullptr;
    std::vector<Part> parts;
};

namespace {

// the sub-mesh of part p: its elements, their geometry and quadrature, local node numbering
bool build_sub_mesh(const Mesh& g, Part& P, std::string& err) {
    Mesh* s = new Mesh();
    P.mesh = s;
    s->device = g.device;
    std::memcpy(s->lo, g.lo, sizeof(g.lo));
    std::memcpy(s->hi, g.hi, sizeof(g.hi));
    std::memcpy(s->hiI, g.hiI, sizeof(g.hiI));
    s->scale = g.scale;
    s->base_level = g.base_level;
    s->lmax = g.lmax;
    s->n_sm = g.n_sm;
    const int64_t gn = g.n_nodes(), ne = P.e1 - P.e0, nl = (int64_t)P.nodes.size();
    std::vector<int64_t> g2l(gn, -1);
    for (int64_t i = 0; i < nl; ++i) g2l[P.nodes[i]] = i;
    // hanging corners of the part, renumbered
    std::vector<int64_t> h2l(g.n_hang(), -1);
    int64_t nh = 0;
    s->anc.assign(g.anc.begin() + 3 * P.e0, g.anc.begin() + 3 * P.e1);
    s->lev.assign(g.lev.begin() + P.e0, g.lev.begin() + P.e1);
    s->marker.assign(g.marker.begin() + P.e0, g.marker.begin() + P.e1);
    s->cflags.assign(g.cflags.begin() + P.e0, g.cflags.begin() + P.e1);
    s->conn.resize(8 * ne);
    std::vector<int64_t> hang_g;
    for (int64_t e = 0; e < ne; ++e)
        for (int c = 0; c < 8; ++c) {
            const int32_t id = g.conn[8 * (P.e0 + e) + c];
            if (id < gn) { s->conn[8 * e + c] = (int32_t)g2l[id]; continue; }
            const int64_t h = id - gn;
            if (h2l[h] < 0) { h2l[h] = nh++; hang_g.push_back(h); }
            s->conn[8 * e + c] = -1 - (int32_t)h2l[h];   // fixed below, once the node count is known
        }
    for (int32_t& id : s->conn)
        if (id < 0) id = (int32_t)(nl + (-1 - id));
    s->hnp.resize(nh);
    s->hpar.assign(4 * nh, -1);
    for (int64_t j = 0; j < nh; ++j) {
        const int64_t h = hang_g[j];
        s->hnp[j] = g.hnp[h];
        for (int q = 0; q < g.hnp[h]; ++q) s->hpar[4 * j + q] = (int32_t)g2l[g.hpar[4 * h + q]];
    }
    s->nijk.resize(3 * nl);
    for (int64_t i = 0; i < nl; ++i)
        for (int k = 0; k < 3; ++k) s->nijk[3 * i + k] = g.nijk[3 * P.nodes[i] + k];
    // strong rows: the global flags on owned nodes; ghosts carry none (their owner applies them)
    s->bcflag.assign(nl, 0);
    for (int64_t i = 0; i < P.n_owned; ++i) s->bcflag[i] = g.bcflag[P.nodes[i]];
    // quadrature
    for (int32_t e : g.out_list)
        if (e >= P.e0 && e < P.e1) s->out_list.push_back((int32_t)(e - P.e0));
    s->cut_off.push_back(0);
    for (size_t i = 0; i < g.cut_list.size(); ++i) {
        const int32_t e = g.cut_list[i];
        if (e < P.e0 || e >= P.e1) continue;
        s->cut_list.push_back((int32_t)(e - P.e0));
        s->cut_pts.insert(s->cut_pts.end(), g.cut_pts.begin() + 4 * g.cut_off[i], g.cut_pts.begin() + 4 * g.cut_off[i + 1]);
        s->cut_off.push_back((int64_t)s->cut_pts.size() / 4);
    }
    for (size_t i = 0; i < g.sq.size(); i += 10) {
        const int64_t e = (int64_t)g.sq[i + 8];
        if (e < P.e0 || e >= P.e1) continue;
        double rec[10];
        std::memcpy(rec, &g.sq[i], sizeof(rec));
        rec[8] = (double)(e - P.e0);
        s->sq.insert(s->sq.end(), rec, rec + 10);
    }
    s->cut_off_elem.assign(ne + 1, 0);
    for (size_t i = 0; i < s->cut_list.size(); ++i) s->cut_off_elem[s->cut_list[i] + 1] = s->cut_off[i + 1] - s->cut_off[i];
    for (int64_t e = 0; e < ne; ++e) s->cut_off_elem[e + 1] += s->cut_off_elem[e];
    return device_upload_part(*s, err);
}

}  // namespace

void partition_free(Partition* P) {
    if (!P) return;
    for (Part& p : P->parts) {
        if (p.mesh) {
            graphs_free(*p.mesh);
            device_free(*p.mesh);
            delete p.mesh;
        }
        cudaFree(p.d_nodes);
        for (double* v : p.d_vec) cudaFree(v);
        for (int64_t* q : p.d_send) cudaFree(q);
        for (int64_t* q : p.d_recv) cudaFree(q);
        for (double* q : p.d_sbuf) cudaFree(q);
        for (double* q : p.d_rbuf) cudaFree(q);
    }
    delete P;
}

// Eq. (Wpart) weights (unit weights on a host-only mesh) and the k-way split with halo lists.
int partition_build(const Mesh& m, int k, double ts_over_tv, Partition** out, std::string& err) {
    const int64_t ne = m.n_elem(), nn = m.n_nodes();
    if (k < 1 || k > 1024 || k > std::max<int64_t>(1, ne)) { err = "partition: 1 <= k <= min(1024, elements)"; return 1; }
    Partition* P = new Partition();
    P->k = k;
    P->device = !m.host_only;
    P->global = &m;
    // W(e)
    std::vector<double> W(ne, 1.0);
    if (P->device) {
        std::vector<int64_t> nsq(ne, 0);
        for (size_t i = 0; i < m.sq.size(); i += 10) nsq[(int64_t)m.sq[i + 8]] += 1;
        for (int64_t e = 0; e < ne; ++e) {
            const double nv = m.marker[e] == 0 ? 8.0 : (m.marker[e] == 2 ? (double)(m.cut_off_elem[e + 1] - m.cut_off_elem[e]) : 0.0);
            W[e] = nv / 8.0 + ts_over_tv * (double)nsq[e] / 8.0;
        }
    }
    // contiguous Morton ranges of equal weight: cut p at the element boundary whose prefix weight is
    // nearest to p / k of the total, every part keeping at least one element
    std::vector<double> pre(ne + 1, 0.0);
    for (int64_t e = 0; e < ne; ++e) pre[e + 1] = pre[e] + W[e];
    std::vector<int64_t> cut(k + 1, 0);
    cut[k] = ne;
    for (int p = 1; p < k; ++p) {
        const double target = pre[ne] * (double)p / (double)k;
        int64_t c = std::lower_bound(pre.begin(), pre.end(), target) - pre.begin();
        if (c > 0 && target - pre[c - 1] < pre[std::min(c, ne)] - target) --c;
        cut[p] = std::min(std::max(c, cut[p - 1] + 1), ne - (k - p));
    }
    P->parts.resize(k);
    for (int p = 0; p < k; ++p) {
        P->parts[p].e0 = cut[p];
        P->parts[p].e1 = cut[p + 1];
        P->parts[p].weight = pre[cut[p + 1]] - pre[cut[p]];
    }
    // owners: the lowest part that touches a node
    std::vector<int> owner(nn, k);
    auto touch = [&](int64_t el, auto&& fn) {
        for (int c = 0; c < 8; ++c) {
            const int32_t id = m.conn[8 * el + c];
            if (id < nn) { fn(id); continue; }
            const int64_t h = id - nn;
            for (int q = 0; q < m.hnp[h]; ++q) fn(m.hpar[4 * h + q]);
        }
    };
    for (int p = 0; p < k; ++p)
        for (int64_t el = P->parts[p].e0; el < P->parts[p].e1; ++el)
            touch(el, [&](int64_t n) { owner[n] = std::min(owner[n], p); });
    std::vector<int64_t> g2l(nn, -1);
    for (int p = 0; p < k; ++p) {
        Part& q = P->parts[p];
        std::vector<char> seen(nn, 0);
        std::vector<int64_t> mine;
        for (int64_t el = q.e0; el < q.e1; ++el)
            touch(el, [&](int64_t n) { if (!seen[n]) { seen[n] = 1; mine.push_back(n); } });
        std::sort(mine.begin(), mine.end());
        for (int64_t n : mine)
            if (owner[n] == p) q.nodes.push_back(n);
        q.n_owned = (int64_t)q.nodes.size();
        for (int64_t n : mine)
            if (owner[n] != p) { q.nodes.push_back(n); q.ghost_owner.push_back(owner[n]); }
    }
    // nodes no part touches (none on a valid mesh) belong to part 0
    for (int64_t n = 0; n < nn; ++n)
        if (owner[n] == k) { owner[n] = 0; P->parts[0].nodes.insert(P->parts[0].nodes.begin() + P->parts[0].n_owned, n); P->parts[0].n_owned++; }
    // halo lists: part p receives from q its ghosts owned by q (p's ghost order); q sends the same rows
    for (int p = 0; p < k; ++p) {
        P->parts[p].send_idx.assign(k, {});
        P->parts[p].recv_idx.assign(k, {});
    }
    for (int p = 0; p < k; ++p) {
        Part& q = P->parts[p];
        for (int64_t i = 0; i < q.n_owned; ++i) g2l[q.nodes[i]] = i;   // owned rows are unique across parts
    }
    for (int p = 0; p < k; ++p) {
        Part& q = P->parts[p];
        for (int64_t j = 0; j < (int64_t)q.ghost_owner.size(); ++j) {
            const int o = q.ghost_owner[j];
            const int64_t gnode = q.nodes[q.n_owned + j];
            q.recv_idx[o].push_back(q.n_owned + j);
            P->parts[o].send_idx[p].push_back(g2l[gnode]);
        }
    }
    *out = P;
    if (!P->device) return 0;
    // device side: sub-meshes, local vectors, halo index lists and buffers
    for (int p = 0; p < k; ++p) {
        Part& q = P->parts[p];
        if (!build_sub_mesh(m, q, err)) { partition_free(P); *out = nullptr; return 1; }
        const int64_t nl = (int64_t)q.nodes.size();
        bool ok = cudaMalloc((void**)&q.d_nodes, std::max<int64_t>(1, nl) * sizeof(int64_t)) == cudaSuccess &&
                  cudaMemcpy(q.d_nodes, q.nodes.data(), nl * sizeof(int64_t), cudaMemcpyHostToDevice) == cudaSuccess;
        for (int v = 0; v < 6 && ok; ++v) ok = cudaMalloc((void**)&q.d_vec[v], std::max<int64_t>(1, nl) * 4 * sizeof(double)) == cudaSuccess;
        q.d_send.assign(k, nullptr);
        q.d_recv.assign(k, nullptr);
        q.d_sbuf.assign(k, nullptr);
        q.d_rbuf.assign(k, nullptr);
        for (int o = 0; o < k && ok; ++o) {
            const int64_t ns = (int64_t)q.send_idx[o].size(), nr = (int64_t)q.recv_idx[o].size();
            if (ns) ok = cudaMalloc((void**)&q.d_send[o], ns * sizeof(int64_t)) == cudaSuccess &&
                         cudaMemcpy(q.d_send[o], q.send_idx[o].data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice) == cudaSuccess &&
                         cudaMalloc((void**)&q.d_sbuf[o], 5 * ns * 4 * sizeof(double)) == cudaSuccess;
            if (ok && nr) ok = cudaMalloc((void**)&q.d_recv[o], nr * sizeof(int64_t)) == cudaSuccess &&
                               cudaMemcpy(q.d_recv[o], q.recv_idx[o].data(), nr * sizeof(int64_t), cudaMemcpyHostToDevice) == cudaSuccess &&
                               cudaMalloc((void**)&q.d_rbuf[o], 5 * nr * 4 * sizeof(double)) == cudaSuccess;
        }
        if (!ok) { err = "partition: device allocation failed"; cudaGetLastError(); partition_free(P); *out = nullptr; return 1; }
    }
    return 0;
}

// Residual (v == nullptr) or J v over the k parts, with the halo exchanges of the multi-GPU step.
int partition_apply(Partition* P, const double* u, const double* up, const double* up2, const double* f,
                    const imga_physics& ph, int precision, const double* v, double* out, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const int k = P->k;
    const double* in[5] = {u, up, up2 ? up2 : up, f, v};
    const int nin = 5;
    // 1. owned rows from the global vectors
    for (Part& q : P->parts)
        for (int j = 0; j < nin; ++j)
            if (in[j]) rows_gather<<<nblocks(4 * q.n_owned), 256, 0, s>>>(q.n_owned, q.d_nodes, in[j], q.d_vec[j]);
    // 2. halo gather: pack, move, unpack
    for (int p = 0; p < k; ++p) {
        Part& q = P->parts[p];
        for (int o = 0; o < k; ++o) {
            const int64_t ns = (int64_t)q.send_idx[o].size();
            if (!ns) continue;
            for (int j = 0; j < nin; ++j)
                if (in[j]) rows_gather<<<nblocks(4 * ns), 256, 0, s>>>(ns, q.d_send[o], q.d_vec[j], q.d_sbuf[o] + 4 * ns * j);
            cudaMemcpyAsync(P->parts[o].d_rbuf[p], q.d_sbuf[o], 5 * ns * 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        }
    }
    for (int p = 0; p < k; ++p) {
        Part& q = P->parts[p];
        for (int o = 0; o < k; ++o) {
            const int64_t nr = (int64_t)q.recv_idx[o].size();
            if (!nr) continue;
            for (int j = 0; j < nin; ++j)
                if (in[j]) rows_scatter<<<nblocks(4 * nr), 256, 0, s>>>(nr, q.d_recv[o], q.d_rbuf[o] + 4 * nr * j, q.d_vec[j]);
        }
    }
    // 3. every part's element kernels
    for (Part& q : P->parts) {
        if (vms_apply(*q.mesh, q.d_vec[0], q.d_vec[1], up2 ? q.d_vec[2] : nullptr, f ? q.d_vec[3] : nullptr, ph, precision,
                      v ? q.d_vec[4] : nullptr, q.d_vec[5], s))
            return 1;
    }
    // 4. halo reduce-add: ghosts' partial rows back to their owners, added in part order
    for (int p = 0; p < k; ++p) {
        Part& q = P->parts[p];
        for (int o = 0; o < k; ++o) {
            const int64_t nr = (int64_t)q.recv_idx[o].size();
            if (!nr) continue;
            rows_gather<<<nblocks(4 * nr), 256, 0, s>>>(nr, q.d_recv[o], q.d_vec[5], q.d_rbuf[o]);
            cudaMemcpyAsync(P->parts[o].d_sbuf[p], q.d_rbuf[o], nr * 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        }
    }
    for (int p = 0; p < k; ++p) {
        Part& q = P->parts[p];
        for (int o = 0; o < k; ++o) {
            const int64_t ns = (int64_t)q.send_idx[o].size();
            if (!ns) continue;
            rows_add_free<<<nblocks(4 * ns), 256, 0, s>>>(ns, q.d_send[o], q.d_sbuf[o], q.mesh->d.bcflag, q.d_vec[5]);
        }
    }
    // 5. owned rows to the global output
    for (Part& q : P->parts)
        rows_scatter<<<nblocks(4 * q.n_owned), 256, 0, s>>>(q.n_owned, q.d_nodes, q.d_vec[5], out);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int partition_info(const Partition* P, int64_t* elem_off, double* weight, int64_t* n_owned, int64_t* n_ghost) {
    for (int p = 0; p < P->k; ++p) {
        const Part& q = P->parts[p];
        if (elem_off) { elem_off[p] = q.e0; elem_off[p + 1] = q.e1; }
        if (weight) weight[p] = q.weight;
        if (n_owned) n_owned[p] = q.n_owned;
        if (n_ghost) n_ghost[p] = (int64_t)q.nodes.size() - q.n_owned;
    }
    return 0;
}

int partition_count(const Partition* P) { return (int)P->parts.size(); }

int partition_nodes(const Partition* P, int p, int64_t* nodes, int32_t* ghost_owner) {
    const Part& q = P->parts[p];
    if (nodes) std::copy(q.nodes.begin(), q.nodes.end(), nodes);
    if (ghost_owner) std::copy(q.ghost_owner.begin(), q.ghost_owner.end(), ghost_owner);
    return 0;
}

}  // namespace imga
