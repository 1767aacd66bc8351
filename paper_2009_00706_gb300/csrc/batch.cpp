// Batched meshes: several independent problems merged into one mesh, so that one launch of each
// residual / J v kernel covers all of them (element -> problem map, per-problem viscosity).
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "imga_internal.h"

namespace imga {

// append problem `s` (built on its own) to the merged mesh `m`
static bool append(Mesh& m, const Mesh& s, uint16_t p, double mu, std::string& err) {
    const int64_t eoff = m.n_elem(), noff = m.n_nodes();
    const int64_t hoff = m.n_hang();
    if (m.prob_elem_off.empty()) {
        std::memcpy(m.lo, s.lo, sizeof(m.lo));
        std::memcpy(m.hi, s.hi, sizeof(m.hi));
        std::memcpy(m.hiI, s.hiI, sizeof(m.hiI));
        m.scale = s.scale;
    } else if (s.scale != m.scale || s.lo[0] != m.lo[0] || s.lo[1] != m.lo[1] || s.lo[2] != m.lo[2]) {
        err = "batched problems must share the box origin and the root size";
        return false;
    }
    m.prob_elem_off.push_back(eoff);
    m.prob_node_off.push_back(noff);
    m.pmu.push_back(mu);
    m.anc.insert(m.anc.end(), s.anc.begin(), s.anc.end());
    m.lev.insert(m.lev.end(), s.lev.begin(), s.lev.end());
    m.nijk.insert(m.nijk.end(), s.nijk.begin(), s.nijk.end());
    m.hnp.insert(m.hnp.end(), s.hnp.begin(), s.hnp.end());
    for (int32_t q : s.hpar) m.hpar.push_back(q >= 0 ? (int32_t)(q + noff) : -1);
    m.marker.insert(m.marker.end(), s.marker.begin(), s.marker.end());
    m.cflags.insert(m.cflags.end(), s.cflags.begin(), s.cflags.end());
    m.bcflag.insert(m.bcflag.end(), s.bcflag.begin(), s.bcflag.end());
    m.eprob.insert(m.eprob.end(), s.n_elem(), p);
    for (int32_t e : s.out_list) m.out_list.push_back((int32_t)(e + eoff));
    const int64_t poff = m.cut_off.empty() ? 0 : m.cut_off.back();
    if (m.cut_off.empty()) m.cut_off.push_back(0);
    for (size_t i = 0; i < s.cut_list.size(); ++i) {
        m.cut_list.push_back((int32_t)(s.cut_list[i] + eoff));
        m.cut_off.push_back(s.cut_off[i + 1] + poff);
    }
    m.cut_pts.insert(m.cut_pts.end(), s.cut_pts.begin(), s.cut_pts.end());
    for (size_t i = 0; i + 9 < s.sq.size() + 9 && i < s.sq.size(); i += 10) {
        double rec[10];
        std::memcpy(rec, &s.sq[i], sizeof(rec));
        rec[8] += (double)eoff;
        m.sq.insert(m.sq.end(), rec, rec + 10);
    }
    m.n_in += s.n_in;
    m.n_rays += s.n_rays;
    return true;
}

// hanging corners are addressed as n_nodes + h; once every problem is in, shift them past all nodes
static void finish_conn(Mesh& m, const std::vector<const Mesh*>& parts) {
    const int64_t nn = m.n_nodes();
    m.conn.clear();
    int64_t hoff = 0;
    for (size_t p = 0; p < parts.size(); ++p) {
        const Mesh& s = *parts[p];
        const int64_t noff = m.prob_node_off[p], snn = s.n_nodes();
        for (int32_t id : s.conn) m.conn.push_back(id < snn ? (int32_t)(id + noff) : (int32_t)(nn + hoff + (id - snn)));
        hoff += s.n_hang();
    }
}

bool merge_meshes(Mesh& m, const std::vector<const Mesh*>& parts, const std::vector<double>& mu, std::string& err) {
    if (parts.size() > 65535) { err = "too many problems"; return false; }
    for (size_t p = 0; p < parts.size(); ++p)
        if (!append(m, *parts[p], (uint16_t)p, mu[p], err)) return false;
    finish_conn(m, parts);
    m.cut_off_elem.assign(m.n_elem() + 1, 0);
    for (size_t i = 0; i < m.cut_list.size(); ++i) m.cut_off_elem[m.cut_list[i] + 1] = m.cut_off[i + 1] - m.cut_off[i];
    for (int64_t e = 0; e < m.n_elem(); ++e) m.cut_off_elem[e + 1] += m.cut_off_elem[e];
    m.key.clear();
    return device_upload_batch(m, err);
}

}  // namespace imga
