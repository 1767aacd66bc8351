// VMS residual R(u) and Jacobian-vector product J(u) v on Q1 octree elements.
//
// Weak form: Eqs. (ALE-VMS-form) and (vms), fine scales Eqs. (uprime) and (pprime), Nitsche
// terms Eq. (weakbc); In elements skipped, Out elements on the 2x2x2 Gauss rule, Intercepted
// elements on their adaptive sub-cell points (Algorithm 1); element vectors scattered to the
// nodes through the hanging-node operator M_e^T (Algorithms 2 and 3).
//
// Every quadrature point is reduced to 16 coefficients: with w = phi_a e_i and q = phi_a,
//     r_{a,i} += wq [ phi_a F_i + d_j phi_a S_ij ],     r_{a,p} += wq [ phi_a G + d_j phi_a H_j ],
//   F_i  = rho (du_i/dt + (u.grad u)_i - f_i) + (u'.grad u)_i                    terms 1, 6, -F
//   S_ij = sigma_ij - u'_i u_j - p' delta_ij - u'_i u'_j / rho + taubar (u'.grad u)_i u'_j
//                                                                                terms 2, 4, 5, 7, 8
//   G    = div u,   H_j = -u'_j / rho                                             terms 3, 4
// J v is the forward-mode derivative of the same code (dual numbers value + tangent): the
// matrix of Algorithms 2/4 applied to v without being formed.
//
// Kernels (T = float or double element arithmetic, nodal gathers always float64, scatter by
// float64 atomics):
//   vms_interior  8 threads per Out element: thread c gathers corner c, evaluates Gauss point c,
//                 then contracts node c's four rows over the 8 points; interpolation and test
//                 functions both run in the monomial form of the trilinear basis.
//   vms_cut       one warp per Intercepted element; lane l evaluates sub-cell points l, l + 32, ...
//                 and accumulates their monomial moments, summed over the lanes at the end.
//   nitsche       one thread per surface point, for elements hosting few points;
//   nitsche_el    one warp per element hosting many, lanes over its points (moments).
//   strong_rows   Dirichlet rows U - g and In-only rows, written after every scatter.

#include <cuda_runtime.h>

#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "imga_internal.h"
#include "vms_device.cuh"

namespace imga {

namespace {

// ------------------------------------------------------------------------------------------
// Out elements: 8 threads per element
// ------------------------------------------------------------------------------------------
template <class T> struct Epb { static constexpr int value = 16; };   // elements per block

template <class T> struct IntShape {
    static constexpr int EPB = Epb<T>::value;                                   // elements per block
    static constexpr int THREADS = 8 * EPB;
    // element stride of the corner rows: 8 rows of CS plus 8 T, so the elements of a warp start 8
    // (float) or 16 (double) banks apart and column and broadcast row reads are conflict-free
    static constexpr int ESTR = 8 * CS + 8;
    static constexpr int MSTR = 32 + 16 / (int)sizeof(T);   // row stride of the per-point moments
    static constexpr size_t smem = (size_t)(2 * EPB * ESTR + EPB * 8 * MSTR) * sizeof(T);
};

// One Out element on 8 lanes of a warp (lane & 7 = corner c): the element's rows `nd` are in
// shared memory (8 rows of CS, stride CS); the warp's moment rows s_mw [32][MSTR].  Thread c
// transforms column c of the rows into monomial coefficients, evaluates Gauss point c (monomials m),
// writes the point's 32 monomial moments, then sums moment column S = c over the 8 points and runs
// the backward butterfly: node c's rows, scattered (or stored to the element's slot).  Every lane of
// the warp takes part (valid: this lane's element exists).
// IL: with packed float duals, rewrite the rows with (value, tangent) interleaved so every 16-byte
// row load yields two dual pairs in place (off in the fused kernel, whose register budget it strains)
template <class T, bool JV, bool IL = (JV && sizeof(T) == 4)>
__device__ __forceinline__ void interior_element(const Args& A, T* nd, T* s_mw, const T m[8], int lane, int64_t idx,
                                                 bool valid, int lv, int prob, int32_t id) {
    typedef typename std::conditional<JV, Dual<T, sizeof(T) == 4>, T>::type S;
    constexpr int MSTR = IntShape<T>::MSTR;
    const int c = lane & 7;
    T* mrow = s_mw + lane * MSTR;
    const T* mcol = s_mw + (lane >> 3) * 8 * MSTR + 4 * c;
    __syncwarp();
    {   // corner values -> monomial coefficients: thread c transforms column c of the element's rows
        if constexpr (IL) {
            columns_to_monomial_interleaved<T>(nd, c);
        } else if (c < 7) {
            column_to_monomial<T>(nd + c);
            if (JV) column_to_monomial<T>(nd + CT + c);
        }
        if (A.ndf && c < 3) column_to_monomial<T>(nd + CF + c);
    }
    __syncwarp();
    const T g = lvl_g<T>(A, lv);
    const Phys<T> P(A, prob);
    S cf[16];
    vms_point_modal<S, T, IL>(A, P, m, nd, CS, g, cf);
    const T wq = lvl_w<T>(A, lv), wqg = wq * g;
    // F, G multiply phi; S, H multiply physical gradients = g x reference gradients
    T w16[16];
    for (int k = 0; k < 16; ++k) w16[k] = ((k < 3 || k == 12) ? wq : wqg) * Pick<T, JV>::get(cf[k]);
    T M[32];
    for (int k = 0; k < 32; ++k) M[k] = T(0);
    add_moments<T>(m, w16, M);
    for (int k = 0; k < 32; k += 4) st4s<T>(mrow + k, M[k], M[k + 1], M[k + 2], M[k + 3]);
    __syncwarp();
    T r[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        T v[4];
        ld4s<T>(mcol + q * MSTR, v);
        r[0] += v[0]; r[1] += v[1]; r[2] += v[2]; r[3] += v[3];
    }
    for (int k = 0; k < 4; ++k) r[k] = hadamard_bwd<1>(r[k], c);
    if (A.sv) {
        // deterministic scatter: node c's 4 rows into the element's slot (one 16- or 32-byte store)
        if (valid) st4s<T>((T*)A.sv + 32 * idx + 4 * c, r[0], r[1], r[2], r[3]);
    } else if constexpr (sizeof(T) == 4) {
        // corners of this warp's 4 elements that are the same node add their rows in shared memory
        // first; one lane per node scatters (fewer float64 atomics; float64: the plain scatter is faster)
        const unsigned grp = __match_any_sync(0xffffffffu, valid ? id : -1 - lane);
        __syncwarp();   // every lane has read its moment columns
        st4s<T>(mrow, r[0], r[1], r[2], r[3]);
        __syncwarp();
        if (valid && lane == __ffs(grp) - 1) {
            T t[4] = {T(0), T(0), T(0), T(0)};
            for (unsigned gm = grp; gm; gm &= gm - 1) {
                T v[4];
                ld4s<T>(s_mw + (__ffs(gm) - 1) * MSTR, v);
                for (int k = 0; k < 4; ++k) t[k] += v[k];
            }
            scatter_t(A, id, t);
        }
    } else {
        if (valid) scatter_t(A, id, r);
    }
    __syncwarp();   // the rows and the moments are rewritten by later elements
}

// Gauss point c of the 2x2x2 rule (xi_k = +-1/sqrt(3) by bit k of c) in monomial form
template <class T>
__device__ __forceinline__ void gauss_monomials(int c, T m[8]) {
    const T gauss = (T)0.57735026918962576451;
    T xi[3];
    for (int k = 0; k < 3; ++k) xi[k] = ((c >> k) & 1) ? gauss : -gauss;
    monomials<T>(xi, m);
}

// Persistent: a block walks element groups with a grid stride; while it computes group g its
// threads already stream the node rows of group g + stride into the other shared buffer
// (cp.async), so the gather latency hides behind the arithmetic.  Each warp computes 4 of the
// group's 16 elements (interior_element).
// MINB: resident blocks per SM the register allocation is made for (4: up to 128 registers per thread;
// 5: up to 102, a few spills, one more block of warps to hide latency with)
template <class T, bool JV, int MINB = (sizeof(T) == 4 ? 4 : 2)>
__global__ void __launch_bounds__(IntShape<T>::THREADS, MINB) vms_interior(Args A, const int32_t* __restrict__ oconn,
                                                    const uint8_t* __restrict__ olev,
                                                    const uint16_t* __restrict__ oprob, int64_t n) {
    constexpr int EPB = IntShape<T>::EPB, ESTR = IntShape<T>::ESTR, MSTR = IntShape<T>::MSTR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s_nd = reinterpret_cast<T*>(smem_raw);          // [2][EPB][ESTR]: 8 rows of CS per element
    T* s_m = s_nd + 2 * EPB * ESTR;                     // [EPB][8][MSTR]
    const int c = threadIdx.x & 7, le = threadIdx.x >> 3, lane = threadIdx.x & 31;
    const int64_t ngroups = (n + EPB - 1) / EPB;
    int64_t gi = blockIdx.x;
    if (A.skip && *A.skip) return;   // a captured solver step after its cycle ended
    if (gi >= ngroups) return;
    auto corner_id = [&](int64_t grp) -> int32_t {
        int64_t idx = grp * EPB + le;
        if (idx >= n) idx = n - 1;
        return __ldg(oconn + 8 * idx + c);
    };
    // level (and problem) of this lane's element of a group, loaded a group ahead of its use
    auto level_prob = [&](int64_t grp) -> int {
        int64_t idx = grp * EPB + le;
        if (idx >= n) idx = n - 1;
        return (int)__ldg(olev + idx) | (oprob ? (int)oprob[idx] << 8 : -256);
    };
    auto row = [&](int buf) -> T* { return s_nd + (buf * EPB + le) * ESTR + c * CS; };
    int32_t id_cur = corner_id(gi);
    corner_async<T, JV>(A, id_cur, row(0));
    cp_commit();
    int32_t id_next = gi + gridDim.x < ngroups ? corner_id(gi + gridDim.x) : 0;
    int lp_cur = level_prob(gi);
    T m[8];
    gauss_monomials<T>(c, m);
    T* s_mw = s_m + (threadIdx.x & ~31u) * MSTR;
    int buf = 0;
    for (; gi < ngroups; gi += gridDim.x) {
        const int64_t gnext = gi + gridDim.x;
        if (gnext < ngroups) corner_async<T, JV>(A, id_next, row(buf ^ 1));
        cp_commit();
        const int32_t id_after = gnext + gridDim.x < ngroups ? corner_id(gnext + gridDim.x) : 0;
        const int lp_next = gnext < ngroups ? level_prob(gnext) : 0;
        cp_wait<1>();
        const int64_t idx = gi * EPB + le;
        interior_element<T, JV>(A, s_nd + (buf * EPB + le) * ESTR, s_mw, m, lane, idx, idx < n, lp_cur & 255,
                                lp_cur >> 8, id_cur);
        id_cur = id_next;
        id_next = id_after;
        lp_cur = lp_next;
        buf ^= 1;
    }
    cp_wait<0>();
}

// ------------------------------------------------------------------------------------------
// Intercepted elements: one warp per element
// ------------------------------------------------------------------------------------------
constexpr int WPB = 4;   // warps per block of the per-element surface kernel

// Warp epilogue of the per-element kernels: lane l holds the monomial moments M of its points;
// sum them over the lanes (transpose through shared memory s_m [32][32 + pad]), run the backward
// butterfly so lane 4 a + k holds row (node a, component k), and scatter node a from lane 4 a.
// my_id: the node id of corner (lane & 7).
// extra: a float64 addend of this lane's row (node a = lane / 4, component lane % 4).  With the
// deterministic scatter the 32 rows go to a slot instead: vdst (element precision, volume terms)
// or sdst (float64, surface terms), row a * 4 + k at lane 4 a + k.
template <class T>
__device__ __forceinline__ void warp_scatter_moments(const Args& A, const T M[32], T* s_m, int lane, int32_t my_id,
                                                     double extra = 0.0, T* vdst = nullptr, double* sdst = nullptr) {
    constexpr int MSTR = 32 + 16 / (int)sizeof(T);
    T* mrow = s_m + lane * MSTR;
    for (int k = 0; k < 32; k += 4) st4s<T>(mrow + k, M[k], M[k + 1], M[k + 2], M[k + 3]);
    __syncwarp();
    T acc = T(0);
#pragma unroll 8
    for (int t = 0; t < 32; ++t) acc += s_m[t * MSTR + lane];
    acc = hadamard_bwd<4>(acc, lane >> 2);
    if (vdst) { vdst[lane] = acc; return; }
    const double row = (double)acc + extra;
    if (sdst) { sdst[lane] = row; return; }
    const int a = lane >> 2;
    double r[4];
    for (int k = 0; k < 4; ++k) r[k] = __shfl_sync(0xffffffffu, row, (lane & ~3) + k);
    const int32_t id = __shfl_sync(0xffffffffu, my_id, a);
    if ((lane & 3) == 0) scatter(A, id, r);
}

// One Intercepted element on one warp: lane l evaluates sub-cell points l, l + 32, ... and accumulates
// their monomial moments, summed over the lanes at the end (warp_scatter_moments).  s_nd [8 * CS] and
// s_m [32 * MSTR] are the warp's shared rows; idx the element's position in the list.
template <class T, bool JV>
__device__ __forceinline__ void cut_element(const Args& A, const int32_t* __restrict__ list, const int64_t* __restrict__ off,
                                            const void* __restrict__ pts, int64_t idx, T* s_nd, T* s_m, int lane) {
    typedef typename std::conditional<JV, Dual<T>, T>::type S;
    const int32_t e = list[idx];
    // every 8-lane group gathers the 8 corner rows and forms their monomial coefficients; lanes 0-7 store them
    const int c8 = lane & 7;
    const int32_t my_id = A.conn[8 * (int64_t)e + c8];
    {
        T rw[CS];
        corner_data<T, JV>(A, my_id, rw);
        for (int j = 0; j < 7; ++j) rw[j] = hadamard_fwd(rw[j], c8);
        if (JV)
            for (int j = 0; j < 7; ++j) rw[CT + j] = hadamard_fwd(rw[CT + j], c8);
        if (A.ndf)
            for (int j = 0; j < 3; ++j) rw[CF + j] = hadamard_fwd(rw[CF + j], c8);
        if (lane < 8)
            for (int j = 0; j < CS; ++j) s_nd[lane * CS + j] = rw[j];
    }
    __syncwarp();
    const T g = lvl_g<T>(A, A.lev[e]);
    const T det = lvl_w<T>(A, A.lev[e]);
    const Phys<T> P(A, prob_of(A, e));
    // lane l evaluates points q0 + l, q0 + l + 32, ... and accumulates their monomial moments
    T M[32];
    for (int k = 0; k < 32; ++k) M[k] = T(0);
    const int64_t q0 = off[idx], q1 = off[idx + 1];
    for (int64_t q = q0 + lane; q < q1; q += 32) {
        T pt[4];
        load_pt<T>(pts, q, pt);
        T m[8];
        monomials<T>(pt, m);
        S cf[16];
        vms_point_modal<S, T>(A, P, m, s_nd, CS, g, cf);
        const T wq = pt[3] * det, wqg = wq * g;
        T w16[16];
        for (int k = 0; k < 16; ++k) w16[k] = ((k < 3 || k == 12) ? wq : wqg) * Pick<T, JV>::get(cf[k]);
        add_moments<T>(m, w16, M);
    }
    warp_scatter_moments<T>(A, M, s_m, lane, my_id, 0.0, A.sv ? (T*)A.sv + 32 * (A.n_out_slots + idx) : nullptr);
}

// W warps per block (a tile shape the autotuner picks); `order` (or null) permutes the list
template <class T, bool JV, int W>
__global__ void __launch_bounds__(32 * W, (sizeof(T) == 4 ? 16 : 8) / W) vms_cut(Args A, const int32_t* __restrict__ list,
                                                    const int64_t* __restrict__ off, const void* __restrict__ pts,
                                                    const int32_t* __restrict__ order, int64_t n) {
    constexpr int PAD = 16 / (int)sizeof(T), MSTR = 32 + PAD;
    __shared__ __align__(16) T s_nd[W][8 * CS];
    __shared__ __align__(16) T s_m[W][32 * MSTR];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t slot = (int64_t)blockIdx.x * W + w;
    if (A.skip && *A.skip) return;   // a captured solver step after its cycle ended
    if (slot >= n) return;
    cut_element<T, JV>(A, list, off, pts, order ? (int64_t)order[slot] : slot, &s_nd[w][0], &s_m[w][0], lane);
}

// ------------------------------------------------------------------------------------------
// Nitsche surface terms (Eq. weakbc), one thread per surface point: elements hosting few points
// ------------------------------------------------------------------------------------------
template <class T, bool JV>
__device__ __forceinline__ void surface_point(const Args& A, const int32_t* __restrict__ el, const double* __restrict__ xr,
                                              const double* __restrict__ nr, const double* __restrict__ wr, int64_t i) {
    typedef typename std::conditional<JV, Dual<T>, T>::type S;
    NitschePoint<S, T> P;
    const int32_t e = el[i];
    nitsche_fields<S, T, JV, false>(A, e, i, xr + 3 * i, nr + 3 * i, P);
    const T w = (T)wr[i];
    // (the penalty is added per element in float64 by nitsche_penalty)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        S t[4];
        nitsche_rows<S, T, false>(A, P, c, T(0), t);
        double r[4];
        for (int k = 0; k < 4; ++k) r[k] = (double)(w * Pick<T, JV>::get(t[k]));
        if (A.ss) {
            double* d = A.ss + 32 * (A.n_dense_slots + i) + 4 * c;
            reinterpret_cast<double2*>(d)[0] = make_double2(r[0], r[1]);
            reinterpret_cast<double2*>(d)[1] = make_double2(r[2], r[3]);
        } else {
            scatter(A, P.ids[c], r);
        }
    }
}

template <class T, bool JV>
__global__ void __launch_bounds__(128) nitsche(Args A, const int32_t* __restrict__ el, const double* __restrict__ xr,
                                               const double* __restrict__ nr, const double* __restrict__ wr,
                                               const double* __restrict__ taub, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (A.skip && *A.skip) return;   // a captured solver step after its cycle ended
    surface_point<T, JV>(A, el, xr, nr, wr, i);
}

// ------------------------------------------------------------------------------------------
// Nitsche surface terms (Eq. weakbc), one warp per element hosting many surface points; lane l takes
// points l, l + 32, ... of the element.  Per point the 4 rows of corner c are
//   t_k = phi_c [tau_B d_k - tr_k - [u.n < 0] rho (u.n) d_k] - mu g sum_j d_j phi_c (n_j d_k + n_k d_j),
//   t_p = -phi_c (d.n),   d = u_s - g, tr = -p n + 2 mu eps(u) n,
// i.e. coefficients of phi_c and of its reference gradient, accumulated as monomial moments.
// ------------------------------------------------------------------------------------------
template <class T, bool JV>
__device__ __forceinline__ void surface_element(const Args& A, const int32_t* __restrict__ list, const int64_t* __restrict__ off,
                                                const double* __restrict__ xr, const double* __restrict__ nr,
                                                const double* __restrict__ wr, int64_t idx, T* s_nd, T* s_m, int lane) {
    typedef typename std::conditional<JV, Dual<T>, T>::type S;
    const int32_t e = list[idx];
    // corner rows: u_s (0-2), p (3), jump d = u_s - g_body formed in float64 (4-6), tangents at CT
    // (the penalty is added per element in float64 by nitsche_penalty)
    const int c8 = lane & 7;
    const int32_t my_id = A.conn[8 * (int64_t)e + c8];
    {
        T a8[8], t8[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        ld8<T>(A.ndv, my_id, a8);
        if (JV) ld8<T>(A.ndt, my_id, t8);
        double u4[4], up4[4];
        gather(A, A.U, my_id, u4);
        if (!A.theta1) gather(A, A.Up, my_id, up4);
        T rw[CS];
        for (int k = 0; k < 3; ++k) {
            const double usk = A.theta1 ? u4[k] : A.theta * u4[k] + (1.0 - A.theta) * up4[k];
            rw[k] = a8[k];
            rw[4 + k] = (T)(usk - A.g[k]);
            rw[CT + k] = t8[k];
            rw[CT + 4 + k] = t8[k];
        }
        rw[3] = a8[3];
        rw[CT + 3] = t8[3];
        for (int j = 0; j < 7; ++j) rw[j] = hadamard_fwd(rw[j], c8);
        if (JV)
            for (int j = 0; j < 7; ++j) rw[CT + j] = hadamard_fwd(rw[CT + j], c8);
        if (lane < 8) {
            for (int j = 0; j < 7; ++j) s_nd[lane * CS + j] = rw[j];
            if (JV)
                for (int j = 0; j < 7; ++j) s_nd[lane * CS + CT + j] = rw[CT + j];
        }
    }
    __syncwarp();
    const T g = lvl_g<T>(A, A.lev[e]);
    T mu, rho;
    {
        const Phys<T> Ph(A, prob_of(A, e));
        mu = Ph.mu;
        rho = Ph.rho;
    }
    T M[32];
    for (int k = 0; k < 32; ++k) M[k] = T(0);
    const int64_t q0 = off[idx], q1 = off[idx + 1];
    for (int64_t q = q0 + lane; q < q1; q += 32) {
        T xi[3], nn[3], m[8];
        for (int k = 0; k < 3; ++k) { xi[k] = (T)xr[3 * q + k]; nn[k] = (T)nr[3 * q + k]; }
        // the jump relative to g_body at the corners, corrected to this point's g (its value enters
        // the tangent of the inflow term)
        T dg[3] = {T(0), T(0), T(0)};
        if (A.gpts) {
            const double* gq = point_g(A, q);
            for (int k = 0; k < 3; ++k) dg[k] = (T)(A.g[k] - gq[k]);
        }
        monomials<T>(xi, m);
        // u_s, grad u_s, p, d at the point
        S us[3], Gu[3][3], p, d[3];
        for (int i = 0; i < 3; ++i) { us[i] = zero<S>(); d[i] = zero<S>(); for (int j = 0; j < 3; ++j) Gu[i][j] = zero<S>(); }
        p = zero<S>();
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const T* r = &s_nd[t * CS];
            S a[7];
            for (int j = 0; j < 7; ++j) a[j] = make<S, T>(r[j], JV ? r[CT + j] : T(0));
            for (int i = 0; i < 3; ++i) {
                us[i] = madd(m[t], a[i], us[i]);
                d[i] = madd(m[t], a[4 + i], d[i]);
            }
            p = madd(m[t], a[3], p);
            for (int k = 0; k < 3; ++k)
                if (t & (1 << k))
                    for (int i = 0; i < 3; ++i) Gu[i][k] = madd(m[t ^ (1 << k)], a[i], Gu[i][k]);
        }
        for (int i = 0; i < 3; ++i) {
            d[i] = d[i] + dg[i];
            for (int j = 0; j < 3; ++j) Gu[i][j] = g * Gu[i][j];
        }
        const S un = mmadd(us[2], S(make<S, T>(nn[2], T(0))), mmadd(us[1], S(make<S, T>(nn[1], T(0))), us[0] * nn[0]));
        const S dn = madd(nn[2], d[2], madd(nn[1], d[1], nn[0] * d[0]));
        const bool inflow = value(un) < T(0);
        const T wq = (T)wr[q], wqg = wq * g;
        T c[16];
        for (int k = 0; k < 3; ++k) {
            S tr = (-nn[k]) * p;
            for (int j = 0; j < 3; ++j) tr = madd(mu * nn[j], Gu[k][j] + Gu[j][k], tr);
            S fk = T(-1) * tr;
            if (inflow) fk = fk - rho * (un * d[k]);
            c[k] = wq * Pick<T, JV>::get(fk);
            for (int j = 0; j < 3; ++j) c[3 + 3 * k + j] = (-wqg * mu) * Pick<T, JV>::get(madd(nn[j], d[k], nn[k] * d[j]));
        }
        c[12] = -wq * Pick<T, JV>::get(dn);
        c[13] = c[14] = c[15] = T(0);
        add_moments<T>(m, c, M);
    }
    warp_scatter_moments<T>(A, M, s_m, lane, my_id, 0.0, nullptr, A.ss ? A.ss + 32 * idx : nullptr);
}

template <class T, bool JV>
__global__ void __launch_bounds__(32 * WPB, sizeof(T) == 4 ? 2 : 1) nitsche_el(Args A, const int32_t* __restrict__ list,
                                                    const int64_t* __restrict__ off, const double* __restrict__ xr,
                                                    const double* __restrict__ nr, const double* __restrict__ wr,
                                                    const double* __restrict__ taub, int64_t n) {
    constexpr int PAD = 16 / (int)sizeof(T), MSTR = 32 + PAD;
    __shared__ __align__(16) T s_nd[WPB][8 * CS];
    __shared__ __align__(16) T s_m[WPB][32 * MSTR];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t idx = (int64_t)blockIdx.x * WPB + w;
    if (A.skip && *A.skip) return;   // a captured solver step after its cycle ended
    if (idx >= n) return;
    surface_element<T, JV>(A, list, off, xr, nr, wr, idx, &s_nd[w][0], &s_m[w][0], lane);
}

// ------------------------------------------------------------------------------------------
// One persistent launch over the volume quadrature buckets.  Every warp drains a device work queue
// on its own: first the Intercepted elements (8 .. 4096 sub-cell points), one per claim, longest
// first (the cost model of Eq. Wpart: a warp's time grows with its rounds of 32 points); then the
// Out elements, 4 per warp item, kFusedChunk items per claim, with their node rows double-buffered
// by cp.async as in vms_interior.  Longest items first, then small uniform ones, keeps every SM
// busy to the end whatever the mix (one mesh or many problems of a batch).  The surface terms run
// as their own kernels beside this one (their register budget would spill in it).
// ------------------------------------------------------------------------------------------
constexpr int kFusedWarps = 4;   // warps per block
constexpr int kFusedChunk = 8;   // Out warp items per claim

struct FusedQueue {
    const uint32_t* items;       // Intercepted-list positions, by decreasing point count
    int64_t n_items;
    unsigned long long* cnt;     // [3] claimed items, claimed Out warp items, finished blocks (zero at launch)
    const int32_t* oconn;
    const uint8_t* olev;
    const uint16_t* oprob;
    int64_t n_out;
    const int32_t* cut_list;
    const int64_t* cut_off;
    const void* cut_pts;
    int heavy_warps;             // warps per block that take the costly items before the Out elements
};

template <class T> struct FusedShape {
    static constexpr int ESTR = IntShape<T>::ESTR, MSTR = IntShape<T>::MSTR;
    // per warp: the Out layout (2 buffers x 4 elements of rows, 32 moment rows); the per-element
    // layouts (8 rows, 32 moment rows) fit inside it
    static constexpr int WARP = 2 * 4 * ESTR + 32 * MSTR;
    static_assert(8 * CS + 32 * MSTR <= WARP, "per-element layout");
    static_assert((WARP * sizeof(T)) % 16 == 0 && (8 * CS * sizeof(T)) % 16 == 0, "16-byte rows");
    static constexpr size_t smem = (size_t)kFusedWarps * WARP * sizeof(T);
};

template <class T, bool JV>
__global__ void __launch_bounds__(32 * kFusedWarps, sizeof(T) == 4 ? 4 : 2) vms_fused(Args A, FusedQueue Q) {
    constexpr int ESTR = FusedShape<T>::ESTR, MSTR = FusedShape<T>::MSTR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    T* base = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * FusedShape<T>::WARP;
    if (A.skip && *A.skip) return;   // a captured solver step after its cycle ended
    // the costly items, one per claim
    auto drain_costly = [&]() {
        for (;;) {
            unsigned long long h = 0;
            if (lane == 0) h = atomicAdd(Q.cnt, 1ull);
            h = __shfl_sync(0xffffffffu, h, 0);
            if ((int64_t)h >= Q.n_items) break;
            cut_element<T, JV>(A, Q.cut_list, Q.cut_off, Q.cut_pts, (int64_t)Q.items[h], base, base + 8 * CS, lane);
            __syncwarp();   // the shared rows are reused by the next item
        }
    };
    // 1. the first heavy_warps warps of every block start on the costly items (the others go straight
    //    to the Out elements, so latency-bound costly work shares each SM with arithmetic-bound Out work)
    const bool heavy_first = (int)(threadIdx.x >> 5) < Q.heavy_warps;
    // 2. Out elements
    auto drain_out = [&]() {
        if (Q.n_out > 0) {
            const int c = lane & 7, le = lane >> 3;
            const int64_t n_wi = (Q.n_out + 3) / 4;
            int64_t pos = 0, end = 0;
            bool more = true;
            auto claim = [&]() -> int64_t {   // warp-uniform
                if (pos < end) return pos++;
                if (!more) return -1;
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(Q.cnt + 1, (unsigned long long)kFusedChunk);
                b = __shfl_sync(0xffffffffu, b, 0);
                if ((int64_t)b >= n_wi) { more = false; return -1; }
                pos = (int64_t)b + 1;
                end = (int64_t)b + kFusedChunk < n_wi ? (int64_t)b + kFusedChunk : n_wi;
                return (int64_t)b;
            };
            auto corner_id = [&](int64_t wi) -> int32_t {
                int64_t idx = 4 * wi + le;
                if (idx >= Q.n_out) idx = Q.n_out - 1;
                return __ldg(Q.oconn + 8 * idx + c);
            };
            auto level_prob = [&](int64_t wi) -> int {   // loaded an item ahead of its use
                int64_t idx = 4 * wi + le;
                if (idx >= Q.n_out) idx = Q.n_out - 1;
                return (int)__ldg(Q.olev + idx) | (Q.oprob ? (int)Q.oprob[idx] << 8 : -256);
            };
            auto row = [&](int buf) -> T* { return base + (buf * 4 + le) * ESTR + c * CS; };
            T* s_mw = base + 8 * ESTR;
            int64_t cur = claim();
            if (cur >= 0) {
                T m[8];
                gauss_monomials<T>(c, m);
                int32_t id_cur = corner_id(cur);
                corner_async<T, JV>(A, id_cur, row(0));
                cp_commit();
                int lp_cur = level_prob(cur);
                int64_t nxt = claim();
                int32_t id_next = nxt >= 0 ? corner_id(nxt) : 0;
                int buf = 0;
                while (cur >= 0) {
                    if (nxt >= 0) corner_async<T, JV>(A, id_next, row(buf ^ 1));
                    cp_commit();
                    const int64_t aft = nxt >= 0 ? claim() : -1;
                    const int32_t id_after = aft >= 0 ? corner_id(aft) : 0;
                    const int lp_next = nxt >= 0 ? level_prob(nxt) : 0;
                    cp_wait<1>();
                    const int64_t idx = 4 * cur + le;
                    interior_element<T, JV>(A, base + (buf * 4 + le) * ESTR, s_mw, m, lane, idx, idx < Q.n_out,
                                            lp_cur & 255, lp_cur >> 8, id_cur);
                    cur = nxt;
                    nxt = aft;
                    id_cur = id_next;
                    id_next = id_after;
                    lp_cur = lp_next;
                    buf ^= 1;
                }
                cp_wait<0>();
            }
        }
    };
    // one call site each (the bodies are inlined once): costly items then Out elements, or the reverse
    for (int phase = 0; phase < 2; ++phase) {
        if ((phase == 0) == heavy_first) drain_costly();
        else drain_out();
    }
    // 3. the last block to finish zeroes the counters for the next launch (every claim of every block
    //    precedes its count here)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(Q.cnt + 2, 1ull) == (unsigned long long)gridDim.x - 1) {
            Q.cnt[0] = 0;
            Q.cnt[1] = 0;
            Q.cnt[2] = 0;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------------------------------
// Nitsche penalty in float64, one thread per surface-hosting element.  Over the element's surface
// points the penalty rows are linear in the corner values with a matrix that does not depend on the
// state,
//   r_{a,k} = sum_q w_q tau_B(q) phi_a(x_q) (u_s(x_q) - g(x_q))_k
//           = C_b mu sum_b Pen_ab (u_s,b - g_body)_k + C_b mu sum_q (w_q / h_b) phi_a (g_body - g_q)_k,
//   Pen_ab = sum_q (w_q / h_b) phi_a(x_q) phi_b(x_q)      (float64, built with the mesh),
// so each call costs one 8 x 8 x 3 product per element instead of float64 work per point (the second
// sum only with per-point velocities).  J v: the tangent theta v in place of u_s - g_body.  The rows
// go to the element's surface slot (dense bucket) or to the slot of its first point (sparse bucket),
// after the surface kernel wrote it, or by float64 atomics.
// ------------------------------------------------------------------------------------------
template <bool JV>
__global__ void __launch_bounds__(128) nitsche_penalty(Args A, const int32_t* __restrict__ pe,
                                                       const int64_t* __restrict__ pq, const int64_t* __restrict__ pslot,
                                                       const double* __restrict__ pen, const double* __restrict__ xr,
                                                       const double* __restrict__ wr, const double* __restrict__ taub,
                                                       int64_t n) {
    // eight threads per element: thread c fetches corner c's jump, then forms row c
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t >> 3;
    const int c = (int)(t & 7);
    if (A.skip && *A.skip) return;   // a captured solver step after its cycle ended (uniform over the grid)
    const bool live = i < n;
    const int64_t ii = live ? i : n - 1;
    const int32_t e = pe[ii];
    const double cbmu = A.Cb * Phys<double>(A, prob_of(A, e)).mu;
    const int32_t id = A.conn[8 * (int64_t)e + c];
    double dc[3];
    if (JV) {
        double v4[4];
        gather(A, A.V, id, v4);
        for (int k = 0; k < 3; ++k) dc[k] = A.theta * v4[k];
    } else {
        double u4[4], up4[4];
        gather(A, A.U, id, u4);
        if (!A.theta1) gather(A, A.Up, id, up4);
        for (int k = 0; k < 3; ++k) dc[k] = (A.theta1 ? u4[k] : A.theta * u4[k] + (1.0 - A.theta) * up4[k]) - A.g[k];
    }
    const double* P = pen + 36 * ii;   // upper triangle, row by row: (a, b >= a) at a * 8 - a (a - 1) / 2 + b - a
    double r[3] = {0.0, 0.0, 0.0};
    const unsigned base = threadIdx.x & 31 & ~7u;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int lo = c < b ? c : b, hi = c < b ? b : c;
        const double m = cbmu * P[lo * 8 - lo * (lo - 1) / 2 + hi - lo];
        for (int k = 0; k < 3; ++k) r[k] = fma(m, __shfl_sync(0xffffffffu, dc[k], base | b), r[k]);
    }
    if (!live) return;
    if (!JV && A.gpts) {
        for (int64_t q = pq[i]; q < pq[i + 1]; ++q) {
            const double* gq = point_g(A, q);
            double phi[8];
            basis_values_d(xr + 3 * q, phi);
            const double cq = cbmu * wr[q] * taub[q] * phi[c];
            for (int k = 0; k < 3; ++k) r[k] = fma(cq, A.g[k] - gq[k], r[k]);
        }
    }
    if (A.ss) {
        double* dst = A.ss + 32 * pslot[i] + 4 * c;
        for (int k = 0; k < 3; ++k) dst[k] += r[k];
    } else {
        const double rr[4] = {r[0], r[1], r[2], 0.0};
        scatter(A, id, rr);
    }
}

// ------------------------------------------------------------------------------------------
// strong rows
// ------------------------------------------------------------------------------------------
__global__ void strong_rows(Args A, const uint8_t* __restrict__ flag, const uint8_t* __restrict__ umask,
                            const double* __restrict__ uval, double ux, double uy, double uz, int jv) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= A.n_nodes) return;
    if (A.skip && *A.skip) return;   // a captured solver step after its cycle ended
    const uint8_t f = flag[n];
    uint8_t mask;
    double gv[4];
    if (umask) {
        mask = umask[n];
        for (int k = 0; k < 4; ++k) gv[k] = uval[4 * n + k];
    } else {
        mask = f & 15;
        gv[0] = ux; gv[1] = uy; gv[2] = uz; gv[3] = 0.0;
    }
    if (f & 16) {
        for (int k = 0; k < 4; ++k)
            if (!((mask >> k) & 1)) { mask |= (uint8_t)(1 << k); gv[k] = k < 3 ? A.g[k] : 0.0; }
    }
    if (!mask) return;
    const double* src = jv ? A.V : A.U;
    for (int k = 0; k < 4; ++k)
        if ((mask >> k) & 1) A.out[4 * n + k] = jv ? src[4 * n + k] : src[4 * n + k] - gv[k];
}

// float-float accumulation on the FP32 pipe (Knuth's TwoSum): hi + lo carries the sum of floats to
// about 48 bits, in a fixed order
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// Deterministic o2n (Algorithm 2): one thread per node sums the slot rows of its incidence list in
// list order (a hanging corner's rows times 1/2 or 1/4 for each parent; float-float in mixed
// precision), then the node's strong rows take U - g (R) or v (J v) as in strong_rows.  The kernel is
// bound by the latency of dependent loads, so: the first kIncHead codes of a node sit at a fixed
// place (one aligned 32-byte load, no list offset to fetch first), the rest follow in CSR form; and
// every batch of codes has all its row loads issued before the first sum.  Writes every row of out:
// no zeroing before the call.
template <class T> struct GatherBatch { static constexpr int value = sizeof(T) == 4 ? 8 : 4; };

// sums the rows of entries e[0 .. B) (kIncNone: none) in order
template <class T, int B>
__device__ __forceinline__ void gather_batch(const Args& A, const uint32_t e[B], int64_t nv, double acc[4], float hi[4],
                                             float lo[4]) {
    T v[B][4];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const int64_t sl = (int64_t)(e[i] >> 5);
        if (e[i] != kIncNone && sl < nv) ld4<T>((const T*)A.sv + 32 * sl, e[i] & 7, v[i]);
    }
#pragma unroll
    for (int i = 0; i < B; ++i) {
        if (e[i] == kIncNone) continue;
        const int c = (int)(e[i] & 7), wc = (int)((e[i] >> 3) & 3);
        const int64_t sl = (int64_t)(e[i] >> 5);
        if (sl < nv) {
            const T w = wc == 0 ? T(1) : (wc == 1 ? T(0.5) : T(0.25));
            if constexpr (sizeof(T) == 4) {
                for (int k = 0; k < 4; ++k) ff_add(hi[k], lo[k], w * v[i][k]);
            } else {
                for (int k = 0; k < 4; ++k) acc[k] += w * v[i][k];
            }
        } else {   // a float64 surface slot
            const double* d = A.ss + 32 * (sl - nv) + 4 * c;
            const double2 x = reinterpret_cast<const double2*>(d)[0], y = reinterpret_cast<const double2*>(d)[1];
            const double w = wc == 0 ? 1.0 : (wc == 1 ? 0.5 : 0.25);
            acc[0] += w * x.x; acc[1] += w * x.y; acc[2] += w * y.x; acc[3] += w * y.y;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) node_gather(Args A, const uint32_t* __restrict__ head,
                                                   const int64_t* __restrict__ ptr, const uint32_t* __restrict__ inc,
                                                   int64_t nv, const uint8_t* __restrict__ flag,
                                                   const uint8_t* __restrict__ umask, const double* __restrict__ uval,
                                                   double ux, double uy, double uz, int jv) {
    static_assert(kIncHead == 8, "head of two 16-byte loads");
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= A.n_nodes) return;
    if (A.skip && *A.skip) return;   // a captured solver step after its cycle ended
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    const uint4* hp = reinterpret_cast<const uint4*>(head + kIncHead * n);
    const uint4 h0 = __ldg(hp), h1 = __ldg(hp + 1);
    const int64_t q0 = ptr[n], q1 = ptr[n + 1];   // independent of the head: loaded alongside
    {
        constexpr int B = GatherBatch<T>::value;
        const uint32_t e8[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
        for (int b = 0; b < 8; b += B) gather_batch<T, B>(A, e8 + b, nv, acc, hi, lo);
    }
    for (int64_t q = q0; q < q1; q += GatherBatch<T>::value) {
        constexpr int B = GatherBatch<T>::value;
        uint32_t e[B];
#pragma unroll
        for (int i = 0; i < B; ++i) e[i] = q + i < q1 ? __ldg(inc + q + i) : kIncNone;
        gather_batch<T, B>(A, e, nv, acc, hi, lo);
    }
    if constexpr (sizeof(T) == 4)
        for (int k = 0; k < 4; ++k) acc[k] += f2d(hi[k]) + f2d(lo[k]);
    // strong rows (as strong_rows)
    const uint8_t f = flag[n];
    uint8_t mask;
    double gv[4];
    if (umask) {
        mask = umask[n];
        for (int k = 0; k < 4; ++k) gv[k] = uval[4 * n + k];
    } else {
        mask = f & 15;
        gv[0] = ux; gv[1] = uy; gv[2] = uz; gv[3] = 0.0;
    }
    if (f & 16) {
        for (int k = 0; k < 4; ++k)
            if (!((mask >> k) & 1)) { mask |= (uint8_t)(1 << k); gv[k] = k < 3 ? A.g[k] : 0.0; }
    }
    if (mask) {
        const double* src = jv ? A.V : A.U;
        for (int k = 0; k < 4; ++k)
            if ((mask >> k) & 1) acc[k] = jv ? src[4 * n + k] : src[4 * n + k] - gv[k];
    }
    double2* o = reinterpret_cast<double2*>(A.out + 4 * n);
    o[0] = make_double2(acc[0], acc[1]);
    o[1] = make_double2(acc[2], acc[3]);
}

// optional event pair around a launch (profiling); never for calls on a caller's workspace
// (imga_jvp_noalloc), which create no events and leave the mesh untouched
struct Timed {
    Mesh* m;
    int k, nk;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    Timed(const Mesh& mesh, int kind, cudaStream_t st, int launches = 1, bool enable = true)
        : m(const_cast<Mesh*>(&mesh)), k(kind), nk(launches), s(st) {
        if (!enable || !m->profiling) return;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    ~Timed() {
        if (!a) return;
        cudaEventRecord(b, s);
        m->prof_ev[k].push_back({(void*)a, (void*)b, nk});
    }
};

template <class T, bool JV>
void launch_cut(const Mesh& m, const Args& A, cudaStream_t s, int wpb, int lpt) {
    const int64_t nc = (int64_t)m.cut_list.size();
    const void* pts = std::is_same<T, float>::value ? (const void*)m.d.cut_pts_f : (const void*)m.d.cut_pts;
    const int32_t* order = lpt ? m.d.cut_order : nullptr;
    switch (wpb) {
        case 2: vms_cut<T, JV, 2><<<(unsigned)((nc + 1) / 2), 64, 0, s>>>(A, m.d.cut_list, m.d.cut_off, pts, order, nc); break;
        case 8:
            if constexpr (sizeof(T) == 4) {
                vms_cut<T, JV, 8><<<(unsigned)((nc + 7) / 8), 256, 0, s>>>(A, m.d.cut_list, m.d.cut_off, pts, order, nc);
                break;
            }
            [[fallthrough]];
        default: vms_cut<T, JV, 4><<<(unsigned)((nc + 3) / 4), 128, 0, s>>>(A, m.d.cut_list, m.d.cut_off, pts, order, nc);
    }
}

template <class T, bool JV, int MINB = (sizeof(T) == 4 ? 4 : 2)>
int interior_blocks_per_sm();
template <class T, bool JV>
void launch_interior(const Mesh& m, const Args& A, cudaStream_t s, int bps);

// Autotuner of the Intercepted-element bucket: with the node data of this call prepared, time every
// (warps per block, element order) candidate on the call's own inputs (3 launches each after one
// untimed) and keep the fastest; then the Out-element bucket: the persistent interior kernel with
// 1 .. 4 resident blocks per SM, and 5 with the smaller register allocation (float).  Writes into the output vector, which the call then recomputes.
template <class T, bool JV>
int autotune_cut(Mesh& m, Args A, cudaStream_t s) {
    const int64_t nc = (int64_t)m.cut_list.size();
    Mesh::CutTune& ct = m.cut_tune[sizeof(T) == 4][JV];
    m.tune_pending[sizeof(T) == 4][JV] = false;
    if (nc > 0 && !m.d.cut_order) {   // longest first: positions of the list by decreasing point count
        std::vector<int32_t> ord(nc);
        for (int64_t i = 0; i < nc; ++i) ord[i] = (int32_t)i;
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
            return m.cut_off[a + 1] - m.cut_off[a] > m.cut_off[b + 1] - m.cut_off[b];
        });
        if (cudaMalloc((void**)&m.d.cut_order, nc * sizeof(int32_t)) != cudaSuccess ||
            cudaMemcpy(m.d.cut_order, ord.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
            return 1;
    }
    const int64_t next = m.n_nodes() + m.n_hang();
    T* ndv = node_workspace<T>(m, nullptr);
    A.ndv = ndv;
    A.ndt = ndv + 8 * next;
    A.ndf = A.F ? ndv + 16 * next : nullptr;
    launch_node_prep<T, JV>(A, ndv, (T*)A.ndt, (T*)A.ndf, s);
    const int wpbs[3] = {2, 4, 8};
    const int nw = sizeof(T) == 4 ? 3 : 2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int wi = 0; wi < nw && nc > 0; ++wi)
        for (int lpt = 0; lpt < 2; ++lpt) {
            launch_cut<T, JV>(m, A, s, wpbs[wi], lpt);
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3; ++r) launch_cut<T, JV>(m, A, s, wpbs[wi], lpt);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.f;
            m.cut_tune_ms[sizeof(T) == 4][JV][2 * wi + lpt] = ms;
            if (ms < best) { best = ms; ct.wpb = wpbs[wi]; ct.lpt = lpt; }
        }
    // the Out-element bucket: the persistent interior kernel with 1 .. (occupancy limit) blocks per SM
    const int64_t no = (int64_t)m.out_list.size();
    constexpr int EPB = Epb<T>::value;
    int maxb = std::min(4, interior_blocks_per_sm<T, JV>());
    if constexpr (sizeof(T) == 4)
        if (maxb == 4 && interior_blocks_per_sm<T, JV, 5>() >= 5) maxb = 5;
    float best_out = 1e30f;
    for (int b = 1; b <= maxb && no > 0; ++b) {
        auto run = [&]() { launch_interior<T, JV>(m, A, s, b); };
        run();
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) run();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        m.out_tune_ms[sizeof(T) == 4][JV][b - 1] = ms;
        if (ms < best_out) { best_out = ms; m.out_bps[sizeof(T) == 4][JV] = b; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// Resident CTAs of the persistent interior kernel per SM (queried once; also sets its dynamic smem opt-in).
template <class T, bool JV, int MINB>
int interior_blocks_per_sm() {
    static int bps = 0;
    if (bps == 0) {
        const size_t smem = IntShape<T>::smem;
        int b = 0;
        cudaFuncSetAttribute(vms_interior<T, JV, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, vms_interior<T, JV, MINB>, 8 * Epb<T>::value, smem);
        bps = b < 1 ? 1 : b;
    }
    return bps;
}

// The persistent interior kernel at bps resident blocks per SM: the 5-block register allocation for
// bps = 5 (float only), else the default one.
template <class T, bool JV>
void launch_interior(const Mesh& m, const Args& A, cudaStream_t s, int bps) {
    const int64_t no = (int64_t)m.out_list.size();
    constexpr int EPB = Epb<T>::value;
    const int64_t grid = std::min<int64_t>((no + EPB - 1) / EPB, (int64_t)bps * m.n_sm);
    if constexpr (sizeof(T) == 4) {
        if (bps >= 5) {
            vms_interior<T, JV, 5><<<(unsigned)grid, 8 * EPB, IntShape<T>::smem, s>>>(A, m.d.out_conn, m.d.out_lev, m.d.out_prob, no);
            return;
        }
    }
    vms_interior<T, JV><<<(unsigned)grid, 8 * EPB, IntShape<T>::smem, s>>>(A, m.d.out_conn, m.d.out_lev, m.d.out_prob, no);
}

// Resident CTAs of the fused kernel per SM (queried once; also sets its dynamic smem opt-in).
template <class T, bool JV>
int fused_blocks_per_sm() {
    static int bps = 0;
    if (bps == 0) {
        const size_t smem = FusedShape<T>::smem;
        int b = 0;
        cudaFuncSetAttribute(vms_fused<T, JV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, vms_fused<T, JV>, 32 * kFusedWarps, smem);
        bps = b < 1 ? 1 : b;
    }
    return bps;
}

template <class T, bool JV>
void launch_penalty(const Mesh& m, const Args& A, cudaStream_t s, bool timed) {
    const int64_t np = (int64_t)m.pen_elem.size();
    if (np <= 0) return;
    Timed t(m, 2, s, 1, timed);
    nitsche_penalty<JV><<<(unsigned)((8 * np + 127) / 128), 128, 0, s>>>(A, m.d.pen_elem, m.d.pen_q, m.d.pen_slot, m.d.pen,
                                                                        m.d.sq_x, m.d.sq_w, m.d.sq_taub, np);
}

// the surface buckets: thread-per-point and warp-per-element Nitsche kernels, then the float64
// penalty (same stream: the slots hold their rows first)
template <class T, bool JV>
void launch_surface(const Mesh& m, const Args& A, cudaStream_t ss, bool timed) {
    const int64_t nsp = m.n_sq_sparse, nse = m.n_sq_elem;
    if (nsp > 0) {
        Timed t(m, 2, ss, 1, timed);
        nitsche<T, JV><<<(unsigned)((nsp + 127) / 128), 128, 0, ss>>>(A, m.d.sq_elem, m.d.sq_x, m.d.sq_n, m.d.sq_w,
                                                                      m.d.sq_taub, nsp);
    }
    if (nse > 0) {
        Timed t(m, 2, ss, 1, timed);
        nitsche_el<T, JV><<<(unsigned)((nse + WPB - 1) / WPB), 32 * WPB, 0, ss>>>(A, m.d.sq_list, m.d.sq_off, m.d.sq_x,
                                                                                m.d.sq_n, m.d.sq_w, m.d.sq_taub, nse);
    }
    launch_penalty<T, JV>(m, A, ss, timed);
}

// the Out and Intercepted buckets in one persistent launch (vms_fused); the surface kernels beside
// it on the side stream ss (forked and joined with the events ev), or after it on s
template <class T, bool JV>
void launch_fused(const Mesh& m, const Args& A, cudaStream_t s, cudaStream_t ss, cudaEvent_t* ev, bool timed) {
    const bool fork = ev && ss && ss != s;
    if (fork) {   // the surface kernels first: their blocks take their SMs, the persistent queue fills the rest
        cudaEventRecord(ev[0], s);
        cudaStreamWaitEvent(ss, ev[0], 0);
        launch_surface<T, JV>(m, A, ss, timed);
    }
    FusedQueue Q;
    Q.items = m.d.fq_items;
    Q.n_items = m.fq_n;
    Q.cnt = m.d.fq_cnt;
    Q.oconn = m.d.out_conn;
    Q.olev = m.d.out_lev;
    Q.oprob = m.d.out_prob;
    Q.n_out = (int64_t)m.out_list.size();
    Q.cut_list = m.d.cut_list;
    Q.cut_off = m.d.cut_off;
    Q.cut_pts = std::is_same<T, float>::value ? (const void*)m.d.cut_pts_f : (const void*)m.d.cut_pts;
    Q.heavy_warps = m.fused_heavy_warps;
    if (Q.n_items + Q.n_out > 0) {
        Timed t(m, 5, s, 1, timed);
        const int64_t work = Q.n_items + (Q.n_out + 3) / 4;   // warp items
        const int64_t blocks = (work + kFusedWarps - 1) / kFusedWarps;
        const int64_t grid = std::min<int64_t>(blocks, (int64_t)fused_blocks_per_sm<T, JV>() * m.n_sm);
        vms_fused<T, JV><<<(unsigned)grid, 32 * kFusedWarps, FusedShape<T>::smem, s>>>(A, Q);
    }
    if (fork) {
        cudaEventRecord(ev[2], ss);
        cudaStreamWaitEvent(s, ev[2], 0);
    } else {
        launch_surface<T, JV>(m, A, s, timed);
    }
}

template <class T, bool JV>
void launch_all(const Mesh& m, Args A, cudaStream_t s, void* ws = nullptr, cudaStream_t s_cut = nullptr,
                cudaStream_t s_sur = nullptr, cudaEvent_t* ev = nullptr) {
    const int64_t next = m.n_nodes() + m.n_hang();
    T* ndv = node_workspace<T>(m, ws);
    T* ndt = ndv + 8 * next;
    T* ndf = A.F ? ndt + 8 * next : nullptr;
    A.ndv = ndv;
    A.ndt = ndt;
    A.ndf = ndf;
    if (next > 0) {
        Timed t(m, 4, s, (A.n_nodes > 0) + (A.n_hang > 0), !ws);
        launch_node_prep<T, JV>(A, ndv, ndt, ndf, s);
    }
    if (m.fused && m.d.fq_cnt) {
        launch_fused<T, JV>(m, A, s, s_sur, ev, !ws);
        return;
    }
    // fork: the Intercepted-element and surface kernels run beside the Out-element kernel
    const cudaStream_t sc = s_cut ? s_cut : s, ss = s_sur ? s_sur : s;
    if (ev) {
        cudaEventRecord(ev[0], s);
        cudaStreamWaitEvent(sc, ev[0], 0);
        cudaStreamWaitEvent(ss, ev[0], 0);
    }
    const int64_t no = (int64_t)m.out_list.size(), nc = (int64_t)m.cut_list.size();
    constexpr int EPB = Epb<T>::value;
    if (no > 0) {
        Timed t(m, 0, s, 1, !ws);
        const int tuned = m.out_bps[sizeof(T) == 4][JV];
        launch_interior<T, JV>(m, A, s, tuned > 0 ? tuned : interior_blocks_per_sm<T, JV>());
    }
    if (nc > 0) {
        Timed t(m, 1, sc, 1, !ws);
        const Mesh::CutTune& ct = m.cut_tune[sizeof(T) == 4][JV];
        launch_cut<T, JV>(m, A, sc, ct.wpb, ct.lpt);
    }
    launch_surface<T, JV>(m, A, ss, !ws);
    if (ev) {   // join
        cudaEventRecord(ev[1], sc);
        cudaEventRecord(ev[2], ss);
        cudaStreamWaitEvent(s, ev[1], 0);
        cudaStreamWaitEvent(s, ev[2], 0);
    }
}

// strong rows; with the deterministic scatter, the node sums (which write every row) and the strong rows
void launch_strong_rows(const Mesh& m, const Args& A, const imga_physics& ph, bool jv, cudaStream_t s,
                        bool timed = true, int precision = 0) {
    const int64_t nn = m.n_nodes();
    Timed t(m, 3, s, 1, timed);
    if (nn > 0 && A.sv) {
        const uint8_t* um = m.user_bc ? m.d.bcmask_user : nullptr;
        const double* uv = m.user_bc ? m.d.bcval_user : nullptr;
        const unsigned g4 = (unsigned)((nn + 255) / 256);
        if (precision == 0)
            node_gather<double><<<g4, 256, 0, s>>>(A, m.d.inc_head, m.d.inc_ptr, m.d.inc, m.n_vslots, m.d.bcflag, um, uv, ph.u_inf[0],
                                                  ph.u_inf[1], ph.u_inf[2], jv ? 1 : 0);
        else
            node_gather<float><<<g4, 256, 0, s>>>(A, m.d.inc_head, m.d.inc_ptr, m.d.inc, m.n_vslots, m.d.bcflag, um, uv, ph.u_inf[0],
                                                 ph.u_inf[1], ph.u_inf[2], jv ? 1 : 0);
        return;
    }
    if (nn > 0)
        strong_rows<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(A, m.d.bcflag, m.user_bc ? m.d.bcmask_user : nullptr,
                                                                m.user_bc ? m.d.bcval_user : nullptr, ph.u_inf[0],
                                                                ph.u_inf[1], ph.u_inf[2], jv ? 1 : 0);
}

}  // namespace

// The work queue of the fused launch: the Intercepted elements by decreasing point count (the cost
// of an element on a warp is its rounds of 32 sub-cell points, Eq. Wpart's volume term), claimed
// first; the Out elements follow in Morton order, claimed in chunks.
int fused_prepare(Mesh& m, std::string& err) {
    const int64_t nc = (int64_t)m.cut_list.size();
    std::vector<uint32_t> items((size_t)nc);
    for (int64_t i = 0; i < nc; ++i) items[i] = (uint32_t)i;
    std::stable_sort(items.begin(), items.end(), [&](uint32_t a, uint32_t b) {
        return m.cut_off[a + 1] - m.cut_off[a] > m.cut_off[b + 1] - m.cut_off[b];
    });
    if (m.d.fq_items) { cudaFree(m.d.fq_items); m.d.fq_items = nullptr; }
    if (m.d.fq_cnt) { cudaFree(m.d.fq_cnt); m.d.fq_cnt = nullptr; }
    if (cudaMalloc((void**)&m.d.fq_items, std::max<size_t>(1, items.size()) * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc((void**)&m.d.fq_cnt, 3 * sizeof(unsigned long long)) != cudaSuccess ||
        (!items.empty() && cudaMemcpy(m.d.fq_items, items.data(), items.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemset(m.d.fq_cnt, 0, 3 * sizeof(unsigned long long)) != cudaSuccess) {
        err = "fused queue upload";
        return 1;
    }
    m.fq_n = nc;
    m.fq_counts[0] = nc;
    m.fq_counts[1] = m.n_sq_elem;
    m.fq_counts[2] = m.n_sq_sparse;
    fused_blocks_per_sm<double, true>();
    fused_blocks_per_sm<double, false>();
    fused_blocks_per_sm<float, true>();
    fused_blocks_per_sm<float, false>();
    return 0;
}

void graphs_free(Mesh& m) {
    for (auto& g : m.graphs) cudaGraphExecDestroy((cudaGraphExec_t)g.second);
    m.graphs.clear();
    for (int k = 0; k < 3; ++k) if (m.side[k]) { cudaStreamDestroy((cudaStream_t)m.side[k]); m.side[k] = nullptr; }
    for (int k = 0; k < 5; ++k) if (m.fork_ev[k]) { cudaEventDestroy((cudaEvent_t)m.fork_ev[k]); m.fork_ev[k] = nullptr; }
}

// the mesh's side streams and fork / join events (created on first use)
static int side_streams(Mesh& mm) {
    if (mm.side[0]) return 0;
    for (int k = 0; k < 3; ++k)
        if (cudaStreamCreateWithFlags((cudaStream_t*)&mm.side[k], cudaStreamNonBlocking) != cudaSuccess) return 1;
    for (int k = 0; k < 5; ++k)
        if (cudaEventCreateWithFlags((cudaEvent_t*)&mm.fork_ev[k], cudaEventDisableTiming) != cudaSuccess) return 1;
    return 0;
}

static int vms_apply_ws(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                        const imga_physics& ph, int precision, const double* v, double* out, void* stream, void* ws) {
    cudaStream_t s = (cudaStream_t)stream;
    Args A = make_args(m, u, up, up2, f, ph, v, out);
    const bool jv = v != nullptr;
    if (m.tune_pending[precision != 0][jv] && !ws) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &cs);
        if (cs == cudaStreamCaptureStatusNone) {
            Mesh& mm = const_cast<Mesh&>(m);
            const int rc = precision == 0 ? (jv ? autotune_cut<double, true>(mm, A, s) : autotune_cut<double, false>(mm, A, s))
                                          : (jv ? autotune_cut<float, true>(mm, A, s) : autotune_cut<float, false>(mm, A, s));
            if (rc) return 1;
            graphs_free(mm);   // captured launches carry the old tile shapes
        }
    }
    if (m.use_graphs && !ws && !m.profiling) {
        // Replay (or capture once) the whole call as a CUDA graph with parallel branches.  Capture runs on
        // a private stream (the legacy default stream cannot be captured); the graph is launched on a
        // private stream too, ordered after the caller's stream by events and joined back into it.
        Mesh& mm = const_cast<Mesh&>(m);
        GraphKey key;
        std::memset(&key, 0, sizeof(key));
        key.u = u; key.up = up; key.up2 = up2; key.f = f; key.v = v; key.out = out;
        key.precision = precision;
        key.ph = ph;
        key.user_bc = m.user_bc;
        if (side_streams(mm)) return 1;
        cudaStream_t s1 = (cudaStream_t)mm.side[0], s2 = (cudaStream_t)mm.side[1], cs = (cudaStream_t)mm.side[2];
        cudaEvent_t* ev = (cudaEvent_t*)mm.fork_ev;
        cudaGraphExec_t exec = nullptr;
        for (auto& g : mm.graphs)
            if (std::memcmp(&g.first, &key, sizeof(key)) == 0) { exec = (cudaGraphExec_t)g.second; break; }
        if (!exec) {
            vms_prepare();
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return 1;
            if (!A.sv) cudaMemsetAsync(out, 0, (size_t)m.n_nodes() * 4 * sizeof(double), cs);
            cudaStream_t b1 = m.concurrent ? s1 : cs, b2 = m.concurrent ? s2 : cs;
            cudaEvent_t* bev = m.concurrent ? ev : nullptr;
            if (precision == 0) {
                if (jv) launch_all<double, true>(m, A, cs, nullptr, b1, b2, bev); else launch_all<double, false>(m, A, cs, nullptr, b1, b2, bev);
            } else {
                if (jv) launch_all<float, true>(m, A, cs, nullptr, b1, b2, bev); else launch_all<float, false>(m, A, cs, nullptr, b1, b2, bev);
            }
            launch_strong_rows(m, A, ph, jv, cs, true, precision);
            const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
            if (ec != cudaSuccess || !graph) return 1;
            const cudaError_t rc = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (rc != cudaSuccess) return 1;
            if (mm.graphs.size() >= 32) {   // bounded cache: drop the oldest
                cudaGraphExecDestroy((cudaGraphExec_t)mm.graphs.front().second);
                mm.graphs.erase(mm.graphs.begin());
            }
            mm.graphs.push_back({key, (void*)exec});
        }
        if (cudaEventRecord(ev[3], s) != cudaSuccess || cudaStreamWaitEvent(cs, ev[3], 0) != cudaSuccess) return 1;
        if (cudaGraphLaunch(exec, cs) != cudaSuccess) return 1;
        if (cudaEventRecord(ev[4], cs) != cudaSuccess || cudaStreamWaitEvent(s, ev[4], 0) != cudaSuccess) return 1;
        return 0;
    }
    if (!A.sv && cudaMemsetAsync(out, 0, (size_t)m.n_nodes() * 4 * sizeof(double), s) != cudaSuccess) return 1;
    // the Intercepted-element and surface kernels on the mesh's side streams, beside the Out-element
    // kernel, as in the captured graph (not for calls on a caller's workspace, which create nothing)
    cudaStream_t s1 = nullptr, s2 = nullptr;
    cudaEvent_t* ev = nullptr;
    if (!ws && m.concurrent) {
        Mesh& mm = const_cast<Mesh&>(m);
        if (side_streams(mm)) return 1;
        s1 = (cudaStream_t)mm.side[0];
        s2 = (cudaStream_t)mm.side[1];
        ev = (cudaEvent_t*)mm.fork_ev;
    }
    if (precision == 0) {
        if (jv) launch_all<double, true>(m, A, s, ws, s1, s2, ev); else launch_all<double, false>(m, A, s, ws, s1, s2, ev);
    } else {
        if (jv) launch_all<float, true>(m, A, s, ws, s1, s2, ev); else launch_all<float, false>(m, A, s, ws, s1, s2, ev);
    }
    launch_strong_rows(m, A, ph, jv, s, !ws, precision);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// ------------------------------------------------------------------------------------------
// Force of the fluid on the body: the surface terms of Eq. (weakbc) tested with w = e_i, i.e. summed
// over every node's momentum rows (partition of unity), in float64.  Per surface point
//   w_q [ -(sigma(u_s, p) n)_i - [u.n < 0] rho (u.n) (u - g)_i + tau_B (u - g)_i ],
// n the fluid-outward normal: the force that keeps the discrete momentum balance of weak Dirichlet
// conditions.  Each block sums its points in a fixed order, then one block sums the partials in
// block order (same bits on every call).
// ------------------------------------------------------------------------------------------
constexpr int kForceBlocks = 256;

__global__ void __launch_bounds__(256) surface_force_partial(Args A, const int32_t* __restrict__ el,
                                                             const double* __restrict__ xr, const double* __restrict__ nr,
                                                             const double* __restrict__ wr, const double* __restrict__ taub,
                                                             int64_t n, double* __restrict__ part) {
    double f[3] = {0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        NitschePoint<double, double> P;
        nitsche_fields<double, double, false>(A, el[i], i, xr + 3 * i, nr + 3 * i, P);
        const double tauB = A.Cb * P.mu * taub[i];
        for (int k = 0; k < 3; ++k) {
            double t = -P.tr[k] + tauB * P.dd[k];
            if (P.inflow) t -= P.rho * P.un * P.dd[k];
            f[k] += wr[i] * t;
        }
    }
    __shared__ double red[3][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 3; ++k) {
        double v = f[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) v += red[threadIdx.x][j];
        part[3 * blockIdx.x + threadIdx.x] = v;
    }
}

__global__ void surface_force_final(int nb, const double* __restrict__ part, double* __restrict__ F) {
    if (threadIdx.x >= 3) return;
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += part[3 * b + threadIdx.x];
    F[threadIdx.x] = v;
}

// ------------------------------------------------------------------------------------------
// self-check of f2d / d2f against the hardware conversions
// ------------------------------------------------------------------------------------------
namespace {
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void conversion_check(int64_t n, uint64_t seed, unsigned long long* bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t r = mix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1));
    const uint64_t r2 = mix64(r ^ 0xD1B54A32D192ED03ull);
    uint64_t bits;
    const uint64_t sign = r2 & 0x8000000000000000ull, frac = r & 0x000FFFFFFFFFFFFFull;
    switch (i & 7) {
        case 0: bits = r; break;                                                    // anything
        case 1: bits = sign | ((uint64_t)(897 + (r2 >> 8) % 254) << 52) | frac; break;   // float32 normal range
        case 2: bits = sign | ((uint64_t)(897 + (r2 >> 8) % 254) << 52) | (frac & ~0x1FFFFFFFull) | 0x10000000ull; break;  // tie
        case 3: {                                                                   // edges of the range
            const uint32_t E[6] = {0, 1, 896, 897, 1150, 1151};
            bits = sign | ((uint64_t)E[(r2 >> 8) % 6] << 52) | frac;
            break;
        }
        case 4: bits = sign | ((uint64_t)1150 << 52) | (0x000FFFFFF0000000ull | (frac & 0x0FFFFFFFull)); break;  // rounds to inf
        case 5: bits = sign | ((uint64_t)(r2 % 3 == 0 ? 2047 : (r2 % 3 == 1 ? 0 : 1)) << 52) | ((r2 >> 4) & 1 ? frac : 0); break;
        case 6: bits = sign | ((uint64_t)(897 + (r2 >> 8) % 254) << 52) | (frac | 0x000FFFFFE0000000ull); break;   // carry into the exponent
        default: bits = sign | ((uint64_t)(897 + (r2 >> 8) % 254) << 52) | (frac & ~0x1FFFFFFFull); break;        // exact in float32
    }
    const double x = __longlong_as_double((long long)bits);
    const float a = d2f(x), b = (float)x;
    bool ok = (a != a) ? (b != b) : (__float_as_uint(a) == __float_as_uint(b));
    const float y = __uint_as_float((uint32_t)(r2 >> 17));
    const double c = f2d(y), d = (double)y;
    ok = ok && ((c != c) ? (d != d) : (__double_as_longlong(c) == __double_as_longlong(d)));
    if (!ok) atomicAdd(bad, 1ull);
}
}  // namespace

int conversion_selftest(int64_t n, uint64_t seed, int64_t* mismatches, std::string& err) {
    unsigned long long* bad = nullptr;
    if (cudaMalloc((void**)&bad, sizeof(*bad)) != cudaSuccess) { err = "cudaMalloc failed"; return 1; }
    cudaMemset(bad, 0, sizeof(*bad));
    if (n > 0) conversion_check<<<(unsigned)((n + 255) / 256), 256>>>(n, seed, bad);
    unsigned long long h = 0;
    const cudaError_t rc = cudaMemcpy(&h, bad, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    if (rc != cudaSuccess) { err = cudaGetErrorString(rc); return 1; }
    *mismatches = (int64_t)h;
    return 0;
}

// Residual / J v on `stream` without the graph path, every kernel returning at once while *skip is
// nonzero (steps of a solver loop that is itself captured in a graph).
int vms_apply_skip(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                   const imga_physics& ph, int precision, const double* v, double* out, void* stream,
                   const int* skip) {
    cudaStream_t s = (cudaStream_t)stream;
    Args A = make_args(m, u, up, up2, f, ph, v, out);
    A.skip = skip;
    const bool jv = v != nullptr;
    if (!A.sv && cudaMemsetAsync(out, 0, (size_t)m.n_nodes() * 4 * sizeof(double), s) != cudaSuccess) return 1;
    if (precision == 0) {
        if (jv) launch_all<double, true>(m, A, s); else launch_all<double, false>(m, A, s);
    } else {
        if (jv) launch_all<float, true>(m, A, s); else launch_all<float, false>(m, A, s);
    }
    launch_strong_rows(m, A, ph, jv, s, true, precision);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// one-time launch attributes of the element kernels (call before any stream capture)
void vms_prepare() {
    interior_blocks_per_sm<double, true>();
    interior_blocks_per_sm<double, false>();
    interior_blocks_per_sm<float, true>();
    interior_blocks_per_sm<float, false>();
    interior_blocks_per_sm<float, true, 5>();
    interior_blocks_per_sm<float, false, 5>();
}

int vms_apply(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
              const imga_physics& ph, int precision, const double* v, double* out, void* stream) {
    return vms_apply_ws(m, u, up, up2, f, ph, precision, v, out, stream, nullptr);
}

// ------------------------------------------------------------------------------------------
// J v with no allocation at all: the per-call node workspace lives in this fixed array, which
// every GPU that loads the library holds until the process exits.  Host code must not pass the
// array's name to a kernel (on the host it names a shadow, not device memory): its device
// address is looked up once per device with cudaGetSymbolAddress.
// ------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kMaxDevices] = {};

int vms_jvp_noalloc(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                    const imga_physics& ph, int precision, const double* v, double* out, void* stream,
                    std::string& err) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) { err = "no usable current device"; return 1; }
    if (dev != m.device) { err = "the mesh's device must be current"; return 1; }
    const size_t next = (size_t)(m.n_nodes() + m.n_hang());
    const size_t per_node = (size_t)(f ? 20 : 16) * (precision == 0 ? sizeof(double) : sizeof(float));
    if (next * per_node > kNoAllocScratchBytes) {
        err = "mesh too large for the fixed scratch: needs " + std::to_string(next * per_node) + " bytes, limit " +
              std::to_string(kNoAllocScratchBytes);
        return 1;
    }
    void* ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (rc != cudaSuccess || !p) { err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(rc); return 1; }
            g_noalloc_addr[dev] = p;
        }
        ws = g_noalloc_addr[dev];
    }
    if (vms_apply_ws(m, u, up, up2, f, ph, precision, v, out, stream, ws)) { err = "launch failed"; return 1; }
    return 0;
}

// F [3] (device) = force of the fluid on the body at the state (u, u_prev); part: kForceBlocks x 3
// doubles of workspace
int surface_force(const Mesh& m, const double* u, const double* up, const imga_physics& ph, double* F, double* part,
                  void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    Args A = make_args(m, u, up, up, nullptr, ph, nullptr, nullptr);
    const int64_t next = m.n_nodes() + m.n_hang();
    double* ndv = node_workspace<double>(m, nullptr);
    A.ndv = ndv;
    A.ndt = ndv + 8 * next;
    A.ndf = nullptr;
    if (next > 0) launch_node_prep<double, false>(A, ndv, ndv + 8 * next, nullptr, s);
    const int64_t ns = (int64_t)m.sq.size() / 10;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kForceBlocks, (ns + 255) / 256));
    surface_force_partial<<<nb, 256, 0, s>>>(A, m.d.sq_elem, m.d.sq_x, m.d.sq_n, m.d.sq_w, m.d.sq_taub, ns, part);
    surface_force_final<<<1, 32, 0, s>>>(nb, part, F);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

void profile_reset(Mesh& m) {
    for (int k = 0; k < kProfKinds; ++k) {
        for (auto& p : m.prof_ev[k]) { cudaEventDestroy((cudaEvent_t)p.a); cudaEventDestroy((cudaEvent_t)p.b); }
        m.prof_ev[k].clear();
        m.prof_ms[k] = 0.0;
        m.prof_n[k] = 0;
    }
}

int profile_collect(Mesh& m) {
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    for (int k = 0; k < kProfKinds; ++k) {
        for (auto& p : m.prof_ev[k]) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, (cudaEvent_t)p.a, (cudaEvent_t)p.b);
            m.prof_ms[k] += ms;
            m.prof_n[k] += p.launches;
            cudaEventDestroy((cudaEvent_t)p.a);
            cudaEventDestroy((cudaEvent_t)p.b);
        }
        m.prof_ev[k].clear();
    }
    return 0;
}

}  // namespace imga
