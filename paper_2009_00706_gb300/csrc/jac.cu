// Element Jacobians k_e = d r_e / d u_e (the 32 x 32 element matrix of Algorithm 4, before the
// hanging correction M_e^T k_e M_e of Algorithm 2) and the nodal block-Jacobi diagonal.
//
// Every column of k_e is the derivative of the element residual in the direction of one local
// degree of freedom (corner b, component k).  The fields of the point are interpolated once
// (values); the seed's tangent fields are read off the basis of corner b at the point, then the
// pointwise VMS coefficients are differentiated exactly (dual numbers), weighted and contracted
// with the test functions.  No global matrix is ever formed.
//
//   jac_out     8 threads per Out element (thread c: Gauss point c, then node c's 4 rows)
//   jac_cut     one warp per Intercepted element, 32 sub-cell points per step, lane = row
//   jac_nitsche one thread per surface point
// Mode FULL writes k_e for requested elements (slot map); mode DIAG adds the 4x4 diagonal blocks
// of sum_e M_e^T k_e M_e (each corner's own block times the squared hanging weights; the
// couplings of two different corners of one element that share a parent are left out) to a
// float64 [n_nodes][4][4] array.

#include <cuda_runtime.h>

#include "imga_internal.h"
#include "vms_device.cuh"

namespace imga {

namespace {

enum { FULL = 0, DIAG = 1, BSR = 2 };

// Position of block (row, col) in the block pattern (columns increasing within a row), or -1.
__device__ __forceinline__ int64_t bsr_find(const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                            int32_t row, int32_t col) {
    int64_t lo = ptr[row], hi = ptr[row + 1] - 1;
    while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t c = idx[mid];
        if (c == col) return mid;
        if (c < col) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// node ids and weights a corner enters through M_e: itself, or the 2 / 4 parents of a hanging node
__device__ __forceinline__ int corner_nodes(const Args& A, int32_t id, int32_t nd[4], double& w) {
    if (id < A.n_nodes) { nd[0] = id; w = 1.0; return 1; }
    const int32_t* hp = A.hpar + 4 * (int64_t)(id - A.n_nodes);
    const int np = hp[2] >= 0 ? 4 : 2;
    for (int p = 0; p < np; ++p) nd[p] = hp[p];
    w = np == 4 ? 0.25 : 0.5;
    return np;
}

// entry (row i of corner ida, column k of corner idb) of k_e added to the assembled matrix through
// M_e^T k_e M_e (Algorithm 2): every parent pair (p, q) receives w_p w_q v in block (p, q)
__device__ __forceinline__ void bsr_add(const Args& A, int32_t ida, int32_t idb, int i, int k, double v,
                                        double* __restrict__ val) {
    if (v == 0.0) return;
    int32_t na[4], nb[4];
    double wa, wb;
    const int ca = corner_nodes(A, ida, na, wa), cb = corner_nodes(A, idb, nb, wb);
    const double vw = wa * wb * v;
    for (int p = 0; p < ca; ++p)
        for (int q = 0; q < cb; ++q) {
            const int64_t pos = bsr_find(A.bptr, A.bidx, na[p], nb[q]);
            if (pos >= 0) atomicAdd(val + 16 * pos + 4 * i + k, vw);
        }
}

// tangent fields of the seed (corner b, component k) at a point whose corner-b basis values are
// phb, reference gradient dphb and reference mixed second derivatives d2b (01, 02, 12)
template <class T>
__device__ __forceinline__ void seed_fields(const Args& A, const Fields<T, T>& V, T g, T phb, const T dphb[3],
                                            const T d2b[3], int k, Fields<Dual<T>, T>& F) {
    const T th = (T)A.theta, c0 = (T)A.c0, g2 = g * g;
    for (int i = 0; i < 3; ++i) {
        F.us[i] = {V.us[i], T(0)};
        F.at[i] = {V.at[i], T(0)};
        F.gp[i] = {V.gp[i], T(0)};
        F.H2[i] = {V.H2[i], T(0)};
        F.f[i] = V.f[i];
        for (int j = 0; j < 3; ++j) F.Gu[i][j] = {V.Gu[i][j], T(0)};
    }
    F.p = {V.p, T(0)};
    if (k < 3) {
        F.us[k].d = th * phb;
        F.at[k].d = c0 * phb;
        for (int j = 0; j < 3; ++j) F.Gu[k][j].d = th * g * dphb[j];
        // (grad div u)_i = sum_{j != i} d_i d_j u_j: a unit u_k at corner b feeds every i != k
        const int pair[3][3] = {{-1, 0, 1}, {0, -1, 2}, {1, 2, -1}};
        for (int i = 0; i < 3; ++i)
            if (i != k) F.H2[i].d = th * g2 * d2b[pair[i][k]];
    } else {
        F.p.d = phb;
        for (int j = 0; j < 3; ++j) F.gp[j].d = g * dphb[j];
    }
}

template <class T>
__device__ __forceinline__ void corner_basis(const T fm[3], const T fp[3], int b, T& ph, T dph[3], T d2[3]) {
    const T f0 = (b & 1) ? fp[0] : fm[0], f1 = (b & 2) ? fp[1] : fm[1], f2 = (b & 4) ? fp[2] : fm[2];
    const T h0 = (b & 1) ? T(0.5) : T(-0.5), h1 = (b & 2) ? T(0.5) : T(-0.5), h2 = (b & 4) ? T(0.5) : T(-0.5);
    ph = f0 * f1 * f2;
    dph[0] = h0 * (f1 * f2);
    dph[1] = h1 * (f0 * f2);
    dph[2] = h2 * (f0 * f1);
    d2[0] = (h0 * h1) * f2;
    d2[1] = (h0 * h2) * f1;
    d2[2] = (h1 * h2) * f0;
}

// add a corner's 4x4 block to the diagonal of its node(s) through the hanging weights
__device__ __forceinline__ void add_diag(const Args& A, int32_t id, const double blk[16], double* D) {
    if (id < A.n_nodes) {
        for (int q = 0; q < 16; ++q) atomicAdd(D + 16 * (int64_t)id + q, blk[q]);
        return;
    }
    const int32_t* hp = A.hpar + 4 * (int64_t)(id - A.n_nodes);
    const int np = hp[2] >= 0 ? 4 : 2;
    const double w2 = np == 4 ? 0.0625 : 0.25;
    for (int p = 0; p < np; ++p)
        for (int q = 0; q < 16; ++q) atomicAdd(D + 16 * (int64_t)hp[p] + q, w2 * blk[q]);
}

template <class T> struct JacShape { static constexpr int EPB = sizeof(T) == 8 ? 8 : 16; };

template <class T, int MODE>
__global__ void __launch_bounds__(8 * JacShape<T>::EPB) jac_out(Args A, const int32_t* __restrict__ list, int64_t n,
                                                                const int32_t* __restrict__ slot, double* __restrict__ K,
                                                                double* __restrict__ D) {
    constexpr int EPB = JacShape<T>::EPB;
    __shared__ __align__(16) T s_nd[EPB][8][CS];
    __shared__ T s_cf[EPB][8][17];
    const int c = threadIdx.x & 7, le = threadIdx.x >> 3;
    const int64_t idx = (int64_t)blockIdx.x * EPB + le;
    const bool valid = idx < n;
    const int32_t e = list[valid ? idx : n - 1];
    const int32_t sl = MODE == FULL ? slot[e] : 0;
    const bool work = valid && sl >= 0;
    const int32_t id = A.conn[8 * (int64_t)e + c];
    corner_data<T, false>(A, id, &s_nd[le][c][0]);
    __syncwarp();
    const int lv = A.lev[e];
    const T g = lvl_g<T>(A, lv);
    const T gauss = (T)0.57735026918962576451;
    const T wp = T(0.5) * (T(1) + gauss), wm = T(0.5) * (T(1) - gauss);
    T fm[3], fp[3];
    for (int k = 0; k < 3; ++k) {
        const bool plus = (c >> k) & 1;
        fm[k] = plus ? wm : wp;
        fp[k] = plus ? wp : wm;
    }
    Fields<T, T> V;
    interp<T, T>(A, fm, fp, &s_nd[le][0][0], CS, g, V);
    const T wq = lvl_w<T>(A, lv), wqg = wq * g;
    double diag[16];
    for (int q = 0; q < 16; ++q) diag[q] = 0.0;
    for (int b = 0; b < 8; ++b) {
        T phb, dphb[3], d2b[3];
        corner_basis<T>(fm, fp, b, phb, dphb, d2b);
        for (int k = 0; k < 4; ++k) {
            Fields<Dual<T>, T> F;
            seed_fields<T>(A, V, g, phb, dphb, d2b, k, F);
            Dual<T> cf[16];
            pointwise<Dual<T>, T>(A, Phys<T>(A, prob_of(A, e)), F, g, cf);
            for (int q = 0; q < 16; ++q) s_cf[le][c][q] = ((q < 3 || q == 12) ? wq : wqg) * cf[q].d;
            __syncwarp();
            T r[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                T f[3], d[3];
                for (int kk = 0; kk < 3; ++kk) {
                    bool same = (((c >> kk) & 1) == ((q >> kk) & 1));
                    f[kk] = same ? wp : wm;
                    d[kk] = ((c >> kk) & 1) ? T(0.5) : T(-0.5);
                }
                T ph = f[0] * f[1] * f[2];
                T dp[3] = {d[0] * f[1] * f[2], d[1] * f[0] * f[2], d[2] * f[0] * f[1]};
                const T* C = s_cf[le][q];
                for (int i = 0; i < 3; ++i) r[i] += ph * C[i] + dp[0] * C[3 + 3 * i] + dp[1] * C[4 + 3 * i] + dp[2] * C[5 + 3 * i];
                r[3] += ph * C[12] + dp[0] * C[13] + dp[1] * C[14] + dp[2] * C[15];
            }
            __syncwarp();
            if (MODE == FULL) {
                if (work)
                    for (int i = 0; i < 4; ++i) K[(int64_t)sl * 1024 + (c * 4 + i) * 32 + b * 4 + k] = (double)r[i];
            } else if (MODE == BSR) {
                const int32_t idb = __shfl_sync(0xffffffffu, id, (threadIdx.x & 31 & ~7) | b);
                if (work)
                    for (int i = 0; i < 4; ++i) bsr_add(A, id, idb, i, k, (double)r[i], K);
            } else if (b == c) {
                for (int i = 0; i < 4; ++i) diag[i * 4 + k] = (double)r[i];
            }
        }
    }
    if (MODE == DIAG && work) add_diag(A, id, diag, D);
}

constexpr int JWPB = 2;   // warps per block of jac_cut

template <class T, int MODE>
__global__ void __launch_bounds__(32 * JWPB) jac_cut(Args A, const int32_t* __restrict__ list,
                                                     const int64_t* __restrict__ off, const void* __restrict__ pts,
                                                     int64_t n, const int32_t* __restrict__ slot,
                                                     double* __restrict__ K, double* __restrict__ D) {
    __shared__ __align__(16) T s_nd[JWPB][8][CS];
    __shared__ T s_cf[JWPB][32][20];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t idx = (int64_t)blockIdx.x * JWPB + w;
    if (idx >= n) return;
    const int32_t e = list[idx];
    const int32_t sl = MODE == FULL ? slot[e] : 0;
    if (sl < 0) return;
    int32_t my_id = 0;
    if (lane < 8) {
        my_id = A.conn[8 * (int64_t)e + lane];
        corner_data<T, false>(A, my_id, &s_nd[w][lane][0]);
    }
    __syncwarp();
    const T g = lvl_g<T>(A, A.lev[e]);
    const T det = lvl_w<T>(A, A.lev[e]);
    const int a = lane >> 2, comp = lane & 3;
    const T sa[3] = {(a & 1) ? T(1) : T(-1), (a & 2) ? T(1) : T(-1), (a & 4) ? T(1) : T(-1)};
    T acc[32];
    for (int s = 0; s < 32; ++s) acc[s] = T(0);
    const int64_t q0 = off[idx], q1 = off[idx + 1];
    for (int64_t base = q0; base < q1; base += 32) {
        const int64_t q = base + lane;
        const bool have = q < q1;
        T pt[4] = {T(0), T(0), T(0), T(0)};
        if (have) load_pt<T>(pts, q, pt);
        T fm[3], fp[3];
        for (int k = 0; k < 3; ++k) { fm[k] = T(0.5) * (T(1) - pt[k]); fp[k] = T(0.5) * (T(1) + pt[k]); }
        Fields<T, T> V;
        interp<T, T>(A, fm, fp, &s_nd[w][0][0], CS, g, V);
        const T wq = have ? pt[3] * det : T(0), wqg = wq * g;
        const int m = (int)min((int64_t)32, q1 - base);
        for (int s = 0; s < 32; ++s) {
            const int b = s >> 2, k = s & 3;
            T phb, dphb[3], d2b[3];
            corner_basis<T>(fm, fp, b, phb, dphb, d2b);
            Fields<Dual<T>, T> F;
            seed_fields<T>(A, V, g, phb, dphb, d2b, k, F);
            Dual<T> cf[16];
            pointwise<Dual<T>, T>(A, Phys<T>(A, prob_of(A, e)), F, g, cf);
            for (int qq = 0; qq < 16; ++qq) s_cf[w][lane][qq] = ((qq < 3 || qq == 12) ? wq : wqg) * cf[qq].d;
            s_cf[w][lane][16] = pt[0];
            s_cf[w][lane][17] = pt[1];
            s_cf[w][lane][18] = pt[2];
            __syncwarp();
            T sum = T(0);
            for (int j = 0; j < m; ++j) {
                const T* C = s_cf[w][j];
                T f0 = T(0.5) * (T(1) + sa[0] * C[16]), f1 = T(0.5) * (T(1) + sa[1] * C[17]), f2 = T(0.5) * (T(1) + sa[2] * C[18]);
                T ph = f0 * f1 * f2;
                T d0 = T(0.5) * sa[0] * f1 * f2, d1 = T(0.5) * sa[1] * f0 * f2, d2 = T(0.5) * sa[2] * f0 * f1;
                if (comp < 3) sum += ph * C[comp] + d0 * C[3 + 3 * comp] + d1 * C[4 + 3 * comp] + d2 * C[5 + 3 * comp];
                else sum += ph * C[12] + d0 * C[13] + d1 * C[14] + d2 * C[15];
            }
            acc[s] += sum;
            __syncwarp();
        }
    }
    if (MODE == FULL) {
        for (int s = 0; s < 32; ++s) K[(int64_t)sl * 1024 + lane * 32 + s] = (double)acc[s];
    } else if (MODE == BSR) {
        const int32_t ida = __shfl_sync(0xffffffffu, my_id, a);
        for (int s = 0; s < 32; ++s) {
            const int32_t idb = __shfl_sync(0xffffffffu, my_id, s >> 2);
            bsr_add(A, ida, idb, comp, s & 3, (double)acc[s], K);
        }
    } else {
        // lane (a, comp) holds row comp of corner a's own block in acc[4a .. 4a+3]
        double blk[16];
        for (int i = 0; i < 4; ++i)
            for (int k = 0; k < 4; ++k) blk[i * 4 + k] = (double)__shfl_sync(0xffffffffu, acc[4 * a + k], 4 * a + i);
        const int32_t id = __shfl_sync(0xffffffffu, my_id, a);
        if (comp == 0) add_diag(A, id, blk, D);
    }
}

template <class T, int MODE>
__global__ void __launch_bounds__(128) jac_nitsche(Args A, const int32_t* __restrict__ el,
                                                   const double* __restrict__ xr, const double* __restrict__ nr,
                                                   const double* __restrict__ wr, const double* __restrict__ taub,
                                                   int64_t n, const int32_t* __restrict__ slot, double* __restrict__ K,
                                                   double* __restrict__ D) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t e = el[i];
    const int32_t sl = MODE == FULL ? slot[e] : 0;
    if (sl < 0) return;
    NitschePoint<T, T> V;
    nitsche_fields<T, T, false>(A, e, i, xr + 3 * i, nr + 3 * i, V);
    const T w = (T)wr[i];
    const T tauB = (T)(A.Cb * (double)V.mu * taub[i]);
    for (int b = 0; b < 8; ++b) {
        for (int k = 0; k < 4; ++k) {
            // tangent point data of the seed (corner b, component k)
            NitschePoint<Dual<T>, T> P;
            P.g = V.g;
            P.mu = V.mu;
            P.rho = V.rho;
            P.B = V.B;
            for (int c = 0; c < 8; ++c) P.ids[c] = V.ids[c];
            for (int j = 0; j < 3; ++j) P.nn[j] = V.nn[j];
            const T th = (T)A.theta, phb = V.B.phi[b];
            P.p = {V.p, k == 3 ? phb : T(0)};
            for (int kk = 0; kk < 3; ++kk) {
                P.us[kk] = {V.us[kk], kk == k ? th * phb : T(0)};
                P.d[kk] = {V.d[kk], kk == k ? th * phb : T(0)};
                for (int j = 0; j < 3; ++j)
                    P.Gu[kk][j] = {V.Gu[kk][j], kk == k ? th * V.B.dphi[b][j] : T(0)};   // reference; scaled below
            }
            // finish_nitsche scales Gu by g: undo for the values (already physical)
            for (int kk = 0; kk < 3; ++kk)
                for (int j = 0; j < 3; ++j) P.Gu[kk][j].v = V.Gu[kk][j] / V.g;
            finish_nitsche(A, P);
            P.inflow = V.inflow;
            if (MODE == FULL) {
                for (int c = 0; c < 8; ++c) {
                    Dual<T> t[4];
                    nitsche_rows<Dual<T>, T>(A, P, c, tauB, t);
                    for (int r = 0; r < 4; ++r)
                        atomicAdd(K + (int64_t)sl * 1024 + (c * 4 + r) * 32 + b * 4 + k, (double)(w * t[r].d));
                }
            } else {
                Dual<T> t[4];
                nitsche_rows<Dual<T>, T>(A, P, b, tauB, t);
                double blk[16];
                for (int q = 0; q < 16; ++q) blk[q] = 0.0;
                for (int r = 0; r < 4; ++r) blk[r * 4 + k] = (double)(w * t[r].d);
                add_diag(A, P.ids[b], blk, D);
            }
        }
    }
}

// rows of prescribed components become identity rows
__global__ void jac_strong_rows(int64_t nn, const uint8_t* __restrict__ flag, const uint8_t* __restrict__ umask,
                                double* __restrict__ D) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    uint8_t mask = umask ? umask[n] : (uint8_t)(flag[n] & 15);
    if (flag[n] & 16) mask = 15;
    for (int k = 0; k < 4; ++k)
        if ((mask >> k) & 1)
            for (int j = 0; j < 4; ++j) D[16 * n + 4 * k + j] = j == k ? 1.0 : 0.0;
}

// invert every 4x4 block (Gauss-Jordan, partial pivoting, float64); a singular block -> identity
__global__ void bj_invert(int64_t nn, const double* __restrict__ D, double* __restrict__ Dinv) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    double a[4][8];
    double scale = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            a[i][j] = D[16 * n + 4 * i + j];
            a[i][4 + j] = i == j ? 1.0 : 0.0;
            scale = fmax(scale, fabs(a[i][j]));
        }
    bool ok = scale > 0.0;
    for (int col = 0; col < 4 && ok; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (!(fabs(a[piv][col]) > 1e-14 * scale)) { ok = false; break; }
        if (piv != col)
            for (int j = 0; j < 8; ++j) { double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
        const double inv = 1.0 / a[col][col];
        for (int j = 0; j < 8; ++j) a[col][j] *= inv;
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            const double f = a[r][col];
            if (f != 0.0)
                for (int j = 0; j < 8; ++j) a[r][j] -= f * a[col][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Dinv[16 * n + 4 * i + j] = ok ? a[i][4 + j] : (i == j ? 1.0 : 0.0);
}

// y_n = Dinv_n x_n
__global__ void bj_apply(int64_t nn, const double* __restrict__ Dinv, const double* __restrict__ x,
                         double* __restrict__ y) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    const double* M = Dinv + 16 * n;
    double xv[4] = {x[4 * n], x[4 * n + 1], x[4 * n + 2], x[4 * n + 3]};
    for (int i = 0; i < 4; ++i) y[4 * n + i] = M[4 * i] * xv[0] + M[4 * i + 1] * xv[1] + M[4 * i + 2] * xv[2] + M[4 * i + 3] * xv[3];
}

__global__ void fill_slots(int64_t n, const int32_t* __restrict__ list, int32_t* __restrict__ slot) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) slot[list[i]] = (int32_t)i;
}

template <class T, int MODE>
void launch_jac(const Mesh& m, Args A, const int32_t* slot, double* K, double* D, cudaStream_t s) {
    const int64_t next = m.n_nodes() + m.n_hang();
    T* ndv = node_workspace<T>(m, nullptr);
    A.ndv = ndv;
    A.ndt = ndv + 8 * next;
    A.ndf = A.F ? ndv + 16 * next : nullptr;
    if (next > 0)
        launch_node_prep<T, false>(A, ndv, ndv + 8 * next, (T*)A.ndf, s);
    const int64_t no = (int64_t)m.out_list.size(), nc = (int64_t)m.cut_list.size(), ns = (int64_t)m.sq.size() / 10;
    constexpr int EPB = JacShape<T>::EPB;
    if (no > 0) jac_out<T, MODE><<<(unsigned)((no + EPB - 1) / EPB), 8 * EPB, 0, s>>>(A, m.d.out_list, no, slot, K, D);
    if (nc > 0) {
        const void* pts = sizeof(T) == 4 ? (const void*)m.d.cut_pts_f : (const void*)m.d.cut_pts;
        jac_cut<T, MODE><<<(unsigned)((nc + JWPB - 1) / JWPB), 32 * JWPB, 0, s>>>(A, m.d.cut_list, m.d.cut_off, pts, nc,
                                                                               slot, K, D);
    }
    if (ns > 0)
        jac_nitsche<T, MODE><<<(unsigned)((ns + 127) / 128), 128, 0, s>>>(A, m.d.sq_elem, m.d.sq_x, m.d.sq_n, m.d.sq_w,
                                                                        m.d.sq_taub, ns, slot, K, D);
}

// k_e of the surface terms (one per host element, slot order) added to the assembled matrix
__global__ void scatter_kmat(Args A, const int32_t* __restrict__ list, int64_t n, const double* __restrict__ Ks,
                             double* __restrict__ val) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // (element, row, column block)
    if (t >= n * 256) return;
    const int64_t s = t >> 8;
    const int row = (int)((t >> 3) & 31), b = (int)(t & 7);
    const int32_t e = list[s];
    const int32_t ida = A.conn[8 * (int64_t)e + (row >> 2)], idb = A.conn[8 * (int64_t)e + b];
    for (int k = 0; k < 4; ++k) bsr_add(A, ida, idb, row & 3, k, Ks[s * 1024 + row * 32 + 4 * b + k], val);
}

// rows of prescribed components become identity rows of the assembled matrix
__global__ void bsr_strong_rows(int64_t nn, const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                const uint8_t* __restrict__ flag, const uint8_t* __restrict__ umask, double* __restrict__ val) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    uint8_t mask = umask ? umask[n] : (uint8_t)(flag[n] & 15);
    if (flag[n] & 16) mask = 15;
    if (!mask) return;
    for (int64_t q = ptr[n]; q < ptr[n + 1]; ++q)
        for (int k = 0; k < 4; ++k)
            if ((mask >> k) & 1)
                for (int j = 0; j < 4; ++j) val[16 * q + 4 * k + j] = (idx[q] == n && j == k) ? 1.0 : 0.0;
}

template <class T>
void launch_bsr_assembly(const Mesh& m, Args A, double* val, double* Ks, cudaStream_t s) {
    const int64_t next = m.n_nodes() + m.n_hang();
    T* ndv = node_workspace<T>(m, nullptr);
    A.ndv = ndv;
    A.ndt = ndv + 8 * next;
    A.ndf = A.F ? ndv + 16 * next : nullptr;
    if (next > 0) launch_node_prep<T, false>(A, ndv, ndv + 8 * next, (T*)A.ndf, s);
    const int64_t no = (int64_t)m.out_list.size(), nc = (int64_t)m.cut_list.size(), ns = (int64_t)m.sq.size() / 10;
    const int64_t nh = (int64_t)m.sq_hosts.size();
    constexpr int EPB = JacShape<T>::EPB;
    if (no > 0) jac_out<T, BSR><<<(unsigned)((no + EPB - 1) / EPB), 8 * EPB, 0, s>>>(A, m.d.out_list, no, nullptr, val, nullptr);
    if (nc > 0) {
        const void* pts = sizeof(T) == 4 ? (const void*)m.d.cut_pts_f : (const void*)m.d.cut_pts;
        jac_cut<T, BSR><<<(unsigned)((nc + JWPB - 1) / JWPB), 32 * JWPB, 0, s>>>(A, m.d.cut_list, m.d.cut_off, pts, nc,
                                                                              nullptr, val, nullptr);
    }
    if (ns > 0 && nh > 0) {
        cudaMemsetAsync(m.d.slot, 0xff, (size_t)m.n_elem() * sizeof(int32_t), s);
        fill_slots<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(nh, m.d.sq_hosts, m.d.slot);
        cudaMemsetAsync(Ks, 0, (size_t)nh * 1024 * sizeof(double), s);
        jac_nitsche<T, FULL><<<(unsigned)((ns + 127) / 128), 128, 0, s>>>(A, m.d.sq_elem, m.d.sq_x, m.d.sq_n, m.d.sq_w,
                                                                        m.d.sq_taub, ns, m.d.slot, Ks, nullptr);
        scatter_kmat<<<(unsigned)((nh * 256 + 255) / 256), 256, 0, s>>>(A, m.d.sq_hosts, nh, Ks, val);
    }
}

}  // namespace

// The Jacobian assembled in 4 x 4 blocks on the mesh's block pattern: val [n_blocks][4][4] float64
// (row component, column component), K = sum_e M_e^T k_e M_e with identity rows for the prescribed
// components; Ks: workspace of 1024 doubles per surface-hosting element.
int bsr_assemble(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                 const imga_physics& ph, int precision, const int64_t* bptr, const int32_t* bidx, double* val,
                 double* Ks, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nb = (int64_t)m.bsr_idx.size(), nn = m.n_nodes();
    Args A = make_args(m, u, up, up2, f, ph, nullptr, nullptr);
    A.bptr = bptr;
    A.bidx = bidx;
    cudaMemsetAsync(val, 0, (size_t)nb * 16 * sizeof(double), s);
    if (precision == 0) launch_bsr_assembly<double>(m, A, val, Ks, s);
    else launch_bsr_assembly<float>(m, A, val, Ks, s);
    if (nn > 0)
        bsr_strong_rows<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(nn, bptr, bidx, m.d.bcflag,
                                                                    m.user_bc ? m.d.bcmask_user : nullptr, val);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int element_jacobians(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                      const imga_physics& ph, int precision, const int32_t* elems, int64_t n, double* K, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= 0) return 0;
    Args A = make_args(m, u, up, up2, f, ph, nullptr, nullptr);
    int32_t* slot = m.d.slot;
    cudaMemsetAsync(slot, 0xff, (size_t)m.n_elem() * sizeof(int32_t), s);
    fill_slots<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, elems, slot);
    cudaMemsetAsync(K, 0, (size_t)n * 1024 * sizeof(double), s);
    if (precision == 0) launch_jac<double, FULL>(m, A, slot, K, nullptr, s);
    else launch_jac<float, FULL>(m, A, slot, K, nullptr, s);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int block_jacobi_setup(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                       const imga_physics& ph, int precision, double* D, double* Dinv, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nn = m.n_nodes();
    Args A = make_args(m, u, up, up2, f, ph, nullptr, nullptr);
    cudaMemsetAsync(D, 0, (size_t)nn * 16 * sizeof(double), s);
    if (precision == 0) launch_jac<double, DIAG>(m, A, nullptr, nullptr, D, s);
    else launch_jac<float, DIAG>(m, A, nullptr, nullptr, D, s);
    if (nn > 0) {
        jac_strong_rows<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(nn, m.d.bcflag, m.user_bc ? m.d.bcmask_user : nullptr, D);
        bj_invert<<<(unsigned)((nn + 127) / 128), 128, 0, s>>>(nn, D, Dinv);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int block_jacobi_apply(const Mesh& m, const double* Dinv, const double* x, double* y, void* stream) {
    const int64_t nn = m.n_nodes();
    if (nn > 0) bj_apply<<<(unsigned)((nn + 255) / 256), 256, 0, (cudaStream_t)stream>>>(nn, Dinv, x, y);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace imga
