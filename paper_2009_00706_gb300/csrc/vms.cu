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
//                 then contracts node c's four rows over the 8 points through shared memory.
//   vms_cut       one warp per Intercepted element, 32 sub-cell points per step; lane l owns
//                 row (node l/4, component l%4) of the element vector.
//   nitsche       one thread per surface point (points sorted by element).
//   strong_rows   Dirichlet rows U - g and In-only rows, written after every scatter.

#include <cuda_runtime.h>

#include <cstdio>
#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>

#include "imga_internal.h"

namespace imga {

namespace {

// ------------------------------------------------------------------------------------------
// scalars: plain T or dual (value, tangent)
// ------------------------------------------------------------------------------------------
template <class T> struct Dual { T v, d; };

template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return {a * b.v, a * b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return {a.v * b, a.d * b}; }
template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return {a.v + b, a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, T b) { return {a.v - b, a.d}; }

template <class S> struct Base { typedef S type; };
template <class T> struct Base<Dual<T>> { typedef T type; };

template <class T> __device__ __forceinline__ T value(T a) { return a; }
template <class T> __device__ __forceinline__ T value(Dual<T> a) { return a.v; }
template <class T> __device__ __forceinline__ T tangent(T) { return T(0); }
template <class T> __device__ __forceinline__ T tangent(Dual<T> a) { return a.d; }

template <class S> __device__ __forceinline__ S zero() { return S(0); }
template <> __device__ __forceinline__ Dual<float> zero<Dual<float>>() { return {0.f, 0.f}; }
template <> __device__ __forceinline__ Dual<double> zero<Dual<double>>() { return {0.0, 0.0}; }

template <class S, class T> __device__ __forceinline__ S make(T v, T d);
template <> __device__ __forceinline__ float make<float, float>(float v, float) { return v; }
template <> __device__ __forceinline__ double make<double, double>(double v, double) { return v; }
template <> __device__ __forceinline__ Dual<float> make<Dual<float>, float>(float v, float d) { return {v, d}; }
template <> __device__ __forceinline__ Dual<double> make<Dual<double>, double>(double v, double d) { return {v, d}; }

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
template <class T> __device__ __forceinline__ Dual<T> rsq(Dual<T> x) {
    T r = rsq(x.v);
    return {r, T(-0.5) * r * r * r * x.d};
}
__device__ __forceinline__ float rcp(float x) { return 1.0f / x; }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
template <class T> __device__ __forceinline__ Dual<T> rcp(Dual<T> x) {
    T r = rcp(x.v);
    return {r, -r * r * x.d};
}

template <class T> __device__ __forceinline__ T tiny();
template <> __device__ __forceinline__ float tiny<float>() { return 1e-37f; }
template <> __device__ __forceinline__ double tiny<double>() { return 1e-300; }

// ------------------------------------------------------------------------------------------
// launch parameters
// ------------------------------------------------------------------------------------------
struct Args {
    const int32_t* conn;
    const int32_t* hpar;
    const uint8_t* lev;
    int64_t n_nodes, n_hang;
    double scale;
    float gf[16], wf[16];                // per level: 2/h and h^3/8 (Jacobian of the cube map)
    double gd[16], wd[16];
    const void* ndv;                     // node data [n_nodes + n_hang][8] of T: us(3), p, at(3), 0
    const void* ndt;                     // tangents  [n_nodes + n_hang][8] of T: dus(3), dp, dat(3), 0
    const void* ndf;                     // body force [n_nodes + n_hang][4] of T, or null
    const double* U;
    const double* Up;
    const double* Up2;
    const double* F;
    const double* V;
    double* out;
    double rho, mu, theta, c0, c1, c2;   // c_k = time coefficients / dt
    double K0dt;                         // 4 / dt^2
    double CInu2;                        // C_I nu^2
    double irho;
    float rhof, muf, irhof, K0f, CI3f;   // float copies (CI3 = 3 C_I nu^2, the G:G factor)
    double CI3;
    double Cb;
    double g[3];
    int drop_visc;
};

// node values through the hanging-node interpolation (u_e = M_e U)
__device__ __forceinline__ void load4(const double* a, int64_t i, double o[4]) {
    const double2* p = reinterpret_cast<const double2*>(a + 4 * i);
    double2 x = __ldg(p), y = __ldg(p + 1);
    o[0] = x.x; o[1] = x.y; o[2] = y.x; o[3] = y.y;
}
__device__ __forceinline__ void gather(const Args& A, const double* arr, int32_t id, double o[4]) {
    if (id < A.n_nodes) { load4(arr, id, o); return; }
    const int32_t* hp = A.hpar + 4 * (int64_t)(id - A.n_nodes);
    int np = hp[2] >= 0 ? 4 : 2;
    double t[4];
    o[0] = o[1] = o[2] = o[3] = 0.0;
    for (int k = 0; k < np; ++k) {
        load4(arr, hp[k], t);
        o[0] += t[0]; o[1] += t[1]; o[2] += t[2]; o[3] += t[3];
    }
    double w = np == 4 ? 0.25 : 0.5;
    o[0] *= w; o[1] *= w; o[2] *= w; o[3] *= w;
}

// scatter one node's 4 values through M_e^T
__device__ __forceinline__ void scatter(const Args& A, int32_t id, const double r[4]) {
    if (id < A.n_nodes) {
        double* o = A.out + 4 * (int64_t)id;
        for (int k = 0; k < 4; ++k) atomicAdd(o + k, r[k]);
        return;
    }
    const int32_t* hp = A.hpar + 4 * (int64_t)(id - A.n_nodes);
    int np = hp[2] >= 0 ? 4 : 2;
    double w = np == 4 ? 0.25 : 0.5;
    for (int p = 0; p < np; ++p) {
        double* o = A.out + 4 * (int64_t)hp[p];
        for (int k = 0; k < 4; ++k) atomicAdd(o + k, w * r[k]);
    }
}

// Node data, prepared once per call by node_prep for every independent node and every hanging
// node (the latter interpolated from its parents, u_e = M_e U), so the element kernels gather
// with plain loads and no float64 arithmetic:
//   us = theta u + (1-theta) u_prev (spatial state; theta = 1/2 is Crank-Nicolson), p,
//   at = (c0 u + c1 u_prev + c2 u_prev2)/dt = c0 (u - u_prev) + c2 (u_prev2 - u_prev)
//        (c0 + c1 + c2 = 0), the differences taken in float64 before rounding to T,
//   and for J v the tangents dus = theta v, dp = v_p, dat = c0 v.
// corner row in shared memory: node value row (us, p, at, 0) | tangent row (dus, dp, dat, 0) |
// force row (f, 0); 20 T, a multiple of 16 bytes so rows can be filled by 16-byte async copies
constexpr int CT = 8, CF = 16, CS = 20;

template <class T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { typedef double4 type; };

template <class T>
__device__ __forceinline__ void ld8(const void* base, int64_t i, T o[8]) {
    if constexpr (sizeof(T) == 4) {
        const float4* p = reinterpret_cast<const float4*>(base) + 2 * i;
        float4 a = __ldg(p), b = __ldg(p + 1);
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    } else {
        const double2* p = reinterpret_cast<const double2*>(base) + 4 * i;
        double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y; o[4] = c.x; o[5] = c.y; o[6] = d.x; o[7] = d.y;
    }
}
template <class T>
__device__ __forceinline__ void ld4(const void* base, int64_t i, T o[4]) {
    if constexpr (sizeof(T) == 4) {
        float4 a = __ldg(reinterpret_cast<const float4*>(base) + i);
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    } else {
        const double2* p = reinterpret_cast<const double2*>(base) + 2 * i;
        double2 a = __ldg(p), b = __ldg(p + 1);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
}

template <class T, bool JV>
__device__ __forceinline__ void corner_data(const Args& A, int32_t id, T* dst) {
    ld8<T>(A.ndv, id, dst);
    if (JV) ld8<T>(A.ndt, id, dst + CT);
    if (A.ndf) ld4<T>(A.ndf, id, dst + CF);
    else dst[CF] = dst[CF + 1] = dst[CF + 2] = dst[CF + 3] = T(0);
}

// 16-byte asynchronous global -> shared copy (bypasses registers and L1)
__device__ __forceinline__ void cp16(void* sdst, const void* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <class T, bool JV>
__device__ __forceinline__ void corner_async(const Args& A, int32_t id, T* dst) {
    constexpr int C8 = 8 * sizeof(T) / 16;   // 16-byte chunks in a row of 8 T
    const char* v = reinterpret_cast<const char*>(A.ndv) + (size_t)id * 8 * sizeof(T);
    for (int k = 0; k < C8; ++k) cp16(reinterpret_cast<char*>(dst) + 16 * k, v + 16 * k);
    if (JV) {
        const char* t = reinterpret_cast<const char*>(A.ndt) + (size_t)id * 8 * sizeof(T);
        for (int k = 0; k < C8; ++k) cp16(reinterpret_cast<char*>(dst + CT) + 16 * k, t + 16 * k);
    }
    if (A.ndf) {
        const char* f = reinterpret_cast<const char*>(A.ndf) + (size_t)id * 4 * sizeof(T);
        for (int k = 0; k < C8 / 2; ++k) cp16(reinterpret_cast<char*>(dst + CF) + 16 * k, f + 16 * k);
    } else {
        dst[CF] = dst[CF + 1] = dst[CF + 2] = dst[CF + 3] = T(0);
    }
}

template <class T, bool JV>
__global__ void __launch_bounds__(256) node_prep(Args A, T* __restrict__ ndv, T* __restrict__ ndt, T* __restrict__ ndf) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= A.n_nodes + A.n_hang) return;
    const int32_t id = (int32_t)n;
    double u[4], up[4], up2[4] = {0, 0, 0, 0};
    gather(A, A.U, id, u);
    gather(A, A.Up, id, up);
    if (A.c2 != 0.0) gather(A, A.Up2, id, up2);
    T v8[8];
    for (int k = 0; k < 3; ++k) {
        v8[k] = A.theta == 1.0 ? (T)u[k] : (T)(A.theta * u[k] + (1.0 - A.theta) * up[k]);
        T d1 = (T)(u[k] - up[k]);
        T d2 = A.c2 != 0.0 ? (T)(up2[k] - up[k]) : T(0);
        v8[4 + k] = (T)A.c0 * d1 + (T)A.c2 * d2;
    }
    v8[3] = (T)u[3];
    v8[7] = T(0);
    for (int k = 0; k < 8; ++k) ndv[8 * n + k] = v8[k];
    if (ndf) {
        double f[4];
        gather(A, A.F, id, f);
        for (int k = 0; k < 3; ++k) ndf[4 * n + k] = (T)f[k];
        ndf[4 * n + 3] = T(0);
    }
    if (JV) {
        double v[4];
        gather(A, A.V, id, v);
        T vt[4] = {(T)v[0], (T)v[1], (T)v[2], (T)v[3]};
        T t8[8];
        for (int k = 0; k < 3; ++k) { t8[k] = (T)A.theta * vt[k]; t8[4 + k] = (T)A.c0 * vt[k]; }
        t8[3] = vt[3];
        t8[7] = T(0);
        for (int k = 0; k < 8; ++k) ndt[8 * n + k] = t8[k];
    }
}

// physical constants in the element precision
template <class T> struct Phys;
template <> struct Phys<float> {
    float rho, mu, irho, K0, CI3;
    __device__ Phys(const Args& A) : rho(A.rhof), mu(A.muf), irho(A.irhof), K0(A.K0f), CI3(A.CI3f) {}
};
template <> struct Phys<double> {
    double rho, mu, irho, K0, CI3;
    __device__ Phys(const Args& A) : rho(A.rho), mu(A.mu), irho(A.irho), K0(A.K0dt), CI3(A.CI3) {}
};

template <class T> __device__ __forceinline__ T lvl_g(const Args& A, int l);
template <> __device__ __forceinline__ float lvl_g<float>(const Args& A, int l) { return A.gf[l]; }
template <> __device__ __forceinline__ double lvl_g<double>(const Args& A, int l) { return A.gd[l]; }
template <class T> __device__ __forceinline__ T lvl_w(const Args& A, int l);
template <> __device__ __forceinline__ float lvl_w<float>(const Args& A, int l) { return A.wf[l]; }
template <> __device__ __forceinline__ double lvl_w<double>(const Args& A, int l) { return A.wd[l]; }

// Q1 basis at reference point xi: values, reference-cube first derivatives d/dxi and mixed
// second derivatives; physical derivatives are these times g = 2/h (g^2), applied to the
// interpolated fields rather than to every basis function.
template <class T>
struct Basis {
    T phi[8], dphi[8][3], d2[8][3];   // d2: (01, 02, 12) mixed second derivatives
};
template <class T>
__device__ __forceinline__ void basis(const T xi[3], Basis<T>& B) {
    T fm[3], fp[3];
    for (int k = 0; k < 3; ++k) { fm[k] = T(0.5) * (T(1) - xi[k]); fp[k] = T(0.5) * (T(1) + xi[k]); }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        T f0 = (c & 1) ? fp[0] : fm[0], f1 = (c & 2) ? fp[1] : fm[1], f2 = (c & 4) ? fp[2] : fm[2];
        T h0 = (c & 1) ? T(0.5) : T(-0.5), h1 = (c & 2) ? T(0.5) : T(-0.5), h2 = (c & 4) ? T(0.5) : T(-0.5);
        T f01 = f0 * f1;
        B.phi[c] = f01 * f2;
        B.dphi[c][0] = h0 * (f1 * f2);
        B.dphi[c][1] = h1 * (f0 * f2);
        B.dphi[c][2] = h2 * f01;
        B.d2[c][0] = (h0 * h1) * f2;
        B.d2[c][1] = (h0 * h2) * f1;
        B.d2[c][2] = (h1 * h2) * f0;
    }
}

// Pointwise VMS: fields at a quadrature point -> the 16 coefficients (F, S, G, H).  The S and H
// coefficients come out divided by g (they multiply reference derivatives in the contraction).
template <class S, class T>
__device__ __forceinline__ void vms_point(const Args& A, const T fm[3], const T fp[3], const T* nd /*[8][CS]*/,
                                          int stride, T g, S out[16]) {
    S us[3], Gu[3][3], p = zero<S>(), gp[3], at[3], H2[3];
    T f[3] = {T(0), T(0), T(0)};
    for (int i = 0; i < 3; ++i) {
        us[i] = zero<S>(); at[i] = zero<S>(); gp[i] = zero<S>(); H2[i] = zero<S>();
        for (int j = 0; j < 3; ++j) Gu[i][j] = zero<S>();
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const T* q = nd + c * stride;
        // basis of corner c at the point, formed on the fly (keeps no 8-corner tables live)
        const T f0 = (c & 1) ? fp[0] : fm[0], f1 = (c & 2) ? fp[1] : fm[1], f2 = (c & 4) ? fp[2] : fm[2];
        const T h0 = (c & 1) ? T(0.5) : T(-0.5), h1 = (c & 2) ? T(0.5) : T(-0.5), h2 = (c & 4) ? T(0.5) : T(-0.5);
        const T f01 = f0 * f1;
        const T ph = f01 * f2;
        const T dph[3] = {h0 * (f1 * f2), h1 * (f0 * f2), h2 * f01};
        const T d2[3] = {(h0 * h1) * f2, (h0 * h2) * f1, (h1 * h2) * f0};
        S vu[3], vp, va[3];
        if constexpr (std::is_same<S, T>::value) {
            for (int k = 0; k < 3; ++k) { vu[k] = q[k]; va[k] = q[4 + k]; }
            vp = q[3];
        } else {
            for (int k = 0; k < 3; ++k) { vu[k] = make<S, T>(q[k], q[CT + k]); va[k] = make<S, T>(q[4 + k], q[CT + 4 + k]); }
            vp = make<S, T>(q[3], q[CT + 3]);
        }
        p = p + ph * vp;
        for (int i = 0; i < 3; ++i) {
            us[i] = us[i] + ph * vu[i];
            at[i] = at[i] + ph * va[i];
            gp[i] = gp[i] + dph[i] * vp;
            for (int j = 0; j < 3; ++j) Gu[i][j] = Gu[i][j] + dph[j] * vu[i];
        }
        // (grad div u)_i = sum_{j != i} d_i d_j u_j  (trilinear: d_j d_j phi = 0)
        H2[0] = H2[0] + d2[0] * vu[1] + d2[1] * vu[2];
        H2[1] = H2[1] + d2[0] * vu[0] + d2[2] * vu[2];
        H2[2] = H2[2] + d2[1] * vu[0] + d2[2] * vu[1];
    }
    if (A.ndf) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const T ph = ((c & 1) ? fp[0] : fm[0]) * ((c & 2) ? fp[1] : fm[1]) * ((c & 4) ? fp[2] : fm[2]);
            for (int i = 0; i < 3; ++i) f[i] = f[i] + ph * nd[c * stride + CF + i];
        }
    }
    const Phys<T> P(A);
    const T g2 = g * g;
    for (int i = 0; i < 3; ++i) {
        gp[i] = g * gp[i];
        H2[i] = g2 * H2[i];
        for (int j = 0; j < 3; ++j) Gu[i][j] = g * Gu[i][j];
    }
    S divu = Gu[0][0] + Gu[1][1] + Gu[2][2];
    S conv[3], rM[3];
    for (int i = 0; i < 3; ++i) {
        conv[i] = Gu[i][0] * us[0] + Gu[i][1] * us[1] + Gu[i][2] * us[2];
        S r = P.rho * (at[i] + conv[i] - f[i]) + gp[i];
        rM[i] = A.drop_visc ? r : r - P.mu * H2[i];
    }
    // tau_M = (4/dt^2 + u.G u + C_I nu^2 G:G)^(-1/2), G = g^2 I;  tau_C = 1 / (tau_M tr G)
    S uu = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
    S tauM = rsq(g2 * uu + (P.K0 + P.CI3 * (g2 * g2)));
    S tauC = rcp((T(3) * g2) * tauM);
    S up[3];
    for (int i = 0; i < 3; ++i) up[i] = -(tauM * rM[i]);
    S pp = -(P.rho * tauC * divu);
    S q = g2 * (up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
    bool bar = value(q) > tiny<T>();
    S taubar = bar ? rsq(q) : zero<S>();
    S Gup[3];
    for (int i = 0; i < 3; ++i) Gup[i] = Gu[i][0] * up[0] + Gu[i][1] * up[1] + Gu[i][2] * up[2];
    const T ig = T(1) / g;
    for (int i = 0; i < 3; ++i) {
        out[i] = P.rho * (at[i] + conv[i] - f[i]) + Gup[i];
        S tb = taubar * Gup[i];
        for (int j = 0; j < 3; ++j) {
            S sij = P.mu * (Gu[i][j] + Gu[j][i]) - up[i] * us[j] - P.irho * (up[i] * up[j]) + tb * up[j];
            if (i == j) sij = sij - p - pp;
            out[3 + 3 * i + j] = sij;
        }
        out[13 + i] = -(P.irho * up[i]);
    }
    out[12] = divu;
    (void)ig;
}

template <class T, bool JV> struct Pick;
template <class T> struct Pick<T, false> { template <class S> __device__ static T get(S x) { return value(x); } };
template <class T> struct Pick<T, true> { template <class S> __device__ static T get(S x) { return tangent(x); } };

// ------------------------------------------------------------------------------------------
// Out elements: 8 threads per element
// ------------------------------------------------------------------------------------------
template <class T> struct Epb { static constexpr int value = sizeof(T) == 8 ? 16 : 32; };   // elements per block

template <class T> struct IntShape {
    static constexpr int EPB = Epb<T>::value;                                   // elements per block
    static constexpr int THREADS = 8 * EPB;
    static constexpr size_t smem = (size_t)(2 * EPB * 8 * CS + EPB * 8 * 17) * sizeof(T);
};

// Persistent: a block walks element groups with a grid stride; while it computes group g its
// threads already stream the node rows of group g + stride into the other shared buffer
// (cp.async), so the gather latency hides behind the arithmetic.  Thread c of an element
// gathers corner c, evaluates Gauss point c, then contracts node c's four rows.
template <class T, bool JV>
__global__ void __launch_bounds__(IntShape<T>::THREADS, 2) vms_interior(Args A, const int32_t* __restrict__ oconn,
                                                    const uint8_t* __restrict__ olev, int64_t n) {
    typedef typename std::conditional<JV, Dual<T>, T>::type S;
    constexpr int EPB = IntShape<T>::EPB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s_nd = reinterpret_cast<T*>(smem_raw);          // [2][EPB][8][CS]
    T* s_cf = s_nd + 2 * EPB * 8 * CS;                  // [EPB][8][17]
    const int c = threadIdx.x & 7, le = threadIdx.x >> 3;
    const int64_t ngroups = (n + EPB - 1) / EPB;
    int64_t gi = blockIdx.x;
    if (gi >= ngroups) return;
    auto corner_id = [&](int64_t grp) -> int32_t {
        int64_t idx = grp * EPB + le;
        if (idx >= n) idx = n - 1;
        return __ldg(oconn + 8 * idx + c);
    };
    auto row = [&](int buf) -> T* { return s_nd + ((buf * EPB + le) * 8 + c) * CS; };
    int32_t id_cur = corner_id(gi);
    corner_async<T, JV>(A, id_cur, row(0));
    cp_commit();
    int32_t id_next = gi + gridDim.x < ngroups ? corner_id(gi + gridDim.x) : 0;
    const T gauss = (T)0.57735026918962576451;
    const T wp = T(0.5) * (T(1) + gauss), wm = T(0.5) * (T(1) - gauss);
    // Gauss point c: 1D factors (1 -/+ xi_k)/2 take the values wp, wm
    T fm[3], fp[3];
    for (int k = 0; k < 3; ++k) {
        const bool plus = (c >> k) & 1;
        fm[k] = plus ? wm : wp;
        fp[k] = plus ? wp : wm;
    }
    int buf = 0;
    for (; gi < ngroups; gi += gridDim.x) {
        const int64_t gnext = gi + gridDim.x;
        if (gnext < ngroups) corner_async<T, JV>(A, id_next, row(buf ^ 1));
        cp_commit();
        const int32_t id_after = gnext + gridDim.x < ngroups ? corner_id(gnext + gridDim.x) : 0;
        cp_wait<1>();
        __syncwarp();
        const int64_t idx = gi * EPB + le;
        const bool valid = idx < n;
        const int lv = __ldg(olev + (valid ? idx : n - 1));
        const T g = lvl_g<T>(A, lv);
        S cf[16];
        vms_point<S, T>(A, fm, fp, s_nd + (buf * EPB + le) * 8 * CS, CS, g, cf);
        const T wq = lvl_w<T>(A, lv), wqg = wq * g;
        T* mycf = s_cf + (le * 8 + c) * 17;
        // F, G multiply phi; S, H multiply physical gradients = g x reference gradients
        for (int k = 0; k < 16; ++k) mycf[k] = ((k < 3 || k == 12) ? wq : wqg) * Pick<T, JV>::get(cf[k]);
        __syncwarp();
        T r[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            T f[3], d[3];
            for (int k = 0; k < 3; ++k) {
                bool same = (((c >> k) & 1) == ((q >> k) & 1));
                f[k] = same ? wp : wm;
                d[k] = ((c >> k) & 1) ? T(0.5) : T(-0.5);
            }
            T ph = f[0] * f[1] * f[2];
            T dp[3] = {d[0] * f[1] * f[2], d[1] * f[0] * f[2], d[2] * f[0] * f[1]};
            const T* C = s_cf + (le * 8 + q) * 17;
            for (int i = 0; i < 3; ++i) r[i] += ph * C[i] + dp[0] * C[3 + 3 * i] + dp[1] * C[4 + 3 * i] + dp[2] * C[5 + 3 * i];
            r[3] += ph * C[12] + dp[0] * C[13] + dp[1] * C[14] + dp[2] * C[15];
        }
        if (valid) {
            double rd[4] = {(double)r[0], (double)r[1], (double)r[2], (double)r[3]};
            scatter(A, id_cur, rd);
        }
        __syncwarp();   // this buffer and s_cf are rewritten by later iterations
        id_cur = id_next;
        id_next = id_after;
        buf ^= 1;
    }
    cp_wait<0>();
}

// ------------------------------------------------------------------------------------------
// Intercepted elements: one warp per element
// ------------------------------------------------------------------------------------------
constexpr int WPB = 4;   // warps per block

template <class T> __device__ __forceinline__ void load_pt(const void* pts, int64_t q, T o[4]);
template <> __device__ __forceinline__ void load_pt<double>(const void* pts, int64_t q, double o[4]) {
    const double2* p = reinterpret_cast<const double2*>(pts) + 2 * q;
    double2 a = __ldg(p), b = __ldg(p + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
template <> __device__ __forceinline__ void load_pt<float>(const void* pts, int64_t q, float o[4]) {
    float4 a = __ldg(reinterpret_cast<const float4*>(pts) + q);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}

template <class T, bool JV>
__global__ void __launch_bounds__(32 * WPB) vms_cut(Args A, const int32_t* __restrict__ list, const int64_t* __restrict__ off,
                                                    const void* __restrict__ pts, int64_t n) {
    typedef typename std::conditional<JV, Dual<T>, T>::type S;
    __shared__ T s_nd[WPB][8][CS];
    __shared__ T s_cf[WPB][32][20];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t idx = (int64_t)blockIdx.x * WPB + w;
    if (idx >= n) return;
    const int32_t e = list[idx];
    int32_t my_id = 0;
    if (lane < 8) {
        my_id = A.conn[8 * (int64_t)e + lane];
        corner_data<T, JV>(A, my_id, &s_nd[w][lane][0]);
    }
    __syncwarp();
    const T g = lvl_g<T>(A, A.lev[e]);
    const T det = lvl_w<T>(A, A.lev[e]);
    const int a = lane >> 2, comp = lane & 3;
    const T sa[3] = {(a & 1) ? T(1) : T(-1), (a & 2) ? T(1) : T(-1), (a & 4) ? T(1) : T(-1)};
    T acc = T(0);
    const int64_t q0 = off[idx], q1 = off[idx + 1];
    for (int64_t base = q0; base < q1; base += 32) {
        const int64_t q = base + lane;
        if (q < q1) {
            T pt[4];
            load_pt<T>(pts, q, pt);
            T fm[3], fp[3];
            for (int k = 0; k < 3; ++k) { fm[k] = T(0.5) * (T(1) - pt[k]); fp[k] = T(0.5) * (T(1) + pt[k]); }
            S cf[16];
            vms_point<S, T>(A, fm, fp, &s_nd[w][0][0], CS, g, cf);
            const T wq = pt[3] * det, wqg = wq * g;
            for (int k = 0; k < 16; ++k) s_cf[w][lane][k] = ((k < 3 || k == 12) ? wq : wqg) * Pick<T, JV>::get(cf[k]);
            s_cf[w][lane][16] = pt[0];
            s_cf[w][lane][17] = pt[1];
            s_cf[w][lane][18] = pt[2];
        } else {
            for (int k = 0; k < 19; ++k) s_cf[w][lane][k] = T(0);
        }
        __syncwarp();
        const int m = (int)min((int64_t)32, q1 - base);
        for (int j = 0; j < m; ++j) {
            const T* C = s_cf[w][j];
            T f0 = T(0.5) * (T(1) + sa[0] * C[16]), f1 = T(0.5) * (T(1) + sa[1] * C[17]), f2 = T(0.5) * (T(1) + sa[2] * C[18]);
            T ph = f0 * f1 * f2;
            T d0 = T(0.5) * sa[0] * f1 * f2, d1 = T(0.5) * sa[1] * f0 * f2, d2 = T(0.5) * sa[2] * f0 * f1;
            if (comp < 3) acc += ph * C[comp] + d0 * C[3 + 3 * comp] + d1 * C[4 + 3 * comp] + d2 * C[5 + 3 * comp];
            else acc += ph * C[12] + d0 * C[13] + d1 * C[14] + d2 * C[15];
        }
        __syncwarp();
    }
    // gather the four components of node a into lane 4a, then scatter
    double r[4];
    for (int k = 0; k < 4; ++k) r[k] = (double)__shfl_sync(0xffffffffu, acc, (lane & ~3) + k);
    int32_t id = __shfl_sync(0xffffffffu, my_id, a);
    if (comp == 0) scatter(A, id, r);
}

// ------------------------------------------------------------------------------------------
// Nitsche surface terms, one thread per surface point
// ------------------------------------------------------------------------------------------
template <class T, bool JV>
__global__ void __launch_bounds__(128) nitsche(Args A, const int32_t* __restrict__ el, const double* __restrict__ xr,
                                               const double* __restrict__ nr, const double* __restrict__ wr,
                                               const double* __restrict__ taub, int64_t n) {
    typedef typename std::conditional<JV, Dual<T>, T>::type S;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t e = el[i];
    const T g = lvl_g<T>(A, A.lev[e]);
    T xi[3] = {(T)xr[3 * i], (T)xr[3 * i + 1], (T)xr[3 * i + 2]};
    const T nn[3] = {(T)nr[3 * i], (T)nr[3 * i + 1], (T)nr[3 * i + 2]};
    Basis<T> B;
    basis<T>(xi, B);
    // u_s, p and grad u_s from the node data; the velocity jump d = u_s - g from corner values
    // formed in float64 (the penalty multiplies it by tau_B, up to 100 C_b mu / h on slivers)
    S us[3], Gu[3][3], p = zero<S>(), d[3];
    int32_t ids[8];
    for (int k = 0; k < 3; ++k) { us[k] = zero<S>(); d[k] = zero<S>(); for (int j = 0; j < 3; ++j) Gu[k][j] = zero<S>(); }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        ids[c] = A.conn[8 * (int64_t)e + c];
        T a8[8], t8[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        ld8<T>(A.ndv, ids[c], a8);
        if (JV) ld8<T>(A.ndt, ids[c], t8);
        double u4[4], up4[4];
        gather(A, A.U, ids[c], u4);
        if (A.theta != 1.0) gather(A, A.Up, ids[c], up4);
        const T ph = B.phi[c];
        for (int k = 0; k < 3; ++k) {
            S vu = make<S, T>(a8[k], t8[k]);
            double usk = A.theta == 1.0 ? u4[k] : A.theta * u4[k] + (1.0 - A.theta) * up4[k];
            S jump = make<S, T>((T)(usk - A.g[k]), t8[k]);
            us[k] = us[k] + ph * vu;
            d[k] = d[k] + ph * jump;
            for (int j = 0; j < 3; ++j) Gu[k][j] = Gu[k][j] + B.dphi[c][j] * vu;
        }
        p = p + ph * make<S, T>(a8[3], t8[3]);
    }
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) Gu[k][j] = g * Gu[k][j];
    const Phys<T> P(A);
    S un = us[0] * nn[0] + us[1] * nn[1] + us[2] * nn[2];
    S dn = d[0] * nn[0] + d[1] * nn[1] + d[2] * nn[2];
    const bool inflow = value(un) < T(0);
    S tr[3];
    for (int k = 0; k < 3; ++k)
        tr[k] = P.mu * ((Gu[k][0] + Gu[0][k]) * nn[0] + (Gu[k][1] + Gu[1][k]) * nn[1] + (Gu[k][2] + Gu[2][k]) * nn[2]) - p * nn[k];
    const T w = (T)wr[i];
    const T tauB = (T)(A.Cb * A.mu * taub[i]);    // tau_TAN = tau_NOR: both penalty parts sum to tau_B (u - g)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const T ph = B.phi[c];
        const T gn = g * (B.dphi[c][0] * nn[0] + B.dphi[c][1] * nn[1] + B.dphi[c][2] * nn[2]);
        S gd = g * (B.dphi[c][0] * d[0] + B.dphi[c][1] * d[1] + B.dphi[c][2] * d[2]);
        double r[4];
        for (int k = 0; k < 3; ++k) {
            S t = (tauB * ph) * d[k] - ph * tr[k] - P.mu * (gn * d[k] + nn[k] * gd);
            if (inflow) t = t - (ph * P.rho) * (un * d[k]);
            r[k] = (double)(w * Pick<T, JV>::get(t));
        }
        r[3] = (double)(w * Pick<T, JV>::get(-(ph * dn)));
        scatter(A, ids[c], r);
    }
}

// ------------------------------------------------------------------------------------------
// strong rows
// ------------------------------------------------------------------------------------------
__global__ void strong_rows(Args A, const uint8_t* __restrict__ flag, const uint8_t* __restrict__ umask,
                            const double* __restrict__ uval, double ux, double uy, double uz, int jv) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= A.n_nodes) return;
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

// optional event pair around a launch (profiling)
struct Timed {
    Mesh* m;
    int k;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    Timed(const Mesh& mesh, int kind, cudaStream_t st) : m(const_cast<Mesh*>(&mesh)), k(kind), s(st) {
        if (!m->profiling) return;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    ~Timed() {
        if (!a) return;
        cudaEventRecord(b, s);
        m->prof_ev[k].push_back({(void*)a, (void*)b});
    }
};

template <class T, bool JV>
void launch_all(const Mesh& m, Args A, cudaStream_t s, void* ws = nullptr) {
    const int64_t next = m.n_nodes() + m.n_hang();
    T* ndv = ws ? (T*)ws : sizeof(T) == 4 ? (T*)(void*)m.d.nd_f : (T*)(void*)m.d.nd_d;
    T* ndt = ndv + 8 * next;
    T* ndf = A.F ? ndt + 8 * next : nullptr;
    A.ndv = ndv;
    A.ndt = ndt;
    A.ndf = ndf;
    if (next > 0) {
        Timed t(m, 4, s);
        node_prep<T, JV><<<(unsigned)((next + 255) / 256), 256, 0, s>>>(A, ndv, ndt, ndf);
    }
    const int64_t no = (int64_t)m.out_list.size(), nc = (int64_t)m.cut_list.size(), ns = (int64_t)m.sq.size() / 10;
    constexpr int EPB = Epb<T>::value;
    if (no > 0) {
        Timed t(m, 0, s);
        static int per_sm[2][2] = {{0, 0}, {0, 0}};
        int& bps = per_sm[sizeof(T) == 8][JV];
        const size_t smem = IntShape<T>::smem;
        if (bps == 0) {
            cudaFuncSetAttribute(vms_interior<T, JV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, vms_interior<T, JV>, 8 * EPB, smem);
            if (bps < 1) bps = 1;
        }
        const int64_t groups = (no + EPB - 1) / EPB;
        const int64_t grid = std::min<int64_t>(groups, (int64_t)bps * m.n_sm);
        vms_interior<T, JV><<<(unsigned)grid, 8 * EPB, smem, s>>>(A, m.d.out_conn, m.d.out_lev, no);
    }
    if (nc > 0) {
        Timed t(m, 1, s);
        const void* pts = std::is_same<T, float>::value ? (const void*)m.d.cut_pts_f : (const void*)m.d.cut_pts;
        vms_cut<T, JV><<<(unsigned)((nc + WPB - 1) / WPB), 32 * WPB, 0, s>>>(A, m.d.cut_list, m.d.cut_off, pts, nc);
    }
    if (ns > 0) {
        Timed t(m, 2, s);
        nitsche<T, JV><<<(unsigned)((ns + 127) / 128), 128, 0, s>>>(A, m.d.sq_elem, m.d.sq_x, m.d.sq_n, m.d.sq_w,
                                                                    m.d.sq_taub, ns);
    }
}

}  // namespace

static int vms_apply_ws(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                        const imga_physics& ph, int precision, const double* v, double* out, void* stream, void* ws) {
    cudaStream_t s = (cudaStream_t)stream;
    Args A;
    A.conn = m.d.conn;
    A.hpar = m.d.hpar;
    A.lev = m.d.lev;
    A.n_nodes = m.n_nodes();
    A.scale = m.scale;
    A.n_hang = m.n_hang();
    for (int l = 0; l < 16; ++l) {
        double h = (double)(1u << (kMaxDepth - l)) * m.scale;
        A.gd[l] = 2.0 / h;
        A.wd[l] = 0.125 * h * h * h;
        A.gf[l] = (float)A.gd[l];
        A.wf[l] = (float)A.wd[l];
    }
    A.ndv = A.ndt = A.ndf = nullptr;
    A.U = u;
    A.Up = up;
    A.Up2 = up2 ? up2 : up;
    A.F = f;
    A.V = v;
    A.out = out;
    A.rho = ph.rho;
    A.mu = ph.mu;
    double c[3], theta;
    if (ph.time_scheme == 2) { c[0] = 1.5; c[1] = -2.0; c[2] = 0.5; theta = 1.0; }
    else if (ph.time_scheme == 1) { c[0] = 1.0; c[1] = -1.0; c[2] = 0.0; theta = 0.5; }
    else { c[0] = 1.0; c[1] = -1.0; c[2] = 0.0; theta = 1.0; }
    A.theta = theta;
    A.c0 = c[0] / ph.dt;
    A.c1 = c[1] / ph.dt;
    A.c2 = c[2] / ph.dt;
    A.K0dt = 4.0 / (ph.dt * ph.dt);
    const double nu = ph.mu / ph.rho;
    A.CInu2 = ph.C_I * nu * nu;
    A.CI3 = 3.0 * A.CInu2;
    A.irho = 1.0 / ph.rho;
    A.rhof = (float)ph.rho;
    A.muf = (float)ph.mu;
    A.irhof = (float)A.irho;
    A.K0f = (float)A.K0dt;
    A.CI3f = (float)A.CI3;
    A.Cb = ph.C_b;
    for (int k = 0; k < 3; ++k) A.g[k] = ph.g_body[k];
    A.drop_visc = ph.drop_visc_strong;
    const bool jv = v != nullptr;
    if (cudaMemsetAsync(out, 0, (size_t)m.n_nodes() * 4 * sizeof(double), s) != cudaSuccess) return 1;
    if (precision == 0) {
        if (jv) launch_all<double, true>(m, A, s, ws); else launch_all<double, false>(m, A, s, ws);
    } else {
        if (jv) launch_all<float, true>(m, A, s, ws); else launch_all<float, false>(m, A, s, ws);
    }
    const int64_t nn = m.n_nodes();
    Timed t(m, 3, s);
    if (nn > 0)
        strong_rows<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(A, m.d.bcflag, m.user_bc ? m.d.bcmask_user : nullptr,
                                                                m.user_bc ? m.d.bcval_user : nullptr, ph.u_inf[0],
                                                                ph.u_inf[1], ph.u_inf[2], jv ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
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

void profile_reset(Mesh& m) {
    for (int k = 0; k < 5; ++k) {
        for (auto& p : m.prof_ev[k]) { cudaEventDestroy((cudaEvent_t)p.first); cudaEventDestroy((cudaEvent_t)p.second); }
        m.prof_ev[k].clear();
        m.prof_ms[k] = 0.0;
        m.prof_n[k] = 0;
    }
}

int profile_collect(Mesh& m) {
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    for (int k = 0; k < 5; ++k) {
        for (auto& p : m.prof_ev[k]) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, (cudaEvent_t)p.first, (cudaEvent_t)p.second);
            m.prof_ms[k] += ms;
            m.prof_n[k] += 1;
            cudaEventDestroy((cudaEvent_t)p.first);
            cudaEventDestroy((cudaEvent_t)p.second);
        }
        m.prof_ev[k].clear();
    }
    return 0;
}

}  // namespace imga
