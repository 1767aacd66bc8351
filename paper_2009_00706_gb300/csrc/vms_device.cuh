// Device building blocks of the VMS residual / J v kernels, shared by the residual and J v
// kernels (vms.cu) and the element-Jacobian kernels (jac.cu): scalars and dual numbers, launch
// arguments, node gathers through the hanging-node operator, the per-call node data, the Q1
// basis and the pointwise VMS coefficients of Eqs. (vms), (uprime), (pprime).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
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
    // batched meshes: element -> problem and the viscosity of every problem (null: the scalars)
    const uint16_t* eprob;
    const double* pmu;
    const float* pmuf;
    double CI;
    float CIf;
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
    // p: problem of the element in a batched mesh, or -1
    __device__ Phys(const Args& A, int p) : rho(A.rhof), mu(A.muf), irho(A.irhof), K0(A.K0f), CI3(A.CI3f) {
        if (p >= 0) { mu = A.pmuf[p]; const float nu = mu * irho; CI3 = 3.f * A.CIf * nu * nu; }
    }
};
template <> struct Phys<double> {
    double rho, mu, irho, K0, CI3;
    __device__ Phys(const Args& A, int p) : rho(A.rho), mu(A.mu), irho(A.irho), K0(A.K0dt), CI3(A.CI3) {
        if (p >= 0) { mu = A.pmu[p]; const double nu = mu * irho; CI3 = 3.0 * A.CI * nu * nu; }
    }
};

// problem of element e in a batched mesh, -1 otherwise
__device__ __forceinline__ int prob_of(const Args& A, int32_t e) { return A.eprob ? (int)A.eprob[e] : -1; }

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

// Fields of the VMS integrand at one point (physical derivatives): spatial-state velocity u_s,
// its gradient, pressure and gradient, time derivative, (grad div u)_i, body force.
template <class S, class T>
struct Fields {
    S us[3], Gu[3][3], p, gp[3], at[3], H2[3];
    T f[3];
};

// Interpolate the fields at the point with 1D factors fm = (1 - xi)/2, fp = (1 + xi)/2 from the
// 8 corner rows nd (stride `stride`); reference derivatives are scaled by g = 2/h at the end.
template <class S, class T>
__device__ __forceinline__ void interp(const Args& A, const T fm[3], const T fp[3], const T* nd, int stride, T g,
                                       Fields<S, T>& F) {
    for (int i = 0; i < 3; ++i) {
        F.us[i] = zero<S>(); F.at[i] = zero<S>(); F.gp[i] = zero<S>(); F.H2[i] = zero<S>(); F.f[i] = T(0);
        for (int j = 0; j < 3; ++j) F.Gu[i][j] = zero<S>();
    }
    F.p = zero<S>();
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
        F.p = F.p + ph * vp;
        for (int i = 0; i < 3; ++i) {
            F.us[i] = F.us[i] + ph * vu[i];
            F.at[i] = F.at[i] + ph * va[i];
            F.gp[i] = F.gp[i] + dph[i] * vp;
            for (int j = 0; j < 3; ++j) F.Gu[i][j] = F.Gu[i][j] + dph[j] * vu[i];
        }
        // (grad div u)_i = sum_{j != i} d_i d_j u_j  (trilinear: d_j d_j phi = 0)
        F.H2[0] = F.H2[0] + d2[0] * vu[1] + d2[1] * vu[2];
        F.H2[1] = F.H2[1] + d2[0] * vu[0] + d2[2] * vu[2];
        F.H2[2] = F.H2[2] + d2[1] * vu[0] + d2[2] * vu[1];
    }
    if (A.ndf) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const T ph = ((c & 1) ? fp[0] : fm[0]) * ((c & 2) ? fp[1] : fm[1]) * ((c & 4) ? fp[2] : fm[2]);
            for (int i = 0; i < 3; ++i) F.f[i] = F.f[i] + ph * nd[c * stride + CF + i];
        }
    }
    const T g2 = g * g;
    for (int i = 0; i < 3; ++i) {
        F.gp[i] = g * F.gp[i];
        F.H2[i] = g2 * F.H2[i];
        for (int j = 0; j < 3; ++j) F.Gu[i][j] = g * F.Gu[i][j];
    }
}

// Pointwise VMS: fields -> the 16 coefficients (F, S, G, H) of Eq. (vms).
template <class S, class T>
__device__ __forceinline__ void pointwise(const Args& A, const Phys<T>& P, const Fields<S, T>& F, T g, S out[16]) {
    const T g2 = g * g;
    S divu = F.Gu[0][0] + F.Gu[1][1] + F.Gu[2][2];
    S conv[3], rM[3];
    for (int i = 0; i < 3; ++i) {
        conv[i] = F.Gu[i][0] * F.us[0] + F.Gu[i][1] * F.us[1] + F.Gu[i][2] * F.us[2];
        S r = P.rho * (F.at[i] + conv[i] - F.f[i]) + F.gp[i];
        rM[i] = A.drop_visc ? r : r - P.mu * F.H2[i];
    }
    // tau_M = (4/dt^2 + u.G u + C_I nu^2 G:G)^(-1/2), G = g^2 I;  tau_C = 1 / (tau_M tr G)
    S uu = F.us[0] * F.us[0] + F.us[1] * F.us[1] + F.us[2] * F.us[2];
    S tauM = rsq(g2 * uu + (P.K0 + P.CI3 * (g2 * g2)));
    S tauC = rcp((T(3) * g2) * tauM);
    S up[3];
    for (int i = 0; i < 3; ++i) up[i] = -(tauM * rM[i]);
    S pp = -(P.rho * tauC * divu);
    S q = g2 * (up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
    bool bar = value(q) > tiny<T>();
    S taubar = bar ? rsq(q) : zero<S>();
    S Gup[3];
    for (int i = 0; i < 3; ++i) Gup[i] = F.Gu[i][0] * up[0] + F.Gu[i][1] * up[1] + F.Gu[i][2] * up[2];
    for (int i = 0; i < 3; ++i) {
        out[i] = P.rho * (F.at[i] + conv[i] - F.f[i]) + Gup[i];
        S tb = taubar * Gup[i];
        for (int j = 0; j < 3; ++j) {
            S sij = P.mu * (F.Gu[i][j] + F.Gu[j][i]) - up[i] * F.us[j] - P.irho * (up[i] * up[j]) + tb * up[j];
            if (i == j) sij = sij - F.p - pp;
            out[3 + 3 * i + j] = sij;
        }
        out[13 + i] = -(P.irho * up[i]);
    }
    out[12] = divu;
}

template <class S, class T>
__device__ __forceinline__ void vms_point(const Args& A, const Phys<T>& P, const T fm[3], const T fp[3], const T* nd,
                                          int stride, T g, S out[16]) {
    Fields<S, T> F;
    interp<S, T>(A, fm, fp, nd, stride, g, F);
    pointwise<S, T>(A, P, F, g, out);
}

template <class T, bool JV> struct Pick;
template <class T> struct Pick<T, false> { template <class S> __device__ static T get(S x) { return value(x); } };
template <class T> struct Pick<T, true> { template <class S> __device__ static T get(S x) { return tangent(x); } };


// sub-cell point (xi, reference weight) in the element precision
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

// ------------------------------------------------------------------------------------------
// Nitsche terms of Eq. (weakbc) at one surface point
// ------------------------------------------------------------------------------------------
template <class S, class T>
struct NitschePoint {
    T g, nn[3];
    T mu, rho;
    Basis<T> B;
    int32_t ids[8];
    S us[3], Gu[3][3], p, d[3], un, dn, tr[3];
    bool inflow;
};

template <class S, class T>
__device__ __forceinline__ void finish_nitsche(const Args& A, NitschePoint<S, T>& P) {
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) P.Gu[k][j] = P.g * P.Gu[k][j];
    const T* nn = P.nn;
    P.un = P.us[0] * nn[0] + P.us[1] * nn[1] + P.us[2] * nn[2];
    P.dn = P.d[0] * nn[0] + P.d[1] * nn[1] + P.d[2] * nn[2];
    P.inflow = value(P.un) < T(0);
    for (int k = 0; k < 3; ++k)
        P.tr[k] = P.mu * ((P.Gu[k][0] + P.Gu[0][k]) * nn[0] + (P.Gu[k][1] + P.Gu[1][k]) * nn[1] +
                           (P.Gu[k][2] + P.Gu[2][k]) * nn[2]) - P.p * nn[k];
}

// u_s, p and grad u_s from the node data; the velocity jump d = u_s - g from corner values formed
// in float64 (the penalty multiplies it by tau_B, up to 100 C_b mu / h on sliver cut cells).
template <class S, class T, bool JV>
__device__ __forceinline__ void nitsche_fields(const Args& A, int32_t e, const double* xr, const double* nr,
                                               NitschePoint<S, T>& P) {
    P.g = lvl_g<T>(A, A.lev[e]);
    {
        const Phys<T> Ph(A, prob_of(A, e));
        P.mu = Ph.mu;
        P.rho = Ph.rho;
    }
    T xi[3] = {(T)xr[0], (T)xr[1], (T)xr[2]};
    for (int k = 0; k < 3; ++k) P.nn[k] = (T)nr[k];
    basis<T>(xi, P.B);
    P.p = zero<S>();
    for (int k = 0; k < 3; ++k) { P.us[k] = zero<S>(); P.d[k] = zero<S>(); for (int j = 0; j < 3; ++j) P.Gu[k][j] = zero<S>(); }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        P.ids[c] = A.conn[8 * (int64_t)e + c];
        T a8[8], t8[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        ld8<T>(A.ndv, P.ids[c], a8);
        if (JV) ld8<T>(A.ndt, P.ids[c], t8);
        double u4[4], up4[4];
        gather(A, A.U, P.ids[c], u4);
        if (A.theta != 1.0) gather(A, A.Up, P.ids[c], up4);
        const T ph = P.B.phi[c];
        for (int k = 0; k < 3; ++k) {
            S vu = make<S, T>(a8[k], t8[k]);
            double usk = A.theta == 1.0 ? u4[k] : A.theta * u4[k] + (1.0 - A.theta) * up4[k];
            S jump = make<S, T>((T)(usk - A.g[k]), t8[k]);
            P.us[k] = P.us[k] + ph * vu;
            P.d[k] = P.d[k] + ph * jump;
            for (int j = 0; j < 3; ++j) P.Gu[k][j] = P.Gu[k][j] + P.B.dphi[c][j] * vu;
        }
        P.p = P.p + ph * make<S, T>(a8[3], t8[3]);
    }
    finish_nitsche(A, P);
}

// the 4 rows of corner c (test functions phi_c e_i and q = phi_c), not yet times the weight;
// tau_TAN = tau_NOR: both penalty parts sum to tau_B (u - g)
template <class S, class T>
__device__ __forceinline__ void nitsche_rows(const Args& A, const NitschePoint<S, T>& P, int c, T tauB, S t[4]) {
    const T ph = P.B.phi[c];
    const T* nn = P.nn;
    const T gn = P.g * (P.B.dphi[c][0] * nn[0] + P.B.dphi[c][1] * nn[1] + P.B.dphi[c][2] * nn[2]);
    S gd = P.g * (P.B.dphi[c][0] * P.d[0] + P.B.dphi[c][1] * P.d[1] + P.B.dphi[c][2] * P.d[2]);
    for (int k = 0; k < 3; ++k) {
        S v = (tauB * ph) * P.d[k] - ph * P.tr[k] - P.mu * (gn * P.d[k] + nn[k] * gd);
        if (P.inflow) v = v - (ph * P.rho) * (P.un * P.d[k]);
        t[k] = v;
    }
    t[3] = -(ph * P.dn);
}

// Launch arguments from the mesh and the caller's vectors (host side).
inline Args make_args(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                      const imga_physics& ph, const double* v, double* out) {
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
    A.eprob = m.d.eprob;
    A.pmu = m.d.pmu;
    A.pmuf = m.d.pmuf;
    A.CI = ph.C_I;
    A.CIf = (float)ph.C_I;
    return A;
}

// node workspace of precision T (float or double) of the mesh: value rows, tangent rows, forces
template <class T>
inline T* node_workspace(const Mesh& m, void* ws) {
    return ws ? (T*)ws : sizeof(T) == 4 ? (T*)(void*)m.d.nd_f : (T*)(void*)m.d.nd_d;
}

}  // namespace
}  // namespace imga
