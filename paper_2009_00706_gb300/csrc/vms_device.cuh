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
// K = 1: float duals on the packed FP32x2 pipe (see below); K = 0: plain scalar arithmetic
template <class T, int K = 0> struct alignas(2 * sizeof(T)) Dual { T v, d; };

template <class T, int K> __device__ __forceinline__ Dual<T, K> operator+(Dual<T, K> a, Dual<T, K> b) { return {a.v + b.v, a.d + b.d}; }
template <class T, int K> __device__ __forceinline__ Dual<T, K> operator-(Dual<T, K> a, Dual<T, K> b) { return {a.v - b.v, a.d - b.d}; }
template <class T, int K> __device__ __forceinline__ Dual<T, K> operator-(Dual<T, K> a) { return {-a.v, -a.d}; }
template <class T, int K> __device__ __forceinline__ Dual<T, K> operator*(Dual<T, K> a, Dual<T, K> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T, int K> __device__ __forceinline__ Dual<T, K> operator*(T a, Dual<T, K> b) { return {a * b.v, a * b.d}; }
template <class T, int K> __device__ __forceinline__ Dual<T, K> operator*(Dual<T, K> a, T b) { return {a.v * b, a.d * b}; }
template <class T, int K> __device__ __forceinline__ Dual<T, K> operator+(Dual<T, K> a, T b) { return {a.v + b, a.d}; }
template <class T, int K> __device__ __forceinline__ Dual<T, K> operator-(Dual<T, K> a, T b) { return {a.v - b, a.d}; }

// Packed float duals: (value, tangent) is one register pair, so a sum, a real multiple or a fused
// real multiply-add of duals is one FP32x2 instruction.  Pays where scalars broadcast into pairs
// are reused (the Out-element kernel); kernels with higher register pressure keep K = 0.
typedef Dual<float, 1> PDual;
__device__ __forceinline__ float2 f2(PDual a) { return make_float2(a.v, a.d); }
__device__ __forceinline__ PDual df(float2 a) { return {a.x, a.y}; }
__device__ __forceinline__ PDual operator+(PDual a, PDual b) { return df(__fadd2_rn(f2(a), f2(b))); }
__device__ __forceinline__ PDual operator-(PDual a, PDual b) { return df(__ffma2_rn(f2(b), make_float2(-1.f, -1.f), f2(a))); }
__device__ __forceinline__ PDual operator*(float a, PDual b) { return df(__fmul2_rn(make_float2(a, a), f2(b))); }
__device__ __forceinline__ PDual operator*(PDual a, float b) { return df(__fmul2_rn(f2(a), make_float2(b, b))); }
__device__ __forceinline__ PDual operator*(PDual a, PDual b) {
    const float2 t = __fmul2_rn(f2(a), make_float2(b.v, b.v));
    return {t.x, fmaf(a.v, b.d, t.y)};
}

// acc + s a (s real) and acc + a b, fused
template <class T> __device__ __forceinline__ T madd(T s, T a, T acc) { return fma(s, a, acc); }
template <class T, int K> __device__ __forceinline__ Dual<T, K> madd(T s, Dual<T, K> a, Dual<T, K> acc) {
    return {fma(s, a.v, acc.v), fma(s, a.d, acc.d)};
}
__device__ __forceinline__ PDual madd(float s, PDual a, PDual acc) { return df(__ffma2_rn(make_float2(s, s), f2(a), f2(acc))); }
template <class T> __device__ __forceinline__ T mmadd(T a, T b, T acc) { return fma(a, b, acc); }
template <class T, int K> __device__ __forceinline__ Dual<T, K> mmadd(Dual<T, K> a, Dual<T, K> b, Dual<T, K> acc) {
    return {fma(a.v, b.v, acc.v), fma(a.d, b.v, fma(a.v, b.d, acc.d))};
}
__device__ __forceinline__ PDual mmadd(PDual a, PDual b, PDual acc) {
    const float2 t = __ffma2_rn(f2(a), make_float2(b.v, b.v), f2(acc));
    return {t.x, fmaf(a.v, b.d, t.y)};
}
template <class S> struct Base { typedef S type; };
template <class T, int K> struct Base<Dual<T, K>> { typedef T type; };

template <class T> __device__ __forceinline__ T value(T a) { return a; }
template <class T, int K> __device__ __forceinline__ T value(Dual<T, K> a) { return a.v; }
template <class T> __device__ __forceinline__ T tangent(T) { return T(0); }
template <class T, int K> __device__ __forceinline__ T tangent(Dual<T, K> a) { return a.d; }

template <class S> struct Zero { __device__ static S get() { return S(0); } };
template <class T, int K> struct Zero<Dual<T, K>> { __device__ static Dual<T, K> get() { return {T(0), T(0)}; } };
template <class S> __device__ __forceinline__ S zero() { return Zero<S>::get(); }

template <class S, class T> struct Make { __device__ static S get(T v, T) { return v; } };
template <class T, int K> struct Make<Dual<T, K>, T> { __device__ static Dual<T, K> get(T v, T d) { return {v, d}; } };
template <class S, class T> __device__ __forceinline__ S make(T v, T d) { return Make<S, T>::get(v, d); }

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
template <class T, int K> __device__ __forceinline__ Dual<T, K> rsq(Dual<T, K> x) {
    T r = rsq(x.v);
    return {r, T(-0.5) * r * r * r * x.d};
}
// float: the approximate reciprocal (at most 2 ulp; the mixed path's tolerance is orders above it)
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
template <class T, int K> __device__ __forceinline__ Dual<T, K> rcp(Dual<T, K> x) {
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
    int theta1;                           // theta == 1
    const int* skip;                      // non-null and nonzero: return at once (solver steps captured in graphs)
    double K0dt;                         // 4 / dt^2
    double CInu2;                        // C_I nu^2
    double irho;
    float rhof, muf, irhof, K0f, CI3f;   // float copies (CI3 = 3 C_I nu^2, the G:G factor)
    double CI3;
    double Cb;
    double g[3];
    const double* gpts;                   // g per surface point [n][3] in export order, or null: g
    const int32_t* sq_src;                // export position of every surface point (device order)
    int drop_visc;
    // batched meshes: element -> problem and the viscosity of every problem (null: the scalars)
    const uint16_t* eprob;
    const double* pmu;
    const float* pmuf;
    double CI;
    float CIf;
    // assembled-matrix block pattern (element-Jacobian assembly only)
    const int64_t* bptr;
    const int32_t* bidx;
    // deterministic scatter: element contributions go to slots (sv: volume, element precision;
    // ss: surface, float64) instead of atomic additions into out; null: atomics
    void* sv;
    double* ss;
    int64_t n_out_slots;                  // volume slots of the Out elements (Intercepted ones follow)
    int64_t n_dense_slots;                // surface slots of the dense bucket (sparse points follow)
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

// Node data, prepared once per call by node_prep for every independent node and by
// node_prep_hanging for every hanging node (from its parents' rows, u_e = M_e U), so the element
// kernels gather with plain loads and no float64 arithmetic:
//   us = theta u + (1-theta) u_prev (spatial state; theta = 1/2 is Crank-Nicolson), p,
//   at = (c0 u + c1 u_prev + c2 u_prev2)/dt = c0 (u - u_prev) + c2 (u_prev2 - u_prev)
//        (c0 + c1 + c2 = 0), the differences taken in float64 before rounding to T,
//   and for J v the tangents dus = theta v, dp = v_p, dat = c0 v.
// corner row in shared memory: node value row (us, p, at, 0) | tangent row (dus, dp, dat, 0) |
// force row (f, 0); 20 T, a multiple of 16 bytes so rows can be filled by 16-byte async copies
constexpr int CT = 8, CF = 16, CS = 20;


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

// 8 T to a 16-byte aligned global row with 16-byte stores
template <class T>
__device__ __forceinline__ void st8g(T* dst, const T v[8]) {
    if constexpr (sizeof(T) == 4) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
        for (int k = 0; k < 4; ++k) reinterpret_cast<double2*>(dst)[k] = make_double2(v[2 * k], v[2 * k + 1]);
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
    if (A.ndf) {   // (without a body force the force columns are never read)
        const char* f = reinterpret_cast<const char*>(A.ndf) + (size_t)id * 4 * sizeof(T);
        for (int k = 0; k < C8 / 2; ++k) cp16(reinterpret_cast<char*>(dst + CF) + 16 * k, f + 16 * k);
    }
}

// Conversions between float64 and float32 on the integer pipes (this GPU's float64 unit is narrow),
// written from the IEEE-754 binary64 / binary32 layouts: exponent bias 1023 / 127, fraction 52 / 23
// bits.  Normal numbers by re-biasing the exponent and shifting the fraction (rounding to nearest,
// ties to even, on the 29 dropped bits going down); zeros by their sign; subnormal, infinite and NaN
// operands take the hardware conversion.  Results equal the hardware's for every input.
__device__ __forceinline__ double f2d(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = b & 0x7F800000u;
    if ((b & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    if (e == 0u || e == 0x7F800000u) return (double)x;
    const uint32_t hi = (b & 0x80000000u) | (((b & 0x7FFFFFFFu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ float d2f(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t E = (hi >> 20) & 0x7FFu;
    if (E == 0u) return __uint_as_float(hi & 0x80000000u);   // zero or float64 subnormal: rounds to +-0
    if (E - 897u >= 254u) return (float)x;                   // below / above the float32 normal range
    uint32_t f = ((((hi & 0x7FFFFFFFu) << 3) | (lo >> 29)) - (896u << 23)) | (hi & 0x80000000u);
    const uint32_t rest = lo & 0x1FFFFFFFu, half = 0x10000000u;
    f += (rest > half || (rest == half && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
}
template <class T> __device__ __forceinline__ T to_t(double x);
template <> __device__ __forceinline__ float to_t<float>(double x) { return d2f(x); }
template <> __device__ __forceinline__ double to_t<double>(double x) { return x; }

// scatter one node's 4 values in the element precision: widened to float64 on the float64 unit,
// which the element kernels leave idle while their integer pipe is busy
__device__ __forceinline__ void scatter_t(const Args& A, int32_t id, const double r[4]) { scatter(A, id, r); }
__device__ __forceinline__ void scatter_t(const Args& A, int32_t id, const float r[4]) {
    const double rd[4] = {(double)r[0], (double)r[1], (double)r[2], (double)r[3]};
    scatter(A, id, rd);
}

// Node data, pass 1: independent nodes (float64 differences, then rounding to T)
template <class T, bool JV>
__global__ void __launch_bounds__(256) node_prep(Args A, T* __restrict__ ndv, T* __restrict__ ndt, T* __restrict__ ndf) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= A.n_nodes) return;
    if (A.skip && *A.skip) return;   // a captured solver step after its cycle ended
    double u[4], up[4], up2[4] = {0, 0, 0, 0};
    load4(A.U, n, u);
    load4(A.Up, n, up);
    if (A.c2 != 0.0) load4(A.Up2, n, up2);
    const T c0 = (T)A.c0, c2 = (T)A.c2, th = (T)A.theta;
    T v8[8];
    for (int k = 0; k < 3; ++k) {
        v8[k] = A.theta == 1.0 ? to_t<T>(u[k]) : to_t<T>(A.theta * u[k] + (1.0 - A.theta) * up[k]);
        T d1 = to_t<T>(u[k] - up[k]);
        T d2 = A.c2 != 0.0 ? to_t<T>(up2[k] - up[k]) : T(0);
        v8[4 + k] = c0 * d1 + c2 * d2;
    }
    v8[3] = to_t<T>(u[3]);
    v8[7] = T(0);
    st8g<T>(ndv + 8 * n, v8);
    if (ndf) {
        double f[4];
        load4(A.F, n, f);
        for (int k = 0; k < 3; ++k) ndf[4 * n + k] = to_t<T>(f[k]);
        ndf[4 * n + 3] = T(0);
    }
    if (JV) {
        double v[4];
        load4(A.V, n, v);
        T vt[4] = {to_t<T>(v[0]), to_t<T>(v[1]), to_t<T>(v[2]), to_t<T>(v[3])};
        T t8[8];
        for (int k = 0; k < 3; ++k) { t8[k] = th * vt[k]; t8[4 + k] = c0 * vt[k]; }
        t8[3] = vt[3];
        t8[7] = T(0);
        st8g<T>(ndt + 8 * n, t8);
    }
}

// Node data, pass 2: a hanging node's rows are the mean of its 2 (edge) or 4 (face) parents' rows
// (every entry is linear in the nodal vectors, so this is u_e = M_e U applied to the rows)
template <class T, bool JV>
__global__ void __launch_bounds__(256) node_prep_hanging(Args A, T* __restrict__ ndv, T* __restrict__ ndt,
                                                         T* __restrict__ ndf) {
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= A.n_hang) return;
    if (A.skip && *A.skip) return;   // a captured solver step after its cycle ended
    const int64_t n = A.n_nodes + h;
    const int32_t* hp = A.hpar + 4 * h;
    const int np = hp[2] >= 0 ? 4 : 2;
    const T w = np == 4 ? T(0.25) : T(0.5);
    T a[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)}, b[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    T c[4] = {T(0), T(0), T(0), T(0)};
    for (int p = 0; p < np; ++p) {
        T r[8];
        ld8<T>(ndv, hp[p], r);
        for (int k = 0; k < 8; ++k) a[k] += r[k];
        if (JV) {
            ld8<T>(ndt, hp[p], r);
            for (int k = 0; k < 8; ++k) b[k] += r[k];
        }
        if (ndf) {
            ld4<T>(ndf, hp[p], r);
            for (int k = 0; k < 4; ++k) c[k] += r[k];
        }
    }
    for (int k = 0; k < 8; ++k) { a[k] *= w; b[k] *= w; }
    st8g<T>(ndv + 8 * n, a);
    if (JV) st8g<T>(ndt + 8 * n, b);
    if (ndf)
        for (int k = 0; k < 4; ++k) ndf[4 * n + k] = w * c[k];
}

// both passes on stream s
template <class T, bool JV>
inline void launch_node_prep(const Args& A, T* ndv, T* ndt, T* ndf, cudaStream_t s) {
    if (A.n_nodes > 0) node_prep<T, JV><<<(unsigned)((A.n_nodes + 255) / 256), 256, 0, s>>>(A, ndv, ndt, ndf);
    if (A.n_hang > 0) node_prep_hanging<T, JV><<<(unsigned)((A.n_hang + 255) / 256), 256, 0, s>>>(A, ndv, ndt, ndf);
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
    S acc[3], rM[3];   // acc = d_t u + u . grad u - f (per unit density)
    for (int i = 0; i < 3; ++i) {
        const S conv = mmadd(F.Gu[i][2], F.us[2], mmadd(F.Gu[i][1], F.us[1], F.Gu[i][0] * F.us[0]));
        acc[i] = F.at[i] + conv - F.f[i];
        const S r = madd(P.rho, acc[i], F.gp[i]);
        rM[i] = A.drop_visc ? r : madd(-P.mu, F.H2[i], r);
    }
    // tau_M = (4/dt^2 + u.G u + C_I nu^2 G:G)^(-1/2), G = g^2 I;  tau_C = 1 / (tau_M tr G)
    S uu = mmadd(F.us[2], F.us[2], mmadd(F.us[1], F.us[1], F.us[0] * F.us[0]));
    S tauM = rsq(g2 * uu + (P.K0 + P.CI3 * (g2 * g2)));
    S tauC = rcp((T(3) * g2) * tauM);
    const S ntauM = T(-1) * tauM;
    S up[3];
    for (int i = 0; i < 3; ++i) up[i] = ntauM * rM[i];
    S pp = (-P.rho) * (tauC * divu);
    S q = g2 * mmadd(up[2], up[2], mmadd(up[1], up[1], up[0] * up[0]));
    bool bar = value(q) > tiny<T>();
    S taubar = bar ? rsq(q) : zero<S>();
    const S ppp = F.p + pp;
    for (int i = 0; i < 3; ++i) {
        const S Gup = mmadd(F.Gu[i][2], up[2], mmadd(F.Gu[i][1], up[1], F.Gu[i][0] * up[0]));
        out[i] = madd(P.rho, acc[i], Gup);
        const S wi = (-P.irho) * up[i];                 // -(u'_i / rho)
        const S ci = mmadd(taubar, Gup, wi);           // coefficient of u'_j in S_ij
        const S nup = T(-1) * up[i];
        for (int j = 0; j < 3; ++j) {
            // S_ij = 2 mu eps_ij - u'_i u_j - u'_i u'_j / rho + taubar (u' . grad u)_i u'_j  (- p - p' on i = j)
            S sij = mmadd(ci, up[j], mmadd(nup, F.us[j], P.mu * (F.Gu[i][j] + F.Gu[j][i])));
            if (i == j) sij = sij - ppp;
            out[3 + 3 * i + j] = sij;
        }
        out[13 + i] = wi;
    }
    out[12] = divu;
}


// ------------------------------------------------------------------------------------------
// Monomial (Hadamard) form of the trilinear interpolant on the reference cube [-1,1]^3.
// With s_{c,k} = +1 where bit k of corner c is set and -1 otherwise,
//   phi_c(xi) = prod_k (1 + s_{c,k} xi_k) / 2 = sum_S sigma_{c,S} m_S(xi),
//   sigma_{c,S} = prod_{k in S} s_{c,k},   m_S(xi) = prod_{k in S} xi_k / 8,
// S a subset of the three axes numbered by bits like the corners.  So a field is
//   u(xi) = sum_S a_S m_S(xi)  with  a_S = sum_c sigma_{c,S} u_c          (forward butterfly),
// d m_S / d xi_k = m_{S - k} for k in S, and a test-function sum over points is
//   sum_q [phi_c r_q + grad phi_c . s_q] = sum_S sigma_{c,S} M_S,
//   M_S = sum_q [m_S r_q + sum_{k in S} m_{S - k} s_{q,k}]                 (backward butterfly).
// Each butterfly is three stages of sums and differences, one per axis.
// ------------------------------------------------------------------------------------------
// four consecutive T in shared memory, 16-byte aligned (float4, or two double2)
template <class T>
__device__ __forceinline__ void st4s(T* p, T a, T b, T c, T d) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
        reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
    }
}
template <class T>
__device__ __forceinline__ void ld4s(const T* p, T o[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        const double2 v = reinterpret_cast<const double2*>(p)[0], w = reinterpret_cast<const double2*>(p)[1];
        o[0] = v.x; o[1] = v.y; o[2] = w.x; o[3] = w.y;
    }
}

template <class T>
__device__ __forceinline__ void monomials(const T xi[3], T m[8]) {
    const T e = T(0.125);
    m[0] = e;
    m[1] = e * xi[0];
    m[2] = e * xi[1];
    m[3] = m[1] * xi[1];
    m[4] = e * xi[2];
    m[5] = m[1] * xi[2];
    m[6] = m[2] * xi[2];
    m[7] = m[3] * xi[2];
}

// forward butterfly across the lanes (lane & 7) = corner c of an 8-lane group: corner value -> a_c.
// Each stage is one fused multiply-add by +-1 (exact: the same bits as the sum or difference).
template <class T>
__device__ __forceinline__ T hadamard_fwd(T x, int c) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T o = __shfl_xor_sync(0xffffffffu, x, 1 << k);
        x = fma(((c >> k) & 1) ? T(-1) : T(1), o, x);
    }
    return x;
}

// backward butterfly: lane holds M_S with S = (lane / LS) & 7; returns the sum for corner c = S's slot
template <int LS, class T>
__device__ __forceinline__ T hadamard_bwd(T x, int c) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T o = __shfl_xor_sync(0xffffffffu, x, LS << k);
        x = fma(((c >> k) & 1) ? T(1) : T(-1), o, x);
    }
    return x;
}

// Fields at a point from the monomial coefficients of the 8 corner rows (row S holds a_S of every
// column; layout as the corner rows: values | tangents at CT | force at CF; rows 16-byte aligned),
// monomials m of the point.  Rows are read whole and accumulated into every field they enter.
// IL: the rows hold (value, tangent) pairs interleaved in their first 16 entries (the packed float
// duals of the interior kernel: each 16-byte load yields two dual pairs in place).
template <class S, class T, bool IL = false>
__device__ __forceinline__ void interp_modal(const Args& A, const T m[8], const T* nd, int stride, T g,
                                             Fields<S, T>& F) {
    constexpr bool JV = !std::is_same<S, T>::value;
    static_assert(!IL || JV, "interleaved rows carry tangents");
    for (int i = 0; i < 3; ++i) {
        F.us[i] = zero<S>(); F.at[i] = zero<S>(); F.gp[i] = zero<S>(); F.f[i] = T(0);
        for (int j = 0; j < 3; ++j) F.Gu[i][j] = zero<S>();
    }
    F.p = zero<S>();
    S d01[2] = {zero<S>(), zero<S>()}, d02[2] = {zero<S>(), zero<S>()}, d12[2] = {zero<S>(), zero<S>()};
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const T* r = nd + t * stride;
        S a[7];
        if constexpr (IL) {
            T q[16];
            for (int k = 0; k < 16; k += 4) ld4s<T>(r + k, q + k);
#pragma unroll
            for (int j = 0; j < 7; ++j) a[j] = make<S, T>(q[2 * j], q[2 * j + 1]);
        } else {
            T v[8], d[8];
            ld4s<T>(r, v);
            ld4s<T>(r + 4, v + 4);
            if constexpr (JV) {
                ld4s<T>(r + CT, d);
                ld4s<T>(r + CT + 4, d + 4);
            }
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                if constexpr (JV) a[j] = make<S, T>(v[j], d[j]);
                else a[j] = v[j];
            }
        }
        const T mv = m[t];
        for (int i = 0; i < 3; ++i) {
            F.us[i] = madd(mv, a[i], F.us[i]);
            F.at[i] = madd(mv, a[4 + i], F.at[i]);
        }
        F.p = madd(mv, a[3], F.p);
        // d m_S / d xi_k = m_{S - k}: row t enters the k-derivative with monomial m[t ^ (1 << k)]
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (t & (1 << k)) {
                const T mk = m[t ^ (1 << k)];
                for (int i = 0; i < 3; ++i) F.Gu[i][k] = madd(mk, a[i], F.Gu[i][k]);
                F.gp[k] = madd(mk, a[3], F.gp[k]);
            }
        }
        if ((t & 3) == 3) { const T q = m[t ^ 3]; d01[0] = madd(q, a[0], d01[0]); d01[1] = madd(q, a[1], d01[1]); }
        if ((t & 5) == 5) { const T q = m[t ^ 5]; d02[0] = madd(q, a[0], d02[0]); d02[1] = madd(q, a[2], d02[1]); }
        if ((t & 6) == 6) { const T q = m[t ^ 6]; d12[0] = madd(q, a[1], d12[0]); d12[1] = madd(q, a[2], d12[1]); }
        if (A.ndf) {
            T f4[4];
            ld4s<T>(r + CF, f4);
            for (int i = 0; i < 3; ++i) F.f[i] = F.f[i] + mv * f4[i];
        }
    }
    // (grad div u)_i = sum_{j != i} d_i d_j u_j   (d01 holds u0, u1; d02 u0, u2; d12 u1, u2)
    F.H2[0] = d01[1] + d02[1];
    F.H2[1] = d01[0] + d12[1];
    F.H2[2] = d02[0] + d12[0];
    const T g2 = g * g;
    for (int i = 0; i < 3; ++i) {
        F.gp[i] = g * F.gp[i];
        F.H2[i] = g2 * F.H2[i];
        for (int j = 0; j < 3; ++j) F.Gu[i][j] = g * F.Gu[i][j];
    }
}

// forward butterfly down one column of an element's 8 corner rows (row stride CS), in place
template <class T>
__device__ __forceinline__ void column_to_monomial(T* col) {
    T x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = col[t * CS];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (!(t & (1 << k))) {
                const T lo = x[t], hi = x[t | (1 << k)];
                x[t] = lo + hi;
                x[t | (1 << k)] = hi - lo;
            }
#pragma unroll
    for (int t = 0; t < 8; ++t) col[t * CS] = x[t];
}

// forward butterfly of value column c and tangent column c (c < 7) of an element's 8 corner rows,
// then, after every lane of the warp has read its columns, the results stored interleaved as
// (value, tangent) pairs at entries 2c, 2c + 1 of each row (layout of interp_modal<IL = true>)
template <class T>
__device__ __forceinline__ void columns_to_monomial_interleaved(T* nd, int c) {
    T x[8], y[8];
    if (c < 7) {
#pragma unroll
        for (int t = 0; t < 8; ++t) { x[t] = nd[t * CS + c]; y[t] = nd[t * CS + CT + c]; }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if (!(t & (1 << k))) {
                    const T lo = x[t], hi = x[t | (1 << k)], lod = y[t], hid = y[t | (1 << k)];
                    x[t] = lo + hi;
                    x[t | (1 << k)] = hi - lo;
                    y[t] = lod + hid;
                    y[t | (1 << k)] = hid - lod;
                }
    }
    __syncwarp();
    if (c < 7) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if constexpr (sizeof(T) == 4) *reinterpret_cast<float2*>(nd + t * CS + 2 * c) = make_float2(x[t], y[t]);
            else *reinterpret_cast<double2*>(nd + t * CS + 2 * c) = make_double2(x[t], y[t]);
        }
    }
}

template <class S, class T, bool IL = false>
__device__ __forceinline__ void vms_point_modal(const Args& A, const Phys<T>& P, const T m[8], const T* nd,
                                                int stride, T g, S out[16]) {
    Fields<S, T> F;
    interp_modal<S, T, IL>(A, m, nd, stride, g, F);
    pointwise<S, T>(A, P, F, g, out);
}

// M[4 S + k] += monomial moments of one point's weighted coefficients c (F | S | G | H, the 16 of
// pointwise() times the quadrature weight, S and H in reference-gradient scaling), k = component.
// Scalar fused multiply-adds: the packed FP32x2 form needs its operand pairs assembled by register
// moves here, and measured 2.5 % slower in the interior kernel.
template <class T>
__device__ __forceinline__ void add_moments(const T m[8], const T c[16], T M[32]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T f = k < 3 ? c[k] : c[12];
        const T sx = k < 3 ? c[3 + 3 * k] : c[13];
        const T sy = k < 3 ? c[4 + 3 * k] : c[14];
        const T sz = k < 3 ? c[5 + 3 * k] : c[15];
        auto add = [&](int S, T s, T x) { M[4 * S + k] = fma(s, x, M[4 * S + k]); };
        add(0, m[0], f);
        add(1, m[1], f); add(1, m[0], sx);
        add(2, m[2], f); add(2, m[0], sy);
        add(3, m[3], f); add(3, m[2], sx); add(3, m[1], sy);
        add(4, m[4], f); add(4, m[0], sz);
        add(5, m[5], f); add(5, m[4], sx); add(5, m[1], sz);
        add(6, m[6], f); add(6, m[4], sy); add(6, m[2], sz);
        add(7, m[7], f); add(7, m[6], sx); add(7, m[5], sy); add(7, m[3], sz);
    }
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
    // float64 copies for the penalty: basis values, the jump u_s - g and (J v) its tangent theta v
    double phid[8], dd[3], ddt[3];
};

// g of Eq. (weakbc) at surface point q (device order)
__device__ __forceinline__ const double* point_g(const Args& A, int64_t q) {
    return A.gpts ? A.gpts + 3 * (int64_t)A.sq_src[q] : A.g;
}

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

// Q1 basis values in float64 at reference point xi (corner c = bits along x, y, z)
__device__ __forceinline__ void basis_values_d(const double* xi, double phi[8]) {
    double fm[3], fp[3];
    for (int k = 0; k < 3; ++k) { fm[k] = 0.5 * (1.0 - xi[k]); fp[k] = 0.5 * (1.0 + xi[k]); }
#pragma unroll
    for (int c = 0; c < 8; ++c) phi[c] = ((c & 1) ? fp[0] : fm[0]) * ((c & 2) ? fp[1] : fm[1]) * ((c & 4) ? fp[2] : fm[2]);
}

// u_s, p and grad u_s from the node data at surface point q (device order), and the velocity jump
// d = u_s - g.  DJ: the jump in float64 from the float64 nodal values at the point (dd; for J v its
// tangent theta v in ddt), as the force on the body needs; otherwise the jump from corner values
// u_s - g_body formed in float64 and rounded, plus g_body - g at the point (the float64 penalty is
// applied per element by nitsche_penalty).
template <class S, class T, bool JV, bool DJ = true>
__device__ __forceinline__ void nitsche_fields(const Args& A, int32_t e, int64_t q, const double* xr,
                                               const double* nr, NitschePoint<S, T>& P) {
    P.g = lvl_g<T>(A, A.lev[e]);
    {
        const Phys<T> Ph(A, prob_of(A, e));
        P.mu = Ph.mu;
        P.rho = Ph.rho;
    }
    T xi[3] = {(T)xr[0], (T)xr[1], (T)xr[2]};
    for (int k = 0; k < 3; ++k) P.nn[k] = (T)nr[k];
    basis<T>(xi, P.B);
    if (DJ) basis_values_d(xr, P.phid);
    const double* gq = point_g(A, q);
    P.p = zero<S>();
    double us_d[3] = {0.0, 0.0, 0.0};
    T dtan[3] = {T(0), T(0), T(0)}, dval[3] = {T(0), T(0), T(0)};
    for (int k = 0; k < 3; ++k) { P.us[k] = zero<S>(); P.ddt[k] = 0.0; for (int j = 0; j < 3; ++j) P.Gu[k][j] = zero<S>(); }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        P.ids[c] = A.conn[8 * (int64_t)e + c];
        T a8[8], t8[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        ld8<T>(A.ndv, P.ids[c], a8);
        if (JV) ld8<T>(A.ndt, P.ids[c], t8);
        double u4[4], up4[4];
        gather(A, A.U, P.ids[c], u4);
        if (!A.theta1) gather(A, A.Up, P.ids[c], up4);
        if (JV && DJ) {
            double v4[4];
            gather(A, A.V, P.ids[c], v4);
            for (int k = 0; k < 3; ++k) P.ddt[k] = fma(P.phid[c], A.theta * v4[k], P.ddt[k]);
        }
        const T ph = P.B.phi[c];
        for (int k = 0; k < 3; ++k) {
            S vu = make<S, T>(a8[k], t8[k]);
            const double usk = A.theta1 ? u4[k] : A.theta * u4[k] + (1.0 - A.theta) * up4[k];
            if (DJ) us_d[k] = fma(P.phid[c], usk, us_d[k]);
            else dval[k] = dval[k] + ph * (T)(usk - A.g[k]);
            dtan[k] = dtan[k] + ph * t8[k];
            P.us[k] = P.us[k] + ph * vu;
            for (int j = 0; j < 3; ++j) P.Gu[k][j] = P.Gu[k][j] + P.B.dphi[c][j] * vu;
        }
        P.p = P.p + ph * make<S, T>(a8[3], t8[3]);
    }
    for (int k = 0; k < 3; ++k) {
        if (DJ) {
            P.dd[k] = us_d[k] - gq[k];
            P.d[k] = make<S, T>((T)P.dd[k], dtan[k]);
        } else {
            P.d[k] = make<S, T>(dval[k] + (T)(A.g[k] - gq[k]), dtan[k]);
        }
    }
    finish_nitsche(A, P);
}

// the 4 rows of corner c (test functions phi_c e_i and q = phi_c), not yet times the weight;
// tau_TAN = tau_NOR: both penalty parts sum to tau_B (u - g).  PEN = false leaves the penalty out
// (the residual and J v kernels add it in float64).
template <class S, class T, bool PEN = true>
__device__ __forceinline__ void nitsche_rows(const Args& A, const NitschePoint<S, T>& P, int c, T tauB, S t[4]) {
    const T ph = P.B.phi[c];
    const T* nn = P.nn;
    const T gn = P.g * (P.B.dphi[c][0] * nn[0] + P.B.dphi[c][1] * nn[1] + P.B.dphi[c][2] * nn[2]);
    S gd = P.g * (P.B.dphi[c][0] * P.d[0] + P.B.dphi[c][1] * P.d[1] + P.B.dphi[c][2] * P.d[2]);
    for (int k = 0; k < 3; ++k) {
        S v = T(-1) * (ph * P.tr[k] + P.mu * (gn * P.d[k] + nn[k] * gd));
        if (PEN) v = v + (tauB * ph) * P.d[k];
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
    A.skip = nullptr;
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
    A.theta1 = A.theta == 1.0;
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
    A.gpts = ph.g_points;
    A.sq_src = m.d.sq_src;
    A.drop_visc = ph.drop_visc_strong;
    A.eprob = m.d.eprob;
    A.pmu = m.d.pmu;
    A.pmuf = m.d.pmuf;
    A.CI = ph.C_I;
    A.CIf = (float)ph.C_I;
    A.bptr = nullptr;
    A.bidx = nullptr;
    A.sv = m.deterministic ? m.d.sv : nullptr;
    A.ss = m.deterministic ? m.d.ss : nullptr;
    A.n_out_slots = (int64_t)m.out_list.size();
    A.n_dense_slots = m.n_sq_elem;
    return A;
}

// node workspace of precision T (float or double) of the mesh: value rows, tangent rows, forces
template <class T>
inline T* node_workspace(const Mesh& m, void* ws) {
    return ws ? (T*)ws : sizeof(T) == 4 ? (T*)(void*)m.d.nd_f : (T*)(void*)m.d.nd_d;
}

}  // namespace
}  // namespace imga
