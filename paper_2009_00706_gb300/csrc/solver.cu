// Newton iterations with right-preconditioned GMRES(m) on the device (appendix "Details of solver
// selection": a Newton line-search method with a Krylov solver; here GMRES replaces BiCGStab and
// the preconditioner is block-Jacobi over the nodal 4x4 blocks instead of additive Schwarz).
//
// All vectors and reductions are float64.  The Arnoldi basis is orthogonalised by classical
// Gram-Schmidt applied twice (CGS2): one multi-dot kernel h = V^T w over all previous basis vectors
// and one multi-axpy w -= V h per pass, so each pass reads the basis once.  The Hessenberg matrix
// and its Givens rotations (m x m, tiny) live on the host.  J v is imga_jvp's kernels in the
// requested precision; the true residual that decides convergence is always the float64 residual.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "imga_internal.h"

namespace imga {

namespace {

constexpr int kRedBlocks = 1024;   // blocks of the reduction kernels
constexpr int kDotGroup = 8;       // basis vectors per multi-dot pass

// partial[b][k] = sum over block b's slice of V[k0+k] . w   (k < nv)
template <int NV>
__global__ void __launch_bounds__(256) mdot_kernel(int64_t n, const double* __restrict__ V, int64_t ld, int k0, int nv,
                                                   const double* __restrict__ w, double* __restrict__ partial) {
    double acc[NV];
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (k < nv) acc[k] += V[(int64_t)(k0 + k) * ld + i] * wi;
    }
    __shared__ double red[NV][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < NV && (int)threadIdx.x < nv) {
        double v = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) v += red[threadIdx.x][j];
        partial[(int64_t)blockIdx.x * 64 + k0 + threadIdx.x] = v;
    }
}

// h[k] = sum_b partial[b][k], k < nk
__global__ void mdot_final(int nblocks, int nk, const double* __restrict__ partial, double* __restrict__ h) {
    const int k = blockIdx.x;
    if (k >= nk) return;
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[(int64_t)b * 64 + k];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += red[j];
        h[k] = s;
    }
}

// w = alpha w + beta * sum_{k<nk} h[k] V[k]
__global__ void __launch_bounds__(256) maxpy_kernel(int64_t n, const double* __restrict__ V, int64_t ld, int nk,
                                                    const double* __restrict__ h, double beta, double alpha,
                                                    double* __restrict__ w) {
    __shared__ double hs[64];
    if (threadIdx.x < nk) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nk; ++k) s += hs[k] * V[(int64_t)k * ld + i];
        w[i] = alpha * w[i] + beta * s;
    }
}

__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

// out = a x + b y + c z (out may be y)
__global__ void lincomb3_kernel(int64_t n, double a, const double* __restrict__ x, double b, const double* y, double c,
                                const double* __restrict__ z, double* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * x[i] + b * y[i] + c * z[i];
}

__global__ void scale_copy_kernel(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}

// ------------------------------------------------------------------------------------------
// Device-resident GMRES: the Arnoldi step reads the iteration index k and writes the Hessenberg
// column, the Givens rotations and the residual estimate in device memory, so one captured step
// graph serves every k.  A step that starts after its cycle ended (stop != 0) does nothing.
// ------------------------------------------------------------------------------------------
constexpr int kMaxM = 63;

struct GState {
    int k;          // Arnoldi index in the current cycle
    int its;        // iterations of this solve
    int stop;       // the cycle has ended: converged, breakdown, max iterations or k + 1 = m
    int kdone;      // Arnoldi vectors of the ended cycle
    int m, max_its;
    double target, hn, res;
    double H[(kMaxM + 1) * kMaxM];
    double cs[kMaxM], sn[kMaxM], g[kMaxM + 1], y[kMaxM];
    double h[64], h2[64];
};

__global__ void dg_start(GState* G, int m, int max_its, double target, double beta, int its) {
    G->k = 0;
    G->its = its;
    G->stop = 0;
    G->kdone = 0;
    G->m = m;
    G->max_its = max_its;
    G->target = target;
    G->res = beta;
    for (int i = 0; i <= m; ++i) G->g[i] = 0.0;
    G->g[0] = beta;
}

__global__ void dg_copy_basis(const GState* __restrict__ G, int64_t n, const double* __restrict__ V, double* __restrict__ y) {
    if (G->stop) return;
    const double* src = V + (int64_t)G->k * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = src[i];
}

// partial[b][j] = block b's share of V[j] . w for j <= k; blockIdx.y = group of 8 basis vectors
__global__ void __launch_bounds__(256) dg_mdot(const GState* __restrict__ G, int64_t n, const double* __restrict__ V,
                                               const double* __restrict__ w, double* __restrict__ partial) {
    if (G->stop) return;
    const int nk = G->k + 1, k0 = kDotGroup * blockIdx.y;
    if (k0 >= nk) return;
    const int nv = min(kDotGroup, nk - k0);
    double acc[kDotGroup];
    for (int j = 0; j < kDotGroup; ++j) acc[j] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int j = 0; j < kDotGroup; ++j)
            if (j < nv) acc[j] += V[(int64_t)(k0 + j) * n + i] * wi;
    }
    __shared__ double red[kDotGroup][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kDotGroup; ++j) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[j][wid] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nv) {
        double v = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[threadIdx.x][q];
        partial[(int64_t)blockIdx.x * 64 + k0 + threadIdx.x] = v;
    }
}

// out[j] = sum_b partial[b][j], j <= k (one block per j)
__global__ void dg_mdot_final(const GState* __restrict__ G, int nblocks, const double* __restrict__ partial,
                              double* __restrict__ out) {
    if (G->stop) return;
    const int j = blockIdx.x;
    if (j > G->k) return;
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[(int64_t)b * 64 + j];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        out[j] = t;
    }
}

// w -= sum_{j <= k} c[j] V[j]
__global__ void __launch_bounds__(256) dg_maxpy(const GState* __restrict__ G, int64_t n, const double* __restrict__ V,
                                                const double* __restrict__ c, double* __restrict__ w) {
    if (G->stop) return;
    const int nk = G->k + 1;
    __shared__ double cs[64];
    if ((int)threadIdx.x < nk) cs[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int j = 0; j < nk; ++j) t += cs[j] * V[(int64_t)j * n + i];
        w[i] -= t;
    }
}

// partial[b][0] = block b's share of w . w
__global__ void __launch_bounds__(256) dg_dot(const GState* __restrict__ G, int64_t n, const double* __restrict__ w,
                                              double* __restrict__ partial) {
    if (G->stop) return;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += w[i] * w[i];
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        partial[(int64_t)blockIdx.x * 64] = t;
    }
}

// hn = sqrt(sum_b partial[b][0])
__global__ void dg_norm_final(GState* G, int nblocks, const double* __restrict__ partial) {
    if (G->stop) return;
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[(int64_t)b * 64];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        G->hn = sqrt(fmax(t, 0.0));
    }
}

// V[k+1] = w / hn
__global__ void dg_normalize(const GState* __restrict__ G, int64_t n, const double* __restrict__ w, double* __restrict__ V) {
    if (G->stop) return;
    const double hn = G->hn;
    if (!(hn > 0.0)) return;
    double* dst = V + (int64_t)(G->k + 1) * n;
    const double inv = 1.0 / hn;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = inv * w[i];
}

// Hessenberg column k (CGS2 coefficients h + h2, norm hn), previous rotations, the new rotation,
// the residual estimate |g[k+1]|; ends the cycle or advances k.  One thread.
__global__ void dg_givens(GState* G) {
    if (G->stop) return;
    const int k = G->k, m = G->m;
    double* H = G->H;
    for (int i = 0; i <= k; ++i) H[i * m + k] = G->h[i] + G->h2[i];
    H[(k + 1) * m + k] = G->hn;
    for (int i = 0; i < k; ++i) {
        const double t = G->cs[i] * H[i * m + k] + G->sn[i] * H[(i + 1) * m + k];
        H[(i + 1) * m + k] = -G->sn[i] * H[i * m + k] + G->cs[i] * H[(i + 1) * m + k];
        H[i * m + k] = t;
    }
    const double a = H[k * m + k], b = H[(k + 1) * m + k];
    const double den = hypot(a, b);
    const double c = den > 0.0 ? a / den : 1.0, sn = den > 0.0 ? b / den : 0.0;
    G->cs[k] = c;
    G->sn[k] = sn;
    H[k * m + k] = c * a + sn * b;
    H[(k + 1) * m + k] = 0.0;
    G->g[k + 1] = -sn * G->g[k];
    G->g[k] = c * G->g[k];
    G->its += 1;
    G->res = fabs(G->g[k + 1]);
    if (G->res <= G->target || !(G->hn > 0.0) || G->its >= G->max_its || k + 1 >= m) {
        G->stop = 1;
        G->kdone = k + 1;
    } else {
        G->k = k + 1;
    }
}

// y = H^-1 g over the kdone columns of the ended cycle (back substitution).  One thread.
__global__ void dg_solve_y(GState* G) {
    const int kk = G->kdone, m = G->m;
    for (int i = kk - 1; i >= 0; --i) {
        double t = G->g[i];
        for (int j = i + 1; j < kk; ++j) t -= G->H[i * m + j] * G->y[j];
        G->y[i] = t / G->H[i * m + i];
    }
}

// w = sum_{j < kdone} y[j] V[j]
__global__ void __launch_bounds__(256) dg_combine(const GState* __restrict__ G, int64_t n, const double* __restrict__ V,
                                                  double* __restrict__ w) {
    const int kk = G->kdone;
    __shared__ double ys[64];
    if ((int)threadIdx.x < kk) ys[threadIdx.x] = G->y[threadIdx.x];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int j = 0; j < kk; ++j) t += ys[j] * V[(int64_t)j * n + i];
        w[i] = t;
    }
}

// ------------------------------------------------------------------------------------------
// A whole Newton solve replayed as one CUDA graph: WHILE conditional nodes (Newton iterations ->
// GMRES restart cycles -> Arnoldi steps, and the line search) whose conditions device kernels set.
// Every loop is bounded in its decision kernel (m steps per cycle, max_krylov iterations, 12
// line-search trials, max_newton iterations), so the graph always ends.
// ------------------------------------------------------------------------------------------
struct NState {
    double rn, target, lam, rt, bnorm, gtarget, beta;
    double krylov_rtol;
    int it, max_newton, line_search, trials, its, max_krylov, cycles, steps, nonfinite;
    double res_hist[33];
    int kpn[32];
    double krel[32];
};

// out = sqrt(sum_b partial[b][0]) (with sqrt = 1) or the sum
__global__ void ng_dot_final(int nblocks, const double* __restrict__ partial, double* __restrict__ out, int take_sqrt) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[(int64_t)b * 64];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        *out = take_sqrt ? sqrt(fmax(t, 0.0)) : t;
    }
}

// partial[b][0] = block b's share of x . x
__global__ void __launch_bounds__(256) ng_dot(int64_t n, const double* __restrict__ x, double* __restrict__ partial) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += x[i] * x[i];
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        partial[(int64_t)blockIdx.x * 64] = t;
    }
}

// y = x / *den
__global__ void ng_scale_inv(int64_t n, const double* __restrict__ x, const double* __restrict__ den, double* __restrict__ y) {
    const double inv = 1.0 / *den;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = inv * x[i];
}

// ut = u + *lam du
__global__ void ng_trial(int64_t n, const double* __restrict__ u, const double* __restrict__ du, const double* __restrict__ lam,
                         double* __restrict__ ut) {
    const double l = *lam;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        ut[i] = u[i] + l * du[i];
}

// linear solve starts: target, first residual, whether GMRES runs at all
__global__ void ng_gmres_init(NState* N, cudaGraphConditionalHandle h) {
    N->its = 0;
    N->cycles = 0;
    N->gtarget = N->krylov_rtol * N->bnorm;
    N->beta = N->bnorm;
    cudaGraphSetConditional(h, (N->beta > N->gtarget && N->beta != 0.0 && N->max_krylov > 0) ? 1u : 0u);
}

// a restart cycle starts from V[0] = r / beta
__global__ void ng_cycle_start(GState* G, NState* N, int m, cudaGraphConditionalHandle h) {
    G->k = 0;
    G->its = N->its;
    G->stop = 0;
    G->kdone = 0;
    G->m = m;
    G->max_its = N->max_krylov;
    G->target = N->gtarget;
    G->res = N->beta;
    for (int i = 0; i <= m; ++i) G->g[i] = 0.0;
    G->g[0] = N->beta;
    N->steps = 0;
    N->cycles += 1;
    cudaGraphSetConditional(h, 1u);
}

// after an Arnoldi step: continue while the cycle runs (at most m + 1 steps)
__global__ void ng_step_cond(GState* G, NState* N, cudaGraphConditionalHandle h) {
    N->steps += 1;
    if (N->steps > G->m + 1) G->stop = 1;
    cudaGraphSetConditional(h, G->stop ? 0u : 1u);
}

// after a cycle: the true residual norm beta of the iterate decides (as the host-driven solver)
__global__ void ng_gmres_decide(const GState* G, NState* N, cudaGraphConditionalHandle h) {
    N->its = G->its;
    bool cont = true;
    if (G->res <= N->gtarget || N->its >= N->max_krylov)
        cont = !(N->beta <= N->gtarget * 1.0000001 || N->its >= N->max_krylov);
    if (!(N->beta > 0.0) || N->cycles > N->max_krylov + 2) cont = false;
    cudaGraphSetConditional(h, cont ? 1u : 0u);
}

__global__ void ng_ls_init(NState* N, cudaGraphConditionalHandle h) {
    N->lam = 1.0;
    N->trials = 0;
    cudaGraphSetConditional(h, 1u);
}

// Armijo backtracking (c = 1e-4, halving, at most 12 trials)
__global__ void ng_ls_decide(NState* N, cudaGraphConditionalHandle h) {
    N->trials += 1;
    const bool ok = !N->line_search || (isfinite(N->rt) && N->rt <= (1.0 - 1e-4 * N->lam) * N->rn);
    if (ok || N->trials >= 12) {
        cudaGraphSetConditional(h, 0u);
    } else {
        N->lam *= 0.5;
        cudaGraphSetConditional(h, 1u);
    }
}

// the step is taken: record it and decide whether Newton goes on
__global__ void ng_newton_next(NState* N, cudaGraphConditionalHandle h) {
    N->rn = N->rt;
    if (N->it < 32) {
        N->kpn[N->it] = N->its;
        N->krel[N->it] = N->bnorm > 0.0 ? N->beta / N->bnorm : 0.0;
    }
    N->it += 1;
    if (N->it <= 32) N->res_hist[N->it] = N->rn;
    if (!isfinite(N->rn)) N->nonfinite = 1;
    const bool cont = isfinite(N->rn) && N->rn > N->target && N->it < N->max_newton && N->it < 32;
    cudaGraphSetConditional(h, cont ? 1u : 0u);
}

// During a capture on s: a conditional handle of the graph being captured (its value set by kernels).
int capture_handle(cudaStream_t s, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    if (cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess || !g) return 1;
    return cudaGraphConditionalHandleCreate(h, g, 0, 0) == cudaSuccess ? 0 : 1;
}

// During a capture on s: append a WHILE node on h after the captured work; later work depends on it.
int capture_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &ed, &nd) != cudaSuccess || !g) return 1;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, deps, ed, nd, &cp) != cudaSuccess) return 1;
    *body = cp.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) == cudaSuccess ? 0 : 1;
}

constexpr int kVecs = 14;          // work vectors of n doubles

struct Work {
    int m = 0;
    int64_t n = 0;
    double* V = nullptr;       // [(m+1)][n]
    double* vec = nullptr;     // kVecs vectors of n
    double* D = nullptr;       // [n_nodes][16]
    double* Dinv = nullptr;
    double* partial = nullptr; // [kRedBlocks][64]
    double* h = nullptr;       // [64]
    double* hh = nullptr;      // pinned host [128]: dot products in, coefficients out
    GState* G = nullptr;       // device-resident GMRES state
    NState* N = nullptr;       // device-resident Newton state (graph-replayed solve)
    double* gh = nullptr;      // pinned host [8]: the head of G read back once per chunk of steps
};

class Solver {
public:
    Solver(Mesh& m, const imga_physics& ph, const imga_solver_opts& o, cudaStream_t s, const double* up,
           const double* up2, const double* f)
        : M(m), P(ph), O(o), st(s), Up(up), Up2(up2), F(f) {
        n = 4 * m.n_nodes();
    }

    int alloc(std::string& err) {
        Work& w = W;
        const int mm = std::max(1, std::min(O.gmres_m, 63));
        if (M.solver_work && ((Work*)M.solver_work)->m >= mm && ((Work*)M.solver_work)->n == n) {
            W = *(Work*)M.solver_work;
            return 0;
        }
        free_work(M);
        w.m = mm;
        w.n = n;
        size_t bytes = (size_t)(mm + 1) * n * sizeof(double);
        if (cudaMalloc((void**)&w.V, bytes) != cudaSuccess || cudaMalloc((void**)&w.vec, kVecs * n * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&w.D, 4 * n * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&w.Dinv, 4 * n * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&w.partial, kRedBlocks * 64 * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&w.h, 64 * sizeof(double)) != cudaSuccess ||
            cudaMallocHost((void**)&w.hh, 128 * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&w.G, sizeof(GState)) != cudaSuccess || cudaMalloc((void**)&w.N, sizeof(NState)) != cudaSuccess ||
            cudaMallocHost((void**)&w.gh, 8 * sizeof(double)) != cudaSuccess) {
            err = "solver workspace allocation failed";
            cudaGetLastError();
            return 1;
        }
        M.solver_work = new Work(w);
        return 0;
    }

    static void free_work(Mesh& m) {
        if (!m.solver_work) return;
        Work* w = (Work*)m.solver_work;
        cudaFree(w->V); cudaFree(w->vec); cudaFree(w->D); cudaFree(w->Dinv); cudaFree(w->partial); cudaFree(w->h);
        cudaFreeHost(w->hh);
        cudaFree(w->G);
        cudaFree(w->N);
        cudaFreeHost(w->gh);
        delete w;
        m.solver_work = nullptr;
    }

    double* vec(int k) { return W.vec + (int64_t)k * n; }
    double* basis(int k) { return W.V + (int64_t)k * n; }

    // h[0..nk) = V[0..nk)^T w, copied to the host
    void mdot(const double* V, int nk, const double* w, double* host) {
        const int grid = (int)std::min<int64_t>(kRedBlocks, (n + 255) / 256);
        for (int k0 = 0; k0 < nk; k0 += kDotGroup)
            mdot_kernel<kDotGroup><<<grid, 256, 0, st>>>(n, V, n, k0, std::min(kDotGroup, nk - k0), w, W.partial);
        mdot_final<<<nk, 256, 0, st>>>(grid, nk, W.partial, W.h);
        cudaMemcpyAsync(W.hh, W.h, nk * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        std::memcpy(host, W.hh, nk * sizeof(double));
    }
    double norm(const double* x) {
        double v;
        mdot(x, 1, x, &v);
        return std::sqrt(std::max(v, 0.0));
    }
    void maxpy(const double* V, int nk, const double* hhost, double beta, double alpha, double* w) {
        // upload half of the pinned buffer (the other half receives the dot products)
        std::memcpy(W.hh + 64, hhost, nk * sizeof(double));
        cudaMemcpyAsync(W.h, W.hh + 64, nk * sizeof(double), cudaMemcpyHostToDevice, st);
        const int grid = (int)std::min<int64_t>(4 * M.n_sm, (n + 255) / 256);
        maxpy_kernel<<<grid, 256, 0, st>>>(n, V, n, nk, W.h, beta, alpha, w);
    }
    void axpby(double a, const double* x, double b, double* y) {
        axpby_kernel<<<(unsigned)std::min<int64_t>(4 * M.n_sm, (n + 255) / 256), 256, 0, st>>>(n, a, x, b, y);
    }
    void scale_copy(double a, const double* x, double* y) {
        scale_copy_kernel<<<(unsigned)std::min<int64_t>(4 * M.n_sm, (n + 255) / 256), 256, 0, st>>>(n, a, x, y);
    }

    int residual(const double* u, double* R) {
        return vms_apply(M, u, Up, Up2, F, P, 0, nullptr, R, st);
    }
    int jv(const double* u, const double* v, double* out) {
        return vms_apply(M, u, Up, Up2, F, P, O.precision, v, out, st);
    }
    // the true linear residual of a restart in float64: with float32 element arithmetic J v is linear
    // only to rounding (~1e-7 relative), so the restarts form b - J x with the float64 J v and every
    // cycle refines the float64 solution (iterative refinement); the Arnoldi steps keep O.precision
    int jv_true(const double* u, const double* v, double* out) {
        return vms_apply(M, u, Up, Up2, F, P, 0, v, out, st);
    }
    int pmode = 0;   // preconditioner in use for the current linear solve (block-Jacobi fallback)
    static bool learned_mode(int p) { return p == 2 || p == 3; }
    void precond(const double* x, double* y) {
        if (pmode == 4) { multilevel_apply(M, x, y, st); return; }
        if (pmode >= 1) block_jacobi_apply(M, W.Dinv, x, y, st);
        else cudaMemcpyAsync(y, x, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (learned_mode(pmode))
            precond_correction(M, P, L.elems, L.n, L.C, L.scale, (float)O.learned_omega, x, L.zc, y, st);
    }
    void lincomb3(double a, const double* x, double b, const double* y, double c, const double* z, double* out) {
        lincomb3_kernel<<<(unsigned)std::min<int64_t>(4 * M.n_sm, (n + 255) / 256), 256, 0, st>>>(n, a, x, b, y, c, z, out);
    }
    double dot(const double* x, const double* y) {
        double v;
        mdot(x, 1, y, &v);
        return v;
    }

    // BiCGStab (van der Vorst) with right preconditioning on the assembled Jacobian A: x = A^-1 b to
    // ||b - A x|| <= rtol ||b|| (appendix "Details of solver selection"); x starts at 0
    int bicgstab(const double* A, const double* b, double* x, double rtol, int max_its, int* its_out, double* res_out) {
        double *r = vec(4), *rh = vec(5), *pv = vec(6), *v = vec(8), *sv = vec(9), *ph = vec(10), *sh = vec(11),
               *t = vec(12);
        std::string err;
        auto Amul = [&](const double* in, double* out) { return bsr_spmv(M, A, in, out, st, err); };
        cudaMemsetAsync(x, 0, n * sizeof(double), st);
        cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(rh, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        cudaMemsetAsync(v, 0, n * sizeof(double), st);
        cudaMemsetAsync(pv, 0, n * sizeof(double), st);
        const double bn = norm(b), tol = rtol * bn;
        double res = bn, rho_old = 1.0, alpha = 1.0, omega = 1.0;
        int it = 0;
        if (res > tol) {
            for (it = 1; it <= max_its; ++it) {
                const double rho = dot(rh, r);
                if (rho == 0.0) break;
                const double beta = (rho / rho_old) * (alpha / omega);
                lincomb3(1.0, r, beta, pv, -beta * omega, v, pv);
                precond(pv, ph);
                if (Amul(ph, v)) return 1;
                alpha = rho / dot(rh, v);
                axpby(1.0, r, 0.0, sv);
                axpby(-alpha, v, 1.0, sv);
                const double sn = norm(sv);
                if (sn <= tol) { axpby(alpha, ph, 1.0, x); res = sn; break; }
                precond(sv, sh);
                if (Amul(sh, t)) return 1;
                const double tt = dot(t, t);
                omega = tt > 0.0 ? dot(t, sv) / tt : 0.0;
                lincomb3(alpha, ph, 1.0, x, omega, sh, x);
                lincomb3(1.0, sv, 0.0, sv, -omega, t, r);
                res = norm(r);
                if (res <= tol || omega == 0.0) break;
                rho_old = rho;
            }
        }
        *its_out = std::min(it, max_its);
        *res_out = res;
        return 0;
    }

    // learned correction: network inputs of every active element, one inference per Newton iteration
    struct Learned {
        int64_t n = 0;
        int ldx = 0;
        int32_t* elems = nullptr;
        float *X = nullptr, *C = nullptr, *scale = nullptr;
        double *K = nullptr, *zc = nullptr;
    } L;

    int learned_alloc(std::string& err) {
        std::vector<int32_t> act(M.out_list);
        act.insert(act.end(), M.cut_list.begin(), M.cut_list.end());
        L.n = (int64_t)act.size();
        L.ldx = O.precond == 2 ? mlp_nin_pad((const Mlp*)O.learned) : 1040;
        if (L.ldx < 1027) { err = "learned preconditioner: the network must take 1027 inputs"; return 1; }
        bool ok = cudaMalloc((void**)&L.elems, std::max<int64_t>(1, L.n) * 4) == cudaSuccess &&
                  cudaMalloc((void**)&L.X, std::max<int64_t>(1, L.n) * L.ldx * 4) == cudaSuccess &&
                  cudaMalloc((void**)&L.C, std::max<int64_t>(1, L.n) * 1024 * 4) == cudaSuccess &&
                  cudaMalloc((void**)&L.scale, std::max<int64_t>(1, L.n) * 4) == cudaSuccess &&
                  cudaMalloc((void**)&L.K, std::max<int64_t>(1, L.n) * 1024 * 8) == cudaSuccess &&
                  cudaMalloc((void**)&L.zc, n * 8) == cudaSuccess;
        if (!ok) { err = "learned preconditioner allocation failed"; cudaGetLastError(); return 1; }
        cudaMemcpyAsync(L.elems, act.data(), L.n * 4, cudaMemcpyHostToDevice, st);
        return 0;
    }
    void learned_free() {
        cudaFree(L.elems); cudaFree(L.X); cudaFree(L.C); cudaFree(L.scale); cudaFree(L.K); cudaFree(L.zc);
        L = Learned();
    }
    int learned_setup(const double* u) {
        // precond 2: the network's correction; precond 3: the exact element-block correction it is trained on
        float* T = O.precond == 3 ? L.C : nullptr;
        if (precond_dataset(M, u, Up, Up2, F, P, O.precision, L.elems, L.n, L.ldx, L.X, T, L.scale, L.K, st)) return 1;
        if (O.precond == 3) return 0;
        return mlp_forward((Mlp*)O.learned, L.X, L.ldx, L.n, L.C, st);
    }

    ~Solver() {
        for (auto& g : step_graph)
            if (g) cudaGraphExecDestroy(g);
        if (cap) cudaStreamDestroy(cap);
    }

    // ---- device-resident GMRES: one Arnoldi step per replay of a captured graph ----
    static constexpr int kChunk = 8;   // steps launched between two reads of the stop flag
    cudaGraphExec_t step_graph[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t cap = nullptr;

    double* dev_field(size_t off) { return reinterpret_cast<double*>(reinterpret_cast<char*>(W.G) + off); }

    // precondition V[k], J v, CGS2 against V[0..k], normalise into V[k+1], Givens update
    int step_launches(const double* u) {
        GState* G = W.G;
        double* vk = vec(4);
        double* z = vec(5);
        double* w = vec(6);
        const int grid = (int)std::min<int64_t>(kRedBlocks, (n + 255) / 256);
        const int grid2 = (int)std::min<int64_t>(4 * M.n_sm, (n + 255) / 256);
        dg_copy_basis<<<grid2, 256, 0, st>>>(G, n, W.V, vk);
        precond(vk, z);
        if (vms_apply_skip(M, u, Up, Up2, F, P, O.precision, z, w, st, &G->stop)) return 1;
        for (int pass = 0; pass < 2; ++pass) {
            double* c = dev_field(pass ? offsetof(GState, h2) : offsetof(GState, h));
            dg_mdot<<<dim3(grid, (kMaxM + 1 + kDotGroup - 1) / kDotGroup), 256, 0, st>>>(G, n, W.V, w, W.partial);
            dg_mdot_final<<<64, 256, 0, st>>>(G, grid, W.partial, c);
            dg_maxpy<<<grid2, 256, 0, st>>>(G, n, W.V, c, w);
        }
        dg_dot<<<grid, 256, 0, st>>>(G, n, w, W.partial);
        dg_norm_final<<<1, 256, 0, st>>>(G, grid, W.partial);
        dg_normalize<<<grid2, 256, 0, st>>>(G, n, w, W.V);
        dg_givens<<<1, 1, 0, st>>>(G);
        return cudaGetLastError() == cudaSuccess ? 0 : 1;
    }

    int capture_step(const double* u) {
        if (step_graph[pmode]) return 0;
        if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return 1;
        vms_prepare();
        cudaStream_t keep = st;
        st = cap;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { st = keep; return 1; }
        const int rc = step_launches(u);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cap, &g);
        st = keep;
        if (rc || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return 1;
        }
        const cudaError_t ei = cudaGraphInstantiate(&step_graph[pmode], g, 0);
        cudaGraphDestroy(g);
        return ei == cudaSuccess ? 0 : 1;
    }

    struct Head { int stop, its; double res; };
    Head read_head() {
        cudaMemcpyAsync(W.gh, W.G, offsetof(GState, H), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        GState h;
        std::memcpy(&h, W.gh, offsetof(GState, H));
        return {h.stop, h.its, h.res};
    }

    // the same solve as gmres(), with the Arnoldi steps replayed as a graph and no host round trip
    // inside a chunk of steps
    int gmres_dev(const double* u, const double* b, double* x, double rtol, int max_its, int* its_out, double* res_out) {
        const int m = std::min(W.m, kMaxM);
        double* r = vec(4);
        double* z = vec(5);
        double* w = vec(6);
        cudaMemsetAsync(x, 0, n * sizeof(double), st);
        const double bnorm = norm(b);
        const double target = rtol * bnorm;
        int its = 0;
        double res = bnorm, beta = bnorm;
        if (capture_step(u)) return 1;
        cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        const int grid2 = (int)std::min<int64_t>(4 * M.n_sm, (n + 255) / 256);
        while (true) {
            res = beta;
            if (beta <= target || its >= max_its || beta == 0.0) break;
            scale_copy(1.0 / beta, r, basis(0));
            dg_start<<<1, 1, 0, st>>>(W.G, m, max_its, target, beta, its);
            Head h{0, its, beta};
            for (int chunk = 0; !h.stop; ++chunk) {
                if (chunk > m) return 1;   // every step advances k or ends the cycle
                for (int c = 0; c < kChunk; ++c)
                    if (cudaGraphLaunch(step_graph[pmode], st) != cudaSuccess) return 1;
                h = read_head();
            }
            its = h.its;
            dg_solve_y<<<1, 1, 0, st>>>(W.G);
            dg_combine<<<grid2, 256, 0, st>>>(W.G, n, W.V, w);
            precond(w, z);
            axpby(1.0, z, 1.0, x);
            // residual of the iterate: the true one decides at the end, the restart starts from it
            if (jv_true(u, x, w)) return 1;
            cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
            axpby(-1.0, w, 1.0, r);
            const double beta0 = beta;
            beta = norm(r);
            if (h.res <= target || its >= max_its) {
                res = beta;
                if (beta <= target * 1.0000001 || its >= max_its) break;
            }
            if (stalled(beta, beta0)) { res = beta; break; }
        }
        *its_out = its;
        *res_out = res;
        return 0;
    }

    // with a learned correction in use, a restart cycle that does not halve the residual ends the
    // solve early: the caller then redoes it with block-Jacobi
    bool stalled(double r, double r_cycle_start) const { return learned_mode(pmode) && r > 0.5 * r_cycle_start; }

    int solve(const double* u, const double* b, double* x, double rtol, int max_its, int* its_out, double* res_out) {
        if (M.use_graphs && !M.profiling) return gmres_dev(u, b, x, rtol, max_its, its_out, res_out);
        return gmres(u, b, x, rtol, max_its, its_out, res_out);
    }

    // solve J(u) x = b to ||b - J x|| <= rtol ||b|| (or max_its); x starts at 0
    int gmres(const double* u, const double* b, double* x, double rtol, int max_its, int* its_out, double* res_out) {
        const int m = W.m;
        double* r = vec(4);
        double* z = vec(5);
        double* w = vec(6);
        cudaMemsetAsync(x, 0, n * sizeof(double), st);
        const double bnorm = norm(b);
        const double target = rtol * bnorm;
        int its = 0;
        double res = bnorm;
        std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m), h(m + 1), h2(m + 1);
        cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        while (true) {
            const double beta = its == 0 ? bnorm : norm(r);
            res = beta;
            if (beta <= target || its >= max_its || beta == 0.0) break;
            scale_copy(1.0 / beta, r, basis(0));
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int k = 0;
            for (; k < m && its < max_its; ++k) {
                precond(basis(k), z);
                if (jv(u, z, w)) return 1;
                // CGS2
                mdot(W.V, k + 1, w, h.data());
                maxpy(W.V, k + 1, h.data(), -1.0, 1.0, w);
                mdot(W.V, k + 1, w, h2.data());
                maxpy(W.V, k + 1, h2.data(), -1.0, 1.0, w);
                for (int i = 0; i <= k; ++i) H[i * m + k] = h[i] + h2[i];
                const double hn = norm(w);
                H[(k + 1) * m + k] = hn;
                if (hn > 0.0) scale_copy(1.0 / hn, w, basis(k + 1));
                for (int i = 0; i < k; ++i) {
                    const double t = cs[i] * H[i * m + k] + sn[i] * H[(i + 1) * m + k];
                    H[(i + 1) * m + k] = -sn[i] * H[i * m + k] + cs[i] * H[(i + 1) * m + k];
                    H[i * m + k] = t;
                }
                const double den = std::hypot(H[k * m + k], H[(k + 1) * m + k]);
                cs[k] = den > 0.0 ? H[k * m + k] / den : 1.0;
                sn[k] = den > 0.0 ? H[(k + 1) * m + k] / den : 0.0;
                H[k * m + k] = cs[k] * H[k * m + k] + sn[k] * H[(k + 1) * m + k];
                H[(k + 1) * m + k] = 0.0;
                g[k + 1] = -sn[k] * g[k];
                g[k] = cs[k] * g[k];
                ++its;
                res = std::fabs(g[k + 1]);
                if (res <= target || hn == 0.0) { ++k; break; }
            }
            for (int i = k - 1; i >= 0; --i) {
                double s = g[i];
                for (int j = i + 1; j < k; ++j) s -= H[i * m + j] * y[j];
                y[i] = s / H[i * m + i];
            }
            // x += M^{-1} (V y)
            cudaMemsetAsync(w, 0, n * sizeof(double), st);
            maxpy(W.V, k, y.data(), 1.0, 0.0, w);
            precond(w, z);
            axpby(1.0, z, 1.0, x);
            if (res <= target || its >= max_its) {
                // true residual of the returned solution
                if (jv_true(u, x, w)) return 1;
                cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
                axpby(-1.0, w, 1.0, r);
                res = norm(r);
                if (res <= target * 1.0000001 || its >= max_its) break;
                continue;
            }
            if (jv_true(u, x, w)) return 1;
            cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
            axpby(-1.0, w, 1.0, r);
            const double rn = norm(r);
            if (stalled(rn, beta)) { res = rn; break; }
        }
        *its_out = its;
        *res_out = res;
        return 0;
    }

    // preconditioner setup at the iterate u (block-Jacobi or multilevel), launches only (capturable)
    int precond_setup(const double* u, std::string& err) {
        if (O.precond >= 1 && O.precond <= 3 && block_jacobi_setup(M, u, Up, Up2, F, P, O.precision, W.D, W.Dinv, st)) {
            err = "block-Jacobi setup failed";
            return 1;
        }
        if (O.precond == 4 && multilevel_setup(M, u, Up, Up2, F, P, O.precision, O.ml_sweeps > 0 ? O.ml_sweeps : 1,
                                               O.ml_omega > 0.0 ? O.ml_omega : 0.5, st, err))
            return 1;
        return 0;
    }

    // *out = ||x|| computed on the device (launches only)
    void norm_dev(const double* x, double* out) {
        const int grid = (int)std::min<int64_t>(kRedBlocks, (n + 255) / 256);
        ng_dot<<<grid, 256, 0, st>>>(n, x, W.partial);
        ng_dot_final<<<1, 256, 0, st>>>(grid, W.partial, out, 1);
    }

    double* nfield(size_t off) { return reinterpret_cast<double*>(reinterpret_cast<char*>(W.N) + off); }

    // The Newton solve of newton() as one graph launch: Newton iterations, GMRES restart cycles, Arnoldi
    // steps and line-search trials are WHILE nodes whose conditions device kernels set, so the host
    // waits once.  Returns -1 (nothing done) when the graph cannot be built; newton() then drives it.
    int newton_graph(double* u, imga_solver_stats* S, std::string& err) {
        auto t0 = std::chrono::steady_clock::now();
        double *R = vec(0), *b = vec(1), *du = vec(2), *ut = vec(3), *r = vec(4), *z = vec(5), *w = vec(6), *Rt = vec(7);
        if (residual(u, R)) { err = "residual launch failed"; return 1; }
        const double r0 = norm(R);
        if (!std::isfinite(r0)) { err = "NaN/Inf in the initial residual"; return 2; }
        S->res_norm[0] = r0;
        const double target = std::max(O.rtol * r0, O.atol);
        if (r0 <= target || O.max_newton <= 0) {
            S->newton_its = 0;
            S->converged = r0 <= target ? 1 : 0;
            S->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            return 0;
        }
        // set-up work that allocates or sets launch attributes runs once before the capture
        if (precond_setup(u, err)) return 1;
        vms_prepare();
        pmode = O.precond;
        NState h;
        std::memset(&h, 0, sizeof(h));
        h.rn = r0;
        h.target = target;
        h.krylov_rtol = O.krylov_rtol;
        h.max_newton = O.max_newton;
        h.line_search = O.line_search;
        h.max_krylov = O.max_krylov;
        h.res_hist[0] = r0;
        if (cudaMemcpyAsync(W.N, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
            return -1;
        const int m = std::min(W.m, kMaxM);
        NState* N = W.N;
        GState* G = W.G;
        cudaStream_t keep = st, c[3] = {nullptr, nullptr, nullptr};
        cudaGraph_t top = nullptr;
        cudaGraphExec_t exec = nullptr;
        bool ok = true;
        for (int i = 0; i < 3 && ok; ++i) ok = cudaStreamCreateWithFlags(&c[i], cudaStreamNonBlocking) == cudaSuccess;
        cudaGraphConditionalHandle hN, hG, hA, hL;
        cudaGraph_t bN = nullptr, bC = nullptr, bS = nullptr, bL = nullptr;
        auto end = [&](cudaStream_t cs, cudaGraph_t* g) {
            cudaGraph_t out = *g;
            const bool e = cudaStreamEndCapture(cs, &out) == cudaSuccess;
            ok = ok && e;
        };
        ok = ok && cudaGraphCreate(&top, 0) == cudaSuccess &&
             cudaGraphConditionalHandleCreate(&hN, top, 1, cudaGraphCondAssignDefault) == cudaSuccess;
        if (ok) {   // top: WHILE (Newton goes on) { one Newton iteration }
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = hN;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            ok = cudaGraphAddNode(&node, top, nullptr, nullptr, 0, &cp) == cudaSuccess;
            if (ok) bN = cp.conditional.phGraph_out[0];
        }
        if (ok) ok = cudaStreamBeginCaptureToGraph(c[0], bN, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            st = c[0];
            std::string e2;
            ok = precond_setup(u, e2) == 0;
            scale_copy(-1.0, R, b);
            cudaMemsetAsync(du, 0, n * sizeof(double), st);
            cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
            norm_dev(b, nfield(offsetof(NState, bnorm)));
            ok = ok && capture_handle(st, &hG) == 0;
            if (ok) ng_gmres_init<<<1, 1, 0, st>>>(N, hG);
            ok = ok && capture_while(st, hG, &bC) == 0;
            // GMRES restart cycle
            if (ok) ok = cudaStreamBeginCaptureToGraph(c[1], bC, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                st = c[1];
                ng_scale_inv<<<(unsigned)std::min<int64_t>(4 * M.n_sm, (n + 255) / 256), 256, 0, st>>>(
                    n, r, nfield(offsetof(NState, beta)), basis(0));
                ok = capture_handle(st, &hA) == 0;
                if (ok) ng_cycle_start<<<1, 1, 0, st>>>(G, N, m, hA);
                ok = ok && capture_while(st, hA, &bS) == 0;
                if (ok) ok = cudaStreamBeginCaptureToGraph(c[2], bS, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {   // one Arnoldi step
                    st = c[2];
                    ok = step_launches(u) == 0;
                    ng_step_cond<<<1, 1, 0, st>>>(G, N, hA);
                    end(c[2], &bS);
                }
                st = c[1];
                const int grid2 = (int)std::min<int64_t>(4 * M.n_sm, (n + 255) / 256);
                dg_solve_y<<<1, 1, 0, st>>>(G);
                dg_combine<<<grid2, 256, 0, st>>>(G, n, W.V, w);
                precond(w, z);
                axpby(1.0, z, 1.0, du);
                ok = ok && vms_apply_skip(M, u, Up, Up2, F, P, 0, du, w, st, nullptr) == 0;   // float64: jv_true
                cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
                axpby(-1.0, w, 1.0, r);
                norm_dev(r, nfield(offsetof(NState, beta)));
                ng_gmres_decide<<<1, 1, 0, st>>>(G, N, hG);
                end(c[1], &bC);
            }
            // line search
            st = c[0];
            ok = ok && capture_handle(st, &hL) == 0;
            if (ok) ng_ls_init<<<1, 1, 0, st>>>(N, hL);
            ok = ok && capture_while(st, hL, &bL) == 0;
            if (ok) ok = cudaStreamBeginCaptureToGraph(c[1], bL, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                st = c[1];
                ng_trial<<<(unsigned)std::min<int64_t>(4 * M.n_sm, (n + 255) / 256), 256, 0, st>>>(
                    n, u, du, nfield(offsetof(NState, lam)), ut);
                ok = vms_apply_skip(M, ut, Up, Up2, F, P, 0, nullptr, Rt, st, nullptr) == 0;
                norm_dev(Rt, nfield(offsetof(NState, rt)));
                ng_ls_decide<<<1, 1, 0, st>>>(N, hL);
                end(c[1], &bL);
            }
            st = c[0];
            cudaMemcpyAsync(u, ut, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(R, Rt, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
            ng_newton_next<<<1, 1, 0, st>>>(N, hN);
            end(c[0], &bN);
        }
        st = keep;
        ok = ok && cudaGraphInstantiate(&exec, top, 0) == cudaSuccess;
        int rc = -1;
        if (ok) {
            rc = 0;
            if (cudaGraphLaunch(exec, st) != cudaSuccess || cudaMemcpyAsync(&h, W.N, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                err = "graph-replayed Newton failed";
                rc = 1;
            }
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (top) cudaGraphDestroy(top);
        for (cudaStream_t cs : c)
            if (cs) cudaStreamDestroy(cs);
        if (rc != 0) {
            cudaGetLastError();
            return rc;
        }
        S->newton_its = h.it;
        for (int i = 0; i < std::min(h.it, 32); ++i) {
            S->krylov_per_newton[i] = h.kpn[i];
            S->krylov_rel[i] = h.krel[i];
            S->krylov_its += h.kpn[i];
            S->res_norm[i + 1] = h.res_hist[i + 1];
        }
        if (h.nonfinite) { err = "NaN/Inf in the residual"; return 2; }
        S->converged = h.rn <= target ? 1 : 0;
        S->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return 0;
    }

    int newton(double* u, imga_solver_stats* S, std::string& err) {
        if (M.use_graphs && !M.profiling && O.linear_solver == 0 && !learned_mode(O.precond)) {
            const int rc = newton_graph(u, S, err);
            if (rc >= 0) return rc;
            std::memset(S, 0, sizeof(*S));   // the graph could not be built: drive the same solve from the host
        }
        auto t0 = std::chrono::steady_clock::now();
        double* R = vec(0);
        double* b = vec(1);
        double* du = vec(2);
        double* ut = vec(3);
        double* Rt = vec(7);
        if (residual(u, R)) { err = "residual launch failed"; return 1; }
        double r0 = norm(R), rn = r0;
        if (!std::isfinite(r0)) { err = "NaN/Inf in the initial residual"; return 2; }
        S->res_norm[0] = r0;
        const double target = std::max(O.rtol * r0, O.atol);
        int it = 0;
        for (; it < O.max_newton && it < 32; ++it) {
            if (rn <= target) break;
            if (O.precond >= 1 && O.precond <= 3 &&
                block_jacobi_setup(M, u, Up, Up2, F, P, O.precision, W.D, W.Dinv, st)) {
                err = "block-Jacobi setup failed";
                return 1;
            }
            if (learned_mode(O.precond) && learned_setup(u)) { err = "learned preconditioner setup failed"; return 1; }
            const double* Aasm = nullptr;
            if (O.precond == 4) {
                if (multilevel_setup(M, u, Up, Up2, F, P, O.precision, O.ml_sweeps > 0 ? O.ml_sweeps : 1,
                                     O.ml_omega > 0.0 ? O.ml_omega : 0.5, st, err))
                    return 1;
                Aasm = multilevel_matrix(M);
            } else if (O.linear_solver == 1) {
                const int64_t* bp;
                const int32_t* bi;
                double* ks;
                if (bsr_device_pattern(M, &bp, &bi, &ks, err)) return 3;
                double* A0 = multilevel_matrix(M);
                if (bsr_assemble(M, u, Up, Up2, F, P, O.precision, bp, bi, A0, ks, st)) { err = "assembly failed"; return 1; }
                Aasm = A0;
            }
            scale_copy(-1.0, R, b);
            int kits = 0;
            double kres = 0.0;
            pmode = O.precond;
            if (O.linear_solver == 1) {
                if (bicgstab(Aasm, b, du, O.krylov_rtol, O.max_krylov, &kits, &kres)) { err = "BiCGStab failed"; return 1; }
            } else if (solve(u, b, du, O.krylov_rtol, O.max_krylov, &kits, &kres)) { err = "GMRES failed"; return 1; }
            if (learned_mode(pmode) && !(kres <= O.krylov_rtol * rn * 1.0000001)) {
                // the correction did not bring GMRES to its tolerance: redo the solve with block-Jacobi
                S->fallbacks += 1;
                S->krylov_its += kits;
                pmode = 1;
                if (solve(u, b, du, O.krylov_rtol, O.max_krylov, &kits, &kres)) { err = "GMRES failed"; return 1; }
            }
            S->krylov_per_newton[it] = kits;
            S->krylov_rel[it] = rn > 0.0 ? kres / rn : 0.0;
            S->krylov_its += kits;
            double lam = 1.0, rt = 0.0;
            for (int ls = 0; ls < 12; ++ls) {
                cudaMemcpyAsync(ut, u, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
                axpby(lam, du, 1.0, ut);
                if (residual(ut, Rt)) { err = "residual launch failed"; return 1; }
                rt = norm(Rt);
                if (!O.line_search || (std::isfinite(rt) && rt <= (1.0 - 1e-4 * lam) * rn)) break;
                lam *= 0.5;
            }
            if (!std::isfinite(rt)) { err = "NaN/Inf in the residual"; return 2; }
            cudaMemcpyAsync(u, ut, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(R, Rt, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
            rn = rt;
            S->res_norm[it + 1] = rn;
        }
        cudaStreamSynchronize(st);
        S->newton_its = it;
        S->converged = rn <= target ? 1 : 0;
        S->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return 0;
    }

    Mesh& M;
    imga_physics P;
    imga_solver_opts O;
    cudaStream_t st;
    const double *Up, *Up2, *F;
    int64_t n;
    Work W;
};

}  // namespace

int newton_solve(Mesh& m, double* u, const double* up, const double* up2, const double* f, const imga_physics& ph,
                 const imga_solver_opts& o, imga_solver_stats* stats, void* stream, std::string& err) {
    std::memset(stats, 0, sizeof(*stats));
    Solver S(m, ph, o, (cudaStream_t)stream, up, up2, f);
    if (S.alloc(err)) return 3;
    if ((o.precond == 2 || o.precond == 3) && S.learned_alloc(err)) return 3;
    if ((o.precond == 4 || o.linear_solver == 1) &&
        multilevel_prepare(m, o.ml_agg > 0 ? o.ml_agg : 6, o.ml_coarse_max > 0 ? o.ml_coarse_max : 16, err))
        return 3;
    int rc = S.newton(u, stats, err);
    if (o.precond == 2 || o.precond == 3) { cudaStreamSynchronize((cudaStream_t)stream); S.learned_free(); }
    return rc;
}

void solver_free(Mesh& m) { Solver::free_work(m); }

}  // namespace imga
