// Learned block preconditioner: a 3-layer MLP (BF16 weights and activations on the tensor cores,
// FP32 accumulation, FP32 master weights, Adam) that maps an element's normalised Jacobian block
// k_e (32 x 32) plus features (log h, Intercepted flag, log10 local Re) to a 32 x 32 correction C_e;
// GMRES is then right-preconditioned by
//     P^-1 v = D^-1 v + omega sum_e M_e^T (C_e / s_e) M_e v,
// D the nodal block-Jacobi diagonal (its fallback), s_e the element's mean |diagonal| entry.
// Training target: the element's exact inverse correction (K + 0.1 I)^-1 - blockdiag4(K + 0.1 I)^-1
// of the normalised block, from the Jacobians the method itself forms (imga_element_jacobians).
// The paper has no learned component; its conclusion asks for method-specific preconditioners
// for matrix-free solvers (Sec. "Conclusion", footnote of Sec. "Matrix Assembly").
//
// GEMMs: C[m, n] = alpha sum_k A(m, k) B(n, k) + beta C[m, n] with arbitrary strides, mma.sync
// m16n8k16 BF16 x BF16 -> FP32; CTA tile 64 x 64 x 32, four warps of 32 x 32.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "imga_internal.h"
#include "vms_device.cuh"

namespace imga {

namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int GT = 64, GK = 32, GPAD = 8;

__global__ void __launch_bounds__(128) gemm_bf16(int M, int N, int K, const bf16* __restrict__ A, int64_t sam,
                                                 int64_t sak, const bf16* __restrict__ B, int64_t sbn, int64_t sbk,
                                                 float* __restrict__ C, int64_t ldc, float alpha, float beta) {
    __shared__ __align__(16) bf16 sA[GT][GK + GPAD];
    __shared__ __align__(16) bf16 sB[GT][GK + GPAD];
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gid = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int i = threadIdx.x; i < GT * GK; i += blockDim.x) {
            const int r = i / GK, kk = i % GK;
            const int gm = m0 + r, gn = n0 + r, gk = k0 + kk;
            sA[r][kk] = (gm < M && gk < K) ? A[(int64_t)gm * sam + (int64_t)gk * sak] : zero;
            sB[r][kk] = (gn < N && gk < K) ? B[(int64_t)gn * sbn + (int64_t)gk * sbk] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GK; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + gid;
                af[i][0] = pack2(sA[r][ks + 2 * tig], sA[r][ks + 2 * tig + 1]);
                af[i][1] = pack2(sA[r + 8][ks + 2 * tig], sA[r + 8][ks + 2 * tig + 1]);
                af[i][2] = pack2(sA[r][ks + 2 * tig + 8], sA[r][ks + 2 * tig + 9]);
                af[i][3] = pack2(sA[r + 8][ks + 2 * tig + 8], sA[r + 8][ks + 2 * tig + 9]);
            }
            for (int j = 0; j < 4; ++j) {
                const int c = wn + 8 * j + gid;
                bfr[j][0] = pack2(sB[c][ks + 2 * tig], sB[c][ks + 2 * tig + 1]);
                bfr[j][1] = pack2(sB[c][ks + 2 * tig + 8], sB[c][ks + 2 * tig + 9]);
            }
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 4; ++q) {
                const int r = m0 + wm + 16 * i + gid + (q >= 2 ? 8 : 0);
                const int c = n0 + wn + 8 * j + 2 * tig + (q & 1);
                if (r < M && c < N) {
                    float* dst = C + (int64_t)r * ldc + c;
                    *dst = beta == 0.f ? alpha * acc[i][j][q] : alpha * acc[i][j][q] + beta * *dst;
                }
            }
}

void gemm(cudaStream_t s, int M, int N, int K, const bf16* A, int64_t sam, int64_t sak, const bf16* B, int64_t sbn,
          int64_t sbk, float* C, int64_t ldc, float alpha = 1.f, float beta = 0.f) {
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    gemm_bf16<<<grid, 128, 0, s>>>(M, N, K, A, sam, sak, B, sbn, sbk, C, ldc, alpha, beta);
}

__global__ void to_bf16(int64_t n, const float* __restrict__ x, bf16* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}
// rows of x [n][ld_in] (first n_in columns) -> bf16 [n][ld_out] zero padded
__global__ void rows_to_bf16(int64_t n, int n_in, int64_t ld_in, const float* __restrict__ x, int ld_out,
                             bf16* __restrict__ y) {
    const int64_t tot = n * ld_out;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / ld_out;
        const int c = (int)(i % ld_out);
        y[i] = __float2bfloat16(c < n_in ? x[r * ld_in + c] : 0.f);
    }
}
// z = c + b (kept for the backward mask), h = relu(z) in bf16
__global__ void bias_relu(int64_t n, int w, float* __restrict__ z, const float* __restrict__ b, bf16* __restrict__ h) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * w; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = z[i] + b[i % w];
        z[i] = v;
        h[i] = __float2bfloat16(v > 0.f ? v : 0.f);
    }
}
__global__ void bias_add(int64_t n, int w, float* __restrict__ y, const float* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * w; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += b[i % w];
}
// dy = (y - t) / scale (bf16), loss partial sum of (y - t)^2
__global__ void mse_grad(int64_t n, const float* __restrict__ y, const float* __restrict__ t, float inv_scale,
                         bf16* __restrict__ dy, double* __restrict__ loss) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        s += (double)d * (double)d;
        dy[i] = __float2bfloat16(d * inv_scale);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}
// dz = dh * (z > 0), bf16
__global__ void relu_back(int64_t n, const float* __restrict__ dh, const float* __restrict__ z, bf16* __restrict__ dz) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dz[i] = __float2bfloat16(z[i] > 0.f ? dh[i] : 0.f);
}
// db[j] (+)= sum_r d[r][j]  (d bf16 [n][w])
__global__ void col_sum(int64_t n, int w, const bf16* __restrict__ d, float* __restrict__ db, int accumulate) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= w) return;
    float s = 0.f;
    for (int64_t r = 0; r < n; ++r) s += __bfloat162float(d[r * w + j]);
    db[j] = accumulate ? db[j] + s : s;
}
__global__ void adam(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                     float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// one warp per 32 x 32 matrix: Gauss-Jordan with partial pivoting, lane r owns row r of [A | I]
__device__ bool warp_inverse32(float a[32], float inv[32], int lane) {
    for (int j = 0; j < 32; ++j) inv[j] = j == lane ? 1.f : 0.f;
    for (int c = 0; c < 32; ++c) {
        // pivot: largest |a[c]| among rows >= c
        float best = lane >= c ? fabsf(a[c]) : -1.f;
        int bl = lane;
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (ob > best || (ob == best && ol < bl)) { best = ob; bl = ol; }
        }
        if (!(best > 0.f)) return false;
        // swap rows c and bl
        if (bl != c) {
            for (int j = 0; j < 32; ++j) {
                const float x = a[j], y = inv[j];
                const float xc = __shfl_sync(0xffffffffu, x, c), xb = __shfl_sync(0xffffffffu, x, bl);
                const float yc = __shfl_sync(0xffffffffu, y, c), yb = __shfl_sync(0xffffffffu, y, bl);
                if (lane == c) { a[j] = xb; inv[j] = yb; }
                if (lane == bl) { a[j] = xc; inv[j] = yc; }
            }
        }
        const float piv = __shfl_sync(0xffffffffu, a[c], c);
        const float ip = 1.f / piv;
        if (lane == c)
            for (int j = 0; j < 32; ++j) { a[j] *= ip; inv[j] *= ip; }
        const float f = a[c];
        for (int j = 0; j < 32; ++j) {
            const float pr = __shfl_sync(0xffffffffu, a[j], c), pi = __shfl_sync(0xffffffffu, inv[j], c);
            if (lane != c) { a[j] -= f * pr; inv[j] -= f * pi; }
        }
    }
    return true;
}

// features + targets of one element per warp from K (float64 [n][32][32])
// X [n][ldx]: 1024 normalised entries, log(h), Intercepted flag, log10(1 + Re_local); T [n][1024]
__global__ void dataset_kernel(Args A, int64_t n, const int32_t* __restrict__ elems, const double* __restrict__ K,
                               const int8_t* __restrict__ marker, float eps, int ldx, float* __restrict__ X,
                               float* __restrict__ Tg, float* __restrict__ scale_out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    const double* Ke = K + w * 1024;
    float row[32], inv[32];
    double d = fabs(Ke[lane * 32 + lane]);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    const double s = d / 32.0 > 0.0 ? d / 32.0 : 1.0;
    for (int j = 0; j < 32; ++j) row[j] = (float)(Ke[lane * 32 + j] / s);
    float* xo = X + w * ldx;
    for (int j = 0; j < 32; ++j) xo[lane * 32 + j] = row[j];
    const int32_t e = elems[w];
    if (lane == 0) {
        const double h = 2.0 / A.gd[A.lev[e]];
        double uu = 0.0;
        for (int c = 0; c < 8; ++c) {
            double u4[4];
            gather(A, A.U, A.conn[8 * (int64_t)e + c], u4);
            uu += sqrt(u4[0] * u4[0] + u4[1] * u4[1] + u4[2] * u4[2]) / 8.0;
        }
        const double nu = (A.eprob ? A.pmu[A.eprob[e]] : A.mu) / A.rho;
        xo[1024] = (float)log(h);
        xo[1025] = marker[e] == 2 ? 1.f : 0.f;
        xo[1026] = (float)log10(1.0 + uu * h / (nu > 0.0 ? nu : 1e-300));
        for (int j = 1027; j < ldx; ++j) xo[j] = 0.f;
        scale_out[w] = (float)s;
    }
    if (!Tg) return;
    // target: (Khat + eps I)^-1 - blockdiag4(Khat + eps I)^-1
    row[lane] += eps;
    float full[32];
    for (int j = 0; j < 32; ++j) full[j] = row[j];
    bool ok = warp_inverse32(full, inv, lane);
    // block-diagonal inverse of the 4x4 blocks, computed by the same routine on the block-masked matrix
    float bd[32], binv[32];
    for (int j = 0; j < 32; ++j) bd[j] = ((j >> 2) == (lane >> 2)) ? row[j] : (j == lane ? 1.f : 0.f);
    // masking keeps only the 4x4 diagonal blocks (off-block entries are zero), so the inverse is
    // block-diagonal too
    for (int j = 0; j < 32; ++j) if ((j >> 2) != (lane >> 2)) bd[j] = 0.f;
    bool ok2 = warp_inverse32(bd, binv, lane);
    float* to = Tg + w * 1024;
    for (int j = 0; j < 32; ++j) to[lane * 32 + j] = (ok && ok2) ? inv[j] - binv[j] : 0.f;
}

// z_corr += omega M_e^T (C_e / s_e) M_e v, one warp per active element, lane = local dof (a, i)
__global__ void correction_apply(Args A, int64_t n, const int32_t* __restrict__ elems, const float* __restrict__ C,
                                 const float* __restrict__ scale, float omega, const double* __restrict__ v,
                                 double* __restrict__ z) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    const int32_t e = elems[w];
    const int a = lane >> 2, comp = lane & 3;
    const int32_t id = A.conn[8 * (int64_t)e + a];
    double vv[4];
    gather(A, v, id, vv);
    const float x = (float)vv[comp];
    const float* Ce = C + w * 1024 + lane * 32;
    float y = 0.f;
    for (int j = 0; j < 32; ++j) y += Ce[j] * __shfl_sync(0xffffffffu, x, j);
    y *= omega / scale[w];
    // gather the node's 4 components to lane 4a and scatter through M_e^T
    double r[4];
    for (int k = 0; k < 4; ++k) r[k] = (double)__shfl_sync(0xffffffffu, y, (lane & ~3) + k);
    if (comp == 0) {
        Args B = A;
        B.out = z;
        scatter(B, id, r);
    }
}

// z = Dinv v + corr on free rows (prescribed rows keep Dinv v, which is v there)
__global__ void combine_rows(int64_t nn, const uint8_t* __restrict__ flag, const uint8_t* __restrict__ umask,
                             const double* __restrict__ corr, double* __restrict__ z) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    uint8_t mask = umask ? umask[n] : (uint8_t)(flag[n] & 15);
    if (flag[n] & 16) mask = 15;
    for (int k = 0; k < 4; ++k)
        if (!((mask >> k) & 1)) z[4 * n + k] += corr[4 * n + k];
}

// shift of the normalised element block before inversion: the element's constant-pressure mode is
// nearly singular, and a small shift would make the local inverse (and the correction) huge there
constexpr float kTargetShift = 0.1f;

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::min<int64_t>(4096, (n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------------------------------------
// MLP object
// ------------------------------------------------------------------------------------------
struct Mlp {
    int nin, nin_pad, w, nout;
    int64_t nparam;
    float* P = nullptr;    // master weights: W1 [w][nin_pad], b1 [w], W2 [w][w], b2 [w], W3 [nout][w], b3 [nout]
    float* G = nullptr;    // gradients, same layout
    float* Mm = nullptr;   // Adam moments
    float* Vm = nullptr;
    bf16* Pb = nullptr;    // bf16 copy of the weights
    int64_t cap = 0;       // batch capacity of the activation buffers
    bf16 *xb = nullptr, *h1 = nullptr, *h2 = nullptr, *dyb = nullptr, *dz2 = nullptr, *dz1 = nullptr;
    float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dh2 = nullptr, *dh1 = nullptr;
    double* loss = nullptr;
    int64_t step = 0;
    int64_t off(int k) const {
        const int64_t o1 = (int64_t)w * nin_pad, o2 = o1 + w, o3 = o2 + (int64_t)w * w, o4 = o3 + w,
                      o5 = o4 + (int64_t)nout * w;
        const int64_t o[6] = {0, o1, o2, o3, o4, o5};
        return o[k];
    }
};

static bool mlp_reserve(Mlp& M, int64_t b) {
    if (b <= M.cap) return true;
    cudaFree(M.xb); cudaFree(M.h1); cudaFree(M.h2); cudaFree(M.dyb); cudaFree(M.dz2); cudaFree(M.dz1);
    cudaFree(M.z1); cudaFree(M.z2); cudaFree(M.y); cudaFree(M.dh2); cudaFree(M.dh1);
    bool ok = cudaMalloc((void**)&M.xb, b * M.nin_pad * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&M.h1, b * M.w * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&M.h2, b * M.w * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&M.dyb, b * M.nout * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&M.dz2, b * M.w * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&M.dz1, b * M.w * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&M.z1, b * M.w * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&M.z2, b * M.w * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&M.y, b * M.nout * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&M.dh2, b * M.w * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&M.dh1, b * M.w * sizeof(float)) == cudaSuccess;
    M.cap = ok ? b : 0;
    return ok;
}

static void mlp_sync_bf16(Mlp& M, cudaStream_t s) { to_bf16<<<nblk(M.nparam), 256, 0, s>>>(M.nparam, M.P, M.Pb); }

// forward of a batch: X float [b][ldx] (first nin columns) -> M.y float [b][nout]
static void mlp_forward_batch(Mlp& M, const float* X, int64_t ldx, int64_t b, cudaStream_t s) {
    rows_to_bf16<<<nblk(b * M.nin_pad), 256, 0, s>>>(b, M.nin, ldx, X, M.nin_pad, M.xb);
    const bf16 *W1 = M.Pb + M.off(0), *W2 = M.Pb + M.off(2), *W3 = M.Pb + M.off(4);
    gemm(s, (int)b, M.w, M.nin_pad, M.xb, M.nin_pad, 1, W1, M.nin_pad, 1, M.z1, M.w);
    bias_relu<<<nblk(b * M.w), 256, 0, s>>>(b, M.w, M.z1, M.P + M.off(1), M.h1);
    gemm(s, (int)b, M.w, M.w, M.h1, M.w, 1, W2, M.w, 1, M.z2, M.w);
    bias_relu<<<nblk(b * M.w), 256, 0, s>>>(b, M.w, M.z2, M.P + M.off(3), M.h2);
    gemm(s, (int)b, M.nout, M.w, M.h2, M.w, 1, W3, M.w, 1, M.y, M.nout);
    bias_add<<<nblk(b * M.nout), 256, 0, s>>>(b, M.nout, M.y, M.P + M.off(5));
}

// gradient of sum((y - t)^2) / (2 n_total) over a batch, accumulated into M.G (beta = 1) or written (beta = 0)
static void mlp_backward_batch(Mlp& M, const float* T, int64_t b, double n_total, float beta, cudaStream_t s) {
    mse_grad<<<nblk(b * M.nout), 256, 0, s>>>(b * M.nout, M.y, T, (float)(1.0 / n_total), M.dyb, M.loss);
    const bf16 *W2 = M.Pb + M.off(2), *W3 = M.Pb + M.off(4);
    // dW3 [nout][w] = dy^T h2 : A(m = o, k = r) = dy[r][o], B(n = j, k = r) = h2[r][j]
    gemm(s, M.nout, M.w, (int)b, M.dyb, 1, M.nout, M.h2, 1, M.w, M.G + M.off(4), M.w, 1.f, beta);
    col_sum<<<(M.nout + 127) / 128, 128, 0, s>>>(b, M.nout, M.dyb, M.G + M.off(5), beta != 0.f);
    // dh2 [b][w] = dy W3 : A(m = r, k = o) = dy[r][o], B(n = j, k = o) = W3[o][j]
    gemm(s, (int)b, M.w, M.nout, M.dyb, M.nout, 1, W3, 1, M.w, M.dh2, M.w);
    relu_back<<<nblk(b * M.w), 256, 0, s>>>(b * M.w, M.dh2, M.z2, M.dz2);
    gemm(s, M.w, M.w, (int)b, M.dz2, 1, M.w, M.h1, 1, M.w, M.G + M.off(2), M.w, 1.f, beta);
    col_sum<<<(M.w + 127) / 128, 128, 0, s>>>(b, M.w, M.dz2, M.G + M.off(3), beta != 0.f);
    gemm(s, (int)b, M.w, M.w, M.dz2, M.w, 1, W2, 1, M.w, M.dh1, M.w);
    relu_back<<<nblk(b * M.w), 256, 0, s>>>(b * M.w, M.dh1, M.z1, M.dz1);
    gemm(s, M.w, M.nin_pad, (int)b, M.dz1, 1, M.w, M.xb, 1, M.nin_pad, M.G + M.off(0), M.nin_pad, 1.f, beta);
    col_sum<<<(M.w + 127) / 128, 128, 0, s>>>(b, M.w, M.dz1, M.G + M.off(1), beta != 0.f);
}

int mlp_create(int nin, int width, int nout, uint64_t seed, Mlp** out, std::string& err) {
    Mlp* M = new Mlp();
    M->nin = nin;
    M->nin_pad = (nin + 15) / 16 * 16;
    M->w = width;
    M->nout = nout;
    M->nparam = M->off(5) + nout;
    std::vector<float> h(M->nparam, 0.f);
    // He-uniform initial weights from SplitMix64 (biases zero)
    uint64_t st = seed * 0x9E3779B97F4A7C15ull + 1;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](int k, int fan_in, int rows, int cols, int ld) {
        const double lim = std::sqrt(6.0 / fan_in);
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) h[M->off(k) + (int64_t)r * ld + c] = (float)((2.0 * next() - 1.0) * lim);
    };
    fill(0, nin, width, nin, M->nin_pad);
    fill(2, width, width, width, width);
    fill(4, width, nout, width, width);
    for (int64_t i = M->off(4); i < M->off(5); ++i) h[i] *= 0.1f;   // small initial output
    bool ok = cudaMalloc((void**)&M->P, M->nparam * 4) == cudaSuccess && cudaMalloc((void**)&M->G, M->nparam * 4) == cudaSuccess &&
              cudaMalloc((void**)&M->Mm, M->nparam * 4) == cudaSuccess && cudaMalloc((void**)&M->Vm, M->nparam * 4) == cudaSuccess &&
              cudaMalloc((void**)&M->Pb, M->nparam * 2) == cudaSuccess && cudaMalloc((void**)&M->loss, 8) == cudaSuccess;
    if (!ok) { err = "MLP allocation failed"; delete M; return 1; }
    cudaMemcpy(M->P, h.data(), M->nparam * 4, cudaMemcpyHostToDevice);
    cudaMemset(M->G, 0, M->nparam * 4);
    cudaMemset(M->Mm, 0, M->nparam * 4);
    cudaMemset(M->Vm, 0, M->nparam * 4);
    mlp_sync_bf16(*M, 0);
    *out = M;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}

void mlp_destroy(Mlp* M) {
    if (!M) return;
    void* p[] = {M->P, M->G, M->Mm, M->Vm, M->Pb, M->loss, M->xb, M->h1, M->h2, M->dyb, M->dz2, M->dz1, M->z1, M->z2, M->y, M->dh2, M->dh1};
    for (void* q : p) if (q) cudaFree(q);
    delete M;
}

int64_t mlp_nparam(const Mlp* M) { return M->nparam; }
int mlp_nin_pad(const Mlp* M) { return M->nin_pad; }

int mlp_params(Mlp* M, float* host, int set) {
    if (set) {
        cudaMemcpy(M->P, host, M->nparam * 4, cudaMemcpyHostToDevice);
        cudaMemset(M->Mm, 0, M->nparam * 4);
        cudaMemset(M->Vm, 0, M->nparam * 4);
        M->step = 0;
        mlp_sync_bf16(*M, 0);
    } else {
        cudaMemcpy(host, M->P, M->nparam * 4, cudaMemcpyDeviceToHost);
    }
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}

int mlp_grads(Mlp* M, float* host) { return cudaMemcpy(host, M->G, M->nparam * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : 1; }

int mlp_forward(Mlp* M, const float* X, int64_t ldx, int64_t n, float* Y, cudaStream_t s) {
    const int64_t B = 4096;
    if (!mlp_reserve(*M, std::min(n, B))) return 1;
    for (int64_t r = 0; r < n; r += B) {
        const int64_t b = std::min(B, n - r);
        mlp_forward_batch(*M, X + r * ldx, ldx, b, s);
        cudaMemcpyAsync(Y + r * M->nout, M->y, b * M->nout * 4, cudaMemcpyDeviceToDevice, s);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// gradient of the mean loss over all n samples (one pass, no update); returns the loss
int mlp_gradient(Mlp* M, const float* X, int64_t ldx, const float* T, int64_t n, double* loss, cudaStream_t s) {
    const int64_t B = 4096;
    if (!mlp_reserve(*M, std::min(n, B))) return 1;
    cudaMemsetAsync(M->loss, 0, 8, s);
    for (int64_t r = 0; r < n; r += B) {
        const int64_t b = std::min(B, n - r);
        mlp_forward_batch(*M, X + r * ldx, ldx, b, s);
        mlp_backward_batch(*M, T + r * M->nout, b, (double)n, r == 0 ? 0.f : 1.f, s);
    }
    double h = 0.0;
    cudaMemcpyAsync(&h, M->loss, 8, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    *loss = h / (2.0 * (double)n);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// Adam over shuffled-free mini-batches; loss_hist[e] = mean training loss of epoch e
int mlp_train(Mlp* M, const float* X, int64_t ldx, const float* T, int64_t n, int epochs, int batch, float lr,
              double* loss_hist, cudaStream_t s) {
    if (!mlp_reserve(*M, std::min<int64_t>(n, batch))) return 1;
    for (int ep = 0; ep < epochs; ++ep) {
        cudaMemsetAsync(M->loss, 0, 8, s);
        for (int64_t r = 0; r < n; r += batch) {
            const int64_t b = std::min<int64_t>(batch, n - r);
            mlp_forward_batch(*M, X + r * ldx, ldx, b, s);
            mlp_backward_batch(*M, T + r * M->nout, b, (double)b, 0.f, s);
            ++M->step;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f / (1.f - std::pow(b1, (float)M->step)), c2 = 1.f / (1.f - std::pow(b2, (float)M->step));
            adam<<<nblk(M->nparam), 256, 0, s>>>(M->nparam, M->P, M->G, M->Mm, M->Vm, lr, b1, b2, 1e-8f, c1, c2);
            mlp_sync_bf16(*M, s);
        }
        double h = 0.0;
        cudaMemcpyAsync(&h, M->loss, 8, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (loss_hist) loss_hist[ep] = h / (2.0 * (double)n);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// ------------------------------------------------------------------------------------------
// preconditioner data: features, targets, corrections
// ------------------------------------------------------------------------------------------
int precond_dataset(const Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                    const imga_physics& ph, int precision, const int32_t* elems, int64_t n, int ldx, float* X,
                    float* T, float* scale, double* Kbuf, cudaStream_t s) {
    if (n <= 0) return 0;
    if (element_jacobians(m, u, up, up2, f, ph, precision, elems, n, Kbuf, s)) return 1;
    Args A = make_args(m, u, up, up2, f, ph, nullptr, nullptr);
    dataset_kernel<<<(unsigned)((n * 32 + 127) / 128), 128, 0, s>>>(A, n, elems, Kbuf, m.d.marker, kTargetShift, ldx, X, T, scale);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int precond_correction(const Mesh& m, const imga_physics& ph, const int32_t* elems, int64_t n, const float* C,
                       const float* scale, float omega, const double* v, double* zc, double* z, cudaStream_t s) {
    const int64_t nn = m.n_nodes();
    cudaMemsetAsync(zc, 0, nn * 4 * sizeof(double), s);
    Args A = make_args(m, v, v, v, nullptr, ph, nullptr, zc);
    if (n > 0) correction_apply<<<(unsigned)((n * 32 + 127) / 128), 128, 0, s>>>(A, n, elems, C, scale, omega, v, zc);
    if (nn > 0)
        combine_rows<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(nn, m.d.bcflag, m.user_bc ? m.d.bcmask_user : nullptr, zc, z);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int gemm_bf16_test(int M, int N, int K, const float* A, const float* B, float* C, cudaStream_t s) {
    bf16 *a = nullptr, *b = nullptr;
    if (cudaMalloc((void**)&a, (size_t)M * K * 2) != cudaSuccess || cudaMalloc((void**)&b, (size_t)N * K * 2) != cudaSuccess) return 1;
    to_bf16<<<nblk((int64_t)M * K), 256, 0, s>>>((int64_t)M * K, A, a);
    to_bf16<<<nblk((int64_t)N * K), 256, 0, s>>>((int64_t)N * K, B, b);
    gemm(s, M, N, K, a, K, 1, b, K, 1, C, N);
    cudaStreamSynchronize(s);
    cudaFree(a);
    cudaFree(b);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace imga
