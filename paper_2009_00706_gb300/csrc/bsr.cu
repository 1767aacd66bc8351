// Matrix-based path: the Jacobian assembled in 4 x 4 blocks (Algorithms 2 and 4: K = sum_e M_e^T
// k_e M_e, identity rows for prescribed components), its product with a vector, and a multilevel
// preconditioner built from it by block coarsening.
//
// Multilevel hierarchy.  Level 0 is the assembled matrix, one block row per node, nodes in Morton
// order.  Level l + 1 aggregates `agg` consecutive block rows of level l (Morton ranges, so aggregates
// stay compact) with a piecewise-constant prolongation P_l per unknown that leaves out the rows of
// level l that are not free (identity rows and empty rows of level 0, dead rows of coarser levels):
//     A_{l+1} = P_l^T A_l P_l,   block (I, J) = sum over i in I, j in J of F_i A_l(i, j) F_j,
// F the diagonal 0/1 mask of free unknowns.  Every row of P has at most one nonzero, so this is a
// block coarsening: no general sparse product.  Since the columns of a fine row are sorted, the fine
// blocks of coarse block (I, J) in fine row i are one contiguous range, and each coarse block is a
// gather in a fixed order (deterministic).  A coarse unknown that no free row reaches (a dead row)
// gets an identity row.  The last level (at most `coarse_max` block rows) is inverted densely.
// One V-cycle applies `nu` damped block-Jacobi sweeps (weight omega), the coarse correction, and `nu`
// sweeps more.  The paper preconditions its Krylov solver with additive Schwarz; its conclusion asks
// for preconditioners suited to the method.  Block coarsening needs only the assembled blocks.
//
// Arithmetic: the hierarchy and the V-cycle run in T = double (plain FP64 path) or T = float (mixed
// path; the assembly itself accumulates in float64).

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "imga_internal.h"

namespace imga {

namespace {

constexpr int kMaxLevels = 24;

// ------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------
// y = b - A x (b null: y = A x); four threads per block row, thread i forms component i
template <class T>
__global__ void __launch_bounds__(256) bsr_resid(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                                 const T* __restrict__ val, const T* __restrict__ x,
                                                 const T* __restrict__ b, T* __restrict__ y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = t >> 2;
    const int i = (int)(t & 3);
    if (row >= n) return;
    T acc = T(0);
    for (int64_t q = ptr[row], q1 = ptr[row + 1]; q < q1; ++q) {
        const int64_t c = idx[q];
        const T* v = val + 16 * q + 4 * i;
        const T* xc = x + 4 * c;
        acc += v[0] * xc[0] + v[1] * xc[1] + v[2] * xc[2] + v[3] * xc[3];
    }
    y[4 * row + i] = b ? b[4 * row + i] - acc : acc;
}

// free mask of level 0 from the assembled float64 matrix: bit k set unless row (node, k) is an
// identity row (diagonal 1, absolute row sum 1) or empty (absolute row sum 0)
__global__ void ml_free0(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                         const double* __restrict__ val, uint8_t* __restrict__ fr) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    uint8_t m = 0;
    for (int k = 0; k < 4; ++k) {
        double s = 0.0, d = 0.0;
        for (int64_t q = ptr[row]; q < ptr[row + 1]; ++q) {
            const double* v = val + 16 * q + 4 * k;
            s += fabs(v[0]) + fabs(v[1]) + fabs(v[2]) + fabs(v[3]);
            if (idx[q] == row) d = v[k];
        }
        const bool fixed = (d == 1.0 && s == 1.0) || s == 0.0;
        if (!fixed) m |= (uint8_t)(1 << k);
    }
    fr[row] = m;
}

template <class S, class D>
__global__ void convert_kernel(int64_t n, const S* __restrict__ a, D* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (D)a[i];
}

// coarse block (I, J) = sum over fine rows i of aggregate I and their blocks with column in aggregate J
// of the masked fine block; 16 threads per coarse block, thread (k, m) forms entry (k, m)
template <class T>
__global__ void __launch_bounds__(256) ml_coarsen(int64_t nc, const int64_t* __restrict__ cptr,
                                                  const int32_t* __restrict__ cidx, int64_t nbc, int64_t nf,
                                                  const int64_t* __restrict__ fptr, const int32_t* __restrict__ fidx,
                                                  const T* __restrict__ fval, const uint8_t* __restrict__ ffree, int agg,
                                                  const int64_t* __restrict__ crow, T* __restrict__ cval) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cb = t >> 4;
    if (cb >= nbc) return;
    const int k = (int)((t >> 2) & 3), mm = (int)(t & 3);
    const int64_t I = crow[cb];
    const int32_t J = cidx[cb];
    const int64_t j0 = (int64_t)J * agg, j1 = j0 + agg;
    double acc = 0.0;
    for (int64_t i = I * agg, iend = (I * agg + agg < nf ? I * agg + agg : nf); i < iend; ++i) {
        if (!((ffree[i] >> k) & 1)) continue;
        int64_t lo = fptr[i], hi = fptr[i + 1];
        while (lo < hi) {   // first column >= j0
            const int64_t mid = (lo + hi) >> 1;
            if (fidx[mid] < j0) lo = mid + 1;
            else hi = mid;
        }
        for (int64_t q = lo; q < fptr[i + 1] && fidx[q] < j1; ++q)
            if ((ffree[fidx[q]] >> mm) & 1) acc += (double)fval[16 * q + 4 * k + mm];
    }
    cval[16 * cb + 4 * k + mm] = (T)acc;
}

// dead rows of a coarse level (no free fine row reaches them) get an identity row; fr = the rest
template <class T>
__global__ void ml_dead(int64_t n, const int64_t* __restrict__ ptr, const int64_t* __restrict__ diag,
                        T* __restrict__ val, uint8_t* __restrict__ fr) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    uint8_t m = 0;
    for (int k = 0; k < 4; ++k) {
        T s = T(0);
        for (int64_t q = ptr[row]; q < ptr[row + 1]; ++q) {
            const T* v = val + 16 * q + 4 * k;
            s += fabs(v[0]) + fabs(v[1]) + fabs(v[2]) + fabs(v[3]);
        }
        if (s == T(0)) val[16 * diag[row] + 5 * k] = T(1);
        else m |= (uint8_t)(1 << k);
    }
    fr[row] = m;
}

// inverse of every diagonal block (Gauss-Jordan with partial pivoting in float64); a block whose
// pivot falls below 1e-14 of its largest entry is replaced by the identity
template <class T>
__global__ void ml_diag_inv(int64_t n, const int64_t* __restrict__ diag, const T* __restrict__ val, T* __restrict__ Dinv) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double a[4][8];
    double scale = 0.0;
    const T* v = val + 16 * diag[r];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            a[i][j] = (double)v[4 * i + j];
            a[i][4 + j] = i == j ? 1.0 : 0.0;
            scale = fmax(scale, fabs(a[i][j]));
        }
    bool ok = scale > 0.0;
    for (int col = 0; col < 4 && ok; ++col) {
        int piv = col;
        for (int i = col + 1; i < 4; ++i)
            if (fabs(a[i][col]) > fabs(a[piv][col])) piv = i;
        if (!(fabs(a[piv][col]) > 1e-14 * scale)) { ok = false; break; }
        if (piv != col)
            for (int j = 0; j < 8; ++j) { const double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
        const double inv = 1.0 / a[col][col];
        for (int j = 0; j < 8; ++j) a[col][j] *= inv;
        for (int i = 0; i < 4; ++i) {
            if (i == col) continue;
            const double f = a[i][col];
            if (f != 0.0)
                for (int j = 0; j < 8; ++j) a[i][j] -= f * a[col][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Dinv[16 * r + 4 * i + j] = (T)(ok ? a[i][4 + j] : (i == j ? 1.0 : 0.0));
}

// dense copy [N][N] (N = 4 n) of the last level; an all-zero row gets a 1 on the diagonal
template <class T>
__global__ void ml_densify(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                           const T* __restrict__ val, double* __restrict__ dense) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int64_t N = 4 * n;
    for (int k = 0; k < 4; ++k) {
        double* d = dense + (4 * row + k) * N;
        for (int64_t j = 0; j < N; ++j) d[j] = 0.0;
        double s = 0.0;
        for (int64_t q = ptr[row]; q < ptr[row + 1]; ++q)
            for (int mm = 0; mm < 4; ++mm) {
                const double x = (double)val[16 * q + 4 * k + mm];
                d[4 * (int64_t)idx[q] + mm] = x;
                s += fabs(x);
            }
        if (s == 0.0) d[4 * row + k] = 1.0;
    }
}

// Inverse of the dense N x N matrix by Gauss-Jordan with partial pivoting, one block, the
// augmented [A | I] in shared memory (float64).  A singular column leaves *bad set and the identity.
template <class T>
__global__ void __launch_bounds__(512) ml_dense_inverse(int N, const double* __restrict__ A, T* __restrict__ Ainv,
                                                        int* __restrict__ bad) {
    extern __shared__ double sa[];   // [N][2N]
    __shared__ int s_piv;
    __shared__ double s_scale;
    const int W = 2 * N;
    for (int t = threadIdx.x; t < N * W; t += blockDim.x) {
        const int i = t / W, j = t % W;
        sa[t] = j < N ? A[(int64_t)i * N + j] : (j - N == i ? 1.0 : 0.0);
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < N * N; ++t) s = fmax(s, fabs(A[t]));
        s_scale = s;
    }
    __syncthreads();
    bool ok = true;
    for (int col = 0; col < N; ++col) {
        if (threadIdx.x == 0) {
            int p = col;
            for (int i = col + 1; i < N; ++i)
                if (fabs(sa[i * W + col]) > fabs(sa[p * W + col])) p = i;
            s_piv = fabs(sa[p * W + col]) > 1e-300 + 1e-15 * s_scale ? p : -1;
        }
        __syncthreads();
        const int p = s_piv;
        if (p < 0) { ok = false; break; }
        if (p != col)
            for (int j = threadIdx.x; j < W; j += blockDim.x) {
                const double t = sa[col * W + j];
                sa[col * W + j] = sa[p * W + j];
                sa[p * W + j] = t;
            }
        __syncthreads();
        const double inv = 1.0 / sa[col * W + col];
        __syncthreads();
        for (int j = threadIdx.x; j < W; j += blockDim.x) sa[col * W + j] *= inv;
        __syncthreads();
        for (int t = threadIdx.x; t < N * W; t += blockDim.x) {
            const int i = t / W, j = t % W;
            if (i == col || j == col) continue;
            const double f = sa[i * W + col];
            if (f != 0.0) sa[t] -= f * sa[col * W + j];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += blockDim.x)
            if (i != col) sa[i * W + col] = 0.0;
        __syncthreads();
    }
    if (!ok && threadIdx.x == 0) *bad = 1;
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
        const int i = t / N, j = t % N;
        Ainv[t] = (T)(ok ? sa[i * W + N + j] : (i == j ? 1.0 : 0.0));
    }
}

// x = omega Dinv r   (first sweep from x = 0)
template <class T>
__global__ void ml_smooth0(int64_t n, const T* __restrict__ Dinv, T omega, const T* __restrict__ r, T* __restrict__ x) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = t >> 2;
    const int i = (int)(t & 3);
    if (row >= n) return;
    const T* M = Dinv + 16 * row + 4 * i;
    const T* v = r + 4 * row;
    x[4 * row + i] = omega * (M[0] * v[0] + M[1] * v[1] + M[2] * v[2] + M[3] * v[3]);
}

// x += omega Dinv res
template <class T>
__global__ void ml_smooth(int64_t n, const T* __restrict__ Dinv, T omega, const T* __restrict__ res, T* __restrict__ x) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = t >> 2;
    const int i = (int)(t & 3);
    if (row >= n) return;
    const T* M = Dinv + 16 * row + 4 * i;
    const T* v = res + 4 * row;
    x[4 * row + i] += omega * (M[0] * v[0] + M[1] * v[1] + M[2] * v[2] + M[3] * v[3]);
}

// rc[I][k] = sum over the rows i of aggregate I of F_i res[i][k]
template <class T>
__global__ void ml_restrict(int64_t nc, int64_t nf, int agg, const uint8_t* __restrict__ fr, const T* __restrict__ res,
                            T* __restrict__ rc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t I = t >> 2;
    const int k = (int)(t & 3);
    if (I >= nc) return;
    T s = T(0);
    for (int64_t i = I * agg, iend = (I * agg + agg < nf ? I * agg + agg : nf); i < iend; ++i)
        if ((fr[i] >> k) & 1) s += res[4 * i + k];
    rc[4 * I + k] = s;
}

// x[i][k] += F_i xc[I(i)][k]
template <class T>
__global__ void ml_prolong(int64_t nf, int agg, const uint8_t* __restrict__ fr, const T* __restrict__ xc, T* __restrict__ x) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t >> 2;
    const int k = (int)(t & 3);
    if (i >= nf) return;
    if ((fr[i] >> k) & 1) x[4 * i + k] += xc[4 * (i / agg) + k];
}

// y = Ainv r for the dense last level (N <= 4 * coarse_max); one block
template <class T>
__global__ void ml_dense_apply(int N, const T* __restrict__ Ainv, const T* __restrict__ r, T* __restrict__ y) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        T s = T(0);
        for (int j = 0; j < N; ++j) s += Ainv[(int64_t)i * N + j] * r[j];
        y[i] = s;
    }
}

inline unsigned blocks(int64_t threads, int per = 256) { return (unsigned)std::max<int64_t>(1, (threads + per - 1) / per); }

}  // namespace

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
struct MLPattern {
    int64_t n = 0;                  // block rows
    std::vector<int64_t> ptr;       // [n + 1]
    std::vector<int32_t> idx;
    int64_t *dptr = nullptr, *ddiag = nullptr, *drow = nullptr;   // device: pattern, diagonal position, row of each block
    int32_t* didx = nullptr;
};

template <class T>
struct MLValues {
    T* A[kMaxLevels] = {};
    T* Dinv[kMaxLevels] = {};
    T *r[kMaxLevels] = {}, *x[kMaxLevels] = {}, *res[kMaxLevels] = {};
    T* Cinv = nullptr;
    bool alloc = false;
};

struct Multilevel {
    int agg = 0, coarse_max = 0;
    std::vector<MLPattern> lev;     // lev.back() is the dense level
    uint8_t* fr[kMaxLevels] = {};   // free masks per level (device)
    double* A0 = nullptr;           // assembled fine matrix, float64
    double* Ks = nullptr;           // surface element matrices (assembly workspace)
    double* dense = nullptr;        // [N][N] last level, float64
    int* bad = nullptr;
    MLValues<double> vd;
    MLValues<float> vf;
    int precision = -1;             // precision of the last setup
    int nu = 1;
    double omega = 0.5;
};

namespace {

template <class T>
void free_values(MLValues<T>& v, size_t nlev) {
    for (size_t l = 0; l < nlev; ++l) {
        if (l > 0 || !std::is_same<T, double>::value) cudaFree(v.A[l]);
        cudaFree(v.Dinv[l]); cudaFree(v.r[l]); cudaFree(v.x[l]); cudaFree(v.res[l]);
    }
    cudaFree(v.Cinv);
    v = MLValues<T>();
}

// the coarse pattern of aggregating `agg` consecutive block rows and columns
void coarsen_pattern(const MLPattern& f, int agg, MLPattern& c) {
    c.n = (f.n + agg - 1) / agg;
    c.ptr.assign(c.n + 1, 0);
    std::vector<std::vector<int32_t>> rows(c.n);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t I = 0; I < c.n; ++I) {
        std::vector<int32_t>& cols = rows[I];
        for (int64_t i = I * agg; i < std::min<int64_t>(I * agg + agg, f.n); ++i)
            for (int64_t q = f.ptr[i]; q < f.ptr[i + 1]; ++q) cols.push_back(f.idx[q] / agg);
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    }
    for (int64_t I = 0; I < c.n; ++I) c.ptr[I + 1] = c.ptr[I] + (int64_t)rows[I].size();
    c.idx.resize(c.ptr[c.n]);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t I = 0; I < c.n; ++I) std::copy(rows[I].begin(), rows[I].end(), c.idx.begin() + c.ptr[I]);
}

bool upload_pattern(MLPattern& p, std::string& err) {
    const int64_t nb = p.ptr.back();
    std::vector<int64_t> diag(std::max<int64_t>(1, p.n), -1), row(std::max<int64_t>(1, nb), 0);
    for (int64_t i = 0; i < p.n; ++i)
        for (int64_t q = p.ptr[i]; q < p.ptr[i + 1]; ++q) {
            row[q] = i;
            if (p.idx[q] == i) diag[i] = q;
        }
    for (int64_t i = 0; i < p.n; ++i)
        if (diag[i] < 0) { err = "block pattern without a diagonal block"; return false; }
    auto up = [&](auto** d, const auto& v) {
        using E = typename std::remove_reference<decltype(v)>::type::value_type;
        const size_t bytes = std::max<size_t>(1, v.size()) * sizeof(E);
        if (cudaMalloc((void**)d, bytes) != cudaSuccess) return false;
        return v.empty() || cudaMemcpy(*d, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!up(&p.dptr, p.ptr) || !up(&p.didx, p.idx) || !up(&p.ddiag, diag) || !up(&p.drow, row)) {
        err = "multilevel pattern upload failed";
        cudaGetLastError();
        return false;
    }
    return true;
}

template <class T>
MLValues<T>& values(Multilevel& L);
template <> MLValues<double>& values<double>(Multilevel& L) { return L.vd; }
template <> MLValues<float>& values<float>(Multilevel& L) { return L.vf; }

template <class T>
bool alloc_values(Multilevel& L, std::string& err) {
    MLValues<T>& v = values<T>(L);
    if (v.alloc) return true;
    const size_t nl = L.lev.size();
    bool ok = true;
    for (size_t l = 0; l < nl && ok; ++l) {
        const MLPattern& p = L.lev[l];
        const int64_t nb = p.ptr.back(), n = std::max<int64_t>(1, p.n);
        if (l == 0 && std::is_same<T, double>::value) v.A[0] = (T*)L.A0;
        else ok = ok && cudaMalloc((void**)&v.A[l], std::max<int64_t>(1, nb) * 16 * sizeof(T)) == cudaSuccess;
        ok = ok && cudaMalloc((void**)&v.Dinv[l], n * 16 * sizeof(T)) == cudaSuccess &&
             cudaMalloc((void**)&v.r[l], n * 4 * sizeof(T)) == cudaSuccess &&
             cudaMalloc((void**)&v.x[l], n * 4 * sizeof(T)) == cudaSuccess &&
             cudaMalloc((void**)&v.res[l], n * 4 * sizeof(T)) == cudaSuccess;
    }
    const int64_t N = 4 * L.lev.back().n;
    ok = ok && cudaMalloc((void**)&v.Cinv, std::max<int64_t>(1, N * N) * sizeof(T)) == cudaSuccess;
    if (!ok) { err = "multilevel allocation failed"; cudaGetLastError(); return false; }
    v.alloc = true;
    return true;
}

template <class T>
int setup_values(const Mesh& m, Multilevel& L, cudaStream_t s) {
    MLValues<T>& v = values<T>(L);
    const size_t nl = L.lev.size();
    const MLPattern& p0 = L.lev[0];
    if (!std::is_same<T, double>::value)
        convert_kernel<double, T><<<blocks(16 * p0.ptr.back()), 256, 0, s>>>(16 * p0.ptr.back(), L.A0, v.A[0]);
    for (size_t l = 0; l + 1 < nl; ++l) {
        const MLPattern &f = L.lev[l], &c = L.lev[l + 1];
        ml_diag_inv<T><<<blocks(f.n, 128), 128, 0, s>>>(f.n, f.ddiag, v.A[l], v.Dinv[l]);
        const int64_t nbc = c.ptr.back();
        ml_coarsen<T><<<blocks(16 * nbc), 256, 0, s>>>(c.n, c.dptr, c.didx, nbc, f.n, f.dptr, f.didx, v.A[l], L.fr[l],
                                                         L.agg, c.drow, v.A[l + 1]);
        ml_dead<T><<<blocks(c.n), 256, 0, s>>>(c.n, c.dptr, c.ddiag, v.A[l + 1], L.fr[l + 1]);
    }
    const MLPattern& d = L.lev.back();
    const int N = (int)(4 * d.n);
    if (N > 0) {
        ml_densify<T><<<blocks(d.n), 256, 0, s>>>(d.n, d.dptr, d.didx, v.A[nl - 1], L.dense);
        const size_t smem = (size_t)N * 2 * N * sizeof(double);
        ml_dense_inverse<T><<<1, 512, smem, s>>>(N, L.dense, v.Cinv, L.bad);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <class T>
void vcycle(Multilevel& L, size_t l, cudaStream_t s) {
    MLValues<T>& v = values<T>(L);
    const MLPattern& p = L.lev[l];
    if (l + 1 == L.lev.size()) {
        ml_dense_apply<T><<<1, 256, 0, s>>>((int)(4 * p.n), v.Cinv, v.r[l], v.x[l]);
        return;
    }
    const T om = (T)L.omega;
    const int64_t th = 4 * p.n;
    ml_smooth0<T><<<blocks(th), 256, 0, s>>>(p.n, v.Dinv[l], om, v.r[l], v.x[l]);
    for (int k = 1; k < L.nu; ++k) {
        bsr_resid<T><<<blocks(th), 256, 0, s>>>(p.n, p.dptr, p.didx, v.A[l], v.x[l], v.r[l], v.res[l]);
        ml_smooth<T><<<blocks(th), 256, 0, s>>>(p.n, v.Dinv[l], om, v.res[l], v.x[l]);
    }
    bsr_resid<T><<<blocks(th), 256, 0, s>>>(p.n, p.dptr, p.didx, v.A[l], v.x[l], v.r[l], v.res[l]);
    const MLPattern& c = L.lev[l + 1];
    ml_restrict<T><<<blocks(4 * c.n), 256, 0, s>>>(c.n, p.n, L.agg, L.fr[l], v.res[l], v.r[l + 1]);
    vcycle<T>(L, l + 1, s);
    ml_prolong<T><<<blocks(th), 256, 0, s>>>(p.n, L.agg, L.fr[l], v.x[l + 1], v.x[l]);
    for (int k = 0; k < L.nu; ++k) {
        bsr_resid<T><<<blocks(th), 256, 0, s>>>(p.n, p.dptr, p.didx, v.A[l], v.x[l], v.r[l], v.res[l]);
        ml_smooth<T><<<blocks(th), 256, 0, s>>>(p.n, v.Dinv[l], om, v.res[l], v.x[l]);
    }
}

}  // namespace

void multilevel_free(Mesh& m) {
    Multilevel* L = (Multilevel*)m.mlev;
    if (!L) return;
    free_values(L->vd, L->lev.size());
    free_values(L->vf, L->lev.size());
    for (auto& p : L->lev) { cudaFree(p.dptr); cudaFree(p.didx); cudaFree(p.ddiag); cudaFree(p.drow); }
    for (int l = 0; l < kMaxLevels; ++l) cudaFree(L->fr[l]);
    cudaFree(L->A0); cudaFree(L->Ks); cudaFree(L->dense); cudaFree(L->bad);
    delete L;
    m.mlev = nullptr;
}

// Patterns of the hierarchy (host, once per mesh and (agg, coarse_max)) and the device arrays.
int multilevel_prepare(Mesh& m, int agg, int coarse_max, std::string& err) {
    Multilevel* L = (Multilevel*)m.mlev;
    if (L && L->agg == agg && L->coarse_max == coarse_max) return 0;
    multilevel_free(m);
    if (agg < 2 || coarse_max < 1 || 4 * coarse_max > 96) { err = "multilevel: agg >= 2 and 1 <= coarse_max <= 24"; return 1; }
    if (m.bsr_ptr.empty()) build_bsr_pattern(m);
    L = new Multilevel();
    m.mlev = L;
    L->agg = agg;
    L->coarse_max = coarse_max;
    MLPattern p0;
    p0.n = m.n_nodes();
    p0.ptr = m.bsr_ptr;
    p0.idx = m.bsr_idx;
    L->lev.push_back(std::move(p0));
    while (L->lev.back().n > coarse_max) {
        if ((int)L->lev.size() >= kMaxLevels) { err = "multilevel: too many levels"; multilevel_free(m); return 1; }
        MLPattern c;
        coarsen_pattern(L->lev.back(), agg, c);
        L->lev.push_back(std::move(c));
    }
    for (auto& p : L->lev)
        if (!upload_pattern(p, err)) { multilevel_free(m); return 1; }
    const int64_t N = 4 * L->lev.back().n;
    bool ok = cudaMalloc((void**)&L->A0, std::max<int64_t>(1, m.bsr_ptr.back()) * 16 * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&L->Ks, std::max<size_t>(1, m.sq_hosts.size()) * 1024 * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&L->dense, std::max<int64_t>(1, N * N) * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&L->bad, sizeof(int)) == cudaSuccess;
    for (size_t l = 0; l < L->lev.size() && ok; ++l)
        ok = cudaMalloc((void**)&L->fr[l], std::max<int64_t>(1, L->lev[l].n)) == cudaSuccess;
    if (!ok) { err = "multilevel allocation failed"; cudaGetLastError(); multilevel_free(m); return 1; }
    cudaMemset(L->bad, 0, sizeof(int));
    // the dense inverse keeps [N][2N] doubles in shared memory
    const int smem = (int)(N * 2 * N * sizeof(double));
    cudaFuncSetAttribute(ml_dense_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, std::max(smem, 1));
    cudaFuncSetAttribute(ml_dense_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, std::max(smem, 1));
    return 0;
}

// Assemble the fine matrix at the state (u, ...) and build every level's values in the precision.
int multilevel_setup(Mesh& m, const double* u, const double* up, const double* up2, const double* f,
                     const imga_physics& ph, int precision, int nu, double omega, void* stream, std::string& err) {
    Multilevel* L = (Multilevel*)m.mlev;
    if (!L) { err = "multilevel: not prepared"; return 1; }
    cudaStream_t s = (cudaStream_t)stream;
    L->nu = std::max(1, nu);
    L->omega = omega;
    L->precision = precision;
    const MLPattern& p0 = L->lev[0];
    if (bsr_assemble(m, u, up, up2, f, ph, precision, p0.dptr, p0.didx, L->A0, L->Ks, s)) { err = "assembly failed"; return 1; }
    ml_free0<<<blocks(p0.n), 256, 0, s>>>(p0.n, p0.dptr, p0.didx, L->A0, L->fr[0]);
    if (precision == 0) {
        if (!alloc_values<double>(*L, err)) return 1;
        return setup_values<double>(m, *L, s) ? (err = "multilevel setup launch failed", 1) : 0;
    }
    if (!alloc_values<float>(*L, err)) return 1;
    return setup_values<float>(m, *L, s) ? (err = "multilevel setup launch failed", 1) : 0;
}

// z = V-cycle(r), float64 vectors [n_nodes][4]
int multilevel_apply(Mesh& m, const double* r, double* z, void* stream) {
    Multilevel* L = (Multilevel*)m.mlev;
    if (!L || L->precision < 0) return 1;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n4 = 4 * L->lev[0].n;
    if (n4 == 0) return 0;
    if (L->precision == 0) {
        cudaMemcpyAsync(L->vd.r[0], r, n4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        vcycle<double>(*L, 0, s);
        cudaMemcpyAsync(z, L->vd.x[0], n4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    } else {
        convert_kernel<double, float><<<blocks(n4), 256, 0, s>>>(n4, r, L->vf.r[0]);
        vcycle<float>(*L, 0, s);
        convert_kernel<float, double><<<blocks(n4), 256, 0, s>>>(n4, L->vf.x[0], z);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// block rows per level (host array of n_levels entries, may be null) and whether the dense
// inverse met a singular pivot; returns the number of levels
int multilevel_info(Mesh& m, int64_t* rows, int* singular) {
    Multilevel* L = (Multilevel*)m.mlev;
    if (!L) return 0;
    if (rows)
        for (size_t l = 0; l < L->lev.size(); ++l) rows[l] = L->lev[l].n;
    if (singular) {
        int h = 0;
        cudaMemcpy(&h, L->bad, sizeof(int), cudaMemcpyDeviceToHost);
        *singular = h;
    }
    return (int)L->lev.size();
}

// y = A x with the assembled float64 matrix val on the mesh's block pattern
int bsr_spmv(Mesh& m, const double* val, const double* x, double* y, void* stream, std::string& err) {
    if (m.bsr_ptr.empty()) build_bsr_pattern(m);
    Multilevel* L = (Multilevel*)m.mlev;
    if (!L) { err = "the block pattern is not on the device (call the assembly first)"; return 1; }
    const MLPattern& p = L->lev[0];
    if (p.n > 0)
        bsr_resid<double><<<blocks(4 * p.n), 256, 0, (cudaStream_t)stream>>>(p.n, p.dptr, p.didx, val, x, nullptr, y);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// the assembled float64 fine matrix of the hierarchy (valid after multilevel_setup)
double* multilevel_matrix(Mesh& m) { return m.mlev ? ((Multilevel*)m.mlev)->A0 : nullptr; }

// the device pattern of level 0 (prepared on first use with default hierarchy parameters)
int bsr_device_pattern(Mesh& m, const int64_t** ptr, const int32_t** idx, double** ks, std::string& err) {
    if (!m.mlev && multilevel_prepare(m, 6, 16, err)) return 1;
    Multilevel* L = (Multilevel*)m.mlev;
    *ptr = L->lev[0].dptr;
    *idx = L->lev[0].didx;
    *ks = L->Ks;
    return 0;
}

}  // namespace imga
