// Sparse kernels: CSR SpMV (with the CG dot (A p, p) fused), the FP64 true residual
// b - A x with the restart / refinement decision, the SpMM A W of stage one, the Jacobi
// diagonal, and precision conversions.
//
// CSR rows are mapped to groups of L lanes (L in {1,2,4,8,16,32}, chosen per matrix from
// its mean row length); the lanes of a group stride through the row, so wide rows
// (elasticity, ~80 entries) load col/val coalesced while short stencil rows use L = 1.
#include <type_traits>

#include "common.cuh"
#include "launch.h"

namespace podcg {

// Row loop shared by the SpMV variants. Returns the group's row sum in lane 0 of the group.
// Loop bounds are uniform per warp so the group shuffles never diverge. With one lane per
// row, rows of up to 8 entries (stencils) issue all index/value loads first and then all
// gathers, so a row costs two memory round trips instead of one per entry.
template <int L, typename TV, typename TX>
__device__ __forceinline__ void spmv_rows(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                          const TV* __restrict__ val, const TX* __restrict__ x, int n,
                                          int row, bool valid, TX& out)
{
    TX s = TX(0);
    if (valid) {
        const int beg = __ldg(rp + row), end = __ldg(rp + row + 1);
        if (L == 1 && end - beg <= 8) {
            const int len = end - beg;
            int c[8];
            TV v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                c[t] = (t < len) ? __ldg(col + beg + t) : 0;
                v[t] = (t < len) ? __ldg(val + beg + t) : TV(0);
            }
            TX g[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) g[t] = (t < len) ? __ldg(x + c[t]) : TX(0);
#pragma unroll
            for (int t = 0; t < 8; ++t) s += TX(v[t]) * g[t];
        } else {
            const int lane = threadIdx.x & (L - 1);
            for (int k = beg + lane; k < end; k += L) s += TX(__ldg(val + k)) * __ldg(x + __ldg(col + k));
        }
    }
    if (L > 1) {
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    out = s;
}

// y = A x (stateless product; also timed by the lanes autotuner in either precision).
template <int L, typename TV = double, typename TX = double>
__global__ void __launch_bounds__(kBlock) k_spmv_plain(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                       const TV* __restrict__ val, const TX* __restrict__ x,
                                                       TX* __restrict__ y, int n)
{
    const int gpb = kBlock / L;
    const int g = threadIdx.x / L;
    const int warp_first = (blockIdx.x * gpb + (threadIdx.x & ~31) / L);
    const int stride = gridDim.x * gpb;
    for (int base = warp_first; base < n; base += stride) {
        const int row = base + (g - (threadIdx.x & ~31) / L);
        TX s;
        spmv_rows<L, TV, TX>(rp, col, val, x, n, row, row < n, s);
        if ((threadIdx.x & (L - 1)) == 0 && row < n) y[row] = s;
    }
}

// CG product: q = A p and gamma = (A p, p); the last block forms alpha = (r, z)/gamma and
// flags a breakdown when gamma is not positive (the matrix is then not SPD). CHAIN (the FP32
// inner loop): every block stores its share of gamma instead and the update pass forms
// alpha (chain_alpha).
template <int L, typename T, bool CHAIN>
__global__ void __launch_bounds__(kBlock) k_spmv_cg(const ProbDesc* __restrict__ pd, const T* __restrict__ p,
                                                    T* __restrict__ q, double* __restrict__ partials,
                                                    unsigned int* counter, DevState* st)
{
    pdl_wait_then_release();
    if (blockIdx.x == 0 && threadIdx.x == 0) st->dir_pending = 0;
    if (st->done) return;   // uniform: `done` is written by k_init / k_update only
    const int n = pd->n;
    const int32_t* rp = pd->rp;
    const int32_t* col = pd->col;
    const int gpb = kBlock / L;
    const int g = threadIdx.x / L;
    const int wg0 = (threadIdx.x & ~31) / L;
    const int stride = gridDim.x * gpb;
    // direction record (FP64): column `iters` of the Krylov-vector store while below its cap
    double* rec = nullptr;
    if constexpr (!CHAIN) {
        if (pd->krec != nullptr) {
            const int it = st->iters;
            if (it < pd->krec_cap) rec = pd->krec + (size_t)it * pd->ld;
        }
    }
    T dot = T(0);
    if constexpr (L == 1 && CHAIN) {
        // FP32, one thread per row: the next row's bounds are loaded before this row's entries, so
        // every row after a thread's first starts with its bounds already in registers (the
        // rows, and the order of each row's sum, are those of the general loop below)
        const T* __restrict__ val;
        if constexpr (std::is_same<T, double>::value) val = pd->val;
        else val = pd->val32;
        int row = blockIdx.x * gpb + threadIdx.x;
        int beg = 0, end = 0;
        if (row < n) {
            beg = __ldg(rp + row);
            end = __ldg(rp + row + 1);
        }
        for (; row < n; row += stride) {
            const int nrow = row + stride;
            int nbeg = 0, nend = 0;
            if (nrow < n) {
                nbeg = __ldg(rp + nrow);
                nend = __ldg(rp + nrow + 1);
            }
            T s = T(0);
            const int len = end - beg;
            if (len <= 8) {
                int c[8];
                T v[8], gx[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    c[t] = (t < len) ? __ldg(col + beg + t) : 0;
                    v[t] = (t < len) ? __ldg(val + beg + t) : T(0);
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) gx[t] = (t < len) ? __ldg(p + c[t]) : T(0);
#pragma unroll
                for (int t = 0; t < 8; ++t) s += v[t] * gx[t];
            } else {
                for (int k = beg; k < end; ++k) s += __ldg(val + k) * __ldg(p + __ldg(col + k));
            }
            const T pr = p[row];
            q[row] = s;
            dot += s * pr;
            if (rec) rec[row] = double(pr);
            beg = nbeg;
            end = nend;
        }
    } else {
        for (int base = blockIdx.x * gpb + wg0; base < n; base += stride) {
            const int row = base + (g - wg0);
            T s;
            if constexpr (std::is_same<T, double>::value)
                spmv_rows<L, double, double>(rp, col, pd->val, p, n, row, row < n, s);
            else
                spmv_rows<L, float, float>(rp, col, pd->val32, p, n, row, row < n, s);
            if ((threadIdx.x & (L - 1)) == 0 && row < n) {
                const T pr = p[row];
                q[row] = s;
                dot += s * pr;
                if (rec) rec[row] = double(pr);
            }
        }
    }
    if constexpr (CHAIN) {
        chain_store_gamma(double(dot), partials);
    } else {
        double acc[1] = {double(dot)};
        __shared__ double tot[1];
        if (reduce_to_last_block<1>(acc, 1, partials, counter, tot) && threadIdx.x == 0) {
            if (rec) pd->krec_gamma[st->iters] = tot[0];
            cg_product_finish(st, tot[0]);
        }
    }
}

// True residual r = b - A x in FP64 and its norm. The last block takes the outer decision:
//   FP64 mode (mixed = 0): stop when ||r|| <= tol ||b|| or on an error status; otherwise
//     restart the CG from this residual (residual replacement), at most max_refine times.
//   Mixed mode (mixed = 1): same test; otherwise it is the start of the next refinement
//     step, whose inner solve must reduce ||r|| by inner_tol, or by half the factor that
//     reaches the tolerance when that is larger.
// The decision is published to the graph's outer while-loop through `h_outer`.
template <int L, bool COND>
__global__ void __launch_bounds__(kBlock) k_residual(const ProbDesc* __restrict__ pd, const double* __restrict__ x, double* __restrict__ r,
                                                     double* __restrict__ partials, unsigned int* counter,
                                                     DevState* st, int mixed, double inner_tol,
                                                     cudaGraphConditionalHandle h_outer, int use_cond)
{
    const int n = pd->n;
    const double* b = pd->b;
    const int gpb = kBlock / L;
    const int g = threadIdx.x / L;
    const int wg0 = (threadIdx.x & ~31) / L;
    const int stride = gridDim.x * gpb;
    double rr = 0.0;
    for (int base = blockIdx.x * gpb + wg0; base < n; base += stride) {
        const int row = base + (g - wg0);
        double s;
        spmv_rows<L, double, double>(pd->rp, pd->col, pd->val, x, n, row, row < n, s);
        if ((threadIdx.x & (L - 1)) == 0 && row < n) {
            const double ri = b[row] - s;
            r[row] = ri;
            rr += ri * ri;
        }
    }
    double acc[1] = {rr};
    __shared__ double tot[1];
    if (reduce_to_last_block<1>(acc, 1, partials, counter, tot) && threadIdx.x == 0) {
        const double rt = tot[0];
        st->rr_true = rt;
        if (st->rr_stage1 < 0.0) st->rr_stage1 = rt;
        int stop = 0;
        if (st->status != 0) stop = 1;
        else if (!isfinite(rt)) { st->status = 5; stop = 1; }
        else if (rt <= st->tol2) stop = 1;
        else if (st->restarts >= st->max_refine) { st->status = 4; stop = 1; }
        else {
            st->restarts += 1;
            if (mixed) {
                st->rr_outer = rt;
                st->rnorm = sqrt(rt);
                // the inner solve sees r/||r||: it reduces that by inner_tol, or only by half of
                // the factor that reaches tol ||b|| when that is the larger (the last refinement
                // step stops where the tolerance needs it to)
                st->tol2_in = fmax(inner_tol * inner_tol, 0.25 * st->tol2 / rt);
            }
        }
        st->outer_done = stop;
        if constexpr (COND) {
            if (use_cond) cudaGraphSetConditional(h_outer, stop ? 0u : 1u);
        }
    }
}

// AW = A W for column-major W (leading dimension ldw) and AW (leading dimension lda):
// one thread per row, w accumulators in registers. For stencil-like matrices consecutive
// rows touch consecutive columns, so each W column gather is coalesced across the warp.
template <int WB, typename TV, typename T>
__global__ void __launch_bounds__(kBlock) k_spmm(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                 const TV* __restrict__ val, const T* __restrict__ W, int ldw,
                                                 T* __restrict__ AW, int lda, int n, int w)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T acc[WB];
#pragma unroll
        for (int j = 0; j < WB; ++j) acc[j] = T(0);
        const int beg = rp[i], end = rp[i + 1];
        for (int k = beg; k < end; ++k) {
            const T a = T(__ldg(val + k));
            const size_t c = (size_t)__ldg(col + k);
#pragma unroll
            for (int j = 0; j < WB; ++j)
                if (j < w) acc[j] += a * __ldg(W + (size_t)j * ldw + c);
        }
#pragma unroll
        for (int j = 0; j < WB; ++j)
            if (j < w) AW[(size_t)j * lda + i] = acc[j];
    }
}

// Jacobi preconditioner M = diag(A): dinv = 1/a_ii (FP64, plus an FP32 copy). A missing
// or non-positive diagonal sets status NOT_SPD.
__global__ void __launch_bounds__(kBlock) k_dinv(const ProbDesc* __restrict__ pd, double* __restrict__ dinv,
                                                 float* __restrict__ dinv32, DevState* st)
{
    const int n = pd->n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        const int beg = pd->rp[i], end = pd->rp[i + 1];
        for (int k = beg; k < end; ++k)
            if (pd->col[k] == i) d += pd->val[k];
        if (!(d > 0.0)) {
            st->status = 2;
            dinv[i] = 0.0;
            if (dinv32) dinv32[i] = 0.0f;
        } else {
            dinv[i] = 1.0 / d;
            if (dinv32) dinv32[i] = float(1.0 / d);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_to_f32(const double* __restrict__ a, float* __restrict__ b, size_t m)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
        b[i] = float(a[i]);
}

__global__ void __launch_bounds__(kBlock) k_desc_val_to_f32(const ProbDesc* __restrict__ pd, float* __restrict__ v32, int64_t nnz)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
        v32[i] = float(pd->val[i]);
}

// ------------------------------------------------------------------ host launchers

int spmv_lanes_for(double mean_row)
{
    if (mean_row <= 12.0) return 1;
    if (mean_row <= 24.0) return 4;
    if (mean_row <= 48.0) return 8;
    if (mean_row <= 96.0) return 16;
    return 32;
}

#define PODCG_LANES(L, ...)                                   \
    switch (L) {                                              \
    case 1: { constexpr int LL = 1; __VA_ARGS__; } break;     \
    case 2: { constexpr int LL = 2; __VA_ARGS__; } break;     \
    case 4: { constexpr int LL = 4; __VA_ARGS__; } break;     \
    case 8: { constexpr int LL = 8; __VA_ARGS__; } break;     \
    case 16: { constexpr int LL = 16; __VA_ARGS__; } break;   \
    default: { constexpr int LL = 32; __VA_ARGS__; } break;   \
    }

int grid_rows(int rows, int per_block, int sms)
{
    long long need = ((long long)rows + per_block - 1) / per_block;
    long long cap = (long long)sms * 8;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

cudaError_t launch_spmv_plain(int L, const int32_t* rp, const int32_t* col, const double* val, const double* x,
                              double* y, int n, int sms, cudaStream_t s)
{
    const int grid = grid_rows(n, kBlock / L, sms);
    PODCG_LANES(L, (k_spmv_plain<LL, double, double><<<grid, kBlock, 0, s>>>(rp, col, val, x, y, n)));
    return cudaGetLastError();
}

cudaError_t launch_spmv_plain32(int L, const int32_t* rp, const int32_t* col, const float* val, const float* x,
                                float* y, int n, int sms, cudaStream_t s)
{
    const int grid = grid_rows(n, kBlock / L, sms);
    PODCG_LANES(L, (k_spmv_plain<LL, float, float><<<grid, kBlock, 0, s>>>(rp, col, val, x, y, n)));
    return cudaGetLastError();
}

void* kernel_spmv_cg(int L, bool fp32)
{
    void* f = nullptr;
    if (fp32) { PODCG_LANES(L, f = (void*)k_spmv_cg<LL, float, true>); }
    else { PODCG_LANES(L, f = (void*)k_spmv_cg<LL, double, false>); }
    return f;
}

void* kernel_residual(int L, bool cond)
{
    void* f = nullptr;
    if (cond) { PODCG_LANES(L, f = (void*)k_residual<LL, true>); }
    else { PODCG_LANES(L, f = (void*)k_residual<LL, false>); }
    return f;
}

#define PODCG_WB(WB, ...)                                      \
    if ((WB) <= 8) { constexpr int WW = 8; __VA_ARGS__; }      \
    else if ((WB) <= 16) { constexpr int WW = 16; __VA_ARGS__; } \
    else if ((WB) <= 32) { constexpr int WW = 32; __VA_ARGS__; } \
    else if ((WB) <= 48) { constexpr int WW = 48; __VA_ARGS__; } \
    else { constexpr int WW = 64; __VA_ARGS__; }

cudaError_t launch_spmm(const int32_t* rp, const int32_t* col, const double* val, const double* W, int ldw,
                        double* AW, int lda, int n, int w, int sms, cudaStream_t s)
{
    if (w <= 0) return cudaSuccess;
    const int grid = grid_rows(n, kBlock, sms);
    PODCG_WB(w, (k_spmm<WW, double, double><<<grid, kBlock, 0, s>>>(rp, col, val, W, ldw, AW, lda, n, w)));
    return cudaGetLastError();
}

cudaError_t launch_spmm_f32(const int32_t* rp, const int32_t* col, const float* val, const float* W, int ldw,
                            float* AW, int lda, int n, int w, int sms, cudaStream_t s)
{
    if (w <= 0) return cudaSuccess;
    const int grid = grid_rows(n, kBlock, sms);
    PODCG_WB(w, (k_spmm<WW, float, float><<<grid, kBlock, 0, s>>>(rp, col, val, W, ldw, AW, lda, n, w)));
    return cudaGetLastError();
}

cudaError_t launch_dinv(const ProbDesc* pd, int n, double* dinv, float* dinv32, DevState* st, int sms, cudaStream_t s)
{
    k_dinv<<<grid_rows(n, kBlock, sms), kBlock, 0, s>>>(pd, dinv, dinv32, st);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* a, float* b, size_t m, int sms, cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    const size_t need = (m + kBlock - 1) / kBlock;
    const int grid = (int)(need < (size_t)sms * 8 ? need : (size_t)sms * 8);
    k_to_f32<<<grid, kBlock, 0, s>>>(a, b, m);
    return cudaGetLastError();
}

cudaError_t launch_desc_val_to_f32(const ProbDesc* pd, float* v32, int64_t nnz, int sms, cudaStream_t s)
{
    if (nnz == 0) return cudaSuccess;
    k_desc_val_to_f32<<<sms * 8, kBlock, 0, s>>>(pd, v32, nnz);
    return cudaGetLastError();
}

}  // namespace podcg
