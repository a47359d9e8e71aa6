// Kernels of the FP32-inner / FP64-refinement mode.
//
// Each outer step (graph outer while-loop) is:
//   k_residual   r64 = b - A x in FP64 and the stop test (k_sparse.cu)
//   k_mx_proj    r32 = float(r64/||r64||) and c = W32^T r32: the stage-one projection of the
//                correction (augmented CG only searches the A-orthogonal complement of
//                range(W), so the correction's component in range(W) is solved directly
//                with the stage-one factor, as Algorithm 2 does for x)
//   k_mx_start   dhat = R^{-1} R^{-T} c, d = W32 dhat, r32 -= AW32 dhat
//   k_init / inner while { k_spmv_cg, k_update, k_dir } in FP32 on A d = r32
//   k_mx_accum   x += ||r64|| double(d)
// All of them return at once after the outer loop decided to stop (outer_done), because
// the rest of the outer body still runs in that pass.
//
// Also here: the FP32 lift W32 = S32 C, the FP32 Gram partials (FP32 products summed in
// FP32 over 32 rows, then in FP64), and the mixed-mode stage-one lift x0 = W32 what.
#include "common.cuh"
#include "launch.h"

namespace podcg {

template <int WB>
__device__ __forceinline__ void block_mu32(const double* __restrict__ Rinv, const double* __restrict__ c, int w,
                                           double* s_R, double* s_t, double* s_mu)
{
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        const int i = e / w, j = e % w;
        s_R[i * WB + j] = Rinv[i * kWMax + j];
    }
    __syncthreads();
    for (int a = threadIdx.x; a < w; a += blockDim.x) {
        double v = 0.0;
        for (int k = 0; k <= a; ++k) v += s_R[k * WB + a] * c[k];
        s_t[a] = v;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < w; a += blockDim.x) {
        double v = 0.0;
        for (int k = a; k < w; ++k) v += s_R[a * WB + k] * s_t[k];
        s_mu[a] = v;
    }
    __syncthreads();
}

template <int WB>
__global__ void __launch_bounds__(kBlock) k_mx_proj(int n, int ld, const double* __restrict__ r64,
                                                    float* __restrict__ r32, const float* __restrict__ W32,
                                                    double* __restrict__ partials, unsigned int* counter,
                                                    DevState* st)
{
    if (st->outer_done) return;
    constexpr int CPW = WB > 0 ? (WB + kWarps - 1) / kWarps : 1;
    const int w = st->w;
    const double inv = st->rnorm > 0.0 ? 1.0 / st->rnorm : 1.0;
    __shared__ float s_z[kBlock];
    __shared__ double s_blk[WB + 2];
    float cacc[CPW];
#pragma unroll
    for (int k = 0; k < CPW; ++k) cacc[k] = 0.0f;
    for (int row0 = blockIdx.x * kBlock; row0 < n; row0 += gridDim.x * kBlock) {
        const int i = row0 + threadIdx.x;
        float ri = 0.0f;
        if (i < n) {
            ri = float(r64[i] * inv);
            r32[i] = ri;
        }
        if (WB > 0) {
            s_z[threadIdx.x] = ri;
            __syncthreads();
            tile_columns<CPW, float>(W32, ld, w, row0, n, s_z, cacc);
            __syncthreads();
        }
    }
    block_totals<CPW, float>(0.0f, 0.0f, cacc, w, s_blk);
    __shared__ double tot[WB + 2];
    if (partials_to_last_block(s_blk, 2 + w, partials, counter, tot)) {
        for (int a = threadIdx.x; a < w; a += blockDim.x) st->c[a] = tot[2 + a];
    }
}

template <int WB>
__global__ void __launch_bounds__(kBlock) k_mx_start(int n, int ld, float* __restrict__ d32,
                                                     float* __restrict__ r32, const float* __restrict__ W32,
                                                     const float* __restrict__ AW32, const double* __restrict__ Rinv,
                                                     const DevState* st)
{
    if (st->outer_done) return;
    const int w = st->w;
    __shared__ double s_R[WB > 0 ? WB * WB : 1];
    __shared__ double s_t[WB > 0 ? WB : 1], s_mu[WB > 0 ? WB : 1];
    __shared__ float s_dh[WB > 0 ? WB : 1];
    if (WB > 0) {
        block_mu32<WB>(Rinv, st->c, w, s_R, s_t, s_mu);
        for (int j = threadIdx.x; j < WB; j += blockDim.x) s_dh[j] = (j < w) ? float(s_mu[j]) : 0.0f;
        __syncthreads();
    }
    float dh[WB > 0 ? WB : 1];
#pragma unroll
    for (int j = 0; j < WB; ++j) dh[j] = (WB > 0) ? s_dh[j] : 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float di = 0.0f, ai = 0.0f;
#pragma unroll
        for (int j = 0; j < WB; ++j) {
            if (j < w) {
                di += __ldg(W32 + (size_t)j * ld + i) * dh[j];
                ai += __ldg(AW32 + (size_t)j * ld + i) * dh[j];
            }
        }
        d32[i] = di;
        r32[i] -= ai;
    }
}

__global__ void __launch_bounds__(kBlock) k_mx_accum(int n, double* __restrict__ x, const float* __restrict__ d32,
                                                     const DevState* st)
{
    if (st->outer_done) return;
    const double scale = st->rnorm > 0.0 ? st->rnorm : 1.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] += scale * double(d32[i]);
}

// W32[:, j] = sum_k S32[:, k] C[k][j] (C row stride kWMax, FP64 coefficients used in FP32),
// j < st->pod_w, or j < st->pod_y when cols_y (the augmenting basis Y).
template <int SB>
__global__ void __launch_bounds__(kBlock) k_lift32(int n, const float* __restrict__ S, int lds, int s,
                                                   const double* __restrict__ C, const DevState* st,
                                                   float* __restrict__ W, int ldw, int cols_y)
{
    __shared__ float sC[SB * kWMax];
    const int w = cols_y ? st->pod_y : st->pod_w;
    for (int e = threadIdx.x; e < s * kWMax; e += blockDim.x) sC[e] = float(C[e]);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float sv[SB];
#pragma unroll
        for (int k = 0; k < SB; ++k) sv[k] = (k < s) ? __ldg(S + (size_t)k * lds + i) : 0.0f;
        for (int j = 0; j < w; ++j) {
            float t = 0.0f;
#pragma unroll
            for (int k = 0; k < SB; ++k)
                if (k < s) t += sv[k] * sC[k * kWMax + j];
            W[(size_t)j * ldw + i] = t;
        }
    }
}

cudaError_t launch_lift32(int n, const float* S, int lds, int s, const double* C, const DevState* st, float* W,
                          int ldw, int sms, cudaStream_t str, int cols_y)
{
    const int grid = grid_rows(n, kBlock, sms);
    if (s <= 8) k_lift32<8><<<grid, kBlock, 0, str>>>(n, S, lds, s, C, st, W, ldw, cols_y);
    else if (s <= 16) k_lift32<16><<<grid, kBlock, 0, str>>>(n, S, lds, s, C, st, W, ldw, cols_y);
    else if (s <= 32) k_lift32<32><<<grid, kBlock, 0, str>>>(n, S, lds, s, C, st, W, ldw, cols_y);
    else if (s <= 48) k_lift32<48><<<grid, kBlock, 0, str>>>(n, S, lds, s, C, st, W, ldw, cols_y);
    else k_lift32<64><<<grid, kBlock, 0, str>>>(n, S, lds, s, C, st, W, ldw, cols_y);
    return cudaGetLastError();
}

// Mixed-mode stage-one lift: x = W32 what (FP32 products, stored FP64; the FP64
// refinement corrects its rounding), ||b||^2 and the tolerances.
template <int WB>
__global__ void __launch_bounds__(kBlock) k_stage1_mx(const ProbDesc* __restrict__ pd, const float* __restrict__ W32,
                                                      double* __restrict__ x, double* __restrict__ partials,
                                                      unsigned int* counter, DevState* st, double tol)
{
    const int n = pd->n, ld = pd->ld;
    const int w = st->w;
    const double* b = pd->b;
    __shared__ float s_what[WB > 0 ? WB : 1];
    for (int j = threadIdx.x; j < WB; j += blockDim.x) s_what[j] = (j < w) ? float(st->what[j]) : 0.0f;
    __syncthreads();
    double bb = 0.0;
    float wh[WB > 0 ? WB : 1];
#pragma unroll
    for (int j = 0; j < WB; ++j) wh[j] = (WB > 0) ? s_what[j] : 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float xi = 0.0f;
#pragma unroll
        for (int j = 0; j < WB; ++j)
            if (j < w) xi += __ldg(W32 + (size_t)j * ld + i) * wh[j];
        x[i] = double(xi);
        const double bi = b[i];
        bb += bi * bi;
    }
    double acc[1] = {bb};
    __shared__ double tot[1];
    if (reduce_to_last_block<1>(acc, 1, partials, counter, tot) && threadIdx.x == 0) {
        st->bb = tot[0];
        st->tol2 = tol * tol * tot[0];
        st->tol2_in = st->tol2;
        st->rr_stage1 = -1.0;   // filled by the first outer residual
    }
}

cudaError_t launch_stage1_mx(int wb, const ProbDesc* pd, int n, const float* W32, double* x, double* partials,
                             unsigned int* counter, DevState* st, double tol, int sms, cudaStream_t s)
{
    const int grid = grid_rows(n, kBlock, sms);
    if (wb <= 0) k_stage1_mx<0><<<grid, kBlock, 0, s>>>(pd, W32, x, partials, counter, st, tol);
    else if (wb <= 8) k_stage1_mx<8><<<grid, kBlock, 0, s>>>(pd, W32, x, partials, counter, st, tol);
    else if (wb <= 16) k_stage1_mx<16><<<grid, kBlock, 0, s>>>(pd, W32, x, partials, counter, st, tol);
    else if (wb <= 32) k_stage1_mx<32><<<grid, kBlock, 0, s>>>(pd, W32, x, partials, counter, st, tol);
    else if (wb <= 48) k_stage1_mx<48><<<grid, kBlock, 0, s>>>(pd, W32, x, partials, counter, st, tol);
    else k_stage1_mx<64><<<grid, kBlock, 0, s>>>(pd, W32, x, partials, counter, st, tol);
    return cudaGetLastError();
}

// Gram partials of FP32 blocks: FP32 products summed in FP32 over 32 consecutive rows of
// a thread, then in FP64. Same tiling and output layout as the FP64 Gram.
constexpr int kTile32 = 8;
__global__ void __launch_bounds__(kBlock) k_gram_partial32(int n, const float* __restrict__ X, int ldx, int p,
                                                           const float* __restrict__ Y, int ldy, int qy,
                                                           const double* __restrict__ extra, int q, int tiles_j,
                                                           int upper_only, int rows_per_split,
                                                           double* __restrict__ partials)
{
    const int tile = blockIdx.x;
    const int ti = tile / tiles_j, tj = tile % tiles_j;
    const int split = blockIdx.y;
    const int a0 = ti * kTile32, c0 = tj * kTile32;
    double* out = partials + ((size_t)split * gridDim.x + tile) * (kTile32 * kTile32);
    const bool skip = upper_only && (c0 + kTile32 <= a0) && !(extra && c0 + kTile32 > qy);
    double acc[kTile32 * kTile32];
#pragma unroll
    for (int e = 0; e < kTile32 * kTile32; ++e) acc[e] = 0.0;
    if (!skip) {
        const float* xp[kTile32];
        const float* yp[kTile32];
        bool yextra[kTile32];
#pragma unroll
        for (int a = 0; a < kTile32; ++a) xp[a] = (a0 + a < p) ? X + (size_t)(a0 + a) * ldx : nullptr;
#pragma unroll
        for (int c = 0; c < kTile32; ++c) {
            const int cc = c0 + c;
            yp[c] = (cc < qy) ? Y + (size_t)cc * ldy : nullptr;
            yextra[c] = (extra && cc == qy && cc < q);
        }
        const int r0 = split * rows_per_split;
        const int r1 = min(n, r0 + rows_per_split);
        float part[kTile32 * kTile32];
#pragma unroll
        for (int e = 0; e < kTile32 * kTile32; ++e) part[e] = 0.0f;
        int cnt = 0;
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            float xv[kTile32], yv[kTile32];
#pragma unroll
            for (int a = 0; a < kTile32; ++a) xv[a] = xp[a] ? __ldg(xp[a] + i) : 0.0f;
#pragma unroll
            for (int c = 0; c < kTile32; ++c)
                yv[c] = yp[c] ? __ldg(yp[c] + i) : (yextra[c] ? float(extra[i]) : 0.0f);
#pragma unroll
            for (int a = 0; a < kTile32; ++a)
#pragma unroll
                for (int c = 0; c < kTile32; ++c) part[a * kTile32 + c] += xv[a] * yv[c];
            if (++cnt == 32) {
#pragma unroll
                for (int e = 0; e < kTile32 * kTile32; ++e) {
                    acc[e] += double(part[e]);
                    part[e] = 0.0f;
                }
                cnt = 0;
            }
        }
#pragma unroll
        for (int e = 0; e < kTile32 * kTile32; ++e) acc[e] += double(part[e]);
    }
    __shared__ double s_w[kWarps][kTile32 * kTile32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < kTile32 * kTile32; ++e) {
        const double t = warp_sum(acc[e]);
        if (lane == 0) s_w[wid][e] = t;
    }
    __syncthreads();
    if (threadIdx.x < kTile32 * kTile32) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) t += s_w[k][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

cudaError_t launch_gram32(int n, const float* X, int ldx, int p, const float* Y, int ldy, int qy, const double* extra,
                          double* G, int ldg, int upper_only, double* work, size_t work_bytes, int sms,
                          cudaStream_t s)
{
    const int q = qy + (extra ? 1 : 0);
    if (p <= 0 || q <= 0) return cudaSuccess;
    int tj, tiles, splits, rps;
    gram_shape(n, p, q, sms, &tj, &tiles, &splits, &rps);
    if ((size_t)splits * tiles * kTile32 * kTile32 * sizeof(double) > work_bytes) return cudaErrorInvalidValue;
    dim3 grid(tiles, splits);
    k_gram_partial32<<<grid, kBlock, 0, s>>>(n, X, ldx, p, Y, ldy, qy, extra, q, tj, upper_only, rps, work);
    return launch_gram_reduce(work, splits, tiles, tj, p, q, G, ldg, s);
}

void mixed_kernels(int wb, void** proj, void** start)
{
#define PODCG_MX(WW) *proj = (void*)k_mx_proj<WW>; *start = (void*)k_mx_start<WW>;
    if (wb <= 0) { PODCG_MX(0) }
    else if (wb <= 8) { PODCG_MX(8) }
    else if (wb <= 16) { PODCG_MX(16) }
    else if (wb <= 32) { PODCG_MX(32) }
    else if (wb <= 48) { PODCG_MX(48) }
    else { PODCG_MX(64) }
#undef PODCG_MX
}

void* kernel_mx_accum() { return (void*)k_mx_accum; }

}  // namespace podcg
