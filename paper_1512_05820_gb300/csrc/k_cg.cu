// Kernels of the augmented PCG iteration (Section 2.2, Algorithm 1 with Y = W and
// M = diag(A)), in FP64 or FP32 (T), for a basis of at most WB columns (w <= WB read from
// the device state so one captured graph serves every w of its bucket).
//
// One iteration is three launches:
//   k_spmv_cg : q = A p, gamma = (q, p), alpha = (r, z)/gamma            (k_sparse.cu)
//   k_update  : r -= alpha q, z = M^{-1} r, (r, z), ||r||^2, c = (A W)^T z;
//               last block: beta, iteration count, exit test -> graph condition
//   k_dir     : mu = R^{-1} R^{-T} c (every block, from the stage-one factor reused as in
//               Section 4.3), x += alpha p, p = z + beta p - W mu (z recomputed from r)
// (A W)^T z equals the paper's W^T A z because A is symmetric.
//
// The same kernels run inside a conditional while-graph (the loop stops on the device)
// or inside a plain graph of several unrolled iterations whose later launches return
// immediately: k_spmv_cg and k_update skip once `done` is set, and k_dir runs only when
// the k_update of its iteration did (`dir_pending`). COND = false compiles the variants
// with no graph-condition call at all, for plain graphs and direct launches.
#include "common.cuh"
#include "launch.h"

namespace podcg {

// mu = R^{-1} (R^{-T} c) in shared memory: s_R holds R^{-1} (row stride WB), s_c holds c.
template <int WB>
__device__ __forceinline__ void block_mu(const double* __restrict__ Rinv, const double* __restrict__ c, int w,
                                         double* s_R, double* s_c, double* s_t, double* s_mu)
{
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        const int i = e / w, j = e % w;
        s_R[i * WB + j] = Rinv[i * kWMax + j];
    }
    for (int a = threadIdx.x; a < w; a += blockDim.x) s_c[a] = c[a];
    __syncthreads();
    for (int a = threadIdx.x; a < w; a += blockDim.x) {
        double v = 0.0;
        for (int k = 0; k <= a; ++k) v += s_R[k * WB + a] * s_c[k];
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

// Start of a CG pass from the residual r: z0 = M^{-1} r, (r, z0), ||r||^2, c = (A W)^T z0;
// the residual test on r0 (zero iterations allowed). mu0 is formed by k_dir<FIRST>.
// Same column-parallel tiling as k_update.
template <int WB, typename T, bool COND>
__global__ void __launch_bounds__(kBlock) k_init(int n, int ld, const T* __restrict__ r, const T* __restrict__ dinv,
                                                 const T* __restrict__ AW, double* __restrict__ partials,
                                                 unsigned int* counter, DevState* st,
                                                 cudaGraphConditionalHandle h_inner, int use_cond)
{
    constexpr int CPW = WB > 0 ? (WB + kWarps - 1) / kWarps : 1;
    const int w = st->w;
    __shared__ T s_z[kBlock];
    __shared__ double s_blk[WB + 2];
    T cacc[CPW];
#pragma unroll
    for (int k = 0; k < CPW; ++k) cacc[k] = T(0);
    T rho = T(0), rr = T(0);
    const bool skip = st->outer_done != 0;   // mixed precision: the outer loop already stopped
    if (!skip) {
        for (int row0 = blockIdx.x * kBlock; row0 < n; row0 += gridDim.x * kBlock) {
            const int i = row0 + threadIdx.x;
            T zi = T(0);
            if (i < n) {
                const T ri = r[i];
                zi = dinv[i] * ri;
                rho += ri * zi;
                rr += ri * ri;
            }
            if (WB > 0) {
                s_z[threadIdx.x] = zi;
                __syncthreads();
                tile_columns<CPW, T>(AW, ld, w, row0, n, s_z, cacc);
                __syncthreads();
            }
        }
    }
    block_totals<CPW, T>(rho, rr, cacc, w, s_blk);
    __shared__ double tot[WB + 2];
    if (partials_to_last_block(s_blk, 2 + w, partials, counter, tot)) {
        for (int a = threadIdx.x; a < w; a += blockDim.x) st->c[a] = tot[2 + a];
        if (threadIdx.x == 0) {
            st->rho = tot[0];
            st->rr = tot[1];
            st->alpha = 0.0;
            st->beta = 0.0;
            if (st->status == 0 && !(isfinite(tot[0]) && isfinite(tot[1]))) st->status = 5;
            const int done = skip || (st->status != 0) || !(tot[1] > st->tol2_in);
            st->done = done;
            st->dir_pending = 0;
            st->inner_iters = 0;
            st->inner_break = 0;
            if constexpr (COND) {
                if (use_cond) cudaGraphSetConditional(h_inner, done ? 0u : 1u);
            }
        }
    }
}

// Update pass, column-parallel projection: each 256-row tile computes r, z, (r, z) and
// ||r||^2 row-wise, stages z in shared memory, then every warp accumulates (A W)^T z for
// its own columns (j = warp, warp + 8, ...) with coalesced reads of A W. A thread holds at
// most WB/8 column accumulators (32-40 registers), so the kernel stays at high occupancy.
// (A one-row-per-thread form with w accumulators per thread measured no faster in FP32
// and half as fast in FP64 at 96 registers.)
template <int WB, typename T, bool COND>
__global__ void __launch_bounds__(kBlock) k_update(int n, int ld, T* __restrict__ r, const T* __restrict__ q,
                                                   const T* __restrict__ dinv, const T* __restrict__ AW,
                                                   double* __restrict__ partials, unsigned int* counter,
                                                   DevState* st, cudaGraphConditionalHandle h_inner, int use_cond)
{
    if (st->done) return;   // uniform: only this kernel's last block writes `done`
    constexpr int CPW = WB > 0 ? (WB + kWarps - 1) / kWarps : 1;
    const int w = st->w;
    const T alpha = (st->status == 0) ? T(st->alpha) : T(0);
    __shared__ T s_z[kBlock];
    __shared__ double s_blk[WB + 2];
    T cacc[CPW];
#pragma unroll
    for (int k = 0; k < CPW; ++k) cacc[k] = T(0);
    T rho = T(0), rr = T(0);
    for (int row0 = blockIdx.x * kBlock; row0 < n; row0 += gridDim.x * kBlock) {
        const int i = row0 + threadIdx.x;
        T zi = T(0);
        if (i < n) {
            const T ri = r[i] - alpha * q[i];
            r[i] = ri;
            zi = dinv[i] * ri;
            rho += ri * zi;
            rr += ri * ri;
        }
        if (WB > 0) {
            s_z[threadIdx.x] = zi;
            __syncthreads();
            tile_columns<CPW, T>(AW, ld, w, row0, n, s_z, cacc);
            __syncthreads();
        }
    }
    block_totals<CPW, T>(rho, rr, cacc, w, s_blk);
    __shared__ double tot[WB + 2];
    if (partials_to_last_block(s_blk, 2 + w, partials, counter, tot)) {
        for (int a = threadIdx.x; a < w; a += blockDim.x) st->c[a] = tot[2 + a];
        if (threadIdx.x == 0) {
            const double rho_new = tot[0];
            st->beta = rho_new / st->rho;
            st->rho = rho_new;
            st->rr = tot[1];
            st->iters += 1;
            st->inner_iters += 1;
            if (st->status == 0 && !(isfinite(rho_new) && isfinite(tot[1]))) {
                if (st->mixed) st->inner_break = 1;
                else st->status = 5;
            }
            int done = (st->status != 0) || st->inner_break || !(tot[1] > st->tol2_in);
            if (!done && st->iters >= st->k_max) {
                st->status = 4;
                done = 1;
            }
            st->done = done;
            st->dir_pending = 1;
            if constexpr (COND) {
                if (use_cond) cudaGraphSetConditional(h_inner, done ? 0u : 1u);
            }
        }
    }
}

// mu = R^{-1} R^{-T} c; x += alpha p; then (unless the pass has finished)
// p = z + beta p - W mu with z = M^{-1} r. FIRST: p0 = z0 - W mu0, x untouched.
template <int WB, typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock) k_dir(int n, int ld, T* __restrict__ x, T* __restrict__ p,
                                                const T* __restrict__ r, const T* __restrict__ dinv,
                                                const T* __restrict__ W, const double* __restrict__ Rinv,
                                                const DevState* st)
{
    if (!FIRST && !st->dir_pending) return;
    if (FIRST && st->outer_done) return;
    const int w = st->w;
    const bool ok = st->status == 0 && !st->inner_break;
    const T alpha = ok ? T(st->alpha) : T(0);
    const T beta = T(st->beta);
    const bool upd_p = FIRST || (!st->done && ok);
    __shared__ double s_R[WB > 0 ? WB * WB : 1];
    __shared__ double s_c[WB > 0 ? WB : 1], s_t[WB > 0 ? WB : 1], s_mud[WB > 0 ? WB : 1];
    __shared__ T s_mu[WB > 0 ? WB : 1];
    if (WB > 0 && upd_p) {
        block_mu<WB>(Rinv, st->c, w, s_R, s_c, s_t, s_mud);
        for (int j = threadIdx.x; j < WB; j += blockDim.x) s_mu[j] = (j < w) ? T(s_mud[j]) : T(0);
        __syncthreads();
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const T pi = p[i];
        if (!FIRST) x[i] += alpha * pi;
        if (upd_p) {
            T v = dinv[i] * r[i];
            if (!FIRST) v += beta * pi;
#pragma unroll
            for (int j = 0; j < WB; ++j)
                if (j < w) v -= __ldg(W + (size_t)j * ld + i) * s_mu[j];
            p[i] = v;
        }
    }
}

// ------------------------------------------------------------------ kernel pointers

template <typename T, bool COND>
static void pick(int wb, void** init, void** upd, void** dir0, void** dir)
{
#define PODCG_PICK(WW)                                   \
    *init = (void*)k_init<WW, T, COND>;                  \
    *upd = (void*)k_update<WW, T, COND>;                 \
    *dir0 = (void*)k_dir<WW, T, true>;                   \
    *dir = (void*)k_dir<WW, T, false>;
    if (wb <= 0) { PODCG_PICK(0) }
    else if (wb <= 8) { PODCG_PICK(8) }
    else if (wb <= 16) { PODCG_PICK(16) }
    else if (wb <= 32) { PODCG_PICK(32) }
    else if (wb <= 48) { PODCG_PICK(48) }
    else { PODCG_PICK(64) }
#undef PODCG_PICK
}

void cg_kernels(int wb, bool fp32, bool cond, void** init, void** upd, void** dir0, void** dir)
{
    if (fp32) {
        if (cond) pick<float, true>(wb, init, upd, dir0, dir);
        else pick<float, false>(wb, init, upd, dir0, dir);
    } else {
        if (cond) pick<double, true>(wb, init, upd, dir0, dir);
        else pick<double, false>(wb, init, upd, dir0, dir);
    }
}

int wb_bucket(int w)
{
    if (w <= 0) return 0;
    if (w <= 8) return 8;
    if (w <= 16) return 16;
    if (w <= 32) return 32;
    if (w <= 48) return 48;
    return 64;
}

}  // namespace podcg
