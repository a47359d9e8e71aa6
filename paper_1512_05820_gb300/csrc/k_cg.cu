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
#include <cuda.h>
#include <cuda_fp16.h>

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
            int done = skip || (st->status != 0) || !(tot[1] > st->tol2_in);
            if (!done && st->iters >= st->k_max) {   // the cap is checked before an iteration
                st->status = 4;
                done = 1;
            }
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

// Block totals of an update pass, the deterministic cross-block sum, and (last block)
// beta, the iteration count, the exit test and the graph condition.
template <int WB, bool COND>
__device__ __forceinline__ void update_finish(const double* s_blk, int w, double* __restrict__ partials,
                                              unsigned int* counter, DevState* st,
                                              cudaGraphConditionalHandle h_inner, int use_cond)
{
    __shared__ double tot[WB + 2];
    if (partials_to_last_block(s_blk, 2 + w, partials, counter, tot)) {
        for (int a = threadIdx.x; a < w; a += blockDim.x) st->c[a] = tot[2 + a];
        if (threadIdx.x == 0) {
            // read every state field first (independent loads, one round of latency)
            const double rho_old = st->rho, tol2_in = st->tol2_in;
            const int iters = st->iters + 1, inner_iters = st->inner_iters + 1, k_max = st->k_max;
            int status = st->status, inner_break = st->inner_break;
            const int mixed = st->mixed;
            const double rho_new = tot[0];
            if (status == 0 && !(isfinite(rho_new) && isfinite(tot[1]))) {
                if (mixed) inner_break = 1;
                else status = 5;
            }
            int done = (status != 0) || inner_break || !(tot[1] > tol2_in);
            if (!done && iters >= k_max) {
                status = 4;
                done = 1;
            }
            st->beta = rho_new / rho_old;
            st->rho = rho_new;
            st->rr = tot[1];
            st->iters = iters;
            st->inner_iters = inner_iters;
            st->status = status;
            st->inner_break = inner_break;
            st->done = done;
            st->dir_pending = 1;
            if constexpr (COND) {
                if (use_cond) cudaGraphSetConditional(h_inner, done ? 0u : 1u);
            }
        }
    }
}

template <int WB, typename T, bool COND, int CPW>
__device__ __forceinline__ void update_tail(T rho, T rr, const T (&cacc)[CPW], int w, double* s_blk,
                                            double* __restrict__ partials, unsigned int* counter, DevState* st,
                                            cudaGraphConditionalHandle h_inner, int use_cond)
{
    block_totals<CPW, T>(rho, rr, cacc, w, s_blk);
    update_finish<WB, COND>(s_blk, w, partials, counter, st, h_inner, use_cond);
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
    pdl_wait_then_release();
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
    update_tail<WB, T, COND>(rho, rr, cacc, w, s_blk, partials, counter, st, h_inner, use_cond);
}

// mu = R^{-1} R^{-T} c; x += alpha p; then (unless the pass has finished)
// p = z + beta p - W mu with z = M^{-1} r. FIRST: p0 = z0 - W mu0, x untouched.
template <int WB, typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock) k_dir(int n, int ld, T* __restrict__ x, T* __restrict__ p,
                                                const T* __restrict__ r, const T* __restrict__ dinv,
                                                const T* __restrict__ W, const double* __restrict__ Rinv,
                                                const DevState* st)
{
    pdl_wait_then_release();
    if (!FIRST && !st->dir_pending) return;
    if (FIRST && st->outer_done) return;
    const int w = st->w;
    // the step of the iteration that reached the cap (status 4) is valid and is applied
    const bool ok = (st->status == 0 || st->status == 4) && !st->inner_break;
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

// ------------------------------------------------------------------ FP32 loop, TMA-staged
//
// The second FP32 form of the update and direction passes (proj_form = 1). Every CTA
// takes every gridDim-th 256-row tile. One producer lane streams every tile into a
// ring of shared-memory stages: the basis panel (A W for the update, W for the direction)
// as 2D tensor copies (cp.async.bulk.tensor) of 256 rows x 8 FP32 columns, or 256 rows x
// 16 fp16 columns for the direction pass's 16-bit W, and the per-row vectors as 1 KB bulk
// copies (cp.async.bulk), all completing on the stage's `full` mbarrier. The panels' tensor
// maps span exactly the basis width in use, so the columns of a last, partial box past it
// are filled with zeros by the copy engine and cost no memory traffic. Eight consumer
// warps compute from shared memory and release a stage through its `empty` mbarrier (one
// arrival per warp): no block-wide barrier sits in the loop, and the reads in flight do not
// depend on the consumers' register count. A probe streaming the same copies (a 22-column
// panel, three vectors, one vector written back) reached 6.1 TB/s with 130-190 KB in
// flight per SM and less with more (5.8 TB/s at 200 KB in one CTA). The update pass runs
// one CTA per SM with a 160 KB ring (its partials feed every block of the direction pass,
// so fewer CTAs make that pass's prologue shorter); the direction pass two CTAs per SM with
// 88 KB rings when a stage is at most 40 KB, else one with 160 KB (tma_shape).
//
// Every copy stays inside its buffer: vectors and panels are allocated with the padded
// leading dimension ld (a multiple of 32 >= n), a vector copy spans min(256, ld - row0)
// rows, and the tensor maps' row extent is ld (rows past it are filled with zeros). Rows
// >= n inside a tile are never used. Every mbarrier wait is bounded (4e9 SM clocks, about
// 2 s); on expiry the warp records status 7 (timeout) and leaves its loop, the producer
// waits (bounded) for the copies it issued, and the pass ends with that status.

constexpr long long kBulkWaitCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr int kTmTile = 256;                           // rows per tile
constexpr int kTmBoxBytes = 8192;                      // panel box: 256 x 8 FP32 or 256 x 16 fp16
constexpr int kTmVecBytes = kTmTile * 4;               // one FP32 vector tile
constexpr int kTmRingMax = 160 * 1024;                 // ring bytes of a CTA alone on its SM
constexpr int kTmRingPair = 88 * 1024;                 // ring bytes of each of two CTAs per SM
constexpr int kTmMaxStages = 16;
constexpr int kTmConsumers = 8;                        // consumer warps (one row per thread)
constexpr int kTmThreads = 32 * (kTmConsumers + 1);    // + the producer warp
constexpr int kTmSmemMax = kTmRingMax + 1024;          // + alignment slack of the ring base

__device__ __forceinline__ uint32_t bulk_smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tensor_copy_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ bool bulk_try(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait of `budget` SM clocks: the clock is read only once the first try fails.
__device__ __forceinline__ bool bulk_wait(uint32_t mbar, uint32_t parity, long long budget)
{
    if (bulk_try(mbar, parity)) return true;
    const long long c0 = clock64();
    while (!bulk_try(mbar, parity))
        if (clock64() - c0 > budget) return false;
    return true;
}

// The wait override of pod_cg_debug_wait_timeout for the staged passes (zero: normal).
static __device__ WaitTest g_cg_wait_test;

// The ring of one CTA: its tiles, the run-time stage size and count, and the waits.
// Stage layout: nbox panel boxes of 8 KB, then NV vector tiles of 1 KB (1024-aligned).
template <int NV>
struct TmaRing {
    unsigned char* base;
    uint64_t* full;
    uint64_t* empty;
    int t0, nloc, S, nbox, cols_per_box, vec_off, stage_bytes;
    long long budget;   // SM clocks a wait may take
    bool starve;        // test of the timeout path: no copy is ever issued

    __device__ void init(unsigned char* raw, uint64_t* f, uint64_t* e, int n, int ncols, int cpb, int ring_bytes)
    {
        const WaitTest wt = g_cg_wait_test;
        starve = (wt.mask & kWaitTestStaged) != 0;
        budget = starve ? wt.cycles : kBulkWaitCycles;
        base = raw + ((1024u - (bulk_smem_u32(raw) & 1023u)) & 1023u);
        full = f;
        empty = e;
        cols_per_box = cpb;
        nbox = (ncols + cpb - 1) / cpb;
        vec_off = nbox * kTmBoxBytes;
        stage_bytes = vec_off + NV * kTmVecBytes;
        S = max(1, min(kTmMaxStages, ring_bytes / stage_bytes));
        // tiles interleaved over the CTAs (tile blockIdx.x + k gridDim.x): at any moment the
        // CTAs read neighbouring tiles, so every column is read in long sequential runs
        const int ntiles = (n + kTmTile - 1) / kTmTile;
        t0 = blockIdx.x;
        nloc = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        if (threadIdx.x == 0) {
            for (int i = 0; i < S; ++i) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bulk_smem_u32(&full[i])));
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bulk_smem_u32(&empty[i])),
                             "r"(kTmConsumers));
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    __device__ unsigned char* stage(int t) const { return base + (t % S) * stage_bytes; }
    __device__ int row0(int t) const { return (t0 + t * (int)gridDim.x) * kTmTile; }

    // Producer lane: stream every local tile (waiting for its stage to be released), then
    // wait (bounded) until every copy issued has landed, so none is in flight at exit. The
    // tensor map lives in global memory (rewritten by the host when the basis width
    // changes), so the tensor-map proxy acquires it first.
    __device__ void produce(int ld, const CUtensorMap* tm, const float* const* vec)
    {
        if (starve) return;
        if (nbox > 0) asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm) : "memory");
        int t = 0;
        for (; t < nloc; ++t) {
            const int s = t % S;
            if (t >= S && !bulk_wait(bulk_smem_u32(&empty[s]), (uint32_t)((t / S - 1) & 1), budget)) break;
            const int r0 = row0(t);
            const uint32_t vbytes = (uint32_t)min(kTmTile, ld - r0) * 4u;
            unsigned char* sg = stage(t);
            const uint32_t mb = bulk_smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                         "r"((uint32_t)(nbox * kTmBoxBytes) + (uint32_t)NV * vbytes)
                         : "memory");
            for (int b = 0; b < nbox; ++b) tensor_copy_2d(bulk_smem_u32(sg + b * kTmBoxBytes), tm, r0, b * cols_per_box, mb);
#pragma unroll
            for (int v = 0; v < NV; ++v) bulk_copy(bulk_smem_u32(sg + vec_off + v * kTmVecBytes), vec[v] + r0, vbytes, mb);
        }
        for (int u = t > S ? t - S : 0; u < t; ++u) bulk_wait(bulk_smem_u32(&full[u % S]), (uint32_t)((u / S) & 1), budget);
    }
    // consumer warp: wait for tile t (every lane), false after a timeout (warp-uniform)
    __device__ bool acquire(int t) const
    {
        const bool ok = bulk_wait(bulk_smem_u32(&full[t % S]), (uint32_t)((t / S) & 1), budget);
        return __all_sync(0xffffffffu, ok);
    }
    __device__ void release(int t) const
    {
        __syncwarp();
        if ((threadIdx.x & 31) == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bulk_smem_u32(&empty[t % S])) : "memory");
    }
};

__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

// Update pass: r -= alpha q, z = M^{-1} r, (r, z), ||r||^2, c = (A W)^T z. Consumer warp cw
// takes rows 32 cw + lane for the row part and basis columns cw, cw + 8, ... for the
// column part, whose lanes cover the tile's 256 rows as two float4 groups each (z is
// formed again from the staged r, q, M^{-1} by every warp, so no warp waits for another).
template <int WB>
__global__ void __launch_bounds__(kTmThreads, 2) k_update_tma(int n, int ld, int ring_bytes, float* __restrict__ r,
                                                              const float* __restrict__ q,
                                                              const float* __restrict__ dinv,
                                                              const CUtensorMap* __restrict__ tmAW,
                                                              double* __restrict__ partials, int g_spmv,
                                                              DevState* st)
{
    pdl_wait_then_release();
    if (st->done) return;   // uniform: `done` is written by k_init / the direction pass only
    constexpr int CPW = (WB + kTmConsumers - 1) / kTmConsumers;
    extern __shared__ __align__(1024) unsigned char tm_raw[];
    __shared__ uint64_t full[kTmMaxStages], empty[kTmMaxStages];
    __shared__ float s_red[kTmConsumers][2];
    __shared__ double s_blk[WB + 2];
    const int w = st->w;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    TmaRing<3> ring;
    ring.init(tm_raw, full, empty, n, w, 8, ring_bytes);
    float acc[CPW];
#pragma unroll
    for (int k = 0; k < CPW; ++k) acc[k] = 0.0f;
    float rho = 0.0f, rr = 0.0f;
    bool timeout = false;
    if (warp == kTmConsumers) {
        if (lane == 0) {
            const float* const vec[3] = {r, q, dinv};
            ring.produce(ld, tmAW, vec);
        }
    } else {
        // alpha from the SpMV's partials while the producer already streams (consumers only)
        const float alpha = float(chain_alpha(st, partials, g_spmv));
        for (int t = 0; t < ring.nloc; ++t) {
            if (!ring.acquire(t)) {
                timeout = true;
                break;
            }
            const unsigned char* sg = ring.stage(t);
            const float* sP = reinterpret_cast<const float*>(sg);
            const float* sr = reinterpret_cast<const float*>(sg + ring.vec_off);
            const float* sq = sr + kTmTile;
            const float* sd = sq + kTmTile;
            const int row0 = ring.row0(t);
            const int valid = min(kTmTile, n - row0);
            {
                const int i = 32 * warp + lane;
                if (i < valid) {
                    const float ri = sr[i] - alpha * sq[i];
                    r[row0 + i] = ri;
                    const float zi = sd[i] * ri;
                    rho += ri * zi;
                    rr += ri * ri;
                }
            }
            if (valid == kTmTile) {
                float4 z4[2];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const float4 a = reinterpret_cast<const float4*>(sr)[lane + 32 * m];
                    const float4 b = reinterpret_cast<const float4*>(sq)[lane + 32 * m];
                    const float4 d = reinterpret_cast<const float4*>(sd)[lane + 32 * m];
                    z4[m] = make_float4(d.x * (a.x - alpha * b.x), d.y * (a.y - alpha * b.y),
                                        d.z * (a.z - alpha * b.z), d.w * (a.w - alpha * b.w));
                }
#pragma unroll
                for (int k = 0; k < CPW; ++k) {
                    const int j = warp + kTmConsumers * k;
                    if (j < w) {
                        const float4* col = reinterpret_cast<const float4*>(sP + (j >> 3) * 2048 + (j & 7) * kTmTile);
                        acc[k] += dot4(col[lane], z4[0]) + dot4(col[lane + 32], z4[1]);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < CPW; ++k) {
                    const int j = warp + kTmConsumers * k;
                    if (j < w) {
                        const float* col = sP + (j >> 3) * 2048 + (j & 7) * kTmTile;
                        float a = 0.0f;
                        for (int m = 0; m < kTmTile / 32; ++m) {
                            const int i = lane + 32 * m;
                            if (i < valid) a += col[i] * (sd[i] * (sr[i] - alpha * sq[i]));
                        }
                        acc[k] += a;
                    }
                }
            }
            ring.release(t);
        }
    }
    if (timeout && lane == 0) atomicExch(&st->status, 7);
    if (warp < kTmConsumers) {
        rho = warp_sum(rho);
        rr = warp_sum(rr);
#pragma unroll
        for (int k = 0; k < CPW; ++k) {
            const int j = warp + kTmConsumers * k;
            const float t = warp_sum(acc[k]);
            if (lane == 0 && j < w) s_blk[2 + j] = (double)t;
        }
        if (lane == 0) {
            s_red[warp][0] = rho;
            s_red[warp][1] = rr;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int k = 0; k < kTmConsumers; ++k) {
            t0 += (double)s_red[k][0];
            t1 += (double)s_red[k][1];
        }
        s_blk[0] = t0;
        s_blk[1] = t1;
    }
    __syncthreads();
    chain_store(s_blk, w + 2, partials);
}

// Direction pass: mu = R^{-1} R^{-T} c, x += alpha p, p = z + beta p - W mu (FIRST: p0 =
// z0 - W mu0 from st->c, x untouched), one row per consumer thread; otherwise the update
// pass's totals come from its partials (chain_direction, with COND the graph condition).
// H: W is the 16-bit copy W16 with one power-of-two scale per column (W32 = W16 * wscale
// exactly), folded into mu.
template <int WB, bool FIRST, bool H, bool COND>
__global__ void __launch_bounds__(kTmThreads, 2) k_dir_tma(int n, int ld, int ring_bytes, float* __restrict__ x,
                                                           float* __restrict__ p,
                                                           const float* __restrict__ r, const float* __restrict__ dinv,
                                                           const CUtensorMap* __restrict__ tmW,
                                                           const float* __restrict__ wscale,
                                                           const double* __restrict__ Rinv,
                                                           const double* __restrict__ M,
                                                           const double* __restrict__ partials, int g_upd, DevState* st,
                                                           cudaGraphConditionalHandle h_inner, int use_cond)
{
    pdl_wait_then_release();
    if (!FIRST && !st->dir_pending) return;
    if (FIRST && st->outer_done) return;
    constexpr int NV = FIRST ? 3 : 4;
    const int w = st->w;
    extern __shared__ __align__(1024) unsigned char tm_raw[];
    __shared__ uint64_t full[kTmMaxStages], empty[kTmMaxStages];
    __shared__ double s_tot[WB + 2], s_t[WB > 0 ? WB : 1], s_mud[WB > 0 ? WB : 1];
    __shared__ float s_mu[WB > 0 ? WB : 1], s_M[WB > 0 ? WB * WB : 1];
    // the producer streams the whole panel from the start (the loads do not depend on the
    // update pass's totals); a pass that has finished does not use it (its last iteration)
    TmaRing<NV> ring;
    ring.init(tm_raw, full, empty, n, w, H ? 16 : 8, ring_bytes);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool timeout = false;
    if (warp == kTmConsumers) {
        if (lane == 0) {
            const float* vec[NV];
            vec[0] = p;
            vec[1] = r;
            vec[2] = dinv;
            if constexpr (!FIRST) vec[NV - 1] = x;
            ring.produce(ld, tmW, vec);
        }
    } else {
        // consumers only (named barrier): the update pass's totals and decisions, then mu
        float alpha = 0.0f, beta = 0.0f;
        bool upd_p = true;
        if constexpr (!FIRST) {
            const ChainStep cs = chain_direction<WB, COND>(st, partials, g_upd, w, M, s_tot, s_M, s_mud, h_inner,
                                                           use_cond);
            alpha = float(cs.alpha);
            beta = float(cs.beta);
            upd_p = cs.upd_p;
        } else {
            block_mu_global(Rinv, st->c, w, s_t, s_mud);
        }
        if (upd_p) {
            for (int j = threadIdx.x; j < WB; j += kBlock)
                s_mu[j] = (j < w) ? float(s_mud[j]) * (H ? wscale[j] : 1.0f) : 0.0f;
            bar_compute();
        }
        const int wc = upd_p ? w : 0;
        const int i = threadIdx.x;
        for (int t = 0; t < ring.nloc; ++t) {
            if (!ring.acquire(t)) {
                timeout = true;
                break;
            }
            const unsigned char* sg = ring.stage(t);
            const float* sv = reinterpret_cast<const float*>(sg + ring.vec_off);
            const int row0 = ring.row0(t);
            if (row0 + i < n) {
                const float pi = sv[i];
                if constexpr (!FIRST) x[row0 + i] = sv[3 * kTmTile + i] + alpha * pi;
                if (upd_p) {
                    float v = sv[2 * kTmTile + i] * sv[kTmTile + i];
                    if (!FIRST) v += beta * pi;
                    if constexpr (H) {
                        const __half* sW = reinterpret_cast<const __half*>(sg);
#pragma unroll
                        for (int j = 0; j < WB; ++j)
                            if (j < wc) v -= __half2float(sW[(j >> 4) * 4096 + (j & 15) * kTmTile + i]) * s_mu[j];
                    } else {
                        const float* sW = reinterpret_cast<const float*>(sg);
#pragma unroll
                        for (int j = 0; j < WB; ++j)
                            if (j < wc) v -= sW[(j >> 3) * 2048 + (j & 7) * kTmTile + i] * s_mu[j];
                    }
                    p[row0 + i] = v;
                }
            }
            ring.release(t);
        }
    }
    if (timeout && lane == 0) atomicExch(&st->status, 7);
}

// W16 = fp16(W32 / 2^e_j) with 2^e_j the smallest power of two >= max_i |W32[i][j]|, then
// W32 = float(W16) * 2^e_j, which FP32 holds exactly: W32 becomes the 16-bit basis, so
// every use of W32 (stage one, the correction's projection, A W32 formed after this) and
// the direction pass's W16 see the same basis. cmax: per-column maxima as float bit
// patterns (non-negative floats order as unsigned integers, so atomicMax gives a result
// that does not depend on the order); zero on entry.
__global__ void __launch_bounds__(kBlock) k_colmax(int n, int ld, const float* __restrict__ W, const DevState* st,
                                                   unsigned int* cmax)
{
    __shared__ float s_m[kWarps];
    const int w = st->pod_w;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = 0; j < w; ++j) {
        float m = 0.0f;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
            m = fmaxf(m, fabsf(W[(size_t)j * ld + i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_m[wid] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            float b = 0.0f;
            for (int k = 0; k < kWarps; ++k) b = fmaxf(b, s_m[k]);
            atomicMax(cmax + j, __float_as_uint(b));
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) k_quant16(int n, int ld, float* __restrict__ W, __half* __restrict__ W16,
                                                    const unsigned int* __restrict__ cmax, float* __restrict__ wscale,
                                                    const DevState* st)
{
    const int w = st->pod_w;
    for (int j = 0; j < w; ++j) {
        const float m = __uint_as_float(cmax[j]);
        int e = 0;
        if (m > 0.0f && isfinite(m)) frexpf(m, &e);   // m = f 2^e, 0.5 <= f < 1, so m <= 2^e
        const float scale = ldexpf(1.0f, e), inv = ldexpf(1.0f, -e);
        if (blockIdx.x == 0 && threadIdx.x == 0) wscale[j] = scale;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            const __half hv = __float2half_rn(W[(size_t)j * ld + i] * inv);
            W16[(size_t)j * ld + i] = hv;
            W[(size_t)j * ld + i] = __half2float(hv) * scale;
        }
    }
}

cudaError_t launch_quant16(int n, int ld, float* W32, __half* W16, unsigned int* cmax, float* wscale,
                           const DevState* st, int sms, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(cmax, 0, sizeof(unsigned int) * kWMax, s);
    if (e != cudaSuccess) return e;
    const int grid = grid_rows(n, kBlock, sms);
    k_colmax<<<grid, kBlock, 0, s>>>(n, ld, W32, st, cmax);
    k_quant16<<<grid, kBlock, 0, s>>>(n, ld, W32, W16, cmax, wscale, st);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP32 loop, row-parallel float4
//
// The other FP32 form of the update and direction passes: each thread owns groups of four
// consecutive rows (one float4 of every vector and panel column), so a warp streams 512
// contiguous bytes of a column per load. Under full load this GPU's HBM needs about
// 200 KB of reads in flight per SM.
// Direction: one float4 result per row group; W mu is subtracted column by column with a
// low register count (48: 5 blocks of 256 per SM), so many warps keep loads in flight.
// Update: one FP32 accumulator per basis column in registers, panel loads in batches of
// eight independent float4 per thread (two blocks per SM), and one reduction per block
// (warp shuffle tree, then warps in fixed order). (A split of the columns over lane groups,
// to lower the register count, measured slower at every width: every row group then paid
// one more dependent step before its panel loads.)
// Rows past the last full group of four are handled one per thread.

constexpr int kV4Batch = 8;
constexpr int kV4Blocks = 6;   // resident blocks per SM the register budget is set for

template <int WB>
__global__ void __launch_bounds__(kBlock, WB <= 8 ? 4 : 2) k_update_v4(int n, int ld, float* __restrict__ r,
                                                                     const float* __restrict__ q,
                                                                     const float* __restrict__ dinv,
                                                                     const float* __restrict__ AW,
                                                                     double* __restrict__ partials, int g_spmv,
                                                                     DevState* st)
{
    pdl_wait_then_release();
    if (st->done) return;   // uniform: `done` is written by k_init / the direction pass only
    constexpr int NA = WB > 0 ? WB : 1;
    __shared__ float s_red[kWarps][WB + 2];
    __shared__ double s_blk[WB + 2];
    const int w = st->w;
    const float alpha = float(chain_alpha(st, partials, g_spmv));
    float acc[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) acc[j] = 0.0f;
    float rho = 0.0f, rr = 0.0f;
    const int n4 = n >> 2;
    const int stride = gridDim.x * blockDim.x;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += stride) {
        float4 r4 = reinterpret_cast<const float4*>(r)[g];
        const float4 q4 = __ldg(reinterpret_cast<const float4*>(q) + g);
        const float4 d4 = __ldg(reinterpret_cast<const float4*>(dinv) + g);
        r4.x -= alpha * q4.x;
        r4.y -= alpha * q4.y;
        r4.z -= alpha * q4.z;
        r4.w -= alpha * q4.w;
        reinterpret_cast<float4*>(r)[g] = r4;
        const float4 z4 = make_float4(d4.x * r4.x, d4.y * r4.y, d4.z * r4.z, d4.w * r4.w);
        rho += r4.x * z4.x + r4.y * z4.y + r4.z * z4.z + r4.w * z4.w;
        rr += r4.x * r4.x + r4.y * r4.y + r4.z * r4.z + r4.w * r4.w;
#pragma unroll
        for (int jb = 0; jb < WB; jb += kV4Batch) {
            float4 a[kV4Batch];
#pragma unroll
            for (int u = 0; u < kV4Batch; ++u)
                if (jb + u < w) a[u] = __ldg(reinterpret_cast<const float4*>(AW + (size_t)(jb + u) * ld) + g);
#pragma unroll
            for (int u = 0; u < kV4Batch; ++u)
                if (jb + u < w) acc[jb + u] += a[u].x * z4.x + a[u].y * z4.y + a[u].z * z4.z + a[u].w * z4.w;
        }
    }
    for (int i = 4 * n4 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float ri = r[i] - alpha * q[i];
        r[i] = ri;
        const float zi = dinv[i] * ri;
        rho += ri * zi;
        rr += ri * ri;
#pragma unroll
        for (int j = 0; j < WB; ++j)
            if (j < w) acc[j] += AW[(size_t)j * ld + i] * zi;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    rho = warp_sum(rho);
    rr = warp_sum(rr);
#pragma unroll
    for (int j = 0; j < WB; ++j)
        if (j < w) acc[j] = warp_sum(acc[j]);
    if (lane == 0) {
        s_red[wid][0] = rho;
        s_red[wid][1] = rr;
#pragma unroll
        for (int j = 0; j < WB; ++j)
            if (j < w) s_red[wid][2 + j] = acc[j];
    }
    __syncthreads();
    for (int v = threadIdx.x; v < w + 2; v += blockDim.x) {
        double t = 0.0;
        for (int k = 0; k < kWarps; ++k) t += (double)s_red[k][v];
        s_blk[v] = t;
    }
    __syncthreads();
    chain_store(s_blk, w + 2, partials);
}

// FIRST: mu0 from st->c (k_init), p0 = z0 - W mu0, x untouched. Otherwise the update pass's
// totals come from its partials (chain_direction, which also takes the exit decisions and,
// with COND, sets the graph condition), then mu = R^{-1} R^{-T} c, x += alpha p and
// p = z + beta p - W mu.
template <int WB, bool FIRST, bool COND, bool H = false>
__global__ void __launch_bounds__(kBlock, WB <= 8 ? 4 : WB <= 32 ? kV4Blocks - 1 : 4) k_dir_v4(int n, int ld, float* __restrict__ x,
                                                              float* __restrict__ p, const float* __restrict__ r,
                                                              const float* __restrict__ dinv,
                                                              const float* __restrict__ W,
                                                              const __half* __restrict__ W16,
                                                              const float* __restrict__ wscale,
                                                              const double* __restrict__ Rinv,
                                                              const double* __restrict__ M,
                                                              const double* __restrict__ partials, int g_upd,
                                                              DevState* st, cudaGraphConditionalHandle h_inner,
                                                              int use_cond)
{
    pdl_wait_then_release();
    if (!FIRST && !st->dir_pending) return;
    if (FIRST && st->outer_done) return;
    constexpr int NB = WB > 0 ? WB : 1;
    const int w = st->w;
    __shared__ double s_tot[WB + 2];
    __shared__ float s_M[NB * NB];
    __shared__ double s_c[NB], s_t[NB], s_mud[NB];
    __shared__ float s_mu[NB];
    float alpha = 0.0f, beta = 0.0f;
    bool upd_p = true;
    // narrow bases: the thread's first group of p, x, r and M^{-1} is loaded before the
    // prologue (which needs none of them), so its latency hides behind the partials' sums
    constexpr bool kPre = !FIRST && WB <= 8;
    const int g_first = blockIdx.x * blockDim.x + threadIdx.x;
    float4 pre_p = make_float4(0.f, 0.f, 0.f, 0.f), pre_x = pre_p, pre_r = pre_p, pre_d = pre_p;
    if (kPre && g_first < (n >> 2)) {
        pre_p = reinterpret_cast<const float4*>(p)[g_first];
        pre_x = reinterpret_cast<const float4*>(x)[g_first];
        pre_r = __ldg(reinterpret_cast<const float4*>(r) + g_first);
        pre_d = __ldg(reinterpret_cast<const float4*>(dinv) + g_first);
    }
    if constexpr (!FIRST) {
        const ChainStep cs = chain_direction<WB, COND>(st, partials, g_upd, w, M, s_tot, s_M, s_mud, h_inner, use_cond);
        alpha = float(cs.alpha);
        beta = float(cs.beta);
        upd_p = cs.upd_p;
    } else if (WB > 0) {
        block_mu_global(Rinv, st->c, w, s_t, s_mud);
    }
    __shared__ float s_sc[NB];   // H: the 16-bit basis's column scales (W = W16 * scale exactly)
    if (WB > 0 && upd_p) {
        for (int j = threadIdx.x; j < WB; j += blockDim.x) {
            s_mu[j] = (j < w) ? float(s_mud[j]) : 0.0f;
            if (H) s_sc[j] = (j < w) ? wscale[j] : 0.0f;
        }
        __syncthreads();
    }
    const int wc = upd_p ? w : 0;
    const int n4 = n >> 2;
    const int stride = gridDim.x * blockDim.x;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += stride) {
        const bool first = kPre && g == g_first;
        const float4 p4 = first ? pre_p : reinterpret_cast<const float4*>(p)[g];
        if (!FIRST) {
            float4 x4 = first ? pre_x : reinterpret_cast<const float4*>(x)[g];
            x4.x += alpha * p4.x;
            x4.y += alpha * p4.y;
            x4.z += alpha * p4.z;
            x4.w += alpha * p4.w;
            reinterpret_cast<float4*>(x)[g] = x4;
        }
        if (upd_p) {
            const float4 r4 = first ? pre_r : __ldg(reinterpret_cast<const float4*>(r) + g);
            const float4 d4 = first ? pre_d : __ldg(reinterpret_cast<const float4*>(dinv) + g);
            float4 v = make_float4(d4.x * r4.x, d4.y * r4.y, d4.z * r4.z, d4.w * r4.w);
            if (!FIRST) {
                v.x += beta * p4.x;
                v.y += beta * p4.y;
                v.z += beta * p4.z;
                v.w += beta * p4.w;
            }
            if constexpr (WB > 0) {
#pragma unroll 4
                for (int j = 0; j < wc; ++j) {
                    float4 a;
                    if constexpr (H) {   // four 16-bit entries, dequantised exactly
                        const uint2 u = __ldg(reinterpret_cast<const uint2*>(W16 + (size_t)j * ld) + g);
                        const float sc = s_sc[j];
                        const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
                        const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
                        a = make_float4(lo.x * sc, lo.y * sc, hi.x * sc, hi.y * sc);
                    } else {
                        a = __ldg(reinterpret_cast<const float4*>(W + (size_t)j * ld) + g);
                    }
                    const float m = s_mu[j];
                    v.x -= a.x * m;
                    v.y -= a.y * m;
                    v.z -= a.z * m;
                    v.w -= a.w * m;
                }
            }
            reinterpret_cast<float4*>(p)[g] = v;
        }
    }
    for (int i = 4 * n4 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float pi = p[i];
        if (!FIRST) x[i] += alpha * pi;
        if (upd_p) {
            float v = dinv[i] * r[i];
            if (!FIRST) v += beta * pi;
#pragma unroll
            for (int j = 0; j < WB; ++j)
                if (j < wc) {
                    const float a = H ? __half2float(W16[(size_t)j * ld + i]) * s_sc[j] : W[(size_t)j * ld + i];
                    v -= a * s_mu[j];
                }
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

// FP32 with a basis: the TMA-staged update and direction passes (one CTA of kTmThreads
// threads per SM, kTmSmem bytes of dynamic shared memory).
template <int WB, bool COND>
static void pick_tma(bool w16, void** upd, void** dir0, void** dir)
{
    *upd = (void*)k_update_tma<WB>;
    *dir0 = w16 ? (void*)k_dir_tma<WB, true, true, false> : (void*)k_dir_tma<WB, true, false, false>;
    *dir = w16 ? (void*)k_dir_tma<WB, false, true, COND> : (void*)k_dir_tma<WB, false, false, COND>;
    static bool attr = false;
    if (!attr) {
        const void* fs[] = {(void*)k_update_tma<WB>, (void*)k_dir_tma<WB, true, true, false>,
                            (void*)k_dir_tma<WB, true, false, false>, (void*)k_dir_tma<WB, false, true, true>,
                            (void*)k_dir_tma<WB, false, false, true>, (void*)k_dir_tma<WB, false, true, false>,
                            (void*)k_dir_tma<WB, false, false, false>};
        for (const void* f : fs) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmSmemMax);
        attr = true;
    }
}

template <bool COND>
static void pick_tma_wb(int wb, bool w16, void** upd, void** dir0, void** dir)
{
    if (wb <= 8) pick_tma<8, COND>(w16, upd, dir0, dir);
    else if (wb <= 16) pick_tma<16, COND>(w16, upd, dir0, dir);
    else if (wb <= 32) pick_tma<32, COND>(w16, upd, dir0, dir);
    else if (wb <= 48) pick_tma<48, COND>(w16, upd, dir0, dir);
    else pick_tma<64, COND>(w16, upd, dir0, dir);
}

// FP32 with a basis, row-parallel float4 form.
template <int WB, bool COND>
static void pick_v4(bool w16, void** upd, void** dir0, void** dir)
{
    *upd = (void*)k_update_v4<WB>;
    *dir0 = w16 ? (void*)k_dir_v4<WB, true, false, true> : (void*)k_dir_v4<WB, true, false, false>;
    *dir = w16 ? (void*)k_dir_v4<WB, false, COND, true> : (void*)k_dir_v4<WB, false, COND, false>;
}

template <bool COND>
static void pick_v4_wb(int wb, bool w16, void** upd, void** dir0, void** dir)
{
    if (wb <= 0) pick_v4<0, COND>(false, upd, dir0, dir);
    else if (wb <= 8) pick_v4<8, COND>(w16, upd, dir0, dir);
    else if (wb <= 16) pick_v4<16, COND>(w16, upd, dir0, dir);
    else if (wb <= 32) pick_v4<32, COND>(w16, upd, dir0, dir);
    else if (wb <= 48) pick_v4<48, COND>(w16, upd, dir0, dir);
    else pick_v4<64, COND>(w16, upd, dir0, dir);
}

void cg_kernels(int wb, bool fp32, bool cond, int form, bool w16, void** init, void** upd, void** dir0, void** dir,
                int* smem_upd, int* smem_dir)
{
    *smem_upd = 0;
    *smem_dir = 0;
    if (fp32) {
        if (cond) pick<float, true>(wb, init, upd, dir0, dir);
        else pick<float, false>(wb, init, upd, dir0, dir);
        if (wb > 0 && form == kProjStaged) {
            if (cond) pick_tma_wb<true>(wb, w16, upd, dir0, dir);
            else pick_tma_wb<false>(wb, w16, upd, dir0, dir);
            *smem_upd = kTmSmemMax;
            *smem_dir = kTmSmemMax;
        } else {   // every FP32 width, 0 included: row-parallel float4, reductions without tails
            if (cond) pick_v4_wb<true>(wb, w16, upd, dir0, dir);
            else pick_v4_wb<false>(wb, w16, upd, dir0, dir);
        }
    } else {
        if (cond) pick<double, true>(wb, init, upd, dir0, dir);
        else pick<double, false>(wb, init, upd, dir0, dir);
    }
}

cudaError_t cg_set_wait_test(int mask, long long cycles)
{
    const WaitTest wt{cycles, mask, 0};
    return cudaMemcpyToSymbol(g_cg_wait_test, &wt, sizeof(wt));
}

int tma_block_threads() { return kTmThreads; }

void tma_shape(int n, int sms, int ncols, int cols_per_box, int nvec, bool allow_pair, int* grid, int* ring_bytes,
               int* smem)
{
    const int stage = (ncols + cols_per_box - 1) / cols_per_box * kTmBoxBytes + nvec * kTmVecBytes;
    const int pair = allow_pair && stage <= 40 * 1024;
    *ring_bytes = pair ? kTmRingPair : kTmRingMax;
    *smem = *ring_bytes + 1024;
    const int ntiles = (n + kTmTile - 1) / kTmTile;
    const int g = sms * (pair ? 2 : 1);
    *grid = ntiles < g ? ntiles : g;
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
