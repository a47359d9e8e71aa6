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

// ------------------------------------------------------------------ FP32 loop with staged tiles
//
// The FP32 update and direction passes stream 256-row tiles of the basis panel (A W for the
// update, W for the direction) and of the per-row vectors through a ring of shared-memory
// stages filled by bulk asynchronous copies (cp.async.bulk, the TMA engine) that complete
// on one mbarrier per stage. One block per SM owns a contiguous range of tiles. The ring is
// sized at run time from the basis width: a stage holds w + NV column tiles of 1 KB, and
// as many stages as fit in kBulkSmem are kept in flight (7 at w = 22), because under full
// load this GPU needs about 200 KB of reads in flight per SM to reach its HBM bandwidth.
// Copies are issued per basis column j < w (w from the device state), one per lane of
// warp 0. Every copy stays inside its buffer: a tile spans min(256, ld - row0) rows and all
// panels and vectors are allocated with the padded leading dimension ld (a multiple of 32
// >= n). Rows >= n inside a tile are never used. Every mbarrier wait is bounded (4e9 SM
// clocks, about 2 s); on expiry the block records status 7 (timeout), waits (bounded) for
// its own copies in flight and leaves the loop, and the pass ends with that status.

constexpr long long kBulkWaitCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr int kBulkSmem = 200 * 1024;                  // ring bytes per block (one block per SM)
constexpr int kBulkMaxStages = 32;
constexpr int kBulkBarBytes = kBulkMaxStages * 8;
constexpr int kBulkTile = kBlock * 4;                  // bytes of one 256-row FP32 column tile

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

// The ring of one block: tile range, run-time stage size and count, copy issue and waits.
// Stage layout: w panel column tiles, then the NV vector tiles, 1 KB each.
template <int NV>
struct BulkRing {
    unsigned char* smem;
    uint64_t* full;
    int t0, nloc, issued, S, w, stage_bytes;
    long long budget;   // SM clocks a wait may take
    bool starve;        // test of the timeout path: no copy is ever issued

    __device__ void init(unsigned char* sm, int n, int w_)
    {
        const WaitTest wt = g_cg_wait_test;
        starve = (wt.mask & kWaitTestStaged) != 0;
        budget = starve ? wt.cycles : kBulkWaitCycles;
        full = reinterpret_cast<uint64_t*>(sm);
        smem = sm + kBulkBarBytes;
        w = w_;
        stage_bytes = (w + NV) * kBulkTile;
        S = min(kBulkMaxStages, (kBulkSmem - kBulkBarBytes) / stage_bytes);
        const int ntiles = (n + kBlock - 1) / kBlock;
        t0 = (int)(((long long)blockIdx.x * ntiles) / gridDim.x);
        nloc = (int)(((long long)(blockIdx.x + 1) * ntiles) / gridDim.x) - t0;
        if (threadIdx.x == 0) {
            for (int i = 0; i < S; ++i)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bulk_smem_u32(&full[i])));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        issued = starve ? 0 : (nloc < S ? nloc : S);
        __syncthreads();
    }
    __device__ const float* stage(int t) const
    {
        return reinterpret_cast<const float*>(smem + (t % S) * stage_bytes);
    }
    __device__ int row0(int t) const { return (t0 + t) * kBlock; }

    // warp 0: copies of local tile t, one copy per lane so the w + NV copies leave
    // together; lane 0 posts the byte count first
    __device__ void issue(int t, int ld, const float* panel, const float* const* vec)
    {
        if (starve) return;
        const int lane = threadIdx.x & 31;
        const int r0 = row0(t);
        const int rows = min(kBlock, ld - r0);
        const uint32_t bytes = (uint32_t)rows * 4u;
        unsigned char* sg = smem + (t % S) * stage_bytes;
        const uint32_t mb = bulk_smem_u32(&full[t % S]);
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                         "r"(bytes * (uint32_t)(w + NV))
                         : "memory");
        __syncwarp();
        for (int c = lane; c < w + NV; c += 32) {
            const float* src;
            if (c < w) {
                src = panel + (size_t)c * ld;
            } else {
                const int v = c - w;   // select without indexing the array at run time
                src = vec[0];
#pragma unroll
                for (int u = 1; u < NV; ++u)
                    if (v == u) src = vec[u];
            }
            bulk_copy(bulk_smem_u32(sg + c * kBulkTile), src + r0, bytes, mb);
        }
    }
    __device__ bool wait(int t) const
    {
        return bulk_wait(bulk_smem_u32(&full[t % S]), (uint32_t)((t / S) & 1), budget);
    }
    // after a timeout: bounded waits for the copies still in flight
    __device__ void drain(int consumed) const
    {
        for (int t = consumed; t < issued; ++t) wait(t);
    }
};

template <int WB, bool COND>
__global__ void __launch_bounds__(kBlock) k_update_bulk(int n, int ld, float* __restrict__ r,
                                                        const float* __restrict__ q, const float* __restrict__ dinv,
                                                        const float* __restrict__ AW, double* __restrict__ partials,
                                                        unsigned int* counter, DevState* st,
                                                        cudaGraphConditionalHandle h_inner, int use_cond)
{
    if (st->done) return;   // uniform: only the last block of a pass writes `done`
    constexpr int CPW = (WB + kWarps - 1) / kWarps;
    extern __shared__ __align__(128) unsigned char bulk_sm[];
    __shared__ double s_blk[WB + 2];
    const int w = st->w;
    const float alpha = (st->status == 0) ? float(st->alpha) : 0.0f;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    BulkRing<3> ring;
    ring.init(bulk_sm, n, w);
    const float* const vec[3] = {r, q, dinv};
    if (threadIdx.x < 32)
        for (int t = 0; t < ring.issued; ++t) ring.issue(t, ld, AW, vec);
    float cacc[CPW];
#pragma unroll
    for (int k = 0; k < CPW; ++k) cacc[k] = 0.0f;
    float rho = 0.0f, rr = 0.0f;
    int t = 0;
    for (; t < ring.nloc; ++t) {
        // one barrier per tile: tile t has landed and every thread is done with tile t-1
        if (!__syncthreads_and(ring.wait(t))) break;
        if (t > 0 && t - 1 + ring.S < ring.nloc) {
            if (threadIdx.x < 32) ring.issue(t - 1 + ring.S, ld, AW, vec);   // refill tile t-1's stage
            if (!ring.starve) ++ring.issued;
        }
        const float* sg = ring.stage(t);
        const float* sr = sg + w * kBlock;
        const float* sq = sr + kBlock;
        const float* sd = sq + kBlock;
        const int row0 = ring.row0(t);
        const int valid = min(kBlock, n - row0);
        // row part: r -= alpha q (written back), z = M^{-1} r, (r, z), ||r||^2
        if ((int)threadIdx.x < valid) {
            const float ri = sr[threadIdx.x] - alpha * sq[threadIdx.x];
            r[row0 + threadIdx.x] = ri;
            const float zi = sd[threadIdx.x] * ri;
            rho += ri * zi;
            rr += ri * ri;
        }
        // column part: every warp forms z for the whole tile in registers (the same
        // arithmetic as the row part) and accumulates (A W)^T z for its columns
        if (valid == kBlock) {
            float4 z4[kBlock / 128];
#pragma unroll
            for (int m = 0; m < kBlock / 128; ++m) {
                const float4 a = reinterpret_cast<const float4*>(sr)[lane + 32 * m];
                const float4 b = reinterpret_cast<const float4*>(sq)[lane + 32 * m];
                const float4 d = reinterpret_cast<const float4*>(sd)[lane + 32 * m];
                z4[m] = make_float4(d.x * (a.x - alpha * b.x), d.y * (a.y - alpha * b.y), d.z * (a.z - alpha * b.z),
                                    d.w * (a.w - alpha * b.w));
            }
#pragma unroll
            for (int k = 0; k < CPW; ++k) {
                const int j = wid + kWarps * k;
                if (j < w) {
                    const float4* col = reinterpret_cast<const float4*>(sg + j * kBlock);
                    float a = 0.0f;
#pragma unroll
                    for (int m = 0; m < kBlock / 128; ++m) {
                        const float4 av = col[lane + 32 * m];
                        a += av.x * z4[m].x + av.y * z4[m].y + av.z * z4[m].z + av.w * z4[m].w;
                    }
                    cacc[k] += a;
                }
            }
        } else {
            for (int k = 0; k < CPW; ++k) {
                const int j = wid + kWarps * k;
                if (j < w) {
                    const float* col = sg + j * kBlock;
                    float a = 0.0f;
                    for (int m = 0; m < kBlock / 32; ++m) {
                        const int rr2 = lane + 32 * m;
                        if (rr2 < valid) a += col[rr2] * (sd[rr2] * (sr[rr2] - alpha * sq[rr2]));
                    }
                    cacc[k] += a;
                }
            }
        }
    }
    if (t < ring.nloc) {
        if (threadIdx.x == 0) atomicExch(&st->status, 7);
        ring.drain(t);
    }
    update_tail<WB, float, COND>(rho, rr, cacc, w, s_blk, partials, counter, st, h_inner, use_cond);
}

// FP32 direction pass with staged W tiles: mu = R^{-1} R^{-T} c, x += alpha p,
// p = z + beta p - W mu (FIRST: p0 = z0 - W mu0, x untouched), as k_dir. x is staged too,
// except in the FIRST pass, which does not read it.
template <int WB, bool FIRST>
__global__ void __launch_bounds__(kBlock) k_dir_bulk(int n, int ld, float* __restrict__ x, float* __restrict__ p,
                                                     const float* __restrict__ r, const float* __restrict__ dinv,
                                                     const float* __restrict__ W, const double* __restrict__ Rinv,
                                                     const DevState* st)
{
    if (!FIRST && !st->dir_pending) return;
    if (FIRST && st->outer_done) return;
    constexpr int NV = FIRST ? 3 : 4;
    const int w = st->w;
    const bool ok = (st->status == 0 || st->status == 4) && !st->inner_break;
    const float alpha = ok ? float(st->alpha) : 0.0f;
    const float beta = float(st->beta);
    const bool upd_p = FIRST || (!st->done && ok);
    extern __shared__ __align__(128) unsigned char bulk_sm[];
    __shared__ float s_mu[WB];
    if (upd_p) {
        // the ring's memory is scratch for mu until the first copy is issued
        double* s_R = reinterpret_cast<double*>(bulk_sm);
        double* s_c = s_R + WB * WB;
        double* s_t = s_c + WB;
        double* s_mud = s_t + WB;
        block_mu<WB>(Rinv, st->c, w, s_R, s_c, s_t, s_mud);
        for (int j = threadIdx.x; j < WB; j += blockDim.x) s_mu[j] = (j < w) ? float(s_mud[j]) : 0.0f;
        __syncthreads();
    }
    // without a p update only x += alpha p remains: no panel needed
    const int wc = upd_p ? w : 0;
    BulkRing<NV> ring;
    ring.init(bulk_sm, n, wc);
    const float* vec[NV];
    vec[0] = p;
    vec[1] = r;
    vec[2] = dinv;
    if constexpr (!FIRST) vec[NV - 1] = x;
    if (threadIdx.x < 32)
        for (int t = 0; t < ring.issued; ++t) ring.issue(t, ld, W, vec);
    int t = 0;
    for (; t < ring.nloc; ++t) {
        // one barrier per tile: tile t has landed and every thread is done with tile t-1
        if (!__syncthreads_and(ring.wait(t))) break;
        if (t > 0 && t - 1 + ring.S < ring.nloc) {
            if (threadIdx.x < 32) ring.issue(t - 1 + ring.S, ld, W, vec);
            if (!ring.starve) ++ring.issued;
        }
        const float* sg = ring.stage(t);
        const float* sv = sg + wc * kBlock;
        const int i = ring.row0(t) + threadIdx.x;
        if (i < n) {
            const float pi = sv[threadIdx.x];
            if constexpr (!FIRST) x[i] = sv[3 * kBlock + threadIdx.x] + alpha * pi;
            if (upd_p) {
                float v = sv[2 * kBlock + threadIdx.x] * sv[kBlock + threadIdx.x];
                if (!FIRST) v += beta * pi;
#pragma unroll
                for (int j = 0; j < WB; ++j)
                    if (j < wc) v -= sg[j * kBlock + threadIdx.x] * s_mu[j];
                p[i] = v;
            }
        }
    }
    if (t < ring.nloc) {
        if (threadIdx.x == 0) atomicExch(const_cast<int*>(&st->status), 7);
        ring.drain(t);
    }
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

template <int WB, bool COND>
__global__ void __launch_bounds__(kBlock, 2) k_update_v4(int n, int ld, float* __restrict__ r,
                                                         const float* __restrict__ q, const float* __restrict__ dinv,
                                                         const float* __restrict__ AW, double* __restrict__ partials,
                                                         unsigned int* counter, DevState* st,
                                                         cudaGraphConditionalHandle h_inner, int use_cond)
{
    if (st->done) return;   // uniform: only the last block of a pass writes `done`
    __shared__ float s_red[kWarps][WB + 2];
    __shared__ double s_blk[WB + 2];
    const int w = st->w;
    const float alpha = (st->status == 0) ? float(st->alpha) : 0.0f;
    float acc[WB];
#pragma unroll
    for (int j = 0; j < WB; ++j) acc[j] = 0.0f;
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
    update_finish<WB, COND>(s_blk, w, partials, counter, st, h_inner, use_cond);
}

template <int WB, bool FIRST>
__global__ void __launch_bounds__(kBlock, WB <= 32 ? kV4Blocks - 1 : 4) k_dir_v4(int n, int ld, float* __restrict__ x,
                                                              float* __restrict__ p, const float* __restrict__ r,
                                                              const float* __restrict__ dinv,
                                                              const float* __restrict__ W,
                                                              const double* __restrict__ Rinv, const DevState* st)
{
    if (!FIRST && !st->dir_pending) return;
    if (FIRST && st->outer_done) return;
    const int w = st->w;
    const bool ok = (st->status == 0 || st->status == 4) && !st->inner_break;
    const float alpha = ok ? float(st->alpha) : 0.0f;
    const float beta = float(st->beta);
    const bool upd_p = FIRST || (!st->done && ok);
    __shared__ double s_R[WB * WB];
    __shared__ double s_c[WB], s_t[WB], s_mud[WB];
    __shared__ float s_mu[WB];
    if (upd_p) {
        block_mu<WB>(Rinv, st->c, w, s_R, s_c, s_t, s_mud);
        for (int j = threadIdx.x; j < WB; j += blockDim.x) s_mu[j] = (j < w) ? float(s_mud[j]) : 0.0f;
        __syncthreads();
    }
    const int wc = upd_p ? w : 0;
    const int n4 = n >> 2;
    const int stride = gridDim.x * blockDim.x;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n4; g += stride) {
        const float4 p4 = reinterpret_cast<const float4*>(p)[g];
        if (!FIRST) {
            float4 x4 = reinterpret_cast<const float4*>(x)[g];
            x4.x += alpha * p4.x;
            x4.y += alpha * p4.y;
            x4.z += alpha * p4.z;
            x4.w += alpha * p4.w;
            reinterpret_cast<float4*>(x)[g] = x4;
        }
        if (upd_p) {
            const float4 r4 = __ldg(reinterpret_cast<const float4*>(r) + g);
            const float4 d4 = __ldg(reinterpret_cast<const float4*>(dinv) + g);
            float4 v = make_float4(d4.x * r4.x, d4.y * r4.y, d4.z * r4.z, d4.w * r4.w);
            if (!FIRST) {
                v.x += beta * p4.x;
                v.y += beta * p4.y;
                v.z += beta * p4.z;
                v.w += beta * p4.w;
            }
#pragma unroll 4
            for (int j = 0; j < wc; ++j) {
                const float4 a = __ldg(reinterpret_cast<const float4*>(W + (size_t)j * ld) + g);
                const float m = s_mu[j];
                v.x -= a.x * m;
                v.y -= a.y * m;
                v.z -= a.z * m;
                v.w -= a.w * m;
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
                if (j < wc) v -= W[(size_t)j * ld + i] * s_mu[j];
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

// FP32 with a basis: the staged-tile update and direction passes.
template <int WB, bool COND>
static void pick_bulk(void** upd, void** dir0, void** dir, int* smem_upd, int* smem_dir)
{
    *upd = (void*)k_update_bulk<WB, COND>;
    *dir0 = (void*)k_dir_bulk<WB, true>;
    *dir = (void*)k_dir_bulk<WB, false>;
    *smem_upd = kBulkSmem;
    *smem_dir = kBulkSmem;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_update_bulk<WB, COND>, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem_upd);
        cudaFuncSetAttribute(k_dir_bulk<WB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem_dir);
        cudaFuncSetAttribute(k_dir_bulk<WB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem_dir);
        attr = true;
    }
}

template <bool COND>
static void pick_bulk_wb(int wb, void** upd, void** dir0, void** dir, int* su, int* sd)
{
    if (wb <= 8) pick_bulk<8, COND>(upd, dir0, dir, su, sd);
    else if (wb <= 16) pick_bulk<16, COND>(upd, dir0, dir, su, sd);
    else if (wb <= 32) pick_bulk<32, COND>(upd, dir0, dir, su, sd);
    else if (wb <= 48) pick_bulk<48, COND>(upd, dir0, dir, su, sd);
    else pick_bulk<64, COND>(upd, dir0, dir, su, sd);
}

// FP32 with a basis, row-parallel float4 form.
template <int WB, bool COND>
static void pick_v4(void** upd, void** dir0, void** dir)
{
    *upd = (void*)k_update_v4<WB, COND>;
    *dir0 = (void*)k_dir_v4<WB, true>;
    *dir = (void*)k_dir_v4<WB, false>;
}

template <bool COND>
static void pick_v4_wb(int wb, void** upd, void** dir0, void** dir)
{
    if (wb <= 8) pick_v4<8, COND>(upd, dir0, dir);
    else if (wb <= 16) pick_v4<16, COND>(upd, dir0, dir);
    else if (wb <= 32) pick_v4<32, COND>(upd, dir0, dir);
    else if (wb <= 48) pick_v4<48, COND>(upd, dir0, dir);
    else pick_v4<64, COND>(upd, dir0, dir);
}

void cg_kernels(int wb, bool fp32, bool cond, int form, void** init, void** upd, void** dir0, void** dir,
                int* smem_upd, int* smem_dir)
{
    *smem_upd = 0;
    *smem_dir = 0;
    if (fp32) {
        if (cond) pick<float, true>(wb, init, upd, dir0, dir);
        else pick<float, false>(wb, init, upd, dir0, dir);
        if (wb > 0 && form == kProjStaged) {
            if (cond) pick_bulk_wb<true>(wb, upd, dir0, dir, smem_upd, smem_dir);
            else pick_bulk_wb<false>(wb, upd, dir0, dir, smem_upd, smem_dir);
        } else if (wb > 0) {
            if (cond) pick_v4_wb<true>(wb, upd, dir0, dir);
            else pick_v4_wb<false>(wb, upd, dir0, dir);
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
