// Device-side helpers shared by the kernels of the POD-augmented CG library.
//
// Reductions are deterministic: each block reduces in a fixed shuffle/shared-memory
// order, writes one partial per value, and the last block to finish (found with one
// atomic ticket, no waiting) sums the partials in block order. Results are therefore
// identical from run to run for a given launch shape; no floating-point atomics are used.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace podcg {

constexpr int kBlock = 256;             // threads per block of every streaming kernel
constexpr int kWarps = kBlock / 32;
constexpr int kWMax = 64;               // largest basis dimension (w) supported
constexpr int kSMax = 64;               // largest snapshot window (s) supported

// Scalars of the iteration, resident in device memory for the whole solve so the loop
// needs no host round trip. One instance per solve in flight.
struct DevState {
    double rho;        // (r, z)
    double gamma;      // (A p, p)
    double alpha, beta;
    double rr;         // ||r||^2 of the recursive residual
    double bb;         // ||b||^2
    double tol2;       // (tol * ||b||)^2: the outer (true-residual) test
    double tol2_in;    // the inner loop's test on the recursive residual
    double rr_true;    // ||b - A x||^2 from the last true-residual product
    double rr_stage1;  // ||b - A x0||^2 after stage one
    double rr_outer;   // mixed precision: ||r||^2 of the current outer residual
    double rnorm;      // mixed precision: ||r|| of the current outer residual; the FP32
                       // inner solve works on r/||r|| (no underflow or overflow in FP32)
    double cond;       // cond_2(W^T A W) diagnostic
    double mu[kWMax];  // reduced coordinates of the A-orthogonalisation (Algorithm 1)
    double c[kWMax];   // (A W)^T z of the current iterate; mu = R^{-1} R^{-T} c
    double what[kWMax];// stage-one reduced solution
    int w;             // basis dimension in use (0 = plain PCG)
    int iters;         // CG iterations so far (all passes)
    int k_max;
    int restarts;      // residual replacements (FP64) / outer refinement steps (mixed)
    int max_refine;
    int status;        // pod_cg_status code
    int done;          // inner loop finished
    int chol_failed;
    int pod_w;         // w chosen by the POD (before a possible Cholesky failure)
    int outer_done;
    int inner_iters;   // mixed precision: iterations of the current inner solve
    int dir_pending;   // the direction kernel of this iteration has work (chunked loops)
    int mixed;         // FP32 inner loop: a breakdown ends the inner pass instead of the solve
    int inner_break;   // set by an FP32 inner breakdown (mixed mode)
    // stage two of the three-stage algorithm (Section 4.2)
    int pod_y;         // augmenting-basis dimension y chosen by the POD (0: no stage two)
    int w1;            // stage-one dimension after its Cholesky; stage two's basis starts here
    int k2;            // iterations of the current reduced solve (stage two, or an inner solve)
    int m_dirs;        // reduced directions stored so far (stage two's, then inner solves')
    int m_cap;         // at most min(y, basis capacity) - w1 of them
    int inner_total;   // inner reduced iterations of the whole-Y stage three
    int s2_done;       // the current reduced solve finished
    int s2_break;      // it ended on a non-positive or non-finite (Y^T A Y p, p)
    double tol_rel;    // the solve's relative tolerance (host-written)
    double rho2;       // (rhat, rhat)
    double tol2_s2;    // squared absolute stage-two tolerance
    double rh[kSMax];  // reduced residual
    double ph[kSMax];  // reduced direction
    double xh[kSMax];  // solution of the current inner reduced solve (whole-Y stage three)
    // FP32 inner loop without grid-reduction tails: copies the direction pass reads while its
    // block 0 rewrites the originals (written by block 0 of the update pass)
    double rho_prev;   // (r, z) before this iteration
    int iters_prev;    // iterations before this iteration
    int inner_prev;    // inner iterations before this iteration
    unsigned long long loop_ns;   // device time of the persistent inner-loop launches (ns)
};

// Borrowed problem pointers of the current solve, read by the kernels of a captured
// graph so the graph can be replayed for every system of a sequence.
struct ProbDesc {
    const int32_t* rp;
    const int32_t* col;
    const double* val;
    const float* val32;
    const double* b;
    double* x;
    int n;
    int ld;            // leading dimension of the n-by-k blocks (W, AW, S)
    // 3x3 block form of the same matrix (k_bsr.cu), when its pattern has one
    const int32_t* brp;   // block-row pointers, nb + 1
    const int32_t* bcol;  // block-column indices, nnzb
    const double* bval;   // values by block entry: entry (r, c) of block t at bval[(3r + c) nnzb + t]
    const float* bval32;  // the same in FP32 (mixed precision)
    int nb;               // block rows (n / 3)
    int nnzb;             // blocks (nnz / 9)
    // record of the stage-three search directions (accumulated Krylov vectors, Section 3.1):
    // while iters < krec_cap the FP64 CSR CG product stores p_k in column k of krec (row
    // stride ld) and (A p_k, p_k) in krec_gamma[k]; krec = NULL records nothing
    double* krec;
    double* krec_gamma;
    int krec_cap;
};

// Programmatic dependent launch inside the stage-three loop's graphs: the update and
// direction kernels hang off their predecessor by a programmatic edge, so their blocks may
// be scheduled while the predecessor's last blocks still run. Every loop kernel therefore
// waits for its prerequisite grids (completion and memory visibility) before its first
// access (a no-op when launched without such an edge), then lets its own dependents be
// scheduled: they too wait before touching anything this kernel writes.
__device__ __forceinline__ void pdl_wait_then_release()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// The scalar step after the CG product (Algorithm 1): gamma = (A p, p) given, the last
// block records it, flags a breakdown when it is not positive (an FP32 inner pass ends
// instead of the solve in mixed precision) and forms alpha = (r, z)/gamma. Thread 0 only.
__device__ __forceinline__ void cg_product_finish(DevState* st, double gamma)
{
    // read the state fields first (independent loads, one round of latency)
    int status = st->status, inner_break = st->inner_break;
    const int mixed = st->mixed;
    const double rho = st->rho;
    const bool bad = !isfinite(gamma) || !(gamma > 0.0);
    if (bad && status == 0) {
        if (mixed) inner_break = 1;
        else status = !isfinite(gamma) ? 5 : 3;
    }
    st->gamma = gamma;
    st->status = status;
    st->inner_break = inner_break;
    st->alpha = (status == 0 && !inner_break) ? rho / gamma : 0.0;
}

// Test support for the failure path of the bounded device waits
// (pod_cg_debug_wait_timeout): while a kernel's bit is set in `mask`, its producers issue no
// copies and each of its waits gives up after `cycles` SM clocks, so the timeout path runs
// with nothing in flight. Each translation unit with bounded waits keeps its own copy in
// device memory, read by the kernels at run time (captured graphs see changes).
struct WaitTest {
    long long cycles;
    int mask;
    int pad_;
};
constexpr int kWaitTestGramTc = 1;   // k_gram_tc
constexpr int kWaitTestStaged = 2;   // k_update_tma, k_dir_tma
constexpr int kWaitTestLoop = 4;     // k_cg_loop's grid barrier

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Stride between the partials of two values: partials are stored value-major
// (partials[v * kPartialStride + block], then the group partials at G + g).
constexpr int kPartialStride = 4096;   // >= any grid of a reducing kernel + kRedGroups

// Counters of one reduction site: kRedGroups first-level group tickets, then the top ticket.
constexpr int kRedGroups = 16;
constexpr int kCounterStride = 32;

// s_out[v] = sum of partials[v][first + i * step] over i < count, for v < nv <= NV: warp wid
// takes values wid, wid + kWarps, ...; lanes take rows i = lane, lane + 32, ... with U rows
// unrolled into independent sums, so up to 32 U rows cost one round of latency (partials
// written by other SMs a moment earlier take microseconds to read). Fixed order per value:
// lane strides, the U sums in order, then the warp's shuffle tree.
template <int NV, int U>
__device__ __forceinline__ void sum_rows(const double* __restrict__ partials, int nv, int first, int step, int count,
                                         double* s_out)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid >= kWarps) return;   // blocks with more warps (a producer warp) sum with the first kWarps
    constexpr int kR = (NV + kWarps - 1) / kWarps;
    double t[kR][U];
#pragma unroll
    for (int k = 0; k < kR; ++k)
#pragma unroll
        for (int u = 0; u < U; ++u) t[k][u] = 0.0;
    for (int i0 = lane; i0 < count; i0 += 32 * U) {
#pragma unroll
        for (int k = 0; k < kR; ++k) {
            const int v = wid + kWarps * k;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + 32 * u;
                if (v < nv && i < count) t[k][u] += __ldcg(partials + (size_t)v * kPartialStride + first + i * step);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kR; ++k) {
        const int v = wid + kWarps * k;
        if (v < nv) {   // uniform per warp
            double a = t[k][0];
#pragma unroll
            for (int u = 1; u < U; ++u) a += t[k][u];
            a = warp_sum(a);
            if (lane == 0) s_out[v] = a;
        }
    }
}

// Tail of a deterministic grid reduction, called by every block after thread 0 has published
// (and fenced) the block's nv partials at partials[v][blockIdx.x]. Two levels, so no block
// walks all G partials: block b belongs to group b mod NG (NG = min(G, kRedGroups)); the last
// block of each group to arrive sums its group's partials and publishes them at
// partials[v][G + g]; the last group to finish sums the NG group partials into s_tot[0..nv)
// and returns true (every other block returns false). Fixed summation order throughout, so
// results repeat bit for bit for a given grid. Needs G + kRedGroups <= kPartialStride and
// counter[0..kRedGroups] zero on entry (each level resets its own counters).
template <int NV, int U>
__device__ __forceinline__ bool grid_tail(double* __restrict__ partials, int nv, unsigned int* counter, double* s_tot)
{
    __shared__ int s_role;
    __shared__ double s_grp[kWMax + 2];
    const int G = gridDim.x;
    const int NG = G < kRedGroups ? G : kRedGroups;
    const int g = blockIdx.x % NG;
    const int members = (G - g + NG - 1) / NG;
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(counter + g, 1u);
        s_role = (t == (unsigned int)members - 1) ? 1 : 0;
    }
    __syncthreads();
    if (s_role == 0) return false;
    __threadfence();
    sum_rows<NV, U>(partials, nv, g, NG, members, s_grp);
    __syncthreads();
    if ((int)threadIdx.x < nv) {
        partials[(size_t)threadIdx.x * kPartialStride + G + g] = s_grp[threadIdx.x];
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        counter[g] = 0u;   // every member of the group has taken its ticket
        const unsigned int t = atomicAdd(counter + kRedGroups, 1u);
        s_role = (t == (unsigned int)NG - 1) ? 2 : 0;
    }
    __syncthreads();
    if (s_role != 2) return false;
    __threadfence();
    sum_rows<NV, U>(partials, nv, G, 1, NG, s_tot);
    __syncthreads();
    if (threadIdx.x == 0) counter[kRedGroups] = 0u;
    return true;
}

// Block-reduce acc[0..nv) (nv uniform over the grid, nv <= NV), store one partial per
// block, and return true in exactly one block, which then holds the grid totals in
// s_tot[0..nv) (grid_tail). Every thread of every block must call this exactly once per
// launch; `counter` points at the site's kCounterStride counters, zero on entry.
template <int NV>
__device__ __forceinline__ bool reduce_to_last_block(const double (&acc)[NV], int nv,
                                                     double* __restrict__ partials,
                                                     unsigned int* counter, double* s_tot)
{
    __shared__ double s_w[kWarps][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if (v < nv) {
            double t = warp_sum(acc[v]);
            if (lane == 0) s_w[wid][v] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int v = 0; v < nv; ++v) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < kWarps; ++k) t += s_w[k][v];
            partials[(size_t)v * kPartialStride + blockIdx.x] = t;
        }
        __threadfence();
    }
    return grid_tail<NV, 1>(partials, nv, counter, s_tot);
}

// Publish block totals s_blk[0..nv) (shared memory, complete before the call) as this
// block's partials; returns true in the last block to finish, which then holds the grid
// totals in s_tot[0..nv) (same fixed summation order as reduce_to_last_block).
__device__ __forceinline__ bool partials_to_last_block(const double* s_blk, int nv, double* __restrict__ partials,
                                                       unsigned int* counter, double* s_tot)
{
    // one thread publishes the block's partials and fences: the other threads never wait on
    // a memory fence
    if (threadIdx.x == 0) {
        for (int v = 0; v < nv; ++v) partials[(size_t)v * kPartialStride + blockIdx.x] = s_blk[v];
        __threadfence();
    }
    return grid_tail<kWMax + 2, 1>(partials, nv, counter, s_tot);
}

// ------------------------------------------------------------------ reductions without tails
//
// The FP32 inner loop (mixed precision) reduces across the grid without a last-block tail,
// whose fences, tickets and serialised sums cost about 7 us per launch on this GPU: every
// block of a producing kernel stores its partials and exits; every block of the consuming
// kernel sums all of them itself in one fixed order, so all blocks hold identical totals and
// the kernel boundary orders the stores before the loads. The SpMV's (A p, p) partials sit
// in row kSpmvRow of `partials`, the update pass's (r, z), ||r||^2 and (A W)^T z in rows
// 0 .. w+1 (value-major, kPartialStride apart). The helpers below synchronise the first
// kBlock threads of the block only (named barrier 1), so a TMA producer warp past them keeps
// streaming while they run.
constexpr int kSpmvRow = kWMax + 2;
constexpr int kPartialRows = kWMax + 3;

__device__ __forceinline__ void bar_compute() { asm volatile("bar.sync 1, %0;" ::"n"(kBlock) : "memory"); }

// s_out[v] = sum over b < G of partials[v * kPartialStride + b] for v < nv, in a fixed order:
// a group of TPV threads (the largest power of two with TPV nv <= kBlock, aligned) takes one
// value; thread k of the group sums b = k, k + TPV, ... into U interleaved accumulators (U
// independent loads in flight), combined in a fixed tree; then the group combines by a
// shuffle tree (and, for groups wider than a warp, the warp sums in order). Called by
// threads 0 .. kBlock-1 only (named barrier).
template <int U>
__device__ __forceinline__ void block_sum_rows(const double* __restrict__ partials, int nv, int G, double* s_out)
{
    __shared__ double s_wsum[kWarps];
    const int t = threadIdx.x;
    int tpv = kBlock;
    while (tpv * nv > kBlock) tpv >>= 1;
    const int v = t / tpv, k = t % tpv;
    double acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = 0.0;
    if (v < nv) {
        const double* row = partials + (size_t)v * kPartialStride;
        for (int b0 = k; b0 < G; b0 += U * tpv) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int b = b0 + u * tpv;
                if (b < G) acc[u] += __ldcg(row + b);
            }
        }
    }
#pragma unroll
    for (int h = U / 2; h > 0; h >>= 1)
#pragma unroll
        for (int u = 0; u < h; ++u) acc[u] += acc[u + h];
    double a = acc[0];
    if (tpv <= 32) {
        for (int o = tpv / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (k == 0 && v < nv) s_out[v] = a;
    } else {
        a = warp_sum(a);
        if ((t & 31) == 0) s_wsum[t >> 5] = a;
        bar_compute();
        if (t < nv) {
            const int wpg = tpv >> 5;   // warps per group
            double b = 0.0;
            for (int j = 0; j < wpg; ++j) b += s_wsum[t * wpg + j];
            s_out[t] = b;
        }
    }
    bar_compute();
}

// mu = R^{-1} R^{-T} c (reading R^{-1}, row stride kWMax, from global memory) into s_mu,
// c in shared or global memory; s_t: w doubles of shared scratch. Threads 0 .. kBlock-1 only.
__device__ __forceinline__ void block_mu_global(const double* __restrict__ Rinv, const double* c, int w, double* s_t,
                                                double* s_mu)
{
    for (int a = threadIdx.x; a < w; a += kBlock) {
        double v = 0.0;
        for (int k = 0; k <= a; ++k) v += __ldg(Rinv + (size_t)k * kWMax + a) * c[k];
        s_t[a] = v;
    }
    bar_compute();
    for (int a = threadIdx.x; a < w; a += kBlock) {
        double v = 0.0;
        for (int k = a; k < w; ++k) v += __ldg(Rinv + (size_t)a * kWMax + k) * s_t[k];
        s_mu[a] = v;
    }
    bar_compute();
}

// Update-pass prologue: gamma = (A p, p) from the SpMV's G partials, then the scalar step of
// cg_product_finish computed by every block from the same gamma (a breakdown ends an FP32
// inner pass, or the solve in FP64). Block 0 records gamma, alpha and the status, the copies
// the direction pass reads (rho, iters, inner_iters) and that the direction pass has work.
// Returns alpha (0 when the step is not valid). Threads 0 .. kBlock-1 only.
__device__ __forceinline__ double chain_alpha(DevState* st, const double* __restrict__ partials, int G)
{
    __shared__ double s_g[1];
    block_sum_rows<8>(partials + (size_t)kSpmvRow * kPartialStride, 1, G, s_g);
    const double gamma = s_g[0];
    int status = st->status, inner_break = st->inner_break;
    const int mixed = st->mixed;
    const double rho = st->rho;
    const bool bad = !isfinite(gamma) || !(gamma > 0.0);
    if (bad && status == 0) {
        if (mixed) inner_break = 1;
        else status = !isfinite(gamma) ? 5 : 3;
    }
    const double alpha = (status == 0 && !inner_break) ? rho / gamma : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int iters = st->iters, inner = st->inner_iters;
        st->gamma = gamma;
        st->alpha = alpha;
        st->status = status;
        st->inner_break = inner_break;
        st->rho_prev = rho;
        st->iters_prev = iters;
        st->inner_prev = inner;
        st->dir_pending = 1;
    }
    return alpha;
}

// SpMV epilogue without a tail: this block's share of (A p, p) (fixed shuffle tree, warps in
// order) stored as its partial in row kSpmvRow. Every thread of the block must call.
__device__ __forceinline__ void chain_store_gamma(double v, double* __restrict__ partials)
{
    __shared__ double s_g[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) s_g[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kWarps; ++k) t += s_g[k];
        partials[(size_t)kSpmvRow * kPartialStride + blockIdx.x] = t;
    }
}

// Store this block's nv totals s_blk[0..nv) as its partials in rows 0 .. nv-1 (no tail).
__device__ __forceinline__ void chain_store(const double* s_blk, int nv, double* __restrict__ partials)
{
    for (int v = threadIdx.x; v < nv; v += blockDim.x) partials[(size_t)v * kPartialStride + blockIdx.x] = s_blk[v];
}

// What a direction pass needs from the update pass it follows.
struct ChainStep {
    double beta;
    double alpha;   // 0 when the step of this iteration is not applied
    bool upd_p;     // the direction is updated (the pass has not finished)
};

// Direction-pass prologue: the update pass's totals ((r, z), ||r||^2, c = (A W)^T z) from its
// G partials into s_tot[0 .. w+2), then the decisions update_finish takes in the tailed form
// (beta, the iteration count, the exit test, the iteration cap, non-finite scalars), taken by
// every block from the same totals and the copies chain_alpha made, so they agree, and
// mu = M c into s_mu with M = R^{-1} R^{-T} (row stride kWMax), read into s_M (w x w, FP32:
// mu is used in FP32) in the same round as the partials. Block 0 writes the state and the graph condition. Threads
// 0 .. kBlock-1 only.
template <int WB, bool COND>
__device__ __forceinline__ ChainStep chain_direction(DevState* st, const double* __restrict__ partials, int G, int w,
                                                     const double* __restrict__ M, double* s_tot, float* s_M,
                                                     double* s_mu, cudaGraphConditionalHandle h_inner, int use_cond)
{
    constexpr int MPT = (WB * WB + kBlock - 1) / kBlock;   // entries of M per thread
    double m[MPT > 0 ? MPT : 1];
#pragma unroll
    for (int u = 0; u < MPT; ++u) {
        const int e = threadIdx.x + u * kBlock;
        m[u] = (e < w * w) ? __ldg(M + (size_t)(e / w) * kWMax + e % w) : 0.0;
    }
    block_sum_rows<16>(partials, w + 2, G, s_tot);
#pragma unroll
    for (int u = 0; u < MPT; ++u) {
        const int e = threadIdx.x + u * kBlock;
        if (e < w * w) s_M[e] = float(m[u]);
    }
    bar_compute();
    for (int a = threadIdx.x; a < w; a += kBlock) {
        double v = 0.0;
        for (int k = 0; k < w; ++k) v += (double)s_M[a * w + k] * s_tot[2 + k];
        s_mu[a] = v;
    }
    bar_compute();
    const double rho_old = st->rho_prev, tol2_in = st->tol2_in;
    const int iters = st->iters_prev + 1, inner_iters = st->inner_prev + 1, k_max = st->k_max;
    int status = st->status, inner_break = st->inner_break;
    const int mixed = st->mixed;
    const double rho_new = s_tot[0], rr = s_tot[1];
    if (status == 0 && !(isfinite(rho_new) && isfinite(rr))) {
        if (mixed) inner_break = 1;
        else status = 5;
    }
    int done = (status != 0) || inner_break || !(rr > tol2_in);
    if (!done && iters >= k_max) {
        status = 4;
        done = 1;
    }
    ChainStep cs;
    cs.beta = rho_new / rho_old;
    // the step of the iteration that reached the cap (status 4) is valid and is applied
    const bool ok = (status == 0 || status == 4) && !inner_break;
    cs.alpha = ok ? st->alpha : 0.0;
    cs.upd_p = !done && ok;
    if (blockIdx.x == 0) {
        for (int a = threadIdx.x; a < w; a += kBlock) st->c[a] = s_tot[2 + a];
        if (threadIdx.x == 0) {
            st->beta = cs.beta;
            st->rho = rho_new;
            st->rr = rr;
            st->iters = iters;
            st->inner_iters = inner_iters;
            st->status = status;
            st->inner_break = inner_break;
            st->done = done;
            if constexpr (COND) {
                if (use_cond) cudaGraphSetConditional(h_inner, done ? 0u : 1u);
            }
        }
    }
    return cs;
}

// Column-parallel accumulation of c_j += sum_rows col_j[row] * s_z[row - row0] over one
// 256-row tile: warp `wid` owns columns j = wid, wid + kWarps, ... (CPW of them), lanes read
// 32 consecutive rows of a column per access (coalesced 128/256-byte segments).
template <int CPW, typename T>
__device__ __forceinline__ void tile_columns(const T* __restrict__ M, int ld, int w, int row0, int n, const T* s_z,
                                             T (&cacc)[CPW])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < CPW; ++k) {
        const int j = wid + kWarps * k;
        if (j < w) {
            const T* col = M + (size_t)j * ld + row0;
            T a = T(0);
#pragma unroll
            for (int m = 0; m < kBlock / 32; ++m) {
                const int rr = lane + 32 * m;
                if (row0 + rr < n) a += __ldg(col + rr) * s_z[rr];
            }
            cacc[k] += a;
        }
    }
}

// Block totals of (two row sums, CPW column sums per warp) into s_blk[0..2+w).
template <int CPW, typename T>
__device__ __forceinline__ void block_totals(T v0, T v1, const T (&cacc)[CPW], int w, double* s_blk)
{
    __shared__ double s_two[kWarps][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double a0 = warp_sum(double(v0)), a1 = warp_sum(double(v1));
    if (lane == 0) {
        s_two[wid][0] = a0;
        s_two[wid][1] = a1;
    }
#pragma unroll
    for (int k = 0; k < CPW; ++k) {
        const int j = wid + kWarps * k;
        const double t = warp_sum(double(cacc[k]));
        if (lane == 0 && j < w) s_blk[2 + j] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int k = 0; k < kWarps; ++k) {
            t0 += s_two[k][0];
            t1 += s_two[k][1];
        }
        s_blk[0] = t0;
        s_blk[1] = t1;
    }
    __syncthreads();
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

}  // namespace podcg
