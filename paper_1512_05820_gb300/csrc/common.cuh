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
};

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
constexpr int kWaitTestStaged = 2;   // k_update_bulk, k_dir_bulk

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
