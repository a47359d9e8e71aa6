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
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Stride between the partials of two values: partials are stored value-major
// (partials[v * kPartialStride + block]) so the last block reads them coalesced.
constexpr int kPartialStride = 4096;   // >= any grid of a reducing kernel

// Block-reduce acc[0..nv) (nv uniform over the grid, nv <= NV), store one partial per
// block, and return true in the last block to finish, which then holds the grid totals
// in s_tot[0..nv). Every thread of every block must call this exactly once per launch.
// `counter` must be 0 on entry; the last block resets it.
template <int NV>
__device__ __forceinline__ bool reduce_to_last_block(const double (&acc)[NV], int nv,
                                                     double* __restrict__ partials,
                                                     unsigned int* counter, double* s_tot)
{
    __shared__ double s_w[kWarps][NV];
    __shared__ bool s_last;
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
        unsigned int ticket = atomicAdd(counter, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const int G = gridDim.x;
    for (int v = wid; v < nv; v += kWarps) {
        const double* pv = partials + (size_t)v * kPartialStride;
        double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
        int b = lane;
        for (; b + 96 < G; b += 128) {
            t0 += __ldcg(pv + b);
            t1 += __ldcg(pv + b + 32);
            t2 += __ldcg(pv + b + 64);
            t3 += __ldcg(pv + b + 96);
        }
        for (; b < G; b += 32) t0 += __ldcg(pv + b);
        double t = warp_sum((t0 + t1) + (t2 + t3));
        if (lane == 0) s_tot[v] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

// Publish block totals s_blk[0..nv) (shared memory, complete before the call) as this
// block's partials; returns true in the last block to finish, which then holds the grid
// totals in s_tot[0..nv) (same fixed summation order as reduce_to_last_block).
__device__ __forceinline__ bool partials_to_last_block(const double* s_blk, int nv, double* __restrict__ partials,
                                                       unsigned int* counter, double* s_tot)
{
    __shared__ bool s_last;
    // one thread publishes the block's partials, fences and takes the ticket: the other
    // threads never wait on a memory fence
    if (threadIdx.x == 0) {
        for (int v = 0; v < nv; ++v) partials[(size_t)v * kPartialStride + blockIdx.x] = s_blk[v];
        __threadfence();
        unsigned int ticket = atomicAdd(counter, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int G = gridDim.x;
    for (int v = wid; v < nv; v += kWarps) {
        const double* pv = partials + (size_t)v * kPartialStride;
        double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
        int b = lane;
        for (; b + 96 < G; b += 128) {
            t0 += __ldcg(pv + b);
            t1 += __ldcg(pv + b + 32);
            t2 += __ldcg(pv + b + 64);
            t3 += __ldcg(pv + b + 96);
        }
        for (; b < G; b += 32) t0 += __ldcg(pv + b);
        const double t = warp_sum((t0 + t1) + (t2 + t3));
        if (lane == 0) s_tot[v] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
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
