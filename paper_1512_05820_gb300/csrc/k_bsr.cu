// 3x3 block-sparse (BSR) form of the CG product, for matrices whose CSR pattern consists of
// full 3x3 blocks (three unknowns per mesh node, as the elasticity operator's). The same
// product as the CSR kernel (Algorithm 1's A p with gamma = (A p, p)), with one column
// index per 9 values instead of one per value: in FP32 4.44 bytes per nonzero instead of 8.
//
// Layout: block rows I = 0..nb-1 (rows 3I..3I+2), block-row pointers brp[nb + 1], block
// columns bcol[nnzb], values structure-of-arrays by block entry (entry (r, c) of block t at
// val[(3r + c) nnzb + t]), so lanes that read consecutive blocks read consecutive words.
//
// Built from the caller's CSR: k_bsr_check tests the pattern once (each row's columns come
// in aligned triplets c, c+1, c+2 with c divisible by 3, and the three rows of a block row
// share one block-column list), k_bsr_pattern derives brp and bcol, and k_bsr_values
// gathers the values of each system (FP64 and, in mixed precision, FP32).
#include "common.cuh"
#include "launch.h"

namespace podcg {

__global__ void __launch_bounds__(kBlock) k_bsr_check(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                      int n, int* __restrict__ bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int beg = rp[i], len = rp[i + 1] - beg;
        const int i0 = i - i % 3;
        const int beg0 = rp[i0], len0 = rp[i0 + 1] - beg0;
        bool ok = (len % 3 == 0) && (len == len0) && (beg0 % 9 == 0);
        for (int t = 0; ok && 3 * t < len; ++t) {
            const int c = col[beg + 3 * t];
            ok = (c % 3 == 0) && col[beg + 3 * t + 1] == c + 1 && col[beg + 3 * t + 2] == c + 2 &&
                 col[beg0 + 3 * t] == c;
        }
        if (!ok) atomicOr(bad, 1);
    }
}

__global__ void __launch_bounds__(kBlock) k_bsr_pattern(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                        int nb, int32_t* __restrict__ brp, int32_t* __restrict__ bcol)
{
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nb; I += gridDim.x * blockDim.x) {
        const int beg = rp[3 * I], nbk = (rp[3 * I + 1] - beg) / 3;
        const int b0 = beg / 9;
        brp[I] = b0;
        if (I == nb - 1) brp[nb] = rp[3 * nb] / 9;
        for (int t = 0; t < nbk; ++t) bcol[b0 + t] = col[beg + 3 * t] / 3;
    }
}

// One thread per row i = 3I + r: its 3 nbk values go to entries (r, 0..2) of the blocks.
__global__ void __launch_bounds__(kBlock) k_bsr_values(const int32_t* __restrict__ rp, const double* __restrict__ val,
                                                       int n, int nnzb, double* __restrict__ bval,
                                                       float* __restrict__ bval32)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = i % 3;
        const int beg = rp[i], nbk = (rp[i + 1] - beg) / 3;
        const int b0 = rp[i - r] / 9;
        for (int t = 0; t < nbk; ++t)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double v = val[beg + 3 * t + c];
                const size_t e = (size_t)(3 * r + c) * nnzb + b0 + t;
                bval[e] = v;
                if (bval32) bval32[e] = float(v);
            }
    }
}

// q = A p and gamma = (A p, p): L lanes per block row stride through its blocks (lane l
// takes blocks l, l + L, ...: consecutive lanes read consecutive value words), then the
// group sums its three row sums by shuffles. In FP32 (the inner loop of mixed precision)
// every block stores its share of gamma and the update pass forms alpha (chain_alpha); in
// FP64 the last block does.
template <int L, typename T>
__global__ void __launch_bounds__(kBlock) k_bsr_spmv_cg(const ProbDesc* __restrict__ pd, const T* __restrict__ p,
                                                        T* __restrict__ q, double* __restrict__ partials,
                                                        unsigned int* counter, DevState* st)
{
    pdl_wait_then_release();
    if (blockIdx.x == 0 && threadIdx.x == 0) st->dir_pending = 0;
    if (st->done) return;   // uniform: `done` is written by k_init / k_update only
    const int nb = pd->nb, nnzb = pd->nnzb;
    const int32_t* __restrict__ brp = pd->brp;
    const int32_t* __restrict__ bcol = pd->bcol;
    const T* __restrict__ v;
    if constexpr (sizeof(T) == 8) v = reinterpret_cast<const T*>(pd->bval);
    else v = reinterpret_cast<const T*>(pd->bval32);
    const int gpb = kBlock / L;
    const int g = threadIdx.x / L;
    const int lane = threadIdx.x & (L - 1);
    const int wg0 = (threadIdx.x & ~31) / L;
    const int stride = gridDim.x * gpb;
    T dot = T(0);
    for (int base = blockIdx.x * gpb + wg0; base < nb; base += stride) {
        const int I = base + (g - wg0);
        T s0 = T(0), s1 = T(0), s2 = T(0);
        if (I < nb) {
            const int end = __ldg(brp + I + 1);
            for (int b = __ldg(brp + I) + lane; b < end; b += L) {
                const int c = 3 * __ldg(bcol + b);
                const T x0 = __ldg(p + c), x1 = __ldg(p + c + 1), x2 = __ldg(p + c + 2);
                s0 += __ldg(v + b) * x0 + __ldg(v + (size_t)nnzb + b) * x1 + __ldg(v + (size_t)2 * nnzb + b) * x2;
                s1 += __ldg(v + (size_t)3 * nnzb + b) * x0 + __ldg(v + (size_t)4 * nnzb + b) * x1 +
                      __ldg(v + (size_t)5 * nnzb + b) * x2;
                s2 += __ldg(v + (size_t)6 * nnzb + b) * x0 + __ldg(v + (size_t)7 * nnzb + b) * x1 +
                      __ldg(v + (size_t)8 * nnzb + b) * x2;
            }
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0 && I < nb) {
            q[3 * I] = s0;
            q[3 * I + 1] = s1;
            q[3 * I + 2] = s2;
            dot += s0 * p[3 * I] + s1 * p[3 * I + 1] + s2 * p[3 * I + 2];
        }
    }
    if constexpr (sizeof(T) == 4) {
        chain_store_gamma(double(dot), partials);
    } else {
        double acc[1] = {double(dot)};
        __shared__ double tot[1];
        if (reduce_to_last_block<1>(acc, 1, partials, counter, tot) && threadIdx.x == 0) cg_product_finish(st, tot[0]);
    }
}

// ------------------------------------------------------------------------------ host side

cudaError_t launch_bsr_check(const int32_t* rp, const int32_t* col, int n, int* bad, int sms, cudaStream_t s)
{
    if (n % 3 != 0) return cudaErrorInvalidValue;
    k_bsr_check<<<grid_rows(n, kBlock, sms), kBlock, 0, s>>>(rp, col, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_bsr_pattern(const int32_t* rp, const int32_t* col, int nb, int32_t* brp, int32_t* bcol, int sms,
                               cudaStream_t s)
{
    k_bsr_pattern<<<grid_rows(nb, kBlock, sms), kBlock, 0, s>>>(rp, col, nb, brp, bcol);
    return cudaGetLastError();
}

cudaError_t launch_bsr_values(const int32_t* rp, const double* val, int n, int nnzb, double* bval, float* bval32,
                              int sms, cudaStream_t s)
{
    k_bsr_values<<<grid_rows(n, kBlock, sms), kBlock, 0, s>>>(rp, val, n, nnzb, bval, bval32);
    return cudaGetLastError();
}

int bsr_lanes_for(double blocks_per_row)
{
    if (blocks_per_row <= 3.0) return 2;
    if (blocks_per_row <= 8.0) return 4;
    if (blocks_per_row <= 20.0) return 8;
    return 16;
}

void* kernel_bsr_spmv_cg(int L, bool fp32)
{
    switch (L) {
    case 2: return fp32 ? (void*)k_bsr_spmv_cg<2, float> : (void*)k_bsr_spmv_cg<2, double>;
    case 4: return fp32 ? (void*)k_bsr_spmv_cg<4, float> : (void*)k_bsr_spmv_cg<4, double>;
    case 8: return fp32 ? (void*)k_bsr_spmv_cg<8, float> : (void*)k_bsr_spmv_cg<8, double>;
    case 16: return fp32 ? (void*)k_bsr_spmv_cg<16, float> : (void*)k_bsr_spmv_cg<16, double>;
    default: return fp32 ? (void*)k_bsr_spmv_cg<32, float> : (void*)k_bsr_spmv_cg<32, double>;
    }
}

}  // namespace podcg
