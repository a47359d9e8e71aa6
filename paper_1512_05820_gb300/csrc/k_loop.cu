// The FP32 inner loop of Algorithm 1 (mixed precision) as one persistent cooperative kernel:
// every iteration's three passes (the CG product q = A p with (A p, p); the update
// r -= alpha q, z = M^{-1} r, (r, z), ||r||^2, c = (A W)^T z; the direction x += alpha p,
// p = z + beta p - W mu) run in one launch, separated by grid-wide barriers instead of kernel
// boundaries. The arithmetic and the fixed-order reductions are those of the three-kernel
// chain (k_spmv_cg / k_update_v4 / k_dir_v4 with chain_alpha and chain_direction), so the
// iterates are the same; what goes away is the launch, ramp-up and tail of three kernels per
// iteration, which at small basis widths cost as much as the streaming itself.
//
// Every CTA of the grid must be resident (cooperative launch; the launch fails otherwise).
// Vectors written inside the launch (p, q, r, x) are written with st.global.cg and read with
// coherent loads after the barrier's acquire fence (the CG product's gathers of p through L1,
// where a stencil's neighbours reuse lines; the streams through L2); read-only data (the
// matrix, M^{-1}, the panels, M) keep the non-coherent read-only path, which is never used
// for data written inside the launch. The barrier's waits are bounded:
// a wait that runs out sets the timeout status (7), and each CTA leaves the loop at its next
// barrier, so the launch always ends.
#include "common.cuh"
#include "launch.h"

namespace podcg {

// the wait override of pod_cg_debug_wait_timeout (bit kWaitTestLoop)
static __device__ WaitTest g_loop_wait_test;

constexpr long long kLoopWaitPolls = 1ll << 24;   // ~1.7 s of 64 ns sleeps

// Grid barrier over G CTAs: bar[0] counts arrivals (zero between barriers), bar[1] is the
// generation, read by every CTA at the start of the launch (no barrier can complete before
// every CTA has arrived, so all read the same value). Thread 0 releases the block's writes
// (fence), arrives, and waits for the generation to pass `gen`; the last arrival resets the
// count and publishes the generation.
// Every thread then fences (acquire) before its next loads. Returns false when the wait ran
// out (or the test override made it run out).
__device__ __forceinline__ bool grid_sync(unsigned int* bar, unsigned int G, unsigned int& gen, DevState* st)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int test = g_loop_wait_test.mask & kWaitTestLoop;
        const long long polls = test ? g_loop_wait_test.cycles / 64 : kLoopWaitPolls;
        const unsigned int target = gen + 1;
        int ok = 1;
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar[0], 1u);
        if (arrived == G - 1 && !test) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicExch(&bar[1], target);
        } else {
            long long k = 0;
            while (*(volatile unsigned int*)&bar[1] != target) {
                if (++k > polls) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (!ok) st->status = 7;
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    __threadfence();
    gen += 1;
    return s_ok != 0;
}

template <int WB>
__global__ void __launch_bounds__(kBlock, 4) k_cg_loop(const ProbDesc* __restrict__ pd, float* p, float* q, float* r,
                                                       float* x, const float* __restrict__ dinv,
                                                       const float* __restrict__ AW, const float* __restrict__ W,
                                                       const double* __restrict__ M, double* partials,
                                                       unsigned int* bar, DevState* st,
                                                       cudaGraphConditionalHandle h_inner, int use_cond)
{
    constexpr int NA = WB > 0 ? WB : 1;
    __shared__ float s_red[kWarps][WB + 2];
    __shared__ double s_blk[WB + 2];
    __shared__ double s_tot[WB + 2];
    __shared__ float s_M[NA * NA];
    __shared__ double s_mud[NA];
    __shared__ float s_mu[NA];
    const int n = pd->n, ld = pd->ld;
    const int32_t* __restrict__ rp = pd->rp;
    const int32_t* __restrict__ col = pd->col;
    const float* __restrict__ val = pd->val32;
    const unsigned int G = gridDim.x;
    const int tid = blockIdx.x * kBlock + threadIdx.x, stride = (int)G * kBlock;
    const int n4 = n >> 2;
    unsigned int gen = *(volatile unsigned int*)&bar[1];
    unsigned long long t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    bool run = st->done == 0;   // written by k_init before the launch: the same for every CTA
    const int w = st->w;
    while (run) {
        // ---- the CG product: q = A p, this block's share of (A p, p)
        float dot = 0.0f;
        for (int row = tid; row < n; row += stride) {
            const int beg = __ldg(rp + row), end = __ldg(rp + row + 1);
            float s = 0.0f;
            if (end - beg <= 8) {
                const int len = end - beg;
                int c[8];
                float v[8], g[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    c[t] = (t < len) ? __ldg(col + beg + t) : 0;
                    v[t] = (t < len) ? __ldg(val + beg + t) : 0.0f;
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) g[t] = (t < len) ? p[c[t]] : 0.0f;
#pragma unroll
                for (int t = 0; t < 8; ++t) s += v[t] * g[t];
            } else {
                for (int k = beg; k < end; ++k) s += __ldg(val + k) * p[__ldg(col + k)];
            }
            __stcg(q + row, s);
            dot += s * p[row];
        }
        chain_store_gamma(double(dot), partials);
        if (!grid_sync(bar, G, gen, st)) break;

        // ---- update: alpha from the product's partials, then r, z, (r, z), ||r||^2, (A W)^T z
        const float alpha = float(chain_alpha(st, partials, (int)G));
        float acc[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) acc[j] = 0.0f;
        float rho = 0.0f, rr = 0.0f;
        for (int g = tid; g < n4; g += stride) {
            float4 r4 = __ldcg(reinterpret_cast<const float4*>(r) + g);
            const float4 q4 = __ldcg(reinterpret_cast<const float4*>(q) + g);
            const float4 d4 = __ldg(reinterpret_cast<const float4*>(dinv) + g);
            r4.x -= alpha * q4.x;
            r4.y -= alpha * q4.y;
            r4.z -= alpha * q4.z;
            r4.w -= alpha * q4.w;
            __stcg(reinterpret_cast<float4*>(r) + g, r4);
            const float4 z4 = make_float4(d4.x * r4.x, d4.y * r4.y, d4.z * r4.z, d4.w * r4.w);
            rho += r4.x * z4.x + r4.y * z4.y + r4.z * z4.z + r4.w * z4.w;
            rr += r4.x * r4.x + r4.y * r4.y + r4.z * r4.z + r4.w * r4.w;
#pragma unroll
            for (int j = 0; j < WB; ++j)
                if (j < w) {
                    const float4 a = __ldg(reinterpret_cast<const float4*>(AW + (size_t)j * ld) + g);
                    acc[j] += a.x * z4.x + a.y * z4.y + a.z * z4.z + a.w * z4.w;
                }
        }
        for (int i = 4 * n4 + tid; i < n; i += stride) {
            const float ri = __ldcg(r + i) - alpha * __ldcg(q + i);
            __stcg(r + i, ri);
            const float zi = __ldg(dinv + i) * ri;
            rho += ri * zi;
            rr += ri * ri;
#pragma unroll
            for (int j = 0; j < WB; ++j)
                if (j < w) acc[j] += __ldg(AW + (size_t)j * ld + i) * zi;
        }
        {
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
            for (int v = threadIdx.x; v < w + 2; v += kBlock) {
                double t = 0.0;
                for (int k = 0; k < kWarps; ++k) t += (double)s_red[k][v];
                s_blk[v] = t;
            }
            __syncthreads();
            chain_store(s_blk, w + 2, partials);
        }
        if (!grid_sync(bar, G, gen, st)) break;

        // ---- direction: beta, mu and the exit decision from the update's partials (every
        // CTA takes the same decision), x += alpha p, p = z + beta p - W mu
        const ChainStep cs = chain_direction<WB, true>(st, partials, (int)G, w, M, s_tot, s_M, s_mud, h_inner, use_cond);
        const float a_x = float(cs.alpha), beta = float(cs.beta);
        if (WB > 0 && cs.upd_p) {
            for (int j = threadIdx.x; j < NA; j += kBlock) s_mu[j] = (j < w) ? float(s_mud[j]) : 0.0f;
            __syncthreads();
        }
        const int wc = cs.upd_p ? w : 0;
        for (int g = tid; g < n4; g += stride) {
            const float4 p4 = __ldcg(reinterpret_cast<const float4*>(p) + g);
            float4 x4 = __ldcg(reinterpret_cast<const float4*>(x) + g);
            x4.x += a_x * p4.x;
            x4.y += a_x * p4.y;
            x4.z += a_x * p4.z;
            x4.w += a_x * p4.w;
            __stcg(reinterpret_cast<float4*>(x) + g, x4);
            if (cs.upd_p) {
                const float4 r4 = __ldcg(reinterpret_cast<const float4*>(r) + g);
                const float4 d4 = __ldg(reinterpret_cast<const float4*>(dinv) + g);
                float4 v = make_float4(d4.x * r4.x + beta * p4.x, d4.y * r4.y + beta * p4.y,
                                       d4.z * r4.z + beta * p4.z, d4.w * r4.w + beta * p4.w);
                if constexpr (WB > 0) {
#pragma unroll 4
                    for (int j = 0; j < wc; ++j) {
                        const float4 a = __ldg(reinterpret_cast<const float4*>(W + (size_t)j * ld) + g);
                        const float m = s_mu[j];
                        v.x -= a.x * m;
                        v.y -= a.y * m;
                        v.z -= a.z * m;
                        v.w -= a.w * m;
                    }
                }
                __stcg(reinterpret_cast<float4*>(p) + g, v);
            }
        }
        for (int i = 4 * n4 + tid; i < n; i += stride) {
            const float pi = __ldcg(p + i);
            __stcg(x + i, __ldcg(x + i) + a_x * pi);
            if (cs.upd_p) {
                float v = __ldg(dinv + i) * __ldcg(r + i) + beta * pi;
#pragma unroll
                for (int j = 0; j < WB; ++j)
                    if (j < wc) v -= __ldg(W + (size_t)j * ld + i) * s_mu[j];
                __stcg(p + i, v);
            }
        }
        if (!cs.upd_p) break;   // converged, capped or broken down: the same in every CTA
        if (!grid_sync(bar, G, gen, st)) break;
    }
    // the inner while-loop runs this body once per outer pass; block 0 adds the launch's time
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (use_cond) cudaGraphSetConditional(h_inner, 0u);
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        st->loop_ns += t1 - t0;
    }
}

void* kernel_cg_loop(int wb)
{
    if (wb <= 0) return (void*)k_cg_loop<0>;
    if (wb <= 8) return (void*)k_cg_loop<8>;
    return nullptr;
}

int cg_loop_grid(int wb, int sms)
{
    void* f = kernel_cg_loop(wb);
    if (!f) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kBlock, 0) != cudaSuccess) return 0;
    return per_sm * sms;
}

cudaError_t loop_set_wait_test(int mask, long long cycles)
{
    const WaitTest wt{cycles, mask, 0};
    return cudaMemcpyToSymbol(g_loop_wait_test, &wt, sizeof(wt));
}

}  // namespace podcg
