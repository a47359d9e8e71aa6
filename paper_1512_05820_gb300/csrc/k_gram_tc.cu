// Tall-skinny Gram G = X^T [Y, e] on the tensor cores (tcgen05) with split-bf16 products.
//
// This is the reduced-matrix product of stage one (Algorithm 2: W^T (A W) and W^T b) for
// FP32 or FP64 column blocks X (n x p), Y (n x qy) and an optional FP64 column e; p, qy
// <= 64. In FP64 it is bound by the FP64 pipe (2 p q n flops on (p + q) n words), so here
// the contraction runs on the bf16 tensor cores with an error-free splitting: every value,
// rounded to FP32, is written exactly as v = v_hi + v_mid + v_lo with three bf16 parts
// (successive 8-bit slices of the 24-bit significand, cut by truncation), in the manner of
// the multi-word splittings of Henry, Tang & Heinecke (2019, bfloat16 for higher-precision
// computations) and Ootomo & Yokota (2022). Products of bf16 parts are exact in FP32.
//
// Layout of one MMA (M = 128, N = round16(q), K = 16): the A operand stacks the parts of
// X along M — rows [hi; mid; lo] when 3p <= 128 (all nine part products, three MMAs per
// K step), else [hi; mid] plus a second operand [lo; 0] (seven products, four MMAs); the
// B operand is one part of [Y, e]. All MMAs of a window accumulate into one FP32 TMEM
// accumulator D; row part*p + a of D holds part(X_a) . [Y, e], so G[a][c] is the sum of
// the part rows. Every kTcFlush chunks (one window) the epilogue warps read D (tcgen05.ld)
// and add it into Kahan-compensated FP32 sums in shared memory; the CTA's sums go to FP64
// at the end and a deterministic reduction over CTAs (launch_gram_reduce) forms G.
//
// Pipeline per CTA (one per SM, persistent over a contiguous range of 32-row chunks), warp
// specialised and coupled by mbarriers only: a producer lane keeps a ring of TMA loads in
// flight (cp.async.bulk.tensor, 128-byte swizzle, zero fill past row n); eight converter
// warps split each chunk from the ring into the bf16 tiles of one of two MMA stages
// (canonical K-major layout, no swizzle); one lane issues the MMAs and commits them; four
// epilogue warps drain finished windows from two alternating TMEM accumulators, so the
// tensor cores never wait for the read-back. Every mbarrier wait is bounded (4e9 SM clocks,
// about 2 s); on expiry the role records the error and stops, the others stop at their
// next check or their own bounded wait, the CTA waits (bounded) for its own copies and
// MMAs in flight, frees its TMEM, writes NaN into its partial sums and sets the error flag
// (if given) to 7, the library's timeout status.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "common.cuh"
#include "launch.h"

namespace podcg {

constexpr int kTcRows = 32;        // contraction rows per chunk
constexpr int kTcM = 128;          // MMA M
constexpr int kTcNMax = 80;        // MMA N bound (q <= 65 rounded up to 16)
constexpr int kTcColsMax = 64;     // p and qy bounds
constexpr int kTcFlush = 4;        // chunks per TMEM accumulation window (128 rows)
constexpr int kTcBox = 8192;       // bytes of one TMA box slot: 64 columns x 128 bytes
constexpr int kTcRingBytes = 65536;
constexpr int kTcTileA = kTcM * kTcRows * 2;         // 8 KB
constexpr int kTcTileB = kTcNMax * kTcRows * 2;      // 5 KB
constexpr int kTcStageMma = 2 * kTcTileA + 3 * kTcTileB;
constexpr int kTcAccLd = kTcNMax + 1;                // padded row of the Kahan sums
constexpr uint32_t kTcTmemCols = 256;   // two accumulators of up to 128 columns
constexpr long long kTcWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

// shared-memory plan (offsets from a 1024-byte aligned base)
constexpr int kOffRing = 0;
constexpr int kOffExtra = kOffRing + kTcRingBytes;                 // up to 4 x 256 B
constexpr int kOffTiles = kOffExtra + 4 * 256;
constexpr int kOffSum = kOffTiles + 2 * kTcStageMma;
constexpr int kOffComp = kOffSum + kTcM * kTcAccLd * 4;
constexpr int kOffBar = kOffComp + kTcM * kTcAccLd * 4;           // 16 mbarriers
constexpr int kOffMisc = kOffBar + 16 * 8;
constexpr int kTcSmemBytes = kOffMisc + 64 + 1024;                 // + alignment slack

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of bf16 element (r, k) in an R x 32 tile, canonical K-major layout without
// swizzle: 8 x 8 core matrices of 128 contiguous bytes, K-adjacent cores 128 B apart (LBO),
// 8-row groups 512 B apart (SBO).
__host__ __device__ constexpr int tc_canon(int r, int k)
{
    return (r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// tcgen05 shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29),
// SBO >> 4 (32-45), fixed version 1 (46-48), base offset 0, no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B bf16 (7-9 = 1,
// 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool tc_try(uint32_t mbar, uint32_t parity)
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

// Wait for the phase of parity `parity` of an mbarrier; false after `budget` SM clocks
// (kTcWaitCycles, about 2 s at the maximum clock, unless a test shortened it). The clock is
// read only once the first try fails.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity, long long budget)
{
    if (tc_try(mbar, parity)) return true;
    const long long c0 = clock64();
    while (!tc_try(mbar, parity))
        if (clock64() - c0 > budget) return false;
    return true;
}

// The wait override of pod_cg_debug_wait_timeout for this kernel (zero: normal operation).
static __device__ WaitTest g_tc_wait_test;

// 4 consecutive values -> three packed bf16 quads (hi, mid, lo) with v = hi + mid + lo
// exactly. Truncation split: hi keeps the top 8 significant bits of v (its bf16 bit pattern
// is the upper half of v's), mid the next 8 of the exact remainder v - hi, lo the last 8
// of the exact remainder (at most 8 significant bits, so its upper half holds it exactly).
// Two logic ops and two subtractions per value, no conversion instructions.
__device__ __forceinline__ void tc_split4(const float v[4], uint2& hi, uint2& mid, uint2& lo)
{
    uint32_t h[4], m[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        h[t] = __float_as_uint(v[t]) & 0xFFFF0000u;
        const float r1 = v[t] - __uint_as_float(h[t]);
        m[t] = __float_as_uint(r1) & 0xFFFF0000u;
        l[t] = __float_as_uint(r1 - __uint_as_float(m[t]));
    }
    // element k at the lower address: low half = element 0 of the pair
    hi = make_uint2(__byte_perm(h[0], h[1], 0x7632), __byte_perm(h[2], h[3], 0x7632));
    mid = make_uint2(__byte_perm(m[0], m[1], 0x7632), __byte_perm(m[2], m[3], 0x7632));
    lo = make_uint2(__byte_perm(l[0], l[1], 0x7632), __byte_perm(l[2], l[3], 0x7632));
}

template <typename TI>
struct TcGeom {
    static constexpr int kBoxRows = 128 / (int)sizeof(TI);      // rows per 128-byte box row
    static constexpr int kBoxes = kTcRows / kBoxRows;          // boxes per chunk per operand
    static constexpr int kStageBytes = 2 * kBoxes * kTcBox;
    static constexpr int kStages = kTcRingBytes / kStageBytes;  // 4 (FP32) or 2 (FP64)
};

// Rows 4*k4 .. 4*k4+3 of column `col` of a box group (kBoxes boxes of [64][128 B] each,
// 128-byte swizzle: 16-byte chunk j of box row c sits at chunk j ^ (c & 7)).
template <typename TI>
__device__ __forceinline__ void tc_read4(const unsigned char* group, int col, int k4, float v[4])
{
    if constexpr (sizeof(TI) == 4) {
        const float4 f = *reinterpret_cast<const float4*>(group + col * 128 + ((k4 ^ (col & 7)) << 4));
        v[0] = f.x;
        v[1] = f.y;
        v[2] = f.z;
        v[3] = f.w;
    } else {
        const unsigned char* box = group + (k4 >> 2) * kTcBox + col * 128;
        const int ch = 2 * (k4 & 3);
        const double2 a = *reinterpret_cast<const double2*>(box + ((ch ^ (col & 7)) << 4));
        const double2 b = *reinterpret_cast<const double2*>(box + (((ch + 1) ^ (col & 7)) << 4));
        v[0] = (float)a.x;
        v[1] = (float)a.y;
        v[2] = (float)b.x;
        v[3] = (float)b.y;
    }
}

__device__ __forceinline__ void tc_tma2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tc_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Warp roles of the warp-specialised pipeline.
constexpr int kTcProducerWarp = 0;     // TMA loads (one lane); allocates and frees TMEM
constexpr int kTcMmaWarp = 1;          // tcgen05.mma issue (one lane)
constexpr int kTcConvWarp0 = 2;        // 8 converter warps: FP32 -> three bf16 tiles
constexpr int kTcConvWarps = 8;
constexpr int kTcEpiWarp0 = kTcConvWarp0 + kTcConvWarps;   // 4 epilogue warps: TMEM -> Kahan sums
constexpr int kTcWarps = kTcEpiWarp0 + 4;
constexpr int kTcThreads = 32 * kTcWarps;

// mbarrier slots
constexpr int kBarFull = 0;        // [4] TMA landed in ring slot s            (1 arrive + bytes)
constexpr int kBarRingFree = 4;    // [4] converters done with ring slot s      (8 arrives)
constexpr int kBarTileFull = 8;    // [2] bf16 tiles of stage st written        (8 arrives)
constexpr int kBarTileFree = 10;   // [2] MMAs of stage st complete             (commit)
constexpr int kBarAccFull = 12;    // [2] accumulator a holds a finished window (commit)
constexpr int kBarAccFree = 14;    // [2] epilogue done reading accumulator a   (4 arrives)
constexpr int kTcBars = 16;

template <typename TI>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
              const __grid_constant__ CUtensorMap tmE, int n, int p, int qy, int has_extra, int tiles_j,
              double* __restrict__ partials, int* err_flag)
{
    using G = TcGeom<TI>;
    constexpr int S = G::kStages;
    extern __shared__ unsigned char tc_raw[];
    unsigned char* base = tc_raw + ((1024u - (tc_smem_u32(tc_raw) & 1023u)) & 1023u);
    unsigned char* ring = base + kOffRing;
    unsigned char* extra = base + kOffExtra;
    unsigned char* tiles = base + kOffTiles;
    float* accS = reinterpret_cast<float*>(base + kOffSum);
    float* accC = reinterpret_cast<float*>(base + kOffComp);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + kOffBar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + kOffMisc);
    volatile int* s_err = reinterpret_cast<volatile int*>(base + kOffMisc + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = qy + has_extra;
    const int N = (q + 15) & ~15;
    const int parts1 = (3 * p <= kTcM) ? 3 : 2;   // parts stacked in the first A operand
    const int rows_used = parts1 * p;
    const int ncols = p + q;
    const int nchunks = (n + kTcRows - 1) / kTcRows;
    const int c0 = (int)(((long long)blockIdx.x * nchunks) / gridDim.x);
    const int nloc = (int)(((long long)(blockIdx.x + 1) * nchunks) / gridDim.x) - c0;
    const int nwin = (nloc + kTcFlush - 1) / kTcFlush;
    const uint32_t tx_bytes = (uint32_t)(G::kBoxes * 128 * (p + qy) + (has_extra ? 256 : 0));
    const WaitTest wt = g_tc_wait_test;
    const bool starve = (wt.mask & kWaitTestGramTc) != 0;   // test: no copies, short waits
    const long long budget = starve ? wt.cycles : kTcWaitCycles;
    auto B = [&](int i) { return tc_smem_u32(&bar[i]); };

    // zero the MMA tiles (rows beyond the used ones stay zero) and the Kahan sums
    {
        uint4* t = reinterpret_cast<uint4*>(tiles);
        for (int e = tid; e < 2 * kTcStageMma / 16; e += kTcThreads) t[e] = make_uint4(0, 0, 0, 0);
        for (int e = tid; e < kTcM * kTcAccLd; e += kTcThreads) {
            accS[e] = 0.0f;
            accC[e] = 0.0f;
        }
    }
    if (tid == 0) {
        *s_err = 0;
        for (int i = 0; i < kTcBars; ++i) {
            int cnt = 1;
            if ((i >= kBarRingFree && i < kBarRingFree + 4) || (i >= kBarTileFull && i < kBarTileFull + 2))
                cnt = 32 * kTcConvWarps;   // every converter thread arrives
            if (i >= kBarAccFree && i < kBarAccFree + 2) cnt = 128;   // every epilogue thread arrives
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(B(i)), "r"(cnt));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kTcProducerWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tmem_slot)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    auto fail = [&]() {
        *s_err = 1;
        if (err_flag) atomicExch(err_flag, 7);
    };

    if (warp == kTcProducerWarp) {
        if (lane == 0) {
            int issued = 0;
            for (int c = 0; c < nloc && !*s_err && !starve; ++c) {
                const int s = c % S;
                if (c >= S && !tc_wait(B(kBarRingFree + s), (uint32_t)((c / S - 1) & 1), budget)) {
                    fail();
                    break;
                }
                unsigned char* stage = ring + s * G::kStageBytes;
                const int row0 = (c0 + c) * kTcRows;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(B(kBarFull + s)),
                             "r"(tx_bytes)
                             : "memory");
                for (int b = 0; b < G::kBoxes; ++b) {
                    const int x = row0 + b * G::kBoxRows;
                    tc_tma2d(tc_smem_u32(stage + b * kTcBox), &tmX, x, 0, B(kBarFull + s));
                    if (qy > 0) tc_tma2d(tc_smem_u32(stage + (G::kBoxes + b) * kTcBox), &tmY, x, 0, B(kBarFull + s));
                }
                if (has_extra)
                    asm volatile(
                        "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];" ::"r"(
                            tc_smem_u32(extra + s * 256)),
                        "l"(reinterpret_cast<uint64_t>(&tmE)), "r"(row0), "r"(B(kBarFull + s))
                        : "memory");
                ++issued;
            }
            // every copy this CTA issued has landed before the CTA may exit (bounded)
            for (int s = 0; s < S && s < issued; ++s)
                tc_wait(B(kBarFull + s), (uint32_t)(((issued - s + S - 1) / S - 1) & 1), budget);
        }
    } else if (warp == kTcMmaWarp) {
        if (lane == 0) {
            const uint32_t idesc = tc_idesc(kTcM, N);
            const int pairs = parts1 == 3 ? 3 : 4;
            int last_c = -1;
            for (int c = 0; c < nloc && !*s_err; ++c) {
                const int st = c & 1;
                const int wnd = c / kTcFlush, a = wnd & 1;
                const bool first = (c % kTcFlush) == 0;
                const bool last = (c % kTcFlush) == kTcFlush - 1 || c == nloc - 1;
                if (!tc_wait(B(kBarTileFull + st), (uint32_t)((c >> 1) & 1), budget) ||
                    (first && wnd >= 2 && !tc_wait(B(kBarAccFree + a), (uint32_t)(((wnd >> 1) - 1) & 1), budget))) {
                    fail();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char* A1 = tiles + st * kTcStageMma;
                const uint32_t a1 = tc_smem_u32(A1), a2 = a1 + kTcTileA, bp = a1 + 2 * kTcTileA;
                const uint32_t d = tmem + (uint32_t)(a * 128);
                for (int kk = 0; kk < kTcRows / 16; ++kk) {
                    for (int pr = 0; pr < pairs; ++pr) {
                        const uint32_t aaddr = (pr < 3 ? a1 : a2) + (uint32_t)(kk * 256);
                        const uint32_t baddr = bp + (uint32_t)((pr < 3 ? pr : 0) * kTcTileB + kk * 256);
                        const uint32_t accumulate = (!first || kk > 0 || pr > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred pa;\n\t"
                            "setp.ne.u32 pa, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n\t}" ::"r"(d),
                            "l"(tc_desc(aaddr)), "l"(tc_desc(baddr)), "r"(idesc), "r"(accumulate)
                            : "memory");
                    }
                }
                tc_commit(B(kBarTileFree + st));
                if (last) tc_commit(B(kBarAccFull + a));
                last_c = c;
            }
            // the CTA's MMAs are complete before TMEM is freed (bounded)
            if (last_c >= 0) tc_wait(B(kBarTileFree + (last_c & 1)), (uint32_t)((last_c >> 1) & 1), budget);
        }
    } else if (warp < kTcEpiWarp0) {
        // converters: split the chunk in ring slot s into the bf16 tiles of stage st
        const int ctid = tid - 32 * kTcConvWarp0;
        const int groups = (ncols + 7) >> 3;
        for (int c = 0; c < nloc && !*s_err; ++c) {
            const int s = c % S, st = c & 1;
            if (!tc_wait(B(kBarFull + s), (uint32_t)((c / S) & 1), budget) ||
                (c >= 2 && !tc_wait(B(kBarTileFree + st), (uint32_t)(((c >> 1) - 1) & 1), budget))) {
                fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned char* stage = ring + s * G::kStageBytes;
            const double* ex = reinterpret_cast<const double*>(extra + s * 256);
            unsigned char* A1 = tiles + st * kTcStageMma;
            unsigned char* A2 = A1 + kTcTileA;
            unsigned char* Bp = A2 + kTcTileA;
            for (int e = ctid; e < groups * 64; e += 32 * kTcConvWarps) {
                const int g = e >> 5;
                const int col = (g >> 1) * 8 + (e & 7);
                const int k4 = ((e & 31) >> 3) + 4 * (g & 1);
                if (col >= ncols) continue;
                float v[4];
                if (col < p) tc_read4<TI>(stage, col, k4, v);
                else if (col < p + qy) tc_read4<TI>(stage + G::kBoxes * kTcBox, col - p, k4, v);
                else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) v[u] = (float)ex[4 * k4 + u];
                }
                uint2 hi, mid, lo;
                tc_split4(v, hi, mid, lo);
                if (col < p) {
                    *reinterpret_cast<uint2*>(A1 + tc_canon(col, 4 * k4)) = hi;
                    *reinterpret_cast<uint2*>(A1 + tc_canon(p + col, 4 * k4)) = mid;
                    if (parts1 == 3) *reinterpret_cast<uint2*>(A1 + tc_canon(2 * p + col, 4 * k4)) = lo;
                    else *reinterpret_cast<uint2*>(A2 + tc_canon(col, 4 * k4)) = lo;
                } else {
                    const int cc = col - p;
                    *reinterpret_cast<uint2*>(Bp + tc_canon(cc, 4 * k4)) = hi;
                    *reinterpret_cast<uint2*>(Bp + kTcTileB + tc_canon(cc, 4 * k4)) = mid;
                    *reinterpret_cast<uint2*>(Bp + 2 * kTcTileB + tc_canon(cc, 4 * k4)) = lo;
                }
            }
            // generic-proxy tile writes must be visible to the tensor cores' async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_arrive(B(kBarTileFull + st));
            tc_arrive(B(kBarRingFree + s));
        }
    } else {
        // epilogue: each finished window of accumulator a -> Kahan-compensated FP32 sums
        const int quarter = warp & 3;
        const int r = quarter * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
        for (int wnd = 0; wnd < nwin && !*s_err; ++wnd) {
            const int a = wnd & 1;
            if (!tc_wait(B(kBarAccFull + a), (uint32_t)((wnd >> 1) & 1), budget)) {
                fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (quarter * 32 < rows_used) {
                for (int cb = 0; cb < N / 16; ++cb) {
                    uint32_t d[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];"
                        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]),
                          "=r"(d[7]), "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]),
                          "=r"(d[14]), "=r"(d[15])
                        : "r"(taddr + (uint32_t)(a * 128 + cb * 16)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (r < rows_used) {
                        float* Sr = accS + r * kTcAccLd + cb * 16;
                        float* Cr = accC + r * kTcAccLd + cb * 16;
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const float y = __uint_as_float(d[u]) - Cr[u];
                            const float tt = Sr[u] + y;
                            Cr[u] = (tt - Sr[u]) - y;
                            Sr[u] = tt;
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            tc_arrive(B(kBarAccFree + a));
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == kTcProducerWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");

    // this CTA's partial Gram in the 8x8-tile layout of the Gram reduction
    const int ntiles = ((p + 7) / 8) * tiles_j;
    double* out = partials + (size_t)blockIdx.x * ntiles * 64;
    const bool bad = *s_err != 0;
    for (int e = tid; e < ntiles * 64; e += kTcThreads) {
        const int tile = e >> 6, el = e & 63;
        const int ai = (tile / tiles_j) * 8 + (el >> 3), cc = (tile % tiles_j) * 8 + (el & 7);
        double v = 0.0;
        if (ai < p && cc < q) {
            for (int part = 0; part < parts1; ++part) {
                const int rr = part * p + ai;
                v += (double)accS[rr * kTcAccLd + cc] - (double)accC[rr * kTcAccLd + cc];
            }
            if (bad) v = __longlong_as_double(0x7ff8000000000000LL);
        }
        out[e] = v;
    }
}

// ---------------------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    return fn;
}

bool encode_panel_map(CUtensorMap* tm, const void* base, int elem_bytes, int ld, int cols, int box_cols)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc || !base || cols < 1 || ld < 1 || (reinterpret_cast<uintptr_t>(base) & 15) ||
        ((size_t)ld * elem_bytes) % 16)
        return false;
    const CUtensorMapDataType dt = elem_bytes == 2   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    memset(tm, 0, sizeof(*tm));
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)cols};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * (cuuint64_t)elem_bytes};
    const cuuint32_t box[2] = {256u, (cuuint32_t)box_cols};
    const cuuint32_t estr[2] = {1, 1};
    return enc(tm, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int tc_grid(int n, int sms)
{
    const int nchunks = (n + kTcRows - 1) / kTcRows;
    return nchunks < sms ? nchunks : sms;
}

size_t gram_tc_workspace_bytes(int n, int p, int q, int sms)
{
    const int tiles = ((p + 7) / 8) * ((q + 7) / 8);
    return (size_t)tc_grid(n, sms) * tiles * 64 * sizeof(double);
}

bool gram_tc_aligned(const void* ptr, size_t ld_bytes)
{
    return (reinterpret_cast<uintptr_t>(ptr) & 15) == 0 && ld_bytes % 16 == 0;
}

template <typename TI>
static cudaError_t launch_gram_tc_t(int n, const TI* X, int ldx, int p, const TI* Y, int ldy, int qy,
                                    const double* extra, double* G, int ldg, double* work, size_t work_bytes,
                                    int* err_flag, int sms, cudaStream_t s)
{
    const int q = qy + (extra ? 1 : 0);
    if (n < 1 || p < 1 || p > kTcColsMax || qy < 0 || qy > kTcColsMax || q < 1) return cudaErrorInvalidValue;
    if (gram_tc_workspace_bytes(n, p, q, sms) > work_bytes) return cudaErrorInvalidValue;
    // TMA: 16-byte aligned bases and strides
    if (!gram_tc_aligned(X, (size_t)ldx * sizeof(TI))) return cudaErrorInvalidValue;
    if (qy > 0 && !gram_tc_aligned(Y, (size_t)ldy * sizeof(TI))) return cudaErrorInvalidValue;
    if (extra && !gram_tc_aligned(extra, 16)) return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;

    using Gm = TcGeom<TI>;
    const CUtensorMapDataType dt = sizeof(TI) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    CUtensorMap tmX, tmY, tmE;
    memset(&tmX, 0, sizeof(tmX));
    memset(&tmY, 0, sizeof(tmY));
    memset(&tmE, 0, sizeof(tmE));
    const cuuint32_t estr[2] = {1, 1};
    {
        const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)p};
        const cuuint64_t strides[1] = {(cuuint64_t)ldx * sizeof(TI)};
        const cuuint32_t box[2] = {(cuuint32_t)Gm::kBoxRows, (cuuint32_t)p};
        if (enc(&tmX, dt, 2, (void*)X, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    if (qy > 0) {
        const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)qy};
        const cuuint64_t strides[1] = {(cuuint64_t)ldy * sizeof(TI)};
        const cuuint32_t box[2] = {(cuuint32_t)Gm::kBoxRows, (cuuint32_t)qy};
        if (enc(&tmY, dt, 2, (void*)Y, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    if (extra) {
        const cuuint64_t dims[1] = {(cuuint64_t)n};
        const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(double)};   // unused for rank 1
        const cuuint32_t box[1] = {(cuuint32_t)kTcRows};
        if (enc(&tmE, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 1, (void*)extra, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    static bool attr[2] = {false, false};
    if (!attr[sizeof(TI) == 8]) {
        cudaError_t e = cudaFuncSetAttribute(k_gram_tc<TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
        if (e != cudaSuccess) return e;
        attr[sizeof(TI) == 8] = true;
    }
    const int grid = tc_grid(n, sms);
    const int tj = (q + 7) / 8;
    k_gram_tc<TI><<<grid, kTcThreads, kTcSmemBytes, s>>>(tmX, tmY, tmE, n, p, qy, extra ? 1 : 0, tj, work, err_flag);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_gram_reduce(work, grid, ((p + 7) / 8) * tj, tj, p, q, G, ldg, s);
}

cudaError_t launch_gram_tc(int n, const float* X, int ldx, int p, const float* Y, int ldy, int qy,
                           const double* extra, double* G, int ldg, double* work, size_t work_bytes, int* err_flag,
                           int sms, cudaStream_t s)
{
    return launch_gram_tc_t<float>(n, X, ldx, p, Y, ldy, qy, extra, G, ldg, work, work_bytes, err_flag, sms, s);
}

cudaError_t launch_gram_tc(int n, const double* X, int ldx, int p, const double* Y, int ldy, int qy,
                           const double* extra, double* G, int ldg, double* work, size_t work_bytes, int* err_flag,
                           int sms, cudaStream_t s)
{
    return launch_gram_tc_t<double>(n, X, ldx, p, Y, ldy, qy, extra, G, ldg, work, work_bytes, err_flag, sms, s);
}

cudaError_t gram_tc_set_wait_test(int mask, long long cycles)
{
    const WaitTest wt{cycles, mask, 0};
    return cudaMemcpyToSymbol(g_tc_wait_test, &wt, sizeof(wt));
}

}  // namespace podcg
