// Batched persistent solver: many independent sequences of uneven sizes in one launch.
//
// A worker is one thread-block cluster (CL CTAs). Workers take whole sequences from a
// queue ordered by decreasing estimated work (one atomic ticket per sequence, no waiting)
// and solve every system of the sequence in order, recycling the previous solutions:
//   POD of the snapshots (Gram row per new snapshot, Jacobi eigensolve, energy truncation,
//   Algorithm 4), FP32 lift W = S C, FP32 A W, Gram W^T [A W, b] with FP64 sums, FP64
//   Cholesky (Algorithm 2), x0 = W what, then FP64 refinement around FP32 augmented PCG
//   (Algorithm 1 with Y = W on the correction) until ||b - A x|| <= tol ||b|| in FP64.
// Rows of a sequence are spread over all threads of the cluster. Sums over rows are
// block-reduced, then combined across the cluster through distributed shared memory; each
// combination costs one hardware cluster barrier (double-buffered slots), and every CTA
// ends with identical totals. The cluster barrier also orders the global-memory vector
// updates between phases (release/acquire at cluster scope). No spin waits: all loops are
// bounded by the iteration and refinement caps.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "pod_cg.h"

namespace cg = cooperative_groups;

namespace podcg {

constexpr int kBW = 32;        // largest basis dimension of the batched solver
constexpr int kBS = 16;        // largest snapshot window of the batched solver
constexpr int kBThreads = 512; // threads per CTA
constexpr int kBWarps = kBThreads / 32;
constexpr int kRedMax = 64;    // values per cluster reduction (>= kBW + 2 and 8x8 Gram tiles)

// Device descriptor of one sequence (arena pointers filled by the host).
struct BatchSeqDev {
    int n, nnz, p, w_max, s_max;
    double tol, energy;
    const int32_t* rp;
    const int32_t* col;
    const double* val;   // p x nnz
    const double* b;     // p x n
    double* x;           // p x n (output)
    // workspace
    double* S;           // s_max x n
    float* S32;          // s_max x n
    float* W;            // w_max x n
    float* AW;           // w_max x n
    float* val32;        // nnz
    double* r64;         // n
    float *r, *p32, *q, *d, *dinv;   // n each
    // tiles of the inner CG loop (chosen per size class by the autotuner): lanes per row of
    // the CSR product (1, 2, 4 or 8) and rows per thread of the update and direction passes
    // (1, or 4 as float4 when n is a multiple of 4)
    int lanes, vec;
    unsigned long long* t_ns;   // device time of this sequence's solve (global timer, ns)
    // per-system statistics
    int* st_status;
    int* st_iters;
    int* st_refine;
    int* st_w;
    double* st_relres;
    double* st_stage1;
};

struct BatchSmem {
    double red_w[kBWarps][kRedMax];
    double slot[2][kRedMax];
    double tot[kRedMax];
    double GS[kBS * kBS];
    double A[kBS * kBS];
    double V[kBS * kBS];
    double C[kBS * kBW];       // lift coefficients (s x w)
    double G[kBW * (kBW + 1)]; // stage-one Gram W^T [AW, b]
    double R[kBW * kBW];       // Cholesky factor, then its inverse
    double Rinv[kBW * kBW];
    double mu[kBW];
    double t[kBW];
    double what[kBW];
    float muf[kBW];
    double ev[kBS];
    int seq;
    int w;
};

struct Team {
    cg::cluster_group cl;
    int rank, nctas, tid, nthr;
    int phase;
};

// Sum acc[0..nv) over all threads of the cluster; totals land in sm.tot (every CTA).
template <int NV>
__device__ void team_sum(Team& T, BatchSmem& sm, const double (&acc)[NV], int nv)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if (v < nv) {
            const double t = warp_sum(acc[v]);
            if (lane == 0) sm.red_w[wid][v] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int k = 0; k < kBWarps; ++k) s += sm.red_w[k][threadIdx.x];
        sm.slot[T.phase][threadIdx.x] = s;
    }
    T.cl.sync();
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int r = 0; r < T.nctas; ++r) s += *T.cl.map_shared_rank(&sm.slot[T.phase][threadIdx.x], r);
        sm.tot[threadIdx.x] = s;
    }
    T.phase ^= 1;
    __syncthreads();
}

// Cyclic-by-row Jacobi on the s x s matrix in sm.A (row stride kBS), one thread; results:
// sm.ev (decreasing), sm.V columns (largest-magnitude entry positive).
__device__ void small_jacobi(BatchSmem& sm, int s)
{
    double* A = sm.A;
    double U[kBS * kBS];
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) U[i * kBS + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) fro += A[i * kBS + j] * A[i * kBS + j];
    for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j)
                if (i != j) off += A[i * kBS + j] * A[i * kBS + j];
        if (off <= 1e-32 * fro || off == 0.0) break;
        for (int p = 0; p < s - 1; ++p)
            for (int q = p + 1; q < s; ++q) {
                const double apq = A[p * kBS + q];
                if (apq == 0.0) continue;
                const double th = (A[q * kBS + q] - A[p * kBS + p]) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                for (int k = 0; k < s; ++k) {
                    const double a1 = A[k * kBS + p], a2 = A[k * kBS + q];
                    A[k * kBS + p] = c * a1 - sn * a2;
                    A[k * kBS + q] = sn * a1 + c * a2;
                }
                for (int k = 0; k < s; ++k) {
                    const double a1 = A[p * kBS + k], a2 = A[q * kBS + k];
                    A[p * kBS + k] = c * a1 - sn * a2;
                    A[q * kBS + k] = sn * a1 + c * a2;
                }
                for (int k = 0; k < s; ++k) {
                    const double u1 = U[k * kBS + p], u2 = U[k * kBS + q];
                    U[k * kBS + p] = c * u1 - sn * u2;
                    U[k * kBS + q] = sn * u1 + c * u2;
                }
            }
    }
    bool used[kBS];
    for (int i = 0; i < s; ++i) used[i] = false;
    for (int i = 0; i < s; ++i) {
        int best = -1;
        for (int j = 0; j < s; ++j)
            if (!used[j] && (best < 0 || A[j * kBS + j] > A[best * kBS + best])) best = j;
        used[best] = true;
        sm.ev[i] = A[best * kBS + best];
        int arg = 0;
        for (int k = 1; k < s; ++k)
            if (fabs(U[k * kBS + best]) > fabs(U[arg * kBS + best])) arg = k;
        const double sg = U[arg * kBS + best] < 0.0 ? -1.0 : 1.0;
        for (int k = 0; k < s; ++k) sm.V[k * kBS + i] = sg * U[k * kBS + best];
    }
}

// Upper Cholesky of sm.G[:, :w] (row stride kBW+1) into sm.R, R^{-1} into sm.Rinv,
// what = R^{-1} R^{-T} G[:, w]. One thread. Returns false if not numerically SPD.
__device__ bool small_chol(BatchSmem& sm, int w)
{
    const int ldg = kBW + 1;
    for (int i = 0; i < w; ++i)
        for (int j = 0; j < w; ++j) sm.R[i * kBW + j] = 0.0;
    for (int i = 0; i < w; ++i) {
        double d = sm.G[i * ldg + i];
        for (int k = 0; k < i; ++k) d -= sm.R[k * kBW + i] * sm.R[k * kBW + i];
        if (!(d > 0.0) || !isfinite(d)) return false;
        const double rii = sqrt(d);
        sm.R[i * kBW + i] = rii;
        for (int j = i + 1; j < w; ++j) {
            double s = sm.G[i * ldg + j];
            for (int k = 0; k < i; ++k) s -= sm.R[k * kBW + i] * sm.R[k * kBW + j];
            sm.R[i * kBW + j] = s / rii;
        }
    }
    for (int j = 0; j < w; ++j)
        for (int i = j; i >= 0; --i) {
            double t = (i == j) ? 1.0 : 0.0;
            for (int k = i + 1; k <= j; ++k) t -= sm.R[i * kBW + k] * sm.Rinv[k * kBW + j];
            sm.Rinv[i * kBW + j] = t / sm.R[i * kBW + i];
        }
    for (int i = 0; i < w; ++i)
        for (int j = 0; j < i; ++j) sm.Rinv[i * kBW + j] = 0.0;
    for (int a = 0; a < w; ++a) {
        double v = 0.0;
        for (int k = 0; k <= a; ++k) v += sm.Rinv[k * kBW + a] * sm.G[k * ldg + w];
        sm.t[a] = v;
    }
    for (int a = 0; a < w; ++a) {
        double v = 0.0;
        for (int k = a; k < w; ++k) v += sm.Rinv[a * kBW + k] * sm.t[k];
        sm.what[a] = v;
    }
    return true;
}

// mu = R^{-1} R^{-T} c for c in sm.tot[off..off+w) (thread 0), float copy in sm.muf.
__device__ void apply_rinv_small(BatchSmem& sm, int w, int off)
{
    if (threadIdx.x == 0) {
        for (int a = 0; a < w; ++a) {
            double v = 0.0;
            for (int k = 0; k <= a; ++k) v += sm.Rinv[k * kBW + a] * sm.tot[off + k];
            sm.t[a] = v;
        }
        for (int a = 0; a < w; ++a) {
            double v = 0.0;
            for (int k = a; k < w; ++k) v += sm.Rinv[a * kBW + k] * sm.t[k];
            sm.mu[a] = v;
            sm.muf[a] = float(v);
        }
    }
    __syncthreads();
}

// q = A p (FP32) and (A p, p): groups of q.lanes consecutive threads take one row, their
// lanes striding through its entries, then a shuffle tree; loop bounds are uniform per warp
// so the shuffles never diverge.
__device__ float batch_spmv(const Team& T, const BatchSeqDev& q, int n)
{
    const int L = q.lanes;
    float dot = 0.0f;
    if (L <= 1) {
        for (int i = T.tid; i < n; i += T.nthr) {
            float s = 0.0f;
            for (int k = q.rp[i]; k < q.rp[i + 1]; ++k) s += q.val32[k] * q.p32[q.col[k]];
            q.q[i] = s;
            dot += s * q.p32[i];
        }
        return dot;
    }
    const int lane = T.tid & 31, gl = lane & (L - 1);
    const int gpw = 32 / L;                 // row groups per warp
    const int wg = T.tid >> 5, nw = T.nthr >> 5;
    for (int r0 = wg * gpw; r0 < n; r0 += nw * gpw) {
        const int row = r0 + lane / L;
        float s = 0.0f;
        if (row < n)
            for (int k = q.rp[row] + gl; k < q.rp[row + 1]; k += L) s += q.val32[k] * q.p32[q.col[k]];
        for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (gl == 0 && row < n) {
            q.q[row] = s;
            dot += s * q.p32[row];
        }
    }
    return dot;
}

// Update pass of one inner iteration over V rows per thread (V = 4: float4 loads of every
// vector and basis column; n a multiple of 4): d += alpha p, r -= alpha q, z = M^{-1} r,
// (r, z), ||r||^2 and c = (A W)^T z, summed into the thread's registers.
template <int V>
__device__ void batch_update(const Team& T, const BatchSeqDev& q, int n, int w, float alpha, float (&cl)[kBW],
                             float& rho_l, float& rr_l)
{
    if constexpr (V == 1) {
        for (int i = T.tid; i < n; i += T.nthr) {
            q.d[i] += alpha * q.p32[i];
            const float ri = q.r[i] - alpha * q.q[i];
            q.r[i] = ri;
            const float zi = q.dinv[i] * ri;
            rho_l += ri * zi;
            rr_l += ri * ri;
#pragma unroll
            for (int c = 0; c < kBW; ++c)
                if (c < w) cl[c] += q.AW[(size_t)c * n + i] * zi;
        }
    } else {
        const int n4 = n >> 2;
        for (int g = T.tid; g < n4; g += T.nthr) {
            float4 d4 = reinterpret_cast<const float4*>(q.d)[g];
            const float4 p4 = reinterpret_cast<const float4*>(q.p32)[g];
            float4 r4 = reinterpret_cast<const float4*>(q.r)[g];
            const float4 q4 = reinterpret_cast<const float4*>(q.q)[g];
            const float4 m4 = reinterpret_cast<const float4*>(q.dinv)[g];
            d4.x += alpha * p4.x; d4.y += alpha * p4.y; d4.z += alpha * p4.z; d4.w += alpha * p4.w;
            r4.x -= alpha * q4.x; r4.y -= alpha * q4.y; r4.z -= alpha * q4.z; r4.w -= alpha * q4.w;
            reinterpret_cast<float4*>(q.d)[g] = d4;
            reinterpret_cast<float4*>(q.r)[g] = r4;
            const float4 z4 = make_float4(m4.x * r4.x, m4.y * r4.y, m4.z * r4.z, m4.w * r4.w);
            rho_l += r4.x * z4.x + r4.y * z4.y + r4.z * z4.z + r4.w * z4.w;
            rr_l += r4.x * r4.x + r4.y * r4.y + r4.z * r4.z + r4.w * r4.w;
#pragma unroll
            for (int c = 0; c < kBW; ++c) {
                if (c < w) {
                    const float4 a = reinterpret_cast<const float4*>(q.AW + (size_t)c * n)[g];
                    cl[c] += a.x * z4.x + a.y * z4.y + a.z * z4.z + a.w * z4.w;
                }
            }
        }
    }
}

// Direction pass: p = M^{-1} r + beta p - W mu, V rows per thread as batch_update.
template <int V>
__device__ void batch_direction(const Team& T, const BatchSmem& sm, const BatchSeqDev& q, int n, int w, float beta)
{
    if constexpr (V == 1) {
        for (int i = T.tid; i < n; i += T.nthr) {
            float v = q.dinv[i] * q.r[i] + beta * q.p32[i];
#pragma unroll
            for (int c = 0; c < kBW; ++c)
                if (c < w) v -= q.W[(size_t)c * n + i] * sm.muf[c];
            q.p32[i] = v;
        }
    } else {
        const int n4 = n >> 2;
        for (int g = T.tid; g < n4; g += T.nthr) {
            const float4 r4 = reinterpret_cast<const float4*>(q.r)[g];
            const float4 m4 = reinterpret_cast<const float4*>(q.dinv)[g];
            const float4 p4 = reinterpret_cast<const float4*>(q.p32)[g];
            float4 v = make_float4(m4.x * r4.x + beta * p4.x, m4.y * r4.y + beta * p4.y, m4.z * r4.z + beta * p4.z,
                                   m4.w * r4.w + beta * p4.w);
#pragma unroll
            for (int c = 0; c < kBW; ++c) {
                if (c < w) {
                    const float4 a = reinterpret_cast<const float4*>(q.W + (size_t)c * n)[g];
                    const float m = sm.muf[c];
                    v.x -= a.x * m; v.y -= a.y * m; v.z -= a.z * m; v.w -= a.w * m;
                }
            }
            reinterpret_cast<float4*>(q.p32)[g] = v;
        }
    }
}

__device__ void solve_sequence(Team& T, BatchSmem& sm, const BatchSeqDev& q, int k_max, int max_refine,
                               double inner_tol, double rank_tol)
{
    const int n = q.n, nnz = q.nnz;
    int s_count = 0, s_next = 0;
    for (int e = threadIdx.x; e < kBS * kBS; e += blockDim.x) sm.GS[e] = 0.0;
    __syncthreads();
    for (int j = 0; j < q.p; ++j) {
        const double* val = q.val + (size_t)j * nnz;
        const double* b = q.b + (size_t)j * n;
        double* x = q.x + (size_t)j * n;
        int status = 0, iters = 0, refine = 0;
        // FP32 values and the Jacobi diagonal
        for (int i = T.tid; i < nnz; i += T.nthr) q.val32[i] = float(val[i]);
        for (int i = T.tid; i < n; i += T.nthr) {
            double dg = 0.0;
            for (int k = q.rp[i]; k < q.rp[i + 1]; ++k)
                if (q.col[k] == i) dg += val[k];
            q.dinv[i] = dg > 0.0 ? float(1.0 / dg) : 0.0f;
            if (!(dg > 0.0)) status = 2;
        }
        {
            double acc[1] = {double(status)};
            team_sum<1>(T, sm, acc, 1);
            status = sm.tot[0] > 0.0 ? 2 : 0;
        }
        // POD of the snapshots (Algorithm 4): eigensolve, truncation, lift
        int w = 0;
        if (s_count > 0) {
            if (threadIdx.x == 0) {
                for (int a = 0; a < s_count; ++a)
                    for (int c = 0; c < s_count; ++c) sm.A[a * kBS + c] = sm.GS[a * kBS + c];
                small_jacobi(sm, s_count);
                int ww = 0;
                const double lam1 = sm.ev[0];
                if (lam1 > 0.0) {
                    int rank = 0;
                    for (int i = 0; i < s_count; ++i)
                        if (sm.ev[i] > rank_tol * lam1) rank = i + 1;
                    double total = 0.0;
                    for (int i = 0; i < s_count; ++i) total += fmax(sm.ev[i], 0.0);
                    ww = rank;
                    double cum = 0.0;
                    for (int i = 0; i < rank; ++i) {
                        cum += sm.ev[i];
                        if (cum / total >= q.energy) { ww = i + 1; break; }
                    }
                    ww = min(ww, q.w_max);
                }
                for (int k = 0; k < s_count; ++k)
                    for (int c = 0; c < ww; ++c) sm.C[k * kBW + c] = sm.V[k * kBS + c] / sqrt(sm.ev[c]);
                sm.w = ww;
            }
            __syncthreads();
            w = sm.w;
            for (int i = T.tid; i < n; i += T.nthr) {
                float sv[kBS];
#pragma unroll
                for (int k = 0; k < kBS; ++k) sv[k] = (k < s_count) ? q.S32[(size_t)k * n + i] : 0.0f;
                for (int c = 0; c < w; ++c) {
                    float t = 0.0f;
#pragma unroll
                    for (int k = 0; k < kBS; ++k)
                        if (k < s_count) t += sv[k] * float(sm.C[k * kBW + c]);
                    q.W[(size_t)c * n + i] = t;
                }
            }
            T.cl.sync();
        }
        // stage one (Algorithm 2): A W, W^T [A W, b], Cholesky, x0 = W what
        if (w > 0) {
            for (int i = T.tid; i < n; i += T.nthr) {
                float acc[kBW];
#pragma unroll
                for (int c = 0; c < kBW; ++c) acc[c] = 0.0f;
                for (int k = q.rp[i]; k < q.rp[i + 1]; ++k) {
                    const float a = q.val32[k];
                    const int cc = q.col[k];
#pragma unroll
                    for (int c = 0; c < kBW; ++c)
                        if (c < w) acc[c] += a * q.W[(size_t)c * n + cc];
                }
#pragma unroll
                for (int c = 0; c < kBW; ++c)
                    if (c < w) q.AW[(size_t)c * n + i] = acc[c];
            }
            T.cl.sync();
            const int tiles = (w + 3) / 4, tiles_c = (w + 1 + 7) / 8;
            for (int ta = 0; ta < tiles; ++ta)
                for (int tc = (ta * 4) / 8; tc < tiles_c; ++tc) {
                    double acc[32];
                    float part[32];
#pragma unroll
                    for (int e = 0; e < 32; ++e) { acc[e] = 0.0; part[e] = 0.0f; }
                    int cnt = 0;
                    for (int i = T.tid; i < n; i += T.nthr) {
                        float xa[4], yc[8];
#pragma unroll
                        for (int a = 0; a < 4; ++a) xa[a] = (ta * 4 + a < w) ? q.W[(size_t)(ta * 4 + a) * n + i] : 0.0f;
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const int cc = tc * 8 + c;
                            yc[c] = (cc < w) ? q.AW[(size_t)cc * n + i] : (cc == w ? float(b[i]) : 0.0f);
                        }
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int c = 0; c < 8; ++c) part[a * 8 + c] += xa[a] * yc[c];
                        if (++cnt == 16) {
#pragma unroll
                            for (int e = 0; e < 32; ++e) { acc[e] += double(part[e]); part[e] = 0.0f; }
                            cnt = 0;
                        }
                    }
#pragma unroll
                    for (int e = 0; e < 32; ++e) acc[e] += double(part[e]);
                    team_sum<32>(T, sm, acc, 32);
                    if (threadIdx.x < 32) {
                        const int a = ta * 4 + threadIdx.x / 8, c = tc * 8 + threadIdx.x % 8;
                        if (a < w && c <= w) sm.G[a * (kBW + 1) + c] = sm.tot[threadIdx.x];
                    }
                    __syncthreads();
                }
            if (threadIdx.x == 0) sm.w = small_chol(sm, w) ? w : -1;
            __syncthreads();
            if (sm.w < 0) w = 0;   // basis not numerically SPD: plain PCG for this system
        }
        for (int i = T.tid; i < n; i += T.nthr) {
            float xi = 0.0f;
#pragma unroll
            for (int c = 0; c < kBW; ++c)
                if (c < w) xi += q.W[(size_t)c * n + i] * float(sm.what[c]);
            x[i] = double(xi);
        }
        // FP64 refinement around FP32 augmented CG (Algorithm 1 on the correction)
        double bb = 0.0, rr_true = 0.0, rr_stage1 = -1.0;
        for (int pass = 0; pass <= max_refine + 1; ++pass) {
            T.cl.sync();   // x complete
            double acc2[2] = {0.0, 0.0};
            for (int i = T.tid; i < n; i += T.nthr) {
                double s = 0.0;
                for (int k = q.rp[i]; k < q.rp[i + 1]; ++k) s += val[k] * x[q.col[k]];
                const double ri = b[i] - s;
                q.r64[i] = ri;
                acc2[0] += ri * ri;
                acc2[1] += b[i] * b[i];
            }
            team_sum<2>(T, sm, acc2, 2);
            rr_true = sm.tot[0];
            bb = sm.tot[1];
            if (rr_stage1 < 0.0) rr_stage1 = rr_true;
            const double tol2 = q.tol * q.tol * bb;
            if (status != 0 || !(rr_true > tol2)) break;
            if (!isfinite(rr_true)) { status = 5; break; }
            if (refine >= max_refine) { status = 4; break; }
            ++refine;
            // the FP32 inner solve works on r/||r|| (no underflow or overflow in FP32)
            const double rnorm = sqrt(rr_true), rinv = 1.0 / rnorm;
            // reduce r/||r|| by inner_tol, or only by half of the factor that reaches the
            // tolerance when that is the larger (the last refinement step stops where needed)
            const double tol2_in = fmax(inner_tol * inner_tol, 0.25 * tol2 / rr_true);
            // projection of the correction onto W: c = W^T r
            {
                double acc[kBW];
                float cl[kBW];
#pragma unroll
                for (int c = 0; c < kBW; ++c) cl[c] = 0.0f;
                for (int i = T.tid; i < n; i += T.nthr) {
                    const float ri = float(q.r64[i] * rinv);
                    q.r[i] = ri;
#pragma unroll
                    for (int c = 0; c < kBW; ++c)
                        if (c < w) cl[c] += q.W[(size_t)c * n + i] * ri;
                }
#pragma unroll
                for (int c = 0; c < kBW; ++c) acc[c] = double(cl[c]);
                if (w > 0) {
                    team_sum<kBW>(T, sm, acc, w);
                    apply_rinv_small(sm, w, 0);
                }
            }
            // d = W dhat, r -= AW dhat; z0, (r, z0), ||r||^2, c0 = AW^T z0
            {
                float cl[kBW];
#pragma unroll
                for (int c = 0; c < kBW; ++c) cl[c] = 0.0f;
                float rho = 0.0f, rr = 0.0f;
                for (int i = T.tid; i < n; i += T.nthr) {
                    float di = 0.0f, ai = 0.0f;
#pragma unroll
                    for (int c = 0; c < kBW; ++c) {
                        if (c < w) {
                            di += q.W[(size_t)c * n + i] * sm.muf[c];
                            ai += q.AW[(size_t)c * n + i] * sm.muf[c];
                        }
                    }
                    q.d[i] = di;
                    const float ri = q.r[i] - ai;
                    q.r[i] = ri;
                    const float zi = q.dinv[i] * ri;
                    rho += ri * zi;
                    rr += ri * ri;
#pragma unroll
                    for (int c = 0; c < kBW; ++c)
                        if (c < w) cl[c] += q.AW[(size_t)c * n + i] * zi;
                }
                double acc[kBW + 2];
                acc[0] = rho;
                acc[1] = rr;
#pragma unroll
                for (int c = 0; c < kBW; ++c) acc[2 + c] = cl[c];
                team_sum<kBW + 2>(T, sm, acc, 2 + w);
            }
            double rho = sm.tot[0], rr = sm.tot[1];
            if (w > 0) apply_rinv_small(sm, w, 2);
            for (int i = T.tid; i < n; i += T.nthr) {
                float v = q.dinv[i] * q.r[i];
#pragma unroll
                for (int c = 0; c < kBW; ++c)
                    if (c < w) v -= q.W[(size_t)c * n + i] * sm.muf[c];
                q.p32[i] = v;
            }
            bool inner_done = !(rr > tol2_in);
            while (!inner_done) {
                if (iters >= k_max) { status = 4; break; }
                T.cl.sync();   // p complete
                double acc1[1] = {0.0};
                acc1[0] = batch_spmv(T, q, n);
                team_sum<1>(T, sm, acc1, 1);
                const double gamma = sm.tot[0];
                if (!(gamma > 0.0) || !isfinite(gamma)) break;   // FP32 breakdown ends this inner pass
                const float alpha = float(rho / gamma);
                float cl[kBW];
#pragma unroll
                for (int c = 0; c < kBW; ++c) cl[c] = 0.0f;
                float rho_l = 0.0f, rr_l = 0.0f;
                if (q.vec == 4) batch_update<4>(T, q, n, w, alpha, cl, rho_l, rr_l);
                else batch_update<1>(T, q, n, w, alpha, cl, rho_l, rr_l);
                double acc[kBW + 2];
                acc[0] = rho_l;
                acc[1] = rr_l;
#pragma unroll
                for (int c = 0; c < kBW; ++c) acc[2 + c] = cl[c];
                team_sum<kBW + 2>(T, sm, acc, 2 + w);
                const double rho_new = sm.tot[0];
                rr = sm.tot[1];
                ++iters;
                if (!isfinite(rho_new) || !isfinite(rr)) break;
                const float beta = float(rho_new / rho);
                rho = rho_new;
                inner_done = !(rr > tol2_in);
                if (inner_done) break;
                if (w > 0) apply_rinv_small(sm, w, 2);
                if (q.vec == 4) batch_direction<4>(T, sm, q, n, w, beta);
                else batch_direction<1>(T, sm, q, n, w, beta);
            }
            for (int i = T.tid; i < n; i += T.nthr) x[i] += rnorm * double(q.d[i]);
            if (status != 0) break;
        }
        // statistics of system j
        if (T.rank == 0 && threadIdx.x == 0) {
            q.st_status[j] = status;
            q.st_iters[j] = iters;
            q.st_refine[j] = refine;
            q.st_w[j] = w;
            q.st_relres[j] = bb > 0.0 ? sqrt(rr_true / bb) : 0.0;
            q.st_stage1[j] = bb > 0.0 ? sqrt(fmax(rr_stage1, 0.0) / bb) : 0.0;
        }
        // record x_j as a snapshot and its Gram row (Algorithm 4 step 1)
        T.cl.sync();   // x complete
        const int slot = s_next;
        for (int i = T.tid; i < n; i += T.nthr) {
            const double v = x[i];
            q.S[(size_t)slot * n + i] = v;
            q.S32[(size_t)slot * n + i] = float(v);
        }
        s_next = (s_next + 1) % q.s_max;
        s_count = min(s_count + 1, q.s_max);
        T.cl.sync();
        {
            double acc[kBS];
#pragma unroll
            for (int k = 0; k < kBS; ++k) acc[k] = 0.0;
            for (int i = T.tid; i < n; i += T.nthr) {
                const double v = q.S[(size_t)slot * n + i];
#pragma unroll
                for (int k = 0; k < kBS; ++k)
                    if (k < s_count) acc[k] += v * q.S[(size_t)k * n + i];
            }
            team_sum<kBS>(T, sm, acc, s_count);
            if (threadIdx.x < s_count) {
                sm.GS[slot * kBS + threadIdx.x] = sm.tot[threadIdx.x];
                sm.GS[threadIdx.x * kBS + slot] = sm.tot[threadIdx.x];
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kBThreads, 1) k_batch(const BatchSeqDev* __restrict__ seqs, const int* __restrict__ order,
                                                        int nseq, unsigned int* ticket, int k_max, int max_refine,
                                                        double inner_tol, double rank_tol)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BatchSmem& sm = *reinterpret_cast<BatchSmem*>(smem_raw);
    Team T{cg::this_cluster(), 0, 0, 0, 0, 0};
    T.rank = (int)T.cl.block_rank();
    T.nctas = (int)T.cl.num_blocks();
    T.tid = T.rank * blockDim.x + threadIdx.x;
    T.nthr = T.nctas * blockDim.x;
    for (;;) {
        if (T.rank == 0 && threadIdx.x == 0) sm.seq = (int)atomicAdd(ticket, 1u);
        T.cl.sync();
        const int id = *T.cl.map_shared_rank(&sm.seq, 0);
        T.cl.sync();   // rank 0 may not take the next ticket before everyone read this one
        if (id >= nseq) break;
        unsigned long long t0 = 0, t1 = 0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        solve_sequence(T, sm, seqs[order[id]], k_max, max_refine, inner_tol, rank_tol);
        T.cl.sync();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (T.rank == 0 && threadIdx.x == 0 && seqs[order[id]].t_ns) *seqs[order[id]].t_ns = t1 - t0;
    }
    T.cl.sync();   // no CTA leaves while another may still read its shared memory
}

size_t batch_smem_bytes() { return sizeof(BatchSmem); }

cudaError_t launch_batch(const BatchSeqDev* seqs, const int* order, int nseq, unsigned int* ticket, int cluster,
                         int grid_clusters, int k_max, int max_refine, double inner_tol, double rank_tol,
                         cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BatchSmem));
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_clusters * cluster);
    cfg.blockDim = dim3(kBThreads);
    cfg.dynamicSmemBytes = sizeof(BatchSmem);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch, seqs, order, nseq, ticket, k_max, max_refine, inner_tol, rank_tol);
}

int batch_max_clusters(int cluster)
{
    cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BatchSmem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster * 64);
    cfg.blockDim = dim3(kBThreads);
    cfg.dynamicSmemBytes = sizeof(BatchSmem);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_batch, &cfg) != cudaSuccess) return 0;
    return nc;
}

}  // namespace podcg

// ======================================================================== host side

// Tile candidates of the batch autotuner: lanes per CSR row, rows per thread.
constexpr int kBatchTileCands = 4;
constexpr int kBatchTileLanes[kBatchTileCands] = {1, 1, 2, 4};
constexpr int kBatchTileVec[kBatchTileCands] = {1, 4, 4, 4};

struct pod_cg_batch_t {
    int nseq = 0, total_sys = 0;
    cudaStream_t stream = nullptr;
    pod_cg_config cfg{};
    std::vector<podcg::BatchSeqDev> hseq;
    podcg::BatchSeqDev* dseq = nullptr;
    int* dorder = nullptr;
    unsigned int* dticket = nullptr;
    unsigned char* arena = nullptr;
    int* st_i = nullptr;        // 4 x total_sys ints
    double* st_d = nullptr;     // 2 x total_sys doubles
    int cluster = 0, grid_clusters = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<float> tune_ms;   // autotuner timings for cluster 2, 4, 8
    unsigned long long* t_ns = nullptr;   // per-sequence solve time (device, nseq)
    int tile_lanes[3] = {1, 1, 1}, tile_vec[3] = {1, 1, 1};   // per size class (n < 16k, < 64k, larger)
    float tile_ms[3][kBatchTileCands] = {};                   // autotuner: per class, per candidate
    std::string err;
};

namespace {

pod_cg_status bfail(pod_cg_batch_t* h, pod_cg_status st, const std::string& m)
{
    if (h) h->err = m;
    else podcg::set_last_error(m);
    return st;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

pod_cg_status batch_build_graph(pod_cg_batch_t* h)
{
    if (h->exec) { cudaGraphExecDestroy(h->exec); h->exec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = podcg::launch_batch(h->dseq, h->dorder, h->nseq, h->dticket, h->cluster, h->grid_clusters,
                                             h->cfg.k_max, h->cfg.max_refine, h->cfg.inner_tol, h->cfg.rank_tol, cs);
        e = cudaStreamEndCapture(cs, &h->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->exec, h->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) return bfail(h, POD_CG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    return POD_CG_OK;
}

pod_cg_status batch_run(pod_cg_batch_t* h, float* ms)
{
    cudaError_t e = cudaEventRecord(h->e0, h->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(h->exec, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(h->e1);
    if (e == cudaSuccess && ms) e = cudaEventElapsedTime(ms, h->e0, h->e1);
    if (e != cudaSuccess) return bfail(h, POD_CG_ERR_CUDA, std::string("batch solve: ") + cudaGetErrorString(e));
    return POD_CG_OK;
}

int size_class(int n) { return n < 16384 ? 0 : n < 65536 ? 1 : 2; }

// Per-sequence tiles: the class's lanes, and 4 rows per thread only where n % 4 == 0.
pod_cg_status batch_apply_tiles(pod_cg_batch_t* h, const int* lanes3, const int* vec3)
{
    for (auto& d : h->hseq) {
        const int c = size_class(d.n);
        d.lanes = lanes3[c];
        d.vec = (vec3[c] == 4 && d.n % 4 == 0) ? 4 : 1;
    }
    cudaError_t e = cudaMemcpy(h->dseq, h->hseq.data(), sizeof(podcg::BatchSeqDev) * h->nseq, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(h, POD_CG_ERR_CUDA, std::string("batch tiles: ") + cudaGetErrorString(e));
    return POD_CG_OK;
}

// Tile autotuner: the whole batch runs once per candidate (lanes per row of the CSR product,
// rows per thread of the update and direction passes), every sequence timing its own solve
// on the device; each size class keeps the candidate with the least total time.
pod_cg_status batch_tune_tiles(pod_cg_batch_t* h)
{
    std::vector<unsigned long long> t(h->nseq);
    for (int k = 0; k < kBatchTileCands; ++k) {
        const int lanes3[3] = {kBatchTileLanes[k], kBatchTileLanes[k], kBatchTileLanes[k]};
        const int vec3[3] = {kBatchTileVec[k], kBatchTileVec[k], kBatchTileVec[k]};
        pod_cg_status st = batch_apply_tiles(h, lanes3, vec3);
        if (st == POD_CG_OK) st = batch_run(h, nullptr);
        if (st != POD_CG_OK) return st;
        cudaError_t e = cudaMemcpy(t.data(), h->t_ns, sizeof(unsigned long long) * h->nseq, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bfail(h, POD_CG_ERR_CUDA, std::string("batch tiles: ") + cudaGetErrorString(e));
        for (int i = 0; i < h->nseq; ++i) h->tile_ms[size_class(h->hseq[i].n)][k] += float(t[i] * 1e-6);
    }
    for (int c = 0; c < 3; ++c) {
        int best = 0;
        for (int k = 1; k < kBatchTileCands; ++k)
            if (h->tile_ms[c][k] < h->tile_ms[c][best]) best = k;
        h->tile_lanes[c] = kBatchTileLanes[best];
        h->tile_vec[c] = kBatchTileVec[best];
    }
    return batch_apply_tiles(h, h->tile_lanes, h->tile_vec);
}

pod_cg_status batch_set_cluster(pod_cg_batch_t* h, int cl)
{
    const int maxc = podcg::batch_max_clusters(cl);
    if (maxc < 1) return bfail(h, POD_CG_ERR_CUDA, "cluster size " + std::to_string(cl) + " cannot be scheduled");
    h->cluster = cl;
    h->grid_clusters = std::min(maxc, h->nseq);
    return batch_build_graph(h);
}

}  // namespace

extern "C" {

pod_cg_status pod_cg_batch_create(const pod_cg_batch_seq* seqs, int nseq, const pod_cg_config* cfg, int cluster,
                                  void* cuda_stream, pod_cg_batch_t** out)
{
    if (!out) return bfail(nullptr, POD_CG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!seqs || nseq < 1) return bfail(nullptr, POD_CG_ERR_ARG, "no sequences");
    if (cluster != 0 && cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8)
        return bfail(nullptr, POD_CG_ERR_ARG, "cluster must be 0 (autotune), 1, 2, 4 or 8");
    pod_cg_config c;
    if (cfg) c = *cfg;
    else pod_cg_config_default(&c);
    pod_cg_batch_t* h = new (std::nothrow) pod_cg_batch_t();
    if (!h) return bfail(nullptr, POD_CG_ERR_OOM, "host allocation failed");
    h->cfg = c;
    h->nseq = nseq;
    h->stream = (cudaStream_t)cuda_stream;
    // arena layout
    size_t total = 0;
    std::vector<size_t> off(nseq);
    for (int i = 0; i < nseq; ++i) {
        const pod_cg_batch_seq& q = seqs[i];
        if (q.n < 1 || q.nnz < 1 || q.nnz >= INT32_MAX || q.p < 1 || q.w_max < 1 || q.w_max > podcg::kBW ||
            q.s_max < 1 || q.s_max > podcg::kBS || !q.row_ptr || !q.col || !q.val || !q.b || !q.x ||
            !(q.tol >= 0.0) || !(q.energy >= 0.0 && q.energy <= 1.0)) {
            delete h;
            return bfail(nullptr, POD_CG_ERR_ARG, "bad sequence " + std::to_string(i) +
                                                      " (n, nnz, p >= 1; w_max <= 32; s_max <= 16; pointers)");
        }
        off[i] = total;
        const size_t n = q.n;
        total += align256(8 * n * q.s_max) + align256(4 * n * q.s_max) + 2 * align256(4 * n * q.w_max) +
                 align256(4 * (size_t)q.nnz) + align256(8 * n) + 5 * align256(4 * n);
        h->total_sys += q.p;
    }
    cudaError_t e = cudaMalloc((void**)&h->arena, std::max<size_t>(total, 256));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->st_i, sizeof(int) * 4 * h->total_sys);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->st_d, sizeof(double) * 2 * h->total_sys);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->dseq, sizeof(podcg::BatchSeqDev) * nseq);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->dorder, sizeof(int) * nseq);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->dticket, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->t_ns, sizeof(unsigned long long) * nseq);
    if (e == cudaSuccess) e = cudaEventCreate(&h->e0);
    if (e == cudaSuccess) e = cudaEventCreate(&h->e1);
    if (e != cudaSuccess) {
        pod_cg_status st = bfail(nullptr, e == cudaErrorMemoryAllocation ? POD_CG_ERR_OOM : POD_CG_ERR_CUDA,
                                 std::string("batch create: ") + cudaGetErrorString(e));
        pod_cg_batch_destroy(h);
        return st;
    }
    h->hseq.resize(nseq);
    int sys_off = 0;
    for (int i = 0; i < nseq; ++i) {
        const pod_cg_batch_seq& q = seqs[i];
        podcg::BatchSeqDev& d = h->hseq[i];
        const size_t n = q.n;
        unsigned char* a = h->arena + off[i];
        auto take = [&](size_t bytes) { unsigned char* r = a; a += align256(bytes); return r; };
        d.n = q.n; d.nnz = (int)q.nnz; d.p = q.p; d.w_max = q.w_max; d.s_max = q.s_max;
        d.tol = q.tol; d.energy = q.energy;
        d.rp = q.row_ptr; d.col = q.col; d.val = q.val; d.b = q.b; d.x = q.x;
        d.S = (double*)take(8 * n * q.s_max);
        d.S32 = (float*)take(4 * n * q.s_max);
        d.W = (float*)take(4 * n * q.w_max);
        d.AW = (float*)take(4 * n * q.w_max);
        d.val32 = (float*)take(4 * (size_t)q.nnz);
        d.r64 = (double*)take(8 * n);
        d.r = (float*)take(4 * n);
        d.p32 = (float*)take(4 * n);
        d.q = (float*)take(4 * n);
        d.d = (float*)take(4 * n);
        d.dinv = (float*)take(4 * n);
        d.lanes = 1;
        d.vec = 1;
        d.t_ns = h->t_ns + i;
        d.st_status = h->st_i + 0 * h->total_sys + sys_off;
        d.st_iters = h->st_i + 1 * h->total_sys + sys_off;
        d.st_refine = h->st_i + 2 * h->total_sys + sys_off;
        d.st_w = h->st_i + 3 * h->total_sys + sys_off;
        d.st_relres = h->st_d + 0 * h->total_sys + sys_off;
        d.st_stage1 = h->st_d + 1 * h->total_sys + sys_off;
        sys_off += q.p;
    }
    // longest estimated work first: nnz * p * n^(1/3) (CG iterations grow with the grid edge)
    std::vector<int> order(nseq);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double wa = double(seqs[a].nnz) * seqs[a].p * std::cbrt(double(seqs[a].n));
        const double wb = double(seqs[b].nnz) * seqs[b].p * std::cbrt(double(seqs[b].n));
        return wa > wb;
    });
    e = cudaMemcpy(h->dseq, h->hseq.data(), sizeof(podcg::BatchSeqDev) * nseq, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->dorder, order.data(), sizeof(int) * nseq, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pod_cg_status st = bfail(nullptr, POD_CG_ERR_CUDA, std::string("batch create: ") + cudaGetErrorString(e));
        pod_cg_batch_destroy(h);
        return st;
    }
    pod_cg_status st;
    if (cluster != 0) {
        st = batch_set_cluster(h, cluster);
    } else {
        // autotuner: time the whole batch once per cluster size, keep the fastest
        const int cands[3] = {2, 4, 8};
        float best = 0.0f;
        int best_cl = 0;
        st = POD_CG_OK;
        for (int k = 0; k < 3 && st == POD_CG_OK; ++k) {
            if (batch_set_cluster(h, cands[k]) != POD_CG_OK) {
                h->tune_ms.push_back(-1.0f);
                continue;
            }
            float ms = 0.0f;
            st = batch_run(h, &ms);
            h->tune_ms.push_back(ms);
            if (st == POD_CG_OK && (best_cl == 0 || ms < best)) { best = ms; best_cl = cands[k]; }
        }
        if (st == POD_CG_OK) st = best_cl ? batch_set_cluster(h, best_cl) : bfail(h, POD_CG_ERR_CUDA, "no cluster size runs");
        if (st == POD_CG_OK) st = batch_tune_tiles(h);
    }
    if (st != POD_CG_OK) {
        podcg::set_last_error(h->err);
        pod_cg_batch_destroy(h);
        return st;
    }
    *out = h;
    return POD_CG_OK;
}

pod_cg_status pod_cg_batch_solve(pod_cg_batch_t* h, pod_cg_batch_sysstat* stats, float* ms)
{
    if (!h) return bfail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    pod_cg_status st = batch_run(h, ms);
    if (st != POD_CG_OK) return st;
    int worst = 0;
    if (stats) {
        std::vector<int> si(4 * (size_t)h->total_sys);
        std::vector<double> sd(2 * (size_t)h->total_sys);
        cudaError_t e = cudaMemcpy(si.data(), h->st_i, sizeof(int) * si.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(sd.data(), h->st_d, sizeof(double) * sd.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bfail(h, POD_CG_ERR_CUDA, std::string("batch stats: ") + cudaGetErrorString(e));
        const int T = h->total_sys;
        for (int k = 0; k < T; ++k) {
            stats[k].status = si[k];
            stats[k].iters = si[T + k];
            stats[k].refinements = si[2 * T + k];
            stats[k].w = si[3 * T + k];
            stats[k].final_relres = sd[k];
            stats[k].stage1_relres = sd[T + k];
            if (si[k] != 0 && worst == 0) worst = si[k];
        }
    }
    if (worst != 0) return bfail(h, (pod_cg_status)worst, "a system of the batch did not converge (see its stats)");
    return POD_CG_OK;
}

pod_cg_status pod_cg_batch_info(const pod_cg_batch_t* h, int* cluster, int* workers, float* tune_ms3)
{
    if (!h) return POD_CG_ERR_ARG;
    if (cluster) *cluster = h->cluster;
    if (workers) *workers = h->grid_clusters;
    if (tune_ms3)
        for (int k = 0; k < 3; ++k) tune_ms3[k] = k < (int)h->tune_ms.size() ? h->tune_ms[k] : 0.0f;
    return POD_CG_OK;
}

pod_cg_status pod_cg_batch_set_tiles(pod_cg_batch_t* h, const int* lanes3, const int* rows3)
{
    if (!h || !lanes3 || !rows3) return bfail(h, POD_CG_ERR_ARG, "pod_cg_batch_set_tiles: NULL argument");
    for (int c = 0; c < 3; ++c) {
        const int L = lanes3[c], r = rows3[c];
        if (!(L == 1 || L == 2 || L == 4 || L == 8) || !(r == 1 || r == 4))
            return bfail(h, POD_CG_ERR_ARG, "pod_cg_batch_set_tiles: lanes 1, 2, 4 or 8 and rows 1 or 4");
    }
    for (int c = 0; c < 3; ++c) {
        h->tile_lanes[c] = lanes3[c];
        h->tile_vec[c] = rows3[c];
    }
    return batch_apply_tiles(h, h->tile_lanes, h->tile_vec);
}

pod_cg_status pod_cg_batch_tiles(const pod_cg_batch_t* h, int* lanes3, int* rows3, float* ms12)
{
    if (!h) return POD_CG_ERR_ARG;
    for (int c = 0; c < 3; ++c) {
        if (lanes3) lanes3[c] = h->tile_lanes[c];
        if (rows3) rows3[c] = h->tile_vec[c];
        if (ms12)
            for (int k = 0; k < kBatchTileCands; ++k) ms12[c * kBatchTileCands + k] = h->tile_ms[c][k];
    }
    return POD_CG_OK;
}

const char* pod_cg_batch_last_error(const pod_cg_batch_t* h) { return h ? h->err.c_str() : ""; }

pod_cg_status pod_cg_batch_destroy(pod_cg_batch_t* h)
{
    if (!h) return POD_CG_OK;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    void* bufs[] = {h->arena, h->st_i, h->st_d, h->dseq, h->dorder, h->dticket, h->t_ns};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (h->e0) cudaEventDestroy(h->e0);
    if (h->e1) cudaEventDestroy(h->e1);
    delete h;
    return POD_CG_OK;
}

}  // extern "C"
