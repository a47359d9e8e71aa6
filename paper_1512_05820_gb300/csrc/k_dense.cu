// Tall-skinny and small dense kernels of the POD-augmented path:
//   - Gram G = X^T Y of n-by-p and n-by-q column-major blocks (split over rows, then a
//     fixed-order sum of the splits): the snapshot Gram S^T S (Algorithm 4 step 1) and
//     the reduced matrix W^T [A W, b] (Algorithm 2 step 1);
//   - lift W = S C with C = V_w Sigma_w^{-1} (Algorithm 4 step 4);
//   - stage-one lift x0 = W what, r0 = b - (A W) what (Algorithm 2 then Algorithm 1 steps
//     1-2 with xbar = 0; A x0 = (A W) what needs no extra product);
//   - one-block kernels: Cholesky R^T R = W^T A W with R^{-1} and the stage-one solve
//     (Algorithm 2 step 2), and the symmetric eigensolve of S^T S by parallel cyclic
//     Jacobi (Brent-Luk round-robin ordering of disjoint rotations), energy truncation
//     and the lift coefficients (Algorithm 4 steps 2-3).
#include "common.cuh"
#include "launch.h"

namespace podcg {

constexpr int kTile = 8;   // Gram output tile edge (8x8 accumulators per thread)

// One split of the rows [r0, r1) for one TI x 8 output tile (TI = 8, or 1 for a single
// row such as a new snapshot's Gram row). Y column qy (if `extra`) is the extra vector
// (the right-hand side b of stage one). Partials are stored 8x8 per tile either way.
template <int TI>
__global__ void __launch_bounds__(kBlock) k_gram_partial(int n, const double* __restrict__ X, int ldx, int p,
                                                         const double* __restrict__ Y, int ldy, int qy,
                                                         const double* __restrict__ extra, int q,
                                                         int tiles_j, int upper_only, int rows_per_split,
                                                         double* __restrict__ partials)
{
    int tile = blockIdx.x;
    const int ti = tile / tiles_j, tj = tile % tiles_j;
    const int split = blockIdx.y;
    const int a0 = ti * kTile, c0 = tj * kTile;
    double* out = partials + ((size_t)split * gridDim.x + tile) * (kTile * kTile);
    // upper_only: W^T A W is symmetric; tiles strictly below the diagonal (except the
    // extra right-hand-side column) are not needed by the Cholesky.
    const bool skip = upper_only && (c0 + kTile <= a0) && !(extra && c0 + kTile > qy);
    double acc[kTile * kTile];
#pragma unroll
    for (int e = 0; e < kTile * kTile; ++e) acc[e] = 0.0;
    if (!skip) {
        const double* xp[kTile];
        const double* yp[kTile];
#pragma unroll
        for (int a = 0; a < kTile; ++a) xp[a] = (a < TI && a0 + a < p) ? X + (size_t)(a0 + a) * ldx : nullptr;
#pragma unroll
        for (int c = 0; c < kTile; ++c) {
            const int cc = c0 + c;
            yp[c] = (cc < qy) ? Y + (size_t)cc * ldy : ((extra && cc == qy && cc < q) ? extra : nullptr);
        }
        const int r0 = split * rows_per_split;
        const int r1 = min(n, r0 + rows_per_split);
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            double xv[kTile], yv[kTile];
#pragma unroll
            for (int a = 0; a < TI; ++a) xv[a] = xp[a] ? __ldg(xp[a] + i) : 0.0;
#pragma unroll
            for (int c = 0; c < kTile; ++c) yv[c] = yp[c] ? __ldg(yp[c] + i) : 0.0;
#pragma unroll
            for (int a = 0; a < TI; ++a)
#pragma unroll
                for (int c = 0; c < kTile; ++c) acc[a * kTile + c] += xv[a] * yv[c];
        }
    }
    __shared__ double s_w[kWarps][kTile * kTile];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < kTile * kTile; ++e) {
        const double t = (e < TI * kTile) ? warp_sum(acc[e]) : 0.0;
        if (lane == 0) s_w[wid][e] = t;
    }
    __syncthreads();
    if (threadIdx.x < kTile * kTile) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) t += s_w[k][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// G[a][c] = sum over splits in split order (deterministic). G row-major p x q with row
// stride ldg.
// One warp per output element; lanes take the splits in a fixed interleaved order and a
// fixed shuffle tree combines them (deterministic).
__global__ void k_gram_reduce(const double* __restrict__ partials, int splits, int tiles, int tiles_j,
                              int p, int q, double* __restrict__ G, int ldg)
{
    const int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (idx >= p * q) return;   // uniform per warp
    const int a = idx / q, c = idx % q;
    const int tile = (a / kTile) * tiles_j + (c / kTile);
    const int e = (a % kTile) * kTile + (c % kTile);
    double t = 0.0;
    for (int s = lane; s < splits; s += 32) t += partials[((size_t)s * tiles + tile) * (kTile * kTile) + e];
    t = warp_sum(t);
    if (lane == 0) G[(size_t)a * ldg + c] = t;
}

void gram_shape(int n, int p, int q, int sms, int* tiles_j, int* tiles, int* splits, int* rows_per_split)
{
    *tiles_j = (q + kTile - 1) / kTile;
    *tiles = ((p + kTile - 1) / kTile) * (*tiles_j);
    int want = (sms * 4 + *tiles - 1) / *tiles;
    int maxs = (n + 255) / 256;
    if (want > maxs) want = maxs;
    if (want < 1) want = 1;
    int rps = (n + want - 1) / want;
    rps = ((rps + 31) / 32) * 32;
    if (rps < 32) rps = 32;
    *rows_per_split = rps;
    *splits = (n + rps - 1) / rps;
    if (*splits < 1) *splits = 1;
}

size_t gram_workspace_bytes(int n, int p, int q, int sms)
{
    int tj, tiles, splits, rps;
    gram_shape(n, p, q, sms, &tj, &tiles, &splits, &rps);
    return (size_t)splits * tiles * kTile * kTile * sizeof(double);
}

cudaError_t launch_gram(int n, const double* X, int ldx, int p, const double* Y, int ldy, int qy,
                        const double* extra, double* G, int ldg, int upper_only, double* work,
                        size_t work_bytes, int sms, cudaStream_t s)
{
    const int q = qy + (extra ? 1 : 0);
    if (p <= 0 || q <= 0) return cudaSuccess;
    int tj, tiles, splits, rps;
    gram_shape(n, p, q, sms, &tj, &tiles, &splits, &rps);
    if ((size_t)splits * tiles * kTile * kTile * sizeof(double) > work_bytes) return cudaErrorInvalidValue;
    dim3 grid(tiles, splits);
    if (p == 1) k_gram_partial<1><<<grid, kBlock, 0, s>>>(n, X, ldx, p, Y, ldy, qy, extra, q, tj, upper_only, rps, work);
    else k_gram_partial<8><<<grid, kBlock, 0, s>>>(n, X, ldx, p, Y, ldy, qy, extra, q, tj, upper_only, rps, work);
    return launch_gram_reduce(work, splits, tiles, tj, p, q, G, ldg, s);
}

cudaError_t launch_gram_reduce(const double* work, int splits, int tiles, int tj, int p, int q, double* G, int ldg,
                               cudaStream_t s)
{
    const int m = p * q;
    k_gram_reduce<<<(m * 32 + 127) / 128, 128, 0, s>>>(work, splits, tiles, tj, p, q, G, ldg);
    return cudaGetLastError();
}

// W[:, j] = sum_k S[:, k] C[k][j], k < s, j < w (w = st->pod_w, or st->pod_y when cols_y:
// the augmenting basis Y). C row-major s x w (row stride kWMax).
template <int SB>
__global__ void __launch_bounds__(kBlock) k_lift(int n, const double* __restrict__ S, int lds, int s,
                                                 const double* __restrict__ C, const DevState* st,
                                                 double* __restrict__ W, int ldw, int cols_y)
{
    __shared__ double sC[SB * kWMax];
    const int w = cols_y ? st->pod_y : st->pod_w;
    for (int e = threadIdx.x; e < s * kWMax; e += blockDim.x) sC[e] = C[e];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double sv[SB];
#pragma unroll
        for (int k = 0; k < SB; ++k) sv[k] = (k < s) ? __ldg(S + (size_t)k * lds + i) : 0.0;
        for (int j = 0; j < w; ++j) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < SB; ++k)
                if (k < s) t += sv[k] * sC[k * kWMax + j];
            W[(size_t)j * ldw + i] = t;
        }
    }
}

cudaError_t launch_lift(int n, const double* S, int lds, int s, const double* C, const DevState* st,
                        double* W, int ldw, int sms, cudaStream_t str, int cols_y)
{
    const int grid = grid_rows(n, kBlock, sms);
    if (s <= 8) k_lift<8><<<grid, kBlock, 0, str>>>(n, S, lds, s, C, st, W, ldw, cols_y);
    else if (s <= 16) k_lift<16><<<grid, kBlock, 0, str>>>(n, S, lds, s, C, st, W, ldw, cols_y);
    else if (s <= 32) k_lift<32><<<grid, kBlock, 0, str>>>(n, S, lds, s, C, st, W, ldw, cols_y);
    else if (s <= 48) k_lift<48><<<grid, kBlock, 0, str>>>(n, S, lds, s, C, st, W, ldw, cols_y);
    else k_lift<64><<<grid, kBlock, 0, str>>>(n, S, lds, s, C, st, W, ldw, cols_y);
    return cudaGetLastError();
}

// Stage-one lift: x = W what, r = b - (A W) what; ||r||^2 and ||b||^2. The last block sets
// the tolerances (tol2 = tol^2 ||b||^2) and the stage-one residual.
template <int WB>
__global__ void __launch_bounds__(kBlock) k_stage1(const ProbDesc* __restrict__ pd, const double* __restrict__ W,
                                                   const double* __restrict__ AW, double* __restrict__ x,
                                                   double* __restrict__ r, double* __restrict__ partials,
                                                   unsigned int* counter, DevState* st, double tol)
{
    const int n = pd->n, ld = pd->ld;
    const int w = st->w;
    const double* b = pd->b;
    __shared__ double s_what[WB > 0 ? WB : 1];
    for (int j = threadIdx.x; j < WB; j += blockDim.x) s_what[j] = (j < w) ? st->what[j] : 0.0;
    __syncthreads();
    double rr = 0.0, bb = 0.0;
    double wh[WB > 0 ? WB : 1];
#pragma unroll
    for (int j = 0; j < WB; ++j) wh[j] = (WB > 0) ? s_what[j] : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double xi = 0.0, ai = 0.0;
#pragma unroll
        for (int j = 0; j < WB; ++j) {
            if (j < w) {
                xi += __ldg(W + (size_t)j * ld + i) * wh[j];
                ai += __ldg(AW + (size_t)j * ld + i) * wh[j];
            }
        }
        const double bi = b[i];
        const double ri = bi - ai;
        x[i] = xi;
        r[i] = ri;
        rr += ri * ri;
        bb += bi * bi;
    }
    double acc[2] = {rr, bb};
    __shared__ double tot[2];
    if (reduce_to_last_block<2>(acc, 2, partials, counter, tot) && threadIdx.x == 0) {
        st->rr = tot[0];
        st->rr_stage1 = tot[0];
        st->rr_outer = tot[0];
        st->bb = tot[1];
        st->tol2 = tol * tol * tot[1];
        st->tol2_in = st->tol2;
    }
}

cudaError_t launch_stage1(int wb, const ProbDesc* pd, int n, const double* W, const double* AW, double* x,
                          double* r, double* partials, unsigned int* counter, DevState* st, double tol, int sms,
                          cudaStream_t s)
{
    const int grid = grid_rows(n, kBlock, sms);
    if (wb <= 0) k_stage1<0><<<grid, kBlock, 0, s>>>(pd, W, AW, x, r, partials, counter, st, tol);
    else if (wb <= 8) k_stage1<8><<<grid, kBlock, 0, s>>>(pd, W, AW, x, r, partials, counter, st, tol);
    else if (wb <= 16) k_stage1<16><<<grid, kBlock, 0, s>>>(pd, W, AW, x, r, partials, counter, st, tol);
    else if (wb <= 32) k_stage1<32><<<grid, kBlock, 0, s>>>(pd, W, AW, x, r, partials, counter, st, tol);
    else if (wb <= 48) k_stage1<48><<<grid, kBlock, 0, s>>>(pd, W, AW, x, r, partials, counter, st, tol);
    else k_stage1<64><<<grid, kBlock, 0, s>>>(pd, W, AW, x, r, partials, counter, st, tol);
    return cudaGetLastError();
}

// ------------------------------------------------------------ one-block small kernels

// Parallel cyclic Jacobi on the symmetric m x m matrix A (shared memory, row stride kSMax),
// accumulating the rotations into V. m is even (callers pad an odd order with a zero row
// and column). One sweep applies m-1 rounds of m/2 disjoint rotations (round-robin pairs);
// each rotation is the 2x2 symmetric Schur rotation that zeroes A[p][q]. Stops when the
// off-diagonal Frobenius norm^2 <= 1e-32 * ||A||_F^2 or after max_sweeps sweeps.
__device__ int jacobi_parallel(double* A, double* V, int m, int max_sweeps, int* pos, double* cs, double* sn,
                               int* pp, int* qq, double* red)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < m * kSMax; e += nt) {
        const int i = e / kSMax, j = e % kSMax;
        if (j < m) V[e] = (i == j) ? 1.0 : 0.0;
    }
    // Frobenius norm^2 and off-diagonal norm^2 by a block reduction (fixed order)
    auto block_norms = [&](double* total, double* offd) {
        __shared__ double s_p[2][kBlock / 32];
        double t = 0.0, o = 0.0;
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, j = e % m;
            const double v = A[i * kSMax + j];
            t += v * v;
            if (i != j) o += v * v;
        }
        t = warp_sum(t);
        o = warp_sum(o);
        if ((tid & 31) == 0) {
            s_p[0][tid >> 5] = t;
            s_p[1][tid >> 5] = o;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < nt / 32; ++k) {
                a += s_p[0][k];
                b += s_p[1][k];
            }
            red[0] = a;
            red[1] = b;
        }
        __syncthreads();
        *total = red[0];
        *offd = red[1];
        __syncthreads();
    };
    double fro = 0.0, off0 = 0.0;
    __syncthreads();
    block_norms(&fro, &off0);
    int sweep = 0;
    const int half = m / 2;
    for (; sweep < max_sweeps; ++sweep) {
        double tot_unused = 0.0, off = 0.0;
        block_norms(&tot_unused, &off);
        if (off <= 1e-32 * fro || off == 0.0) break;
        for (int i = tid; i < m; i += nt) pos[i] = i;
        __syncthreads();
        for (int round = 0; round < m - 1; ++round) {
            for (int k = tid; k < half; k += nt) {
                int p = pos[k], q = pos[m - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                pp[k] = p;
                qq[k] = q;
                const double apq = A[p * kSMax + q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    const double theta = (A[q * kSMax + q] - A[p * kSMax + p]) / (2.0 * apq);
                    const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            // columns p, q of A and of V
            for (int e = tid; e < half * m; e += nt) {
                const int k = e / m, r = e % m;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                const double ap = A[r * kSMax + p], aq = A[r * kSMax + q];
                A[r * kSMax + p] = c * ap - s * aq;
                A[r * kSMax + q] = s * ap + c * aq;
                const double vp = V[r * kSMax + p], vq = V[r * kSMax + q];
                V[r * kSMax + p] = c * vp - s * vq;
                V[r * kSMax + q] = s * vp + c * vq;
            }
            __syncthreads();
            // rows p, q of A
            for (int e = tid; e < half * m; e += nt) {
                const int k = e / m, r = e % m;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                const double ap = A[p * kSMax + r], aq = A[q * kSMax + r];
                A[p * kSMax + r] = c * ap - s * aq;
                A[q * kSMax + r] = s * ap + c * aq;
            }
            __syncthreads();
            // round-robin: position 0 fixed, the others rotate by one
            if (tid == 0) {
                const int last = pos[m - 1];
                for (int i = m - 1; i > 1; --i) pos[i] = pos[i - 1];
                pos[1] = last;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    return sweep;
}

// Sort eigenvalues (diagonal of A, first `s` entries) decreasingly by rank counting and
// write ev[s] and the matching columns of V into Vs (row stride kSMax), each signed so its
// entry of largest magnitude (first such index) is positive.
__device__ void sort_eigs(const double* A, const double* V, int s, double* ev, double* Vs, int* order)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < s; i += nt) {
        const double li = A[i * kSMax + i];
        int rank = 0;
        for (int j = 0; j < s; ++j) {
            const double lj = A[j * kSMax + j];
            if (lj > li || (lj == li && j < i)) ++rank;
        }
        order[rank] = i;
    }
    __syncthreads();
    for (int i = tid; i < s; i += nt) {
        const int src = order[i];
        ev[i] = A[src * kSMax + src];
        int arg = 0;
        for (int k = 1; k < s; ++k)
            if (fabs(V[k * kSMax + src]) > fabs(V[arg * kSMax + src])) arg = k;
        const double sg = V[arg * kSMax + src] < 0.0 ? -1.0 : 1.0;
        for (int k = 0; k < s; ++k) Vs[k * kSMax + i] = sg * V[k * kSMax + src];
    }
    __syncthreads();
}

struct SmallSmem {
    double A[kSMax * kSMax];
    double V[kSMax * kSMax];
    double Vs[kSMax * kSMax];
    double T[kSMax * kSMax];
    double ev[kSMax];
    double cs[kSMax / 2], sn[kSMax / 2];
    double red[4];
    int pos[kSMax], pp[kSMax / 2], qq[kSMax / 2], order[kSMax];
};

// POD of the snapshot Gram (Algorithm 4 steps 2-3): eigen-decompose G (s x s, row stride
// kSMax), numerical rank = #{lambda_i > rank_tol lambda_1}, w = smallest index <= rank with
// cumulative energy >= energy, capped at w_max; C[k][j] = v_j[k]/sigma_j (row stride kWMax);
// sigma2[i] = lambda_i. w is written to st->pod_w (and st->w). With y_max > 0 (three-stage
// mode) the augmenting-basis dimension y is chosen the same way with energy_y, capped at
// y_max and raised to w (POD bases are nested, so W is then the first w columns of Y), and
// written to st->pod_y; C then has max(w, y) columns.
//
// Warm start: successive snapshot Grams differ in one row and column, so when the
// eigenvectors of the previous Gram (Vprev, its first prev_s slots) are given, the
// matrix is first rotated to A' = V0^T G V0 with V0 = blockdiag(Vprev, I), which is
// nearly diagonal, Jacobi runs on A', and the eigenvectors are mapped back, V = V0 V'.
// Same eigenpairs (up to rounding) in far fewer sweeps. Vprev receives the new sorted
// eigenvectors for the next call.
__global__ void __launch_bounds__(kBlock) k_pod_eig(const double* __restrict__ G, int ldg, int s, double energy,
                                                    double rank_tol, int w_max, double* __restrict__ C,
                                                    double* __restrict__ sigma2, DevState* st,
                                                    double* __restrict__ Vprev, int prev_s, double energy_y,
                                                    int y_max)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallSmem& sm = *reinterpret_cast<SmallSmem*>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int m = s + (s & 1);
    const bool warm = Vprev != nullptr && prev_s > 0 && prev_s <= s;
    for (int e = tid; e < kSMax * kSMax; e += nt) {
        const int i = e / kSMax, j = e % kSMax;
        sm.A[e] = (i < s && j < s) ? G[(size_t)i * ldg + j] : 0.0;
        if (warm) {
            double v0 = (i == j) ? 1.0 : 0.0;
            if (i < prev_s && j < prev_s) v0 = Vprev[e];
            sm.Vs[e] = (i < s && j < s) ? v0 : 0.0;   // V0
        }
    }
    __syncthreads();
    if (warm) {
        // V = G V0 (in V), then A = V0^T V
        for (int e = tid; e < s * s; e += nt) {
            const int i = e / s, j = e % s;
            double t = 0.0;
            for (int k = 0; k < s; ++k) t += sm.A[i * kSMax + k] * sm.Vs[k * kSMax + j];
            sm.V[i * kSMax + j] = t;
        }
        __syncthreads();
        for (int e = tid; e < s * s; e += nt) {
            const int i = e / s, j = e % s;
            double t = 0.0;
            for (int k = 0; k < s; ++k) t += sm.Vs[k * kSMax + i] * sm.V[k * kSMax + j];
            sm.A[i * kSMax + j] = t;
        }
        __syncthreads();
        // symmetrise the rotated matrix (rounding)
        for (int e = tid; e < s * s; e += nt) {
            const int i = e / s, j = e % s;
            if (i < j) {
                const double v = 0.5 * (sm.A[i * kSMax + j] + sm.A[j * kSMax + i]);
                sm.A[i * kSMax + j] = v;
                sm.A[j * kSMax + i] = v;
            }
        }
        __syncthreads();
    }
    if (s > 0) jacobi_parallel(sm.A, sm.V, m, 40, sm.pos, sm.cs, sm.sn, sm.pp, sm.qq, sm.red);
    if (warm) {
        // V <- V0 V' (V0 in Vs, V' in V, product through T)
        for (int e = tid; e < s * s; e += nt) {
            const int i = e / s, j = e % s;
            double t = 0.0;
            for (int k = 0; k < s; ++k) t += sm.Vs[i * kSMax + k] * sm.V[k * kSMax + j];
            sm.T[i * kSMax + j] = t;
        }
        __syncthreads();
        for (int e = tid; e < s * s; e += nt) {
            const int i = e / s, j = e % s;
            sm.V[i * kSMax + j] = sm.T[i * kSMax + j];
        }
        __syncthreads();
    }
    sort_eigs(sm.A, sm.V, s, sm.ev, sm.Vs, sm.order);
    if (Vprev)
        for (int e = tid; e < kSMax * kSMax; e += nt) {
            const int i = e / kSMax, j = e % kSMax;
            Vprev[e] = (i < s && j < s) ? sm.Vs[i * kSMax + j] : 0.0;
        }
    __shared__ int s_w;
    if (tid == 0) {
        int w = 0, y = 0;
        if (s > 0 && sm.ev[0] > 0.0) {
            const double lam1 = sm.ev[0];
            int rank = 0;
            for (int i = 0; i < s; ++i)
                if (sm.ev[i] > rank_tol * lam1) rank = i + 1;
            double total = 0.0;
            for (int i = 0; i < s; ++i) total += fmax(sm.ev[i], 0.0);
            w = rank;
            y = rank;
            double cum = 0.0;
            bool got_w = false, got_y = false;
            for (int i = 0; i < rank && !(got_w && got_y); ++i) {
                cum += sm.ev[i];
                if (!got_w && cum / total >= energy) { w = i + 1; got_w = true; }
                if (!got_y && cum / total >= energy_y) { y = i + 1; got_y = true; }
            }
            if (w > w_max) w = w_max;
            // the augmenting basis (three-stage mode) holds the stage-one basis: y >= w
            if (y > y_max) y = y_max;
            if (y_max > 0 && y < w) y = w;
            if (y_max <= 0) y = 0;
        }
        s_w = y > w ? y : w;
        st->pod_w = w;
        st->w = w;
        st->pod_y = y;
    }
    __syncthreads();
    const int nc = s_w;   // columns of C: max(w, y)
    for (int i = tid; i < s; i += nt) sigma2[i] = sm.ev[i];
    for (int e = tid; e < s * kWMax; e += nt) {
        const int k = e / kWMax, j = e % kWMax;
        C[e] = (j < nc) ? sm.Vs[k * kSMax + j] / sqrt(sm.ev[j]) : 0.0;
    }
}

size_t pod_eig_smem_bytes() { return sizeof(SmallSmem); }

cudaError_t launch_pod_eig(const double* G, int ldg, int s, double energy, double rank_tol, int w_max, double* C,
                           double* sigma2, DevState* st, double* Vprev, int prev_s, cudaStream_t str,
                           double energy_y, int y_max)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_pod_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(SmallSmem));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_pod_eig<<<1, kBlock, sizeof(SmallSmem), str>>>(G, ldg, s, energy, rank_tol, w_max, C, sigma2, st, Vprev, prev_s,
                                                     energy_y, y_max);
    return cudaGetLastError();
}

// Previous weights of the accumulated Krylov vectors (Section 3.2, Eq. (weightsPrevious) with
// x_bar = 0): coords = (Z^T A Z)^+ Z^T b from G = Z^T [A Z, b] (z x (z + 1), row-major, row
// stride ldg). The symmetric part of Z^T A Z is eigen-decomposed by the parallel Jacobi
// method; eigenvalues of magnitude below rcond * max |lambda| count as zero (the minimum-norm
// least-squares solution: the directions of several systems can be nearly dependent; a
// singular value at or below the cut-off is dropped). The
// weights for the next compression follow: weights 0 (Eq. (weightsRBF), rho(r) = 2^-(r-1)):
// eta <- coords + eta / 2 (the older coordinates, zero-padded, halve with each newer system);
// weights 1 (previous weights alone): eta <- coords. eta holds kSMax entries, zero past z.
__global__ void __launch_bounds__(kBlock) k_krylov_coords(const double* __restrict__ G, int ldg, int z, double rcond,
                                                          double* __restrict__ coords, double* __restrict__ eta,
                                                          int rbf)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallSmem& sm = *reinterpret_cast<SmallSmem*>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int m = z + (z & 1);
    double* rhs = sm.T;              // Z^T b
    double* t = sm.T + kSMax;        // V^T Z^T b / lambda
    __shared__ double s_cut;
    for (int e = tid; e < kSMax * kSMax; e += nt) {
        const int i = e / kSMax, j = e % kSMax;
        sm.A[e] = (i < z && j < z) ? 0.5 * (G[(size_t)i * ldg + j] + G[(size_t)j * ldg + i]) : 0.0;
    }
    for (int i = tid; i < kSMax; i += nt) rhs[i] = (i < z) ? G[(size_t)i * ldg + z] : 0.0;
    __syncthreads();
    if (z > 0) jacobi_parallel(sm.A, sm.V, m, 60, sm.pos, sm.cs, sm.sn, sm.pp, sm.qq, sm.red);
    if (tid == 0) {
        double lmax = 0.0;
        for (int i = 0; i < z; ++i) lmax = fmax(lmax, fabs(sm.A[i * kSMax + i]));
        s_cut = rcond * lmax;
    }
    __syncthreads();
    for (int k = tid; k < z; k += nt) {
        const double lam = sm.A[k * kSMax + k];
        double v = 0.0;
        for (int j = 0; j < z; ++j) v += sm.V[j * kSMax + k] * rhs[j];
        t[k] = (fabs(lam) > s_cut) ? v / lam : 0.0;
    }
    __syncthreads();
    for (int i = tid; i < kSMax; i += nt) {
        double c = 0.0;
        if (i < z)
            for (int k = 0; k < z; ++k) c += sm.V[i * kSMax + k] * t[k];
        coords[i] = c;
        eta[i] = rbf ? c + 0.5 * eta[i] : c;
    }
}

cudaError_t launch_krylov_coords(const double* G, int ldg, int z, double rcond, double* coords, double* eta, int rbf,
                                 cudaStream_t str)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_krylov_coords, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(SmallSmem));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_krylov_coords<<<1, kBlock, sizeof(SmallSmem), str>>>(G, ldg, z, rcond, coords, eta, rbf);
    return cudaGetLastError();
}

// Column scaling of an n x k block (row stride ld): dst[:, c] = src[:, c] / sqrt(f[c])
// (inv_sqrt = 1: the A-normalisation P T^{-1/2} of recorded directions) or src[:, c] * f[c]
// (inv_sqrt = 0: the POD weights, Z diag(eta)). dst may equal src.
__global__ void k_scale_cols(const double* src, double* dst, int ld, int n, int k, const double* __restrict__ f,
                             int inv_sqrt)
{
    const int c = blockIdx.y;
    const double sc = inv_sqrt ? 1.0 / sqrt(f[c]) : f[c];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[(size_t)c * ld + i] = src[(size_t)c * ld + i] * sc;
}

cudaError_t launch_scale_cols(const double* src, double* dst, int ld, int n, int k, const double* f, int inv_sqrt,
                              int sms, cudaStream_t str)
{
    if (k <= 0 || n <= 0) return cudaSuccess;
    const int gx = std::max(1, std::min((n + kBlock - 1) / kBlock, (4 * sms + k - 1) / k));
    k_scale_cols<<<dim3(gx, k), kBlock, 0, str>>>(src, dst, ld, n, k, f, inv_sqrt);
    return cudaGetLastError();
}

// Stage one, small part (Algorithm 2 step 2): upper Cholesky R^T R of Ahat = G[:, :w]
// (row-major, row stride ldg, upper triangle read; w = w_dim, or st->pod_w when w_dim < 0),
// then R^{-1} (stored upper, row stride kWMax) and what = R^{-1} R^{-T} bhat with
// bhat = G[:, w]. With truncate, a non-positive pivot k keeps the leading k columns (whose
// factor is complete) instead of dropping the basis. A non-positive pivot marks the
// basis unusable: chol_failed = 1 and w = 0 (plain PCG for this system). Optionally the
// condition number of Ahat by the Jacobi eigensolver.
__global__ void __launch_bounds__(kBlock) k_chol(const double* __restrict__ G, int ldg, double* __restrict__ Rinv,
                                                 DevState* st, int want_cond, int w_dim, int truncate)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallSmem& sm = *reinterpret_cast<SmallSmem*>(smem_raw);
    double* R = sm.A;     // working copy, row stride kSMax
    double* X = sm.Vs;    // R^{-1}, row stride kSMax
    const int tid = threadIdx.x, nt = blockDim.x;
    const int w = w_dim >= 0 ? w_dim : st->pod_w;
    __shared__ int s_fail, s_kfail;
    if (tid == 0) {
        s_fail = 0;
        s_kfail = 0;
    }
    for (int e = tid; e < kSMax * kSMax; e += nt) {
        const int i = e / kSMax, j = e % kSMax;
        R[e] = (i < w && j < w && j >= i) ? G[(size_t)i * ldg + j] : 0.0;
        X[e] = 0.0;
    }
    __syncthreads();
    // right-looking Cholesky on the upper triangle
    for (int k = 0; k < w; ++k) {
        __shared__ double s_piv;
        if (tid == 0) {
            const double d = R[k * kSMax + k];
            if (!(d > 0.0) || !isfinite(d)) {
                s_fail = 1;
                s_kfail = k;
            }
            s_piv = (d > 0.0) ? sqrt(d) : 1.0;
            R[k * kSMax + k] = s_piv;
        }
        __syncthreads();
        if (s_fail) break;
        for (int j = k + 1 + tid; j < w; j += nt) R[k * kSMax + j] /= s_piv;
        __syncthreads();
        const int m = w - k - 1;
        for (int e = tid; e < m * m; e += nt) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j >= i) R[i * kSMax + j] -= R[k * kSMax + i] * R[k * kSMax + j];
        }
        __syncthreads();
    }
    __syncthreads();
    const int wu = s_fail ? (truncate ? s_kfail : 0) : w;
    // R^{-1}: column j by back substitution (one thread per column)
    for (int j = tid; j < wu; j += nt) {
        for (int i = j; i >= 0; --i) {
            double t = (i == j) ? 1.0 : 0.0;
            for (int k = i + 1; k <= j; ++k) t -= R[i * kSMax + k] * X[k * kSMax + j];
            X[i * kSMax + j] = t / R[i * kSMax + i];
        }
    }
    __syncthreads();
    for (int e = tid; e < kWMax * kWMax; e += nt) {
        const int i = e / kWMax, j = e % kWMax;
        Rinv[e] = (i < wu && j < wu) ? X[i * kSMax + j] : 0.0;
    }
    // what = R^{-1} (R^{-T} bhat)
    double* t = sm.ev;
    for (int a = tid; a < wu; a += nt) {
        double v = 0.0;
        for (int k = 0; k <= a; ++k) v += X[k * kSMax + a] * G[(size_t)k * ldg + w];
        t[a] = v;
    }
    __syncthreads();
    for (int a = tid; a < kWMax; a += nt) {
        double v = 0.0;
        if (a < wu)
            for (int k = a; k < wu; ++k) v += X[a * kSMax + k] * t[k];
        st->what[a] = v;
    }
    if (tid == 0) {
        st->w = wu;
        st->chol_failed = s_fail;
        st->cond = 0.0;
    }
    __syncthreads();
    if (want_cond && wu > 0) {
        // symmetric part of Ahat, from the upper triangle
        for (int e = tid; e < kSMax * kSMax; e += nt) {
            const int i = e / kSMax, j = e % kSMax;
            double v = 0.0;
            if (i < wu && j < wu) v = (j >= i) ? G[(size_t)i * ldg + j] : G[(size_t)j * ldg + i];
            sm.A[e] = v;
        }
        __syncthreads();
        const int m = wu + (wu & 1);
        jacobi_parallel(sm.A, sm.V, m, 40, sm.pos, sm.cs, sm.sn, sm.pp, sm.qq, sm.red);
        if (tid == 0) {
            double lo = sm.A[0], hi = sm.A[0];
            for (int i = 1; i < wu; ++i) {
                lo = fmin(lo, sm.A[i * kSMax + i]);
                hi = fmax(hi, sm.A[i * kSMax + i]);
            }
            st->cond = lo > 0.0 ? hi / lo : INFINITY;
        }
    }
}

// M = R^{-1} R^{-T} (w x w of st->w, row stride kWMax; R^{-1} upper triangular, row stride
// kWMax): the operator of the reduced solve mu = M c that every augmented direction takes
// (Section 4.3: the stage-one factor reused), formed once per solve so a direction pass
// needs one matrix-vector product instead of two triangular solves.
__global__ void __launch_bounds__(kBlock) k_mu_matrix(const double* __restrict__ Rinv, const DevState* st,
                                                      double* __restrict__ M)
{
    const int w = st->w;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < w * w; e += gridDim.x * blockDim.x) {
        const int a = e / w, b = e % w;
        const int k0 = a > b ? a : b;   // R^{-1}[a][k] R^{-1}[b][k] vanish below the diagonal
        double v = 0.0;
        for (int k = k0; k < w; ++k) v += Rinv[(size_t)a * kWMax + k] * Rinv[(size_t)b * kWMax + k];
        M[(size_t)a * kWMax + b] = v;
    }
}

cudaError_t launch_mu_matrix(const double* Rinv, const DevState* st, double* M, cudaStream_t str)
{
    k_mu_matrix<<<(kWMax * kWMax + kBlock - 1) / kBlock, kBlock, 0, str>>>(Rinv, st, M);
    return cudaGetLastError();
}

cudaError_t launch_chol(const double* G, int ldg, double* Rinv, DevState* st, int want_cond, cudaStream_t str,
                        int w_dim, int truncate)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(SmallSmem));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_chol<<<1, kBlock, sizeof(SmallSmem), str>>>(G, ldg, Rinv, st, want_cond, w_dim, truncate);
    return cudaGetLastError();
}

// Gram of the output-functional images of the snapshots (the output-oriented metric C^T C
// of Section 3.3): G[k][l] = sum_i cs[k][i] cs[l][i] for slots k, l < s, with cs[k] = C s_k
// (q values at cs + k * ldc). One thread per entry (s <= 64, q <= 128), fixed order.
__global__ void k_cs_gram(const double* __restrict__ cs, int ldc, int s, int q, double* __restrict__ G, int ldg)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < s * s; e += gridDim.x * blockDim.x) {
        const int k = e / s, l = e % s;
        double v = 0.0;
        for (int i = 0; i < q; ++i) v += cs[(size_t)k * ldc + i] * cs[(size_t)l * ldc + i];
        G[(size_t)k * ldg + l] = v;
    }
}

cudaError_t launch_cs_gram(const double* cs, int ldc, int s, int q, double* G, int ldg, cudaStream_t str)
{
    k_cs_gram<<<(s * s + kBlock - 1) / kBlock > 0 ? (s * s + kBlock - 1) / kBlock : 1, kBlock, 0, str>>>(cs, ldc, s, q,
                                                                                                         G, ldg);
    return cudaGetLastError();
}

// Symmetric part of an s x s matrix in place: G[k][l] = G[l][k] = (G[k][l] + G[l][k]) / 2.
__global__ void k_symmetrize(double* __restrict__ G, int ldg, int s)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < s * s; e += gridDim.x * blockDim.x) {
        const int k = e / s, l = e % s;
        if (k < l) {
            const double m = 0.5 * (G[(size_t)k * ldg + l] + G[(size_t)l * ldg + k]);
            G[(size_t)k * ldg + l] = m;
            G[(size_t)l * ldg + k] = m;
        }
    }
}

cudaError_t launch_symmetrize(double* G, int ldg, int s, cudaStream_t str)
{
    k_symmetrize<<<(s * s + kBlock - 1) / kBlock > 0 ? (s * s + kBlock - 1) / kBlock : 1, kBlock, 0, str>>>(G, ldg, s);
    return cudaGetLastError();
}

// Scatter one new row of the snapshot Gram: G[q][k] = G[k][q] = row[k], k < s.
__global__ void k_gram_scatter(const double* __restrict__ row, int s, int q, double* __restrict__ G, int ldg)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < s) {
        G[(size_t)q * ldg + k] = row[k];
        G[(size_t)k * ldg + q] = row[k];
    }
}

cudaError_t launch_gram_scatter(const double* row, int s, int q, double* G, int ldg, cudaStream_t str)
{
    k_gram_scatter<<<1, kSMax, 0, str>>>(row, s, q, G, ldg);
    return cudaGetLastError();
}

}  // namespace podcg
