// Stage two of the three-stage algorithm (Section 4.2): augmented CG on the reduced system
//
//     (Y^T A Y) yhat = Y^T b                          (xbar = 0)
//
// over the augmenting basis Y (n x y, the POD modes), started from the stage-one solution
// yhat0 = [what; 0], augmented with the stage-one coordinates Phi = [I_w; 0] (W = Y Phi is
// the first w columns of Y) and unpreconditioned. Y^T A Y is never formed: an iteration
// lifts v = Y phat, multiplies u = A v and projects qhat = Y^T u, one sparse product and two
// passes over Y. The augmentation solves reuse the stage-one factor; their right-hand side
// Phi^T (Y^T A Y) zhat = (Y^T A W)^T zhat comes from G = Y^T [A W, b], formed once per
// system by the Gram kernel (its first w rows are stage one's W^T [A W, b]).
//
// Every new reduced direction is re-A-orthogonalised against the directions taken so far,
// phat -= sum_i (qhat_i^T phat / gamma_i) phat_i, with their stored reduced products qhat_i
// (classical Gram-Schmidt, one pass; zero in exact arithmetic). For an identity-metric POD
// basis Y^T A Y is ill-conditioned and plain CG directions lose their mutual A-orthogonality
// once the reduced residual has fallen far; stage three uses them as an explicit basis with
// the block-diagonal factor below, which needs that orthogonality (without it stage three
// diverged on the 128^3 diffusion sequence).
//
// Iteration k keeps v and u as columns w + k of the basis buffers (W and A W), its step
// length as what[w + k] and 1/sqrt(gamma_k) as entry (w + k, w + k) of R^{-1}. Stage three
// (Algorithm 1 with basis [W, V2], Section 4.3) then runs unchanged on the wider basis with
// the block-diagonal factor blockdiag(R, sqrt(T2)) and starts from [what; alpha], the
// stage-two solution.
//
// Stage two computes in FP64 in both precision modes (FP32 products lose the directions'
// mutual A-orthogonality at about eps_32 cond(Y^T A Y), more than stage three's block-diagonal
// factor can absorb); the templates take the element type T = double.
//
// Kernels: k_s2_bb (||b||^2, for the stage-two tolerance), k_s2_init (one block: the
// reduced residual, the first direction), then per iteration k_s2_lift (v = Y phat) and
// k_s2_apply (u = A v, gamma = (u, v), qhat = Y^T u; the last block advances the reduced
// iteration and decides whether to go on). After the stop (st->s2_done) both per-iteration
// kernels return at once.
#include "common.cuh"
#include "launch.h"

namespace podcg {

// Row sums of A x with L lanes per row (lane 0 of each group holds the sum). Loop bounds are
// uniform per warp so the shuffles never diverge.
template <int L, typename T, typename TV>
__device__ __forceinline__ T s2_row(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const TV* __restrict__ val, const T* __restrict__ x, int row, bool valid)
{
    T s = T(0);
    if (valid) {
        const int beg = __ldg(rp + row), end = __ldg(rp + row + 1);
        for (int k = beg + (int)(threadIdx.x & (L - 1)); k < end; k += L) s += T(__ldg(val + k)) * __ldg(x + __ldg(col + k));
    }
    if (L > 1) {
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

// mu = R^{-1} (R^{-T} c) for the upper-triangular R^{-1} (row stride kWMax), w <= kWMax;
// block-wide, result in s_mu (shared).
__device__ __forceinline__ void s2_mu(const double* __restrict__ Rinv, const double* s_c, int w, double* s_t,
                                      double* s_mu)
{
    for (int a = threadIdx.x; a < w; a += blockDim.x) {
        double v = 0.0;
        for (int k = 0; k <= a; ++k) v += Rinv[k * kWMax + a] * s_c[k];
        s_t[a] = v;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < w; a += blockDim.x) {
        double v = 0.0;
        for (int k = a; k < w; ++k) v += Rinv[a * kWMax + k] * s_t[k];
        s_mu[a] = v;
    }
    __syncthreads();
}

// c_j = sum_{a < y} G[a][j] r[a] for j < w (the augmentation right-hand side (Y^T A W)^T r).
__device__ __forceinline__ void s2_rhs(const double* __restrict__ G, int ldg, const double* s_r, int y, int w,
                                       double* s_c)
{
    for (int j = threadIdx.x; j < w; j += blockDim.x) {
        double v = 0.0;
        for (int a = 0; a < y; ++a) v += G[(size_t)a * ldg + j] * s_r[a];
        s_c[j] = v;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBlock) k_s2_bb(const ProbDesc* __restrict__ pd, double* __restrict__ partials,
                                                  unsigned int* counter, DevState* st)
{
    const int n = pd->n;
    const double* b = pd->b;
    double bb = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) bb += b[i] * b[i];
    double acc[1] = {bb};
    __shared__ double tot[1];
    if (reduce_to_last_block<1>(acc, 1, partials, counter, tot) && threadIdx.x == 0) st->bb = tot[0];
}

// One block. G = Y^T [A W, b] (row-major, row stride ldg; column st->pod_w holds Y^T b), w
// the stage-one dimension after its Cholesky (st->w), y = st->pod_y, w_cap the basis
// buffers' column capacity. Algorithm 1 steps 1-5 on the reduced system:
//   rhat0 = Y^T b - (Y^T A W) what, zhat0 = rhat0, mu0 from (Y^T A W)^T zhat0, phat0 = zhat0 - [mu0; 0]
// and the stop test on ||rhat0|| against tol_fac * tol * ||b|| (tol = st->tol_rel).
template <bool COND>
__global__ void __launch_bounds__(kBlock) k_s2_init(const double* __restrict__ G, int ldg,
                                                    const double* __restrict__ Rinv, DevState* st, int w_cap,
                                                    double tol_fac, cudaGraphConditionalHandle h_loop)
{
    __shared__ double s_r[kSMax], s_c[kWMax], s_t[kWMax], s_mu[kWMax];
    __shared__ int s_done;
    const int y = st->pod_y, w = st->w, bcol = st->pod_w;
    for (int a = threadIdx.x; a < y; a += blockDim.x) {
        double v = G[(size_t)a * ldg + bcol];
        for (int j = 0; j < w; ++j) v -= G[(size_t)a * ldg + j] * st->what[j];
        s_r[a] = v;
    }
    __syncthreads();
    s2_rhs(G, ldg, s_r, y, w, s_c);
    s2_mu(Rinv, s_c, w, s_t, s_mu);
    for (int a = threadIdx.x; a < y; a += blockDim.x) {
        st->rh[a] = s_r[a];
        st->ph[a] = s_r[a] - (a < w ? s_mu[a] : 0.0);
    }
    if (threadIdx.x == 0) {
        double rr = 0.0;
        for (int a = 0; a < y; ++a) rr += s_r[a] * s_r[a];
        const double t = st->tol_rel * tol_fac;
        const double t2 = t * t * st->bb;
        const int cap = (y < w_cap ? y : w_cap) - w;
        st->w1 = w;
        st->k2 = 0;
        st->m_dirs = 0;
        st->inner_total = 0;
        st->m_cap = cap > 0 ? cap : 0;
        st->rho2 = rr;
        st->tol2_s2 = t2;
        st->s2_break = 0;
        const int done = (cap <= 0 || !(rr > t2)) ? 1 : 0;
        st->s2_done = done;
        s_done = done;
    }
    __syncthreads();
    if (COND && threadIdx.x == 0) cudaGraphSetConditional(h_loop, s_done ? 0u : 1u);
}

// v = Y phat into column w1 + k2 of the basis buffer B (stage two), or into B itself (an
// inner solve of the whole-Y stage three, inner = 1: its lifted directions are not kept).
template <int YB, typename T>
__global__ void __launch_bounds__(kBlock) k_s2_lift(int n, int ld, const T* __restrict__ Y, T* __restrict__ B,
                                                    const DevState* st, int inner)
{
    if (st->s2_done) return;
    const int y = st->pod_y;
    __shared__ T s_p[YB];
    for (int l = threadIdx.x; l < YB; l += blockDim.x) s_p[l] = (l < y) ? T(st->ph[l]) : T(0);
    __syncthreads();
    T* v = B + (inner ? (size_t)0 : (size_t)(st->w1 + st->k2) * ld);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T t = T(0);
#pragma unroll
        for (int l = 0; l < YB; ++l)
            if (l < y) t += __ldg(Y + (size_t)l * ld + i) * s_p[l];
        v[i] = t;
    }
}

// u = A v (column w1 + k2 of AB; inner = 1: AB itself), gamma = (u, v) and qhat = Y^T u in
// one pass; the last block then takes the reduced step (Algorithm 1 on Y^T A Y, M = I):
//   alpha = rho/gamma, xhat += alpha phat, rhat -= alpha qhat, beta = (rhat, rhat)/rho,
//   mu from (Y^T A W)^T rhat, phat = rhat + beta phat - [mu; 0], then the re-A-
//   orthogonalisation against the stored directions (hist: phat_i at hist[i * kSMax],
//   qhat_i at hist[(kWMax + i) * kSMax], gamma_i at hist[2 * kWMax * kSMax + i]; the one
//   just taken is stored at i = m_dirs first). Stage two (inner = 0) records alpha and
//   1/sqrt(gamma) for stage three. It stops on ||rhat|| <= tolerance, when m_cap directions
//   are stored, or on a non-positive / non-finite gamma (that direction is dropped).
template <int L, int YB, typename T, bool COND>
__global__ void __launch_bounds__(kBlock) k_s2_apply(const ProbDesc* __restrict__ pd, int ld, const T* __restrict__ Y,
                                                     const T* __restrict__ B, T* __restrict__ AB,
                                                     double* __restrict__ partials, unsigned int* counter,
                                                     DevState* st, double* __restrict__ Rinv,
                                                     const double* __restrict__ G, int ldg,
                                                     double* __restrict__ hist, int inner,
                                                     cudaGraphConditionalHandle h_loop)
{
    if (st->s2_done) return;
    constexpr int CPW = (YB + kWarps - 1) / kWarps;
    const int n = pd->n, y = st->pod_y, w1 = st->w1, k = st->k2, m = st->m_dirs;
    const int colk = w1 + k;
    const T* v = B + (inner ? (size_t)0 : (size_t)colk * ld);
    T* u = AB + (inner ? (size_t)0 : (size_t)colk * ld);
    __shared__ T s_u[kBlock];
    __shared__ double s_blk[YB + 2];
    T cacc[CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) cacc[c] = T(0);
    T dot = T(0);
    constexpr int gpb = kBlock / L;
    const int g = threadIdx.x / L;
    const bool head = (threadIdx.x & (L - 1)) == 0;
    for (int row0 = blockIdx.x * kBlock; row0 < n; row0 += gridDim.x * kBlock) {
#pragma unroll 1
        for (int sub = 0; sub < L; ++sub) {
            const int rl = sub * gpb + g;
            const int row = row0 + rl;
            T s;
            s = s2_row<L, T, double>(pd->rp, pd->col, pd->val, v, row, row < n);
            if (head) {
                s_u[rl] = (row < n) ? s : T(0);
                if (row < n) {
                    u[row] = s;
                    dot += s * v[row];
                }
            }
        }
        __syncthreads();
        tile_columns<CPW, T>(Y, ld, y, row0, n, s_u, cacc);
        __syncthreads();
    }
    block_totals<CPW, T>(dot, T(0), cacc, y, s_blk);
    __shared__ double tot[kWMax + 2];
    if (!partials_to_last_block(s_blk, 2 + y, partials, counter, tot)) return;

    __shared__ double s_r[kSMax], s_c[kWMax], s_t[kWMax], s_mu[kWMax];
    __shared__ double s_beta, s_alpha;
    __shared__ int s_stop;
    if (threadIdx.x == 0) {
        const double gamma = tot[0];
        const double rho = st->rho2;
        const bool bad = !isfinite(gamma) || !(gamma > 0.0);
        s_stop = bad ? 2 : 0;
        s_alpha = bad ? 0.0 : rho / gamma;
        if (!bad && !inner) {
            st->what[colk] = s_alpha;
            Rinv[colk * kWMax + colk] = 1.0 / sqrt(gamma);
        }
    }
    __syncthreads();
    if (s_stop == 2) {
        if (threadIdx.x == 0) {
            st->s2_break = 1;
            st->s2_done = 1;
            if (!inner) st->w = colk;   // directions 0..k-1
            if (COND) cudaGraphSetConditional(h_loop, 0u);
        }
        return;
    }
    double* Ph = hist;
    double* Qh = hist + (size_t)kWMax * kSMax;
    double* gam = hist + (size_t)2 * kWMax * kSMax;
    for (int a = threadIdx.x; a < y; a += blockDim.x) {
        s_r[a] = st->rh[a] - s_alpha * tot[2 + a];
        st->xh[a] += s_alpha * st->ph[a];
        Ph[(size_t)m * kSMax + a] = st->ph[a];
        Qh[(size_t)m * kSMax + a] = tot[2 + a];
    }
    if (threadIdx.x == 0) gam[m] = tot[0];
    __syncthreads();
    if (threadIdx.x == 0) {
        double rr = 0.0;
        for (int a = 0; a < y; ++a) rr += s_r[a] * s_r[a];
        s_beta = rr / st->rho2;
        st->rho2 = rr;
        const int kn = k + 1;
        st->k2 = kn;
        st->m_dirs = m + 1;
        if (inner) st->inner_total += 1;
        const int stop = (!(rr > st->tol2_s2) || m + 1 >= st->m_cap || !isfinite(rr)) ? 1 : 0;
        s_stop = stop;
        if (stop) {
            st->s2_done = 1;
            if (!inner) st->w = w1 + kn;
        }
        if (COND) cudaGraphSetConditional(h_loop, stop ? 0u : 1u);
    }
    __syncthreads();
    if (s_stop) return;
    s2_rhs(G, ldg, s_r, y, w1, s_c);
    s2_mu(Rinv, s_c, w1, s_t, s_mu);
    __shared__ double s_p[kSMax], s_cf[kWMax];
    for (int a = threadIdx.x; a < y; a += blockDim.x) {
        st->rh[a] = s_r[a];
        s_p[a] = s_r[a] + s_beta * st->ph[a] - (a < w1 ? s_mu[a] : 0.0);
    }
    __syncthreads();
    // classical Gram-Schmidt in the reduced A-inner product, stored directions 0..m
    for (int i = threadIdx.x; i <= m; i += blockDim.x) {
        double c = 0.0;
        for (int a = 0; a < y; ++a) c += Qh[(size_t)i * kSMax + a] * s_p[a];
        s_cf[i] = c / gam[i];
    }
    __syncthreads();
    for (int a = threadIdx.x; a < y; a += blockDim.x) {
        double t = 0.0;
        for (int i = 0; i <= m; ++i) t += s_cf[i] * Ph[(size_t)i * kSMax + a];
        st->ph[a] = s_p[a] - t;
    }
}

// ------------------------------------------- stage three over the entire augmenting basis

// The whole-Y stage three (Section 4.3.1) runs Algorithm 1 with the plain Jacobi-PCG
// kernels (st->w = 0: no projection in the update) and these three steps for the
// augmentation solves Y^T A Y mu = Y^T A z:
//   k_it_az    u = A z with z = M^{-1} r formed on the fly, chat = Y^T u (fused), and in
//              the last block the start of the inner reduced solve: the Galerkin solution
//              over the stored reduced basis Psi = [Phi, stored directions],
//                mu0 = Phi R^{-1} R^{-T} chat[:w] + sum_i phat_i (phat_i^T chat)/gamma_i,
//              its residual rhat0 = chat - (Y^T A W) nu - sum_i c_i qhat_i from the stored
//              products, the first direction, and the stop test ||rhat|| <= tol_in ||chat||;
//   then inner iterations of k_s2_lift / k_s2_apply (inner = 1), which append their
//              directions to the store (at most m_cap in all);
//   k_it_dir   x += alpha p (after the first step), p = z + beta p - Y mu.
// Both return at once (k_it_dir after its x update) once the loop has stopped.

// Row sums of A (D^{-1} r): the diagonal scaling is applied to each gathered entry.
template <int L>
__device__ __forceinline__ double it_row(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                         const double* __restrict__ val, const double* __restrict__ dinv,
                                         const double* __restrict__ r, int row, bool valid)
{
    double s = 0.0;
    if (valid) {
        const int beg = __ldg(rp + row), end = __ldg(rp + row + 1);
        for (int k = beg + (int)(threadIdx.x & (L - 1)); k < end; k += L) {
            const int c = __ldg(col + k);
            s += __ldg(val + k) * (__ldg(dinv + c) * r[c]);
        }
    }
    if (L > 1) {
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

template <int L, int YB>
__global__ void __launch_bounds__(kBlock) k_it_az(const ProbDesc* __restrict__ pd, int ld,
                                                  const double* __restrict__ dinv, const double* __restrict__ r,
                                                  const double* __restrict__ Y, double* __restrict__ partials,
                                                  unsigned int* counter, DevState* st,
                                                  const double* __restrict__ Rinv, const double* __restrict__ G,
                                                  int ldg, const double* __restrict__ hist, double tol_in)
{
    if (st->done || st->status != 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->s2_done = 1;
        return;
    }
    constexpr int CPW = (YB + kWarps - 1) / kWarps;
    const int n = pd->n, y = st->pod_y;
    __shared__ double s_u[kBlock];
    __shared__ double s_blk[YB + 2];
    double cacc[CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) cacc[c] = 0.0;
    constexpr int gpb = kBlock / L;
    const int g = threadIdx.x / L;
    const bool head = (threadIdx.x & (L - 1)) == 0;
    for (int row0 = blockIdx.x * kBlock; row0 < n; row0 += gridDim.x * kBlock) {
#pragma unroll 1
        for (int sub = 0; sub < L; ++sub) {
            const int rl = sub * gpb + g;
            const int row = row0 + rl;
            const double sv = it_row<L>(pd->rp, pd->col, pd->val, dinv, r, row, row < n);
            if (head) s_u[rl] = (row < n) ? sv : 0.0;
        }
        __syncthreads();
        tile_columns<CPW, double>(Y, ld, y, row0, n, s_u, cacc);
        __syncthreads();
    }
    block_totals<CPW, double>(0.0, 0.0, cacc, y, s_blk);
    __shared__ double tot[kWMax + 2];
    if (!partials_to_last_block(s_blk, 2 + y, partials, counter, tot)) return;

    const double* Ph = hist;
    const double* Qh = hist + (size_t)kWMax * kSMax;
    const double* gam = hist + (size_t)2 * kWMax * kSMax;
    const int w1 = st->w1, m = st->m_dirs;
    __shared__ double s_ch[kSMax], s_r[kSMax], s_c[kWMax], s_t[kWMax], s_nu[kWMax], s_cf[kWMax], s_p[kSMax];
    for (int a = threadIdx.x; a < y; a += blockDim.x) s_ch[a] = tot[2 + a];
    for (int j = threadIdx.x; j < w1; j += blockDim.x) s_c[j] = tot[2 + j];   // Phi^T chat
    __syncthreads();
    s2_mu(Rinv, s_c, w1, s_t, s_nu);                                          // nu = R^{-1} R^{-T} chat[:w]
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double c = 0.0;
        for (int a = 0; a < y; ++a) c += Ph[(size_t)i * kSMax + a] * s_ch[a];
        s_cf[i] = c / gam[i];
    }
    __syncthreads();
    for (int a = threadIdx.x; a < y; a += blockDim.x) {
        // mu0 and rhat0 = chat - (Y^T A W) nu - sum_i c_i qhat_i
        double x0 = (a < w1) ? s_nu[a] : 0.0, q = 0.0;
        for (int j = 0; j < w1; ++j) q += G[(size_t)a * ldg + j] * s_nu[j];
        for (int i = 0; i < m; ++i) {
            x0 += s_cf[i] * Ph[(size_t)i * kSMax + a];
            q += s_cf[i] * Qh[(size_t)i * kSMax + a];
        }
        st->xh[a] = x0;
        s_r[a] = s_ch[a] - q;
    }
    __syncthreads();
    s2_rhs(G, ldg, s_r, y, w1, s_c);                                          // (Y^T A W)^T zhat, zhat = rhat
    s2_mu(Rinv, s_c, w1, s_t, s_nu);
    for (int a = threadIdx.x; a < y; a += blockDim.x) {
        st->rh[a] = s_r[a];
        s_p[a] = s_r[a] - (a < w1 ? s_nu[a] : 0.0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double c = 0.0;
        for (int a = 0; a < y; ++a) c += Qh[(size_t)i * kSMax + a] * s_p[a];
        s_cf[i] = c / gam[i];
    }
    __syncthreads();
    for (int a = threadIdx.x; a < y; a += blockDim.x) {
        double t = 0.0;
        for (int i = 0; i < m; ++i) t += s_cf[i] * Ph[(size_t)i * kSMax + a];
        st->ph[a] = s_p[a] - t;
    }
    if (threadIdx.x == 0) {
        double rr = 0.0, cc = 0.0;
        for (int a = 0; a < y; ++a) {
            rr += s_r[a] * s_r[a];
            cc += s_ch[a] * s_ch[a];
        }
        st->rho2 = rr;
        st->tol2_s2 = tol_in * tol_in * cc;
        st->k2 = 0;
        st->s2_done = (!(rr > st->tol2_s2) || m >= st->m_cap) ? 1 : 0;
    }
}

// FIRST: p = z - Y mu. Otherwise x += alpha p, then (unless the loop has stopped)
// p = z + beta p - Y mu, with z = M^{-1} r and mu = st->xh.
template <int YB, bool FIRST>
__global__ void __launch_bounds__(kBlock) k_it_dir(int n, int ld, double* __restrict__ x, double* __restrict__ p,
                                                   const double* __restrict__ r, const double* __restrict__ dinv,
                                                   const double* __restrict__ Y, const DevState* st)
{
    if (FIRST && (st->done || st->status != 0)) return;
    const int y = st->pod_y;
    const bool ok = st->status == 0 || st->status == 4;   // 4: the cap, after a valid step
    const double alpha = ok ? st->alpha : 0.0;
    const double beta = st->beta;
    const bool upd_p = FIRST || (!st->done && ok);
    __shared__ double s_mu[YB];
    for (int l = threadIdx.x; l < YB; l += blockDim.x) s_mu[l] = (l < y) ? st->xh[l] : 0.0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double pi = p[i];
        if (!FIRST) x[i] += alpha * pi;
        if (upd_p) {
            double t = 0.0;
#pragma unroll
            for (int l = 0; l < YB; ++l)
                if (l < y) t += __ldg(Y + (size_t)l * ld + i) * s_mu[l];
            const double zi = dinv[i] * r[i];
            p[i] = zi + (FIRST ? 0.0 : beta * pi) - t;
        }
    }
}

// Start of the whole-Y stage three: Algorithm 1's update kernels run without a basis.
__global__ void k_it_begin(DevState* st) { st->w = 0; }


// FP32 copy of stage two's directions for a mixed-precision stage three, each column scaled
// to unit A-norm (by its 1/sqrt(gamma), the diagonal entry of R^{-1}): the last directions of
// a stage two that ran to rounding level are tiny, and their FP32 products would underflow.
// Columns col0 .. col0 + ncols - 1 of W (ld-strided).
__global__ void __launch_bounds__(kBlock) k_s2_to_f32(int n, int ld, const double* __restrict__ W,
                                                      float* __restrict__ W32, int col0, int ncols,
                                                      const double* __restrict__ Rinv)
{
    const size_t total = (size_t)ncols * ld;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int c = col0 + (int)(e / ld);
        const int i = (int)(e % ld);
        if (i < n) W32[(size_t)c * ld + i] = float(W[(size_t)c * ld + i] * Rinv[c * kWMax + c]);
    }
}

cudaError_t launch_s2_to_f32(int n, int ld, const double* W, float* W32, int col0, int ncols, const double* Rinv,
                             int sms, cudaStream_t s)
{
    if (ncols <= 0) return cudaSuccess;
    k_s2_to_f32<<<sms * 8, kBlock, 0, s>>>(n, ld, W, W32, col0, ncols, Rinv);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ host side

#define PODCG_S2_YB(Y, ...)                                       \
    if ((Y) <= 8) { constexpr int YY = 8; __VA_ARGS__; }          \
    else if ((Y) <= 16) { constexpr int YY = 16; __VA_ARGS__; }   \
    else if ((Y) <= 32) { constexpr int YY = 32; __VA_ARGS__; }   \
    else if ((Y) <= 48) { constexpr int YY = 48; __VA_ARGS__; }   \
    else { constexpr int YY = 64; __VA_ARGS__; }

#define PODCG_S2_L(L, ...)                                    \
    switch (L) {                                              \
    case 1: { constexpr int LL = 1; __VA_ARGS__; } break;     \
    case 2: { constexpr int LL = 2; __VA_ARGS__; } break;     \
    case 4: { constexpr int LL = 4; __VA_ARGS__; } break;     \
    case 8: { constexpr int LL = 8; __VA_ARGS__; } break;     \
    case 16: { constexpr int LL = 16; __VA_ARGS__; } break;   \
    default: { constexpr int LL = 32; __VA_ARGS__; } break;   \
    }

void it_kernels(int y, int L, void** az, void** dir0, void** dir, void** begin)
{
    *begin = (void*)k_it_begin;
    PODCG_S2_YB(y, {
        *dir0 = (void*)k_it_dir<YY, true>;
        *dir = (void*)k_it_dir<YY, false>;
        PODCG_S2_L(L, *az = (void*)k_it_az<LL, YY>);
    });
}

void stage2_kernels(int y, int L, bool cond, void** bb, void** init, void** lift, void** apply)
{
    *bb = (void*)k_s2_bb;
    *init = cond ? (void*)k_s2_init<true> : (void*)k_s2_init<false>;
    PODCG_S2_YB(y, {
        *lift = (void*)k_s2_lift<YY, double>;
        PODCG_S2_L(L, *apply = cond ? (void*)k_s2_apply<LL, YY, double, true> : (void*)k_s2_apply<LL, YY, double, false>);
    });
}

}  // namespace podcg
