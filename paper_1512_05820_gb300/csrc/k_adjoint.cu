// Differentiation of a sequence of solves with respect to per-cell log-coefficients theta,
// for the cell-centred finite-volume diffusion operator A(theta) (k = exp(theta); interior
// face conductance k_f = 2 k_a k_b/(k_a + k_b); Dirichlet boundary face conductance 2 k_a).
//
// With L = sum_j l_j(x_j) and A_j x_j = b_j, the adjoint solves A_j lambda_j = dl_j/dx_j
// (A_j symmetric, so A_j^{-T} = A_j^{-1}) and
//     dL/db_j      = lambda_j
//     dL/dtheta_c  = - sum_j lambda_j^T (dA_j/dtheta_c) x_j
//                  = - sum_j [ sum_{faces f=(c,m)} dk_f/dtheta_c (lambda_c - lambda_m)(x_c - x_m)
//                              + (boundary faces of c) 2 k_c lambda_c x_c ]
// with dk_f/dtheta_c = k_f k_m/(k_c + k_m). A diagonal term independent of theta (the
// per-system shift) does not contribute.
//
// Cells are numbered x fastest, then y, then z; the CSR row of a cell lists its z-1, y-1,
// x-1 neighbours, itself, then x+1, y+1, z+1 (absent neighbours omitted).
#include <algorithm>
#include <string>

#include "common.cuh"
#include "launch.h"
#include "pod_cg.h"

namespace podcg {

__device__ __forceinline__ double hmean(double a, double b) { return 2.0 * a * b / (a + b); }

// CSR values of A(theta) + diag(extra): the diagonal sums its face conductances in the
// order x+1, x-1, x boundaries, y+1, y-1, y boundaries, z+1, z-1, z boundaries, extra.
__global__ void __launch_bounds__(kBlock) k_diffusion_assemble(int mx, int my, int mz, const double* __restrict__ theta,
                                                               const double* __restrict__ extra,
                                                               const int32_t* __restrict__ rp, double* __restrict__ val)
{
    const long long n = (long long)mx * my * mz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % mx), y = (int)((i / mx) % my), z = (int)(i / ((long long)mx * my));
        const double kc = exp(theta[i]);
        const long long sx = 1, sy = mx, sz = (long long)mx * my;
        double fxm = 0.0, fxp = 0.0, fym = 0.0, fyp = 0.0, fzm = 0.0, fzp = 0.0;
        if (x > 0) fxm = hmean(exp(theta[i - sx]), kc);
        if (x < mx - 1) fxp = hmean(kc, exp(theta[i + sx]));
        if (y > 0) fym = hmean(exp(theta[i - sy]), kc);
        if (y < my - 1) fyp = hmean(kc, exp(theta[i + sy]));
        if (mz > 1) {
            if (z > 0) fzm = hmean(exp(theta[i - sz]), kc);
            if (z < mz - 1) fzp = hmean(kc, exp(theta[i + sz]));
        }
        double d = 0.0;
        if (x < mx - 1) d += fxp;
        if (x > 0) d += fxm;
        if (x == 0) d += 2.0 * kc;
        if (x == mx - 1) d += 2.0 * kc;
        if (y < my - 1) d += fyp;
        if (y > 0) d += fym;
        if (y == 0) d += 2.0 * kc;
        if (y == my - 1) d += 2.0 * kc;
        if (mz > 1) {
            if (z < mz - 1) d += fzp;
            if (z > 0) d += fzm;
            if (z == 0) d += 2.0 * kc;
            if (z == mz - 1) d += 2.0 * kc;
        }
        if (extra) d = d + extra[i];
        int k = rp[i];
        if (mz > 1 && z > 0) val[k++] = -fzm;
        if (y > 0) val[k++] = -fym;
        if (x > 0) val[k++] = -fxm;
        val[k++] = d;
        if (x < mx - 1) val[k++] = -fxp;
        if (y < my - 1) val[k++] = -fyp;
        if (mz > 1 && z < mz - 1) val[k++] = -fzp;
    }
}

// grad[c] -= sum_j lambda_j^T (dA/dtheta_c) x_j for nsys systems stored row-major
// (system j at offset j*n) in one pass over the checkpoints.
__global__ void __launch_bounds__(kBlock) k_theta_grad(int mx, int my, int mz, const double* __restrict__ theta,
                                                       int nsys, const double* __restrict__ lam,
                                                       const double* __restrict__ xs, double* __restrict__ grad)
{
    const long long n = (long long)mx * my * mz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % mx), y = (int)((i / mx) % my), z = (int)(i / ((long long)mx * my));
        const double kc = exp(theta[i]);
        long long nb[6];
        int cnt = 0, nbound = 0;
        if (x > 0) nb[cnt++] = i - 1; else ++nbound;
        if (x < mx - 1) nb[cnt++] = i + 1; else ++nbound;
        if (y > 0) nb[cnt++] = i - mx; else ++nbound;
        if (y < my - 1) nb[cnt++] = i + mx; else ++nbound;
        if (mz > 1) {
            const long long sz = (long long)mx * my;
            if (z > 0) nb[cnt++] = i - sz; else ++nbound;
            if (z < mz - 1) nb[cnt++] = i + sz; else ++nbound;
        }
        double dk[6];
        for (int f = 0; f < cnt; ++f) {
            const double km = exp(theta[nb[f]]);
            const double s = kc + km;
            dk[f] = (2.0 * kc * km / s) * km / s;   // dk_f/dtheta_c
        }
        double g = 0.0;
        for (int j = 0; j < nsys; ++j) {
            const double* lj = lam + (size_t)j * n;
            const double* xj = xs + (size_t)j * n;
            const double lc = lj[i], xc = xj[i];
            double t = nbound * 2.0 * kc * lc * xc;
            for (int f = 0; f < cnt; ++f) t += dk[f] * (lc - lj[nb[f]]) * (xc - xj[nb[f]]);
            g += t;
        }
        grad[i] -= g;
    }
}

cudaError_t launch_diffusion_assemble(int mx, int my, int mz, const double* theta, const double* extra,
                                      const int32_t* rp, double* val, int sms, cudaStream_t s)
{
    const long long n = (long long)mx * my * mz;
    const int grid = grid_rows((int)std::min<long long>(n, 1 << 30), kBlock, sms);
    k_diffusion_assemble<<<grid, kBlock, 0, s>>>(mx, my, mz, theta, extra, rp, val);
    return cudaGetLastError();
}

cudaError_t launch_theta_grad(int mx, int my, int mz, const double* theta, int nsys, const double* lam,
                              const double* xs, double* grad, int sms, cudaStream_t s)
{
    const long long n = (long long)mx * my * mz;
    const int grid = grid_rows((int)std::min<long long>(n, 1 << 30), kBlock, sms);
    k_theta_grad<<<grid, kBlock, 0, s>>>(mx, my, mz, theta, nsys, lam, xs, grad);
    return cudaGetLastError();
}

}  // namespace podcg

namespace {
int sms_now()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}
}  // namespace

extern "C" pod_cg_status pod_cg_diffusion_assemble(int mx, int my, int mz, const double* theta,
                                                   const double* extra_diag, const int32_t* row_ptr,
                                                   double* val_out, void* cuda_stream)
{
    if (mx < 1 || my < 1 || mz < 1 || (long long)mx * my * mz >= (1LL << 31) || !theta || !row_ptr || !val_out) {
        podcg::set_last_error("pod_cg_diffusion_assemble: bad arguments");
        return POD_CG_ERR_ARG;
    }
    cudaError_t e = podcg::launch_diffusion_assemble(mx, my, mz, theta, extra_diag, row_ptr, val_out, sms_now(),
                                                     (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        podcg::set_last_error(std::string("pod_cg_diffusion_assemble: ") + cudaGetErrorString(e));
        return POD_CG_ERR_CUDA;
    }
    return POD_CG_OK;
}

extern "C" pod_cg_status pod_cg_diffusion_theta_grad(int mx, int my, int mz, const double* theta, int nsys,
                                                     const double* lambdas, const double* xs, double* grad,
                                                     void* cuda_stream)
{
    if (mx < 1 || my < 1 || mz < 1 || (long long)mx * my * mz >= (1LL << 31) || nsys < 0 || !theta || !grad ||
        (nsys > 0 && (!lambdas || !xs))) {
        podcg::set_last_error("pod_cg_diffusion_theta_grad: bad arguments");
        return POD_CG_ERR_ARG;
    }
    cudaError_t e = podcg::launch_theta_grad(mx, my, mz, theta, nsys, lambdas, xs, grad, sms_now(),
                                             (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        podcg::set_last_error(std::string("pod_cg_diffusion_theta_grad: ") + cudaGetErrorString(e));
        return POD_CG_ERR_CUDA;
    }
    return POD_CG_OK;
}
