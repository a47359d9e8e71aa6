// Solver engine and C ABI (include/pod_cg.h).
//
// A handle owns the snapshot ring S (column-major, leading dimension ld = n rounded up to
// 32), its Gram S^T S (kept up to date one row per added snapshot), the POD basis W, A W,
// the stage-one factor R^{-1}, the CG vectors, reduction scratch and the captured graphs.
//
// pod_cg_solve enqueues, on the handle's stream:
//   POD (when the snapshots changed): Jacobi eigensolve of S^T S, truncation, lift W = S C
//   stage one: A W, W^T [A W, b], Cholesky + R^{-1} + what, x0 = W what, r0 = b - A W what
//   one graph launch: outer while (residual replacement / refinement) {
//       init pass: z0, mu0, p0; inner while (CG) { q = A p; update; direction };
//       true residual b - A x in FP64 (sets the outer condition) }
// The loop runs entirely on the device (conditional graph nodes); the host synchronises
// once to learn w (which selects the graph of the basis-width bucket) and once at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "pod_cg.h"

using namespace podcg;

namespace {

thread_local std::string g_last_error;

int device_sms()
{
    int dev = 0;
    cudaGetDevice(&dev);
    static int cache[64] = {0};
    if (dev < 0 || dev >= 64) dev = 0;
    if (cache[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = v > 0 ? v : 1;
    }
    return cache[dev];
}

struct GraphSlot {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int L = 0;
    bool valid = false;
};

// Add a kernel node: the arguments are passed by value and must match the kernel's
// parameter types in size and order.
template <typename... Args>
cudaError_t add_kernel(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps, void* func, int grid,
                       int block, cudaGraphNode_t* out, Args... args)
{
    void* ptrs[] = {(void*)&args...};
    cudaKernelNodeParams p = {};
    p.func = func;
    p.gridDim = dim3(grid);
    p.blockDim = dim3(block);
    p.sharedMemBytes = 0;
    p.kernelParams = ptrs;
    p.extra = nullptr;
    return cudaGraphAddKernelNode(out, g, deps, ndeps, &p);
}

cudaError_t add_while(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps, cudaGraphConditionalHandle h,
                      cudaGraphNode_t* out, cudaGraph_t* body)
{
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(out, g, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess) *body = cp.conditional.phGraph_out[0];
    return e;
}

}  // namespace

struct pod_cg_t {
    int n = 0, ld = 0, sms = 1, device = 0;
    pod_cg_config cfg{};
    cudaStream_t stream = nullptr;
    std::string err;

    // snapshots and POD
    double* S = nullptr;        // ld x s_max
    double* GS = nullptr;       // kSMax x kSMax row-major (slot order)
    double* grow = nullptr;     // one Gram row (kSMax)
    double* C = nullptr;        // kSMax x kWMax lift coefficients
    double* sigma2 = nullptr;   // kSMax eigenvalues
    int s_count = 0, s_next = 0;
    bool pod_dirty = false;
    int pod_w = 0;

    // basis and stage one
    double* W = nullptr;        // ld x w_max
    double* AW = nullptr;       // ld x w_max
    double* G = nullptr;        // kWMax x (kWMax + 1) row-major
    double* Rinv = nullptr;     // kWMax x kWMax

    // CG vectors (FP64)
    double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *dinv = nullptr;
    float* dinv32 = nullptr;

    // reductions
    double* partials = nullptr;
    unsigned int* counters = nullptr;   // 16 counters
    double* gram_work = nullptr;
    size_t gram_work_bytes = 0;

    DevState* st = nullptr;
    DevState* st_host = nullptr;        // pinned
    ProbDesc* pd = nullptr;
    ProbDesc* pd_host = nullptr;        // pinned

    GraphSlot graphs[6][2];             // [width bucket][precision]
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int system_counter = 0;
};

namespace {

pod_cg_status fail(pod_cg_t* h, pod_cg_status st, const std::string& msg)
{
    if (h) h->err = msg;
    else g_last_error = msg;
    return st;
}

pod_cg_status cuda_fail(pod_cg_t* h, const char* what, cudaError_t e)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? POD_CG_ERR_OOM : POD_CG_ERR_CUDA, m);
}

#define PODCG_CK(h, call)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(h, #call, e_); \
    } while (0)

int bucket_index(int wb)
{
    switch (wb) {
    case 0: return 0;
    case 8: return 1;
    case 16: return 2;
    case 32: return 3;
    case 48: return 4;
    default: return 5;
    }
}

pod_cg_status check_csr(pod_cg_t* h, const pod_cg_csr* A, int n)
{
    if (!A) return fail(h, POD_CG_ERR_ARG, "A is NULL");
    if (A->n != n) return fail(h, POD_CG_ERR_ARG, "A->n does not match the handle's order");
    if (A->nnz < 0 || A->nnz >= (int64_t)INT32_MAX) return fail(h, POD_CG_ERR_ARG, "nnz out of range");
    if (n > 0 && (!A->row_ptr || !A->col || (A->nnz > 0 && !A->val)))
        return fail(h, POD_CG_ERR_ARG, "CSR arrays must be non-NULL");
    return POD_CG_OK;
}

// Build the FP64 solve graph for width bucket wb and SpMV lanes L.
pod_cg_status build_graph_fp64(pod_cg_t* h, int wb, int L, GraphSlot& gs)
{
    const int n = h->n, ld = h->ld;
    const int grid = grid_rows(n, kBlock, h->sms);
    const int grid_spmv = grid_rows(n, kBlock / L, h->sms);
    void *k_init_f, *k_upd_f, *k_dir0_f, *k_dir_f;
    cg_kernels(wb, false, &k_init_f, &k_upd_f, &k_dir0_f, &k_dir_f);
    void* k_spmv_f = kernel_spmv_cg(L, false);
    void* k_res_f = kernel_residual(L);

    cudaGraph_t P = nullptr;
    PODCG_CK(h, cudaGraphCreate(&P, 0));
    cudaGraphConditionalHandle h_outer, h_inner;
    PODCG_CK(h, cudaGraphConditionalHandleCreate(&h_outer, P, 1, cudaGraphCondAssignDefault));
    cudaGraphNode_t n_outer;
    cudaGraph_t O = nullptr, I = nullptr;
    PODCG_CK(h, add_while(P, nullptr, 0, h_outer, &n_outer, &O));
    PODCG_CK(h, cudaGraphConditionalHandleCreate(&h_inner, O, 0, 0));

    const double* cW = h->W;
    const double* cAW = h->AW;
    const double* cRinv = h->Rinv;
    const double* cdinv = h->dinv;
    unsigned int* c0 = h->counters + 0;
    unsigned int* c1 = h->counters + 1;
    unsigned int* c2 = h->counters + 2;
    unsigned int* c3 = h->counters + 3;
    int use_cond = 1, zero = 0;
    double inner_tol = h->cfg.inner_tol;

    cudaGraphNode_t n1, n2, n3, n4, m1, m2, m3;
    PODCG_CK(h, add_kernel(O, nullptr, 0, k_init_f, grid, kBlock, &n1, n, ld, (const double*)h->r, cdinv, cAW,
                           cRinv, h->partials, c0, h->st, h_inner, use_cond));
    PODCG_CK(h, add_kernel(O, &n1, 1, k_dir0_f, grid, kBlock, &n2, n, ld, h->x, h->p, (const double*)h->r, cdinv,
                           cW, (const DevState*)h->st));
    PODCG_CK(h, add_while(O, &n2, 1, h_inner, &n3, &I));
    PODCG_CK(h, add_kernel(O, &n3, 1, k_res_f, grid_spmv, kBlock, &n4, (const ProbDesc*)h->pd,
                           (const double*)h->x, h->r, h->partials, c1, h->st, zero, inner_tol, h_outer, use_cond));
    PODCG_CK(h, add_kernel(I, nullptr, 0, k_spmv_f, grid_spmv, kBlock, &m1, (const ProbDesc*)h->pd,
                           (const double*)h->p, h->q, h->partials, c2, h->st));
    PODCG_CK(h, add_kernel(I, &m1, 1, k_upd_f, grid, kBlock, &m2, n, ld, h->r, (const double*)h->q, cdinv, cAW,
                           cRinv, h->partials, c3, h->st, h_inner, use_cond));
    PODCG_CK(h, add_kernel(I, &m2, 1, k_dir_f, grid, kBlock, &m3, n, ld, h->x, h->p, (const double*)h->r, cdinv, cW,
                           (const DevState*)h->st));
    cudaGraphExec_t exec = nullptr;
    PODCG_CK(h, cudaGraphInstantiate(&exec, P, 0));
    gs.graph = P;
    gs.exec = exec;
    gs.L = L;
    gs.valid = true;
    return POD_CG_OK;
}

void destroy_graph(GraphSlot& gs)
{
    if (gs.exec) cudaGraphExecDestroy(gs.exec);
    if (gs.graph) cudaGraphDestroy(gs.graph);
    gs = GraphSlot();
}

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

}  // namespace

void podcg::set_last_error(const std::string& msg) { g_last_error = msg; }

// ======================================================================== C ABI

extern "C" {

pod_cg_status pod_cg_config_default(pod_cg_config* c)
{
    if (!c) return POD_CG_ERR_ARG;
    std::memset(c, 0, sizeof(*c));
    c->w_max = 32;
    c->s_max = 40;
    c->energy = 0.9999;
    c->rank_tol = 1e-13;
    c->k_max = 100000;
    c->max_refine = 5;
    c->precision = POD_CG_FP64;
    c->inner_tol = 1e-5;
    c->use_tc_gram = 0;
    c->cond_diag = 0;
    c->keep_factors = 0;
    return POD_CG_OK;
}

const char* pod_cg_last_error(const pod_cg_t* h)
{
    return h ? h->err.c_str() : g_last_error.c_str();
}

pod_cg_status pod_cg_destroy(pod_cg_t* h)
{
    if (!h) return POD_CG_OK;
    for (auto& row : h->graphs)
        for (auto& g : row) destroy_graph(g);
    void* bufs[] = {h->S, h->GS, h->grow, h->C, h->sigma2, h->W, h->AW, h->G, h->Rinv, h->x, h->r, h->p,
                    h->q, h->dinv, h->dinv32, h->partials, h->counters, h->gram_work, h->st, h->pd};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->pd_host) cudaFreeHost(h->pd_host);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    delete h;
    return POD_CG_OK;
}

pod_cg_status pod_cg_create(int n, const pod_cg_config* cfg, void* cuda_stream, pod_cg_t** out)
{
    if (!out) return fail(nullptr, POD_CG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1) return fail(nullptr, POD_CG_ERR_ARG, "n must be >= 1");
    pod_cg_config c;
    if (cfg) c = *cfg;
    else pod_cg_config_default(&c);
    if (c.w_max < 1 || c.w_max > kWMax || c.s_max < 1 || c.s_max > kSMax || !(c.energy >= 0.0 && c.energy <= 1.0) ||
        c.k_max < 0 || c.max_refine < 0 || (c.precision != POD_CG_FP64 && c.precision != POD_CG_MIXED) ||
        c.keep_factors < 0)
        return fail(nullptr, POD_CG_ERR_ARG, "invalid configuration");
    pod_cg_t* h = new (std::nothrow) pod_cg_t();
    if (!h) return fail(nullptr, POD_CG_ERR_OOM, "host allocation failed");
    h->n = n;
    h->ld = ((n + 31) / 32) * 32;
    h->cfg = c;
    h->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&h->device);
    h->sms = device_sms();
    const size_t ld = (size_t)h->ld;
    cudaError_t e = cudaSuccess;
#define PODCG_ALLOC(ptr, cnt)                                           \
    if (e == cudaSuccess) e = dalloc(&(ptr), (cnt));
    PODCG_ALLOC(h->S, ld * c.s_max)
    PODCG_ALLOC(h->GS, (size_t)kSMax * kSMax)
    PODCG_ALLOC(h->grow, (size_t)kSMax)
    PODCG_ALLOC(h->C, (size_t)kSMax * kWMax)
    PODCG_ALLOC(h->sigma2, (size_t)kSMax)
    PODCG_ALLOC(h->W, ld * c.w_max)
    PODCG_ALLOC(h->AW, ld * c.w_max)
    PODCG_ALLOC(h->G, (size_t)kWMax * (kWMax + 1))
    PODCG_ALLOC(h->Rinv, (size_t)kWMax * kWMax)
    PODCG_ALLOC(h->x, ld)
    PODCG_ALLOC(h->r, ld)
    PODCG_ALLOC(h->p, ld)
    PODCG_ALLOC(h->q, ld)
    PODCG_ALLOC(h->dinv, ld)
    PODCG_ALLOC(h->dinv32, ld)
    PODCG_ALLOC(h->partials, (size_t)h->sms * 8 * (kWMax + 2))
    PODCG_ALLOC(h->counters, 16)
    PODCG_ALLOC(h->st, 1)
    PODCG_ALLOC(h->pd, 1)
#undef PODCG_ALLOC
    if (e == cudaSuccess) {
        h->gram_work_bytes = std::max(gram_workspace_bytes(n, 1, c.s_max, h->sms),
                                      gram_workspace_bytes(n, c.w_max, c.w_max + 1, h->sms));
        e = cudaMalloc((void**)&h->gram_work, h->gram_work_bytes);
    }
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->st_host, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->pd_host, sizeof(ProbDesc));
    for (auto& ev : h->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->counters, 0, 16 * sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->S, 0, sizeof(double) * ld * c.s_max, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->GS, 0, sizeof(double) * kSMax * kSMax, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->p, 0, sizeof(double) * ld, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        pod_cg_status s = cuda_fail(nullptr, "pod_cg_create", e);
        pod_cg_destroy(h);
        return s;
    }
    *out = h;
    return POD_CG_OK;
}

pod_cg_status pod_cg_clear_snapshots(pod_cg_t* h)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    h->s_count = 0;
    h->s_next = 0;
    h->pod_dirty = false;
    h->pod_w = 0;
    return POD_CG_OK;
}

pod_cg_status pod_cg_add_snapshots(pod_cg_t* h, const double* X, int m)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    if (m < 0 || (m > 0 && !X)) return fail(h, POD_CG_ERR_ARG, "bad snapshot block");
    const int n = h->n;
    for (int c = 0; c < m; ++c) {
        const int slot = h->s_next;
        double* col = h->S + (size_t)slot * h->ld;
        PODCG_CK(h, cudaMemcpyAsync(col, X + (size_t)c * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
        h->s_next = (h->s_next + 1) % h->cfg.s_max;
        h->s_count = std::min(h->s_count + 1, h->cfg.s_max);
        // new row of S^T S: s_new^T S (Algorithm 4 step 1, one row at a time)
        PODCG_CK(h, launch_gram(n, col, h->ld, 1, h->S, h->ld, h->s_count, nullptr, h->grow, kSMax, 0, h->gram_work,
                                h->gram_work_bytes, h->sms, h->stream));
        PODCG_CK(h, launch_gram_scatter(h->grow, h->s_count, slot, h->GS, kSMax, h->stream));
    }
    if (m > 0) h->pod_dirty = true;
    return POD_CG_OK;
}

pod_cg_status pod_cg_get_basis(pod_cg_t* h, double* W_out, int* w_out)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    if (w_out) *w_out = h->pod_w;
    if (W_out && h->pod_w > 0) {
        PODCG_CK(h, cudaMemcpy2DAsync(W_out, sizeof(double) * h->n, h->W, sizeof(double) * h->ld,
                                      sizeof(double) * h->n, h->pod_w, cudaMemcpyDeviceToDevice, h->stream));
    }
    PODCG_CK(h, cudaStreamSynchronize(h->stream));
    return POD_CG_OK;
}

pod_cg_status pod_cg_solve(pod_cg_t* h, const pod_cg_csr* A, const double* b, double tol, double* x_out,
                           pod_cg_stats* stats)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    pod_cg_status cs = check_csr(h, A, h->n);
    if (cs != POD_CG_OK) return cs;
    if (!b || !x_out) return fail(h, POD_CG_ERR_ARG, "b and x_out must be non-NULL");
    if (b == x_out) return fail(h, POD_CG_ERR_ARG, "x_out may not alias b");
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(h, POD_CG_ERR_ARG, "tol must be finite and >= 0");
    if (h->cfg.precision != POD_CG_FP64) return fail(h, POD_CG_ERR_ARG, "precision mode not available");
    const int n = h->n;
    cudaStream_t s = h->stream;

    // problem descriptor and fresh device state
    *h->pd_host = ProbDesc{A->row_ptr, A->col, A->val, nullptr, b, nullptr, n, h->ld};
    PODCG_CK(h, cudaMemcpyAsync(h->pd, h->pd_host, sizeof(ProbDesc), cudaMemcpyHostToDevice, s));
    DevState& sh = *h->st_host;
    std::memset(&sh, 0, sizeof(DevState));
    sh.k_max = h->cfg.k_max;
    sh.max_refine = h->cfg.max_refine;
    sh.pod_w = h->pod_w;
    sh.w = h->pod_w;
    PODCG_CK(h, cudaMemcpyAsync(h->st, &sh, sizeof(DevState), cudaMemcpyHostToDevice, s));
    PODCG_CK(h, cudaEventRecord(h->ev[0], s));
    PODCG_CK(h, launch_dinv(h->pd, n, h->dinv, h->dinv32, h->st, h->sms, s));

    int launches = 2;   // dinv, stage-one lift
    // POD of the current snapshots (Algorithm 4)
    if (h->s_count > 0 && h->pod_dirty) {
        launches += 2;
        PODCG_CK(h, launch_pod_eig(h->GS, kSMax, h->s_count, h->cfg.energy, h->cfg.rank_tol, h->cfg.w_max, h->C,
                                   h->sigma2, h->st, s));
        PODCG_CK(h, launch_lift(n, h->S, h->ld, h->s_count, h->C, h->st, h->W, h->ld, h->sms, s));
        PODCG_CK(h, cudaMemcpyAsync(&sh.pod_w, &h->st->pod_w, sizeof(int), cudaMemcpyDeviceToHost, s));
        PODCG_CK(h, cudaStreamSynchronize(s));
        h->pod_w = sh.pod_w;
        h->pod_dirty = false;
    } else if (h->s_count == 0) {
        h->pod_w = 0;
    }
    const int w = h->pod_w;
    PODCG_CK(h, cudaEventRecord(h->ev[1], s));

    // stage one (Algorithm 2)
    if (w > 0) {
        PODCG_CK(h, launch_spmm(A->row_ptr, A->col, A->val, h->W, h->ld, h->AW, h->ld, n, w, h->sms, s));
        PODCG_CK(h, launch_gram(n, h->W, h->ld, w, h->AW, h->ld, w, b, h->G, kWMax + 1, 1, h->gram_work,
                                h->gram_work_bytes, h->sms, s));
        PODCG_CK(h, launch_chol(h->G, kWMax + 1, h->Rinv, h->st, h->cfg.cond_diag, s));
        launches += 4;   // spmm, gram partial + reduce, cholesky
    }
    const int wb = wb_bucket(w);
    PODCG_CK(h, launch_stage1(wb, h->pd, n, h->W, h->AW, h->x, h->r, h->partials, h->counters + 4, h->st, tol,
                              h->sms, s));
    PODCG_CK(h, cudaEventRecord(h->ev[2], s));

    // stage two: the captured loop
    const double mean_row = n > 0 ? double(A->nnz) / n : 1.0;
    const int L = spmv_lanes_for(mean_row);
    GraphSlot& gs = h->graphs[bucket_index(wb)][0];
    if (gs.valid && gs.L != L) destroy_graph(gs);
    if (!gs.valid) {
        pod_cg_status bs = build_graph_fp64(h, wb, L, gs);
        if (bs != POD_CG_OK) return bs;
    }
    PODCG_CK(h, cudaGraphLaunch(gs.exec, s));
    PODCG_CK(h, cudaEventRecord(h->ev[3], s));
    PODCG_CK(h, cudaMemcpyAsync(x_out, h->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    PODCG_CK(h, cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    PODCG_CK(h, cudaStreamSynchronize(s));

    const DevState& d = *h->st_host;
    const int sysid = h->system_counter++;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->status = d.status;
        stats->iters = d.iters;
        stats->refinements = d.restarts;
        stats->w = d.w;
        stats->s = h->s_count;
        stats->chol_failed = d.chol_failed;
        stats->system_id = sysid;
        stats->spmv_count = d.iters + w + d.restarts + 1;
        // graph: per outer pass init + first direction + residual; per iteration 3 kernels
        stats->launches = launches + 3 * (d.restarts + 1) + 3 * d.iters;
        stats->stage1_relres = d.bb > 0.0 ? std::sqrt(d.rr_stage1 / d.bb) : 0.0;
        stats->final_relres = d.bb > 0.0 ? std::sqrt(d.rr_true / d.bb) : 0.0;
        stats->cond_gram = d.cond;
        cudaEventElapsedTime(&stats->ms_pod, h->ev[0], h->ev[1]);
        cudaEventElapsedTime(&stats->ms_stage1, h->ev[1], h->ev[2]);
        cudaEventElapsedTime(&stats->ms_stage2, h->ev[2], h->ev[3]);
    }
    if (d.status != 0) {
        static const char* names[] = {"ok", "arg", "not SPD (non-positive diagonal)", "breakdown: (Ap, p) <= 0",
                                      "iteration/refinement cap reached", "non-finite scalar"};
        const char* nm = (d.status >= 0 && d.status <= 5) ? names[d.status] : "error";
        return fail(h, (pod_cg_status)d.status, std::string("solve: ") + nm);
    }
    return POD_CG_OK;
}

pod_cg_status pod_cg_solve_adjoint(pod_cg_t* h, int system_id, const pod_cg_csr* A, const double* g, double tol,
                                   double* lambda_out, pod_cg_stats* st)
{
    (void)system_id; (void)A; (void)g; (void)tol; (void)lambda_out; (void)st;
    return fail(h, POD_CG_ERR_STATE, "adjoint factors not kept");
}

pod_cg_status pod_cg_time_kernels(pod_cg_t* h, const pod_cg_csr* A, const double* b, int reps, float* ms_out)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    pod_cg_status cs = check_csr(h, A, h->n);
    if (cs != POD_CG_OK) return cs;
    if (!b || !ms_out || reps < 1) return fail(h, POD_CG_ERR_ARG, "bad arguments");
    const int n = h->n, ld = h->ld;
    cudaStream_t s = h->stream;
    *h->pd_host = ProbDesc{A->row_ptr, A->col, A->val, nullptr, b, nullptr, n, h->ld};
    PODCG_CK(h, cudaMemcpyAsync(h->pd, h->pd_host, sizeof(ProbDesc), cudaMemcpyHostToDevice, s));
    const int w = h->pod_w;
    const int wb = wb_bucket(w);
    const int L = spmv_lanes_for(n > 0 ? double(A->nnz) / n : 1.0);
    const int grid = grid_rows(n, kBlock, h->sms);
    const int grid_spmv = grid_rows(n, kBlock / L, h->sms);
    void *k_init_f, *k_upd_f, *k_dir0_f, *k_dir_f;
    cg_kernels(wb, false, &k_init_f, &k_upd_f, &k_dir0_f, &k_dir_f);
    void* k_spmv_f = kernel_spmv_cg(L, false);
    void* k_res_f = kernel_residual(L);
    DevState tmpl;
    std::memset(&tmpl, 0, sizeof(tmpl));
    tmpl.rho = 1.0;
    tmpl.alpha = 1e-30;
    tmpl.beta = 0.5;
    tmpl.w = w;
    tmpl.pod_w = w;
    tmpl.k_max = 1 << 30;
    tmpl.max_refine = 1 << 30;
    tmpl.tol2 = 0.0;
    tmpl.tol2_in = -1.0;
    *h->st_host = tmpl;
    const double* cW = h->W;
    const double* cAW = h->AW;
    const double* cRinv = h->Rinv;
    const double* cdinv = h->dinv;
    const double* cr = h->r;
    const double* cq = h->q;
    const double* cp = h->p;
    const double* cx = h->x;
    const DevState* cst = h->st;
    const ProbDesc* cpd = h->pd;
    cudaGraphConditionalHandle h0 = 0;
    int no_cond = 0, zero = 0;
    double inner_tol = h->cfg.inner_tol;
    unsigned int* c2 = h->counters + 2;
    unsigned int* c3 = h->counters + 3;
    unsigned int* c1 = h->counters + 1;
    void* a_spmv[] = {(void*)&cpd, (void*)&cp, (void*)&h->q, (void*)&h->partials, (void*)&c2, (void*)&h->st};
    void* a_upd[] = {(void*)&n, (void*)&ld, (void*)&h->r, (void*)&cq, (void*)&cdinv, (void*)&cAW, (void*)&cRinv,
                     (void*)&h->partials, (void*)&c3, (void*)&h->st, (void*)&h0, (void*)&no_cond};
    void* a_dir[] = {(void*)&n, (void*)&ld, (void*)&h->x, (void*)&h->p, (void*)&cr, (void*)&cdinv, (void*)&cW,
                     (void*)&cst};
    void* a_res[] = {(void*)&cpd, (void*)&cx, (void*)&h->r, (void*)&h->partials, (void*)&c1, (void*)&h->st,
                     (void*)&zero, (void*)&inner_tol, (void*)&h0, (void*)&no_cond};
    struct K { void* f; int g; void** a; } ks[4] = {{k_spmv_f, grid_spmv, a_spmv}, {k_upd_f, grid, a_upd},
                                                   {k_dir_f, grid, a_dir}, {k_res_f, grid_spmv, a_res}};
    for (int k = 0; k < 4; ++k) {
        float total = 0.0f;
        for (int rep = 0; rep < reps + 1; ++rep) {
            PODCG_CK(h, cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, s));
            PODCG_CK(h, cudaEventRecord(h->ev[0], s));
            PODCG_CK(h, cudaLaunchKernel(ks[k].f, dim3(ks[k].g), dim3(kBlock), ks[k].a, 0, s));
            PODCG_CK(h, cudaEventRecord(h->ev[1], s));
            PODCG_CK(h, cudaEventSynchronize(h->ev[1]));
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
            if (rep > 0) total += ms;   // first launch is a warm-up
        }
        ms_out[k] = total / reps;
    }
    return POD_CG_OK;
}

// ----------------------------------------------------------------- stateless steps

pod_cg_status pod_cg_spmv(const pod_cg_csr* A, const double* x, double* y, void* stream)
{
    if (!A || A->n < 0 || !x || !y) return fail(nullptr, POD_CG_ERR_ARG, "bad arguments");
    if (A->n == 0) return POD_CG_OK;
    const int L = spmv_lanes_for(double(A->nnz) / A->n);
    cudaError_t e = launch_spmv_plain(L, A->row_ptr, A->col, A->val, x, y, A->n, device_sms(), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, "pod_cg_spmv", e);
    return POD_CG_OK;
}

pod_cg_status pod_cg_spmm(const pod_cg_csr* A, const double* W, int w, double* AW, void* stream)
{
    if (!A || A->n < 0 || w < 0 || w > kWMax || (w > 0 && (!W || !AW))) return fail(nullptr, POD_CG_ERR_ARG, "bad arguments");
    if (A->n == 0 || w == 0) return POD_CG_OK;
    cudaError_t e = launch_spmm(A->row_ptr, A->col, A->val, W, A->n, AW, A->n, A->n, w, device_sms(), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, "pod_cg_spmm", e);
    return POD_CG_OK;
}

size_t pod_cg_gram_workspace(int n, int p, int q)
{
    if (n < 1 || p < 1 || q < 1) return 0;
    return gram_workspace_bytes(n, p, q, device_sms());
}

pod_cg_status pod_cg_gram(int n, const double* X, int p, const double* Y, int q, double* G, void* work,
                          size_t work_bytes, void* stream)
{
    if (n < 1 || p < 1 || q < 1 || p > kWMax + 1 || q > kWMax + 1 || !X || !Y || !G || !work)
        return fail(nullptr, POD_CG_ERR_ARG, "bad arguments");
    if (work_bytes < gram_workspace_bytes(n, p, q, device_sms())) return fail(nullptr, POD_CG_ERR_ARG, "workspace too small");
    cudaError_t e = launch_gram(n, X, n, p, Y, n, q, nullptr, G, q, 0, (double*)work, work_bytes, device_sms(),
                                (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, "pod_cg_gram", e);
    return POD_CG_OK;
}

pod_cg_status pod_cg_pod(int n, int s, const double* S, double energy, double rank_tol, int w_max, double* W_out,
                         double* sigma2_out, int* w_out, void* work, size_t work_bytes, void* stream)
{
    if (n < 1 || s < 1 || s > kSMax || w_max < 1 || w_max > kWMax || !S || !W_out || !sigma2_out || !w_out || !work)
        return fail(nullptr, POD_CG_ERR_ARG, "bad arguments");
    cudaStream_t str = (cudaStream_t)stream;
    const int sms = device_sms();
    if (work_bytes < gram_workspace_bytes(n, s, s, sms)) return fail(nullptr, POD_CG_ERR_ARG, "workspace too small");
    double *G = nullptr, *C = nullptr;
    DevState* st = nullptr;
    cudaError_t e = cudaMalloc((void**)&G, sizeof(double) * kSMax * kSMax);
    if (e == cudaSuccess) e = cudaMalloc((void**)&C, sizeof(double) * kSMax * kWMax);
    if (e == cudaSuccess) e = cudaMalloc((void**)&st, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(DevState), str);
    if (e == cudaSuccess) e = launch_gram(n, S, n, s, S, n, s, nullptr, G, kSMax, 0, (double*)work, work_bytes, sms, str);
    if (e == cudaSuccess) e = launch_pod_eig(G, kSMax, s, energy, rank_tol, w_max, C, sigma2_out, st, str);
    if (e == cudaSuccess) e = launch_lift(n, S, n, s, C, st, W_out, n, sms, str);
    int w = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&w, &st->pod_w, sizeof(int), cudaMemcpyDeviceToHost, str);
    if (e == cudaSuccess) e = cudaStreamSynchronize(str);
    cudaFree(G);
    cudaFree(C);
    cudaFree(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, "pod_cg_pod", e);
    *w_out = w;
    return POD_CG_OK;
}

}  // extern "C"
