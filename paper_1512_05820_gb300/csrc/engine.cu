// Solver engine and C ABI (include/pod_cg.h).
//
// A handle owns the snapshot ring S (column-major, leading dimension ld = n rounded up to
// 32), its Gram S^T S (kept up to date one row per added snapshot), the POD basis W, A W,
// the stage-one Gram and R^{-1}, the CG vectors, reduction scratch and the captured graphs.
//
// pod_cg_solve enqueues, on the handle's stream (stages numbered as in Section 4):
//   POD (when the snapshots changed): Jacobi eigensolve of S^T S, truncation, lift W = S C
//     (three-stage mode: lift the augmenting basis Y = S C and copy W = its first w columns)
//   stage one: A W, W^T [A W, b] (three-stage: Y^T [A W, b]), Cholesky + R^{-1} + what
//   stage two (three-stage mode only, k_stage2.cu): reduced augmented CG over range(Y),
//     appending its directions V2 and A V2 to the basis buffers
//   x0 = [W, V2] [what; alpha], r0 = b - [A W, A V2] [what; alpha]
//   the stage-three loop (Algorithm 1 with basis [W, V2]), either
//     loop_mode 0: one graph launch with two nested conditional while-nodes
//        FP64 : outer (residual replacement) { init; first direction;
//                 inner { q = A p; update; direction }; true residual }
//        mixed: outer (refinement) { FP64 residual; projection of the correction onto W;
//                 FP32 init; first direction; inner { ... in FP32 }; x += d }
//     loop_mode 1: the same kernels, the inner loop as a plain graph of 16 unrolled
//        iterations (later ones return at once after convergence), host check per chunk.
//     loop_mode 2: as 0, the mixed inner loop (bases up to 8 wide, one lane per CSR row)
//        as one persistent cooperative launch per refinement step (k_loop.cu).
// The host synchronises once to learn w (which selects the kernel width bucket) and once
// at the end for the statistics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <string>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "pod_cg.h"

using namespace podcg;

namespace {

thread_local std::string g_last_error;
constexpr int kQMax = 128;   // output functionals of the output-oriented POD metric
constexpr int kChunk = 16;   // iterations per plain graph in loop_mode 1

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

// Kernel arguments stored by value with stable addresses (a spec is built in place and
// never copied, so the pointer array stays valid for graph-node creation and launches).
struct KArgs {
    alignas(64) unsigned char buf[512];
    size_t off = 0;
    void* ptrs[24];
    int count = 0;
    template <typename T>
    void add(T v)
    {
        off = (off + alignof(T) - 1) & ~(alignof(T) - 1);
        std::memcpy(buf + off, &v, sizeof(T));
        ptrs[count++] = buf + off;
        off += sizeof(T);
    }
};

struct KSpec {
    void* f = nullptr;
    int grid = 1;
    int block = kBlock;   // threads per block
    int smem = 0;         // dynamic shared memory bytes
    KArgs a;
    KSpec() = default;
    KSpec(const KSpec&) = delete;
    KSpec& operator=(const KSpec&) = delete;
    template <typename... Args>
    void set(void* func, int g, Args... args)
    {
        f = func;
        grid = g;
        a.off = 0;
        a.count = 0;
        (a.add(args), ...);
    }
};

struct Plan {
    KSpec init, dir0, spmv, upd, dir, res, mxproj, mxstart, mxaccum;
    KSpec loop;               // the FP32 inner loop as one persistent cooperative kernel
    bool persistent = false;  // the inner loop body is `loop` alone
};

struct Stage2Plan {
    KSpec bb, init, lift, apply;
};

struct GraphSlot {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int L = 0;
    int yb = 0;   // stage-two graphs: the y bucket they were built for
    bool bsr = false;   // built with the 3x3 block product
    bool valid = false;
};

cudaError_t add_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps, KSpec& k, cudaGraphNode_t* out)
{
    cudaKernelNodeParams p = {};
    p.func = k.f;
    p.gridDim = dim3(k.grid);
    p.blockDim = dim3(k.block);
    p.sharedMemBytes = (unsigned int)k.smem;
    p.kernelParams = k.a.ptrs;
    p.extra = nullptr;
    return cudaGraphAddKernelNode(out, g, deps, ndeps, &p);
}

// A kernel node hanging off `dep` by a programmatic edge (programmatic dependent launch):
// its blocks may be scheduled once every block of `dep` has started; the loop kernels wait
// for their prerequisites' completion before their first access. PODCG_PDL=0 in the
// environment makes it a plain edge (the same graph without the overlap, for comparison).
cudaError_t add_node_after(cudaGraph_t g, cudaGraphNode_t dep, KSpec& k, cudaGraphNode_t* out)
{
    static const bool pdl = [] {
        const char* e = std::getenv("PODCG_PDL");
        return !(e && e[0] == '0');
    }();
    if (!pdl) return add_node(g, &dep, 1, k, out);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeKernel;
    np.kernel.func = k.f;
    np.kernel.gridDim = dim3(k.grid);
    np.kernel.blockDim = dim3(k.block);
    np.kernel.sharedMemBytes = (unsigned int)k.smem;
    np.kernel.kernelParams = k.a.ptrs;
    np.kernel.extra = nullptr;
    cudaGraphEdgeData ed = {};
    ed.from_port = cudaGraphKernelNodePortProgrammatic;
    ed.to_port = cudaGraphKernelNodePortDefault;
    ed.type = cudaGraphDependencyTypeProgrammatic;
    return cudaGraphAddNode(out, g, &dep, &ed, 1, &np);
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

cudaError_t launch_spec(KSpec& k, cudaStream_t s)
{
    return cudaLaunchKernel(k.f, dim3(k.grid), dim3(k.block), k.a.ptrs, (size_t)k.smem, s);
}

}  // namespace

struct pod_cg_t {
    int n = 0, ld = 0, sms = 1, device = 0;
    bool mixed = false;
    pod_cg_config cfg{};
    cudaStream_t stream = nullptr;
    std::string err;

    // snapshots and POD
    double* S = nullptr;        // ld x s_max
    float* S32 = nullptr;       // ld x s_max (mixed)
    double* GS = nullptr;       // kSMax x kSMax row-major (slot order)
    double* grow = nullptr;     // one Gram row (kSMax)
    double* C = nullptr;        // kSMax x kWMax lift coefficients
    double* sigma2 = nullptr;   // kSMax eigenvalues
    double* Vprev = nullptr;    // kSMax x kSMax eigenvectors of the last POD (warm start)
    int vprev_s = 0;            // slots covered by Vprev (0: none)
    int s_count = 0, s_next = 0;
    bool pod_dirty = false;
    int pod_w = 0;

    // basis and stage one
    double* W = nullptr;        // ld x wcap: W, then (three-stage) the stage-two basis V2
    double* AW = nullptr;       // ld x wcap: A W, then A V2
    float* W32 = nullptr;       // mixed
    float* AW32 = nullptr;      // mixed
    __half* W16 = nullptr;      // mixed, two-stage: 16-bit copy of W32 (W32 = W16 * wscale exactly)
    float* wscale = nullptr;    // its power-of-two column scales (kWMax)
    unsigned int* wmax = nullptr;   // scratch of the column maxima (kWMax)
    CUtensorMap* tm_dev = nullptr;    // tensor maps of the panels A W32, W32, W16 (device, 3)
    CUtensorMap* tm_host = nullptr;   // their host copy (pinned)
    int tm_cols = -1;           // basis width the maps were encoded for
    bool tm_ok = false;         // maps can be encoded (else only the float4 form is used)
    bool w16 = false;           // the staged direction pass reads W16
    int wcap = 0;               // columns of the basis buffers: w_max, or kWMax in three-stage mode
    double* Y = nullptr;        // three-stage: augmenting basis, ld x max(y_max, w_max)
    float* Y32 = nullptr;       // three-stage, mixed: its FP32 copy (stage-one panels)
    double* s2_hist = nullptr;  // three-stage: stage-two reduced directions, products, gammas
    double* s2tmp = nullptr;    // whole-Y stage three: the inner solves' lifted v and A v
    int pod_y = 0;              // augmenting-basis dimension of the current POD
    int pod_y_used = 0;         // last solve: y when stage two ran, else 0
    int k2 = 0, k2_launch = 0;  // last solve: stage-two iterations, their loop bodies run
    bool w_clobbered = false;   // stage two wrote over W's columns (stage-one Cholesky failed)
    bool it_mode = false;       // last solve ran stage three over the whole Y

    // output-oriented POD metric C^T C (Section 3.3): the q functionals and C s per slot
    int out_q = 0;
    double* Cout = nullptr;      // q x n row-major (functional i at Cout + i n)
    double* CSv = nullptr;       // C s_k for slot k at CSv + k * kQMax
    double* GSC = nullptr;       // kSMax x kSMax Gram (C S)^T (C S), slot order
    double* out_work = nullptr;  // workspace of the products C s
    size_t out_work_bytes = 0;
    // POD metric A (pod_metric = 1): A S and S^T A S of the system being solved
    double* AS = nullptr;        // ld x s_max
    double* GA = nullptr;        // kSMax x kSMax

    // 3x3 block form of the CG product (k_bsr.cu): pattern cache and buffers
    const int32_t* bsr_key = nullptr;   // row_ptr of the pattern checked last
    int bsr_key_n = 0;
    int64_t bsr_key_nnz = -1;
    bool bsr_ok = false;                // that pattern is made of full 3x3 blocks
    bool use_bsr = false;               // the current solve uses the block form
    int bsr_L = 8;
    bool bsr_timed = false;             // lanes per block row timed for the current pattern
    int32_t *brp = nullptr, *bcol = nullptr;
    double* bval = nullptr;
    float* bval32 = nullptr;
    int64_t bsr_cap = 0;                // blocks the value buffers hold
    int* bsr_flag = nullptr;
    double* G = nullptr;        // kWMax x (kWMax + 1) row-major
    double* Rinv = nullptr;     // kWMax x kWMax
    double* Mmu = nullptr;      // R^{-1} R^{-T} (mixed: the direction passes' mu = M c), kWMax x kWMax

    // vectors
    double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *dinv = nullptr;
    float* dinv32 = nullptr;
    float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;   // mixed
    float* val32 = nullptr;     // mixed: FP32 copy of A's values
    int64_t val32_cap = 0;

    // reductions
    double* partials = nullptr;
    unsigned int* counters = nullptr;   // 8 reduction sites x kCounterStride
    unsigned int* gbar = nullptr;       // the persistent loop's grid barrier (count, generation)
    double* gram_work = nullptr;
    size_t gram_work_bytes = 0;

    DevState* st = nullptr;
    DevState* st_host = nullptr;        // pinned
    ProbDesc* pd = nullptr;
    ProbDesc* pd_host = nullptr;        // pinned

    // factors kept for the adjoint
    double* kW = nullptr;
    double* kAW = nullptr;
    double* kG = nullptr;
    std::vector<int> k_id, k_w;
    int k_next = 0;

    // SpMV lanes-per-row autotuner: one entry per sparsity pattern seen
    struct LaneChoice { const int32_t* rp; int n; int64_t nnz; bool mixed; int L; float ms[6]; };
    std::vector<LaneChoice> lanes;
    int last_L = 0;
    // FP32 projection form per width bucket (kProjDirect / kProjStaged, -1 = not chosen yet)
    // and the update + direction times that chose it (ms, [bucket][form])
    int proj_form[6] = {-1, -1, -1, -1, -1, -1};   // bit 0: update pass staged, bit 1: direction
    float proj_ms[6][2][2] = {};                     // [bucket][form][update, direction]
    DevState* st_save = nullptr;   // device copy of the state while the form is timed

    // the paper's snapshots (Section 3.1, Algorithm 3): accumulated Krylov vectors
    bool kry_on = false;
    pod_cg_krylov_config kc{};
    double* Z = nullptr;        // ld x kSMax: augmenting basis, columns in append order
    double* Zalt = nullptr;     // ld x kSMax: Z diag(eta) during a compression
    double* AZ = nullptr;       // ld x kSMax: A Z (A Z diag(eta) during a compression)
    double* kgam = nullptr;     // kSMax: (A p_k, p_k) of the recorded directions
    double* zG = nullptr;       // kSMax x (kSMax + 1) row-major: Z^T [A Z, b]
    double* zG2 = nullptr;      // kSMax x kSMax: the weighted Gram of a compression
    double* zcoord = nullptr;   // kSMax: coordinates of the last solution in Z
    double* zeta = nullptr;     // kSMax: POD weights accumulated since the last compression
    int z = 0;                  // columns of Z
    std::vector<int> w_idx;     // columns of Z that form the stage-one basis
    int compressions = 0;
    int kry_cap = 0;            // directions the current solve may record

    GraphSlot graphs[6];                // conditional graphs [width bucket]
    GraphSlot chunks[6];                // plain chunk graphs [width bucket]
    GraphSlot s2graph;                  // stage-two conditional graph
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};   // solve timeline (ev[5]: loop start)
    // cost-tuned cap on w (w_select = 1): candidates, visit order, summed device ms and counts
    std::vector<int> wsel_caps, wsel_order;
    std::vector<double> wsel_ms;
    std::vector<int> wsel_n;
    int wsel_pos = 0;           // next position in wsel_order
    bool wsel_done = false;
    int w_cap = 0;              // cap chosen (valid when wsel_done)
    int cap_now = 0;            // cap of the current solve
    // stage-one Gram of MIXED two-stage solves (use_tc_gram = -1): per basis width, -1 = not
    // timed yet, 0 = CUDA cores (FP32 panels), 1 = tensor cores; the times that chose it
    signed char gram_choice[kWMax + 1];
    float gram_ms[kWMax + 1][2] = {};
    int last_gram_tc = 0;       // the last solve's stage-one Gram ran on the tensor cores
    int wsel_slot = -1;         // candidate index timed by the current solve (-1: none)
    cudaEvent_t tev[2] = {nullptr, nullptr};                              // autotuner timing
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

#define PODCG_CK(h, call)                                      \
    do {                                                       \
        cudaError_t e_ = (call);                               \
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

// SpMV lanes per row for this pattern: the mean-row-length heuristic for small systems;
// otherwise the candidates around it are timed on the actual matrix (plain product in the
// solve's precision, CUDA events) and the fastest is kept for the pattern.
pod_cg_status choose_lanes(pod_cg_t* h, const pod_cg_csr* A, int* L_out)
{
    for (auto& c : h->lanes)
        if (c.rp == A->row_ptr && c.n == A->n && c.nnz == A->nnz && c.mixed == h->mixed) {
            *L_out = c.L;
            return POD_CG_OK;
        }
    const double mean = A->n > 0 ? double(A->nnz) / A->n : 1.0;
    pod_cg_t::LaneChoice ch{A->row_ptr, A->n, A->nnz, h->mixed, spmv_lanes_for(mean), {0, 0, 0, 0, 0, 0}};
    if (h->cfg.spmv_lanes > 0) {
        ch.L = h->cfg.spmv_lanes;
    } else if (A->n >= 65536) {
        const int cands[6] = {1, 2, 4, 8, 16, 32};
        const int heur = ch.L;
        float best = -1.0f, t_heur = -1.0f;
        int best_L = heur;
        for (int k = 0; k < 6; ++k) {
            const int L = cands[k];
            if (L > 4 * mean + 4 || L * 16 < mean) { ch.ms[k] = -1.0f; continue; }
            float tot = 0.0f;
            for (int rep = 0; rep < 4; ++rep) {
                PODCG_CK(h, cudaEventRecord(h->tev[0], h->stream));
                if (h->mixed)
                    PODCG_CK(h, launch_spmv_plain32(L, A->row_ptr, A->col, h->val32, h->p32, h->q32, A->n, h->sms,
                                                    h->stream));
                else
                    PODCG_CK(h, launch_spmv_plain(L, A->row_ptr, A->col, A->val, h->p, h->q, A->n, h->sms, h->stream));
                PODCG_CK(h, cudaEventRecord(h->tev[1], h->stream));
                PODCG_CK(h, cudaEventSynchronize(h->tev[1]));
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, h->tev[0], h->tev[1]);
                if (rep > 0) tot += ms;
            }
            ch.ms[k] = tot / 3.0f;
            if (L == heur) t_heur = ch.ms[k];
            if (best < 0.0f || ch.ms[k] < best) { best = ch.ms[k]; best_L = L; }
        }
        // keep the heuristic width unless another is clearly (>= 10%) faster: one noisy
        // timing must not switch the kernel
        ch.L = (t_heur > 0.0f && best >= 0.9f * t_heur) ? heur : best_L;
    }
    h->lanes.push_back(ch);
    *L_out = ch.L;
    return POD_CG_OK;
}

void make_plan(pod_cg_t* h, int wb, int L, bool mixed, int use_cond, cudaGraphConditionalHandle h_inner,
               cudaGraphConditionalHandle h_outer, Plan& P);
pod_cg_status read_state(pod_cg_t* h);

// FP32 projection form for width bucket wb: both forms of the update and direction passes
// are timed once on this system (CUDA events, median-free mean of 3 after a warm-up) and
// the faster pair is kept for the bucket. The device state is saved first and restored
// after; the FP32 vectors the passes touch are scratch until the loop starts. Systems
// under 65,536 rows take the direct form untimed.
// The panels' tensor maps for a basis of `cols` columns (the TMA-staged passes): encoded on
// the host and copied to the device when the width changes (stream-ordered before the loop).
pod_cg_status set_panel_maps(pod_cg_t* h, int cols)
{
    if (!h->tm_ok || cols < 1 || cols == h->tm_cols) return POD_CG_OK;
    if (!encode_panel_map(&h->tm_host[0], h->AW32, 4, h->ld, cols, 8) ||
        !encode_panel_map(&h->tm_host[1], h->W32, 4, h->ld, cols, 8) ||
        !encode_panel_map(&h->tm_host[2], h->W16, 2, h->ld, cols, 16))
        return fail(h, POD_CG_ERR_CUDA, "tensor map encoding failed");
    PODCG_CK(h, cudaMemcpyAsync(h->tm_dev, h->tm_host, 3 * sizeof(CUtensorMap), cudaMemcpyHostToDevice, h->stream));
    PODCG_CK(h, cudaStreamSynchronize(h->stream));   // the host copy may be rewritten by the next solve
    h->tm_cols = cols;
    return POD_CG_OK;
}

pod_cg_status choose_proj_form(pod_cg_t* h, int wb, int L)
{
    const int bi = bucket_index(wb);
    if (!h->mixed || wb == 0 || h->proj_form[bi] >= 0) return POD_CG_OK;
    if (h->n < 65536 || !h->tm_ok) {
        h->proj_form[bi] = kProjDirect;
        return POD_CG_OK;
    }
    cudaStream_t s = h->stream;
    PODCG_CK(h, cudaMemcpyAsync(h->st_save, h->st, sizeof(DevState), cudaMemcpyDeviceToDevice, s));
    pod_cg_status rs = read_state(h);
    if (rs != POD_CG_OK) return rs;
    DevState t = *h->st_host;   // a state under which both passes do their full work
    t.rho = 1.0;
    t.alpha = 1e-30;
    t.beta = 0.5;
    t.k_max = 1 << 30;
    t.tol2_in = -1.0;
    t.dir_pending = 1;
    t.done = 0;
    t.status = 0;
    t.inner_break = 0;
    t.outer_done = 0;
    for (int a = 0; a < kWMax; ++a) t.c[a] = 0.0;
    *h->st_host = t;
    // each form times its update pass, then its direction pass (which reads the partials of
    // the update pass of the same form); each pass keeps its faster form. Before every timed
    // launch 256 MB are written, so the panels are not left in L2 by the previous launch (in
    // the loop the CG product streams the matrix between two passes; a narrow basis would
    // otherwise be timed from L2)
    void* flush = nullptr;
    const size_t flush_bytes = size_t(256) << 20;
    if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        cudaGetLastError();
        flush = nullptr;
    }
    for (int form = kProjDirect; form <= kProjStaged; ++form) {
        h->proj_form[bi] = form == kProjStaged ? 3 : 0;
        Plan pl;
        make_plan(h, wb, L, true, 0, 0, 0, pl);
        KSpec* ks[2] = {&pl.upd, &pl.dir};
        for (int k = 0; k < 2; ++k) {
            float total = 0.0f;
            for (int rep = 0; rep < 4; ++rep) {
                PODCG_CK(h, cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, s));
                if (flush) PODCG_CK(h, cudaMemsetAsync(flush, rep, flush_bytes, s));
                PODCG_CK(h, cudaEventRecord(h->tev[0], s));
                PODCG_CK(h, launch_spec(*ks[k], s));
                PODCG_CK(h, cudaEventRecord(h->tev[1], s));
                PODCG_CK(h, cudaEventSynchronize(h->tev[1]));
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, h->tev[0], h->tev[1]);
                if (rep > 0) total += ms;
            }
            h->proj_ms[bi][form][k] = total / 3.0f;
        }
    }
    if (flush) cudaFree(flush);
    h->proj_form[bi] = (h->proj_ms[bi][kProjStaged][0] < h->proj_ms[bi][kProjDirect][0] ? 1 : 0) |
                       (h->proj_ms[bi][kProjStaged][1] < h->proj_ms[bi][kProjDirect][1] ? 2 : 0);
    PODCG_CK(h, cudaMemcpyAsync(h->st, h->st_save, sizeof(DevState), cudaMemcpyDeviceToDevice, s));
    return read_state(h);
}

// One wave: as many blocks as are resident at once (occupancy), never more than needed.
int occ_grid(pod_cg_t* h, const void* f, int rows, int rows_per_block, int smem = 0)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kBlock, (size_t)smem) != cudaSuccess || nb < 1) nb = 1;
    long long need = ((long long)rows + rows_per_block - 1) / rows_per_block;
    long long cap = (long long)h->sms * nb;
    long long g = std::min(need, cap);
    g = std::min<long long>(g, kPartialStride - kRedGroups);
    return (int)std::max<long long>(g, 1);
}

void make_plan(pod_cg_t* h, int wb, int L, bool mixed, int use_cond, cudaGraphConditionalHandle h_inner,
               cudaGraphConditionalHandle h_outer, Plan& P)
{
    const int n = h->n, ld = h->ld;
    void *f_init, *f_upd, *f_dir0, *f_dir;
    int sm_upd = 0, sm_dir = 0;
    // FP32 with a basis: the form of each pass (bit 0 of the bucket's choice: the update pass
    // staged by the TMA engine, bit 1: the direction pass)
    const int pf = (mixed && wb > 0 && h->tm_ok && h->proj_form[bucket_index(wb)] > 0) ? h->proj_form[bucket_index(wb)] : 0;
    const int form_u = (pf & 1) ? kProjStaged : kProjDirect, form_d = (pf & 2) ? kProjStaged : kProjDirect;
    cg_kernels(wb, mixed, use_cond != 0, form_d, h->w16, &f_init, &f_upd, &f_dir0, &f_dir, &sm_upd, &sm_dir);
    if (form_u != form_d) {
        void *i2, *d02, *d2;
        int sd2 = 0;
        cg_kernels(wb, mixed, use_cond != 0, form_u, h->w16, &i2, &f_upd, &d02, &d2, &sm_upd, &sd2);
    }
    // the CG product: CSR, or the 3x3 block form when the pattern has one (k_bsr.cu)
    void* f_spmv = h->use_bsr ? kernel_bsr_spmv_cg(h->bsr_L, mixed) : kernel_spmv_cg(L, mixed);
    void* f_res = kernel_residual(L, use_cond != 0);
    const int g_init = occ_grid(h, f_init, n, kBlock);
    const int g_upd = occ_grid(h, f_upd, n, kBlock, sm_upd);
    const int g_dir = occ_grid(h, f_dir, n, kBlock, sm_dir);
    const int g_spmv = h->use_bsr ? occ_grid(h, f_spmv, n / 3, kBlock / h->bsr_L) : occ_grid(h, f_spmv, n, kBlock / L);
    const int g_res = occ_grid(h, f_res, n, kBlock / L);
    unsigned int* c = h->counters;
    const ProbDesc* pd = h->pd;
    DevState* st = h->st;
    const DevState* cst = h->st;
    const double* Rinv = h->Rinv;
    const double inner_tol = h->cfg.inner_tol;
    P.res.set(f_res, g_res, pd, (const double*)h->x, h->r, h->partials, c + 1 * kCounterStride, st, (int)mixed, inner_tol, h_outer,
              use_cond);
    if (!mixed) {
        P.init.set(f_init, g_init, n, ld, (const double*)h->r, (const double*)h->dinv, (const double*)h->AW,
                   h->partials, c + 0 * kCounterStride, st, h_inner, use_cond);
        P.dir0.set(f_dir0, g_dir, n, ld, h->x, h->p, (const double*)h->r, (const double*)h->dinv,
                   (const double*)h->W, Rinv, cst);
        P.spmv.set(f_spmv, g_spmv, pd, (const double*)h->p, h->q, h->partials, c + 2 * kCounterStride, st);
        P.upd.set(f_upd, g_upd, n, ld, h->r, (const double*)h->q, (const double*)h->dinv, (const double*)h->AW,
                  h->partials, c + 3 * kCounterStride, st, h_inner, use_cond);
        P.dir.set(f_dir, g_dir, n, ld, h->x, h->p, (const double*)h->r, (const double*)h->dinv,
                  (const double*)h->W, Rinv, cst);
    } else {
        void *f_proj, *f_start;
        mixed_kernels(wb, &f_proj, &f_start);
        void* f_acc = kernel_mx_accum();
        P.mxproj.set(f_proj, occ_grid(h, f_proj, n, kBlock), n, ld, (const double*)h->r, h->r32,
                     (const float*)h->W32, h->partials, c + 5 * kCounterStride, st);
        P.mxstart.set(f_start, occ_grid(h, f_start, n, kBlock), n, ld, h->d32, h->r32, (const float*)h->W32,
                      (const float*)h->AW32, Rinv, cst);
        P.init.set(f_init, g_init, n, ld, (const float*)h->r32, (const float*)h->dinv32, (const float*)h->AW32,
                   h->partials, c + 0 * kCounterStride, st, h_inner, use_cond);
        // the FP32 loop reduces without tails: the SpMV's partials feed the update pass, the
        // update pass's feed the direction pass, which sets the graph condition
        P.spmv.set(f_spmv, g_spmv, pd, (const float*)h->p32, h->q32, h->partials, c + 2 * kCounterStride, st);
        // the update pass at two blocks per SM at most: its partials feed every direction block
        const int gu = std::min(g_upd, 2 * h->sms);
        const double* M = h->Mmu;
        P.upd.set(f_upd, gu, n, ld, h->r32, (const float*)h->q32, (const float*)h->dinv32, (const float*)h->AW32,
                  h->partials, g_spmv, st);
        P.dir0.set(f_dir0, g_dir, n, ld, h->d32, h->p32, (const float*)h->r32, (const float*)h->dinv32,
                   (const float*)h->W32, (const __half*)h->W16, (const float*)h->wscale, Rinv, M,
                   (const double*)h->partials, gu, st, h_inner, 0);
        P.dir.set(f_dir, g_dir, n, ld, h->d32, h->p32, (const float*)h->r32, (const float*)h->dinv32,
                  (const float*)h->W32, (const __half*)h->W16, (const float*)h->wscale, Rinv, M,
                  (const double*)h->partials, gu, st, h_inner, use_cond);
        P.mxaccum.set(f_acc, occ_grid(h, f_acc, n, kBlock), n, h->x, (const float*)h->d32, cst);
        // loop_mode 2: the whole inner loop in one cooperative launch (CSR product with one
        // thread per row, bases up to 8 wide) inside the conditional graph
        const bool allow = h->cfg.loop_mode == 2;
        const int gl = (allow && use_cond && !h->use_bsr && L == 1 && wb <= 8) ? cg_loop_grid(wb, h->sms) : 0;
        if (gl > 0) {
            P.loop.set(kernel_cg_loop(wb), gl, pd, h->p32, h->q32, h->r32, h->d32, (const float*)h->dinv32,
                       (const float*)h->AW32, (const float*)h->W32, (const double*)h->Mmu, h->partials, h->gbar, st,
                       h_inner, use_cond);
            P.persistent = true;
        }
    }
    P.upd.smem = sm_upd;
    P.dir0.smem = sm_dir;
    P.dir.smem = sm_dir;
    if (mixed && wb > 0 && pf != 0) {
        // TMA-staged passes: the panels as tensor maps, ring and grid by the bucket's stage size;
        // the direction pass sums one partial per block of whichever update pass runs
        int gu = std::min(g_upd, 2 * h->sms);
        if (form_u == kProjStaged) {
            int ru, su;
            tma_shape(n, h->sms, wb, 8, 3, false, &gu, &ru, &su);
            P.upd.set(f_upd, gu, n, ld, ru, h->r32, (const float*)h->q32, (const float*)h->dinv32,
                      (const CUtensorMap*)h->tm_dev, h->partials, g_spmv, st);
            P.upd.block = tma_block_threads();
            P.upd.smem = su;
        }
        if (form_d == kProjStaged) {
            const CUtensorMap* tmW = h->tm_dev + (h->w16 ? 2 : 1);
            int gd, rd, sd;
            tma_shape(n, h->sms, wb, h->w16 ? 16 : 8, 4, true, &gd, &rd, &sd);
            P.dir0.set(f_dir0, gd, n, ld, rd, h->d32, h->p32, (const float*)h->r32, (const float*)h->dinv32, tmW,
                       (const float*)h->wscale, Rinv, (const double*)h->Mmu, (const double*)h->partials, gu, st,
                       h_inner, 0);
            P.dir.set(f_dir, gd, n, ld, rd, h->d32, h->p32, (const float*)h->r32, (const float*)h->dinv32, tmW,
                      (const float*)h->wscale, Rinv, (const double*)h->Mmu, (const double*)h->partials, gu, st,
                      h_inner, use_cond);
            P.dir0.block = P.dir.block = tma_block_threads();
            P.dir0.smem = P.dir.smem = sd;
        } else {
            P.dir0.set(f_dir0, g_dir, n, ld, h->d32, h->p32, (const float*)h->r32, (const float*)h->dinv32,
                       (const float*)h->W32, (const __half*)h->W16, (const float*)h->wscale, Rinv,
                       (const double*)h->Mmu, (const double*)h->partials, gu, st, h_inner, 0);
            P.dir.set(f_dir, g_dir, n, ld, h->d32, h->p32, (const float*)h->r32, (const float*)h->dinv32,
                      (const float*)h->W32, (const __half*)h->W16, (const float*)h->wscale, Rinv,
                      (const double*)h->Mmu, (const double*)h->partials, gu, st, h_inner, use_cond);
        }
    }
}

void destroy_graph(GraphSlot& gs)
{
    if (gs.exec) cudaGraphExecDestroy(gs.exec);
    if (gs.graph) cudaGraphDestroy(gs.graph);
    gs = GraphSlot();
}

// The whole stage-three loop as one graph with two nested conditional while-nodes.
pod_cg_status build_conditional(pod_cg_t* h, int wb, int L, GraphSlot& gs)
{
    cudaGraph_t P = nullptr, O = nullptr, I = nullptr;
    PODCG_CK(h, cudaGraphCreate(&P, 0));
    cudaGraphConditionalHandle h_outer, h_inner;
    PODCG_CK(h, cudaGraphConditionalHandleCreate(&h_outer, P, 1, cudaGraphCondAssignDefault));
    cudaGraphNode_t n_outer;
    PODCG_CK(h, add_while(P, nullptr, 0, h_outer, &n_outer, &O));
    PODCG_CK(h, cudaGraphConditionalHandleCreate(&h_inner, O, 0, 0));
    Plan pl;
    make_plan(h, wb, L, h->mixed, 1, h_inner, h_outer, pl);
    cudaGraphNode_t a, b, c, d, e, f, g, m1, m2, m3;
    if (!h->mixed) {
        PODCG_CK(h, add_node(O, nullptr, 0, pl.init, &a));
        PODCG_CK(h, add_node(O, &a, 1, pl.dir0, &b));
        PODCG_CK(h, add_while(O, &b, 1, h_inner, &c, &I));
        PODCG_CK(h, add_node(O, &c, 1, pl.res, &d));
    } else {
        PODCG_CK(h, add_node(O, nullptr, 0, pl.res, &a));
        PODCG_CK(h, add_node(O, &a, 1, pl.mxproj, &b));
        PODCG_CK(h, add_node(O, &b, 1, pl.mxstart, &c));
        PODCG_CK(h, add_node(O, &c, 1, pl.init, &d));
        PODCG_CK(h, add_node(O, &d, 1, pl.dir0, &e));
        PODCG_CK(h, add_while(O, &e, 1, h_inner, &f, &I));
        PODCG_CK(h, add_node(O, &f, 1, pl.mxaccum, &g));
    }
    if (pl.persistent) {   // one body pass runs every inner iteration, then clears the condition
        PODCG_CK(h, add_node(I, nullptr, 0, pl.loop, &m1));
        cudaLaunchAttributeValue v = {};
        v.cooperative = 1;
        PODCG_CK(h, cudaGraphKernelNodeSetAttribute(m1, cudaLaunchAttributeCooperative, &v));
    } else {
        PODCG_CK(h, add_node(I, nullptr, 0, pl.spmv, &m1));
        PODCG_CK(h, add_node_after(I, m1, pl.upd, &m2));
        PODCG_CK(h, add_node_after(I, m2, pl.dir, &m3));
    }
    cudaGraphExec_t exec = nullptr;
    PODCG_CK(h, cudaGraphInstantiate(&exec, P, 0));
    gs.graph = P;
    gs.exec = exec;
    gs.L = L;
    gs.bsr = h->use_bsr;
    gs.valid = true;
    return POD_CG_OK;
}

// kChunk unrolled inner iterations as a plain graph (no conditional nodes).
pod_cg_status build_chunk(pod_cg_t* h, int wb, int L, GraphSlot& gs)
{
    cudaGraph_t P = nullptr;
    PODCG_CK(h, cudaGraphCreate(&P, 0));
    Plan pl;
    make_plan(h, wb, L, h->mixed, 0, 0, 0, pl);
    cudaGraphNode_t prev = nullptr, cur;
    for (int it = 0; it < kChunk; ++it) {
        if (prev) PODCG_CK(h, add_node_after(P, prev, pl.spmv, &cur));
        else PODCG_CK(h, add_node(P, nullptr, 0, pl.spmv, &cur));
        prev = cur;
        PODCG_CK(h, add_node_after(P, prev, pl.upd, &cur));
        prev = cur;
        PODCG_CK(h, add_node_after(P, prev, pl.dir, &cur));
        prev = cur;
    }
    cudaGraphExec_t exec = nullptr;
    PODCG_CK(h, cudaGraphInstantiate(&exec, P, 0));
    gs.graph = P;
    gs.exec = exec;
    gs.L = L;
    gs.bsr = h->use_bsr;
    gs.valid = true;
    return POD_CG_OK;
}

// The 3x3 block form of A for the CG product: the pattern is checked and converted once
// per pattern (block-row pointers and columns), the values of every system are gathered.
// bsr = -1 uses it when the pattern allows, 1 requires it (ERR_ARG otherwise), 0 never.
pod_cg_status setup_bsr(pod_cg_t* h, const pod_cg_csr* A)
{
    h->use_bsr = false;
    if (h->cfg.bsr == 0) return POD_CG_OK;
    cudaStream_t s = h->stream;
    const int n = A->n;
    if (h->bsr_key != A->row_ptr || h->bsr_key_n != n || h->bsr_key_nnz != A->nnz) {
        h->bsr_key = A->row_ptr;
        h->bsr_key_n = n;
        h->bsr_key_nnz = A->nnz;
        h->bsr_ok = false;
        if (n % 3 == 0 && A->nnz % 9 == 0 && A->nnz > 0) {
            if (!h->bsr_flag) PODCG_CK(h, cudaMalloc((void**)&h->bsr_flag, sizeof(int)));
            PODCG_CK(h, cudaMemsetAsync(h->bsr_flag, 0, sizeof(int), s));
            PODCG_CK(h, launch_bsr_check(A->row_ptr, A->col, n, h->bsr_flag, h->sms, s));
            int bad = 1;
            PODCG_CK(h, cudaMemcpyAsync(&bad, h->bsr_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
            PODCG_CK(h, cudaStreamSynchronize(s));
            if (!bad) {
                const int64_t nnzb = A->nnz / 9;
                const int nb = n / 3;
                if (nnzb > h->bsr_cap) {
                    cudaFree(h->bcol);
                    cudaFree(h->bval);
                    cudaFree(h->bval32);
                    h->bcol = nullptr;
                    h->bval = nullptr;
                    h->bval32 = nullptr;
                    h->bsr_cap = 0;
                    PODCG_CK(h, cudaMalloc((void**)&h->bcol, sizeof(int32_t) * nnzb));
                    PODCG_CK(h, cudaMalloc((void**)&h->bval, sizeof(double) * 9 * nnzb));
                    if (h->mixed) PODCG_CK(h, cudaMalloc((void**)&h->bval32, sizeof(float) * 9 * nnzb));
                    h->bsr_cap = nnzb;
                }
                cudaFree(h->brp);
                h->brp = nullptr;
                PODCG_CK(h, cudaMalloc((void**)&h->brp, sizeof(int32_t) * (nb + 1)));
                PODCG_CK(h, launch_bsr_pattern(A->row_ptr, A->col, nb, h->brp, h->bcol, h->sms, s));
                h->bsr_L = bsr_lanes_for(double(nnzb) / std::max(nb, 1));
                h->bsr_timed = false;
                h->bsr_ok = true;
            }
        }
    }
    if (!h->bsr_ok) {
        if (h->cfg.bsr == 1) return fail(h, POD_CG_ERR_ARG, "bsr = 1 but the CSR pattern is not made of full 3x3 blocks");
        return POD_CG_OK;
    }
    const int64_t nnzb = A->nnz / 9;
    PODCG_CK(h, launch_bsr_values(A->row_ptr, A->val, n, (int)nnzb, h->bval, h->mixed ? h->bval32 : nullptr, h->sms, s));
    h->use_bsr = true;
    h->pd_host->brp = h->brp;
    h->pd_host->bcol = h->bcol;
    h->pd_host->bval = h->bval;
    h->pd_host->bval32 = h->bval32;
    h->pd_host->nb = n / 3;
    h->pd_host->nnzb = (int)nnzb;
    return POD_CG_OK;
}

// Lanes per block row of the block CG product, timed once per pattern on the actual
// matrix for systems of >= 65,536 rows (CUDA events, a scratch state, the handle's p and q
// as input and output); the heuristic width is kept unless another is >= 10% faster.
// Needs the problem descriptor with the block arrays on the device.
pod_cg_status choose_bsr_lanes(pod_cg_t* h)
{
    if (!h->use_bsr || h->bsr_timed) return POD_CG_OK;
    h->bsr_timed = true;
    if (h->n < 65536) return POD_CG_OK;
    cudaStream_t s = h->stream;
    const int cands[4] = {4, 8, 16, 32};
    const int heur = h->bsr_L;
    float t_heur = -1.0f, best = -1.0f;
    int best_L = heur;
    for (int L : cands) {
        void* f = kernel_bsr_spmv_cg(L, h->mixed);
        KSpec k;
        if (h->mixed)
            k.set(f, occ_grid(h, f, h->n / 3, kBlock / L), (const ProbDesc*)h->pd, (const float*)h->p32, h->q32,
                  h->partials, h->counters + 2 * kCounterStride, h->st_save);
        else
            k.set(f, occ_grid(h, f, h->n / 3, kBlock / L), (const ProbDesc*)h->pd, (const double*)h->p, h->q,
                  h->partials, h->counters + 2 * kCounterStride, h->st_save);
        PODCG_CK(h, cudaMemsetAsync(h->st_save, 0, sizeof(DevState), s));
        float tot = 0.0f;
        for (int rep = 0; rep < 4; ++rep) {
            PODCG_CK(h, cudaEventRecord(h->tev[0], s));
            PODCG_CK(h, launch_spec(k, s));
            PODCG_CK(h, cudaEventRecord(h->tev[1], s));
            PODCG_CK(h, cudaEventSynchronize(h->tev[1]));
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, h->tev[0], h->tev[1]);
            if (rep > 0) tot += ms;
        }
        tot /= 3.0f;
        if (L == heur) t_heur = tot;
        if (best < 0.0f || tot < best) {
            best = tot;
            best_L = L;
        }
    }
    if (t_heur < 0.0f || best < 0.9f * t_heur) h->bsr_L = best_L;
    return POD_CG_OK;
}

int s2_bucket(int y) { return y <= 8 ? 8 : y <= 16 ? 16 : y <= 32 ? 32 : y <= 48 ? 48 : 64; }

// Stage two (Section 4.2; kernels in k_stage2.cu): ||b||^2, the reduced residual and first
// direction, then lift / apply iterations while the reduced residual is above
// tol_stage2 * tol * ||b|| and fewer than min(y, wcap) - w1 iterations ran. FP64 products
// in both precisions: with FP32 products the reduced iteration's directions lose their
// mutual A-orthogonality at about eps_32 cond(Y^T A Y), which the block-diagonal stage-three
// factor cannot absorb (MIXED solves then stalled in stage three); MIXED converts the
// directions to FP32 afterwards.
void make_s2_plan(pod_cg_t* h, int L, bool cond, cudaGraphConditionalHandle hl, Stage2Plan& P, int inner = 0)
{
    void *f_bb, *f_init, *f_lift, *f_apply;
    stage2_kernels(h->pod_y, L, cond, &f_bb, &f_init, &f_lift, &f_apply);
    const int n = h->n, ld = h->ld;
    unsigned int* c = h->counters;
    const ProbDesc* pd = h->pd;
    P.bb.set(f_bb, occ_grid(h, f_bb, n, kBlock), pd, h->partials, c + 6 * kCounterStride, h->st);
    P.init.set(f_init, 1, (const double*)h->G, kWMax + 1, (const double*)h->Rinv, h->st, h->wcap,
               h->cfg.tol_stage2, hl);
    // inner solves of the whole-Y stage three lift into scratch vectors (v, then u)
    double* Bv = inner ? h->s2tmp : h->W;
    double* Bu = inner ? h->s2tmp + h->ld : h->AW;
    P.lift.set(f_lift, occ_grid(h, f_lift, n, kBlock), n, ld, (const double*)h->Y, Bv, (const DevState*)h->st, inner);
    P.apply.set(f_apply, occ_grid(h, f_apply, n, kBlock), pd, ld, (const double*)h->Y, (const double*)Bv, Bu,
                h->partials, c + 7 * kCounterStride, h->st, h->Rinv, (const double*)h->G, kWMax + 1, h->s2_hist, inner,
                hl);
}

pod_cg_status build_s2_graph(pod_cg_t* h, int L, GraphSlot& gs)
{
    cudaGraph_t P = nullptr, B = nullptr;
    PODCG_CK(h, cudaGraphCreate(&P, 0));
    cudaGraphConditionalHandle hl;
    PODCG_CK(h, cudaGraphConditionalHandleCreate(&hl, P, 0, 0));
    Stage2Plan pl;
    make_s2_plan(h, L, true, hl, pl);
    cudaGraphNode_t a, b, c, d, e;
    PODCG_CK(h, add_node(P, nullptr, 0, pl.bb, &a));
    PODCG_CK(h, add_node(P, &a, 1, pl.init, &b));
    PODCG_CK(h, add_while(P, &b, 1, hl, &c, &B));
    PODCG_CK(h, add_node(B, nullptr, 0, pl.lift, &d));
    PODCG_CK(h, add_node(B, &d, 1, pl.apply, &e));
    cudaGraphExec_t exec = nullptr;
    PODCG_CK(h, cudaGraphInstantiate(&exec, P, 0));
    gs.graph = P;
    gs.exec = exec;
    gs.L = L;
    gs.bsr = h->use_bsr;
    gs.yb = s2_bucket(h->pod_y);
    gs.valid = true;
    return POD_CG_OK;
}

pod_cg_status read_state(pod_cg_t* h);

pod_cg_status run_stage2(pod_cg_t* h, int L)
{
    cudaStream_t s = h->stream;
    if (h->cfg.loop_mode != 1) {
        GraphSlot& gs = h->s2graph;
        if (gs.valid && (gs.L != L || gs.yb != s2_bucket(h->pod_y))) destroy_graph(gs);
        if (!gs.valid) {
            pod_cg_status bs = build_s2_graph(h, L, gs);
            if (bs != POD_CG_OK) return bs;
        }
        PODCG_CK(h, cudaGraphLaunch(gs.exec, s));
        return read_state(h);
    }
    Stage2Plan pl;
    make_s2_plan(h, L, false, 0, pl);
    PODCG_CK(h, launch_spec(pl.bb, s));
    PODCG_CK(h, launch_spec(pl.init, s));
    pod_cg_status rs = read_state(h);
    for (int it = 0; rs == POD_CG_OK && !h->st_host->s2_done && it <= kWMax; ++it) {
        PODCG_CK(h, launch_spec(pl.lift, s));
        PODCG_CK(h, launch_spec(pl.apply, s));
        rs = read_state(h);
    }
    return rs;
}

pod_cg_status read_state(pod_cg_t* h)
{
    PODCG_CK(h, cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    PODCG_CK(h, cudaStreamSynchronize(h->stream));
    return POD_CG_OK;
}

// Stage three over the entire augmenting basis (three_stage = 2, Section 4.3.1; FP64):
// Algorithm 1 with the plain Jacobi-PCG product and update kernels, the augmentation step
// k_it_az, inner reduced iterations (k_s2_lift / k_s2_apply, inner = 1) and k_it_dir, driven
// from the host with one state read per iteration and one per inner reduced iteration (the
// inner iterations of a whole solve are at most y - w: the reduced directions accumulate).
// Passes of residual replacement as in the other loops.
pod_cg_status run_loop_it(pod_cg_t* h, int L, int* launches)
{
    cudaStream_t s = h->stream;
    const int n = h->n, ld = h->ld;
    Plan pl;
    make_plan(h, 0, L, false, 0, 0, 0, pl);   // no basis in the product / update kernels
    void *f_az, *f_dir0, *f_dir, *f_begin;
    it_kernels(h->pod_y, L, &f_az, &f_dir0, &f_dir, &f_begin);
    KSpec az, dir0, dir, begin;
    az.set(f_az, occ_grid(h, f_az, n, kBlock), (const ProbDesc*)h->pd, ld, (const double*)h->dinv, (const double*)h->r,
           (const double*)h->Y, h->partials, h->counters + 6 * kCounterStride, h->st, (const double*)h->Rinv,
           (const double*)h->G, kWMax + 1, (const double*)h->s2_hist, h->cfg.tol_inner);
    dir0.set(f_dir0, occ_grid(h, f_dir0, n, kBlock), n, ld, h->x, h->p, (const double*)h->r, (const double*)h->dinv,
             (const double*)h->Y, (const DevState*)h->st);
    dir.set(f_dir, occ_grid(h, f_dir, n, kBlock), n, ld, h->x, h->p, (const double*)h->r, (const double*)h->dinv,
            (const double*)h->Y, (const DevState*)h->st);
    begin.set(f_begin, 1, h->st);
    Stage2Plan s2;
    make_s2_plan(h, L, false, 0, s2, 1);
    PODCG_CK(h, launch_spec(begin, s));
    int nl = 1;
    auto inner_loop = [&]() -> pod_cg_status {
        for (int it = 0; !h->st_host->s2_done && it <= kWMax; ++it) {
            PODCG_CK(h, launch_spec(s2.lift, s));
            PODCG_CK(h, launch_spec(s2.apply, s));
            nl += 2;
            pod_cg_status rs = read_state(h);
            if (rs != POD_CG_OK) return rs;
        }
        return POD_CG_OK;
    };
    for (int pass = 0; pass <= h->cfg.max_refine + 1; ++pass) {
        PODCG_CK(h, launch_spec(pl.init, s));
        PODCG_CK(h, launch_spec(az, s));
        pod_cg_status rs = read_state(h);
        if (rs != POD_CG_OK) return rs;
        rs = inner_loop();
        if (rs != POD_CG_OK) return rs;
        PODCG_CK(h, launch_spec(dir0, s));
        nl += 3;
        for (long long it = 0; !h->st_host->done && it <= (long long)h->cfg.k_max + 1; ++it) {
            PODCG_CK(h, launch_spec(pl.spmv, s));
            PODCG_CK(h, launch_spec(pl.upd, s));
            PODCG_CK(h, launch_spec(az, s));
            rs = read_state(h);
            if (rs != POD_CG_OK) return rs;
            rs = inner_loop();
            if (rs != POD_CG_OK) return rs;
            PODCG_CK(h, launch_spec(dir, s));
            nl += 4;
        }
        PODCG_CK(h, launch_spec(pl.res, s));
        nl += 1;
        rs = read_state(h);
        if (rs != POD_CG_OK) return rs;
        if (h->st_host->outer_done) break;
    }
    *launches += nl;
    return POD_CG_OK;
}

// Stage three: run the loop in the configured form.
pod_cg_status run_loop(pod_cg_t* h, int wb, int L)
{
    const int bi = bucket_index(wb);
    cudaStream_t s = h->stream;
    if (h->cfg.loop_mode != 1) {
        GraphSlot& gs = h->graphs[bi];
        if (gs.valid && (gs.L != L || gs.bsr != h->use_bsr)) destroy_graph(gs);
        if (!gs.valid) {
            pod_cg_status bs = build_conditional(h, wb, L, gs);
            if (bs != POD_CG_OK) return bs;
        }
        PODCG_CK(h, cudaGraphLaunch(gs.exec, s));
        return POD_CG_OK;
    }
    GraphSlot& gs = h->chunks[bi];
    if (gs.valid && (gs.L != L || gs.bsr != h->use_bsr)) destroy_graph(gs);
    if (!gs.valid) {
        pod_cg_status bs = build_chunk(h, wb, L, gs);
        if (bs != POD_CG_OK) return bs;
    }
    Plan pl;
    make_plan(h, wb, L, h->mixed, 0, 0, 0, pl);
    const long long max_chunks = (long long)h->cfg.k_max / kChunk + 2;
    for (int pass = 0; pass <= h->cfg.max_refine + 1; ++pass) {
        if (h->mixed) {
            PODCG_CK(h, launch_spec(pl.res, s));
            PODCG_CK(h, launch_spec(pl.mxproj, s));
            PODCG_CK(h, launch_spec(pl.mxstart, s));
        }
        PODCG_CK(h, launch_spec(pl.init, s));
        PODCG_CK(h, launch_spec(pl.dir0, s));
        pod_cg_status rs = read_state(h);
        if (rs != POD_CG_OK) return rs;
        for (long long c = 0; !h->st_host->done && c < max_chunks; ++c) {
            PODCG_CK(h, cudaGraphLaunch(gs.exec, s));
            rs = read_state(h);
            if (rs != POD_CG_OK) return rs;
        }
        if (h->mixed) {
            PODCG_CK(h, launch_spec(pl.mxaccum, s));
        } else {
            PODCG_CK(h, launch_spec(pl.res, s));
        }
        rs = read_state(h);
        if (rs != POD_CG_OK) return rs;
        if (h->st_host->outer_done) break;
    }
    return POD_CG_OK;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

void reset_state(pod_cg_t* h, const pod_cg_csr* A, const double* b, double tol)
{
    // the block form's fields are filled by setup_bsr when the pattern has one
    *h->pd_host = ProbDesc{A->row_ptr, A->col, A->val, h->val32, b, nullptr, h->n, h->ld,
                           nullptr, nullptr, nullptr, nullptr, 0, 0};
    DevState& sh = *h->st_host;
    std::memset(&sh, 0, sizeof(DevState));
    sh.k_max = h->cfg.k_max;
    sh.max_refine = h->cfg.max_refine;
    sh.pod_w = h->pod_w;
    sh.w = h->pod_w;
    sh.mixed = h->mixed ? 1 : 0;
    sh.rr_stage1 = -1.0;
    sh.pod_y = h->pod_y;
    sh.w1 = h->pod_w;
    sh.s2_done = 1;
    sh.tol_rel = tol;
}

pod_cg_status finish_solve(pod_cg_t* h, double* out, int w_pod, int launches, pod_cg_stats* stats, int sysid)
{
    cudaStream_t s = h->stream;
    PODCG_CK(h, cudaEventRecord(h->ev[4], s));
    PODCG_CK(h, cudaMemcpyAsync(out, h->x, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, s));
    pod_cg_status rs = read_state(h);
    if (rs != POD_CG_OK) return rs;
    const DevState& d = *h->st_host;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->status = d.status;
        stats->iters = d.iters;
        stats->refinements = d.restarts;
        stats->w = d.w;
        stats->s = h->s_count;
        stats->chol_failed = d.chol_failed;
        stats->system_id = sysid;
        stats->spmv_count = d.iters + w_pod + d.restarts + 1 + h->k2;
        const int per_pass = h->mixed ? 6 : 3;
        stats->launches = launches + per_pass * (d.restarts + 1) + 3 * d.iters;
        stats->y = h->pod_y_used;
        stats->stage2_iters = h->k2;
        if (h->it_mode) {
            stats->w = h->pod_y_used;   // stage three augments with all of Y
            stats->inner_iters = d.inner_total;
            stats->spmv_count += d.inner_total + d.iters + d.restarts + 1;   // A z per iteration and pass
        }
        stats->stage1_relres = d.bb > 0.0 ? std::sqrt(std::max(d.rr_stage1, 0.0) / d.bb) : 0.0;
        stats->final_relres = d.bb > 0.0 ? std::sqrt(d.rr_true / d.bb) : 0.0;
        stats->cond_gram = d.cond;
        stats->gram_tc = h->last_gram_tc;
        stats->ms_loop = float(double(d.loop_ns) * 1e-6);
        cudaEventElapsedTime(&stats->ms_pod, h->ev[0], h->ev[1]);
        cudaEventElapsedTime(&stats->ms_stage1, h->ev[1], h->ev[2]);
        cudaEventElapsedTime(&stats->ms_stage2, h->ev[2], h->ev[3]);
        cudaEventElapsedTime(&stats->ms_stage3, h->ev[3], h->ev[4]);
    }
    if (d.status != 0) {
        static const char* names[] = {"ok", "arg", "not SPD (non-positive diagonal)", "breakdown: (Ap, p) <= 0",
                                      "iteration/refinement cap reached", "non-finite scalar"};
        const char* nm = (d.status >= 0 && d.status <= 5) ? names[d.status] : "error";
        return fail(h, (pod_cg_status)d.status, std::string("solve: ") + nm);
    }
    return POD_CG_OK;
}

// Krylov-vector mode (Section 3.1, Algorithm 3). The augmenting basis of the next solve:
// Y = Z with the stage-one columns first (w of them), so that W is Y's first w columns as
// the three-stage solve expects.
pod_cg_status krylov_gather(pod_cg_t* h)
{
    const size_t ld = (size_t)h->ld;
    std::vector<char> in_w(h->z, 0);
    std::vector<int> order(h->w_idx);
    for (int c : h->w_idx) in_w[c] = 1;
    for (int c = 0; c < h->z; ++c)
        if (!in_w[c]) order.push_back(c);
    for (size_t i = 0; i < order.size(); ++i)
        PODCG_CK(h, cudaMemcpyAsync(h->Y + i * ld, h->Z + (size_t)order[i] * ld, sizeof(double) * h->n,
                                    cudaMemcpyDeviceToDevice, h->stream));
    h->pod_w = (int)h->w_idx.size();
    h->pod_y = h->z;
    h->w_clobbered = h->pod_w > 0;
    h->pod_dirty = false;
    return POD_CG_OK;
}

// Compression (Algorithm 3's truncation): Z <- the first y_keep modes of the POD of
// Z diag(eta) with the metric A (Algorithm 4, Theta = A: Gram (Z diag(eta))^T A (Z diag(eta)),
// symmetrised, eigen-decomposed, lifted; the modes are A-orthonormal); W <- the first w_keep.
pod_cg_status krylov_compress_now(pod_cg_t* h, const pod_cg_csr* A, const double* eta, int y_keep, int w_keep)
{
    cudaStream_t s = h->stream;
    const int n = h->n, z = h->z;
    if (z == 0) return POD_CG_OK;
    PODCG_CK(h, launch_scale_cols(h->Z, h->Zalt, h->ld, n, z, eta, 0, h->sms, s));
    PODCG_CK(h, launch_spmm(A->row_ptr, A->col, A->val, h->Zalt, h->ld, h->AZ, h->ld, n, z, h->sms, s));
    PODCG_CK(h, launch_gram(n, h->Zalt, h->ld, z, h->AZ, h->ld, z, nullptr, h->zG2, kSMax, 0, h->gram_work,
                            h->gram_work_bytes, h->sms, s));
    PODCG_CK(h, launch_symmetrize(h->zG2, kSMax, z, s));
    PODCG_CK(h, launch_pod_eig(h->zG2, kSMax, z, 2.0, h->cfg.rank_tol, y_keep, h->C, h->sigma2, h->st, nullptr, 0, s,
                               0.0, 0));
    PODCG_CK(h, launch_lift(n, h->Zalt, h->ld, z, h->C, h->st, h->Z, h->ld, h->sms, s, 0));
    pod_cg_status rs = read_state(h);
    if (rs != POD_CG_OK) return rs;
    const int yk = h->st_host->pod_w;
    h->z = yk;
    h->w_idx.clear();
    for (int c = 0; c < std::min(w_keep, yk); ++c) h->w_idx.push_back(c);
    PODCG_CK(h, cudaMemsetAsync(h->zeta, 0, sizeof(double) * kSMax, s));
    ++h->compressions;
    return POD_CG_OK;
}

// Coordinates (Z^T A Z)^+ Z^T b (Eq. (weightsPrevious), x_bar = 0) into zcoord; with
// accumulate, the weights zeta are updated from them (RBF or previous weights).
pod_cg_status krylov_coords_now(pod_cg_t* h, const pod_cg_csr* A, const double* b, bool accumulate)
{
    cudaStream_t s = h->stream;
    const int n = h->n, z = h->z;
    if (z == 0) return POD_CG_OK;
    PODCG_CK(h, launch_spmm(A->row_ptr, A->col, A->val, h->Z, h->ld, h->AZ, h->ld, n, z, h->sms, s));
    PODCG_CK(h, launch_gram(n, h->Z, h->ld, z, h->AZ, h->ld, z, b, h->zG, kSMax + 1, 0, h->gram_work,
                            h->gram_work_bytes, h->sms, s));
    double* eta = accumulate ? h->zeta : h->zG2;   // zG2 is scratch outside compressions
    PODCG_CK(h, launch_krylov_coords(h->zG, kSMax + 1, z, 1e-13, h->zcoord, eta, h->kc.weights == 0 ? 1 : 0, s));
    return POD_CG_OK;
}

// After a solve: append its recorded directions, A-normalised (P T^{-1/2}), choose the new
// stage-one columns by nu, form the solution's previous weights and compress when Z has
// passed the storage threshold (Algorithm 3).
pod_cg_status krylov_update(pod_cg_t* h, const pod_cg_csr* A, const double* b)
{
    cudaStream_t s = h->stream;
    const int k = std::min(h->st_host->iters, h->kry_cap);
    if (k > 0) {
        std::vector<double> g(k);
        PODCG_CK(h, cudaMemcpyAsync(g.data(), h->kgam, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
        double* cols = h->Z + (size_t)h->z * h->ld;
        PODCG_CK(h, launch_scale_cols(cols, cols, h->ld, h->n, k, h->kgam, 1, h->sms, s));
        PODCG_CK(h, cudaStreamSynchronize(s));
        double sum = 0.0;
        for (double v : g) sum += v;
        for (int i = 0; i < k; ++i) {
            const bool take = h->kc.nu >= 1.0 ? true : h->kc.nu <= 0.0 ? false : g[i] / sum > h->kc.nu;
            if (take) h->w_idx.push_back(h->z + i);
        }
        h->z += k;
    }
    pod_cg_status cs = krylov_coords_now(h, A, b, true);
    if (cs != POD_CG_OK) return cs;
    if (h->kc.y_threshold > 0 && h->z > h->kc.y_threshold)
        return krylov_compress_now(h, A, h->zeta, h->kc.y_keep, h->kc.w_keep);
    return POD_CG_OK;
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
    c->use_tc_gram = -1;
    c->cond_diag = 0;
    c->keep_factors = 0;
    c->loop_mode = 0;
    c->proj_form = -1;
    c->spmv_lanes = 0;
    c->three_stage = 0;
    c->y_max = 40;
    c->energy_y = 0.99999999;
    c->tol_stage2 = 1e-4;
    c->tol_inner = 1e-12;
    c->bsr = -1;
    c->pod_metric = 0;
    c->w_select = 0;
    return POD_CG_OK;
}

const char* pod_cg_last_error(const pod_cg_t* h)
{
    return h ? h->err.c_str() : g_last_error.c_str();
}

pod_cg_status pod_cg_destroy(pod_cg_t* h)
{
    if (!h) return POD_CG_OK;
    for (auto& g : h->graphs) destroy_graph(g);
    for (auto& g : h->chunks) destroy_graph(g);
    destroy_graph(h->s2graph);
    void* bufs[] = {h->S, h->S32, h->GS, h->grow, h->C, h->sigma2, h->Vprev, h->W, h->AW, h->W32, h->AW32, h->W16, h->wscale, h->wmax, h->Y, h->Y32,
                    h->s2_hist, h->s2tmp, h->brp, h->bcol, h->bval, h->bval32, h->bsr_flag, h->Cout, h->CSv,
                    h->GSC, h->out_work, h->AS, h->GA,
                    h->G, h->Rinv, h->Mmu,
                    h->x, h->r, h->p, h->q, h->dinv, h->dinv32, h->r32, h->p32, h->q32, h->d32, h->val32,
                    h->partials, h->counters, h->gram_work, h->st, h->st_save, h->pd, h->kW, h->kAW, h->kG,
                    h->Z, h->Zalt, h->AZ, h->kgam, h->zG, h->zG2, h->zcoord, h->zeta, h->gbar};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (h->tm_dev) cudaFree(h->tm_dev);
    if (h->tm_host) cudaFreeHost(h->tm_host);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->pd_host) cudaFreeHost(h->pd_host);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : h->tev)
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
        c.keep_factors < 0 || c.keep_factors > 4096 || (c.loop_mode < 0 || c.loop_mode > 2) ||
        c.proj_form < -1 || c.proj_form > 1 ||
        (c.spmv_lanes != 0 && (c.spmv_lanes < 1 || c.spmv_lanes > 32 || (c.spmv_lanes & (c.spmv_lanes - 1)))) ||
        !(c.inner_tol > 0.0 && c.inner_tol < 1.0))
        return fail(nullptr, POD_CG_ERR_ARG, "invalid configuration");
    if (c.three_stage != 0 && (c.three_stage < 0 || c.three_stage > 2 || c.y_max < 1 || c.y_max > c.s_max ||
                               !(c.energy_y >= 0.0 && c.energy_y <= 1.0) ||
                               !(c.tol_stage2 >= 0.0 && std::isfinite(c.tol_stage2)) ||
                               !(c.tol_inner >= 0.0 && c.tol_inner < 1.0)))
        return fail(nullptr, POD_CG_ERR_ARG,
                    "invalid three-stage configuration (three_stage 0/1/2, 1 <= y_max <= s_max, energy_y in [0, 1], "
                    "tol_stage2 >= 0, 0 <= tol_inner < 1)");
    if (c.bsr < -1 || c.bsr > 1) return fail(nullptr, POD_CG_ERR_ARG, "bsr must be -1 (auto), 0 or 1");
    if (c.pod_metric < 0 || c.pod_metric > 1) return fail(nullptr, POD_CG_ERR_ARG, "pod_metric must be 0 or 1");
    if (c.w_select < 0 || c.w_select > 1) return fail(nullptr, POD_CG_ERR_ARG, "w_select must be 0 or 1");
    if (c.three_stage == 2 && c.precision != POD_CG_FP64)
        return fail(nullptr, POD_CG_ERR_ARG, "three_stage = 2 (stage three over the whole Y) runs in FP64 only");
    if (c.use_tc_gram < -1 || c.use_tc_gram > 1 || (c.use_tc_gram == 1 && c.precision != POD_CG_MIXED))
        return fail(nullptr, POD_CG_ERR_ARG,
                    "use_tc_gram is -1, 0 or 1, and 1 needs precision MIXED: the tensor-core Gram rounds W and AW "
                    "to FP32");
    pod_cg_t* h = new (std::nothrow) pod_cg_t();
    if (!h) return fail(nullptr, POD_CG_ERR_OOM, "host allocation failed");
    h->n = n;
    h->ld = ((n + 31) / 32) * 32;
    h->cfg = c;
    h->mixed = c.precision == POD_CG_MIXED;
    // three-stage mode appends up to y - w stage-two directions after W: room for kWMax
    h->wcap = c.three_stage ? kWMax : c.w_max;
    for (auto& g : h->gram_choice) g = -1;
    if (c.w_select) {   // caps 2, 4, 8, ... below w_max, then w_max; visited c1 .. ck ck .. c1
        for (int cp = 2; cp < c.w_max && h->wsel_caps.size() < 7; cp *= 2) h->wsel_caps.push_back(cp);
        h->wsel_caps.push_back(c.w_max);
        const int k = (int)h->wsel_caps.size();
        for (int i = 0; i < k; ++i) h->wsel_order.push_back(i);
        for (int i = k - 1; i >= 0; --i) h->wsel_order.push_back(i);
        h->wsel_ms.assign(k, 0.0);
        h->wsel_n.assign(k, 0);
    }
    if (c.proj_form >= 0)
        for (int& f : h->proj_form) f = c.proj_form == 1 ? 3 : 0;   // both passes in the forced form
    h->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&h->device);
    h->sms = device_sms();
    const size_t ld = (size_t)h->ld;
    cudaError_t e = cudaSuccess;
#define PODCG_ALLOC(ptr, cnt) \
    if (e == cudaSuccess) e = dalloc(&(ptr), (cnt));
    PODCG_ALLOC(h->S, ld * c.s_max)
    PODCG_ALLOC(h->GS, (size_t)kSMax * kSMax)
    PODCG_ALLOC(h->grow, (size_t)kSMax)
    PODCG_ALLOC(h->C, (size_t)kSMax * kWMax)
    PODCG_ALLOC(h->sigma2, (size_t)kSMax)
    PODCG_ALLOC(h->Vprev, (size_t)kSMax * kSMax)
    // stage two runs in FP64 in both precisions: its directions go to the FP64 W/AW buffers
    PODCG_ALLOC(h->W, ld * h->wcap)
    PODCG_ALLOC(h->AW, ld * h->wcap)
    // Y holds y <= max(y_max, w_max) columns (y is raised to w when the energy rule gives less)
    const size_t ycols = (size_t)std::max(c.y_max, c.w_max);
    if (c.three_stage) PODCG_ALLOC(h->Y, ld * ycols)
    if (c.three_stage) PODCG_ALLOC(h->s2_hist, (size_t)2 * kWMax * kSMax + kWMax)
    if (c.three_stage == 2) PODCG_ALLOC(h->s2tmp, ld * 2)
    if (c.pod_metric == 1) {
        PODCG_ALLOC(h->AS, ld * c.s_max)
        PODCG_ALLOC(h->GA, (size_t)kSMax * kSMax)
    }
    PODCG_ALLOC(h->G, (size_t)kWMax * (kWMax + 1))
    PODCG_ALLOC(h->Rinv, (size_t)kWMax * kWMax)
    PODCG_ALLOC(h->Mmu, (size_t)kWMax * kWMax)
    PODCG_ALLOC(h->x, ld)
    PODCG_ALLOC(h->r, ld)
    PODCG_ALLOC(h->p, ld)
    PODCG_ALLOC(h->q, ld)
    PODCG_ALLOC(h->dinv, ld)
    PODCG_ALLOC(h->dinv32, ld)
    PODCG_ALLOC(h->partials, (size_t)kPartialRows * kPartialStride)
    PODCG_ALLOC(h->counters, (size_t)8 * kCounterStride)
    PODCG_ALLOC(h->gbar, (size_t)32)
    PODCG_ALLOC(h->st, 1)
    PODCG_ALLOC(h->st_save, 1)
    PODCG_ALLOC(h->pd, 1)
    if (h->mixed) {
        PODCG_ALLOC(h->S32, ld * c.s_max)
        PODCG_ALLOC(h->W32, ld * h->wcap)
        PODCG_ALLOC(h->AW32, ld * h->wcap)
        PODCG_ALLOC(h->W16, ld * h->wcap)
        PODCG_ALLOC(h->wscale, (size_t)kWMax)
        PODCG_ALLOC(h->wmax, (size_t)kWMax)
        if (c.three_stage) PODCG_ALLOC(h->Y32, ld * ycols)
        PODCG_ALLOC(h->r32, ld)
        PODCG_ALLOC(h->p32, ld)
        PODCG_ALLOC(h->q32, ld)
        PODCG_ALLOC(h->d32, ld)
    }
    if (c.keep_factors > 0) {
        PODCG_ALLOC(h->kW, ld * c.w_max * c.keep_factors)
        PODCG_ALLOC(h->kAW, ld * c.w_max * c.keep_factors)
        PODCG_ALLOC(h->kG, (size_t)kWMax * (kWMax + 1) * c.keep_factors)
        h->k_id.assign(c.keep_factors, -1);
        h->k_w.assign(c.keep_factors, 0);
    }
#undef PODCG_ALLOC
    if (e == cudaSuccess) {
        // the split count of a Gram depends on its shape, and smaller shapes can need more
        // workspace: take the maximum over the shapes each use can take
        for (int k = 1; k <= c.s_max; ++k) {
            h->gram_work_bytes = std::max(h->gram_work_bytes, gram_workspace_bytes(n, 1, k, h->sms));
            if (c.pod_metric == 1)
                h->gram_work_bytes = std::max(h->gram_work_bytes, gram_workspace_bytes(n, k, k, h->sms));
        }
        for (int k = 1; k <= std::max(c.w_max, c.three_stage ? c.y_max : 0); ++k)
            for (int j = 1; j <= c.w_max + 1; ++j)
                h->gram_work_bytes = std::max(h->gram_work_bytes, gram_workspace_bytes(n, k, j, h->sms));
        const int gp = c.three_stage ? std::max(c.w_max, c.y_max) : c.w_max;
        if (c.three_stage && h->mixed)   // the re-formed stage-three Gram, up to kWMax columns
            for (int k = 1; k <= kWMax; ++k)
                h->gram_work_bytes = std::max(h->gram_work_bytes, gram_workspace_bytes(n, k, k + 1, h->sms));
        if (c.use_tc_gram != 0 && h->mixed)
            h->gram_work_bytes = std::max(h->gram_work_bytes, gram_tc_workspace_bytes(n, gp, c.w_max + 1, h->sms));
        e = cudaMalloc((void**)&h->gram_work, h->gram_work_bytes);
    }
    if (e == cudaSuccess && h->mixed) {
        e = cudaMalloc((void**)&h->tm_dev, 3 * sizeof(CUtensorMap));
        if (e == cudaSuccess) e = cudaMallocHost((void**)&h->tm_host, 3 * sizeof(CUtensorMap));
        if (e == cudaSuccess) {
            h->tm_ok = encode_panel_map(&h->tm_host[0], h->AW32, 4, h->ld, h->wcap, 8) &&
                       encode_panel_map(&h->tm_host[1], h->W32, 4, h->ld, h->wcap, 8) &&
                       encode_panel_map(&h->tm_host[2], h->W16, 2, h->ld, h->wcap, 16);
            h->w16 = h->tm_ok && !c.three_stage;   // three-stage W32 also holds stage two's directions
        }
    }
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->st_host, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->pd_host, sizeof(ProbDesc));
    for (auto& ev : h->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    for (auto& ev : h->tev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->counters, 0, (size_t)8 * kCounterStride * sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->S, 0, sizeof(double) * ld * c.s_max, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->GS, 0, sizeof(double) * kSMax * kSMax, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->p, 0, sizeof(double) * ld, h->stream);
    if (e == cudaSuccess && h->mixed) e = cudaMemsetAsync(h->p32, 0, sizeof(float) * ld, h->stream);
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
    h->vprev_s = 0;
    if (h->kry_on) {
        h->z = 0;
        h->w_idx.clear();
        PODCG_CK(h, cudaMemsetAsync(h->zeta, 0, sizeof(double) * kSMax, h->stream));
    }
    return POD_CG_OK;
}

pod_cg_status pod_cg_add_snapshots(pod_cg_t* h, const double* X, int m)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    if (m < 0 || (m > 0 && !X)) return fail(h, POD_CG_ERR_ARG, "bad snapshot block");
    if (h->kry_on && m > 0)
        return fail(h, POD_CG_ERR_STATE, "the handle's snapshots are its Krylov vectors (pod_cg_set_krylov)");
    const int n = h->n;
    for (int c = 0; c < m; ++c) {
        const int slot = h->s_next;
        double* col = h->S + (size_t)slot * h->ld;
        PODCG_CK(h, cudaMemcpyAsync(col, X + (size_t)c * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
        if (h->mixed) PODCG_CK(h, launch_to_f32(col, h->S32 + (size_t)slot * h->ld, n, h->sms, h->stream));
        h->s_next = (h->s_next + 1) % h->cfg.s_max;
        h->s_count = std::min(h->s_count + 1, h->cfg.s_max);
        // new row of S^T S: s_new^T S (Algorithm 4 step 1, one row at a time)
        PODCG_CK(h, launch_gram(n, col, h->ld, 1, h->S, h->ld, h->s_count, nullptr, h->grow, kSMax, 0, h->gram_work,
                                h->gram_work_bytes, h->sms, h->stream));
        PODCG_CK(h, launch_gram_scatter(h->grow, h->s_count, slot, h->GS, kSMax, h->stream));
        if (h->out_q > 0)   // C s_new for the output-oriented metric
            PODCG_CK(h, launch_gram(n, col, h->ld, 1, h->Cout, n, h->out_q, nullptr, h->CSv + (size_t)slot * kQMax,
                                    kQMax, 0, h->out_work, h->out_work_bytes, h->sms, h->stream));
    }
    if (m > 0) h->pod_dirty = true;
    return POD_CG_OK;
}

pod_cg_status pod_cg_set_output_functionals(pod_cg_t* h, const double* C, int q)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    if (q < 0 || q > kQMax || (q > 0 && !C)) return fail(h, POD_CG_ERR_ARG, "q must be 0..128 and C non-NULL");
    if (q > 0 && h->cfg.pod_metric == 1)
        return fail(h, POD_CG_ERR_STATE, "the handle's POD uses the metric A (pod_metric = 1)");
    cudaStream_t s = h->stream;
    const int n = h->n;
    if (q > 0) {
        if (!h->Cout) {
            PODCG_CK(h, cudaMalloc((void**)&h->Cout, sizeof(double) * (size_t)kQMax * n));
            PODCG_CK(h, cudaMalloc((void**)&h->CSv, sizeof(double) * (size_t)kQMax * kSMax));
            PODCG_CK(h, cudaMalloc((void**)&h->GSC, sizeof(double) * (size_t)kSMax * kSMax));
        }
        // the product's split count depends on q: size the workspace for this q
        const size_t wb = gram_workspace_bytes(n, 1, q, h->sms);
        if (wb > h->out_work_bytes) {
            cudaFree(h->out_work);
            h->out_work = nullptr;
            h->out_work_bytes = 0;
            PODCG_CK(h, cudaMalloc((void**)&h->out_work, wb));
            h->out_work_bytes = wb;
        }
        PODCG_CK(h, cudaMemcpyAsync(h->Cout, C, sizeof(double) * (size_t)q * n, cudaMemcpyDeviceToDevice, s));
        // images of the snapshots already held
        for (int k = 0; k < h->s_count; ++k)
            PODCG_CK(h, launch_gram(n, h->S + (size_t)k * h->ld, h->ld, 1, h->Cout, n, q, nullptr,
                                    h->CSv + (size_t)k * kQMax, kQMax, 0, h->out_work, h->out_work_bytes, h->sms, s));
    }
    h->out_q = q;
    h->pod_dirty = h->s_count > 0;
    h->vprev_s = 0;   // the previous eigenvectors belong to the other metric
    PODCG_CK(h, cudaStreamSynchronize(s));
    return POD_CG_OK;
}

pod_cg_status pod_cg_get_basis(pod_cg_t* h, double* W_out, int* w_out)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    if (w_out) *w_out = h->pod_w;
    if (W_out && h->pod_w > 0) {
        if (h->mixed) return fail(h, POD_CG_ERR_STATE, "the FP64 basis is not formed in mixed precision");
        PODCG_CK(h, cudaMemcpy2DAsync(W_out, sizeof(double) * h->n, h->W, sizeof(double) * h->ld,
                                      sizeof(double) * h->n, h->pod_w, cudaMemcpyDeviceToDevice, h->stream));
    }
    PODCG_CK(h, cudaStreamSynchronize(h->stream));
    return POD_CG_OK;
}

pod_cg_status pod_cg_get_stage3_basis(pod_cg_t* h, double* B_out, double* AB_out, int* w3_out)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    const int w3 = h->st_host ? h->st_host->w : 0;
    if (w3_out) *w3_out = w3;
    if ((B_out || AB_out) && w3 > 0) {
        if (h->mixed) return fail(h, POD_CG_ERR_STATE, "the FP64 basis is not formed in mixed precision");
        if (B_out)
            PODCG_CK(h, cudaMemcpy2DAsync(B_out, sizeof(double) * h->n, h->W, sizeof(double) * h->ld,
                                          sizeof(double) * h->n, w3, cudaMemcpyDeviceToDevice, h->stream));
        if (AB_out)
            PODCG_CK(h, cudaMemcpy2DAsync(AB_out, sizeof(double) * h->n, h->AW, sizeof(double) * h->ld,
                                          sizeof(double) * h->n, w3, cudaMemcpyDeviceToDevice, h->stream));
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
    const int n = h->n;
    cudaStream_t s = h->stream;
    if (h->mixed && A->nnz > h->val32_cap) {
        if (h->val32) cudaFree(h->val32);
        h->val32 = nullptr;
        h->val32_cap = 0;
        PODCG_CK(h, cudaMalloc((void**)&h->val32, sizeof(float) * (size_t)std::max<int64_t>(A->nnz, 1)));
        h->val32_cap = A->nnz;
    }

    if (h->kry_on) {   // the basis sizes of this solve are known on the host (the state starts from them)
        h->pod_w = (int)h->w_idx.size();
        h->pod_y = h->z;
    }
    reset_state(h, A, b, tol);
    pod_cg_status bst = setup_bsr(h, A);
    if (bst != POD_CG_OK) return bst;
    h->kry_cap = 0;
    if (h->kry_on && !h->kc.frozen) {   // stage three records its first directions into Z
        h->kry_cap = std::min(h->kc.p_cap, kSMax - h->z);
        h->pd_host->krec = h->Z + (size_t)h->z * h->ld;
        h->pd_host->krec_gamma = h->kgam;
        h->pd_host->krec_cap = h->kry_cap;
    }
    PODCG_CK(h, cudaMemcpyAsync(h->pd, h->pd_host, sizeof(ProbDesc), cudaMemcpyHostToDevice, s));
    PODCG_CK(h, cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, s));
    PODCG_CK(h, cudaMemsetAsync(h->gbar, 0, 2 * sizeof(unsigned int), s));   // the persistent loop's barrier
    PODCG_CK(h, cudaEventRecord(h->ev[0], s));
    PODCG_CK(h, launch_dinv(h->pd, n, h->dinv, h->dinv32, h->st, h->sms, s));
    int launches = 2;   // dinv, stage-one lift
    if (h->mixed) {
        PODCG_CK(h, launch_desc_val_to_f32(h->pd, h->val32, A->nnz, h->sms, s));
        launches += 1;
    }

    // SpMV lanes for this pattern (timed once per pattern, with the autotuner's own events)
    int L = 1;
    pod_cg_status lst = choose_lanes(h, A, &L);
    if (lst != POD_CG_OK) return lst;
    h->last_L = L;
    pod_cg_status blst = choose_bsr_lanes(h);
    if (blst != POD_CG_OK) return blst;

    // POD of the current snapshots (Algorithm 4); in three-stage mode also the augmenting
    // basis Y, whose first w columns are W (nested POD bases)
    const bool three = h->cfg.three_stage != 0;
    // cap on w for this solve (w_select = 1): a candidate while they are timed, then the choice
    int cap = h->cfg.w_max;
    h->wsel_slot = -1;
    if (h->cfg.w_select && !h->kry_on) {
        if (h->wsel_done) cap = h->w_cap;
        else if (h->s_count >= std::min(8, h->cfg.s_max)) {
            h->wsel_slot = h->wsel_order[h->wsel_pos];
            cap = h->wsel_caps[h->wsel_slot];
        }
    }
    if (cap != h->cap_now) h->pod_dirty = h->s_count > 0;
    h->cap_now = cap;
    if (h->cfg.pod_metric == 1 && h->s_count > 0) h->pod_dirty = true;   // the metric is this system's A
    if (h->kry_on) {
        pod_cg_status ks = krylov_gather(h);
        if (ks != POD_CG_OK) return ks;
    } else if (h->s_count > 0 && h->pod_dirty) {
        const double* Gpod = h->GS;
        if (h->out_q > 0) {   // metric C^T C: the Gram of the snapshots' output images
            PODCG_CK(h, launch_cs_gram(h->CSv, kQMax, h->s_count, h->out_q, h->GSC, kSMax, s));
            Gpod = h->GSC;
            launches += 1;
        } else if (h->cfg.pod_metric == 1) {   // metric A: S^T (A S), symmetrised
            PODCG_CK(h, launch_spmm(A->row_ptr, A->col, A->val, h->S, h->ld, h->AS, h->ld, n, h->s_count, h->sms, s));
            PODCG_CK(h, launch_gram(n, h->S, h->ld, h->s_count, h->AS, h->ld, h->s_count, nullptr, h->GA, kSMax, 0,
                                    h->gram_work, h->gram_work_bytes, h->sms, s));
            PODCG_CK(h, launch_symmetrize(h->GA, kSMax, h->s_count, s));
            Gpod = h->GA;
            launches += 4;
        }
        PODCG_CK(h, launch_pod_eig(Gpod, kSMax, h->s_count, h->cfg.energy, h->cfg.rank_tol, cap, h->C,
                                   h->sigma2, h->st, h->Vprev, h->vprev_s, s, h->cfg.energy_y,
                                   three ? h->cfg.y_max : 0));
        h->vprev_s = h->s_count;
        if (three) {
            PODCG_CK(h, launch_lift(n, h->S, h->ld, h->s_count, h->C, h->st, h->Y, h->ld, h->sms, s, 1));
        } else {
            if (h->mixed) {
                PODCG_CK(h, launch_lift32(n, h->S32, h->ld, h->s_count, h->C, h->st, h->W32, h->ld, h->sms, s));
                if (h->w16) {
                    PODCG_CK(h, launch_quant16(n, h->ld, h->W32, h->W16, h->wmax, h->wscale, h->st, h->sms, s));
                    launches += 2;
                }
            }
            else PODCG_CK(h, launch_lift(n, h->S, h->ld, h->s_count, h->C, h->st, h->W, h->ld, h->sms, s));
        }
        launches += 2;
        pod_cg_status rs = read_state(h);
        if (rs != POD_CG_OK) return rs;
        h->pod_w = h->st_host->pod_w;
        h->pod_y = three ? h->st_host->pod_y : 0;
        h->pod_dirty = false;
        h->w_clobbered = three;   // W is copied out of Y below
        if (three && h->mixed && h->pod_y > 0) {
            PODCG_CK(h, launch_to_f32(h->Y, h->Y32, (size_t)h->ld * h->pod_y, h->sms, s));
            launches += 1;
        }
    } else if (h->s_count == 0) {
        h->pod_w = 0;
        h->pod_y = 0;
    }
    const int w = h->pod_w;
    if (three && w > 0 && h->w_clobbered) {
        PODCG_CK(h, cudaMemcpy2DAsync(h->W, sizeof(double) * h->ld, h->Y, sizeof(double) * h->ld,
                                      sizeof(double) * n, w, cudaMemcpyDeviceToDevice, s));
        if (h->mixed)
            PODCG_CK(h, cudaMemcpy2DAsync(h->W32, sizeof(float) * h->ld, h->Y32, sizeof(float) * h->ld,
                                          sizeof(float) * n, w, cudaMemcpyDeviceToDevice, s));
        h->w_clobbered = false;
    }
    const int y = three ? h->pod_y : 0;
    PODCG_CK(h, cudaEventRecord(h->ev[1], s));

    // stage one (Algorithm 2)
    if (w > 0) {
        // Ahat = W^T [AW, b]: FP64 (or FP32-product) CUDA-core Gram, or in mixed precision
        // the tensor-core split-bf16 Gram when use_tc_gram is set (its TMA loads need a
        // 16-byte aligned b; r is free until stage one writes it). In three-stage mode the
        // Gram is Y^T [AW, b]: its first w rows are W^T [AW, b], the rest feed stage two,
        // and it stays on the CUDA cores: stage two's reduced residual Y^T b - Y^T A W what
        // cancels, and the split-bf16 products' error (2^-16 of sum |y| |A w| per entry)
        // left its deflation terms too loose for the block-diagonal stage-three factor.
        const double* bt = b;
        h->last_gram_tc = 0;
        if (h->mixed && h->cfg.use_tc_gram != 0 && !gram_tc_aligned(b, 16)) {
            PODCG_CK(h, cudaMemcpyAsync(h->r, b, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
            bt = h->r;
        }
        int* tc_err = &h->st->status;
        const int p = y > w ? y : w;
        const int upper = y > w ? 0 : 1;
        if (h->mixed && y > 0) {
            // three-stage in mixed precision: stage two runs on FP64 products, so its
            // deflation terms Y^T A W and the stage-one factor come from FP64 data too (an
            // FP32-data Gram left stage two's residual at an inconsistency floor, and its
            // later directions useless); stage three re-forms its FP32 factor below. The
            // FP32 panel A W32 is still formed for stage three.
            PODCG_CK(h, launch_spmm_f32(A->row_ptr, A->col, h->val32, h->W32, h->ld, h->AW32, h->ld, n, w, h->sms, s));
            PODCG_CK(h, launch_spmm(A->row_ptr, A->col, A->val, h->W, h->ld, h->AW, h->ld, n, w, h->sms, s));
            PODCG_CK(h, launch_gram(n, h->Y, h->ld, p, h->AW, h->ld, w, b, h->G, kWMax + 1, upper, h->gram_work,
                                    h->gram_work_bytes, h->sms, s));
            launches += 1;
        } else if (h->mixed) {
            const float* X32 = y > w ? h->Y32 : h->W32;
            PODCG_CK(h, launch_spmm_f32(A->row_ptr, A->col, h->val32, h->W32, h->ld, h->AW32, h->ld, n, w, h->sms, s));
            bool tc = h->cfg.use_tc_gram == 1 && y <= w;
            if (h->cfg.use_tc_gram == -1 && y <= w && n >= 65536) {
                // timed once per basis width on the actual panels (the last call writes G again)
                if (h->gram_choice[w] < 0) {
                    for (int form = 0; form < 2; ++form) {
                        float tot = 0.0f;
                        for (int rep = 0; rep < 4; ++rep) {
                            PODCG_CK(h, cudaEventRecord(h->tev[0], s));
                            if (form == 1)
                                PODCG_CK(h, launch_gram_tc(n, X32, h->ld, p, h->AW32, h->ld, w, bt, h->G, kWMax + 1,
                                                           h->gram_work, h->gram_work_bytes, tc_err, h->sms, s));
                            else
                                PODCG_CK(h, launch_gram32(n, X32, h->ld, p, h->AW32, h->ld, w, b, h->G, kWMax + 1,
                                                          upper, h->gram_work, h->gram_work_bytes, h->sms, s));
                            PODCG_CK(h, cudaEventRecord(h->tev[1], s));
                            PODCG_CK(h, cudaEventSynchronize(h->tev[1]));
                            float ms = 0.0f;
                            cudaEventElapsedTime(&ms, h->tev[0], h->tev[1]);
                            if (rep > 0) tot += ms;
                        }
                        h->gram_ms[w][form] = tot / 3.0f;
                    }
                    h->gram_choice[w] = h->gram_ms[w][1] < h->gram_ms[w][0] ? 1 : 0;
                }
                tc = h->gram_choice[w] == 1;
            }
            h->last_gram_tc = tc ? 1 : 0;
            if (tc)
                PODCG_CK(h, launch_gram_tc(n, X32, h->ld, p, h->AW32, h->ld, w, bt, h->G, kWMax + 1, h->gram_work,
                                           h->gram_work_bytes, tc_err, h->sms, s));
            else
                PODCG_CK(h, launch_gram32(n, X32, h->ld, p, h->AW32, h->ld, w, b, h->G, kWMax + 1, upper, h->gram_work,
                                          h->gram_work_bytes, h->sms, s));
        } else {
            const double* X = y > w ? h->Y : h->W;
            PODCG_CK(h, launch_spmm(A->row_ptr, A->col, A->val, h->W, h->ld, h->AW, h->ld, n, w, h->sms, s));
            PODCG_CK(h, launch_gram(n, X, h->ld, p, h->AW, h->ld, w, b, h->G, kWMax + 1, upper, h->gram_work,
                                    h->gram_work_bytes, h->sms, s));
        }
        PODCG_CK(h, launch_chol(h->G, kWMax + 1, h->Rinv, h->st, h->cfg.cond_diag, s));
        launches += 4;
    } else if (y > 0) {
        // no stage-one basis (cannot happen with y >= w unless the POD is empty): stage two
        // needs Y^T b alone, with w = 0
        PODCG_CK(h, launch_gram(n, h->Y, h->ld, y, nullptr, h->ld, 0, b, h->G, kWMax + 1, 0, h->gram_work,
                                    h->gram_work_bytes, h->sms, s));
        launches += 2;
    }
    PODCG_CK(h, cudaEventRecord(h->ev[2], s));

    // stage two (Section 4.2): iterative solve over range(Y), directions appended to the basis
    h->k2 = 0;
    h->pod_y_used = 0;
    int w3 = w;
    if (y > 0) {
        pod_cg_status s2 = run_stage2(h, L);
        if (s2 != POD_CG_OK) return s2;
        const DevState& d = *h->st_host;
        if (d.status != 0) return fail(h, (pod_cg_status)d.status, "stage two: device error status");
        h->k2 = d.k2;
        h->pod_y_used = y;
        h->k2_launch = d.k2 + d.s2_break;
        w3 = d.w;
        if (d.w1 < w) h->w_clobbered = true;   // stage-one basis dropped: V2 starts at column 0
        launches += 2 + 2 * h->k2_launch;
        if (h->mixed && w3 > 0) {
            // MIXED: stage three iterates on the FP32 basis [W32, V2_32] (V2's columns scaled
            // to unit A-norm), whose A-products come from the FP32 SpMM as A W32's do, and it
            // re-forms that basis' Gram and
            // Cholesky factor instead of taking blockdiag(R, sqrt(T2)): rounded to FP32, and
            // multiplied by the FP32 matrix with its cancellation on smooth vectors, [W, V2]
            // is A-orthogonal only to FP32 accuracy times that cancellation, and the FP32 inner
            // CG needs a factor consistent with the basis it projects with (as stage one's W32
            // gets one). The factor solve also replaces [what; alpha] by the Galerkin
            // coordinates over range([W, V2]), which the stage-two solution equals in exact
            // arithmetic.
            const size_t off = (size_t)d.w1 * h->ld;
            if (h->k2 > 0) {
                PODCG_CK(h, launch_s2_to_f32(n, h->ld, h->W, h->W32, d.w1, h->k2, h->Rinv, h->sms, s));
                PODCG_CK(h, launch_spmm_f32(A->row_ptr, A->col, h->val32, h->W32 + off, h->ld, h->AW32 + off, h->ld,
                                            n, h->k2, h->sms, s));
            }
            PODCG_CK(h, launch_gram32(n, h->W32, h->ld, w3, h->AW32, h->ld, w3, b, h->G, kWMax + 1, 1, h->gram_work,
                                      h->gram_work_bytes, h->sms, s));
            // a non-positive pivot keeps the leading columns: stage two's last directions,
            // taken after its residual had fallen to rounding level, are the ones that turn
            // dependent once rounded to FP32
            PODCG_CK(h, launch_chol(h->G, kWMax + 1, h->Rinv, h->st, h->cfg.cond_diag, s, w3, 1));
            pod_cg_status rs3 = read_state(h);
            if (rs3 != POD_CG_OK) return rs3;
            w3 = h->st_host->w;
            launches += 5;
        }
    }
    const int wb = wb_bucket(w3);
    if (h->mixed)
        PODCG_CK(h, launch_stage1_mx(wb, h->pd, n, h->W32, h->x, h->partials, h->counters + 4 * kCounterStride, h->st, tol, h->sms, s));
    else
        PODCG_CK(h, launch_stage1(wb, h->pd, n, h->W, h->AW, h->x, h->r, h->partials, h->counters + 4 * kCounterStride, h->st, tol,
                                  h->sms, s));
    PODCG_CK(h, cudaEventRecord(h->ev[3], s));

    // stage three (Algorithm 1 with basis [W, V2], or with all of Y: three_stage = 2)
    h->it_mode = h->cfg.three_stage == 2 && y > 0;
    if (h->it_mode) {
        pod_cg_status its = run_loop_it(h, L, &launches);
        if (its != POD_CG_OK) return its;
        const int sysid = h->system_counter++;
        return finish_solve(h, x_out, w, launches, stats, sysid);
    }
    if (h->mixed) {
        pod_cg_status ms = set_panel_maps(h, w3);
        if (ms != POD_CG_OK) return ms;
        // the direction passes' mu = M c, M = R^{-1} R^{-T} of this solve's factor
        PODCG_CK(h, launch_mu_matrix(h->Rinv, h->st, h->Mmu, s));
        launches += 1;
    }
    pod_cg_status ps = choose_proj_form(h, wb, L);
    if (ps != POD_CG_OK) return ps;
    PODCG_CK(h, cudaEventRecord(h->ev[5], s));
    pod_cg_status ls = run_loop(h, wb, L);
    if (ls != POD_CG_OK) return ls;
    const int sysid = h->system_counter++;
    pod_cg_status fs = finish_solve(h, x_out, w, launches, stats, sysid);
    if (fs == POD_CG_OK && h->kry_on && !h->kc.frozen) fs = krylov_update(h, A, b);
    if (fs == POD_CG_OK && h->wsel_slot >= 0) {
        // device time of this solve without the one-time projection-form timing
        float t0 = 0.0f, t1 = 0.0f;
        cudaEventElapsedTime(&t0, h->ev[0], h->ev[3]);
        cudaEventElapsedTime(&t1, h->ev[5], h->ev[4]);
        h->wsel_ms[h->wsel_slot] += double(t0) + double(t1);
        h->wsel_n[h->wsel_slot] += 1;
        if (++h->wsel_pos == (int)h->wsel_order.size()) {
            int best = 0;
            for (int i = 1; i < (int)h->wsel_caps.size(); ++i)
                if (h->wsel_ms[i] / h->wsel_n[i] < h->wsel_ms[best] / h->wsel_n[best]) best = i;
            h->w_cap = h->wsel_caps[best];
            h->wsel_done = true;
        }
    }

    // keep this system's factors for the adjoint
    if (h->cfg.keep_factors > 0 && !h->mixed && fs == POD_CG_OK) {
        const int slot = h->k_next;
        h->k_next = (h->k_next + 1) % h->cfg.keep_factors;
        // the stage-one basis (three-stage mode: without the stage-two directions)
        const int wu = h->pod_y_used > 0 ? h->st_host->w1 : h->st_host->w;
        const size_t blk = (size_t)h->ld * h->cfg.w_max;
        if (wu > 0) {
            PODCG_CK(h, cudaMemcpyAsync(h->kW + slot * blk, h->W, sizeof(double) * h->ld * wu, cudaMemcpyDeviceToDevice, s));
            PODCG_CK(h, cudaMemcpyAsync(h->kAW + slot * blk, h->AW, sizeof(double) * h->ld * wu, cudaMemcpyDeviceToDevice, s));
            PODCG_CK(h, cudaMemcpyAsync(h->kG + (size_t)slot * kWMax * (kWMax + 1), h->G,
                                        sizeof(double) * kWMax * (kWMax + 1), cudaMemcpyDeviceToDevice, s));
        }
        h->k_id[slot] = sysid;
        h->k_w[slot] = wu;
        PODCG_CK(h, cudaStreamSynchronize(s));
    }
    return fs;
}

pod_cg_status pod_cg_solve_adjoint(pod_cg_t* h, int system_id, const pod_cg_csr* A, const double* g, double tol,
                                   double* lambda_out, pod_cg_stats* stats)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    pod_cg_status cs = check_csr(h, A, h->n);
    if (cs != POD_CG_OK) return cs;
    if (!g || !lambda_out || g == lambda_out) return fail(h, POD_CG_ERR_ARG, "bad g / lambda_out");
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(h, POD_CG_ERR_ARG, "tol must be finite and >= 0");
    if (h->mixed) return fail(h, POD_CG_ERR_ARG, "the adjoint solve runs in FP64 mode");
    int slot = -1;
    for (int k = 0; k < (int)h->k_id.size(); ++k)
        if (h->k_id[k] == system_id) slot = k;
    if (slot < 0) return fail(h, POD_CG_ERR_STATE, "factors of this system were not kept (keep_factors too small?)");
    const int n = h->n;
    cudaStream_t s = h->stream;
    const int w = h->k_w[slot];
    const size_t blk = (size_t)h->ld * h->cfg.w_max;
    // restore W_j, A_j W_j and W_j^T A_j W_j of the forward solve (A_j symmetric: same factor)
    if (w > 0) {
        PODCG_CK(h, cudaMemcpyAsync(h->W, h->kW + slot * blk, sizeof(double) * h->ld * w, cudaMemcpyDeviceToDevice, s));
        PODCG_CK(h, cudaMemcpyAsync(h->AW, h->kAW + slot * blk, sizeof(double) * h->ld * w, cudaMemcpyDeviceToDevice, s));
        PODCG_CK(h, cudaMemcpyAsync(h->G, h->kG + (size_t)slot * kWMax * (kWMax + 1),
                                    sizeof(double) * kWMax * (kWMax + 1), cudaMemcpyDeviceToDevice, s));
    }
    h->pod_w = w;
    h->pod_dirty = h->s_count > 0;   // the next forward solve recomputes its own basis
    h->w_clobbered = true;
    reset_state(h, A, g, tol);
    pod_cg_status bst = setup_bsr(h, A);
    if (bst != POD_CG_OK) return bst;
    PODCG_CK(h, cudaMemcpyAsync(h->pd, h->pd_host, sizeof(ProbDesc), cudaMemcpyHostToDevice, s));
    PODCG_CK(h, cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, s));
    PODCG_CK(h, cudaMemsetAsync(h->gbar, 0, 2 * sizeof(unsigned int), s));   // the persistent loop's barrier
    PODCG_CK(h, cudaEventRecord(h->ev[0], s));
    PODCG_CK(h, launch_dinv(h->pd, n, h->dinv, h->dinv32, h->st, h->sms, s));
    PODCG_CK(h, cudaEventRecord(h->ev[1], s));
    int launches = 2;
    if (w > 0) {
        // ghat = W^T g into the right-hand-side column of the saved Gram, then the Cholesky
        PODCG_CK(h, launch_gram(n, h->W, h->ld, w, nullptr, h->ld, 0, g, h->G + w, kWMax + 1, 0, h->gram_work,
                                h->gram_work_bytes, h->sms, s));
        PODCG_CK(h, launch_chol(h->G, kWMax + 1, h->Rinv, h->st, h->cfg.cond_diag, s));
        launches += 3;
    }
    const int wb = wb_bucket(w);
    PODCG_CK(h, cudaEventRecord(h->ev[2], s));
    h->k2 = 0;
    h->pod_y_used = 0;
    h->it_mode = false;
    PODCG_CK(h, launch_stage1(wb, h->pd, n, h->W, h->AW, h->x, h->r, h->partials, h->counters + 4 * kCounterStride, h->st, tol,
                              h->sms, s));
    PODCG_CK(h, cudaEventRecord(h->ev[3], s));
    int L = 1;
    pod_cg_status lst = choose_lanes(h, A, &L);
    if (lst != POD_CG_OK) return lst;
    pod_cg_status ls = run_loop(h, wb, L);
    if (ls != POD_CG_OK) return ls;
    return finish_solve(h, lambda_out, w, launches, stats, system_id);
}

pod_cg_status pod_cg_set_krylov(pod_cg_t* h, const pod_cg_krylov_config* kc)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    if (!kc) return fail(h, POD_CG_ERR_ARG, "cfg is NULL");
    const pod_cg_krylov_config& c = *kc;
    if (c.p_cap < 1 || c.p_cap > kSMax || c.y_threshold < 0 || (c.y_threshold > 0 && c.y_threshold + c.p_cap > kSMax) ||
        c.y_keep < 1 || c.y_keep > kSMax || (c.y_threshold > 0 && c.y_keep > c.y_threshold) || c.w_keep < 0 ||
        c.w_keep > c.y_keep || !std::isfinite(c.nu) || (c.weights != 0 && c.weights != 1) ||
        (c.frozen != 0 && c.frozen != 1))
        return fail(h, POD_CG_ERR_ARG,
                    "invalid Krylov settings (1 <= p_cap <= 64, y_threshold 0 or y_threshold + p_cap <= 64, "
                    "1 <= y_keep <= y_threshold, 0 <= w_keep <= y_keep, finite nu, weights 0/1, frozen 0/1)");
    if (!h->kry_on) {
        if (h->mixed || h->cfg.three_stage != 1 || h->cfg.pod_metric != 0 || h->out_q > 0 || h->s_count > 0 ||
            h->cfg.keep_factors > 0)
            return fail(h, POD_CG_ERR_STATE,
                        "Krylov-vector snapshots need an FP64 handle with three_stage = 1, pod_metric = 0, no output "
                        "functionals, no solution snapshots and keep_factors = 0");
        const size_t ld = (size_t)h->ld;
        cudaError_t e = cudaSuccess;
        // the augmenting basis of a solve can reach kSMax columns
        if (std::max(h->cfg.y_max, h->cfg.w_max) < kSMax) {
            if (h->Y) cudaFree(h->Y);
            h->Y = nullptr;
            e = dalloc(&h->Y, ld * kSMax);
        }
        if (e == cudaSuccess) e = dalloc(&h->Z, ld * kSMax);
        if (e == cudaSuccess) e = dalloc(&h->Zalt, ld * kSMax);
        if (e == cudaSuccess) e = dalloc(&h->AZ, ld * kSMax);
        if (e == cudaSuccess) e = dalloc(&h->kgam, (size_t)kSMax);
        if (e == cudaSuccess) e = dalloc(&h->zG, (size_t)kSMax * (kSMax + 1));
        if (e == cudaSuccess) e = dalloc(&h->zG2, (size_t)kSMax * kSMax);
        if (e == cudaSuccess) e = dalloc(&h->zcoord, (size_t)kSMax);
        if (e == cudaSuccess) e = dalloc(&h->zeta, (size_t)kSMax);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->zeta, 0, sizeof(double) * kSMax, h->stream);
        // Gram workspace for Z^T [A Z, b], the compression's Gram and the stage-one Gram of a
        // basis up to kSMax columns wide
        size_t need = h->gram_work_bytes;
        for (int k = 1; k <= kSMax; ++k) {
            need = std::max(need, gram_workspace_bytes(h->n, k, k + 1, h->sms));
            need = std::max(need, gram_workspace_bytes(h->n, k, k, h->sms));
            for (int j = 1; j <= k + 1 && j <= kWMax + 1; ++j)
                need = std::max(need, gram_workspace_bytes(h->n, k, j, h->sms));
        }
        if (e == cudaSuccess && need > h->gram_work_bytes) {
            cudaFree(h->gram_work);
            h->gram_work = nullptr;
            e = cudaMalloc((void**)&h->gram_work, need);
            if (e == cudaSuccess) h->gram_work_bytes = need;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return fail(h, POD_CG_ERR_OOM, std::string("pod_cg_set_krylov: ") + cudaGetErrorString(e));
        h->kry_on = true;
        h->cfg.bsr = 0;   // the direction record lives in the CSR product
        h->z = 0;
        h->w_idx.clear();
        h->compressions = 0;
    }
    h->kc = c;
    return POD_CG_OK;
}

pod_cg_status pod_cg_krylov_state(pod_cg_t* h, int* z, int* w, int* compressions, double* Z_out, int* w_cols)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    if (!h->kry_on) return fail(h, POD_CG_ERR_STATE, "Krylov-vector mode is off (pod_cg_set_krylov)");
    if (z) *z = h->z;
    if (w) *w = (int)h->w_idx.size();
    if (compressions) *compressions = h->compressions;
    if (w_cols)
        for (size_t i = 0; i < h->w_idx.size(); ++i) w_cols[i] = h->w_idx[i];
    if (Z_out && h->z > 0) {
        PODCG_CK(h, cudaMemcpy2DAsync(Z_out, sizeof(double) * h->n, h->Z, sizeof(double) * h->ld, sizeof(double) * h->n,
                                      h->z, cudaMemcpyDeviceToDevice, h->stream));
        PODCG_CK(h, cudaStreamSynchronize(h->stream));
    }
    return POD_CG_OK;
}

pod_cg_status pod_cg_krylov_coords(pod_cg_t* h, const pod_cg_csr* A, const double* b, double* coords_out,
                                   double* weights_out)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    if (!h->kry_on) return fail(h, POD_CG_ERR_STATE, "Krylov-vector mode is off (pod_cg_set_krylov)");
    pod_cg_status cs = check_csr(h, A, h->n);
    if (cs != POD_CG_OK) return cs;
    if (!b || (!coords_out && h->z > 0)) return fail(h, POD_CG_ERR_ARG, "b and coords_out must be non-NULL");
    if (h->z == 0) return POD_CG_OK;
    cs = krylov_coords_now(h, A, b, false);
    if (cs != POD_CG_OK) return cs;
    PODCG_CK(h, cudaMemcpyAsync(coords_out, h->zcoord, sizeof(double) * h->z, cudaMemcpyDeviceToDevice, h->stream));
    if (weights_out)
        PODCG_CK(h, cudaMemcpyAsync(weights_out, h->zeta, sizeof(double) * h->z, cudaMemcpyDeviceToDevice, h->stream));
    PODCG_CK(h, cudaStreamSynchronize(h->stream));
    return POD_CG_OK;
}

pod_cg_status pod_cg_krylov_compress(pod_cg_t* h, const pod_cg_csr* A, const double* eta, int y_keep, int w_keep)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    if (!h->kry_on) return fail(h, POD_CG_ERR_STATE, "Krylov-vector mode is off (pod_cg_set_krylov)");
    pod_cg_status cs = check_csr(h, A, h->n);
    if (cs != POD_CG_OK) return cs;
    if (y_keep < 1 || y_keep > kSMax || w_keep < 0 || w_keep > y_keep)
        return fail(h, POD_CG_ERR_ARG, "1 <= y_keep <= 64 and 0 <= w_keep <= y_keep");
    if (eta && h->z > 0) {   // the caller's weights, copied: the accumulated ones stay untouched
        PODCG_CK(h, cudaMemcpyAsync(h->zcoord, eta, sizeof(double) * h->z, cudaMemcpyDeviceToDevice, h->stream));
        eta = h->zcoord;
    }
    cs = krylov_compress_now(h, A, eta ? eta : h->zeta, y_keep, w_keep);
    if (cs != POD_CG_OK) return cs;
    PODCG_CK(h, cudaStreamSynchronize(h->stream));
    return POD_CG_OK;
}

pod_cg_status pod_cg_time_kernels(pod_cg_t* h, const pod_cg_csr* A, const double* b, int reps, float* ms_out)
{
    if (!h) return fail(nullptr, POD_CG_ERR_ARG, "handle is NULL");
    pod_cg_status cs = check_csr(h, A, h->n);
    if (cs != POD_CG_OK) return cs;
    if (!b || !ms_out || reps < 1) return fail(h, POD_CG_ERR_ARG, "bad arguments");
    cudaStream_t s = h->stream;
    reset_state(h, A, b, 0.0);
    pod_cg_status bst = setup_bsr(h, A);
    if (bst != POD_CG_OK) return bst;
    PODCG_CK(h, cudaMemcpyAsync(h->pd, h->pd_host, sizeof(ProbDesc), cudaMemcpyHostToDevice, s));
    DevState& t = *h->st_host;
    t.rho = 1.0;
    t.alpha = 1e-30;
    t.beta = 0.5;
    t.k_max = 1 << 30;
    t.max_refine = 1 << 30;
    t.tol2 = 0.0;
    t.tol2_in = -1.0;
    t.dir_pending = 1;
    const int w = h->pod_w;
    const int L = h->last_L > 0 ? h->last_L : spmv_lanes_for(h->n > 0 ? double(A->nnz) / h->n : 1.0);
    Plan pl;
    make_plan(h, wb_bucket(w), L, h->mixed, 0, 0, 0, pl);
    KSpec* ks[4] = {&pl.spmv, &pl.upd, &pl.dir, &pl.res};
    for (int k = 0; k < 4; ++k) {
        float total = 0.0f;
        for (int rep = 0; rep < reps + 1; ++rep) {
            PODCG_CK(h, cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, s));
            PODCG_CK(h, cudaEventRecord(h->ev[0], s));
            PODCG_CK(h, launch_spec(*ks[k], s));
            PODCG_CK(h, cudaEventRecord(h->ev[1], s));
            PODCG_CK(h, cudaEventSynchronize(h->ev[1]));
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
            if (rep > 0) total += ms;   // the first launch is a warm-up
        }
        ms_out[k] = total / reps;
    }
    return POD_CG_OK;
}

pod_cg_status pod_cg_proj_tuning(const pod_cg_t* h, int* forms, float* ms)
{
    if (!h) return POD_CG_ERR_ARG;
    for (int b = 0; b < 6; ++b) {
        if (forms) forms[b] = h->proj_form[b];
        if (ms)
            for (int f = 0; f < 2; ++f)
                for (int k = 0; k < 2; ++k) ms[4 * b + 2 * f + k] = h->proj_ms[b][f][k];
    }
    return POD_CG_OK;
}

pod_cg_status pod_cg_w_tuning(const pod_cg_t* h, int* cap, int* caps, float* ms)
{
    if (!h) return POD_CG_ERR_ARG;
    if (cap) *cap = h->wsel_done ? h->w_cap : h->cfg.w_max;
    for (int i = 0; i < 8; ++i) {
        const bool ok = i < (int)h->wsel_caps.size();
        if (caps) caps[i] = ok ? h->wsel_caps[i] : 0;
        if (ms) ms[i] = (ok && h->wsel_n[i] > 0) ? float(h->wsel_ms[i] / h->wsel_n[i]) : 0.0f;
    }
    return POD_CG_OK;
}

pod_cg_status pod_cg_tuning(const pod_cg_t* h, int* spmv_lanes, float* lane_ms)
{
    if (!h) return POD_CG_ERR_ARG;
    if (spmv_lanes) *spmv_lanes = h->last_L;
    if (lane_ms) {
        for (int k = 0; k < 6; ++k) lane_ms[k] = 0.0f;
        for (const auto& c : h->lanes)
            if (c.L == h->last_L)
                for (int k = 0; k < 6; ++k) lane_ms[k] = c.ms[k];
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

pod_cg_status pod_cg_debug_wait_timeout(int mask, long long cycles)
{
    const int all = kWaitTestGramTc | kWaitTestStaged | kWaitTestLoop;
    if (mask < 0 || mask > all || (mask != 0 && (cycles < 1000 || cycles > 4000000000LL)))
        return fail(nullptr, POD_CG_ERR_ARG, "pod_cg_debug_wait_timeout: mask 0..7 and 1e3 <= cycles <= 4e9");
    const long long c = mask ? cycles : 0;
    cudaError_t e = gram_tc_set_wait_test(mask & kWaitTestGramTc, c);
    if (e == cudaSuccess) e = cg_set_wait_test(mask & kWaitTestStaged, c);
    if (e == cudaSuccess) e = loop_set_wait_test(mask & kWaitTestLoop, c);
    if (e != cudaSuccess) return cuda_fail(nullptr, "pod_cg_debug_wait_timeout", e);
    return POD_CG_OK;
}

size_t pod_cg_gram_workspace_for(int n, int p, int q, int sms)
{
    if (n < 1 || p < 1 || q < 1 || sms < 1) return 0;
    return gram_workspace_bytes(n, p, q, sms);
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

size_t pod_cg_gram_tc_workspace(int n, int p, int q)
{
    if (n < 1 || p < 1 || q < 1) return 0;
    return gram_tc_workspace_bytes(n, p, q, device_sms());
}

pod_cg_status pod_cg_gram_tc(int n, int elem_bytes, const void* X, int p, const void* Y, int qy, const double* e,
                             double* G, void* work, size_t work_bytes, void* stream)
{
    const int q = qy + (e ? 1 : 0);
    if (n < 1 || p < 1 || p > kWMax || qy < 0 || qy > kWMax || q < 1 || (elem_bytes != 4 && elem_bytes != 8) ||
        !X || (qy > 0 && !Y) || !G || !work)
        return fail(nullptr, POD_CG_ERR_ARG, "bad arguments");
    const size_t ldb = (size_t)n * (size_t)elem_bytes;
    if (!gram_tc_aligned(X, ldb) || (qy > 0 && !gram_tc_aligned(Y, ldb)) || (e && !gram_tc_aligned(e, 16)))
        return fail(nullptr, POD_CG_ERR_ARG, "pod_cg_gram_tc: X, Y, e need 16-byte aligned starts and n*elem_bytes a multiple of 16");
    if (work_bytes < gram_tc_workspace_bytes(n, p, q, device_sms()))
        return fail(nullptr, POD_CG_ERR_ARG, "workspace too small");
    cudaError_t err;
    if (elem_bytes == 4)
        err = launch_gram_tc(n, (const float*)X, n, p, (const float*)Y, n, qy, e, G, q, (double*)work, work_bytes,
                             nullptr, device_sms(), (cudaStream_t)stream);
    else
        err = launch_gram_tc(n, (const double*)X, n, p, (const double*)Y, n, qy, e, G, q, (double*)work, work_bytes,
                             nullptr, device_sms(), (cudaStream_t)stream);
    if (err != cudaSuccess) return cuda_fail(nullptr, "pod_cg_gram_tc", err);
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
    if (e == cudaSuccess) e = launch_pod_eig(G, kSMax, s, energy, rank_tol, w_max, C, sigma2_out, st, nullptr, 0, str);
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
