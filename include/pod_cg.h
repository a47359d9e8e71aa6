/*
 * pod_cg.h — C ABI of the GB300 (sm_103a) POD-augmented conjugate-gradient library.
 *
 * Method: K. Carlberg, V. Forstall, R. Tuminaro, "Krylov-subspace recycling via the
 * POD-augmented conjugate-gradient method". A sequence of sparse SPD systems
 * A_j x_j = b_j (Section 2, Eq. (sequence)) is solved to inexact tolerances
 * ||b_j - A_j x_j||_2 <= tol ||b_j||_2 (Eq. (sequenceInexact), with a relative tolerance).
 * For system j the library, with the stages numbered as in Section 4,
 *   1. computes a POD basis W_j of the retained snapshots (previous solutions) with the
 *      eigenvalue route of Algorithm 4 (unit weights): Gram S^T S, symmetric eigensolve,
 *      energy truncation, lift W = S V Sigma^{-1}; in the identity metric by default, in
 *      the metric A_j with pod_metric = 1 (Gram S^T A_j S), or in the output metric C^T C
 *      after pod_cg_set_output_functionals (Section 3.3);
 *   2. stage one (Section 4.1, Algorithm 2): AW = A_j W, Ahat = W^T AW, Cholesky
 *      Ahat = R^T R, Ahat what = W^T b, x0 = W what, r0 = b - AW what;
 *   3. (three_stage = 1 only) stage two (Section 4.2): the POD also gives a larger
 *      augmenting basis Y whose first w columns are W; Algorithm 1 runs on the reduced
 *      system Y^T A Y yhat = Y^T b through products Y^T (A (Y p)) (Y^T A Y is never
 *      formed), augmented with the stage-one coordinates, reusing R and unpreconditioned,
 *      to tol_stage2 * tol * ||b||; its k2 directions V2 = Y Phi2 extend the basis to
 *      [W, V2] with the block-diagonal factor blockdiag(R, sqrt(T2)), T2 = diag(V2^T A V2);
 *   4. stage three (Section 4.3, Algorithm 1 with basis [W, V2], V2 empty without stage
 *      two): Jacobi-preconditioned CG whose directions are A_j-orthogonalised against the
 *      basis through mu = R^{-1} R^{-T} (AW)^T z and p = z + beta p - W mu; or
 *      (three_stage = 2, Section 4.3.1) against all of Y, mu from an inner reduced solve
 *      of Y^T A Y mu = Y^T A z that reuses the reduced directions stored so far. The CG
 *      product A p runs in CSR form, or in 3x3 block form for patterns made of full 3x3
 *      blocks (bsr).
 * Every step runs in hand-written CUDA kernels; this header is the only interface.
 *
 * Conventions for every entry point:
 *  - Array arguments marked "device" are device pointers in the current CUDA context,
 *    borrowed for the duration of the call (the library never frees them and keeps no
 *    reference after the call returns). Arguments marked "host" are host pointers.
 *  - CSR matrices use 32-bit indices: row_ptr[n+1], col[nnz] (sorted within each row,
 *    diagonal present), val[nnz] float64; nnz < 2^31.
 *  - n-by-k dense blocks are column-major with leading dimension n (column j starts at
 *    element j*n). Small k-by-k matrices are row-major.
 *  - Work is ordered on the CUDA stream given at creation (or per call for the stateless
 *    step functions; NULL = the legacy default stream). Handle calls synchronise that
 *    stream before returning, so host outputs (stats, w) are valid on return.
 *  - Every function returns a pod_cg_status. On failure a message is available from
 *    pod_cg_last_error(handle) (or pod_cg_last_error(NULL) for stateless calls); the
 *    handle stays usable and solution outputs hold the best iterate reached.
 */
#ifndef POD_CG_H
#define POD_CG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pod_cg_t pod_cg_t;

typedef enum {
    POD_CG_OK = 0,
    POD_CG_ERR_ARG = 1,        /* invalid argument (sizes, NULL pointers, bad config) */
    POD_CG_ERR_NOT_SPD = 2,    /* non-positive Jacobi diagonal */
    POD_CG_ERR_BREAKDOWN = 3,  /* (A p, p) <= 0 during CG: matrix not SPD */
    POD_CG_ERR_MAXIT = 4,      /* iteration or refinement cap reached above tolerance */
    POD_CG_ERR_NONFINITE = 5,  /* NaN/Inf in a scalar of the iteration */
    POD_CG_ERR_CUDA = 6,       /* a CUDA runtime call failed */
    POD_CG_ERR_TIMEOUT = 7,    /* a bounded device wait expired */
    POD_CG_ERR_OOM = 8,        /* device allocation failed */
    POD_CG_ERR_STATE = 9       /* call not valid in the handle's state (e.g. evicted system) */
} pod_cg_status;

enum { POD_CG_FP64 = 0, POD_CG_MIXED = 1 };

/* Solver settings. Fill with pod_cg_config_default() and override fields. */
typedef struct {
    int    w_max;        /* cap on the POD basis dimension w (1..64) */
    int    s_max;        /* snapshot window: the last s_max added snapshots are kept (1..64) */
    double energy;       /* POD energy criterion (Algorithm 4 step 3), e.g. 0.9999 */
    double rank_tol;     /* eigenvalues <= rank_tol * lambda_1 count as rank deficient (1e-13) */
    int    k_max;        /* cap on CG iterations per solve, summed over restarts (0: stage
                            one only); at the cap x_out holds the k_max-th iterate */
    int    max_refine;   /* FP64: residual-replacement restarts; MIXED: FP64 refinement steps */
    int    precision;    /* POD_CG_FP64, or POD_CG_MIXED (FP32 inner CG, FP64 refinement) */
    double inner_tol;    /* MIXED: each inner solve reduces its residual by this factor, or
                            only by half the factor that reaches the tolerance when that is
                            larger (the last refinement step stops where it is needed) */
    int    use_tc_gram;  /* stage-one Gram W^T [AW, b] of a MIXED two-stage solve: 1 = on the
                            tensor cores with split-bf16 products (pod_cg_gram_tc; MIXED only,
                            else ERR_ARG at create), 0 = on the CUDA cores (FP32 panels, FP64
                            sums), -1 = the faster of the two, timed on the actual panels once
                            per basis width on the first system of >= 65,536 rows (smaller
                            systems: CUDA cores); stats.gram_tc reports which ran. Solves that
                            run stage two keep the CUDA-core Gram (its reduced residual
                            cancels). FP64 mode keeps the FP64 Gram whatever the setting: an
                            FP32-rounded W^T A W leaves the directions A-orthogonal to W only to
                            ~1e-7 cond(W^T A W), too loose for FP64 tolerances */
    int    cond_diag;    /* 1: compute cond_2(W^T A W) per solve (diagnostic, Section 5.2) */
    int    keep_factors; /* systems whose W, AW, R are kept for pod_cg_solve_adjoint (0..) */
    int    loop_mode;    /* 0: the CG loop is one conditional CUDA graph (no host round trip);
                            1: plain graphs of 16 unrolled iterations, host check per chunk
                            (same kernels; a form that kernel profilers can attribute);
                            2: as 0, with the MIXED inner loop of bases up to 8 wide and one
                            lane per CSR row run as one persistent cooperative launch per
                            refinement step (grid barriers between its passes; the same
                            iterates as 0, bit for bit; stats.ms_loop reports its time) */
    int    proj_form;    /* MIXED, FP32 update/direction passes: -1 = timed once per basis-
                            width bucket on the handle's first system of >= 65,536 rows in
                            it (else row-parallel); 0 = row-parallel float4; 1 = 256-row
                            tiles streamed into shared memory by the TMA engine, the
                            direction pass reading a 16-bit copy of W in two-stage solves
                            (see pod_cg_proj_tuning) */
    int    spmv_lanes;   /* CSR SpMV lanes per row: 0 = timed once per sparsity pattern
                            (systems of >= 65,536 rows; the pattern's heuristic width is kept
                            unless another is >= 10% faster); 1, 2, 4, 8, 16 or 32 = forced */
    int    three_stage;  /* 1: the three-stage algorithm of Section 4 (stage two over the
                            augmenting basis Y before stage three, which augments with
                            [W, V2]); 2: the same with stage three augmenting with all of Y,
                            its reduced solves done iteratively (Section 4.3.1; FP64 only,
                            else ERR_ARG); 0: stages one and three */
    int    y_max;        /* three_stage: cap on the augmenting-basis dimension y (1..s_max); y
                            is chosen by the POD energy criterion energy_y (Algorithm 4 step
                            3), capped at y_max, then raised to w when smaller (so y can reach
                            w_max), so that W is the first w columns of Y */
    double energy_y;     /* three_stage: POD energy criterion for Y (>= energy in practice) */
    double tol_stage2;   /* three_stage: stage two stops when ||Y^T (b - A x)||_2 <=
                            tol_stage2 * tol * ||b||_2, or after min(y, 64) - w iterations
                            (the reduced system is then solved exactly in exact arithmetic).
                            Keep it above the reduced residual's rounding floor (the paper's
                            1e-4 .. 1e-7 are): when Y^T A Y is well conditioned (metric A) and
                            stage two runs past that floor, its later directions are rounding
                            noise and re-A-orthogonalisation against them amplifies it.
                            Stage two runs in FP64 in both precisions (MIXED converts its
                            directions to FP32 for stage three) */
    double tol_inner;    /* three_stage = 2: each inner reduced solve stops when its residual
                            is <= tol_inner * ||Y^T A z||_2 (default 1e-12: inexact
                            projections onto range(Y) stall stage three when Y^T A Y is ill-
                            conditioned; the inner directions accumulate, so the inner work
                            of a whole solve is at most y - w reduced products) */
    int    bsr;          /* CG product in 3x3 block-sparse form (one column index per 9 values)
                            when the CSR pattern is made of full 3x3 blocks (three unknowns
                            per node, columns in aligned triplets, n % 3 == 0): -1 = when the
                            pattern allows (checked once per pattern), 0 = never, 1 = required
                            (ERR_ARG at solve time when the pattern does not allow it) */
    int    pod_metric;   /* POD metric (Section 3.3): 0 = identity (S^T S); 1 = the matrix A of
                            the system being solved (S^T A S from one SpMM of the snapshots
                            per solve: W is A-orthonormal, the metric under which POD bounds
                            the A-norm error). Output functionals (pod_cg_set_output_
                            functionals) need 0. */
    int    w_select;     /* 0: w from the energy criterion alone (Algorithm 4 step 3); 1: the
                            energy criterion under a cap on w chosen by measured cost (no
                            counterpart in the paper): once 8 snapshots are held, the next
                            solves try the caps 2, 4, 8, ... (powers of two below w_max) and
                            w_max, each twice in the order c1 .. ck ck .. c1 so that a steady
                            drift of the sequence's difficulty cancels, timing each solve on
                            the device (POD, stages one and two, the stage-three loop); the
                            cap with the least mean time is kept for the rest of the
                            sequence (pod_cg_w_tuning reports it) */
} pod_cg_config;

/* CSR matrix, device arrays, borrowed. */
typedef struct {
    int            n;
    int64_t        nnz;
    const int32_t* row_ptr;
    const int32_t* col;
    const double*  val;
} pod_cg_csr;

/* Per-solve statistics (host). The paper's measures (Section 5.1): matrix-vector
 * products, preconditioner applications (= stage-three iterations) and wall time. */
typedef struct {
    int    status;          /* pod_cg_status of the solve */
    int    iters;           /* stage-three CG iterations (all restarts / inner solves) */
    int    refinements;     /* FP64: residual-replacement restarts; MIXED: outer steps */
    int    w;               /* POD basis dimension used (0 = plain PCG) */
    int    s;               /* snapshots available */
    int    chol_failed;     /* 1 if W^T A W was not numerically SPD (basis dropped) */
    int    system_id;       /* id of this solve for pod_cg_solve_adjoint */
    int    spmv_count;      /* sparse products: iters + w (stage one) + stage2_iters +
                               true-residual products */
    int    launches;        /* kernels launched by this solve (graph-internal ones included) */
    int    y;               /* augmenting-basis dimension when stage two ran, else 0 */
    int    stage2_iters;    /* stage-two iterations k2 (stage three's basis is w + k2 wide) */
    int    inner_iters;     /* three_stage = 2: inner reduced iterations, summed */
    double stage1_relres;   /* ||b - A x0||/||b|| at the start of stage three: after stage
                               one (three_stage: after stages one and two) */
    double final_relres;    /* ||b - A x||/||b|| at exit, from an FP64 product */
    double cond_gram;       /* cond_2(W^T A W) when cond_diag = 1, else 0 */
    float  ms_pod;          /* device time of the POD update (eigensolve + lift) */
    float  ms_stage1;       /* device time of stage one (A W, Gram, Cholesky) */
    float  ms_stage2;       /* device time of stage two and the start x0, r0 of stage three */
    float  ms_stage3;       /* device time of the stage-three CG iteration */
    int    gram_tc;         /* 1 if the stage-one Gram ran on the tensor cores */
    float  ms_loop;         /* device time of the FP32 inner loop when it ran as one
                               persistent launch per refinement step (else 0) */
} pod_cg_stats;

/* ------------------------------------------------------------------ handle lifecycle */

/* Handle lifecycle: no counterpart in the paper (a library's housekeeping).
 * Defaults: w_max 32, s_max 40, energy 0.9999, rank_tol 1e-13, k_max 100000,
 * max_refine 5, FP64, inner_tol 1e-5, use_tc_gram -1, cond_diag 0, keep_factors 0,
 * loop_mode 0, proj_form -1, spmv_lanes 0, three_stage 0, y_max 40, energy_y 0.99999999,
 * tol_stage2 1e-4, tol_inner 1e-12, bsr -1, pod_metric 0, w_select 0. */
pod_cg_status pod_cg_config_default(pod_cg_config* cfg /* host, out */);

/* Create a solver for systems of order n (the problem statement of Section 2) whose work
 * is ordered on `cuda_stream` (a cudaStream_t; NULL = legacy default stream). The handle
 * owns the snapshot ring (s_max columns of n), the basis W and AW (w_max columns each),
 * the stage-one factor and all CG vectors. Errors: ERR_ARG (n < 1, bad config), ERR_OOM. */
pod_cg_status pod_cg_create(int n, const pod_cg_config* cfg /* host, NULL = defaults */,
                            void* cuda_stream, pod_cg_t** out /* host, out */);

/* Release everything the handle owns (no counterpart in the paper). NULL is accepted. */
pod_cg_status pod_cg_destroy(pod_cg_t* h);

/* Message of the last failure on this handle (no counterpart in the paper; NULL: of the
 * last stateless call on this thread). The string stays valid until the next call on the same handle/thread. */
const char* pod_cg_last_error(const pod_cg_t* h);

/* ---------------------------------------------------------------------- the sequence */

/* Append m snapshots (columns of X, device, n-by-m column-major) to the snapshot set S
 * (Section 3.1; here previous solutions, identity metric, unit weights). Once s_max
 * snapshots are held the oldest is replaced. Updates the snapshot Gram S^T S by the new
 * rows (Algorithm 4 step 1). Errors: ERR_ARG. */
pod_cg_status pod_cg_add_snapshots(pod_cg_t* h, const double* X, int m);

/* Output-oriented POD (Section 3.3, metric C^T C; Algorithm 5's POD): set q output
 * functionals (C: device, q-by-n row-major, copied; 1 <= q <= 128) whose values C x the
 * basis should capture. Later PODs then use the Gram (C S)^T (C S) of the snapshots'
 * output images instead of S^T S (the library keeps C s for each held snapshot, one
 * product of C per added snapshot), so W = S V Sigma^{-1} is C^T C-orthonormal. q = 0
 * returns to the identity metric. Errors: ERR_ARG, ERR_STATE (pod_metric = 1), ERR_CUDA. */
pod_cg_status pod_cg_set_output_functionals(pod_cg_t* h, const double* C, int q);

/* Forget all snapshots: the snapshot set of Algorithm 4 becomes empty, so the next solve
 * is Algorithm 1 with an empty basis (plain Jacobi PCG, Section 2.1). */
pod_cg_status pod_cg_clear_snapshots(pod_cg_t* h);

/* Solve A x = b to ||b - A x||_2 <= tol ||b||_2 (Eq. (sequenceInexact)) with the
 * POD-augmented method: POD of the current snapshots (Algorithm 4), stage one
 * (Algorithm 2), stage two when three_stage is set (Section 4.2), and augmented PCG
 * (stage three, Algorithm 1 with basis [W, V2]), then a true-residual check in
 * FP64 with residual replacement (FP64 mode) or FP64 iterative refinement around FP32
 * inner solves (MIXED). A: device CSR of order n; b, x_out: device, length n (x_out is
 * written, caller-owned; it may not alias b). st: host, may be NULL.
 * Errors: ERR_ARG, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_MAXIT, ERR_NONFINITE (x_out then holds
 * the last iterate), ERR_CUDA. */
pod_cg_status pod_cg_solve(pod_cg_t* h, const pod_cg_csr* A, const double* b, double tol,
                           double* x_out, pod_cg_stats* st);

/* Adjoint solve for a loss L(x_j): lambda = A_j^{-1} g (A_j symmetric, Section 2, so
 * A_j^{-T} = A_j^{-1}; no counterpart in the paper beyond that symmetry),
 * by the same POD-augmented method reusing the stage-one basis W_j, A_j W_j and the factor
 * R_j saved by the forward solve whose stats reported `system_id` (three-stage handles keep
 * the stage-one basis only; the adjoint runs stages one and three) (requires
 * keep_factors > 0 and that the system is among the last keep_factors solves).
 * A: the same matrix as that forward solve. g, lambda_out: device, length n.
 * Errors: as pod_cg_solve, plus ERR_STATE when the factors were not kept. */
pod_cg_status pod_cg_solve_adjoint(pod_cg_t* h, int system_id, const pod_cg_csr* A,
                                   const double* g, double tol, double* lambda_out,
                                   pod_cg_stats* st);

/* Copy the POD basis W of the last solve (Algorithm 4's output, Eq.
 * (podAlgebraicDefinition); device out, n-by-w column-major, room for w_max columns) and
 * its dimension (host out). */
pod_cg_status pod_cg_get_basis(pod_cg_t* h, double* W_out, int* w_out);

/* Copy stage three's augmenting basis [W, V2] of the last solve (Section 4.3) and its product
 * A [W, V2] (device outs, n-by-w3 column-major, room for 64 columns; either may be NULL)
 * and w3 = w + k2 (host out, may be NULL). FP64 handles only (ERR_STATE in MIXED, where
 * the basis is held in FP32). */
pod_cg_status pod_cg_get_stage3_basis(pod_cg_t* h, double* B_out, double* AB_out, int* w3_out);

/* Measurement support (no counterpart in the paper): time, with CUDA events on the
 * handle's stream, `reps` separate launches of each kernel of one stage-three iteration
 * (Algorithm 1's loop body) with the launch shapes the solve uses: [0] the CG product
 * q = A p with (A p, p), [1] the update r -= alpha q, z = M^{-1} r, (r, z), ||r||^2,
 * c = (A W)^T z, [2] the direction x += alpha p, p = z + beta p - W mu, [3] the FP64 true
 * residual b - A x. Uses the basis of the last pod_cg_solve; A and b must be that solve's.
 * ms_out (host, 4 floats) receives the mean milliseconds per launch. The handle's
 * iteration vectors are overwritten (the next solve resets them). Errors: ERR_ARG, ERR_CUDA. */
pod_cg_status pod_cg_time_kernels(pod_cg_t* h, const pod_cg_csr* A, const double* b, int reps, float* ms_out);

/* The FP32 projection forms chosen per basis-width bucket (buckets w <= 0, 8, 16, 32, 48,
 * 64): forms[6] receives a bit mask per bucket, bit 0 set when the update pass runs on tiles
 * staged in shared memory by the TMA engine (else row-parallel float4), bit 1 the same for
 * the direction pass, or -1 (bucket not used yet); ms[24] the times (ms) of each bucket as
 * [form 0 update, form 0 direction, form 1 update, form 1 direction], as measured by the
 * handle's one-time timing on the first MIXED system of at least 65,536 rows in that bucket
 * (0 where not timed); each pass keeps its faster form. This is the project's own tuning
 * record, with no counterpart in the paper. Host outputs; either pointer may be NULL. */
pod_cg_status pod_cg_proj_tuning(const pod_cg_t* h, int* forms, float* ms);

/* Record of the cost-tuned basis cap (w_select = 1; no counterpart in the paper): cap (host
 * out) the cap in force, w_max while the caps are still being timed or with w_select = 0;
 * caps[8] the candidates (0 past the last) and ms[8] their mean device time per solve
 * (0 = not timed yet). Either array may be NULL. */
pod_cg_status pod_cg_w_tuning(const pod_cg_t* h, int* cap, int* caps, float* ms);

/* Autotuner record (no counterpart in the paper): the CSR SpMV lanes-per-row used by the
 * last solve (1, 2, ..., 32) and, for systems of at least 65,536 rows, the measured
 * milliseconds of each candidate on that matrix (index k for 2^k lanes; -1 = not tried,
 * 0 = not timed). The first solve on a new sparsity pattern times the candidates on the
 * actual matrix; later solves on the same pattern reuse the choice. lane_ms: host, 6. */
pod_cg_status pod_cg_tuning(const pod_cg_t* h, int* spmv_lanes, float* lane_ms);

/* --------------------------------- the paper's snapshots: accumulated Krylov vectors */

/* Settings of the overall algorithm with Krylov-vector snapshots (Section 3.1, Section 3.2,
 * Algorithm 3). */
typedef struct {
    int    y_threshold;  /* storage threshold: after a solve whose directions take the
                            augmenting basis Z past y_threshold columns, Z is compressed
                            (Algorithm 3's truncation); 0 = never automatically (the caller
                            compresses with pod_cg_krylov_compress). y_threshold + p_cap <= 64 */
    int    y_keep;       /* columns kept by a compression (1..64; <= y_threshold when > 0) */
    int    w_keep;       /* after a compression the stage-one basis W is its first w_keep
                            columns (0..y_keep) */
    double nu;           /* stage-one set rule of Algorithm 3: a new direction k joins W when
                            T_kk / sum_i T_ii > nu (nu >= 1: every direction, nu <= 0: none) */
    int    weights;      /* POD weights of a compression: 0 = RBF weights (Eq. (weightsRBF),
                            rho(r) = 2^-(r-1) over the systems since the last compression),
                            1 = previous weights (Eq. (weightsPrevious)) of the last system */
    int    p_cap;        /* directions kept per system: the first p_cap of stage three (1..64),
                            fewer when Z has less room */
    int    frozen;       /* 1: solves use Z but append nothing and compress nothing */
} pod_cg_krylov_config;

/* Switch the handle to the paper's POD ingredients (Section 3): the augmenting basis Z holds
 * every system's stage-three directions, A_j-normalised, Z <- [Z, P_j T_j^{-1/2}] (T_j the
 * diagonal of (A_j p_k, p_k)); each system runs stage one on W (the columns of Z chosen by
 * nu), stage two over range(Z) and stage three with [W, V2] (Algorithm 3 with the stage-three
 * option of Section 4.3). After each solve the previous weights of its solution,
 * (Z^T A_j Z)^+ Z^T b_j (Eq. (weightsPrevious) with x_bar = 0), are formed; when Z exceeds
 * y_threshold it is replaced by its weighted POD in the metric A_j (Algorithm 4 with
 * Theta = A_j and the chosen weights; the result is A_j-orthonormal, so Algorithm 3's
 * Cholesky re-orthogonalisation is the identity), keeping y_keep columns, the first w_keep
 * of which form W. Requires an FP64 handle with three_stage = 1, pod_metric = 0, no output
 * functionals, no solution snapshots and keep_factors = 0 (else ERR_STATE); the CG product
 * runs in CSR form. Called again, it changes the settings and keeps Z. cfg: host.
 * Errors: ERR_ARG (settings out of range), ERR_STATE, ERR_OOM. pod_cg_clear_snapshots
 * empties Z. */
pod_cg_status pod_cg_set_krylov(pod_cg_t* h, const pod_cg_krylov_config* cfg);

/* The augmenting basis of Section 3.1's accumulated Krylov vectors (Algorithm 3): z, its
 * column count; w, the stage-one columns; compressions so far (host outs, each may be NULL);
 * Z_out (device, n-by-z column-major in Z's storage order, or NULL) a copy of Z and
 * w_cols (host, room for 64, or NULL) the indices of the stage-one columns.
 * Errors: ERR_STATE (Krylov mode off), ERR_CUDA. */
pod_cg_status pod_cg_krylov_state(pod_cg_t* h, int* z, int* w, int* compressions, double* Z_out, int* w_cols);

/* The coordinates (Z^T A Z)^+ Z^T b of a right-hand side in the current Z (Eq.
 * (weightsPrevious) with x_bar = 0; for A, b of the next system these are the ideal weights
 * of Section 3.2 that Section 5's weights experiment compares against). A: device CSR; b:
 * device, length n; coords_out: device, z entries. weights_out (device, z, or NULL): the
 * weights the next compression would use. Errors: ERR_ARG, ERR_STATE, ERR_CUDA. */
pod_cg_status pod_cg_krylov_coords(pod_cg_t* h, const pod_cg_csr* A, const double* b, double* coords_out,
                                   double* weights_out);

/* Compress Z now (Algorithm 3's truncation): Z <- the first y_keep modes of the POD of
 * Z diag(eta) in the metric A (Algorithm 4, Theta = A), W <- its first w_keep columns.
 * eta: device, z entries, or NULL for the accumulated weights of the handle's setting.
 * A: device CSR. Errors: ERR_ARG, ERR_STATE, ERR_CUDA. */
pod_cg_status pod_cg_krylov_compress(pod_cg_t* h, const pod_cg_csr* A, const double* eta, int y_keep, int w_keep);

/* ------------------------------------------------------ stateless steps of the path */

/* y = A x (the product of Algorithm 1's gamma = (A p, p)); x, y device length n. */
pod_cg_status pod_cg_spmv(const pod_cg_csr* A, const double* x, double* y, void* cuda_stream);

/* AW = A W for a device n-by-w column-major W (the w products of Section 4's stage-one
 * cost estimate). AW device n-by-w. */
pod_cg_status pod_cg_spmm(const pod_cg_csr* A, const double* W, int w, double* AW,
                          void* cuda_stream);

/* Bytes of device workspace pod_cg_gram needs for an n-row, p-by-q product (the Gram of
 * Algorithm 2 step 1 and Algorithm 4 step 1). */
size_t pod_cg_gram_workspace(int n, int p, int q);

/* Sizing support with no counterpart in the paper: pod_cg_gram_workspace for a GPU with
 * `sms` multiprocessors, with no device query, so a caller can size the workspace before
 * a CUDA context exists. 0 for bad sizes. */
size_t pod_cg_gram_workspace_for(int n, int p, int q, int sms);

/* G = X^T Y for device X (n-by-p) and Y (n-by-q), column-major; G device row-major p-by-q.
 * This is the snapshot Gram S^T S (Algorithm 4 step 1) and the reduced matrix W^T (A W)
 * (Algorithm 2 step 1). p, q <= 65. work: device, at least pod_cg_gram_workspace(n,p,q)
 * bytes, caller-owned scratch (contents on return are unspecified). */
pod_cg_status pod_cg_gram(int n, const double* X, int p, const double* Y, int q, double* G,
                          void* work, size_t work_bytes, void* cuda_stream);

/* Bytes of device workspace pod_cg_gram_tc needs for an n-row, p-by-q product (the Gram
 * of Algorithm 2 step 1). */
size_t pod_cg_gram_tc_workspace(int n, int p, int q);

/* G = X^T [Y, e] on the tensor cores: the reduced matrix of stage one (Algorithm 2 step 1,
 * W^T (A W) with the extra column W^T b) for X (n-by-p) and Y (n-by-qy), column-major with
 * leading dimension n, of element type FP32 (elem_bytes 4) or FP64 (elem_bytes 8), and an
 * optional FP64 column e (NULL for none); q = qy + (e != NULL); 1 <= p <= 64, 0 <= qy <= 64.
 * G is device row-major p-by-q (leading dimension q), FP64. Every value is rounded to FP32
 * and split exactly into three bf16 parts; the bf16 part products (at least the seven
 * with weight above 2^-24) accumulate in FP32 in tensor memory over 128-row windows,
 * Kahan-compensated in FP32 across windows and summed in FP64 across the GPU. The result
 * is deterministic; its error is that of an FP32-rounded input (about 2^-24 relative per
 * entry of X and Y) plus FP32 accumulation within a window. X, Y and e must start on
 * 16-byte boundaries and n * elem_bytes be a multiple of 16 (TMA); otherwise ERR_ARG.
 * work: device, at least pod_cg_gram_tc_workspace(n, p, q) bytes. Stream-ordered; a device
 * wait that expires (not expected) leaves NaN in G. */
pod_cg_status pod_cg_gram_tc(int n, int elem_bytes, const void* X, int p, const void* Y, int qy,
                             const double* e, double* G, void* work, size_t work_bytes, void* cuda_stream);

/* Test support with no counterpart in the paper: exercise the failure path of the bounded
 * device waits without a GPU fault. While bit 1 (the tensor-core Gram, pod_cg_gram_tc and
 * use_tc_gram solves) or bit 2 (the FP32 update and direction passes staged by the TMA engine,
 * proj_form = 1) is set in `mask`, those kernels issue no copies and every wait of theirs
 * gives up after `cycles` SM clocks (1e3 .. 4e9), so each runs its timeout path with nothing
 * in flight; while bit 4 (the persistent FP32 loop's grid barrier) is set, the last CTA to
 * arrive at a barrier does not release it and every wait gives up after about `cycles`
 * nanoseconds. A solve then ends with ERR_TIMEOUT (the handle stays usable) and
 * pod_cg_gram_tc leaves NaN in G. mask = 0 restores normal operation.
 * Applies to the current device, from the next launch on, captured graphs included; meant
 * for tests of the failure path only. Errors: ERR_ARG, ERR_CUDA. */
pod_cg_status pod_cg_debug_wait_timeout(int mask, long long cycles);

/* Allocation-free G = X^T Y (no counterpart in the paper): a deployment variant
 * of pod_cg_gram with the same arguments minus the workspace, and the same result bit for
 * bit. It is for callers that cannot allocate device memory at the point of use:
 * latency-bound loops where cudaMalloc/cudaFree may synchronise the whole device, and host
 * applications that hand out all device memory themselves under a fixed budget. The
 * scratch is a fixed 512 KiB array compiled into the library (held on every GPU that loads
 * the library until exit); this call allocates nothing. p, q <= 65; a product whose scratch
 * would exceed the array (possible only on a GPU with far more than 152 SMs) is rejected
 * with ERR_ARG and a message naming both sizes. cuda_stream (NULL = legacy default stream)
 * must belong to the current device (else ERR_ARG). The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current and keeps it
 * for the process; make that first call before any stream capture. After cudaDeviceReset
 * on a device the kept address is stale, so this entry point must not be called on that
 * device again in the same process. Every call shares the one array: calls that may overlap
 * on the GPU (different streams, or different host threads) race on it and must be
 * serialised by the caller. Each call overwrites all the scratch it reads, so no clearing
 * is needed. */
pod_cg_status pod_cg_gram_noalloc(int n, const double* X, int p, const double* Y, int q, double* G,
                                  void* cuda_stream);

/* POD by Algorithm 4 (identity metric, unit weights) of the device snapshot block S
 * (n-by-s, column-major, s <= 64): symmetric Jacobi eigensolve of S^T S, eigenvalues in
 * decreasing order, w = smallest index within the numerical rank whose energy fraction
 * reaches `energy`, capped at w_max; W_out (device, n-by-w_max room) = S V_w Sigma_w^{-1};
 * sigma2_out (device, s) = all eigenvalues; w_out (host). work as for pod_cg_gram with
 * p = q = s. */
pod_cg_status pod_cg_pod(int n, int s, const double* S, double energy, double rank_tol,
                         int w_max, double* W_out, double* sigma2_out, int* w_out,
                         void* work, size_t work_bytes, void* cuda_stream);

/* ------------------------------------------- many independent sequences in one launch */

typedef struct pod_cg_batch_t pod_cg_batch_t;

/* One sequence of a batch (device arrays, borrowed for the batch handle's lifetime): p
 * systems sharing one CSR pattern of order n; val holds the p value arrays back to back
 * (system j at j*nnz), b the p right-hand sides (j*n), x receives the p solutions. */
typedef struct {
    int            n;
    int64_t        nnz;
    int            p;
    int            w_max;     /* POD basis cap, 1..32 */
    int            s_max;     /* snapshot window, 1..16 */
    double         tol;       /* relative residual target, Eq. (sequenceInexact) */
    double         energy;    /* POD energy criterion (Algorithm 4) */
    const int32_t* row_ptr;
    const int32_t* col;
    const double*  val;
    const double*  b;
    double*        x;
} pod_cg_batch_seq;

typedef struct {
    int    status;          /* pod_cg_status of this system */
    int    iters;           /* FP32 inner CG iterations, all refinement steps */
    int    refinements;     /* FP64 refinement steps */
    int    w;               /* POD basis dimension used */
    double final_relres;    /* FP64 ||b - A x||/||b|| at exit */
    double stage1_relres;   /* after stage one */
} pod_cg_batch_sysstat;

/* Prepare a batch of nseq independent sequences (the problem of Section 2, many at once)
 * solved by one persistent launch captured in a CUDA graph: each worker (a thread-block
 * cluster) takes whole sequences, longest estimated work first, and runs the recycled-
 * solution form of the overall algorithm (Section 4.4) on each: POD of the previous
 * solutions (Algorithm 4), stage one (Algorithm 2), FP32 augmented PCG (Algorithm 1)
 * inside FP64 refinement. cfg supplies k_max, max_refine, inner_tol, rank_tol (NULL =
 * defaults). cluster: CTAs per worker, 1, 2, 4 or 8, or 0 to autotune (each candidate
 * 2, 4, 8 runs the whole batch once; the fastest is kept; then the inner loop's tiles are
 * tuned per size class, pod_cg_batch_tiles). The handle owns the workspace.
 * Errors: ERR_ARG (a bad sequence is named in the message), ERR_OOM, ERR_CUDA. */
pod_cg_status pod_cg_batch_create(const pod_cg_batch_seq* seqs /* host, nseq */, int nseq,
                                  const pod_cg_config* cfg, int cluster, void* cuda_stream,
                                  pod_cg_batch_t** out);

/* Solve every system of every sequence (one graph launch; synchronises) by the method of
 * pod_cg_batch_create (Section 4.4 per sequence). stats (host,
 * may be NULL) receives one entry per system, sequences in the order given and systems
 * in order within each; ms (host, may be NULL) the device time of the launch. Returns
 * the first non-OK system status, if any. */
pod_cg_status pod_cg_batch_solve(pod_cg_batch_t* h, pod_cg_batch_sysstat* stats, float* ms);

/* Chosen cluster size, number of concurrent workers and the autotuner's timings (ms of
 * the whole batch for cluster 2, 4, 8; 0 when not tuned, -1 when not schedulable).
 * Measurement support, no counterpart in the paper; so are the two calls after it. */
pod_cg_status pod_cg_batch_info(const pod_cg_batch_t* h, int* cluster, int* workers, float* tune_ms3);
const char* pod_cg_batch_last_error(const pod_cg_batch_t* h);
pod_cg_status pod_cg_batch_destroy(pod_cg_batch_t* h);

/* Tile autotuner record of a batch created with cluster = 0 (no counterpart in the paper):
 * per size class (n < 16,384; < 65,536; larger), the lanes per CSR row of the inner CG
 * product (lanes3) and the rows per thread of the update and direction passes (rows3: 1, or
 * 4 as float4 for sequences with n a multiple of 4) chosen by running the whole batch once
 * per candidate (lanes, rows) = (1, 1), (1, 4), (2, 4), (4, 4), each sequence timing its own
 * solve on the device; ms12 (3 x 4) the summed device time of each class per candidate. All
 * pointers host, each may be NULL. Before tuning, or with a forced cluster size: 1 and 1. */
pod_cg_status pod_cg_batch_tiles(const pod_cg_batch_t* h, int* lanes3, int* rows3, float* ms12);

/* Set the inner loop's tiles per size class instead of the autotuner's choice
 * (no counterpart in the paper): lanes3[3] in {1, 2, 4, 8}, rows3[3] in {1, 4} (4 applies to
 * sequences with n a multiple of 4; others use 1). Host arrays. Takes effect from the next
 * pod_cg_batch_solve. Errors: ERR_ARG, ERR_CUDA. */
pod_cg_status pod_cg_batch_set_tiles(pod_cg_batch_t* h, const int* lanes3, const int* rows3);

/* --------------------------------------- differentiation through a sequence of solves */

/* Values of the cell-centred finite-volume diffusion operator A(theta) + diag(extra) on an
 * mx x my x mz grid (mz = 1: five-point 2D), k = exp(theta) per cell, interior faces with
 * the harmonic-mean conductance 2 k_a k_b/(k_a + k_b), Dirichlet boundary faces with 2 k_a.
 * This is the operator whose parameters the adjoint gradient differentiates (the
 * differentiation workload of the sequence problem, Section 2). Cells are numbered x
 * fastest; row i of the CSR pattern (row_ptr, device, n+1) lists the z-1, y-1, x-1
 * neighbours, the cell itself, then x+1, y+1, z+1 (absent ones omitted); val_out (device,
 * nnz) receives the values in that order. theta, extra_diag (nullable): device, length n. */
pod_cg_status pod_cg_diffusion_assemble(int mx, int my, int mz, const double* theta, const double* extra_diag,
                                        const int32_t* row_ptr, double* val_out, void* cuda_stream);

/* Accumulate grad -= sum_j lambda_j^T (dA/dtheta) x_j for nsys systems (the adjoint
 * gradient of a loss over the sequence of Section 2; the paper has no such step) of the operator
 * above: for each cell c, the sum over its faces of dk_f/dtheta_c (lambda_c - lambda_m)
 * (x_c - x_m) with dk_f/dtheta_c = k_f k_m/(k_c + k_m), plus 2 k_c lambda_c x_c per
 * boundary face. With lambda_j the adjoint solutions (pod_cg_solve_adjoint) of a loss
 * L(x_1..x_p), this is dL/dtheta (A_j symmetric). lambdas and xs: device, nsys x n
 * row-major (system j at offset j*n); theta, grad: device, length n (grad accumulated).
 * One pass over all checkpoints. Errors: ERR_ARG, ERR_CUDA. */
pod_cg_status pod_cg_diffusion_theta_grad(int mx, int my, int mz, const double* theta, int nsys,
                                          const double* lambdas, const double* xs, double* grad,
                                          void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* POD_CG_H */
