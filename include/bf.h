/*
 * bf.h -- C ABI of the GB300 (sm_103a) Chebyshev-interpolation butterfly.
 *
 * The operator (Poulson, Demanet, Maxwell, Ying, "A Parallel Butterfly
 * Algorithm", Section 1, Eq. 1 and Eq. "phase"):
 *
 *     f(x_i) ~= sum_j exp(2 pi i Phi(x_i, y_j)) g(y_j),   i, j = 0 .. N^d - 1,
 *
 * applied by the butterfly of Algorithm 1 with the analytic tensor-product
 * Chebyshev interpolation of Section 1.4 (column space below the switch level
 * m, an r x r switch at level m, row space above it), r = q^d.
 *
 * Points.  Targets x_i and sources y_j sit on uniform grids, one per leaf box:
 * with the row-major multi-index (i_0, ..., i_{d-1}) of flat index i (last
 * index fastest),  x_k = x_lo[k] + (i_k + tgt_off) * x_w[k] / N  and likewise
 * y_k = y_lo[k] + (j_k + src_off) * y_w[k] / N.
 *
 * Data.  g and f are contiguous arrays of nrhs x N^d complex numbers
 * (interleaved real, imaginary; right-hand side slowest, then row-major
 * points).  The element type is complex128 (two doubles) for BF_PREC_FP64 and
 * complex64 (two floats) otherwise.  Device pointers must be 16-byte aligned.
 *
 * Streams.  Every apply is asynchronous on the given stream (a cudaStream_t
 * passed as void*; NULL = legacy default stream).  Device-side errors surface
 * at the caller's next synchronisation; launch errors are returned as
 * BF_ERR_CUDA and the CUDA error code is kept in the plan (bf_last_cuda_error).
 *
 * Threads.  A plan owns one workspace; applies on one plan must be ordered on
 * the same stream (or otherwise serialised).  Different plans are independent.
 * An apply (bf_apply, bf_apply_adjoint, bf_apply_host, bf_apply_pass) issued on a
 * stream other than that of the plan's previous apply, while that apply has not
 * completed, returns BF_ERR_UNSUPPORTED and queues nothing (the plan records an
 * event after each apply for this check).  Applies captured into a CUDA graph are not
 * checked: the order of the graph's launches is the caller's.  Persistent batches
 * (bf_batch_apply) use their plans' workspaces and are not checked either.
 *
 * Errors.  Invalid arguments return BF_ERR_INVALID_ARG and write nothing.
 */
#ifndef BF_GB300_H
#define BF_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_plan_s *bf_plan;

typedef enum {
    BF_OK = 0,
    BF_ERR_INVALID_ARG = 1,
    BF_ERR_UNSUPPORTED = 2,
    BF_ERR_NOMEM = 3,
    BF_ERR_CUDA = 4,
    BF_ERR_TIMEOUT = 5,
    BF_ERR_INTERNAL = 6
} bf_status;

/* Phase functions Phi (cycles; the kernel is exp(2 pi i Phi)), Section 3:
 *   BF_PHASE_DOT        Phi = s x.y                                  (Fourier, d = 2, 3)
 *   BF_PHASE_GENRADON   Phi = s (x.y + sqrt(sum_k a_k(x)^2 y_k^2)),  generalized Radon analogue;
 *                       d=2: a_0 = (2 + sin2pi x0 sin2pi x1)/3, a_1 = (2 + cos2pi x0 cos2pi x1)/3;
 *                       d=3: a_k = (2 + sin2pi x_k cos2pi x_{k+1 mod 3})/3
 *   BF_PHASE_HYPRADON   Phi = s x_0 sqrt(y_0^2 + y_1^2 x_1^2),       hyperbolic Radon (d = 2 only)
 *   BF_PHASE_SEPARABLE  Phi = s (sum_k sin 2pi(x_k + (k+1)/7) + sum_k y_k^2/(k+2)), a test phase
 *                       for which the butterfly is exact (s = 0 gives Phi = 0). */
typedef enum {
    BF_PHASE_DOT = 0,
    BF_PHASE_GENRADON = 1,
    BF_PHASE_HYPRADON = 2,
    BF_PHASE_SEPARABLE = 3
} bf_phase_kind;

/* Arithmetic of an apply.
 *   BF_PREC_FP64       complex128 weights, FP64 interpolation, FP64 phase, FP64 sincos.
 *   BF_PREC_MIXED      complex64 weights, FP32 interpolation and sincos; Phi is evaluated
 *                      and reduced mod 1 in double-float (pairs of FP32 numbers, >= 44
 *                      significant bits) before an FP32 polynomial sincos (error ~1e-7).
 *   BF_PREC_MIXED_SFU  as BF_PREC_MIXED but the sin/cos of the reduced phase come from the
 *                      special-function unit (error ~3.4e-7): faster, a few times the
 *                      FP32 weight rounding at the output.
 *   BF_PREC_BF16X3     as BF_PREC_MIXED, except that an apply with several right-hand
 *                      sides (nrhs >= 2; d = 2, q <= 5) runs the middle switch of Section
 *                      1.4 -- per pair the complex r x r phase matrix times the r x nrhs
 *                      weights -- as a GEMM on the tensor cores (tcgen05): every FP32
 *                      operand split into two BF16 parts, three BF16 products accumulated
 *                      in FP32 (relative error per product < 2^-16).  The switch is then
 *                      its own pass (bf_pass_info kind 2).  One right-hand side, d = 3 and
 *                      q > 5 run the BF_PREC_MIXED kernels and equal them bit for bit.  No
 *                      phase tables (BF_ERR_UNSUPPORTED), no persistent batches.
 *                      With bf_params.tc_levels = 1 the column merge levels below the
 *                      switch run on the tensor cores as well: per merge block the
 *                      modulated inputs of its 4 source children times the constant
 *                      Kronecker product of the child->parent interpolation matrices
 *                      (a real 128 x 32 x 128 GEMM per block, BF16x3, FP32 accumulation),
 *                      one level per pass (bf_pass_info kind 3).
 *   BF_PREC_TF32X3     as BF_PREC_BF16X3 (the switch on the tensor cores, the same
 *                      conditions and refusals), with every FP32 operand split into two
 *                      TF32 parts (tcgen05 kind::tf32) and three TF32 products accumulated
 *                      in FP32: relative error per product ~2^-22, so the apply keeps the
 *                      accuracy of BF_PREC_MIXED.  tc_levels has no effect. */
typedef enum {
    BF_PREC_FP64 = 0, BF_PREC_MIXED = 1, BF_PREC_MIXED_SFU = 2, BF_PREC_BF16X3 = 3, BF_PREC_TF32X3 = 4
} bf_precision;

typedef struct {
    double x_lo[3], x_w[3];   /* target domain: prod_k [x_lo[k], x_lo[k] + x_w[k]), x_w > 0  */
    double y_lo[3], y_w[3];   /* source domain, y_w > 0                                     */
    double phase_scale;       /* s in the phase formulas above                              */
    double tgt_off, src_off;  /* point offset inside its leaf box, in [0, 1)               */
    int32_t precision;        /* bf_precision                                               */
    int32_t switch_level;     /* m in [0, L-1]; -1 selects floor(L/2)                       */
    int32_t node_kind;        /* 0 Chebyshev-Lobatto cos(j pi/(q-1))/2, 1 first kind        */
    int32_t max_nrhs;         /* largest nrhs an apply may use (>= 1)                       */
    int32_t fuse_levels;      /* levels fused per kernel pass; 0 selects the default        */
    int32_t phase_tables;     /* 1: evaluate every phase factor once, at plan creation      */
    int32_t tc_levels;        /* BF_PREC_BF16X3: 1 also runs the column merge levels on the  */
                              /* tensor cores (below); 0 keeps them on the CUDA cores       */
    int32_t tc_cpasync;       /* BF16X3, TF32X3: 1 stages the switch's weights with 16-byte  */
                              /* cp.async copies instead of one tiled bulk copy (TMA) per   */
                              /* unit (same results; bf_plan_tc_info)                       */
    int32_t reserved[4];      /* must be zero                                               */
} bf_params;

/* Phase tables (phase_tables = 1; mixed precisions; d = 2 with q <= 5, or d = 3): the
 * precompute trade-off of Section 1.4.  bf_plan_create evaluates the phase factors of the
 * apply once, into device memory, and every bf_apply reads them instead of evaluating Phi.
 * Two forms:
 *  - max_nrhs = 1: the single-RHS kernels record the reduced phase (Phi minus an integer,
 *    one float) of every factor of the merges and of the switch -- (2^d + 1) r L + r^2
 *    floats per point (r^2 only where the switch is not factorised): 7.9 GB at d = 2,
 *    N = 1024, q = 5 and at d = 3, N = 64, q = 4.  The apply reads them with coalesced
 *    loads and evaluates only the sin/cos, so its results equal the evaluating apply bit
 *    for bit.
 *  - max_nrhs > 1 (d = 2 only; BF_ERR_UNSUPPORTED at d = 3): the multi-RHS kernels record
 *    the complex factors themselves (5 r L + r^2
 *    + 2 r + 1 complex64 numbers per point; 16.2 GB at N = 1024) and the apply, for any
 *    nrhs, fetches each CTA's table blocks with bulk copies (the TMA engine, cp.async.bulk)
 *    into two shared-memory buffers two blocks ahead of use; results equal the evaluating
 *    multi-RHS apply bit for bit.
 * BF_ERR_NOMEM if the table does not fit.  The schedule is fixed by the table
 * (bf_plan_autotune only times it).  bf_plan_table_info reports the table's bytes, the time
 * its construction took and (synchronising the device; timed_out may be NULL) whether a
 * wait for a copy ever gave up, or a kernel found a table layout it did not expect (results
 * undefined then).  The adjoint and persistent batches evaluate phases as without tables.
 * For BF_PREC_BF16X3 and BF_PREC_TF32X3 plans timed_out also reports a tensor-core completion wait that gave up
 * (2 s; the switch pass then stops and its outputs are undefined). */

/* Defaults for the problem classes of Section 3: X = [0,1)^d, Y = [-N/2, N/2)^d
 * (integer frequencies), s = 1, points at the lower corner of their leaf boxes,
 * BF_PREC_MIXED, m = floor(L/2), Lobatto nodes, max_nrhs = 1. */
bf_status bf_params_default(int d, int64_t N, bf_params *out);

/* Build a plan for d in {2,3} (d = 1 is not compiled), N = 2^L with 1 <= L and
 * N^d <= 2^30, q nodes per dimension (q in {2,3,4,5,6,8} for d = 2, q in {2,3,4}
 * for d = 3; other q return BF_ERR_UNSUPPORTED),
 * phase kind `phase` (HYPRADON needs d = 2).  The mixed precisions need |Phi| < 2^21
 * cycles over X x Y (bounded from the domain and the phase formula; BF_ERR_UNSUPPORTED
 * otherwise, use BF_PREC_FP64).  Allocates device workspace of
 * 2 * max_nrhs * N^d * q^d complex numbers plus small geometry tables on the
 * current CUDA device.  On success *out owns that memory until bf_destroy. */
bf_status bf_plan_create(int d, int64_t N, int q, bf_phase_kind phase, const bf_params *p,
                         bf_plan *out);

/* f = B g: g and f are device arrays of nrhs x N^d complex numbers (see Data).
 * 0 <= nrhs <= max_nrhs; nrhs = 0 does nothing.  g is read only; f is overwritten.
 * g and f must not overlap. */
bf_status bf_apply(bf_plan plan, const void *g_dev, void *f_dev, int nrhs, void *stream);

/* Sharded apply: one rank's part of f = B g when the source domain is split over G =
 * 2^shard_g ranks (1 <= shard_g <= d; shard_g = 0 is bf_apply), following the distribution of
 * the product space in Section 2 (Algorithms 2 and 4): rank shard_r owns the source boxes whose
 * top shard_g Morton bits (dimension 0 in the lowest bit) equal shard_r.  Every merge below the
 * last level combines the children of one source box, so those passes run the rank's pairs
 * only (1/G of the work); the last pass runs on every pair with the other ranks' weights read
 * as zero and writes f_r, this rank's contribution at every target.  Then f = sum over the
 * ranks of f_r (one all-reduce of nrhs x N^d values), equal to bf_apply's f up to FP32 (FP64)
 * rounding order.  g: all nrhs x N^d sources (only the rank's are read); f_r: nrhs x N^d.
 * Each rank holds its own plan (its own GPU).  BF_ERR_UNSUPPORTED for point-set plans and
 * plans with phase tables; BF_ERR_INVALID_ARG for shard_g > d or shard_r >= 2^shard_g. */
bf_status bf_apply_shard(bf_plan plan, const void *g_dev, void *f_dev, int nrhs, int shard_g, int shard_r,
                         void *stream);

/* g = B^H f, the exact conjugate transpose of the approximate operator applied by
 * bf_apply (every step conjugate-transposed, levels in reverse). */
bf_status bf_apply_adjoint(bf_plan plan, const void *f_dev, void *g_dev, int nrhs, void *stream);

/* Host-buffer variant of bf_apply: copies g_host to plan-owned device memory,
 * applies, copies f back to f_host, and synchronises the stream before returning.
 * Host buffers should be pinned for full copy bandwidth. */
bf_status bf_apply_host(bf_plan plan, const void *g_host, void *f_host, int nrhs, void *stream);

/* count independent problems, in order, on one stream: f[i] = B_i g[i] with nrhs[i]
 * right-hand sides.  Each plan's workspace is used by its own problem only. */
bf_status bf_apply_batched(const bf_plan *plans, const void *const *g_dev, void *const *f_dev,
                           const int *nrhs, int count, void *stream);

/* Persistent batches.  A batch fixes a list of independent problems (plans, d = 2,
 * mixed precision, all with the same q, phase kind and precision) and their numbers
 * of right-hand sides; bf_batch_apply then runs every pass of every problem in ONE
 * kernel launch.  The launch keeps as many CTAs as fit on the device; they take
 * work units (one CTA's tiles of one pass of one problem, for a block of up to 16
 * right-hand sides) from a queue ordered by pass index, and a unit of pass j waits
 * until the same problem's pass j-1 has finished (a counter in device memory).  The
 * butterflies are independent (the many transforms of Section 3.1), so the queue
 * fills the GPU across problems of uneven N.
 *   bf_batch_create: plans[i] with nrhs[i] (1..max_nrhs) right-hand sides, count in
 *     1..256, each plan at most once (its workspace serves one problem).  Allocates
 *     the job table and counters (a few KB).  BF_ERR_UNSUPPORTED if the plans do not
 *     qualify (use bf_apply_batched then).  The plans must outlive the batch.
 *   bf_batch_apply: f_dev[i] = B_i g_dev[i], asynchronous on the stream (device
 *     pointers, 16-byte aligned); one memset and one launch, capturable in a CUDA graph.
 *   bf_batch_status: synchronises the device and reports whether a wait of the last
 *     apply gave up (a dependency not met within 4 s; the unit and every later one are
 *     then skipped, their outputs undefined) -- the kernel never waits unboundedly.
 *   bf_batch_selftest_timeout: runs the batch with every wait's target one above what
 *     can be reached and a 20 ms limit, synchronises, and reports the flag (1 expected;
 *     outputs undefined); shows that a missed dependency ends in an error, not a hang.
 *   bf_batch_info: jobs, work units, CTAs of the launch, shared memory per CTA.
 *   bf_batch_wait_stats: synchronises the device; total time the CTAs of the last
 *     apply spent waiting for dependencies (summed over CTAs, ms) and the number of
 *     waits that did not find their dependency already met. */
typedef struct bf_batch_s *bf_batch;
bf_status bf_batch_create(const bf_plan *plans, const int *nrhs, int count, bf_batch *out);
bf_status bf_batch_apply(bf_batch batch, const void *const *g_dev, void *const *f_dev, void *stream);
bf_status bf_batch_status(bf_batch batch, int *timed_out);
bf_status bf_batch_selftest_timeout(bf_batch batch, const void *const *g_dev, void *const *f_dev, void *stream,
                                    int *timed_out);
bf_status bf_batch_info(bf_batch batch, int *jobs, int *units, int *grid, int64_t *smem_bytes);
bf_status bf_batch_wait_stats(bf_batch batch, double *wait_ms_total, int64_t *waits);
bf_status bf_batch_destroy(bf_batch batch);

/* Arbitrary point sets (Section 1.4: the interpolant of a pair can be evaluated anywhere
 * in its target box, so only the first and last steps see the points; sparse and
 * non-uniform sets are the paper's closing suggestion).  bf_plan_create_points builds a
 * plan as bf_plan_create does for the same (d, N, q, phase, params) -- N fixes the depth
 * of the box trees, N^d leaf boxes per domain -- with nsrc sources src[j*d + k] in the
 * source domain and ntgt targets tgt[i*d + k] in the target domain (host FP64 arrays,
 * copied; a point outside its domain joins the nearest leaf box; a leaf box may hold
 * any number of points, including none).  bf_apply then reads g as nrhs x nsrc values
 * and writes f as nrhs x ntgt values, both in the caller's point order (bf_apply_host
 * and bf_apply_batched likewise).  The per-point Lagrange values and phase factors are
 * computed in FP64 when the plan is made, the leaf boxes' node factors by an FP64 kernel;
 * the merges are the uniform-grid kernels.  bf_apply_adjoint, bf_plan_autotune,
 * bf_apply_pass, bf_pass_info, persistent batches and phase tables return
 * BF_ERR_UNSUPPORTED for such plans.  bf_plan_points_info: 1 and the point counts for
 * them, 0 and N^d, N^d for grid plans. */
bf_status bf_plan_create_points(int d, int64_t N, int q, bf_phase_kind phase, const bf_params *p, int64_t nsrc,
                                const double *src, int64_t ntgt, const double *tgt, bf_plan *out);
bf_status bf_plan_points_info(bf_plan plan, int *is_points, int64_t *nsrc, int64_t *ntgt);

/* Release the plan and its device memory.  bf_destroy(NULL) is a no-op.  The caller
 * must ensure no apply on this plan is still running. */
bf_status bf_destroy(bf_plan plan);

/* Static, human-readable name of a status code. */
const char *bf_status_string(bf_status s);

/* The CUDA error code behind the last BF_ERR_CUDA of this plan (0 if none). */
bf_status bf_last_cuda_error(bf_plan plan, int *cuda_err);

/* Introspection used by tests and the benchmark.
 *   bf_plan_info: d, N, q, switch level m, levels fused per pass, number of kernel
 *   launches per apply (per right-hand-side batch), bytes of device workspace. */
bf_status bf_plan_info(bf_plan plan, int *d, int64_t *N, int *q, int *m, int *fuse_levels,
                       int *launches_per_apply, int64_t *workspace_bytes);
bf_status bf_plan_table_info(bf_plan plan, int64_t *table_bytes, double *build_ms, int *timed_out);
/* Staging of the tensor-core switch: *tiled_copies = 1 when its weights arrive by one tiled
 * bulk copy (cp.async.bulk.tensor, a tensor map of each weight buffer built at plan
 * creation) per unit of two pairs, 0 when by cp.async copies (tc_cpasync = 1, or a driver
 * without the tensor-map encoder) or when the plan has no tensor-core switch. */
bf_status bf_plan_tc_info(bf_plan plan, int *tiled_copies);

/* Autotuner.  Times candidate tile schedules of the apply bf_apply runs for nrhs
 * right-hand sides on this device and keeps the fastest in the plan; the plan's current
 * schedule is timed first and replaced only by a candidate at least 1% faster, so
 * schedules of equal speed do not flip from run to run.  Single-RHS (and
 * FP64) passes: levels fused per pass (1 .. the compiled maximum) and whether the
 * short pass of a run of levels comes first or last.  Multi-RHS passes: fused levels
 * (1, 2), pairs per CTA (1 or 2 switch rounds), right-hand sides per scratch chunk
 * (1, 2, 4, 5, 8, 16),
 * and the short-pass position, among those that fit the shared memory of one CTA.
 * Each candidate runs one warm-up apply and reps timed applies (CUDA events) on
 * scratch buffers the call allocates and frees; synchronises the stream.  Results do
 * not depend on the schedule beyond FP32 rounding order.  best_ms (may be NULL)
 * receives the chosen schedule's time per apply. */
bf_status bf_plan_autotune(bf_plan plan, int nrhs, int reps, void *stream, double *best_ms);

/* Instrumentation.  An apply of nrhs right-hand sides is a fixed schedule of kernel
 * passes: the single-RHS passes for nrhs = 1 (and for FP64 plans), the multi-RHS
 * passes, which evaluate every phase factor once for up to 16 right-hand sides, for
 * nrhs >= 2.  bf_pass_count gives the number of passes of that schedule (= kernel
 * launches of one bf_apply).  bf_apply_pass runs pass i of the schedule only, with
 * the same arguments as bf_apply; running passes 0 .. count-1 in order on one stream
 * is exactly bf_apply.  Used to time individual kernels with events recorded between
 * passes.  bf_pass_info describes pass i of the schedule for nrhs: kind (0 column
 * pass with optional init/switch, 1 row pass with optional final, 2 the tensor-core
 * switch of BF_PREC_BF16X3 or BF_PREC_TF32X3 at level l0 with k = 0), first level l0,
 * number of fused levels k, flags (1 init, 2 switch, 4 final).  nrhs must lie in
 * 1..max_nrhs, i in 0..count-1 (else BF_ERR_INVALID_ARG). */
bf_status bf_pass_count(bf_plan plan, int nrhs, int *count);
bf_status bf_apply_pass(bf_plan plan, int i, const void *g_dev, void *f_dev, int nrhs, void *stream);
bf_status bf_pass_info(bf_plan plan, int nrhs, int i, int *kind, int *l0, int *k, int *flags);

/* Self-checks of the mixed-precision arithmetic on the current device (they
 * allocate and free a few bytes of device memory and synchronise).
 *   bf_selfcheck_sincos: largest |error| of the FP32 sin/cos of 2 pi f used by the
 *     mixed path, against CUDA's FP64 sincospi, over n evenly spaced f in [-1, 1).
 *   bf_selfcheck_phase: largest |error|, in cycles and modulo 1, of the mixed
 *     path's double-float Phi against FP64 arithmetic on the same table features,
 *     over n pseudo-random (target node, source node) pairs of a BF_PREC_MIXED plan
 *     (BF_ERR_INVALID_ARG for an FP64 plan). */
bf_status bf_selfcheck_sincos(int n, double *max_abs_err);
/* Measured FMA rate of the current device in TFLOP/s (an FMA counts 2): fp64 = 0 for
 * FP32, 1 for FP64, 2 for FP32 in packed pairs (one instruction, two FMAs).  Independent
 * dependent-FMA chains on every SM, timed with events; the context for the FP32-issue
 * roofline and for evaluating phases in double-float. */
bf_status bf_measure_fma_rate(int fp64, double *tflops);
/* Phase-evaluation rate of a mixed-precision d = 2 plan, in 10^9 phase factors per second:
 * a compute-only kernel evaluates e^{2 pi i Phi} for (target node, source node) pairs of
 * the plan's tables held in registers, one at a time (paired = 0) or two per float2
 * (paired = 1).  The practical ceiling of the phase work (Section 1.4: every translation
 * and the switch are dominated by these evaluations).  BF_ERR_INVALID_ARG for FP64 or
 * d = 3 plans. */
bf_status bf_measure_phase_rate(bf_plan plan, int paired, double *gphases_per_s);
bf_status bf_selfcheck_phase(bf_plan plan, int n, double *max_err_cycles);
/* Self-check of the tensor-core GEMM blocks that BF_PREC_BF16X3 uses (operand layout in
 * shared memory, descriptors, accumulator in tensor memory): one CTA computes a
 * 128 x 32 x 64 product D = A B^T of fixed operands and the host compares it with the FP64
 * product.  split = 0: small-integer operands, one BF16 product per K step (every product
 * and sum exact: max_rel_err must be 0); split = 1: values in [-1, 1) through the BF16x3
 * split (max_rel_err ~1e-5).  max_rel_err = max |D - D_ref| / max |D_ref|; timed_out = 1
 * if the completion wait (2 s) gave up.  Allocates and frees a few KB, synchronises. */
bf_status bf_selfcheck_umma(int split, double *max_rel_err, int *timed_out);
/* The same for the TF32 blocks of BF_PREC_TF32X3 (kind::tf32, 32-bit operands, K = 32):
 * split = 0 small integers (exact: max_rel_err 0), split = 1 the TF32x3 split of values in
 * [-1, 1) (max_rel_err ~1e-7). */
bf_status bf_selfcheck_umma_tf32(int split, double *max_rel_err, int *timed_out);

/* Forward apply that allocates no device memory.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc themselves or
 * let a library do it -- for example a host application that hands the GPU to
 * a fixed memory pool and forbids allocations after start-up, or code running
 * where an allocation could block or fail mid-stream.  Arguments are those of
 * bf_plan_create followed by those of bf_apply.  It launches the passes of the
 * default schedule of a plan built with the same arguments (before any
 * bf_plan_autotune), with the single-RHS kernels for every nrhs; for nrhs = 1 the
 * result equals that plan's bf_apply up to the last bits of the geometry tables
 * (they are built on the device here), for nrhs >= 2 (where bf_apply runs the
 * multi-RHS kernels) up to FP32 rounding order.  BF_PREC_BF16X3 and BF_PREC_TF32X3 are not accepted.
 *
 * Scratch.  The geometry tables and the two weight buffers live in one static
 * device array of BF_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads the
 * library holds until the process exits.  A problem needs
 *     48 * d * (2^(L+1) - 1) * (q + 2)  +  2 * nrhs * N^d * q^d * c  bytes
 * (c = 16 for BF_PREC_FP64, 8 otherwise; plus up to 256 bytes of alignment per
 * table); larger problems return BF_ERR_INVALID_ARG before any work is queued.
 * For d = 2, q = 5 and one right-hand side this admits N <= 128 in either
 * precision; for d = 3, q = 4 it admits N <= 16.  Nothing is read from the array before this call has written
 * it, so no clearing is needed, but every call uses the same array: calls that
 * overlap on the GPU (different streams, or different host threads without
 * ordering) race on it and must be serialised by the caller.
 *
 * Set-up.  The first call on each device (with that device current) looks up
 * the array's device address with cudaGetSymbolAddress; make that first call
 * before any stream capture begins.  The address is kept for the life of the
 * process: it does not survive cudaDeviceReset (or anything else that destroys
 * the device's primary context), so do not reset a device between calls.
 * Asynchronous on `stream` like bf_apply. */
#define BF_NOALLOC_SCRATCH_BYTES (16u << 20)
bf_status bf_apply_noalloc(int d, int64_t N, int q, bf_phase_kind phase, const bf_params *p,
                           const void *g_dev, void *f_dev, int nrhs, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BF_GB300_H */
