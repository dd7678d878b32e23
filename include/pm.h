/*
 * pm.h -- C ABI of the GB300 performance-modeling library (libpm.so).
 *
 * The library implements the data-parallel hot path of the cross-machine
 * black-box GPU performance-modeling method of Stevens & Kloeckner
 * (arXiv 1904.09538): exact kernel feature counts, device-timed measurement
 * kernels, and calibration / evaluation of user-written time models.
 *
 * Conventions (all entry points):
 *   - Every function returns a pm_status; PM_OK == 0.  On failure a message
 *     is stored in a thread-local buffer returned by pm_last_error().
 *   - Output arrays are owned by the caller.  Handles (pm_model) are owned by
 *     the library and released with the matching destroy call.
 *   - Nothing aborts or exits; CUDA errors become PM_ECUDA plus a message.
 *   - "device pointer" means memory of the current CUDA device (cudaMalloc or
 *     a PyTorch CUDA tensor); "host pointer" means ordinary or pinned host
 *     memory.  A stream argument is a cudaStream_t (NULL = legacy default).
 *   - Sizes are element counts unless stated.
 */
#ifndef PM_H
#define PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PM_OK = 0,
    PM_EINVAL = -1,           /* invalid argument (message says which) */
    PM_ENOMEM = -2,           /* allocation failed */
    PM_ECUDA = -3,            /* CUDA runtime error */
    PM_ENOTCONV = -4,         /* fit reached max_iter; best iterate written */
    PM_ERANK = -5,            /* rank-deficient design; minimum-norm solution written */
    PM_ETIMEOUT = -6,         /* a bounded device wait gave up */
    PM_EUNKNOWN_KERNEL = -7,  /* no kernel of that name / id */
    PM_EPARSE = -8,           /* model expression or feature name does not parse */
    PM_ECAP = -9              /* output array too small; *n_out holds the size needed */
} pm_status;

/* Kernel parameter, e.g. {"n", 1024} -- the size parameters of a kernel's
 * loop domain (Section "Predicting Cost": a dictionary of problem sizes).
 * Integer parameters must hold integral values. */
typedef struct {
    const char *key;
    double value;
} pm_param;

/* ---------------------------------------------------------------- kernels */

/* Kernel registry.  Names: the calibration suite "stream", "fma", "smem",
 * "barrier", "overlap", "empty" (Section "Measurement Kernel Design"), and
 * "smem2d" (local accesses with a lid(1) stride T = 16 or 18 in T x T
 * work-groups, parameters R, T, G: the local-memory pattern of the stencil
 * tiles, for models that split local-memory features by stride);
 * matmul "mm_pf", "mm_nopf" and the work-removed twins "mm_pf_a", "mm_pf_b",
 * "mm_nopf_a", "mm_nopf_b" (Section "Matrix Multiplication", Algorithm 3);
 * DG "dg_nopf", "dg_upf", "dg_dmpf", "dg_dmpft" and twins "dg_nopf_u",
 * "dg_nopf_dm", "dg_dmpf_u", "dg_dmpf_dm", "dg_res", "dg_upf_u", "dg_dmpft_u",
 * "dg_dmpft_res" (Section "DG"; dg_upf needs L0 == L1; dg_dmpft and its twins
 * read u as uT[j, k] (Np x Nel) and write res as resT[m, i, k]); stencil
 * "fd_tile" (16x16 work-group, 14x14 interior), "fd_tile18" (18x18
 * work-group, 16x16 interior), "fd_direct" and twins "fd_tile_u",
 * "fd_tile_res", "fd_tile18_u", "fd_tile18_res", "fd_direct_u",
 * "fd_direct_res" (Section "Finite Differences"); autotuning spaces (the paper's use case
 * of ranking equivalent variants, Section "Assumptions and Limitations"):
 * "mm_simt" (register-tiled fp32 matmul, parameters n, BM, BN, BK); the
 * added BF16 tensor-core matmul "mm_tc" (C = A Bt^T, bf16 in, fp32 out,
 * tcgen05/TMEM/TMA, parameter n, a multiple of 256, and pipe: 0 = 4-stage
 * ring with one CTA per SM, 1 (default) = 2-stage ring with two CTAs per SM,
 * 2 = persistent (one CTA per SM walking the tiles, 4-stage ring, two TMEM
 * accumulators so one tile's epilogue overlaps the next tile's main loop);
 * the counts describe the decomposition into 128 x 256 tiles and do not
 * depend on pipe) and its 256 x 256-tile form "mm_tc256" (parameter n, a
 * multiple of 256: 256-thread work-groups, two 128-row accumulators in 512
 * TMEM columns sharing each Bt box, 3-stage ring, one CTA per SM); the DG
 * tile form "dg_tile" (parameters Np <= 96 and Nel, a multiple of 4; buffers
 * diff_mat, u, res as for dg_nopf; 16 x 16 work-groups of 128 elements, D
 * staged transposed in shared memory, u tiles by one bulk TMA copy); its
 * tensor-core form "dg_tc" (parameters Np, one of the tetrahedral node
 * counts 4, 10, 20, 35, 56, 84, Nel a multiple of 4 (<= 2^24), A the
 * place of the u operand, 0 = shared memory, 1 = tensor memory, -1
 * (default) = 1 for Np = 35 and 84 (20 < Np <= 40 or Np > 64) else 0, and
 * P the persistent CTAs per m-group, 0 (default) = min(ceil(Nel / 128),
 * 152 R / G), one wave of a GB300's 152 SMs with R = 2 CTAs per SM for
 * A = 0 and Np <= 20, else 1, and G = 1 m-group (the three m in one CTA)
 * for Np <= 40 and, with A = 0, for Np <= 64, else 3; the grid is (G, P);
 * buffers as for dg_nopf): the product of each
 * 128-element tile with the stacked operator rows on tcgen05.mma kind::tf32,
 * every operand split into a TF32 head and its FP32 remainder and three
 * passes (head x head, head x remainder, remainder x head) accumulated in
 * FP32 in tensor memory, so the result carries FP32-level accuracy; u tiles
 * by TMA when Np % 4 == 0, the res blocks by bulk copies; the TMA-staged
 * stencil tile family "fd_block" (parameters n, BX, BY, c0, c1, V = 4 or 8
 * outputs per work-item; input u of (n + 2) rows with row pitch n + 4).
 * Returns PM_EUNKNOWN_KERNEL for other names. */
pm_status pm_kernel_lookup(const char *name, int32_t *kernel);
pm_status pm_kernel_count(int32_t *n);
/* Library-owned, static string. */
pm_status pm_kernel_name(int32_t kernel, const char **name);

typedef enum { PM_F32 = 0, PM_F64 = 1, PM_BF16 = 2 } pm_dtype;
typedef enum { PM_IN = 0, PM_OUT = 1 } pm_role;

typedef struct {
    char name[32];      /* "in0".."in3", "out", "seed", "a", "b", "c", "x", "diff_mat", "u", "res", "tgt_dest" */
    int32_t dtype;      /* pm_dtype of one element */
    int32_t role;       /* pm_role */
    uint64_t elems;     /* element count (scalar elements, not vectors) */
} pm_buffer;

/* Buffers kernel `kernel` needs for these parameters, in launch order.
 * PM_ECAP with *n_out set when cap is too small. */
pm_status pm_kernel_buffers(int32_t kernel, const pm_param *p, size_t np,
                            pm_buffer *out, size_t cap, size_t *n_out);

/* ---------------------------------------------------------------- counts */

typedef enum { PM_GRAN_WI = 0, PM_GRAN_SG = 1, PM_GRAN_WG = 2, PM_GRAN_K = 3 } pm_gran;
typedef enum { PM_FEAT_OP = 0, PM_FEAT_MEM = 1, PM_FEAT_SYNC = 2, PM_FEAT_GROUPS = 3, PM_FEAT_LAUNCH = 4 } pm_feat_kind;

/* One exact feature of a kernel instance (Section "Kernel Features").
 *   OP:     name f_op_<dtype>_<add|mul|madd>; count per sub-group (SG),
 *           count_wi per work-item.
 *   MEM:    one memory access site with its pattern (Section "Data Motion
 *           Features"): tag, memory type, data type, direction, local and
 *           group strides along each thread axis (units of the data type),
 *           the stride along the innermost enclosing sequential loop
 *           (Table "ab_pattern"), and accesses/footprint = AFR (Algorithm 2,
 *           per access site).  count is at the site's granularity: global
 *           per work-item unless lid(0) stride is 0 ("uniform"), which is per
 *           sub-group like local memory (Section "Gathering Kernel
 *           Statistics").
 *   SYNC:   f_sync_barrier_local, barriers met by one work-item.
 *   GROUPS: f_thread_groups, the work-group count.
 *   LAUNCH: f_sync_kernel_launch = 1.
 * The sub-group size is 32. */
typedef struct {
    char name[192];        /* canonical feature name */
    int32_t kind;          /* pm_feat_kind */
    int32_t gran;          /* pm_gran of `count` */
    uint64_t count;        /* value at its granularity */
    uint64_t count_wi;     /* OP/MEM: work-item level count */
    uint64_t count_sg;     /* OP/MEM: sub-group level count */
    /* MEM only */
    char tag[32];
    char dtype[16];        /* "float32", "float64", "float32x4", "float64x2" (OP: dtype too) */
    char op[8];            /* OP only: "add", "mul", "madd" */
    int32_t mem;           /* 0 global, 1 local */
    int32_t dir;           /* 0 load, 1 store */
    int32_t dsize;         /* bytes per access */
    int32_t nl, ng;        /* number of meaningful lstride / gstride entries */
    int64_t lstride[3];
    int64_t gstride[3];
    int64_t loop_stride;
    uint64_t accesses;     /* AFR numerator (work-item accesses) */
    uint64_t footprint;    /* AFR denominator (distinct elements touched) */
} pm_feature;

/* Exact integer features of kernel `kernel` at parameters p (Algorithm 1,
 * closed forms per kernel).  Writes up to cap records; *n_out = number of
 * records (PM_ECAP if cap < *n_out).  Pure host computation. */
pm_status pm_counts(int32_t kernel, const pm_param *p, size_t np,
                    pm_feature *out, size_t cap, size_t *n_out);

/* Size parameter over which pm_counts_desc extrapolates: counts are
 * quasi-polynomials in it of the given period and degree bound.  period 0
 * and degree -1 ask the library to derive them from the description (see
 * pm_counts_desc_interp). */
typedef struct {
    const char *name;
    int32_t period;
    int32_t degree;
} pm_interp;

/* Exact features of a kernel given as a text description of its affine loop
 * nest instead of a registry name (Algorithm 1 and Algorithm 2 over a
 * user's kernel; the paper counts such kernels with a polyhedral library,
 * Section "Gathering Kernel Statistics").  Format, one item per line, '#'
 * starts a comment:
 *   params <name>...                      size parameters
 *   grid <e0> [<e1> [<e2>]]               work-group counts per axis
 *   group <e0> [<e1> [<e2>]]              work-items per group per axis
 *   stmt | barrier                        a statement / a local barrier, then:
 *     loop <var> <lo> <hi>                loop (hi exclusive), outermost first
 *     guard <expr>                        executes only where expr >= 0
 *     ops <float32|float64|bfloat16> <add> <mul> <madd>
 *     access <tag> <global|local> <load|store> <dtype> <bytes> <index expr>
 * Expressions: integers, parameters, g0 g1 g2 l0 l1 l2 (group and local
 * ids), the statement's loop variables, + - * / (floor) % min(,) max(,) and
 * parentheses; index expressions must be affine in the ids and loop
 * variables.  Records and granularities are those of pm_counts; tags must be
 * unique (a model can name a tag only if it contains no '_').  With interp
 * (nullable), each listed parameter
 * is extrapolated exactly from degree + 3 enumerated sizes of its residue
 * class, the first at one period above the residue (PM_EINVAL if either of
 * the two extra samples contradicts the degree bound); without it every loop
 * point is enumerated (at most 2^31 statement instances).  Pure host
 * computation; *n_out and PM_ECAP as pm_counts. */
pm_status pm_counts_desc(const char *description, const pm_param *p, size_t np, const pm_interp *interp,
                         size_t ninterp, pm_feature *out, size_t cap, size_t *n_out);

/* Period and degree bound of the counts of a described kernel as
 * quasi-polynomials in the size parameter `param` (the other parameters at
 * their values in p; Section "Gathering Kernel Statistics": counts are
 * piecewise quasi-polynomials in the sizes).  Derived from the description:
 *   period: the lcm of the constant divisors and moduli (/ and %) applied to
 *     expressions that depend on param -- the sources of its periodicity;
 *   degree: over the statements, the larger of the degree of the number of
 *     loop points (grid extents plus, per loop, the larger degree of its
 *     bounds, which also bounds footprints, sub-group counts and barriers)
 *     and the degrees of the access index expressions (their strides); an
 *     index variable has the degree of its range, a product the sum of its
 *     factors' degrees.
 * PM_EINVAL where no bound follows: a work-group extent that depends on
 * param, a divisor or modulus that is not constant and depends on param, a
 * degree above 10 or a period above 2^24.  Pure host computation. */
pm_status pm_counts_desc_interp(const char *description, const char *param, const pm_param *p, size_t np,
                                int32_t *period, int32_t *degree);

/* Compiled resources and launch shape of one kernel instance, for an
 * autotuner's pruning step (the paper's use of a model as a heuristic that
 * narrows the variants worth timing, Section "Assumptions and Limitations"):
 * a variant that spills registers to local memory or cannot keep a CTA
 * resident is not worth timing. */
typedef struct {
    int32_t regs_per_thread;
    int32_t local_bytes_per_thread;  /* stack / register spill */
    int32_t static_smem_bytes;
    int32_t dynamic_smem_bytes;      /* of this launch */
    int32_t threads_per_block;       /* of this launch */
    int32_t max_threads_per_block;   /* of the compiled kernel */
    int32_t blocks_per_sm;           /* resident CTAs per SM at this launch shape (0: cannot run) */
    int32_t sm_count;
    uint64_t grid_blocks;
} pm_resources;

/* Fill *out for `kernel` at parameters p on the current device, without
 * launching it and without touching device memory.  Needs a CUDA device;
 * PM_ECUDA without one. */
pm_status pm_kernel_resources(int32_t kernel, const pm_param *p, size_t np, pm_resources *out);

/* ---------------------------------------------------------------- running */

/* Enqueue one launch of `kernel` on `stream`.  bufs: device pointers in the
 * order pm_kernel_buffers reports, each holding at least `elems` elements.
 * Extra kernel arguments (stencil c0, c1) come from p.  Asynchronous; the
 * launch configuration error (if any) is reported. */
pm_status pm_launch(int32_t kernel, const pm_param *p, size_t np,
                    void *const *bufs, size_t nbufs, void *stream);

typedef struct {
    int32_t warmup;          /* untimed launches first (default 2) */
    int32_t trials;          /* timed launches (default 60, Section "Other Features") */
    double outlier_factor;   /* drop trials > factor * median (default 5; <= 0 keeps all) */
    int32_t flush_l2;        /* 1: before every trial, overwrite a 256 MiB library-owned buffer (larger
                                than L2) outside the timed interval, so each trial starts cache-cold.
                                The buffer is allocated once per device on first use. (default 0) */
} pm_run_opts;

typedef struct {
    double mean_ms;          /* mean over kept trials -- the wall-time feature */
    double median_ms, min_ms, max_ms;
    int32_t n_trials, n_dropped;
} pm_timing;

/* Device-time `kernel` (the paper's wall-time feature, excluding host-device
 * transfer): warmup launches, then `trials` launches each bracketed by CUDA
 * events on `stream`.  trial_ms (nullable, caller-owned, >= trials floats)
 * receives every trial's time.  opts NULL = defaults.  Blocks until done. */
pm_status pm_run(int32_t kernel, const pm_param *p, size_t np,
                 void *const *bufs, size_t nbufs, const pm_run_opts *opts,
                 void *stream, float *trial_ms, pm_timing *out);

/* pm_run with HOST buffers: copies inputs host->device, runs as pm_run, and
 * copies outputs device->host, all on `stream`; device memory is allocated
 * with cudaMallocAsync and freed before returning.  The first call on a device
 * raises the release threshold of that device's default memory pool to the
 * maximum, so freed staging memory stays reserved for later calls (and for
 * any other cudaMallocAsync user of that pool) instead of being unmapped at
 * every synchronisation.  Pinned host buffers copy at the link rate; pageable
 * ones are staged by the driver.  *copy_ms (nullable) receives the total time
 * of the copies. */
pm_status pm_run_host(int32_t kernel, const pm_param *p, size_t np,
                      void *const *host_bufs, size_t nbufs, const pm_run_opts *opts,
                      void *stream, float *trial_ms, pm_timing *out, double *copy_ms);

/* One kernel instance of a host-buffer batch: parameters and host buffers
 * as for pm_run_host, except that an output buffer's host pointer may be
 * NULL: that output stays on the device (the kernel still writes it) and is
 * not copied back -- for calibrations, whose result is the timings.  Input
 * pointers must not be NULL. */
typedef struct {
    int32_t kernel;
    const pm_param *p;
    size_t np;
    void *const *host_bufs;
    size_t nbufs;
} pm_host_job;

/* pm_run_host over a list of kernel instances, pipelined over the two copy
 * directions of the host link: while job i's outputs travel device->host,
 * job i+1's inputs travel host->device (two internal copy streams).  Kernels
 * never overlap a copy, so each job's device timing is as in pm_run_host:
 * job i+1's launches wait for its inputs and for job i's output copy.  When
 * an output buffer of job i overlaps an input buffer of job i+1 in host
 * memory, that pair of copies is serialised instead.  Input buffers that
 * start at the same host address in several jobs are one shared region: it
 * is copied once, at the largest extent any reader reads (every kernel only
 * reads its inputs), and all shared regions are copied back to back at the
 * start of the batch, before the first job's kernels (on GB300 the host ->
 * device path runs copies issued back to back at its full rate, while a
 * copy issued after it has idled for a fraction of a second starts several
 * times slower).  A region that any host
 * output buffer of the batch overlaps is not shared (its host contents may
 * change during the batch); each of its readers copies it.  Device staging
 * is one allocation per batch from the default memory pool (see
 * pm_run_host): the shared regions, then two slots for the jobs' own
 * buffers used by consecutive jobs in turn (a job's input copies wait until
 * the job two before it has copied its outputs out of its slot), so every
 * shared region stays resident for the whole batch.  out: njobs timings;
 * copy_ms (nullable): the copies' own device time -- per job, from the
 * moment its input copies may start to their end, plus its output copies --
 * summed over the jobs (the time between jobs, host work included, is not
 * counted); on error the failing job's index is in the message and later
 * jobs are not run. */
pm_status pm_run_host_batch(const pm_host_job *jobs, size_t njobs, const pm_run_opts *opts, void *stream,
                            pm_timing *out, double *copy_ms);

/* The bytes pm_run_host_batch would copy for these jobs (host only, no GPU
 * work): host->device (shared regions once, at their largest extent) and
 * device->host (outputs with a non-NULL host pointer).  Either output
 * pointer may be NULL.  Same validation and errors as pm_run_host_batch. */
pm_status pm_run_host_batch_bytes(const pm_host_job *jobs, size_t njobs, uint64_t *h2d_bytes, uint64_t *d2h_bytes);

/* Unloaded load latency of the memory level that holds a buffer (the
 * latency in the Little's-law bound of a pattern with few bytes in flight
 * per work-item; not a paper feature).  buf: caller-owned device buffer of
 * `bytes` bytes (128-byte aligned, 256 bytes .. 512 GiB), overwritten with a
 * chain of line indices; one thread then follows `hops` links with L1-
 * bypassing loads, timed with CUDA events on `stream`.  *ns_per_hop: mean
 * time per dependent load -- HBM latency for a buffer much larger than L2,
 * L2 latency for a buffer well inside it.  Blocks until done. */
pm_status pm_probe_latency(void *buf, size_t bytes, int32_t hops, double *ns_per_hop, void *stream);

/* ---------------------------------------------------------------- models */

typedef struct pm_model pm_model;

/* Model = output feature + expression over features f_* and parameters p_*
 * (Section "Modeling Kernel Execution Time").  Grammar: + - * / unary -,
 * parentheses, numbers, tanh exp log sqrt; a name runs to whitespace or one
 * of + * / ( ) (a '-' glued to a name is part of it).  PM_EPARSE on error. */
pm_status pm_model_create(const char *out_feature, const char *expr, pm_model **m);
void pm_model_destroy(pm_model *m);
pm_status pm_model_info(const pm_model *m, size_t *n_features, size_t *n_params);
/* Library-owned strings valid until pm_model_destroy. */
pm_status pm_model_feature_name(const pm_model *m, size_t i, const char **name);
pm_status pm_model_param_name(const pm_model *m, size_t i, const char **name);
/* 1 if g is linear in the parameters (fit by linear least squares). */
pm_status pm_model_is_linear(const pm_model *m, int32_t *linear);

/* Feature assembly: value of each model feature on one kernel's feature
 * records -- the sum of the counts of all matching records (Section "Data
 * Motion Features": tag / memory type / data type / direction / stride and
 * AFR constraints such as lstrides:{0:1;1:>15}).  row_out has n_features
 * doubles.  PM_EPARSE if a model feature name does not parse. */
pm_status pm_feature_values(const pm_model *m, const pm_feature *feats, size_t nfeat, double *row_out);

typedef struct {
    int32_t max_iter;        /* LM iteration cap (default 200); 0: no iteration, a nonlinear
                                fit returns its start point with PM_ENOTCONV */
    double ftol;             /* stop when relative SSR decrease < ftol (default 1e-15) */
    double xtol;             /* stop when |dq| <= xtol (|q| + xtol) in scaled coordinates (default 1e-12) */
    int32_t use_p0;          /* 1: p_inout holds the start point; 0: library start point */
} pm_fit_opts;
/* The library start point (Section "Computing Model Parameters" leaves it
 * open): the linear least-squares fit of the model with every tanh(.)
 * replaced by 0 (each switch at 1/2); a coefficient that comes out <= 0
 * becomes 1e-3 * sum_k t_k / sum_k |h_ki| (h_i its column of that linear
 * design at the origin; for a column zero there, its column at the point
 * reached so far, and 1e-3 * max |p| if that is zero too); every
 * parameter absent from that design (p_edge) starts at 10 / median(t).  The
 * LM then damps by lambda * dmax_i on the diagonal of J^T J (dmax_i the
 * largest value met so far), lambda from 1e-3, /10 on an accepted step, x10
 * on a rejected one (at most 16 per iteration; 16 rejections end the fit).
 * A trial is accepted when its SSR is not larger, or when its predicted
 * decrease is below the SSR's noise floor (4e-13 sqrt(l SSR): float-float
 * residuals), where only the gradient can still direct the step.  The fit
 * stops when |dq| <= xtol (|q| + xtol); when such unverifiable steps have
 * become negligible (max |dq_i| <= 1e-9 max(max |q_i|, 1)) or four of them
 * came in a row; or when a measurable relative SSR decrease is below
 * ftol. */

typedef struct {
    int32_t status;          /* pm_status of this fit */
    int32_t iterations;
    int32_t rank;            /* numerical rank (linear fits) */
    int32_t linear;          /* 1 linear least squares, 0 Levenberg-Marquardt */
    double residual;         /* || 1 - g(p; f_k)/t_k ||_2 at the solution */
    double lambda;           /* final LM damping */
    double cond;             /* condition estimate of the unit-diagonal normal matrix J^T J at the
                                solution over the active parameters: (largest / smallest Cholesky
                                pivot)^2, a lower bound of its 2-norm condition number; the
                                eigenvalue ratio where the factorisation fails; +inf when rank-
                                deficient */
} pm_fit_report;

/* Calibrate one model (Section "Computing Model Parameters") on l rows:
 * X is l x n_features row-major (host, FP64 feature values), t the l output
 * values (host).  Minimises sum_k (1 - g(p; X_k)/t_k)^2 (relative error,
 * scale_features_by_output).  Linear-in-p models: column-scaled least
 * squares (normal equations in float-float with iterative refinement on the
 * GPU); otherwise Levenberg-Marquardt on the GPU (float-float residuals and
 * FP32 Jacobian on the FP32 pipes, J^T J and J^T r accumulated with exact
 * products and compensated sums, the damped normal equations solved in
 * float-float, damping and stopping decisions in FP64).
 * p_inout: n_params doubles (start point if opts->use_p0, result out).
 * Returns PM_ERANK (minimum-norm solution written) or PM_ENOTCONV (best
 * iterate written) where applicable. */
pm_status pm_fit(const pm_model *m, const double *X, const double *t, size_t l,
                 const pm_fit_opts *opts, double *p_inout, pm_fit_report *report);

/* Batched calibration (many models x measurement sets of uneven size in ONE
 * persistent kernel launch, one CTA per model, replayed from a CUDA graph).
 * A plan fixes the models and row counts; it owns device and pinned host
 * staging buffers (allocated at creation) and the captured graph.
 *   threads: CTA size of the fit kernel (64, 128, 256 or 512; 0 = 128).
 * pm_fit_plan_run: X_concat holds, model after model, rows[k] x
 * n_features(k) FP64 values (row-major); t_concat the outputs; p_inout_concat
 * n_params(k) values per model (start points if opts->use_p0); reports one
 * per model.  All host pointers.  Same numerics as pm_fit.  Per-model
 * statuses are in reports[k].status; the call returns PM_OK unless the
 * launch itself failed. */
typedef struct pm_fit_plan pm_fit_plan;
pm_status pm_fit_plan_create(const pm_model *const *models, size_t nmodels, const size_t *rows,
                             const pm_fit_opts *opts, int32_t threads, pm_fit_plan **plan);
pm_status pm_fit_plan_run(pm_fit_plan *plan, const double *X_concat, const double *t_concat,
                          double *p_inout_concat, pm_fit_report *reports, void *stream);
void pm_fit_plan_destroy(pm_fit_plan *plan);
/* One-shot convenience: create a plan, run it once, destroy it. */
pm_status pm_fit_batched(const pm_model *const *models, size_t nmodels, const double *X_concat,
                         const double *t_concat, const size_t *rows, const pm_fit_opts *opts,
                         double *p_inout_concat, pm_fit_report *reports, void *stream);

/* Allocation-free batched calibration.  The paper has no counterpart; this
 * entry point exists for callers that must not allocate GPU memory: a
 * process whose device memory is entirely reserved by another framework's
 * pooling allocator (a cudaMalloc there fails or evicts the pool's cache),
 * or a latency-critical loop that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree may cause.
 *
 * Same arguments, layout and results as pm_fit_batched (host arrays; CTA
 * size 128).  Instead of allocating, it stages the models' programs, the
 * data (FP64 and float-float copies), the parameters and the reports in one
 * static device array of PM_NOALLOC_SCRATCH_BYTES bytes that every GPU which
 * loads the library keeps until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine, and no host allocator either (the
 * job table is built in a static host array).
 *   - Requests whose staged size exceeds PM_NOALLOC_SCRATCH_BYTES, or with
 *     more than 256 models, fail with PM_EINVAL and a message giving the
 *     size needed; nothing is launched then.  A non-finite start point (with
 *     opts->use_p0), feature value or output fails with PM_EINVAL too.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     life of the process.  A cudaDeviceReset in this process invalidates
 *     that address: do not call this entry point after one.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; each call rewrites everything it reads.  Calls whose work
 *     overlapped on the GPU would race on the array, so the library
 *     serialises them: a process-wide lock is held from the first upload
 *     until the results are on the host.
 *   - Blocks: it synchronises `stream` before returning (the results are
 *     copied to host memory).  It must therefore not be called while
 *     `stream` is being captured into a CUDA graph. */
#define PM_NOALLOC_SCRATCH_BYTES (8u << 20)
pm_status pm_fit_batched_noalloc(const pm_model *const *models, size_t nmodels, const double *X_concat,
                                 const double *t_concat, const size_t *rows, const pm_fit_opts *opts,
                                 double *p_inout_concat, pm_fit_report *reports, void *stream);

/* Differentiation entry points (Section "Computing Model Parameters": the
 * model's derivatives with respect to its parameters, obtained here by
 * reverse-mode differentiation of the model program instead of symbolic
 * differentiation).  Device pointers; used by the PyTorch autograd.Function.
 *   X: l x n_features FP64 row-major, t: l FP64 (> 0), p: n_params FP64.
 * Per row the model program runs in float-float arithmetic on the FP32 pipes
 * (each FP64 input split into a hi + lo pair of floats, about 48 bits).
 *   pm_residual:  r_k = 1 - g(p; X_k) / t_k                        (r: l FP64)
 *   pm_residual_vjp: pbar_i = sum_k rbar_k dr_k/dp_i               (rbar: l FP64,
 *                 pbar: n_params FP64, overwritten; float-float reverse sweep and
 *                 products, compensated sums per CTA, combined across CTAs with
 *                 FP64 atomics, so the last bits may differ between runs)
 *   pm_jacobian:  J[k, i] = dr_k/dp_i = -dg/dp_i / t_k             (l x n_params FP32:
 *                 FP32 reverse sweep over the high parts; it steers LM steps)
 * All three are asynchronous on `stream`; l = 0 is a no-op (pbar zeroed).
 * PM_EINVAL for NULL pointers. */
pm_status pm_residual(const pm_model *m, const double *X, const double *t, size_t l, const double *p,
                      double *r, void *stream);
pm_status pm_residual_vjp(const pm_model *m, const double *X, const double *t, size_t l, const double *p,
                          const double *rbar, double *pbar, void *stream);
pm_status pm_jacobian(const pm_model *m, const double *X, const double *t, size_t l, const double *p,
                      float *J, void *stream);

/* Plain Levenberg-Marquardt calibration of one model at a time (Section
 * "Computing Model Parameters"), driven by the caller: the library does the
 * arithmetic of each step, the caller evaluates the residual and its
 * derivatives at the points the library names (pm_residual,
 * pm_residual_vjp, pm_jacobian -- in Python through the autograd.Function)
 * and reads one status word per trial.  Same damping and stopping rules as
 * the batched fit (see pm_fit_opts), with the step solve in FP64.
 *
 *   state:  caller-owned device buffer of PM_LM_STATE_BYTES bytes, opaque.
 *   pm_lm_init:   start point p0 (host, n_params FP64, finite); writes p0
 *                 to the device array p (n_params FP64); opts as for pm_fit
 *                 (use_p0 ignored: p0 is always given; NULL = defaults).
 *   pm_lm_step:   r (l FP64), b = J^T r (n_params FP64, from
 *                 pm_residual_vjp with rbar = r) and J (l x n_params FP32),
 *                 all at the current point p: on the first call after
 *                 pm_lm_init or after an accepted step they are assembled
 *                 into the scaled normal equations (later calls ignore them);
 *                 then the damped system is solved and the trial point
 *                 written to p_try (device, n_params FP64).
 *   pm_lm_update: r_try (l FP64), the residual at p_try: accepts or rejects
 *                 the trial, updates the damping, writes the current point
 *                 to p, and writes flags (device int32[2]) = {status,
 *                 accepted}: status 1 = running, PM_OK = converged,
 *                 PM_ENOTCONV = iteration limit.
 *   pm_lm_report: copies the state to the host (synchronises stream) and
 *                 fills a pm_fit_report (cond is NaN: not estimated).
 * init, step and update are asynchronous on `stream`; init's copies read
 * host memory that may be reused once it returns.  PM_EINVAL for NULL
 * pointers, l = 0, non-finite start points or negative options. */
#define PM_LM_STATE_BYTES 4096
pm_status pm_lm_init(const pm_model *m, const double *p0, const pm_fit_opts *opts, void *state, double *p,
                     void *stream);
pm_status pm_lm_step(void *state, const double *r, const double *b, const float *J, size_t l, double *p_try,
                     void *stream);
pm_status pm_lm_update(void *state, const double *r_try, size_t l, double *p, int32_t *flags, void *stream);
pm_status pm_lm_report(const void *state, pm_fit_report *report, void *stream);

/* Predict (Section "Predicting Cost"): t_out[k] = g(p; X_k) for l rows,
 * evaluated on the GPU in FP64.  X host l x n_features, p host, t_out host.
 * Device staging comes from the default memory pool on the legacy default
 * stream (see pm_run_host: the pool keeps freed memory reserved), so
 * repeated calls make no cudaMalloc / cudaFree.  Blocks until done. */
pm_status pm_predict(const pm_model *m, const double *p, const double *X, size_t l, double *t_out);

/* Thread-local, library-owned message of the last failure ("" if none). */
const char *pm_last_error(void);

/* Test hook (failure injection on the host, no GPU involvement): after
 * pm_test_fail_allocation(n) with n >= 1, the n-th next device or pinned-host
 * allocation the library attempts on the calling thread fails with PM_ENOMEM
 * before any CUDA call is made; n = 0 disarms it.  Every entry point that
 * allocates releases what it had allocated and returns PM_ENOMEM.  Genuine
 * out-of-memory errors from CUDA also map to PM_ENOMEM.  PM_EINVAL for
 * n < 0. */
pm_status pm_test_fail_allocation(int32_t n);

/* Test hook (failure detection without a GPU fault): one CTA waits, with
 * the bounded mbarrier wait and the device error word of the TMA-staged
 * dg_tile kernel, on an mbarrier phase that nothing completes (no arrival,
 * no copy in flight); after `polls` polls (1..2^20) the wait gives up and
 * sets the word, and the host reads and clears it as after a dg_tile
 * launch.  The call synchronizes `stream` (NULL: the legacy default
 * stream).  Returns PM_ETIMEOUT when the wait gave up, as it always does;
 * the context stays usable.  PM_EINVAL for polls out of range. */
pm_status pm_test_bounded_wait(int64_t polls, void *stream);

#ifdef __cplusplus
}
#endif
#endif
