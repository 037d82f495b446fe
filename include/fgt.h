/*
 * fgt.h — C ABI of the GB300 machine fast Gauss transform library (libfgt.so).
 *
 * The library evaluates the continuous Gauss transform of Greengard, Jiang,
 * Rachh and Wang, "A new version of the adaptive fast Gauss transform for
 * discrete and continuous sources" (arXiv 2305.07165):
 *
 *     u(x) = \int_B G(x - y; delta) sigma(y) dy,    B = [-1/2, 1/2]^d,
 *
 * Section 1, eq. (bgt), with the free-space kernel G(x) = exp(-|x|^2/delta)
 * (eq. (gkernel)) or its periodic image sum (eq. (gper_kernel)), d = 2 or 3.
 * sigma is given, and u is returned, at the k^d tensor-product Gauss-Legendre
 * nodes of the leaves of a level-restricted adaptive tree (Section 4,
 * Algorithm 3 output; Definition treedefs).  The transform itself is the box
 * FGT of Section 4.2, Algorithm 4, with the periodic variant of Section 5.
 *
 * Layout (all calls):
 *   - A tree is a list of leaves.  Leaf i has level leaf_level[i] >= 0 and
 *     integer box index leaf_coord[i*d + a] in [0, 2^level) along axis a
 *     (a = 0 is x_1).  Its centre is -1/2 + (coord + 1/2) 2^-level, its side
 *     L = 2^-level.  The leaves must tile B exactly and be 2:1 balanced across
 *     shared boundary points, corners included (Definition treedefs); with
 *     periodic boundary conditions the balance must also hold across the wrap.
 *   - sigma and u are FP64 arrays [n_leaves][k^d] in the caller's leaf order.
 *     Node t = (t_1..t_d) of a leaf sits at centre + (L/2)(eta_{t_1}, ...),
 *     eta the ascending k-point Gauss-Legendre nodes on [-1, 1]; inside a
 *     leaf t_1 is the fastest index.
 *
 * Errors: every call returns an fgt_status; nothing throws across the ABI.
 * fgt_last_error() gives a human-readable message for the calling thread's
 * most recent failure.  All entry points are thread-safe for distinct plans;
 * one plan must not be used from two threads at once.
 */
#ifndef FGT_H
#define FGT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FGT_OK = 0,
  FGT_ERR_ARG = 1,      /* bad argument (d, k, delta, tol, sizes, null pointers) */
  FGT_ERR_TREE = 2,     /* leaves do not tile B, overlap, or are not 2:1 balanced */
  FGT_ERR_OOM = 3,      /* device or host allocation failed */
  FGT_ERR_CUDA = 4,     /* a CUDA call failed (message has the CUDA error string) */
  FGT_ERR_TIMEOUT = 5,  /* a bounded device wait gave up (persistent batches: fgt_batch_status) */
  FGT_ERR_STATE = 6     /* call not valid in the plan's current state */
} fgt_status;

typedef enum { FGT_BC_FREE = 0, FGT_BC_PERIODIC = 1 } fgt_bc;

/* Arithmetic of the plane-wave contractions (form / shift / evaluate).
 * FGT_PREC_FP64: everything in FP64.
 * FGT_PREC_SPLIT: contractions and stored expansions in FP32 (accepted only
 *   when tol >= 1e-7); the near-field 1D tables, the tables' construction and
 *   the final per-leaf accumulation stay FP64.
 * FGT_PREC_FP64_TC: FP64-accurate contractions on the tensor cores.  3D plans in
 *   the fused mode with n_f <= 80 (the plane-wave modes per axis of Section 2.1)
 *   run every contraction of the form and the evaluation (Lemmas pwbox and
 *   pweval) on the BF16 tensor pipe: each FP64 operand is rounded to 47 bits
 *   against its row's (column's) largest exponent and cut into six 8-bit
 *   digits, the digit products are summed exactly in FP32 and recombined in
 *   64-bit integers (error a few units of 2^-47 times the row's and column's
 *   largest entries per term of the contraction); the out->in
 *   phases and the near field run in double-float arithmetic (FP32 pairs,
 *   about 2^-47 per operation), expansions and u stay FP64.  FGT_OZAKI=0 in the environment at plan
 *   creation, and the allocation-free call, use the FP64 tensor cores (DMMA)
 *   for the 3D form's last and the evaluation's first two contractions instead.
 *   2D plans and the kernels without either form run as FGT_PREC_FP64. */
typedef enum { FGT_PREC_FP64 = 0, FGT_PREC_SPLIT = 1, FGT_PREC_FP64_TC = 2 } fgt_prec;

/* How the plane-wave hierarchy of Algorithm 4 is executed.
 * FGT_MODE_FUSED (default): the child-to-parent (T_c->p) and parent-to-child
 *   (T_p->c) diagonal shifts are separable, so they are folded into the 1D form
 *   and evaluation matrices; leaves (or whole uniform subtrees) form their
 *   outgoing expansion directly at their cutoff-level ancestor and evaluate
 *   its incoming expansion directly.  Same arithmetic, reassociated.
 * FGT_MODE_HIERARCHICAL: the literal order of Algorithm 4 — form at each
 *   leaf's own centre, merge level by level with T_c->p, gather with
 *   T_out->in at the cutoff level, push level by level with T_p->c, evaluate
 *   at each leaf.  Needs an expansion slot for every box with f(B) = 1. */
typedef enum { FGT_MODE_FUSED = 0, FGT_MODE_HIERARCHICAL = 1 } fgt_mode;

typedef struct {
  int32_t d;                  /* 2 or 3 */
  int32_t k;                  /* Gauss-Legendre nodes per dimension per leaf, 1..16 */
  int64_t n_leaves;           /* >= 1 */
  const int32_t *leaf_level;  /* [n_leaves], host memory, copied by fgt_plan_create */
  const int32_t *leaf_coord;  /* [n_leaves * d], host memory, copied */
} fgt_tree;

typedef struct fgt_plan fgt_plan;

/* Plan parameters chosen at creation (host values, for inspection and tests). */
typedef struct {
  int32_t d, k, bc;
  int32_t cutoff_level;       /* l_c: boxes at l_c have side 2^-l_c >= D0 sqrt(delta) (Section 3) */
  int32_t fourier;            /* 1: periodic with l_c <= 1, root Fourier series (Section 5) */
  int32_t max_level;          /* deepest leaf level */
  int32_t n_f;                /* paper's n_f = 2M (Theorem 1, eq. (pwterms)); 0 when fourier */
  int32_t n_p;                /* periodic Fourier terms (Section 2.2); 0 unless fourier */
  int32_t modes_1d;           /* modes per dimension actually used: 2M-1, or 2 n_p + 1 */
  int32_t modes_half;         /* stored modes along the last dimension (conjugate symmetry) */
  double delta, tol, eps_pw;  /* eps_pw: the epsilon plugged into Theorem 1 / n_p */
  double D0, R, h;            /* Theorem 1 quantities (R*sqrt(delta) is the covered range) */
  int64_t n_leaves, n_boxes;
  int64_t n_pw_leaves;        /* leaves with f = 1 (evaluated from plane waves) */
  int64_t n_anchor_boxes;     /* boxes at l_c with f = 1 (outgoing/incoming expansion owners) */
  int64_t n_form_blocks;      /* uniform subtrees formed / evaluated as one dense transform */
  int64_t n_direct_pairs;     /* near-field (D-list) leaf pairs, images counted separately */
  int64_t n_gather_pairs;     /* out->in translations at the cutoff level */
  int64_t form_flops, eval_flops, gather_flops, direct_flops; /* per execute, real flops */
  int64_t device_bytes;       /* tables + lists + expansion workspace (excludes host-path staging) */
  int32_t prec, mode;
  int32_t launches;           /* CUDA kernels one execution launches */
  int64_t n_merge_items;      /* hierarchical mode: parents merged from their 2^d children (T_c->p) */
  int64_t n_push_items;       /* hierarchical mode: parents pushed to their 2^d children (T_p->c) */
  int64_t n_tc_eval_blocks;   /* evaluation blocks whose three contractions all run on tcgen05 */
  int64_t n_tc_form_blocks;   /* form blocks whose three contractions all run on tcgen05 */
  int64_t n_sliced_jobs;      /* FP64_TC, 3D: CTAs of the six sliced FP64 tensor-core stages per execution (0: not used) */
} fgt_plan_info;

/* Build a plan: validate the tree, choose l_c, n_f (or n_p), build the lists
 * and the FP64 1D tables (Section 4.1), upload them, size the workspace.
 * delta > 0; tol in [1e-14, 1e-1].  Returns FGT_ERR_TREE for invalid trees.
 *
 * Kernel choices are read from the environment when a plan is created (every choice computes the
 * same transform; the defaults are the measured fastest):
 *   FGT_OZAKI=0         FP64_TC, 3D: DMMA kernels instead of the sliced BF16 tensor-core stages
 *   FGT_FORM7=0 / =1    split, 3D: no form on tcgen05 / the tcgen05 form for K = 8 blocks too
 *   FGT_EVAL7=0         split, 3D: the CUDA-core evaluation instead of the tcgen05 one
 *   FGT_EVAL5=0 / =1    the evaluation order with the half-range axis last: off in FP64 / on in split
 *   FGT_GATHER2=0       FP64: the per-anchor gather instead of the run form
 *   FGT_GATHER3=0       3D: the run-form gather instead of the stencil forms over the cutoff grid
 *   FGT_TC_EVAL=1, FGT_TC_EVAL4=1, FGT_TC_EVAL6=1   earlier split-precision evaluation variants */
fgt_status fgt_plan_create(int d, double delta, double tol, int bc, const fgt_tree *tree, fgt_plan **out);

/* Same, with the plane-wave epsilon given explicitly (eps_pw <= 0 means tol). */
fgt_status fgt_plan_create_ex(int d, double delta, double tol, double eps_pw, int bc, int prec, int mode,
                              const fgt_tree *tree, fgt_plan **out);

/* Host-only dry run of fgt_plan_create_ex: validates the tree, builds the lists and
 * tables and fills `info` (including device_bytes, for admission by HBM footprint)
 * without touching the GPU.  Same error behaviour as plan creation. */
fgt_status fgt_plan_analyze(int d, double delta, double tol, double eps_pw, int bc, int prec, int mode,
                            const fgt_tree *tree, fgt_plan_info *info);

/* Host-only plan (no GPU is touched): the lists and tables are built and kept in host memory
 * for inspection through fgt_plan_host_array(); executing it returns FGT_ERR_STATE. */
fgt_status fgt_plan_create_host(int d, double delta, double tol, double eps_pw, int bc, int prec, int mode,
                                const fgt_tree *tree, fgt_plan **out);

/* Borrow a host-only plan's array by name ("blocks", "block_leaves", "Ff", "Fh", "Ef", "Eh",
 * "gather_dst", "gather_ptr", "gather_src", "gather_segs", "gather_grid", "Pf", "Ph", "near_tgt",
 * "near_flags", "near_ptr",
 * "near_src", "near_tab", "merge<i>_items|qf|qh", "push<i>_items|qf|qh", and for the sliced FP64
 * tensor-core stages "oz_jobs<kind>", "oz_btab", "oz_bexp", "eval_blocks").  "gather_grid", where
 * the plan gathers in stencil form, holds the expansion slot of each box of the cutoff grid (int32,
 * x1 fastest, -1 where a box has no outgoing expansion).  The pointer stays
 * valid until the plan is destroyed or re-planned.  FGT_ERR_STATE for device plans. */
fgt_status fgt_plan_host_array(const fgt_plan *plan, const char *name, const void **data, size_t *bytes);

fgt_status fgt_plan_set_precision(fgt_plan *plan, int prec);  /* fgt_prec; SPLIT needs tol >= 1e-7 */
fgt_status fgt_plan_set_mode(fgt_plan *plan, int mode);       /* fgt_mode */
fgt_status fgt_plan_get_info(const fgt_plan *plan, fgt_plan_info *info);

/* Device bytes the plan holds (tables, lists, expansion workspace). */
size_t fgt_plan_device_bytes(const fgt_plan *plan);

/* Evaluate u from sigma (Algorithm 4).  sigma_dev, u_dev: device pointers to
 * FP64 [n_leaves][k^d]; u is overwritten (not accumulated into); sigma is not
 * modified.  fgt_execute runs on the legacy default stream and returns after
 * the result is complete; fgt_execute_async only enqueues on `stream` (a
 * cudaStream_t, NULL = legacy default stream).  A plan runs one transform at a
 * time: do not overlap two executions of the same plan. */
fgt_status fgt_execute(fgt_plan *plan, const double *sigma_dev, double *u_dev);
fgt_status fgt_execute_async(fgt_plan *plan, const double *sigma_dev, double *u_dev, void *stream);

/* Allocation-free execution.  The paper has no counterpart; this entry point
 * exists for callers that must not allocate device memory at transform time
 * (an application whose allocator owns all device memory, or a thread that may
 * not call cudaMalloc/cudaFree because that would synchronise the device or
 * break its memory pool).  It computes exactly what fgt_execute_async does, on
 * `stream`, but keeps the plane-wave expansions in one fixed array of
 * FGT_NOALLOC_SCRATCH_BYTES (64 MiB) compiled into the library, which every GPU
 * that loads the library holds until the process exits.  It calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *   - The first call on a device looks up that array's device address (a
 *     one-time set-up per device); make that first call before any stream
 *     capture.
 *   - All calls share the array and each call overwrites it (the outgoing
 *     expansions are cleared at the start of every call): calls that overlap on
 *     the GPU race and give wrong results.  Serialise them.
 *   - sigma_dev and u_dev must be device memory on the plan's device; that
 *     device is made current for the call (the array is per device) and the
 *     caller's current device is restored afterwards.  FGT_ERR_ARG otherwise.
 *   - Returns FGT_ERR_ARG (with the sizes in the message) when the plan's
 *     expansion workspace is larger than the array, and FGT_ERR_STATE when the
 *     plan's mode or precision changed since it was last prepared (preparing
 *     again would allocate; fgt_plan_get_info prepares it). */
#define FGT_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
fgt_status fgt_execute_noalloc(fgt_plan *plan, const double *sigma_dev, double *u_dev, void *stream);

/* End to end: sigma_host, u_host are host arrays (pinned for full copy speed);
 * copies in, transforms, copies out on `stream` and synchronises it. */
fgt_status fgt_execute_host(fgt_plan *plan, const double *sigma_host, double *u_host, void *stream);

/* End to end, pipelined (the transform of Algorithm 4, Section 4.2; the pipelining has no counterpart
 * in the paper): the host-buffer transform of fgt_execute_host without the wait, so that
 * successive calls on one plan overlap.  Each call copies sigma_host in on the plan's copy-in
 * stream (into one of two device staging buffers, once the call two before it has copied its
 * result out of that buffer), transforms on `stream` once its input has arrived (calls on one plan
 * run their transforms in call order), and copies u_host out on the plan's copy-out stream.  So a
 * call's copy-in overlaps the previous call's transform, and its copy-out the next call's.
 * sigma_host and u_host (pinned for full copy speed) must stay untouched until fgt_host_sync
 * returns.  fgt_host_sync(plan) waits for every pipelined call on the plan to have written its
 * u_host.  Errors: as fgt_execute_host; FGT_ERR_OOM if the staging buffers or streams cannot be
 * created. */
fgt_status fgt_execute_host_async(fgt_plan *plan, const double *sigma_host, double *u_host, void *stream);
fgt_status fgt_host_sync(fgt_plan *plan);

/* ---- Batched execution: many independent transforms in one launch ----
 * The paper transforms one density at a time; batching is how the GPU is kept busy with many
 * small transforms of uneven depth, k and delta.  fgt_batch_create takes n prepared device
 * plans (any mix of d, k, delta, tol, bc, precision; the batch keeps pointers to them, so they
 * must outlive it and must not change mode or precision).  fgt_batch_execute enqueues all n
 * transforms on `stream` as ONE CUDA graph launch in which every transform is an independent
 * branch, so their kernels run concurrently; sigma_dev[i], u_dev[i] are device FP64 arrays of
 * plan i's size.  The graph is captured on the first call and again only when a pointer
 * changes.  Executions of one batch must not overlap each other or other executions of its
 * plans; a plan listed twice would race with itself and is rejected with FGT_ERR_ARG.
 * fgt_execute_batch = create + execute + synchronise `stream` + destroy. */
typedef struct fgt_batch fgt_batch;
fgt_status fgt_batch_create(fgt_plan *const *plans, int n, fgt_batch **out);

/* Persistent batched execution (no counterpart in the paper).  fgt_batch_create_mode with
 * FGT_BATCH_PERSISTENT lists every kernel launch of every transform as items of one device work
 * queue: an item is one CTA's share of one launch (transform, phase, block, row chunk).
 * fgt_batch_execute then enqueues ONE persistent kernel (one CTA per SM) whose CTAs pop the items in
 * order and run them with the same device code as the single-transform kernels.  Items of a phase
 * (clear, pack, form, gather, evaluate; near field after the clear) wait for their own transform's
 * previous phase through per-transform counters, every wait bounded (about one second); a wait that
 * runs out skips its item and sets the batch status word, read and cleared by fgt_batch_status
 * (0: none ran out, FGT_ERR_TIMEOUT otherwise), so nothing can hang.  The queue uses the CUDA-core
 * kernels (a plan's tcgen05 ranges take their CUDA-core fallbacks) and the plain expansion layout.
 * Plans in hierarchical mode or FP64 tensor-core precision are refused with FGT_ERR_ARG.
 * FGT_BATCH_GRAPH is fgt_batch_create's graph of per-transform branches.  fgt_batch_get_info
 * returns the mode, the number of queue items and the persistent grid size.
 * fgt_selftest_batch_timeout runs the persistent kernel on one item whose dependency nothing
 * satisfies, with a wait of about a millisecond, and returns the status it set (FGT_ERR_TIMEOUT).  Faults
 * nothing, hangs nothing; synchronous. */
#define FGT_BATCH_GRAPH 0
#define FGT_BATCH_PERSISTENT 1
fgt_status fgt_batch_create_mode(fgt_plan *const *plans, int n, int mode, fgt_batch **out);
fgt_status fgt_batch_status(fgt_batch *batch, int *status);
fgt_status fgt_batch_get_info(const fgt_batch *batch, int *mode, int64_t *items, int *grid);
fgt_status fgt_selftest_batch_timeout(int *status);
fgt_status fgt_batch_execute(fgt_batch *batch, const double *const *sigma_dev, double *const *u_dev, void *stream);
void fgt_batch_destroy(fgt_batch *batch);
fgt_status fgt_execute_batch(fgt_plan *const *plans, const double *const *sigma_dev, double *const *u_dev, int n,
                             void *stream);

/* Per-phase device timing (CUDA events on the launching stream) for the executions
 * enqueued while profiling is on.  Phases: 0 form, 1 child->parent merge, 2 out->in
 * gather, 3 parent->child push, 4 evaluate, 5 near field.  fgt_plan_read_profile
 * waits for the recorded events, returns the summed milliseconds per phase in
 * ms[0..5] and the number of executions covered, and starts a new accumulation. */
fgt_status fgt_plan_set_profiling(fgt_plan *plan, int on);
fgt_status fgt_plan_read_profile(fgt_plan *plan, double *ms, int *n_transforms);

/* Output tree (Algorithm 5, tree refinement): evaluate u at the nodes of the leaves of `out`
 * instead of the source tree's own leaves.  Every output leaf must lie inside one source leaf (at
 * its level or finer, levels <= 20) and no output leaf may overlap another; they need not cover
 * the source leaves (u is computed only where asked, as when a refinement round re-evaluates the
 * subdivided leaves alone); FGT_ERR_TREE otherwise.  The transform keeps the source tree's interaction lists: an
 * output leaf takes the plane-wave expansion and the near-field sources of the source leaf that
 * contains it, through evaluation matrices and near-field tables for its own nodes.  After this
 * call fgt_execute* write u as [out->n_leaves][k^d] (leaf order of `out`); sigma is unchanged.
 * out == NULL (or out->n_leaves == 0) restores the source tree.  Fused mode only.  The plan is
 * re-planned at its next execution. */
fgt_status fgt_plan_set_output_tree(fgt_plan *plan, const fgt_tree *out);

/* Refinement and coarsening helpers (Algorithms 5 and 6), on device arrays:
 * fgt_leaf_errors: for n boxes with values vals_dev[n][k^d] at their tensor Gauss-Legendre
 *   nodes, err_dev[i] = the error monitor of eq. (funerr), sqrt(mean |c_alpha|^2 over the tensor
 *   Legendre coefficients with ||alpha||_2 >= k), and, if sumsq_dev is not NULL, sumsq_dev[i] =
 *   sum_t w_t v_t^2 with the product Gauss weights of [-1,1]^d (scale by (L/2)^d for a box of side L).
 * fgt_merge_children: for n_parents parents, the values at the parent's nodes of the piecewise
 *   interpolant of its 2^d children, rows child_rows_dev[p * 2^d + c] of vals_dev, child c holding
 *   the half (c >> a) & 1 along axis a; written to parent_dev[n_parents][k^d].
 * Both: 2 <= d <= 3, 1 <= k <= 16, enqueued on `stream`. */
fgt_status fgt_leaf_errors(int d, int k, int64_t n, const double *vals_dev, double *err_dev, double *sumsq_dev,
                           void *stream);
fgt_status fgt_merge_children(int d, int k, int64_t n_parents, const int64_t *child_rows_dev, const double *vals_dev,
                              double *parent_dev, void *stream);

/* Algorithm 3 on the GPU for a density given as a sum of Gaussians,
 *   sigma(x) = sum_i amps[i] exp(-|x - centers[i]|^2 / alphas[i])   (amps NULL: all 1;
 *   periodic != 0: the minimum-image distance to each centre),
 * centers [n_gauss][d].  Level by level from the root, every box's k^d node values are computed,
 * then their Legendre coefficients and the error monitor of eq. (funerr); a box is subdivided
 * while its level is below min_level, or while e > eps ||sigma||_2 (the norm over the current
 * partition of B) and its level is below max_level.  The leaves are then 2:1 balanced (corners
 * included, across the wrap when periodic) and sigma is evaluated at their nodes.  The result
 * (*out, owned by the caller, freed with fgt_built_tree_destroy) holds the leaves (host arrays,
 * the layout of fgt_tree) and sigma on the device [n_leaves][k^d], ready for fgt_plan_create and
 * fgt_execute.  2 <= d <= 3, 1 <= k <= 16, 0 <= min_level <= max_level <= 20; synchronises `stream`. */
typedef struct fgt_built_tree fgt_built_tree;
fgt_status fgt_build_gaussian_tree(int d, int k, int n_gauss, const double *centers, const double *alphas,
                                   const double *amps, int periodic, double eps, int min_level, int max_level,
                                   void *stream, fgt_built_tree **out);
fgt_status fgt_built_tree_get(const fgt_built_tree *t, int64_t *n_leaves, const int32_t **level,
                              const int32_t **coord, const double **sigma_dev);
/* Copies the tree's sigma into dst_dev [n_leaves][k^d] (device) on `stream`. */
fgt_status fgt_built_tree_copy_sigma(const fgt_built_tree *t, double *dst_dev, void *stream);
void fgt_built_tree_destroy(fgt_built_tree *t);

/* Discrete (point) Gauss transform, free space (Section 3, Algorithms 1 and 2):
 *   u[i] = sum_j exp(-|x_i - y_j|^2 / delta) q_j,  sources src[n_src][d], targets tgt[n_tgt][d] (host,
 *   copied at create), weights q_dev[n_src] and result u_dev[n_tgt] on the device (original orders).
 * The tree is Algorithm 1's at its cutoff level: the bounding cube of all points in 2^l_c boxes of
 * side D0 sqrt(delta) per axis.  Boxes with more than n_s sources are dense: their sources are
 * replaced by a tensor-product proxy grid of k_p^d Gauss-Legendre nodes (in place of the NUFFT),
 * whose plane-wave expansion is formed, translated to every colleague (Eq. diagonaltranslation),
 * evaluated on the colleagues' proxy grids and interpolated to their targets; sources of sparse
 * boxes act on their colleagues' targets directly.  k_p is the smallest grid that reproduces every
 * plane wave of the expansion on a box to 0.1 tol relative to the mode's weight (FGT_ERR_ARG above
 * 40 nodes; about 21 at tol 1e-6 and 33 at 1e-10).
 * prec (fgt_prec): FGT_PREC_FP64 computes everything in FP64.  FGT_PREC_SPLIT (tol >= 1e-7 only)
 * computes the Lagrange weights, the anterpolation and the interpolation in FP32 (sums of at most
 * 32 terms in plain FP32, longer ones compensated) and the plane-wave expansions in FP32; the proxy
 * values Q and U, the direct pairs and the result stay FP64.  Other values: FGT_ERR_ARG. */
typedef struct fgt_point_plan fgt_point_plan;
typedef struct {
  int32_t cutoff_level, proxy_order, modes_1d;
  int64_t n_boxes, n_dense_boxes, n_incoming_boxes, n_direct_pairs;
  double cutoff_length;
  int32_t prec;
} fgt_point_info;
fgt_status fgt_point_plan_create(int d, double delta, double tol, int64_t n_src, const double *src, int64_t n_tgt,
                                 const double *tgt, int n_s, int prec, fgt_point_plan **out);
fgt_status fgt_point_execute(fgt_point_plan *plan, const double *q_dev, double *u_dev, void *stream);
fgt_status fgt_point_plan_get_info(const fgt_point_plan *plan, fgt_point_info *info);
void fgt_point_destroy(fgt_point_plan *plan);

/* Launch-shape knobs of a plan and the autotuner that picks them.
 *   form_group:      at most this many same-size blocks of one anchor per form CTA (1..8)
 *   eval_rows16:     split precision, 3D: rows of a K = 16 block per evaluation CTA (4, 8, 16)
 *   eval_rows_large: split precision, 3D: rows of a K > 16 block per evaluation CTA (4, 8)
 *   near_phase:      the near field runs on a second stream, forked before the form (0), the
 *                    gather (2) or the evaluation (4)
 *   ms:              the step time the autotuner measured for the chosen knobs (0 if never tuned)
 * None of them changes what is computed, only the launch shapes (results differ at most by
 * the order of floating-point sums).  fgt_plan_autotune times the plan on the caller's
 * sigma_dev / u_dev on `stream` (one warm-up and `reps` timed executions per candidate,
 * coordinate descent over the knobs that apply to the plan), keeps the fastest setting, and
 * writes it to *out (may be NULL).  It synchronises `stream`; u_dev holds a valid result
 * afterwards.  fgt_plan_set_tuning applies known settings (e.g. from an earlier run). */
typedef struct {
  int32_t form_group, eval_rows16, eval_rows_large, near_phase;
  double ms;
} fgt_tuning;
fgt_status fgt_plan_autotune(fgt_plan *plan, const double *sigma_dev, double *u_dev, void *stream, int reps,
                             fgt_tuning *out);
fgt_status fgt_plan_get_tuning(const fgt_plan *plan, fgt_tuning *out);
fgt_status fgt_plan_set_tuning(fgt_plan *plan, const fgt_tuning *t);

void fgt_destroy(fgt_plan *plan);

const char *fgt_last_error(void);

/* Status of the tensor-core (tcgen05) evaluation kernels on the current device (no counterpart in the
 * paper).  Those kernels wait
 * on the tensor cores through mbarriers with a time limit of about one second; a wait that runs out
 * makes the kernel skip the rest of its block (u is then wrong there), free its tensor memory and
 * set a device status word instead of hanging.  This call copies that word to *status and clears it:
 *   0: no wait ran out since the last call;
 *   1: a wait ran out, and the copies and MMAs the kernel had in flight completed before it
 *      exited (u is wrong in the skipped blocks, the context is sound);
 *   2: a wait ran out and so did the bounded wait for those copies or MMAs, so one may have
 *      landed after the kernel freed its shared or tensor memory: treat the context as suspect
 *      (results of later kernels on it cannot be trusted until the process restarts the device).
 * The largest value seen since the last call is kept.  It synchronises with the device.
 * FGT_ERR_ARG if status is NULL, FGT_ERR_CUDA if the copy fails. */
fgt_status fgt_device_status(int *status);
/* Self-test of that time-out path (no counterpart in the paper): launches one thread that waits
 * about a millisecond on an mbarrier nothing completes, so that it gives up and sets the status word;
 * the next fgt_device_status returns 1.  Faults nothing and hangs nothing.  Synchronous. */
fgt_status fgt_selftest_tc_timeout(void);

/* Bounds-checked build (libfgt_checked.so, compiled with -DFGT_CHECKED; the paper has no
 * counterpart).  There, every instrumented global access of the kernels (all stores of u, the
 * expansions and the packed density, the streamed loads of sigma and of the expansions) first
 * checks that its bytes lie in the buffers registered for the call (sigma, u, the plan's tables and
 * workspace, or the allocation-free scratch); a failing access is skipped and counted, so an index
 * error is reported instead of faulting.  Batched graphs run unchecked.  Checks assume one transform
 * in flight at a time.  This call reads and clears the first failing access's source line (*site)
 * and the number of failures (*count) since the last call, and sets *checked to 1 in the checked
 * build (in the normal build: *checked = 0, *site = *count = 0).  Synchronous. */
fgt_status fgt_check_status(unsigned *site, unsigned *count, int *checked);

/* ---- Host-side building blocks of the 1D tables (Section 2.4), exposed for tests ---- */

/* k-point Gauss-Legendre rule on [-1,1], ascending nodes. 1 <= k <= 64. */
fgt_status fgt_gauss_legendre(int k, double *nodes, double *weights);

/* Theorem 1 / Section 3 parameters for (delta, eps, bc): cutoff level l_c,
 * D0 = sqrt(log(3/eps)), range R, step h, n_f = 2M; n_p of Section 2.2. */
fgt_status fgt_params(double delta, double eps, int bc, int32_t *cutoff_level, double *D0, double *R,
                      double *h, int32_t *n_f, int32_t *n_p);

/* n_f(R) = 2 ceil(D0 (R + D0) / pi) for a given R (Theorem 1, eq. (pwterms)). */
int32_t fgt_nf_for_range(double eps, double R);

/* J_lambda[P_n](t) = int_{-1}^{1} exp(-(t-x)^2/lambda^2) P_n(x) dx, n = 0..nmax
 * (Section 2.4, eq. (gsintegrals)): erf seeds plus the five-term recurrence
 * (eq. (Jnrecurrence)) when lambda <= 1/8, Gauss-Legendre quadrature above. */
fgt_status fgt_legendre_gauss_integrals(double lambda, double t, int nmax, double *out);

/* Spherical Bessel j_n(x), n = 0..nmax (backward recurrence, normalised). */
fgt_status fgt_spherical_bessel(double x, int nmax, double *out);

/* I[P_n](t) = int_{-1}^{1} exp(i t x) P_n(x) dx = 2 i^n j_n(t), n = 0..nmax
 * (Section 2.4, eq. (pwintegrals2)); real and imaginary parts. */
fgt_status fgt_legendre_fourier_integrals(double t, int nmax, double *re, double *im);

#ifdef __cplusplus
}
#endif

#endif /* FGT_H */
