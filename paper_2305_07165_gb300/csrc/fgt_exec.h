// Device-side execution descriptor: everything one transform launch sequence
// needs, filled by the planner and consumed by fgt_kernels.cu.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "fgt_internal.h"

namespace fgt {

// One launch of a kernel over a contiguous range of items that share a block size K.
struct LaunchRange {
  int first = 0, count = 0, K = 0;
  size_t smem = 0;
  int tensor = 0;  // 1: the tensor-core (3xTF32) variant of the kernel
  int big = 0;     // 1: single blocks of K > 16, sigma streamed from global memory in stage 1
  int rows = 0;    // evaluation: rows of a block per CTA
  int tmem_cols = 0;  // tcgen05 evaluation: tensor-memory columns per CTA
  // tensor: 1 TF32 mma.sync form / evaluation, 2 evaluation stages 2-3 on mma.sync, 3 half-range axis
  // last, 4 evaluation stage 1 on tcgen05, 7 every evaluation stage on tcgen05 (eval7_kernel)
};

// One level of the hierarchical merge (child -> parent) or push (parent -> child).
struct ShiftStep {
  const TreeShift *items = nullptr;  // device
  int64_t n = 0;
  const void *qf = nullptr;          // [2][n1] phase per child half (bit 0 / 1), full-range axes
  const void *qh = nullptr;          // [2][nh] same for the last (half-range) axis
};

constexpr int kSides = 3;

struct ExecDesc {
  int d = 0, k = 0, n1 = 0, nh = 0;
  int prec = 0;                      // 0: FP64 expansions, 1: FP32 expansions
  int tc64 = 0;                      // FP64 contractions on the tensor cores (DMMA) where a kernel has them
  int fourier = 0;                   // 1: no out->in gather, evaluation reads the outgoing slot
  int64_t slot_size = 0;             // complex elements per expansion slot
  int64_t n_phi_slots = 0, n_psi_slots = 0;
  void *phi = nullptr, *psi = nullptr;

  // dense block form / evaluation: all blocks, then the per-kernel lists
  const Block *blocks = nullptr;     // device
  int64_t n_blocks = 0;
  int Kmax = 0;
  const Block *f1_blocks = nullptr;  // per-(block, m_d) form kernel
  int64_t n_f1 = 0;
  int Kmax_f1 = 0;
  const Block *f2_blocks = nullptr;  // grouped form kernel; group g = f2_blocks[gptr[g] .. gptr[g+1])
  const int32_t *f2_gptr = nullptr;
  int64_t n_f2_groups = 0;
  std::vector<LaunchRange> f2_ranges;  // groups by K
  const Block *e1_blocks = nullptr;  // per-(block, row) evaluation kernel
  int64_t n_e1 = 0;
  int Kmax_e1 = 0;
  const Block *e2_blocks = nullptr;  // whole-block evaluation kernel
  int64_t n_e2 = 0;
  std::vector<LaunchRange> e2_ranges;  // blocks by K
  const int64_t *block_leaves = nullptr;  // form blocks' source leaves
  const int64_t *eval_leaves = nullptr;   // evaluation blocks' target leaves (u rows)
  // split precision, 3D: sigma converted to FP32 once per transform, block by block (block b's
  // K^3 values at sigp + b.leaf0 k^3, in (J3, J2, J1) order); nullptr: kernels read sigma itself
  float *sigp = nullptr;
  const int32_t *pack_block = nullptr;  // index into blocks of every block_leaves entry
  int64_t n_pack = 0;                   // block_leaves entries
  const void *Ff = nullptr, *Fh = nullptr, *Ef = nullptr, *Eh = nullptr;
  // tcgen05 evaluation: the expansions it reads in the tensor cores' operand layout (written once
  // per transform after the gather); nullptr: the tcgen05 ranges fall back to the CUDA-core kernel
  void *psi_tc = nullptr;
  int64_t n_psi_tc_slots = 0;
  // all-tcgen05 evaluation (eval7_kernel, split precision, 3D): psi_pitch > 0 stores the incoming
  // expansions padded, slot s at s * nh * pitch^2 complex values, [m3][m2 < pitch][m1 < pitch] (zero
  // beyond n1), read through the tensor map psi_map; 0: the slot layout of phi
  int psi_pitch = 0;
  int psi_map_ready = 0;  // 1 once psi_map has been encoded for psi
  CUtensorMap psi_map;  // 64-byte aligned by its type
  // all-tcgen05 form (form7_kernel): the packed density in (J1, J2, J3) order (sig_order 1; 0: the
  // (J3, J2, J1) order of the CUDA-core forms) read through one tensor map per K = 8, 16, 32
  int sig_order = 0;
  int sig_maps_ready = 0;  // 1 once sig_map has been encoded for sigp (the K in use)
  CUtensorMap sig_map[3];
  // 1: every form block is the only one of its anchor and stores the whole slot (no clear of phi)
  int phi_stored = 0;

  // FP64-accurate form and evaluation on the BF16 tensor cores (precision FP64_TC, 3D, fused mode):
  // six contraction stages (form: x3, x2, x1; evaluation: m1, m2, m3), one launch each over its
  // jobs, every operand cut into six 8-bit slices with exact FP32 accumulation of the slice products
  // (oz_slice_kernel + oz_mma_kernel).  The stages pass their FP64 intermediates through oz_x / oz_y; without them
  // (the allocation-free call) the FP64 kernels of the block lists above run instead.
  int oz = 0;
  int oz_sole = 0;                      // every form block stores its anchor's slot (no clear of phi)
  const OzJob *oz_jobs[6] = {};           // products: (block, tile, part)
  int64_t oz_njobs[6] = {};
  const OzJob *oz_sjobs[6] = {};          // slicing: (block, tile)
  int64_t oz_nsjobs[6] = {};
  unsigned char *oz_dig = nullptr;        // the current stage's operand digit planes
  int *oz_rexp = nullptr;                 // and its row exponents
  const unsigned char *oz_btab = nullptr;  // the sliced 1D matrices (BF16 digit planes)
  const int32_t *oz_bexp = nullptr;        // their column exponents
  const Block *eval_blocks = nullptr;      // the evaluation's blocks (the jobs of stages 3-5 index them)
  const OzGroup *oz_groups = nullptr;      // stage 2's block groups (its jobs index them)
  double *oz_x = nullptr, *oz_y = nullptr;

  // out->in gather at the cutoff level
  int64_t n_gather = 0;
  const int32_t *gather_dst = nullptr;
  const int64_t *gather_ptr = nullptr;
  const GatherSrc *gather_src = nullptr;
  const void *Pf = nullptr, *Ph = nullptr;   // [3][n1], [3][nh]
  const GatherSeg *gather_segs = nullptr;    // separable form of the same gather
  int64_t n_gather_segs = 0;
  int seg_w = 0;                             // target boxes per run (min(kSegW, boxes a side at l_c))
  // every box of the cutoff level an anchor (3D, 4 or 8 boxes a side): the stencil form of the gather
  // over the grid, gather_grid[(x3 nb + x2) nb + x1] = slot of box (x1, x2, x3); grid_nb = 0: not used
  int grid_nb = 0, grid_periodic = 0;
  int grid_lines = 0;  // FP64-TC, gather_grid with boxes without an anchor (-1): the line-stencil kernel
  int gather_sym = 0;  // the phase factors have P(0) = 1 and P(+1) = conj P(-1) exactly (checked at plan time)
  const int32_t *gather_grid = nullptr;

  // hierarchical mode (empty in fused mode); merge in execution order (fine -> coarse)
  std::vector<ShiftStep> merge, push;

  // optional per-phase timing: events[2p] / events[2p+1] recorded around phase p
  // (p: 0 form, 1 merge, 2 gather, 3 push, 4 evaluate, 5 near field); nullptr = off
  cudaEvent_t *events = nullptr;

  // near field (D-list)
  int64_t n_near = 0;
  const int64_t *near_tgt = nullptr;
  const int32_t *near_flags = nullptr;
  const int64_t *near_ptr = nullptr;
  const NearSrc *near_src = nullptr;
  const double *near_tab = nullptr;
  const NearPair *near_pairs = nullptr;  // flattened D-list, one CTA per pair
  const int16_t *near_band = nullptr;    // per table and row: first and last kept column
  int64_t n_near_pairs = 0;
  int64_t n_points = 0;                  // n_leaves * k^d
  int zero_u = 0;                        // clear u first (near field or accumulating evaluation)
  // side streams owned by the plan (nullptr: everything on the caller's stream).  Side 0 runs the
  // near field, forked before phase near_phase (0 form, 2 gather, 4 evaluate) and joined at the
  // end; sides 1 and 2 run the second and later per-size launches of the form and of the
  // evaluation concurrently with the first, joined at the end of their phase.
  cudaStream_t side[kSides] = {};
  cudaEvent_t fork_ev[kSides] = {}, join_ev[kSides] = {};
  int near_phase = 0;
};

constexpr int kPhases = 6;

// Number of kernel launches one transform makes.
int launches_per_transform(const ExecDesc &e);

// Enqueue the whole transform on `stream`.  sigma, u: device FP64 [n_leaves][k^d].
cudaError_t run_transform(const ExecDesc &e, const double *sigma, double *u, cudaStream_t stream);

// Checked build (-DFGT_CHECKED): the buffers the next kernels on `st` may touch (at most
// kCheckRanges; n = 0 turns the checks off), and the first failing access's source line and the
// failure count since the last read (read and cleared; synchronous).  No-ops in the normal build
// (*checked = 0).  One transform at a time: the ranges are global to the device.
constexpr int kCheckRanges = 8;
cudaError_t set_check_ranges(const void *const *base, const size_t *bytes, int n, cudaStream_t st);
cudaError_t read_check(unsigned *site, unsigned *count, int *checked);

// Persistent batched execution: the launches of many transforms (fused mode) as items of one device
// work queue, run by one persistent kernel with per-transform phase counters and bounded waits.
// batch_queue_create sets *why (and *out = nullptr) when a plan cannot be queued.  wait_clocks bounds
// every dependency wait (a wait that runs out sets the batch status word to 1).
struct BatchQueue;
cudaError_t batch_queue_create(const std::vector<const ExecDesc *> &plans, BatchQueue **out, const char **why);
cudaError_t batch_queue_run(BatchQueue *q, const double *const *sigma, double *const *u, cudaStream_t st,
                            long long wait_clocks);
cudaError_t batch_queue_status(BatchQueue *q, int *status);  // read and clear; synchronous
size_t batch_queue_items(const BatchQueue *q);
int batch_queue_grid(const BatchQueue *q);
void batch_queue_destroy(BatchQueue *q);
// One item whose dependency nothing satisfies, with a wait of about a millisecond: *status = 1.
cudaError_t selftest_batch_timeout(int *status);

// Sliced FP64 tensor-core contraction stages (fgt_ozaki.cu).  Stage kinds 0-2: the form's
// contractions over x3, x2, x1; 3-5: the evaluation's over m1, m2, m3.  Per block of K nodes a
// side: R rows, Q contraction length, N columns, split into P parts of Nc (padded to Np) columns,
// nks k-steps of 16.
constexpr int kOzSlices = 6;
constexpr int kOzMaxNp = 32;  // columns per part: 6 accumulators x 32 TMEM columns, two CTAs an SM
struct OzDims { int R, Q, N, P, Nc, Np, nks; };
inline __host__ __device__ OzDims oz_dims(int kind, int K, int n1, int nh) {
  OzDims d{};
  switch (kind) {
    case 0: d.R = K * K; d.Q = K; d.N = 2 * nh; break;
    case 1: d.R = nh * K; d.Q = 2 * K; d.N = 2 * n1; break;
    case 2: d.R = nh * n1; d.Q = 2 * K; d.N = 2 * n1; break;
    case 3: d.R = nh * n1; d.Q = 2 * n1; d.N = 2 * K; break;
    case 4: d.R = K * nh; d.Q = 2 * n1; d.N = 2 * K; break;
    default: d.R = K * K; d.Q = 2 * nh; d.N = K; break;
  }
  d.P = (d.N + kOzMaxNp - 1) / kOzMaxNp;
  d.Nc = (d.N + d.P - 1) / d.P;
  d.Np = (d.Nc + 15) / 16 * 16;
  d.nks = (d.Q + 15) / 16;
  return d;
}
// Stage 2 over a group of blocks: the concatenated contraction length Q replaces 2 K.
inline __host__ __device__ OzDims oz_dims_group(int n1, int nh, int Q) {
  OzDims d = oz_dims(2, 8, n1, nh);
  d.Q = Q;
  d.nks = (Q + 15) / 16;
  return d;
}
// Enqueue stage `kind` over its jobs: src -> dst (sigma -> oz_x -> oz_y -> phi; psi -> oz_x -> oz_y -> u).
cudaError_t run_oz_stage(const ExecDesc &e, int kind, const double *src, double *dst, cudaStream_t st);
// Reads and clears the status word of the sliced stages (1: a wait ran out, 2: its drain as well).
cudaError_t read_oz_status(int *status);

// Reads and clears the status word of the tcgen05 kernels: 1 when a wait on the tensor cores ran
// out since the last read (the affected blocks were skipped), else 0.  Synchronous.
cudaError_t read_tc_status(int *status);
// Runs a kernel whose only wait (about a millisecond) is on an mbarrier that nothing completes, so
// that it sets the status word; synchronous.
cudaError_t selftest_tc_timeout();

// Allocation-free execution: the expansion workspace lives in a fixed device array of
// kNoallocScratchBytes inside the library instead of the plan's own buffers.  The first call
// on a device looks up that array's device address (cudaGetSymbolAddress).  Returns
// cudaErrorInvalidValue when the plan's workspace does not fit.
constexpr size_t kNoallocScratchBytes = size_t(64) << 20;
cudaError_t noalloc_scratch(void **ptr);
cudaError_t run_transform_noalloc(const ExecDesc &e, const double *sigma, double *u, cudaStream_t stream);

// Gauss-Legendre rule passed by value to the refinement / coarsening kernels (k <= kMaxLeafK).
constexpr int kMaxLeafK = 16;
struct GLRule {
  double x[kMaxLeafK], w[kMaxLeafK];
};
// Error monitor (eq. funerr) and quadrature sum of squares of n boxes' node values; device arrays.
cudaError_t leaf_errors(int d, int k, int64_t n, const double *vals, double *err, double *sumsq, cudaStream_t st);
// A sum of Gaussians at the nodes of n boxes (Algorithm 3's density evaluation); device arrays,
// gparams[ng][d + 2] = (centre, alpha, amplitude).
cudaError_t gauss_nodes(int d, int k, int64_t n, const int32_t *level, const int32_t *coord, int ng,
                        const double *gparams, int periodic, double *vals, cudaStream_t st);
// Parent node values from the interpolants of 2^d children (Algorithm 6); device arrays.
cudaError_t merge_children(int d, int k, int64_t n_parents, const int64_t *child_rows, const double *vals,
                           double *parent, cudaStream_t st);

// ---- discrete (point) Gauss transform with proxy grids (Algorithm 2)
constexpr int kMaxProxy = 40;
constexpr int kMaxProxy32 = 30;  // largest k_p of the FP32 (split) point kernels
struct ProxyRule {
  double x[kMaxProxy];   // Gauss-Legendre nodes on [-1, 1]
  double bw[kMaxProxy];  // barycentric weights of the Lagrange basis on them
  float xf[kMaxProxy];   // the nodes rounded to FP32
  float bwf[kMaxProxy];  // the weights over their largest magnitude, rounded to FP32
};
// Points per CTA of the point-FGT kernels (segments of a box's sources or targets).
constexpr int64_t kPointSeg = 1024;
// Q[b][t] = sum_{j in dense box b} q_j prod_a l_{t_a}(s_{j,a}) (sources sorted by box, local
// coordinates s in [-1, 1]^d); segments seg[3s..3s+2] = (box, first, end).  f32: the FP32 kernel.
cudaError_t point_anterp(int d, int kp, bool f32, const ProxyRule &pr, int64_t n_dense, int64_t n_seg,
                         const int64_t *seg,
                         const double *s_local, const double *q_sorted, double *Q, cudaStream_t st);
// u[id_i] = (incoming boxes) sum_t prod_a l_{t_a}(s_{i,a}) U[in(box)][t] + sum over the box's direct
// source boxes of exp(-|x_i - y_j|^2 / delta) q_j; one CTA per target box.
struct PointTargets {
  int d = 0, kp = 0, f32 = 0;          // f32: interpolation in FP32 (direct pairs stay FP64)
  double delta = 0;
  int64_t n_tseg = 0;
  const int64_t *tseg = nullptr;       // segments (target box, first, end) of at most kPointSeg targets
  const double *t_xyz = nullptr;       // sorted targets, coordinates [n][d]
  const double *t_local = nullptr;     // sorted targets, local coordinates in their box [n][d]
  const int64_t *t_id = nullptr;       // original index of each sorted target
  const int32_t *tbox_in = nullptr;    // row of U for the box, -1 if no plane-wave part
  const double *U = nullptr;           // [n_in][kp^d]
  const int64_t *dptr = nullptr;       // CSR over target boxes into dbox
  const int32_t *dbox = nullptr;       // direct source boxes (indices into sptr)
  const int64_t *sptr = nullptr;       // CSR over boxes into the sorted sources
  const double *s_xyz = nullptr;       // sorted sources [n][d]
  const double *q_sorted = nullptr;    // weights of the sorted sources
  double inv_delta = 0;                // 1 / delta
  // FP32 direct pairs (split precision): differences from local coordinates,
  // x - y = (Lc/2) (t_local - s_local - 2 o) for a source box at offset o (in boxes) from the target's
  const int32_t *dcode = nullptr;      // per dbox entry: sum_a (o_a + 1) 3^a
  const float *s_local32 = nullptr;    // sorted sources' local coordinates [n][d], FP32
  const float *q32 = nullptr;          // weights of the sorted sources, FP32
  float dcoef = 0;                     // (Lc/2)^2 / delta
};
cudaError_t point_targets(const PointTargets &pt, const ProxyRule &pr, double *u, cudaStream_t st);
// q permuted into the sources' box order: q_sorted[j] = q[s_id[j]] (and its FP32 copy when q32 != NULL)
cudaError_t point_gather_q(int64_t n, const int64_t *s_id, const double *q, double *q_sorted, float *q32,
                           cudaStream_t st);

// Shared-memory bytes of the grouped form kernel (G blocks of K nodes per axis; r, c: real and
// complex element sizes) and of the whole-block evaluation kernel.
inline size_t form2_bytes(int d, int G, int K, int n1, int nh, size_t r, size_t c) {
  const size_t npb = (d == 3) ? (size_t)K * K * K : (size_t)K * K;
  size_t b = npb * r + (size_t)n1 * K * c + (size_t)nh * K * c + (d == 3 ? (size_t)K * K : (size_t)K) * c;
  if (d == 3) b += 2 * (size_t)n1 * K * c;  // second-axis matrices and Z2
  return (size_t)G * b + 16;                // padding that keeps the complex arrays aligned
}
// Register-tiled 3D form: G blocks of K nodes per axis, planes m_3 in chunks of 4.
inline size_t form3_bytes(int G, int K, int n1, size_t r, size_t c) {
  const size_t GK = (size_t)G * K, Sc = 4;
  const size_t sig = (((size_t)G * K * K * K * r) + 15) & ~(size_t)15;
  return sig + c * (GK * n1 + (size_t)G * n1 * K + (size_t)G * Sc * K + Sc * G * (size_t)K * K +
                    Sc * (size_t)n1 * (GK + 1));
}
// Tensor-core 3D form (FP32 only): F1t and Z2 (rows GK + 2 complex wide) kept, then sigma, F2,
// Fd and Z1, over which the split B operands (2 x 2 n1p x (2GK+4)) are built after stage 2.
// big: one block of K > 16 whose sigma is read from global memory in stage 1 (no sigma tile).
inline size_t form4_bytes(int G, int K, int n1, bool big = false) {
  const size_t GK = (size_t)G * K, n1p = ((size_t)n1 + 7) / 8 * 8, c = 8, Sc = 4;
  const size_t keep = c * (GK * n1 + Sc * (size_t)n1 * (GK + 2));
  const size_t sig = big ? 0 : (((size_t)G * K * K * K * 4) + 15) & ~(size_t)15;
  const size_t s12 = sig + c * ((size_t)G * n1 * K + (size_t)G * Sc * K + Sc * G * (size_t)K * K);
  const size_t bops = 2 * (2 * n1p) * (2 * GK + 4) * 4;
  return keep + (s12 > bops ? s12 : bops);
}
inline size_t form4b_bytes(int K, int n1) { return form4_bytes(1, K, n1, true); }
// Tensor-core 3D evaluation (FP32 only): 8 output rows per CTA.
inline size_t eval3_bytes(int K, int n1, int nh) {
  return 8 * (8 * (size_t)n1 * n1 + 8 * (size_t)K * n1 + 2 * (size_t)K * n1 + 8 * (size_t)nh);
}
// Evaluation with the half-range axis contracted last: `rows` rows I1 of a block per CTA.
inline size_t eval5_bytes(int K, int n1, int nh, size_t c, int rows) {
  const size_t R = (size_t)(K < rows ? K : rows);
  return c * (R * nh * n1 + R * K * nh + R * n1 + (size_t)K * n1 + (size_t)K * nh);
}
// Whole-block evaluation, `rows` rows (along the last axis) of a block per CTA (4, 8 or 16).
inline size_t eval2_bytes(int d, int K, int n1, int nh, size_t c, int rows) {
  const size_t R = (size_t)(K < rows ? K : rows);  // rows held at once
  if (d == 3) return c * (R * n1 * n1 + R * K * n1 + 2 * (size_t)K * n1 + R * nh);
  return c * (R * n1 + (size_t)K * n1 + R * nh);
}

// Whole-block 3D evaluation with stage 1 on tcgen05 (split precision).  The expansion's operand
// copy: per slot, tiles of 128 modes, each a TF32 hi half and a lo half of 128 x kp2 values
// (kp2 = 2 nh padded to a multiple of 8), K-major core matrices.  Shared memory: a ring of
// kEval6Ring half-tiles and the rows' B operand (hi and lo), overlaid after stage 1 by the FP32
// stage-1 result; then the stage-2 result, the E1 / E2 matrices and the barrier words.
inline int eval6_kpad(int nh) { return (2 * nh + 7) / 8 * 8; }
constexpr int kEval6MaxKp2 = 64;  // largest padded 2 nh (nh <= 32)
constexpr int kEval6Ring = 3;
inline int eval6_n(int rows) { return rows <= 8 ? 16 : 2 * rows; }
inline size_t eval6_half_bytes(int nh) { return 128 * (size_t)eval6_kpad(nh) * 4; }
inline size_t eval6_slot_bytes(int n1, int nh) {
  return (size_t)((n1 * n1 + 127) / 128) * 2 * eval6_half_bytes(nh);
}
inline size_t eval6_bytes(int K, int n1, int nh, int rows) {
  const size_t R = (size_t)(K < rows ? K : rows), kp2 = (size_t)eval6_kpad(nh);
  const size_t stage = kEval6Ring * eval6_half_bytes(nh) + 2 * (size_t)eval6_n(rows) * kp2 * 4;
  const size_t y1 = 8 * R * n1 * n1;
  const size_t r1 = ((stage > y1 ? stage : y1) + 127) & ~(size_t)127;
  return r1 + 8 * (R * K * n1 + 2 * (size_t)K * n1) + 64;
}
// Tensor-memory columns of that kernel: one 128 x N accumulator per 128-mode tile, rounded up to a
// power of two (at least 32); 0 when the tiles do not fit the 512 columns of an SM.
inline int eval6_tmem_cols(int n1, int rows) {
  const int tiles = (n1 * n1 + 127) / 128, cols = tiles * eval6_n(rows);
  int c = 32;
  while (c < cols) c *= 2;
  return c <= 512 ? c : 0;
}

// All-tcgen05 evaluation (eval7_kernel): shared-memory bytes per CTA for K = 8, 16, 32, the padded
// mode count per full-range axis of its expansion layout, and the tensor map over the padded
// expansions of e (e.psi, e.psi_pitch, e.nh, e.n_psi_slots set).
size_t eval7_smem_bytes(int K);
int eval7_pitch();
cudaError_t encode_psi_map(ExecDesc &e);
// All-tcgen05 form (form7_kernel): shared-memory bytes per CTA, and the tensor maps over the packed
// density e.sigp (total_floats values) for the block sizes with used[i] (K = 8, 16, 32).
size_t form7_smem_bytes(int K);
cudaError_t encode_sig_maps(ExecDesc &e, int64_t total_floats, const bool *used);

// Shared-memory bytes the form / evaluation kernels need for a block size K.
size_t form_smem_bytes(int d, int K, int n1, int prec);
size_t eval_smem_bytes(int d, int K, int n1, int prec);
int max_dynamic_smem();

}  // namespace fgt
