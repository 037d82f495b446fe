// FP64-accurate contractions of the 3D form (Lemma pwbox) and evaluation (Lemma pweval) on the
// fifth-generation tensor cores.
//
// GB300 issues two FP64 FMAs per clock per SM, on the FP64 pipe and through DMMA alike, so the FP64
// kernels stop at 1.2 TFLOP/s.  These stages take the FP64 products to the BF16 tensor pipe by
// error-free slicing (the splitting of Ozaki, Ogita and Oishi, 2012, here with integer digits):
//
//   - a row r of the matrix operand A carries the exponent e_r of its largest entry, a column n of
//     the 1D matrix B the exponent f_n of its largest; every entry is rounded to a 47-bit integer
//     multiple of that scale and written as six balanced base-256 digits,
//         x = 2^e sum_{s=0..5} d_s 2^(-7 - 8 s),   |d_s| <= 128,
//     each digit an exact BF16 value;
//   - the slice products of equal weight, P_D = sum_q sum_{s+t=D} dA_s dB_t for D = 0..5, are
//     accumulated on the tensor pipe in one FP32 accumulator each (tensor memory): at most
//     6 x 160 products of magnitude <= 2^14 sum to less than 2^24, so every P_D is exact;
//   - C[r][n] = 2^(e_r + f_n - 14) sum_D 2^(-8 D) P_D is recombined in a 64-bit integer and
//     rounded to FP64 once.
// The products dropped (s + t >= 6) and the two 47-bit roundings bound the error of C[r][n] by a
// few units of 2^(e_r + f_n - 47) per term of the contraction (the roundings are relative to the
// row's and the column's largest entries) -- FP64 quality for a contraction, for 21 BF16 products
// per FP64 product where a 3xTF32 product needs 3 TF32 ones.
//
// Each stage is one contraction of the block's separable product (form: x3, x2, x1; evaluation:
// m1, m2, m3, the last one keeping the real part) and takes two launches:
//   - oz_slice_kernel, one CTA per (block, 128-row tile): the rows' exponents and the operand's six
//     digit planes per 16-deep step, written once (a tile's columns are split into parts, and every
//     part reads the same planes) in the tensor cores' K-major core-matrix layout;
//   - oz_mma_kernel, persistent, one CTA per SM over the (block, tile, column part of <= 32 columns)
//     jobs: a copy warp streams the tile's digit planes and the 1D matrix's of each step with bulk
//     asynchronous copies into a 6-stage ring; an MMA warp issues 6 MMAs a step -- A's digit plane s
//     against B's planes 0 .. 5 - s, stored one after another along N, in one MMA of N = (6 - s) 32
//     into accumulators s .. 5 -- so each A plane is read once a step (21 separate MMAs would read it
//     21 times), into one of two accumulator sets; sixteen warps drain the other set (recombine,
//     write FP64 in the layout the next stage's slicing reads, rows fastest), so a job's epilogue
//     runs beside the next job's products.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fgt_exec.h"
#include "fgt_tc.cuh"

namespace fgt {

__device__ int g_oz_status;  // 1: a wait ran out (the CTA skipped its outputs), 2: its drain ran out too

namespace {

constexpr int kNst = 6;                          // pipeline stages (16-deep steps in flight: covers the DRAM latency)
constexpr int kWarps = 16;                       // slicing / epilogue warps; two more copy and issue MMAs
constexpr int kThreads = (kWarps + 2) * 32;
constexpr uint32_t kAPlane = 128 * 16 * 2;       // one digit plane of a 128 x 16 A tile (BF16)
constexpr uint32_t kAStage = kOzSlices * kAPlane;
constexpr uint32_t kBStage = kOzSlices * kOzMaxNp * 32;
constexpr uint32_t kAccCols = 256;               // one accumulator set: 6 x Np <= 192 columns
constexpr uint32_t kTmemCols = 2 * kAccCols;     // two sets: one job's epilogue beside the next one's MMAs
constexpr size_t kSmemBytes = (size_t)kNst * (kAStage + kBStage) + (2 * kNst + 4) * 8 + 16;

struct OzArgs {
  const Block *blocks;
  const OzGroup *groups;  // stage 2: its jobs' block groups
  const int64_t *leaves;
  const double *src;
  double *dst;
  const unsigned char *btab;
  const int32_t *bexp;
  int k, n1, nh;
  int lk;      // log2 k when k is a power of two (divisions by k and K become shifts), else -1
  int64_t ss;  // complex values per expansion slot
};

// x / k and x / K (K = 2^dl k) by shifts when k is a power of two
__device__ __forceinline__ int div_k(int x, const OzArgs &a) { return a.lk >= 0 ? (x >> a.lk) : x / a.k; }
__device__ __forceinline__ int div_K(int x, const Block &blk, const OzArgs &a) {
  return a.lk >= 0 ? (x >> (a.lk + blk.dl)) : x / blk.K;
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Biased exponent field of x (0 for zero and subnormal values, which slice to zero).
__device__ __forceinline__ int exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// The six digits of x against its row's largest biased exponent ebr: n = round(x 2^(47 - e_r)),
// e_r = ebr - 1022 (so |n| <= 2^47), n = sum_s d_s 2^(8 (5 - s)) with |d_s| <= 128.  Integer
// arithmetic only (GB300's FP64 conversions run on the narrow FP64 pipe), and 32-bit after one split:
// n = H 2^24 + L with L the sign-extended low 24 bits, then three balanced base-256 digits of each
// half (the top digit of each absorbs the last carry: |L| <= 2^23 and |H| <= 2^23 + 1 keep it
// within +-128).
__device__ __forceinline__ void slice6(double x, int ebr, int (&dg)[kOzSlices]) {
  const long long b = __double_as_longlong(x);
  const int eb = (int)((b >> 52) & 0x7FF);
  const int sh = ebr - eb + 6;  // >= 6: ebr is the row's largest
  long long n = 0;
  if (eb != 0 && sh >= 6 && sh < 60) {
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    n = (m + (1LL << (sh - 1))) >> sh;
    if (b < 0) n = -n;
  }
  int L = (int)((unsigned)n << 8) >> 8;
  int H = (int)((n - L) >> 24);
  dg[5] = (int)(signed char)L;
  L = (L - dg[5]) >> 8;
  dg[4] = (int)(signed char)L;
  dg[3] = (L - dg[4]) >> 8;
  dg[2] = (int)(signed char)H;
  H = (H - dg[2]) >> 8;
  dg[1] = (int)(signed char)H;
  dg[0] = (H - dg[1]) >> 8;
}

// Two digits (|d| <= 128) as a BF16 pair, d0 in the low half: small integer -> FP32 (exact, by the
// 1.5 2^23 offset) -> BF16 (exact: at most 8 significant bits).
__device__ __forceinline__ uint32_t bf16_pair(int d0, int d1) {
  const float f0 = __int_as_float(0x4B400000 + d0) - 12582912.0f;
  const float f1 = __int_as_float(0x4B400000 + d1) - 12582912.0f;
  const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// Stage layouts (block of K nodes a side, leaves of k nodes, nl = K / k leaves a side):
//   0  rows (J2, J1), q = J3            sigma (leaf values, node j1 fastest)  -> X[(m3, c)][rows]
//   1  rows (m3, J1), q = (c, J2)       X                                      -> Y[(m2, c)][rows]
//   2  rows (m3, m2), q = (c, J1)       Y                                      -> phi slot [m3][m2][m1][c]
//   3  rows (m3, m2), q = (m1, c)       psi slot                               -> X[(c, I1)][rows]
//   4  rows (I1, m3), q = (c, m2)       X                                      -> Y[(c, I2)][rows]
//   5  rows (I2, I1), q = (c, m3)       Y                                      -> u (leaf values), real part
// Row r's fixed part of its operand addresses, then the element index of q.
struct RowAddr {
  int64_t base;
  int a, b;  // kind 0: leaf index part (o2 nl + o1) and node offset (j2 k + j1); kind 2: m3, m2
  int K;     // kind 2, a group of one block: its K (base is then the row's base), else 0
};

template <int KIND>
__device__ __forceinline__ RowAddr row_addr(int r, const OzJob &job, const Block &blk, const OzArgs &a) {
  const int K = blk.K, k = a.k, n1 = a.n1, nh = a.nh, nl = 1 << blk.dl;
  RowAddr ra{0, 0, 0, 0};
  if constexpr (KIND == 0) {
    const int J2 = div_K(r, blk, a), J1 = r - J2 * K, o2 = div_k(J2, a), o1 = div_k(J1, a);
    ra.a = o2 * nl + o1;
    ra.b = (J2 - o2 * k) * k + (J1 - o1 * k);
  } else if constexpr (KIND == 1) {
    const int m3 = div_K(r, blk, a), J1 = r - m3 * K;
    ra.base = job.scr + (int64_t)m3 * 2 * K * K + J1;
  } else if constexpr (KIND == 2) {  // a group of blocks: the member's base is found per q
    ra.a = r / n1;                  // m3
    ra.b = r - ra.a * n1;           // m2
  } else if constexpr (KIND == 3) {
    ra.base = (int64_t)blk.slot * 2 * a.ss + (int64_t)r * 2 * n1;
  } else if constexpr (KIND == 4) {
    const int I1 = r / nh, m3 = r - I1 * nh;
    ra.base = job.scr + (int64_t)I1 * nh * n1 + (int64_t)m3 * n1;
  } else {
    const int I2 = div_K(r, blk, a), I1 = r - I2 * K;
    ra.base = job.scr + (int64_t)I2 * K * nh + (int64_t)I1 * nh;
  }
  return ra;
}

template <int KIND>
__device__ __forceinline__ int64_t a_index(const RowAddr &ra, int q, const int64_t *lv, const Block &blk,
                                           const OzArgs &a, const OzGroup *g = nullptr) {
  const int K = blk.K, k = a.k, n1 = a.n1, nh = a.nh, nl = 1 << blk.dl;
  if constexpr (KIND == 0) {
    const int o3 = div_k(q, a), j3 = q - o3 * k;
    return __ldg(lv + (int64_t)o3 * nl * nl + ra.a) * (int64_t)k * k * k + (int64_t)j3 * k * k + ra.b;
  } else if constexpr (KIND == 1) {
    const int c = q >= K, J2 = q - c * K;
    return ra.base + (int64_t)c * K * K + (int64_t)J2 * K;
  } else if constexpr (KIND == 2) {
    if (ra.K > 0) {  // one member: as for a single block
      const int c = q >= ra.K, J1 = q - c * ra.K;
      return ra.base + (int64_t)c * nh * ra.K + J1;
    }
    int j = 0;  // the member whose contraction holds q
    while (j + 1 < g->n && q >= g->q0[j + 1]) ++j;
    const int Kj = g->K[j], ql = q - g->q0[j], c = ql >= Kj, J1 = ql - c * Kj;
    return g->scr[j] + ((int64_t)ra.b * 2 + c) * nh * Kj + (int64_t)ra.a * Kj + J1;
  } else if constexpr (KIND == 3) {
    return ra.base + q;
  } else if constexpr (KIND == 4) {
    const int c = q >= n1, m2 = q - c * n1;
    return ra.base + (int64_t)c * K * nh * n1 + m2;
  } else {
    const int c = q >= nh, m3 = q - c * nh;
    return ra.base + (int64_t)c * K * K * nh + m3;
  }
}

template <int KIND>
__device__ __forceinline__ void store_out(int r, int n, double v, const OzJob &job, const Block &blk,
                                          const OzDims &dm, const int64_t *lv, const OzArgs &a, int slot = 0) {
  if constexpr (KIND == 2) {
    double *p = a.dst + (int64_t)slot * 2 * a.ss + (int64_t)r * 2 * a.n1 + n;
    if (job.flags & 1) atomicAdd(p, v);
    else *p = v;
  } else if constexpr (KIND == 5) {
    const int K = blk.K, k = a.k, nl = 1 << blk.dl;
    const int I2 = div_K(r, blk, a), I1 = r - I2 * K, I3 = n;
    const int o1 = div_k(I1, a), o2 = div_k(I2, a), o3 = div_k(I3, a);
    double *p = a.dst + __ldg(lv + ((int64_t)o3 * nl + o2) * nl + o1) * (int64_t)k * k * k +
                ((int64_t)(I3 - o3 * k) * k + (I2 - o2 * k)) * k + (I1 - o1 * k);
    if (job.flags & 1) atomicAdd(p, v);
    else *p = v;
  } else {
    a.dst[job.scr + (int64_t)n * dm.R + r] = v;
  }
}

// A job's stage dimensions: its block's, or for stage 2 its group's (the concatenated contraction).
template <int KIND>
__device__ __forceinline__ OzDims job_dims(const OzJob &job, const OzArgs &a) {
  if constexpr (KIND == 2) {
    const OzGroup *g = a.groups + job.blk;
    return oz_dims_group(a.n1, a.nh, __ldg(&g->q0[__ldg(&g->n)]));
  } else {
    return oz_dims(KIND, __ldg(&a.blocks[job.blk].K), a.n1, a.nh);
  }
}

// Slicing: one CTA per (block, 128-row tile).  Sixteen warps, 8 rows each, 4 lanes a row; every
// thread finds its row's largest exponent (with its 3 partner lanes), then cuts its elements into
// the six digit planes of each 16-deep step, in the tensor cores' K-major core-matrix layout
// (conflict-free, coalesced 4-byte stores: a warp writes one 128-byte core-matrix row set).
template <int KIND>
__global__ void __launch_bounds__(kWarps * 32) oz_slice_kernel(const OzArgs a, const OzJob *__restrict__ sjobs,
                                                               unsigned char *__restrict__ dig,
                                                               int *__restrict__ rexp) {
  const OzJob job = sjobs[blockIdx.x];
  __shared__ OzGroup grp;  // stage 2: the job's group of blocks
  Block blk{};
  OzDims dm;
  if constexpr (KIND == 2) {
    if (threadIdx.x == 0) grp = a.groups[job.blk];
    __syncthreads();
    dm = oz_dims_group(a.n1, a.nh, grp.q0[grp.n]);
  } else {
    blk = a.blocks[job.blk];
    dm = oz_dims(KIND, blk.K, a.n1, a.nh);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t *lv = a.leaves + blk.leaf0;
  const int rl = 8 * warp + (lane >> 2), sub = lane & 3;
  const int rg = (int)job.tile * 128 + rl;
  const bool rvalid = rg < dm.R;
  RowAddr ra = row_addr<KIND>(rvalid ? rg : 0, job, blk, a);
  if constexpr (KIND == 2) {
    if (grp.n == 1) {
      ra.K = grp.K[0];
      ra.base = grp.scr[0] + ((int64_t)ra.b * 2 * a.nh + ra.a) * ra.K;  // (m2 2 nh + m3) K
    }
  }
  int ebr = 0;
  if (rvalid)
    for (int q = 2 * sub; q < dm.Q; q += 8) {
      ebr = max(ebr, exp_field(__ldg(a.src + a_index<KIND>(ra, q, lv, blk, a, &grp))));
      if (q + 1 < dm.Q) ebr = max(ebr, exp_field(__ldg(a.src + a_index<KIND>(ra, q + 1, lv, blk, a, &grp))));
    }
  ebr = max(ebr, __shfl_xor_sync(0xffffffffu, ebr, 1));
  ebr = max(ebr, __shfl_xor_sync(0xffffffffu, ebr, 2));
  if (sub == 0) rexp[job.roff + rl] = ebr;
  unsigned char *out = dig + job.aoff;
  const uint32_t off0 = (uint32_t)(rl >> 3) * 256u + (uint32_t)(rl & 7) * 16u + (uint32_t)sub * 4u;
#pragma unroll 2
  for (int ks = 0; ks < dm.nks; ++ks) {
#pragma unroll
    for (int kg = 0; kg < 2; ++kg) {
      const int q = ks * 16 + kg * 8 + 2 * sub;
      const double x0 = (rvalid && q < dm.Q) ? __ldg(a.src + a_index<KIND>(ra, q, lv, blk, a, &grp)) : 0.0;
      const double x1 = (rvalid && q + 1 < dm.Q) ? __ldg(a.src + a_index<KIND>(ra, q + 1, lv, blk, a, &grp)) : 0.0;
      int g0[kOzSlices], g1[kOzSlices];
      slice6(x0, ebr, g0);
      slice6(x1, ebr, g1);
      unsigned char *o = out + (size_t)ks * kAStage + off0 + (uint32_t)kg * 128u;
#pragma unroll
      for (int sl = 0; sl < kOzSlices; ++sl) *reinterpret_cast<uint32_t *>(o + sl * kAPlane) = bf16_pair(g0[sl], g1[sl]);
    }
  }
}

// Bounded wait for a phase that other warps complete: like mbar_wait, but each try may suspend the
// thread for up to about 0.1 ms, so that waiting warps do not take issue slots from working ones.
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t mbar, uint32_t parity, long long limit = 1LL << 31) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity), "r"(100000u)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// Products: a persistent kernel, one CTA per SM over the stage's (block, tile, column part) jobs
// (job j = blockIdx.x + i gridDim.x).  Warp 16 copies the digit planes of every step of every job
// into a 6-stage ring (bulk copies, complete_tx on the stage's `full` barrier), warp 17 issues the
// MMAs into one of two accumulator sets in tensor memory (job i in set i mod 2), and sixteen warps
// drain the other set meanwhile: the epilogue of one job overlaps the products of the next.
template <int KIND>
__global__ void __launch_bounds__(kThreads, 1) oz_mma_kernel(const OzArgs a, const OzJob *__restrict__ jobs,
                                                              int64_t njobs, const unsigned char *__restrict__ dig,
                                                              const int *__restrict__ rexp) {
  extern __shared__ __align__(1024) unsigned char sm_oz[];
  unsigned char *sA = sm_oz;
  unsigned char *sB = sm_oz + kNst * kAStage;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + kNst * kBStage);
  uint64_t *full = bars, *empty = bars + kNst, *tfull = bars + 2 * kNst, *tempty = tfull + 2;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(tempty + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == kWarps * 32) {
    for (int i = 0; i < kNst; ++i) {
      mbar_init(full + i, 2);  // the two bulk copies' expect_tx arrivals
      mbar_init(empty + i, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);        // the MMAs of a job, committed
      mbar_init(tempty + b, kWarps);  // every epilogue warp done reading the set
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int nmine = njobs > blockIdx.x ? (int)((njobs - 1 - blockIdx.x) / gridDim.x) + 1 : 0;

  if (warp == kWarps) {
    // ---- copies: every step of every job, in order, through the ring
    if (lane == 0) {
      int g = 0;  // steps issued so far (all jobs)
      OzJob next = nmine > 0 ? jobs[blockIdx.x] : OzJob{};
      for (int li = 0; li < nmine && !*abort_flag; ++li) {
        const OzJob job = next;
        if (li + 1 < nmine) next = jobs[blockIdx.x + (int64_t)(li + 1) * gridDim.x];  // in flight meanwhile
        const uint32_t bbytes = (uint32_t)(kOzSlices * job.np * 32);
        for (int ks = 0; ks < job.nks; ++ks, ++g) {
          const int st = g % kNst;
          if (g >= kNst && !mbar_wait(smem_addr(empty + st), (uint32_t)((g / kNst - 1) & 1))) {
            *abort_flag = 1;
            atomicMax(&g_oz_status, 1);
            break;
          }
          bulk_copy_g2s(smem_addr(sA + st * kAStage), dig + job.aoff + (size_t)ks * kAStage, kAStage,
                        smem_addr(full + st));
          bulk_copy_g2s(smem_addr(sB + st * kBStage), a.btab + job.boff + (size_t)ks * bbytes, bbytes,
                        smem_addr(full + st));
        }
      }
      // the copies in flight land before the CTA's shared memory is released: the last kNst steps'
      // `full` phases (the MMA warp waits for them too unless it gave up)
      for (int h = max(0, g - kNst); h < g; ++h)
        if (!mbar_wait(smem_addr(full + h % kNst), (uint32_t)((h / kNst) & 1))) atomicMax(&g_oz_status, 2);
    }
  } else if (warp == kWarps + 1) {
    // ---- products: 6 MMAs a step (A's plane s against B's planes 0 .. 5 - s, one N = (6 - s) Np MMA)
    if (lane == 0) {
      int g = 0;
      OzJob next = nmine > 0 ? jobs[blockIdx.x] : OzJob{};
      for (int li = 0; li < nmine && !*abort_flag; ++li) {
        const OzJob job = next;
        if (li + 1 < nmine) next = jobs[blockIdx.x + (int64_t)(li + 1) * gridDim.x];
        const int Np = job.np, nks = job.nks;
        const int b = li & 1;
        if (li >= 2 && !mbar_wait(smem_addr(tempty + b), (uint32_t)((li / 2 - 1) & 1))) {
          *abort_flag = 1;
          atomicMax(&g_oz_status, 1);
          // the epilogue may stop before the previous job's commit: its products (the commit covers
          // every earlier MMA of this thread) finish before the CTA frees tensor memory
          if (!mbar_wait(smem_addr(tfull + (b ^ 1)), (uint32_t)(((li - 1) / 2) & 1))) atomicMax(&g_oz_status, 2);
          break;
        }
        tc_fence_after();
        uint32_t idesc[kOzSlices];
#pragma unroll
        for (int s = 0; s < kOzSlices; ++s) idesc[s] = idesc_bf16(128, (kOzSlices - s) * Np);
        const uint32_t d0 = tmem + (uint32_t)(b * kAccCols);
        bool ok = true;
        for (int ks = 0; ks < nks; ++ks, ++g) {
          const int st = g % kNst;
          if (!mbar_wait(smem_addr(full + st), (uint32_t)((g / kNst) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t aa = smem_addr(sA + st * kAStage), ba = smem_addr(sB + st * kBStage);
#pragma unroll
          for (int s = 0; s < kOzSlices; ++s)
            umma_bf16(d0 + (uint32_t)(s * Np), umma_desc(aa + s * kAPlane, 256), umma_desc(ba, 256), idesc[s],
                      (ks > 0 || s > 0) ? 1u : 0u);
          umma_commit(smem_addr(empty + st));
        }
        if (!ok) {
          *abort_flag = 1;
          atomicMax(&g_oz_status, 1);
        }
        umma_commit(smem_addr(tfull + b));  // this job's accumulators are complete (or abandoned)
        if (!ok) {
          // the abandoned job's products finish before the CTA frees tensor memory
          if (!mbar_wait(smem_addr(tfull + b), (uint32_t)((li / 2) & 1))) atomicMax(&g_oz_status, 2);
          break;
        }
      }
    }
  } else {
    // ---- epilogue: six accumulators per output -> 64-bit integer -> FP64, in the next stage's layout
    const int lq = warp & 3, cg = warp >> 2;  // TMEM lane quarter, column quarter
    const int r = lq * 32 + lane;
    for (int li = 0; li < nmine; ++li) {
      const OzJob job = jobs[blockIdx.x + (int64_t)li * gridDim.x];
      const Block blk = KIND == 2 ? Block{} : a.blocks[job.blk];
      const OzDims dm = job_dims<KIND>(job, a);
      const int slot = KIND == 2 ? __ldg(&a.groups[job.blk].slot) : blk.slot;
      const int b = li & 1;
      int ok = 1;
      if (lane == 0) ok = mbar_wait_sleep(smem_addr(tfull + b), (uint32_t)((li / 2) & 1)) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      tc_fence_after();
      if (!ok) {
        if (lane == 0) atomicMax(&g_oz_status, 2);
        break;
      }
      if (__shfl_sync(0xffffffffu, *abort_flag, 0)) break;
      const int64_t *lv = a.leaves + blk.leaf0;
      const int r0 = (int)job.tile * 128, c0 = (int)job.part * dm.Nc, ncol = min(dm.Nc, dm.N - c0);
      const int rgl = r0 + r, cw = dm.Np / 4, cbeg = cg * cw;  // cw = 4 or 8 columns a warp
      const int sc0 = __ldg(rexp + job.roff + r) - 1022 - 54;
      const uint32_t tl = tmem + (uint32_t)(b * kAccCols) + ((uint32_t)(lq * 32) << 16) + (uint32_t)cbeg;
      uint32_t v[kOzSlices][8];
      if (cw == 8) {
#pragma unroll
        for (int D = 0; D < kOzSlices; ++D) tmem_ld8_nw(tl + (uint32_t)(D * dm.Np), v[D]);
      } else {
#pragma unroll
        for (int D = 0; D < kOzSlices; ++D) tmem_ld4_nw(tl + (uint32_t)(D * dm.Np), v[D]);
      }
      tmem_wait_ld();
      // the accumulator set is in registers: hand it back to the MMA warp before the arithmetic
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty + b);
      if (rgl < dm.R) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int cl = cbeg + j;
          if (j < cw && cl < ncol) {
            long long V = 0;
#pragma unroll
            for (int D = 0; D < kOzSlices; ++D) V = V * 256 + (long long)__float2int_rn(__uint_as_float(v[D][j]));
            store_out<KIND>(rgl, c0 + cl, i64_to_f64_scaled(V, sc0 + __ldg(a.bexp + job.eoff + cl)), job, blk, dm,
                            lv, a, slot);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

template <int KIND>
cudaError_t launch_kind(const OzArgs &a, const ExecDesc &e, cudaStream_t st) {
  const int64_t ns = e.oz_nsjobs[KIND], nj = e.oz_njobs[KIND];
  oz_slice_kernel<KIND><<<(unsigned)ns, kWarps * 32, 0, st>>>(a, e.oz_sjobs[KIND], e.oz_dig, e.oz_rexp);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if ((err = cudaFuncSetAttribute(oz_mma_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmemBytes)) != cudaSuccess)
    return err;
  int dev = 0, nsm = 0;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
  const unsigned grid = (unsigned)std::min<int64_t>(nj, std::max(nsm, 1));
  oz_mma_kernel<KIND><<<grid, kThreads, kSmemBytes, st>>>(a, e.oz_jobs[KIND], nj, e.oz_dig, e.oz_rexp);
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_oz_stage(const ExecDesc &e, int kind, const double *src, double *dst, cudaStream_t st) {
  if (kind < 0 || kind > 5) return cudaErrorInvalidValue;
  const int64_t nj = e.oz_njobs[kind];
  if (nj == 0) return cudaSuccess;
  if (e.oz_dig == nullptr || e.oz_rexp == nullptr) return cudaErrorInvalidValue;
  int lk = -1;
  for (int t = 0; t < 8; ++t)
    if ((1 << t) == e.k) lk = t;
  OzArgs a{kind < 3 ? e.blocks : e.eval_blocks, e.oz_groups, kind < 3 ? e.block_leaves : e.eval_leaves,
           src, dst, e.oz_btab, e.oz_bexp, e.k, e.n1, e.nh, lk, e.slot_size};
  switch (kind) {
    case 0: return launch_kind<0>(a, e, st);
    case 1: return launch_kind<1>(a, e, st);
    case 2: return launch_kind<2>(a, e, st);
    case 3: return launch_kind<3>(a, e, st);
    case 4: return launch_kind<4>(a, e, st);
    default: return launch_kind<5>(a, e, st);
  }
}

cudaError_t read_oz_status(int *status) {
  int v = 0;
  cudaError_t err = cudaMemcpyFromSymbol(&v, g_oz_status, sizeof(int));
  if (err != cudaSuccess) return err;
  if (v != 0) {
    const int zero = 0;
    if ((err = cudaMemcpyToSymbol(g_oz_status, &zero, sizeof(int))) != cudaSuccess) return err;
  }
  *status = v;
  return cudaSuccess;
}

}  // namespace fgt
