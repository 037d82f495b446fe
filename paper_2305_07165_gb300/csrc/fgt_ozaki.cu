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
// The products dropped (s + t >= 6) and the two 47-bit roundings bound the error of C[r][n] by
// about 2^-46 sum_q |A[r][q]| |B[q][n]| -- FP64 quality for a contraction, and 21 BF16 MMAs per
// 16-deep step where a 3xTF32 product needs 3.
//
// Each stage is one contraction of the block's separable product (form: x3, x2, x1; evaluation:
// m1, m2, m3, the last one keeping the real part), one launch over (block, 128-row tile, column
// part) jobs.  A CTA streams its rows' FP64 operand through four pipeline stages: sixteen warps
// read and slice 128 x 16 tiles into shared memory (the K-major no-swizzle operand layout), one
// thread copies the pre-sliced 1D matrix of each 16-deep step with bulk asynchronous copies and
// issues the MMAs; the epilogue reads the six accumulators, recombines and writes FP64 in the
// layout the next stage reads (rows fastest, so that the warp's stores are contiguous).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fgt_exec.h"
#include "fgt_tc.cuh"

namespace fgt {

__device__ int g_oz_status;  // 1: a wait ran out (the CTA skipped its outputs), 2: its drain ran out too

namespace {

constexpr int kNst = 4;                          // pipeline stages (16-deep steps in flight)
constexpr int kWarps = 16;                       // slicing / epilogue warps; one more issues copies + MMAs
constexpr int kThreads = (kWarps + 1) * 32;
constexpr uint32_t kAPlane = 128 * 16 * 2;       // one digit plane of a 128 x 16 A tile (BF16)
constexpr uint32_t kAStage = kOzSlices * kAPlane;
constexpr uint32_t kBStage = kOzSlices * kOzMaxNp * 32;
constexpr uint32_t kTmemCols = 512;              // 6 accumulators x Np <= 480 columns
constexpr size_t kSmemBytes =
    (size_t)kNst * (kAStage + kBStage) + 128 * sizeof(int) + kOzMaxNp * sizeof(int) + (3 * kNst + 1) * 8 + 16;

struct OzArgs {
  const OzJob *jobs;
  const Block *blocks;
  const int64_t *leaves;
  const double *src;
  double *dst;
  const unsigned char *btab;
  const int32_t *bexp;
  int k, n1, nh;
  int64_t ss;  // complex values per expansion slot
};

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

// The six digits of x against its row's largest biased exponent ebr, as BF16 bit patterns:
// n = round(x 2^(47 - e_r)), e_r = ebr - 1022 (so |n| <= 2^47), n = sum_s d_s 2^(8 (5 - s)) with
// balanced digits.  Integer arithmetic only: GB300's FP64 conversions run on the narrow FP64 pipe.
__device__ __forceinline__ void slice6(double x, int ebr, uint32_t (&h)[kOzSlices]) {
  const long long b = __double_as_longlong(x);
  const int eb = (int)((b >> 52) & 0x7FF);
  const int sh = ebr - eb + 6;  // >= 6: ebr is the row's largest
  long long n = 0;
  if (eb != 0 && sh >= 6 && sh < 60) {
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    n = (m + (1LL << (sh - 1))) >> sh;
    if (b < 0) n = -n;
  }
  int dg[kOzSlices];
#pragma unroll
  for (int s = kOzSlices - 1; s >= 1; --s) {
    const int lo = (((int)n + 128) & 255) - 128;  // balanced digit of n mod 256
    dg[s] = lo;
    n = (n - lo) >> 8;
  }
  dg[0] = (int)n;
#pragma unroll
  for (int s = 0; s < kOzSlices; ++s)  // small integer -> FP32 (exact) -> its upper half, the BF16
    h[s] = __float_as_uint(__int_as_float(0x4B400000 + dg[s]) - 12582912.0f) >> 16;
}

// v 2^sc rounded to FP64 (nearest, ties to even), with integer operations.
__device__ __forceinline__ double i64_to_f64_scaled(long long v, int sc) {
  if (v == 0) return 0.0;
  const unsigned long long sg = v < 0 ? (1ULL << 63) : 0ULL;
  unsigned long long a = v < 0 ? 0ULL - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  a <<= lz;
  unsigned long long m = a >> 11;
  const unsigned rem = (unsigned)(a & 0x7FF);
  if (rem > 0x400u || (rem == 0x400u && (m & 1ULL))) ++m;
  int E = 1023 + 63 - lz + sc;
  if (m >> 53) {
    m >>= 1;
    ++E;
  }
  if (E <= 0) return __longlong_as_double((long long)sg);
  if (E >= 2047) return __longlong_as_double((long long)(sg | 0x7FF0000000000000ULL));
  return __longlong_as_double((long long)(sg | ((unsigned long long)E << 52) | (m & 0xFFFFFFFFFFFFFULL)));
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
  int a, b;  // kind 0: leaf index part (o2 nl + o1) and node offset (j2 k + j1)
};

template <int KIND>
__device__ __forceinline__ RowAddr row_addr(int r, const OzJob &job, const Block &blk, const OzArgs &a) {
  const int K = blk.K, k = a.k, n1 = a.n1, nh = a.nh, nl = 1 << blk.dl;
  RowAddr ra{0, 0, 0};
  if constexpr (KIND == 0) {
    const int J2 = r / K, J1 = r - J2 * K, o2 = J2 / k, o1 = J1 / k;
    ra.a = o2 * nl + o1;
    ra.b = (J2 - o2 * k) * k + (J1 - o1 * k);
  } else if constexpr (KIND == 1) {
    const int m3 = r / K, J1 = r - m3 * K;
    ra.base = job.scr + (int64_t)m3 * 2 * K * K + J1;
  } else if constexpr (KIND == 2) {
    const int m3 = r / n1, m2 = r - m3 * n1;
    ra.base = job.scr + (int64_t)m2 * 2 * nh * K + (int64_t)m3 * K;
  } else if constexpr (KIND == 3) {
    ra.base = (int64_t)blk.slot * 2 * a.ss + (int64_t)r * 2 * n1;
  } else if constexpr (KIND == 4) {
    const int I1 = r / nh, m3 = r - I1 * nh;
    ra.base = job.scr + (int64_t)I1 * nh * n1 + (int64_t)m3 * n1;
  } else {
    const int I2 = r / K, I1 = r - I2 * K;
    ra.base = job.scr + (int64_t)I2 * K * nh + (int64_t)I1 * nh;
  }
  return ra;
}

template <int KIND>
__device__ __forceinline__ int64_t a_index(const RowAddr &ra, int q, const int64_t *lv, const Block &blk,
                                           const OzArgs &a) {
  const int K = blk.K, k = a.k, n1 = a.n1, nh = a.nh, nl = 1 << blk.dl;
  if constexpr (KIND == 0) {
    const int o3 = q / k, j3 = q - o3 * k;
    return __ldg(lv + (int64_t)o3 * nl * nl + ra.a) * (int64_t)k * k * k + (int64_t)j3 * k * k + ra.b;
  } else if constexpr (KIND == 1) {
    const int c = q >= K, J2 = q - c * K;
    return ra.base + (int64_t)c * K * K + (int64_t)J2 * K;
  } else if constexpr (KIND == 2) {
    const int c = q >= K, J1 = q - c * K;
    return ra.base + (int64_t)c * nh * K + J1;
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
                                          const OzDims &dm, const int64_t *lv, const OzArgs &a) {
  if constexpr (KIND == 2) {
    double *p = a.dst + (int64_t)blk.slot * 2 * a.ss + (int64_t)r * 2 * a.n1 + n;
    if (job.flags & 1) atomicAdd(p, v);
    else *p = v;
  } else if constexpr (KIND == 5) {
    const int K = blk.K, k = a.k, nl = 1 << blk.dl;
    const int I2 = r / K, I1 = r - I2 * K, I3 = n;
    const int o1 = I1 / k, o2 = I2 / k, o3 = I3 / k;
    double *p = a.dst + __ldg(lv + ((int64_t)o3 * nl + o2) * nl + o1) * (int64_t)k * k * k +
                ((int64_t)(I3 - o3 * k) * k + (I2 - o2 * k)) * k + (I1 - o1 * k);
    if (job.flags & 1) atomicAdd(p, v);
    else *p = v;
  } else {
    a.dst[job.scr + (int64_t)n * dm.R + r] = v;
  }
}

template <int KIND>
__global__ void __launch_bounds__(kThreads, 1) oz_stage_kernel(const OzArgs a) {
  extern __shared__ __align__(1024) unsigned char sm_oz[];
  unsigned char *sA = sm_oz;
  unsigned char *sB = sm_oz + kNst * kAStage;
  int *rowexp = reinterpret_cast<int *>(sB + kNst * kBStage);
  int *colexp = rowexp + 128;
  uint64_t *bars = reinterpret_cast<uint64_t *>(colexp + kOzMaxNp);
  uint64_t *afull = bars, *bfull = bars + kNst, *empty = bars + 2 * kNst, *done = bars + 3 * kNst;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);

  const OzJob job = a.jobs[blockIdx.x];
  const Block blk = a.blocks[job.blk];
  const OzDims dm = oz_dims(KIND, blk.K, a.n1, a.nh);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t *lv = a.leaves + blk.leaf0;
  const int r0 = (int)job.tile * 128;
  const int c0 = (int)job.part * dm.Nc;
  const int ncol = min(dm.Nc, dm.N - c0);
  const int Np = dm.Np;
  const uint32_t bbytes = (uint32_t)(kOzSlices * Np * 32);

  if (threadIdx.x == kWarps * 32) {
    for (int i = 0; i < kNst; ++i) {
      mbar_init(afull + i, kWarps);
      mbar_init(bfull + i, 1);
      mbar_init(empty + i, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int i = threadIdx.x; i < kOzMaxNp; i += blockDim.x) colexp[i] = i < ncol ? __ldg(a.bexp + job.eoff + i) : 0;

  // this thread's row for the operand pass: 8 rows a warp, 4 lanes a row (q = 8 i + 2 sub + {0, 1})
  const int rl = 8 * (warp & (kWarps - 1)) + (lane >> 2), sub = lane & 3;
  const int rg = r0 + rl;
  const bool rvalid = warp < kWarps && rg < dm.R;
  const RowAddr ra = row_addr<KIND>(rvalid ? rg : 0, job, blk, a);
  int ebr = 0;
  if (warp < kWarps) {
    if (rvalid)
      for (int q = 2 * sub; q < dm.Q; q += 8) {
        ebr = max(ebr, exp_field(__ldg(a.src + a_index<KIND>(ra, q, lv, blk, a))));
        if (q + 1 < dm.Q) ebr = max(ebr, exp_field(__ldg(a.src + a_index<KIND>(ra, q + 1, lv, blk, a))));
      }
    ebr = max(ebr, __shfl_xor_sync(0xffffffffu, ebr, 1));
    ebr = max(ebr, __shfl_xor_sync(0xffffffffu, ebr, 2));
    if (sub == 0) rowexp[rl] = ebr;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp < kWarps) {
    // ---- slicing: the rows' 16-deep steps into the digit planes of the ring
    for (int ks = 0; ks < dm.nks; ++ks) {
      const int st = ks % kNst;
      int ok = 1;
      if (lane == 0) {
        if (ks >= kNst) ok = mbar_wait(smem_addr(empty + st), (uint32_t)((ks / kNst - 1) & 1)) ? 1 : 0;
        if (!ok) {
          *abort_flag = 1;
          atomicMax(&g_oz_status, 1);
        }
        ok = ok && !*abort_flag;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      unsigned char *as = sA + st * kAStage;
#pragma unroll
      for (int kg = 0; kg < 2; ++kg) {
        const int q = ks * 16 + kg * 8 + 2 * sub;
        const double x0 = (rvalid && q < dm.Q) ? __ldg(a.src + a_index<KIND>(ra, q, lv, blk, a)) : 0.0;
        const double x1 = (rvalid && q + 1 < dm.Q) ? __ldg(a.src + a_index<KIND>(ra, q + 1, lv, blk, a)) : 0.0;
        uint32_t h0[kOzSlices], h1[kOzSlices];
        slice6(x0, ebr, h0);
        slice6(x1, ebr, h1);
        // K-major core-matrix layout: 8-row groups 256 bytes apart, the two 8-deep halves 128
        const uint32_t off = (uint32_t)(rl >> 3) * 256u + (uint32_t)kg * 128u + (uint32_t)(rl & 7) * 16u + (uint32_t)sub * 4u;
#pragma unroll
        for (int s = 0; s < kOzSlices; ++s) *reinterpret_cast<uint32_t *>(as + s * kAPlane + off) = h0[s] | (h1[s] << 16);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> the MMAs' reads
      __syncwarp();
      if (lane == 0) mbar_arrive(afull + st);
    }
  } else if (lane == 0) {
    // ---- the 1D matrix's digit planes by bulk copies, and the MMAs
    const unsigned char *bsrc = a.btab + job.boff;
    const int nks = dm.nks;
    int issued = 0;
    for (; issued < min(kNst, nks); ++issued)
      bulk_copy_g2s(smem_addr(sB + issued * kBStage), bsrc + (size_t)issued * bbytes, bbytes, smem_addr(bfull + issued));
    const uint32_t idesc = idesc_bf16(128, Np);
    bool ok = true;
    int ks = 0;
    for (; ks < nks; ++ks) {
      const int st = ks % kNst;
      const uint32_t par = (uint32_t)((ks / kNst) & 1);
      if (!mbar_wait(smem_addr(bfull + st), par) || !mbar_wait(smem_addr(afull + st), par)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t aa = smem_addr(sA + st * kAStage), ba = smem_addr(sB + st * kBStage);
#pragma unroll
      for (int s = 0; s < kOzSlices; ++s)
#pragma unroll
        for (int t = 0; t < kOzSlices - s; ++t)
          umma_bf16(tmem + (uint32_t)((s + t) * Np), umma_desc(aa + s * kAPlane, 256),
                    umma_desc(ba + (uint32_t)(t * Np * 32), 256), idesc, (ks > 0 || s > 0) ? 1u : 0u);
      umma_commit(smem_addr(empty + st));
      // refill the stage the previous step used, once its MMAs are done
      const int kn = ks + kNst - 1;
      if (ks >= 1 && kn < nks) {
        const int sp = (ks - 1) % kNst;
        if (!mbar_wait(smem_addr(empty + sp), (uint32_t)(((ks - 1) / kNst) & 1))) {
          ok = false;
          ++ks;
          break;
        }
        bulk_copy_g2s(smem_addr(sB + sp * kBStage), bsrc + (size_t)kn * bbytes, bbytes, smem_addr(bfull + sp));
        ++issued;
      }
    }
    if (!ok) {
      *abort_flag = 1;
      __threadfence_block();
      atomicMax(&g_oz_status, 1);
    }
    umma_commit(smem_addr(done));  // completes when every MMA issued above has
    if (!ok)  // the copies still in flight land before the CTA's shared memory is released
      for (int i = ks; i < issued; ++i)
        if (!mbar_wait(smem_addr(bfull + i % kNst), (uint32_t)((i / kNst) & 1))) atomicMax(&g_oz_status, 2);
  }

  // ---- epilogue: six accumulators per output -> 64-bit integer -> FP64, in the next stage's layout
  if (warp < kWarps) {
    int ok = 1;
    if (lane == 0) ok = mbar_wait(smem_addr(done), 0) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    tc_fence_after();
    if (!ok) {
      if (lane == 0) atomicMax(&g_oz_status, 2);
    } else if (!__shfl_sync(0xffffffffu, *abort_flag, 0)) {
      const int lq = warp & 3, cg = warp >> 2, cw = Np / 4;  // lane quarter, column quarter
      const int r = lq * 32 + lane, rgl = r0 + r;
      const int sc0 = rowexp[r] - 1022 - 54;
      const uint32_t tl = tmem + ((uint32_t)(lq * 32) << 16);
      for (int c = cg * cw; c < (cg + 1) * cw; c += 4) {
        uint32_t v[kOzSlices][4];
#pragma unroll
        for (int D = 0; D < kOzSlices; ++D) tmem_ld<4>(tl + (uint32_t)(D * Np + c), v[D]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int cl = c + j;
          if (rgl < dm.R && cl < ncol) {
            long long V = 0;
#pragma unroll
            for (int D = 0; D < kOzSlices; ++D) V = V * 256 + (long long)__float2int_rn(__uint_as_float(v[D][j]));
            store_out<KIND>(rgl, c0 + cl, i64_to_f64_scaled(V, sc0 + colexp[cl]), job, blk, dm, lv, a);
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
cudaError_t launch_kind(const OzArgs &a, int64_t njobs, cudaStream_t st) {
  cudaError_t err = cudaFuncSetAttribute(oz_stage_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
  if (err != cudaSuccess) return err;
  oz_stage_kernel<KIND><<<(unsigned)njobs, kThreads, kSmemBytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_oz_stage(const ExecDesc &e, int kind, const double *src, double *dst, cudaStream_t st) {
  if (kind < 0 || kind > 5) return cudaErrorInvalidValue;
  const int64_t nj = e.oz_njobs[kind];
  if (nj == 0) return cudaSuccess;
  OzArgs a{e.oz_jobs[kind], kind < 3 ? e.blocks : e.eval_blocks, kind < 3 ? e.block_leaves : e.eval_leaves,
           src, dst, e.oz_btab, e.oz_bexp, e.k, e.n1, e.nh, e.slot_size};
  switch (kind) {
    case 0: return launch_kind<0>(a, nj, st);
    case 1: return launch_kind<1>(a, nj, st);
    case 2: return launch_kind<2>(a, nj, st);
    case 3: return launch_kind<3>(a, nj, st);
    case 4: return launch_kind<4>(a, nj, st);
    default: return launch_kind<5>(a, nj, st);
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
