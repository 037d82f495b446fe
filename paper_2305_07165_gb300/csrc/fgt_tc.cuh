// Helpers shared by the kernel translation units: fifth-generation tensor-core plumbing (shared-
// memory addresses, matrix descriptors of the K-major no-swizzle operand layout, MMA commit,
// bounded mbarrier waits, tensor-memory fences and loads, bulk asynchronous copies; sm_100 family,
// PTX) and an integer-pipe int64 -> FP64 conversion.
#pragma once
#include <cstdint>

namespace fgt {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;                  // leading byte offset: next core matrix along K
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;        // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                            // descriptor version of the sm_100 family
  return d;                                          // base offset 0, no swizzle
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// Waits for the completion of the mbarrier phase of the given parity; gives up after `limit`
// clocks (by default 2^31, about one second) and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit = 1LL << 31) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Bulk asynchronous copy (the copy engine of the sm_90+ memory system): `bytes` (a multiple of 16,
// both addresses 16-byte aligned) from global to shared memory, completing on an mbarrier that
// the issuing thread armed for that many bytes.
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// tcgen05.ld of 4 or 8 consecutive columns for the warp's 32 lanes, without the wait (several loads
// in flight, then one tmem_wait_ld before the registers are read)
__device__ __forceinline__ void tmem_ld4_nw(uint32_t addr, uint32_t *v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(addr));
}
__device__ __forceinline__ void tmem_ld8_nw(uint32_t addr, uint32_t *v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(addr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t addr, uint32_t (&v)[N]) {
  if constexpr (N == 4) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(addr));
  } else if constexpr (N == 8) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(addr));
  } else if constexpr (N == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(addr));
  } else {
    static_assert(N == 32, "tmem_ld: 4, 8, 16 or 32 columns");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(addr));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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

}  // namespace fgt
