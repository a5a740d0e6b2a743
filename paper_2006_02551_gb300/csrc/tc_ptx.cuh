// Inline-PTX helpers of the tensor-core stage kernels for sm_103a: shared-
// memory matrix descriptors, tcgen05 products, commits and tensor-memory
// loads, mbarriers with bounded waits, bulk copies and the TF32 / BF16
// operand element.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace wadg {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, fixed 0b001 at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// instruction descriptor, kind::tf32: D f32, A and B tf32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

// instruction descriptor, kind::f16 with BF16 A and B: D f32, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the given phase parity; gives up (false) after about a second of
// global time, or after 2^24 polls, whichever comes first.  A product or an
// operand tile takes microseconds, so only a signal that never comes reaches
// the limit.
constexpr uint64_t kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  if (mbar_try_wait(a, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int i = 0; i < (1 << 24); ++i) {
    if (mbar_try_wait(a, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) break;
  }
  return false;
}

// try_wait that may suspend the thread in hardware for up to hint_ns
// nanoseconds while the phase is incomplete (instead of returning at once)
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t a, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
// mbar_wait with the waiting thread suspended between polls: gives up after
// about a second of global time (or 2^20 polls)
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t a, uint32_t parity) {
  if (mbar_try_wait(a, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int i = 0; i < (1 << 20); ++i) {
    if (mbar_try_wait_hint(a, parity, 20000u)) return true;
    if (global_ns() - t0 > kWaitLimitNs) break;
  }
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// this thread's lane of 2 / 4 consecutive TMEM columns (load and wait fused so
// the registers are valid when the statement ends)
__device__ __forceinline__ void tld2(uint32_t taddr, float* v) {
  uint32_t r0, r1;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r0), "=r"(r1)
      : "r"(taddr)
      : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
}
__device__ __forceinline__ void tld4(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
      : "r"(taddr)
      : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
}
__device__ __forceinline__ void tld6(uint32_t taddr, float* v) {
  tld4(taddr, v);
  tld2(taddr + 4, v + 4);
}

// 6 consecutive columns at each of two / four column addresses, one wait
// the same at two pairs of column addresses (two elements), one wait
__device__ __forceinline__ void tld_6x2x2(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1,
                                          float* v) {
  uint32_t r[24];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%24];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [%25];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%6, %7, %8, %9}, [%26];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10, %11}, [%27];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12, %13, %14, %15}, [%28];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%16, %17}, [%29];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%18, %19, %20, %21}, [%30];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%22, %23}, [%31];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
      : "r"(a0), "r"(a0 + 4), "r"(a1), "r"(a1 + 4), "r"(b0), "r"(b0 + 4), "r"(b1), "r"(b1 + 4)
      : "memory");
#pragma unroll
  for (int i = 0; i < 24; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tld_6x2(uint32_t a0, uint32_t a1, float* v) {
  uint32_t r[12];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%12];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [%13];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%6, %7, %8, %9}, [%14];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10, %11}, [%15];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11])
      : "r"(a0), "r"(a0 + 4), "r"(a1), "r"(a1 + 4)
      : "memory");
#pragma unroll
  for (int i = 0; i < 12; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tld_6x4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                        float* v) {
  tld_6x2(a0, a1, v);
  tld_6x2(a2, a3, v + 12);
}

// named barrier 1 among the compute warps (warp-aligned, nthreads a multiple of 32)
__device__ __forceinline__ void cbar_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
// the same barrier with an AND reduction of a per-thread flag
__device__ __forceinline__ bool cbar_and(int nthreads, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(nthreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

// bulk global -> shared copy (both addresses 16-byte aligned, size a
// multiple of 16) whose bytes complete on mbarrier `bar`
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// arrive on `bar` and add `bytes` to the transaction count its phase waits for
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// operand element: TF32 held in 32 bits (4 per 16-byte core-matrix row, 8 K
// per instruction) or BF16 (8 per core-matrix row, 16 K per instruction)
template <bool BF>
struct OpT {
  static constexpr int ES = BF ? 2 : 4;    // bytes
  static constexpr int CW = 16 / ES;       // K per core-matrix row
  static constexpr int KS = 2 * CW;        // K per instruction
};

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// TF32 round to nearest (ties away from zero) by integer operations on the
// FP32 bit pattern: add half of the dropped part, clear the 13 low bits
__device__ __forceinline__ float to_tf32_int(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// byte offset of (row r, k) in a K-major canonical tile: 8-row x 16-byte core
// matrices, K-adjacent core matrices lbo bytes apart, 8-row groups sbo apart.
// The field operands use lbo = 144 (one 16-byte gap per core matrix) so that
// consecutive K written by consecutive lanes fall on distinct banks.
template <bool BF>
__host__ __device__ constexpr uint32_t cofs(int r, int k, uint32_t sbo, uint32_t lbo) {
  using O = OpT<BF>;
  return static_cast<uint32_t>(r >> 3) * sbo + static_cast<uint32_t>(k / O::CW) * lbo +
         static_cast<uint32_t>(r & 7) * 16u + static_cast<uint32_t>(k % O::CW) * O::ES;
}

// one operand value, rounded to nearest in the operand type
template <bool BF>
__device__ __forceinline__ void put_op(unsigned char* p, float x) {
  if constexpr (BF) *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(x);
  else *reinterpret_cast<float*>(p) = to_tf32(x);
}

constexpr int rup8(int x) { return (x + 7) & ~7; }
constexpr int rup16(int x) { return (x + 15) & ~15; }


}  // namespace tc
}  // namespace wadg

namespace wadg {
namespace tc {

// this thread's lane of 8 / 16 consecutive TMEM columns (load and wait fused)
__device__ __forceinline__ void tld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// 8 consecutive columns at each of two column addresses, one wait
__device__ __forceinline__ void tld8x2(uint32_t a0, uint32_t a1, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(a0), "r"(a1)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 4 consecutive columns at each of four column addresses, one wait
__device__ __forceinline__ void tld4x4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                       float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%17];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%18];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12, %13, %14, %15}, [%19];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 4 consecutive columns at each of two column addresses, one wait
__device__ __forceinline__ void tld4x2(uint32_t a0, uint32_t a1, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%8];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%9];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(a0), "r"(a1)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// bulk shared -> global copy (both addresses 16-byte aligned, size a
// multiple of 16), tracked by the issuing thread's bulk group
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the issuing thread's committed bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// ... and have completed (their writes are performed)
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// prefetch a 16-byte-aligned global range (size a multiple of 16) into L2
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// named barrier id among nthreads threads (warp-aligned)
__device__ __forceinline__ void nbar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

}  // namespace tc
}  // namespace wadg

namespace wadg {
namespace tc {

// tensor-memory loads without the wait: several are issued back to back and
// one tmem_wait_ld() makes all their registers valid
__device__ __forceinline__ void tld16_nw(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tld8_nw(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tld4_nw(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// n consecutive columns (n a multiple of 4, at most 32) into r, no wait
template <int n>
__device__ __forceinline__ void tld_cols_nw(uint32_t taddr, uint32_t* r) {
  static_assert(n % 4 == 0 && n <= 32, "column count");
  constexpr int a16 = n >= 16 ? 1 : 0;
  constexpr int r1 = n - 16 * a16;
  if constexpr (a16) tld16_nw(taddr, r);
  constexpr int a16b = r1 >= 16 ? 1 : 0;
  if constexpr (a16b) tld16_nw(taddr + 16, r + 16);
  constexpr int r2 = r1 - 16 * a16b;
  constexpr int o2 = n - r2;
  if constexpr (r2 >= 8) tld8_nw(taddr + o2, r + o2);
  constexpr int r3 = r2 >= 8 ? r2 - 8 : r2;
  constexpr int o3 = n - r3;
  if constexpr (r3 >= 4) tld4_nw(taddr + o3, r + o3);
}

}  // namespace tc
}  // namespace wadg
