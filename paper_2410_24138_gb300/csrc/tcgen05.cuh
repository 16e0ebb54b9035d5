// Blackwell (sm_103a) tensor-core building blocks written in inline PTX: mbarriers, tiled TMA
// loads (cp.async.bulk.tensor), tensor-memory allocation, tcgen05.mma of kind::tf32 with FP32
// accumulation in TMEM, and tcgen05.ld for the epilogue.
//
// Operand layout used throughout: K-major tiles in the 128-byte swizzled layout that a TMA load
// with CU_TENSOR_MAP_SWIZZLE_128B produces -- rows of 128 bytes (32 FP32 values of K), eight
// rows per 1024-byte swizzle atom, atoms stacked along M (or N) -- so one operand chunk is
// rows x 32 values.  One MMA consumes K = 8 TF32 values (32 bytes of a row); the k-th step
// inside a chunk starts 32 k bytes further into the atom.
//
// Every wait is bounded (wall clock, %globaltimer): a kernel that gives up sets an error flag
// and returns instead of spinning forever.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace nls {
namespace tc {

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wall-clock limit of one bounded wait.  A tile's copies and MMAs take microseconds; a wait that
// reaches this limit means something is wrong, and the kernel reports it instead of hanging.
constexpr uint64_t kWaitLimitNs = 500ull * 1000ull * 1000ull;

// ---- mbarrier ----------------------------------------------------------------------------
__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Make initialised barriers visible to the async proxy (TMA, tensor cores) and the other threads.
__device__ inline void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete; false after kWaitLimitNs.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
  }
}

// ---- cluster exchange through distributed shared memory ------------------------------------
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ inline uint32_t cluster_addr(const void* local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
  return r;
}
// Two floats into another CTA's shared memory (8-byte aligned address); the store completes 8
// transaction bytes on that CTA's mbarrier `rbar` (both cluster addresses from cluster_addr).
__device__ inline void st_async_f2(uint32_t raddr, float a, float b, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
               "f"(a), "f"(b), "r"(rbar)
               : "memory");
}
// Wait on a local mbarrier whose transactions come from other CTAs of the cluster (acquire at
// cluster scope, so their stores are visible afterwards); false after kWaitLimitNs.
__device__ inline bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ inline bool mbar_wait_cluster(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
  }
}

// ---- TMA ---------------------------------------------------------------------------------
// 2D tiled load of the box at (x, y) (x = innermost coordinate, in elements; x times the
// element size must be a multiple of 16 bytes) into shared memory; completion is signalled on
// `bar` as transaction bytes.
__device__ inline void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Generic-proxy writes to shared memory become visible to the async proxy (tensor cores, TMA).
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- tensor memory -----------------------------------------------------------------------
// Executed by one whole warp: allocates `ncols` (a power of two >= 32) TMEM columns and writes
// their base address to *dst (shared memory).
__device__ inline void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ inline void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ inline void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- descriptors ---------------------------------------------------------------------------
// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzled layout: start
// address, stride between 8-row atoms (SBO) 1024 bytes, leading offset unused for this layout,
// the fixed version bits 46..48 = 0b001, swizzle mode 2 (128 bytes) in bits 61..63.
__device__ inline uint64_t desc_sw128(const void* smem) {
  const uint64_t a = smem_u32(smem);
  uint64_t d = (a & 0x3FFFFull) >> 4;
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor of a dense kind::tf32 MMA: D FP32 (bits 4..5 = 1), A and B TF32
// (bits 7..9 and 10..12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in bits 17..22, M >> 4 in
// bits 24..28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- MMA -----------------------------------------------------------------------------------
// D (TMEM) = A B (+ D when accumulate != 0); issued by one thread.
__device__ inline void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The barrier receives one arrival when every MMA issued so far by this thread has completed.
__device__ inline void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// ---- TMEM -> registers ----------------------------------------------------------------------
// 16 consecutive 32-bit columns of the warp's 32 TMEM lanes (lane = row of the accumulator);
// taddr = base + (first lane << 16) + first column.  Follow with tmem_wait_ld().
__device__ inline void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ inline void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- split of FP32 operands for three-pass TF32 products ------------------------------------
// x = hi + lo with hi = x with its 13 low mantissa bits cleared (exactly representable in TF32)
// and lo = x - hi (exact in FP32).  A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi then carries about
// FP32 accuracy (the dropped A_lo B_lo and the TF32 reading of the lo parts are ~2^-21 relative).
__device__ inline void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

}  // namespace tc
}  // namespace nls
