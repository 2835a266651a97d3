// Shared pieces of the tcgen05 kernels: mbarriers with bounded waits, TMA
// tile loads, shared-memory matrix descriptors, MMA issue/commit, tensor
// memory loads, the TF32 rounding used to split FP32 values, and a cache of
// TMA tensor maps for column-major FP32 blocks.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace trm {
namespace tc {

constexpr uint32_t kMaxPolls = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)),
               "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b))
               : "memory");
}
// One poll. The thread is suspended (it issues nothing) until the phase
// completes or kSuspendNs elapse, so waiting warps leave the issue slots to
// the working ones.
constexpr uint32_t kSuspendNs = 1000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after kMaxPolls polls (a few seconds at most), with
// bit 2 of *err and *failed set, so that every role of the CTA gives up and
// reaches its clean-up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity,
                                          int* err, volatile int* failed) {
  for (uint32_t i = 0; i < kMaxPolls; ++i) {
    if (mbar_try_wait(b, parity)) return true;
    if ((i & 1023u) == 1023u && *failed) break;
  }
  if (err) atomicOr(err, 2);
  *failed = 1;
  return false;
}
// Bounded wait for work this thread issued itself (copies or MMAs in flight
// before it may exit): it does not give up early when another role failed.
__device__ __forceinline__ bool mbar_wait_own(uint64_t* b, uint32_t parity,
                                              int* err) {
  for (uint32_t i = 0; i < kMaxPolls; ++i)
    if (mbar_try_wait(b, parity)) return true;
  if (err) atomicOr(err, 2);
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map,
                                            int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::"
      "complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y),
      "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map,
                                            int x, int y, int z, int w,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::"
      "complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w),
      "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor (descriptor version 1, 128-byte swizzle).
// K-major: rows of 128 bytes along K, 8-row groups `sbo` bytes apart.
// MN-major: 32 FP32 values along M/N per 128-byte line, 8 lines along K per
// 1024-byte atom; atoms `lbo` bytes apart along M/N and `sbo` along K.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo,
                                              uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::tf32 with FP32 accumulation.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, bool a_mn,
                                                  bool b_mn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((a_mn ? 1u : 0u) << 15) |
         ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc,
                                         uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
      "[%0];" ::"r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t cols) {
  asm volatile(
      "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
          smem_u32(dst)),
      "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                   taddr),
               "r"(cols));
}
// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
        "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
        "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 consecutive columns of this thread's TMEM lane, without waiting (the
// registers are valid after tmem_wait_ld).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr,
                                                uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
        "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
        "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 16 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
        "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
        "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Store 16 consecutive columns of this thread's TMEM lane; tmem_wait_st
// makes the stores complete before this thread reads them back or signals.
__device__ __forceinline__ void tmem_st16(uint32_t taddr,
                                          const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]),
      "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]),
      "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Round to the nearest TF32 value (ties away from zero), kept as an FP32
// bit pattern whose low 13 bits are zero.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Form and split half of a 128-byte line (16 values) of a staged tile, in
// place: y = a (+ alpha p, with p read from l), then hi -> a and lo -> l at
// the same offsets. Chunks are visited in a bank-spread order.
__device__ __forceinline__ void split_half(float* a, float* l, int line,
                                           int half, bool axpy, float alpha) {
  float4* pa = reinterpret_cast<float4*>(a + line * 32);
  float4* pl = reinterpret_cast<float4*>(l + line * 32);
  float4 v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = pa[(half * 4 + j) ^ (line & 7)];
  if (axpy) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 p = pl[(half * 4 + j) ^ (line & 7)];
      v[j].x = fmaf(alpha, p.x, v[j].x);
      v[j].y = fmaf(alpha, p.y, v[j].y);
      v[j].z = fmaf(alpha, p.z, v[j].z);
      v[j].w = fmaf(alpha, p.w, v[j].w);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = (half * 4 + j) ^ (line & 7);
    float4 h, o;
    h.x = tf32_rna(v[j].x); o.x = tf32_rna(v[j].x - h.x);
    h.y = tf32_rna(v[j].y); o.y = tf32_rna(v[j].y - h.y);
    h.z = tf32_rna(v[j].z); o.z = tf32_rna(v[j].z - h.z);
    h.w = tf32_rna(v[j].w); o.w = tf32_rna(v[j].w - h.w);
    pa[q] = h;
    pl[q] = o;
  }
}

// Host side: cuTensorMapEncodeTiled through the runtime's driver entry point
// (null when the driver does not offer it).
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t,
                              void*, const cuuint64_t*, const cuuint64_t*,
                              const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encode_fn();

// Tensor map of a column-major rows x cols FP32 matrix (leading dimension
// `ld` >= rows, a multiple of 4) read in boxes of box_rows x box_cols with
// the 128-byte swizzle (box_rows * 4 = 128), or without swizzle (box_rows
// up to 256: the box lands as box_cols columns of box_rows contiguous
// values). Cached per (pointer, shape, box, swizzle); out-of-range elements
// read as zero.
// The FP32 blocks of a grid operator as a 4-D tensor (x, y, z, column), no
// swizzle, boxes of (nx, box_y, 1, 1): one y-band of one plane of a column.
CUtensorMap f32_grid_map(const float* p, int nx, int ny, int nz, int ncols,
                         int box_y);
CUtensorMap f32_map(const float* p, int64_t rows, int64_t cols, int64_t ld,
                    int box_rows, int box_cols, bool swizzle = true);

}  // namespace tc
}  // namespace trm
