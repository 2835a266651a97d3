// Gram products A^T B of FP32 blocks on the 5th-generation tensor cores
// (tcgen05, accumulators in tensor memory), the O(m^2 N) products of
// Fig. EGFIG step (6), Fig. ONFIG step (1) and the line-search projections.
//
// Each FP32 value is split into two TF32 terms, x = hi + lo with
// hi = rna_tf32(x) and lo = rna_tf32(x - hi) (11 + 11 significant bits); the
// three products hi.hi + hi.lo + lo.hi are accumulated in FP32 in tensor
// memory, which keeps FP32-class accuracy (the dropped lo.lo and the rounding
// of lo are near 2^-22 relative). A TMA box of 32 rows x 128 columns of a
// column-major FP32 block, loaded with the 128-byte swizzle, is already the
// K-major operand layout the TF32 MMA reads, so the split happens in place
// (hi overwrites x, lo goes to a twin buffer) and no tile is copied.
//
// One CTA owns a 128 x 128 output tile and a slice of the N rows (split-K);
// its partial tile is written in FP64 and the slices are added in a fixed
// order by k_sum_splits, as in the SIMT path.
//
// Warp roles (192 threads): warp 0 issues the TMA loads (one box of A and one
// of B per 32-row stage, three stages in flight); warp 1 allocates tensor
// memory and issues the MMAs from one thread; warps 2-5 split the stage in
// place, then read the accumulator back (warp w owns TMEM lanes
// 32 (w % 4) .. +31). Every mbarrier wait is bounded: on timeout the kernel
// sets bit 2 of *err and falls through to its clean-up.
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "ops.cuh"

namespace trm {

namespace {

constexpr int BM = 128;        // output rows per CTA (columns of A)
constexpr int BN = 128;        // output columns per CTA (columns of B)
constexpr int BK = 32;         // block rows per stage (one 128-byte box)
constexpr int STAGES = 3;
constexpr int THREADS = 192;
constexpr uint32_t kMaxPolls = 1u << 22;

struct TcSmem {
  // [stage][A hi, B hi, A lo, B lo][128 columns x 32 rows], 128-byte swizzle:
  // 16-byte chunk q of column c sits at chunk q ^ (c % 8).
  float tile[STAGES][4][BM * BK];
  uint64_t full[STAGES], conv[STAGES], empty[STAGES], accdone;
  uint32_t tmem_base;
  int failed;
};

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
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the error bit set) after kMaxPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity,
                                          int* err, int* failed) {
  for (uint32_t i = 0; i < kMaxPolls; ++i)
    if (mbar_try_wait(b, parity)) return true;
  if (err) atomicOr(err, 2);
  *failed = 1;
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
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                            ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc,
                                         uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
      "[%0];" ::"r"(smem_u32(bar))
      : "memory");
}
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

// Round to the nearest TF32 value (ties away from zero), kept as an FP32
// bit pattern whose low 13 bits are zero.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Split one 128-byte line (32 values) of a stage tile in place: hi stays in
// `hi`, lo goes to the same offsets in `lo`.
__device__ __forceinline__ void split_line(float* hi, float* lo, int c) {
  float4* h = reinterpret_cast<float4*>(hi + c * BK);
  float4* l = reinterpret_cast<float4*>(lo + c * BK);
#pragma unroll
  for (int q = 0; q < BK / 4; ++q) {
    const int qs = q ^ (c & 7);  // visit chunks in bank-spread order
    float4 v = h[qs];
    float4 a, b;
    a.x = tf32_rna(v.x); b.x = tf32_rna(v.x - a.x);
    a.y = tf32_rna(v.y); b.y = tf32_rna(v.y - a.y);
    a.z = tf32_rna(v.z); b.z = tf32_rna(v.z - a.z);
    a.w = tf32_rna(v.w); b.w = tf32_rna(v.w - a.w);
    h[qs] = a;
    l[qs] = b;
  }
}

struct TcArgs {
  int64_t N;
  int m, n;               // output is m x n
  int64_t rows_per_split;
  int tiles_m;
  int seg_cols;           // columns per B segment (a multiple of BN if > 1)
  double* part;
  int* err;
};

__global__ void __launch_bounds__(THREADS, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap mapA,
              const __grid_constant__ CUtensorMap mapB0,
              const __grid_constant__ CUtensorMap mapB1,
              const __grid_constant__ CUtensorMap mapB2, TcArgs args) {
  extern __shared__ unsigned char smem_raw[];
  TcSmem* sm = reinterpret_cast<TcSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int split = blockIdx.x;
  const int tile = blockIdx.y;
  const int i0 = (tile % args.tiles_m) * BM;
  const int j0 = (tile / args.tiles_m) * BN;
  const int64_t rb = (int64_t)split * args.rows_per_split;
  const int64_t re = min(args.N, rb + args.rows_per_split);
  const int nk = (int)((re - rb + BK - 1) / BK);
  const int seg = j0 / args.seg_cols;
  const int jb = j0 - seg * args.seg_cols;
  const CUtensorMap* mapB = seg == 0 ? &mapB0 : (seg == 1 ? &mapB1 : &mapB2);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&sm->full[s], 1);
      mbar_init(&sm->conv[s], 128);
      mbar_init(&sm->empty[s], 1);
    }
    mbar_init(&sm->accdone, 1);
    sm->failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::
            "r"(smem_u32(&sm->tmem_base)),
        "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int k = 0; k < nk; ++k) {
        const int s = k % STAGES;
        if (k >= STAGES && !mbar_wait(&sm->empty[s], ((k / STAGES) - 1) & 1,
                                      args.err, &sm->failed))
          break;
        mbar_expect_tx(&sm->full[s], 2 * BM * BK * sizeof(float));
        const int x = (int)(rb + (int64_t)k * BK);
        tma_load_2d(sm->tile[s][0], &mapA, x, i0, &sm->full[s]);
        tma_load_2d(sm->tile[s][1], mapB, x, jb, &sm->full[s]);
        ++issued;
      }
      // Before the CTA may exit, the copies it issued must have landed (they
      // already have unless a wait above gave up).
      for (int k = issued > STAGES ? issued - STAGES : 0; k < issued; ++k)
        mbar_wait(&sm->full[k % STAGES], (k / STAGES) & 1, args.err,
                  &sm->failed);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      for (int k = 0; k < nk && ok; ++k) {
        const int s = k % STAGES;
        if (!mbar_wait(&sm->conv[s], (k / STAGES) & 1, args.err, &sm->failed)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t aH = smem_u32(sm->tile[s][0]);
        const uint32_t bH = smem_u32(sm->tile[s][1]);
        const uint32_t aL = smem_u32(sm->tile[s][2]);
        const uint32_t bL = smem_u32(sm->tile[s][3]);
        const uint32_t pa[3] = {aH, aH, aL};
        const uint32_t pb[3] = {bH, bL, bH};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
#pragma unroll
          for (int kk = 0; kk < BK / 8; ++kk)  // K = 8 per TF32 MMA (32 bytes)
            mma_tf32(tmem, smem_desc(pa[p] + kk * 32), smem_desc(pb[p] + kk * 32),
                     (k > 0 || p > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&sm->empty[s]);  // stage reusable once these MMAs are done
      }
      mma_commit(&sm->accdone);
    }
  } else {
    // ---------------- in-place split, then epilogue ----------------
    const int c = threadIdx.x - 64;  // 0..127: one line of A and one of B
    bool ok = true;
    for (int k = 0; k < nk && ok; ++k) {
      const int s = k % STAGES;
      if (!mbar_wait(&sm->full[s], (k / STAGES) & 1, args.err, &sm->failed)) {
        ok = false;
        break;
      }
      split_line(sm->tile[s][0], sm->tile[s][2], c);
      split_line(sm->tile[s][1], sm->tile[s][3], c);
      fence_proxy_async();
      mbar_arrive(&sm->conv[s]);
    }
    const bool acc_ok =
        ok && nk > 0 && mbar_wait(&sm->accdone, 0, args.err, &sm->failed);
    tc_fence_after();
    const int q = warp & 3;  // TMEM lane quarter of this warp
    const int row = i0 + 32 * q + lane;
    double* out = args.part + (size_t)split * args.m * args.n;
#pragma unroll 1
    for (int cb = 0; cb < BN; cb += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + cb, r);
      if (row < args.m) {
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int col = j0 + cb + e;
          if (col < args.n)
            out[row + (size_t)col * args.m] =
                acc_ok ? (double)__uint_as_float(r[e]) : 0.0;
        }
      }
    }
  }
  __syncwarp();  // lanes that skipped a single-thread role wait for it here
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                     tmem),
                 "r"(BN));
  }
}

// ---------------------------------------------------------------------------
// host side: tensor maps (cached per buffer) and the launch
// ---------------------------------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t,
                              void*, const cuuint64_t*, const cuuint64_t*,
                              const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
    cudaGetLastError();
  });
  return fn;
}

struct MapKey {
  const void* p;
  int64_t N;
  int cols;
  bool operator==(const MapKey& o) const {
    return p == o.p && N == o.N && cols == o.cols;
  }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    return std::hash<const void*>()(k.p) ^ (std::hash<int64_t>()(k.N) << 1) ^
           (std::hash<int>()(k.cols) << 2);
  }
};

std::mutex g_map_mu;
std::unordered_map<MapKey, CUtensorMap, MapKeyHash> g_maps;

// Column-major N x cols FP32 block: dim 0 = rows (contiguous), dim 1 = cols.
CUtensorMap block_map(const float* p, int64_t N, int cols) {
  std::lock_guard<std::mutex> lock(g_map_mu);
  MapKey key{p, N, cols};
  auto it = g_maps.find(key);
  if (it != g_maps.end()) return it->second;
  if (g_maps.size() > 256) g_maps.clear();
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)N * sizeof(float)};
  const cuuint32_t box[2] = {BK, BM};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                           const_cast<float*>(p), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw Error(-5, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  g_maps.emplace(key, map);
  return map;
}

}  // namespace

bool gram_tc_eligible(int64_t N, int m, const Blocks<float>& B) {
  if (N % 4 != 0 || N < BK || m < 64) return false;
  if (B.count > 3) return false;
  if (B.count > 1 && B.cols % BN != 0) return false;
  for (int s = 0; s < B.count; ++s)
    if (reinterpret_cast<uintptr_t>(B.p[s]) % 16 != 0) return false;
  return encode_fn() != nullptr;
}

size_t gram_tc_partials_doubles(int64_t N, int m, int n) {
  const int tiles = ceil_div(m, BM) * ceil_div(n, BN);
  const int splits = std::max(1, std::min(sm_count() / tiles,
                                          ceil_div(N, BK)));
  return (size_t)splits * m * n;
}

void gram_tc(int64_t N, int m, const float* A, const Blocks<float>& B,
             double* out, double* partials, size_t cap, int* err,
             cudaStream_t s) {
  const int n = B.total();
  const int tiles_m = ceil_div(m, BM);
  const int tiles = tiles_m * ceil_div(n, BN);
  int splits = std::max(1, std::min(sm_count() / tiles, ceil_div(N, BK)));
  int64_t rows = (N + splits - 1) / splits;
  rows = ((rows + BK - 1) / BK) * BK;
  splits = (int)((N + rows - 1) / rows);
  if ((size_t)splits * m * n > cap)
    throw Error(-2, "gram_tc: partials buffer too small");
  CUtensorMap mA = block_map(A, N, m);
  const int segcols = B.count > 1 ? B.cols : n;
  CUtensorMap mB[3];
  for (int k = 0; k < 3; ++k)
    mB[k] = block_map(B.p[k < B.count ? k : 0], N, B.cols);
  TcArgs a{N, m, n, rows, tiles_m, segcols, partials, err};
  const size_t smem = sizeof(TcSmem) + 1024;
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  });
  dim3 grid(splits, tiles);
  k_gram_tc<<<grid, THREADS, smem, s>>>(mA, mB[0], mB[1], mB[2], a);
  TRM_CHECK_LAUNCH();
  const size_t count = (size_t)m * n;
  sum_splits(partials, splits, count, out, s);
}

}  // namespace trm
