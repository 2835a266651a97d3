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
// Warp roles (320 threads): warp 0 issues the TMA loads (one box of A and one
// of B per 32-row stage, three stages in flight); warp 1 allocates tensor
// memory and issues the MMAs from one thread; warps 2-9 split the stage in
// place (half a line of A and of B each), then read the accumulator back
// (warp w owns TMEM lanes 32 (w % 4) .. +31 and one 64-column half). Every mbarrier wait is bounded: on timeout the kernel
// sets bit 2 of *err and falls through to its clean-up.
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "ops.cuh"
#include "tc.cuh"

namespace trm {

namespace {

using namespace tc;

constexpr int BM = 128;        // output rows per CTA (columns of A)
constexpr int BN = 128;        // output columns per CTA (columns of B)
constexpr int BK = 32;         // block rows per stage (one 128-byte box)
constexpr int STAGES = 3;
constexpr int THREADS = 320;  // 10 warps

struct TcSmem {
  // [stage][A hi, B hi, A lo, B lo][128 columns x 32 rows], 128-byte swizzle:
  // 16-byte chunk q of column c sits at chunk q ^ (c % 8).
  float tile[STAGES][4][BM * BK];
  uint64_t full[STAGES], conv[STAGES], empty[STAGES], accdone;
  uint32_t tmem_base;
  int failed;
};

// K-major operand descriptor: 128-byte rows, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t kdesc(uint32_t saddr) {
  return smem_desc(saddr, 16, 1024);
}
// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdesc = idesc_tf32(BM, BN, false, false);

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
      mbar_init(&sm->conv[s], 256);
      mbar_init(&sm->empty[s], 1);
    }
    mbar_init(&sm->accdone, 1);
    sm->failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(&sm->tmem_base, BN);
  }
  fence_before();
  __syncthreads();
  fence_after();
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
        mbar_wait_own(&sm->full[k % STAGES], (k / STAGES) & 1, args.err);
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
        fence_after();
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
            mma_tf32(tmem, kdesc(pa[p] + kk * 32), kdesc(pb[p] + kk * 32),
                     kIdesc, (k > 0 || p > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&sm->empty[s]);  // stage reusable once these MMAs are done
      }
      mma_commit(&sm->accdone);
    }
  } else {
    // ---------------- in-place split, then epilogue ----------------
    const int t = threadIdx.x - 64;  // 0..255: half a line of A and of B
    const int c = t >> 1, half = t & 1;
    bool ok = true;
    for (int k = 0; k < nk && ok; ++k) {
      const int s = k % STAGES;
      if (!mbar_wait(&sm->full[s], (k / STAGES) & 1, args.err, &sm->failed)) {
        ok = false;
        break;
      }
      split_half(sm->tile[s][0], sm->tile[s][2], c, half, false, 0.f);
      split_half(sm->tile[s][1], sm->tile[s][3], c, half, false, 0.f);
      fence_proxy_async();
      mbar_arrive(&sm->conv[s]);
    }
    const bool acc_ok =
        ok && nk > 0 && mbar_wait(&sm->accdone, 0, args.err, &sm->failed);
    __syncwarp();  // the TMEM loads below are .sync.aligned
    fence_after();
    const int q = warp & 3;          // TMEM lane quarter of this warp
    const int g = (warp - 2) >> 2;   // column half of the tile
    const int row = i0 + 32 * q + lane;
    double* out = args.part + (size_t)split * args.m * args.n;
#pragma unroll 1
    for (int cb = 64 * g; cb < 64 * g + 64; cb += 32) {
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
  fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    tmem_dealloc(tmem, BN);
  }
}

CUtensorMap block_map(const float* p, int64_t N, int cols) {
  return f32_map(p, N, cols, N, BK, BM);
}

}  // namespace

bool gram_tc_eligible(int64_t N, int m, const Blocks<float>& B) {
  if (N % 4 != 0 || N < BK || m < 64) return false;
  if (B.count > 3) return false;
  if (B.count > 1 && B.cols % BN != 0) return false;
  for (int s = 0; s < B.count; ++s)
    if (reinterpret_cast<uintptr_t>(B.p[s]) % 16 != 0) return false;
  return tc::encode_fn() != nullptr;
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

// ---------------------------------------------------------------------------
// host side of the shared tcgen05 helpers: the tensor-map encoder and cache
// ---------------------------------------------------------------------------
namespace trm {
namespace tc {

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

namespace {
struct MapKey {
  const void* p;
  int64_t rows, cols, ld;
  int br, bc;
  bool operator==(const MapKey& o) const {
    return p == o.p && rows == o.rows && cols == o.cols && ld == o.ld &&
           br == o.br && bc == o.bc;
  }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    size_t h = std::hash<const void*>()(k.p);
    for (int64_t v : {k.rows, k.cols, k.ld, (int64_t)k.br, (int64_t)k.bc})
      h = h * 1000003u ^ std::hash<int64_t>()(v);
    return h;
  }
};
std::mutex g_map_mu;
std::unordered_map<MapKey, CUtensorMap, MapKeyHash> g_maps;
}  // namespace

CUtensorMap f32_map(const float* p, int64_t rows, int64_t cols, int64_t ld,
                    int box_rows, int box_cols) {
  std::lock_guard<std::mutex> lock(g_map_mu);
  MapKey key{p, rows, cols, ld, box_rows, box_cols};
  auto it = g_maps.find(key);
  if (it != g_maps.end()) return it->second;
  if (g_maps.size() > 512) g_maps.clear();
  EncodeFn fn = encode_fn();
  if (!fn) throw Error(-5, "cuTensorMapEncodeTiled is not available");
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<float*>(p), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw Error(-5, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  g_maps.emplace(key, map);
  return map;
}

}  // namespace tc
}  // namespace trm
