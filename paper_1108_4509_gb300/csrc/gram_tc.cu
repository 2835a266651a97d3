// Gram products A^T B of FP32 blocks on the 5th-generation tensor cores
// (tcgen05, accumulators in tensor memory), the O(m^2 N) products of
// Fig. EGFIG step (6), Fig. ONFIG step (1) and the line-search projections.
//
// Each FP32 value is split into two TF32 terms, x = hi + lo. The TF32 MMA
// reads an FP32 bit pattern and ignores its low 13 mantissa bits (measured:
// the raw value as the TF32 operand with lo = rna_tf32(x - trunc(x)) gives
// the product to 2e-8 of sum |a||b|, with lo from rna_tf32(x) instead to
// 1e-5), so hi = trunc_tf32(x) is the TMA-loaded tile itself and only lo is
// formed (lo = rna_tf32(x - hi), |lo| < 2^-10 |x|, rounding error < 2^-21
// |x|). The three products hi.hi + hi.lo + lo.hi are accumulated in FP32 in
// tensor memory; the dropped lo.lo and the rounding of lo are below 2^-19 of
// |a b|: FP32-class accuracy. A TMA box of 32 rows x 128 columns of a
// column-major FP32 block, loaded with the 128-byte swizzle, is already the
// K-major operand layout the TF32 MMA reads, and lo is written at the same
// offsets of a twin buffer.
//
// One CTA owns a 128 x 128 output tile and a slice of the N rows (split-K);
// its partial tile is written as double-float pairs and the slices are added
// in a fixed order by k_sum_splits_pairs (FP64 results).
//
// The tensor core accumulates in FP32 but does not round to nearest: every
// MMA step drops up to an ulp of the running sum, so the error grows with
// the number of steps (measured: 6.7e-4 relative after 98304 rows). The MMA
// therefore accumulates chunks of KC stages (KC * 32 rows) into one of two
// TMEM buffers, and accumulator warps fold each finished chunk into a
// double-float (hi, lo) running sum kept in the other half of TMEM; the bias
// is bounded by KC * 12 steps of 2^-23 of the chunk sums. Row slices of at
// most kSingleChunk stages (3072 rows, all of the 48^3 case) are one chunk:
// the bias is then at most 96 * 12 steps and nothing is folded.
//
// Warp roles (576 threads): warp 0 issues the TMA loads (one box of A and one
// of B per 32-row stage into a ring of raw stages, each freed when the MMAs
// that read it as hi are done); warp 1 allocates tensor memory and issues the
// MMAs from one thread; warps 2-9 form lo of each raw stage into a ring of
// lo stages (half a line of A and of B each), so the split of the next
// stages overlaps the MMAs of this one; warps 10-17 fold the finished
// chunks and write the partial as FP32 pairs (warp w owns TMEM lanes
// 32 (w % 4) .. +31 and one 64-column half). No FP64 instruction runs here
// (GB300's FP64 pipe is 1/64 of its FP32 rate). Every mbarrier wait is
// bounded: on timeout the kernel sets bit 2 of *err and falls through to its
// clean-up.
#include <cuda.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>

#include "dfmath.cuh"
#include "ops.cuh"
#include "tc.cuh"

namespace trm {

namespace {

using namespace tc;

constexpr int BM = 128;        // output rows per CTA (columns of A)
constexpr int BN = 128;        // output columns per CTA (columns of B)
constexpr int BK = 32;         // block rows per stage (one 128-byte box)
#ifndef TRM_GRAM_RSTAGES
#define TRM_GRAM_RSTAGES 3
#endif
#ifndef TRM_GRAM_OSTAGES
#define TRM_GRAM_OSTAGES 3
#endif
constexpr int RSTAGES = TRM_GRAM_RSTAGES;  // raw TMA stages (the hi operands)
constexpr int OSTAGES = TRM_GRAM_OSTAGES;  // lo stages
constexpr int THREADS = 576;  // 18 warps
constexpr int KC = 8;         // stages per accumulation chunk (default)
constexpr int kSingleChunk = 96;  // row slices this short are one chunk
// Row slices of at least this many stages: a small problem takes fewer CTAs
// (each holds a whole SM) and leaves the rest of the GPU to concurrent solves.
constexpr int kMinStages = 16;

struct TcSmem {
  // [stage][A, B][128 columns x 32 rows] as loaded (the hi operands), and
  // the lo operands [stage][A lo, B lo] at the same offsets; 128-byte
  // swizzle: 16-byte chunk q of column c sits at chunk q ^ (c % 8).
  float raw[RSTAGES][2][BM * BK];
  float op[OSTAGES][2][BM * BK];
  uint64_t full[RSTAGES], rawfree[RSTAGES], opfull[OSTAGES], opfree[OSTAGES];
  uint64_t accfull[2], accempty[2], mmadone;
  uint32_t tmem_base;
  int failed;
};

// lo = rna_tf32(x - trunc_tf32(x)) for half of a 128-byte line (16 values)
// of a raw stage, at the same offsets of the lo buffer. Chunks are visited
// in a bank-spread order.
__device__ __forceinline__ float tf32_lo(float x) {
  return tf32_rna(x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u));
}
__device__ __forceinline__ void split_line_half(const float* raw, float* lo,
                                                int line, int half) {
  const float4* pr = reinterpret_cast<const float4*>(raw + line * 32);
  float4* pl = reinterpret_cast<float4*>(lo + line * 32);
  float4 v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = pr[(half * 4 + j) ^ (line & 7)];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = (half * 4 + j) ^ (line & 7);
    pl[q] = make_float4(tf32_lo(v[j].x), tf32_lo(v[j].y), tf32_lo(v[j].z),
                        tf32_lo(v[j].w));
  }
}

// K-major operand descriptor: 128-byte rows, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t kdesc(uint32_t saddr) {
  return smem_desc(saddr, 16, 1024);
}
// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdesc = idesc_tf32(BM, BN, false, false);

// Output tiles of one launch, listed (blockIdx.y indexes the list): all of
// them, or for a symmetric segment only those on or above its diagonal.
constexpr int kMaxTiles = 256;  // 8 x 32: m = 1024, four m-column segments

struct TcArgs {
  int64_t N;
  int m, n;               // output is m x n
  int64_t rows_per_split;
  int kc;                 // stages per accumulation chunk of long slices
  int seg_cols;           // columns per segment
  int tps;                // column tiles per segment (the last one ragged:
                          // its columns past seg_cols load as zeros)
  double* part;
  int* err;
  uint8_t ti[kMaxTiles], tj[kMaxTiles];  // row and column tile of each CTA row
};

// Output column segment k is A_k^T B_k (up to four segments; the line search
// takes [C P P P]^T [P P HP G] in one launch).
struct TcMaps {
  CUtensorMap a[4];
  CUtensorMap b[4];
};

__global__ void __launch_bounds__(THREADS, 1)
    k_gram_tc(const __grid_constant__ TcMaps maps, TcArgs args) {
  extern __shared__ unsigned char smem_raw[];
  TcSmem* sm = reinterpret_cast<TcSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int split = blockIdx.x;
  const int i0 = args.ti[blockIdx.y] * BM;
  const int64_t rb = (int64_t)split * args.rows_per_split;
  const int64_t re = min(args.N, rb + args.rows_per_split);
  const int nk = (int)((re - rb + BK - 1) / BK);
  const int seg = args.tj[blockIdx.y] / args.tps;
  const int jb = (args.tj[blockIdx.y] - seg * args.tps) * BN;  // in segment
  const int j0 = seg * args.seg_cols + jb;  // first output column
  const CUtensorMap* mapA = &maps.a[seg];
  const CUtensorMap* mapB = &maps.b[seg];

  if (threadIdx.x == 0) {
    for (int s = 0; s < RSTAGES; ++s) {
      mbar_init(&sm->full[s], 1);
      mbar_init(&sm->rawfree[s], 1);  // the MMAs that read it are done
    }
    for (int s = 0; s < OSTAGES; ++s) {
      mbar_init(&sm->opfull[s], 256);
      mbar_init(&sm->opfree[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm->accfull[b], 1);
      mbar_init(&sm->accempty[b], 256);  // the eight fold warps
    }
    mbar_init(&sm->mmadone, 1);
    sm->failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // TMEM: chunk buffers at columns 0 and BN, the double-float sum's hi at
  // 2 BN and lo at 3 BN
  if (warp == 1) tmem_alloc(&sm->tmem_base, 4 * BN);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int k = 0; k < nk; ++k) {
        const int s = k % RSTAGES;
        if (k >= RSTAGES &&
            !mbar_wait(&sm->rawfree[s], ((k / RSTAGES) - 1) & 1, args.err,
                       &sm->failed))
          break;
        mbar_expect_tx(&sm->full[s], 2 * BM * BK * sizeof(float));
        const int x = (int)(rb + (int64_t)k * BK);
        tma_load_2d(sm->raw[s][0], mapA, x, i0, &sm->full[s]);
        tma_load_2d(sm->raw[s][1], mapB, x, jb, &sm->full[s]);
        ++issued;
      }
      // Before the CTA may exit, the copies it issued must have landed (they
      // already have unless a wait above gave up).
      for (int k = issued > RSTAGES ? issued - RSTAGES : 0; k < issued; ++k)
        mbar_wait_own(&sm->full[k % RSTAGES], (k / RSTAGES) & 1, args.err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      const int kcl = nk <= kSingleChunk ? nk : args.kc;  // stages per chunk
      for (int k = 0; k < nk && ok; ++k) {
        const int s = k % OSTAGES, r = k % RSTAGES;
        const int kc = k % kcl, c = k / kcl, b = c & 1;
        if (kc == 0 && c >= 2 &&
            !mbar_wait(&sm->accempty[b], ((c / 2) - 1) & 1, args.err,
                       &sm->failed)) {
          ok = false;
          break;
        }
        if (!mbar_wait(&sm->opfull[s], (k / OSTAGES) & 1, args.err,
                       &sm->failed)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(b * BN);
        const uint32_t aH = smem_u32(sm->raw[r][0]);
        const uint32_t bH = smem_u32(sm->raw[r][1]);
        const uint32_t aL = smem_u32(sm->op[s][0]);
        const uint32_t bL = smem_u32(sm->op[s][1]);
        const uint32_t pa[3] = {aH, aH, aL};
        const uint32_t pb[3] = {bH, bL, bH};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
#pragma unroll
          for (int kk = 0; kk < BK / 8; ++kk)  // K = 8 per TF32 MMA (32 bytes)
            mma_tf32(d, kdesc(pa[p] + kk * 32), kdesc(pb[p] + kk * 32),
                     kIdesc, (kc > 0 || p > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&sm->opfree[s]);   // lo and the raw stage reusable
        mma_commit(&sm->rawfree[r]);  // once these MMAs are done
        if (kc == kcl - 1 || k == nk - 1) mma_commit(&sm->accfull[b]);
      }
      // every MMA of this thread completes before the TMEM is released
      mma_commit(&sm->mmadone);
      mbar_wait_own(&sm->mmadone, 0, args.err);
    }
  } else if (warp < 10) {
    // ---------------- split: raw stage -> operand stage ----------------
    const int t = threadIdx.x - 64;  // 0..255: half a line of A and of B
    const int c_line = t >> 1, half = t & 1;
    for (int k = 0; k < nk; ++k) {
      const int s = k % RSTAGES, o = k % OSTAGES;
      if (!mbar_wait(&sm->full[s], (k / RSTAGES) & 1, args.err, &sm->failed))
        break;
      if (k >= OSTAGES &&
          !mbar_wait(&sm->opfree[o], ((k / OSTAGES) - 1) & 1, args.err,
                     &sm->failed))
        break;
      split_line_half(sm->raw[s][0], sm->op[o][0], c_line, half);
      split_line_half(sm->raw[s][1], sm->op[o][1], c_line, half);
      // the lo writes before the MMAs read them, and the raw reads before the
      // TMA refill that follows those MMAs (both across the async proxy)
      fence_proxy_async();
      mbar_arrive(&sm->opfull[o]);
    }
  } else {
    // ------- fold the chunks into the double-float sum, then write -------
    const int q = warp & 3;            // TMEM lane quarter of this warp
    const int g = (warp - 10) >> 2;    // column half of the tile
    const uint32_t lrow = (uint32_t)(32 * q) << 16;
    const int kcl = nk <= kSingleChunk ? nk : args.kc;
    const int nch = nk > 0 ? (nk + kcl - 1) / kcl : 0;
    const int row = i0 + 32 * q + lane;
    // partials as FP32 pairs: split s holds hi at [2 s count, (2 s + 1)
    // count) and lo after it (no FP64 instruction in this kernel)
    const size_t count = (size_t)args.m * args.n;
    float* out_hi = reinterpret_cast<float*>(args.part) + 2 * (size_t)split * count;
    float* out_lo = out_hi + count;
    bool ok = nch > 0;
    for (int c = 0; c < nch && ok; ++c) {
      const int b = c & 1;
      const bool last = c == nch - 1;
      const bool got =
          mbar_wait(&sm->accfull[b], (c / 2) & 1, args.err, &sm->failed);
      if (!__all_sync(0xffffffffu, got)) {  // the TMEM ops are .sync.aligned
        ok = false;
        break;
      }
      fence_after();
#pragma unroll 1
      for (int cb = 64 * g; cb < 64 * g + 64; cb += 16) {
        uint32_t x[16], hi[16], lo[16];
        tmem_ld16_async(tmem + lrow + (uint32_t)(b * BN + cb), x);
        if (c > 0) {
          tmem_ld16_async(tmem + lrow + (uint32_t)(2 * BN + cb), hi);
          tmem_ld16_async(tmem + lrow + (uint32_t)(3 * BN + cb), lo);
        }
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          F2 v = {__uint_as_float(x[e]), 0.f};
          if (c > 0)
            v = df_add(F2{__uint_as_float(hi[e]), __uint_as_float(lo[e])}, v);
          hi[e] = __float_as_uint(v.h);
          lo[e] = __float_as_uint(v.l);
        }
        if (last) {  // the partial of this row slice, as FP32 pairs
          if (row < args.m) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int col = j0 + cb + e;
              if (jb + cb + e < args.seg_cols) {
                const size_t idx = row + (size_t)col * args.m;
                out_hi[idx] = __uint_as_float(hi[e]);
                out_lo[idx] = __uint_as_float(lo[e]);
              }
            }
          }
        } else {
          tmem_st16(tmem + lrow + (uint32_t)(2 * BN + cb), hi);
          tmem_st16(tmem + lrow + (uint32_t)(3 * BN + cb), lo);
        }
      }
      if (!last) {
        tmem_wait_st();
        fence_before();
        mbar_arrive(&sm->accempty[b]);
      }
    }
    __syncwarp();
    if (!ok && row < args.m) {  // a wait gave up: zero partial, error set
      for (int cb = 64 * g; cb < 64 * g + 64; ++cb)
        if (jb + cb < args.seg_cols) {
          out_hi[row + (size_t)(j0 + cb) * args.m] = 0.f;
          out_lo[row + (size_t)(j0 + cb) * args.m] = 0.f;
        }
    }
  }
  __syncwarp();  // lanes that skipped a single-thread role wait for it here
  fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    tmem_dealloc(tmem, 4 * BN);
  }
}

CUtensorMap block_map(const float* p, int64_t N, int cols) {
  return f32_map(p, N, cols, N, BK, BM);
}

}  // namespace

bool gram_tc_eligible(int64_t N, int m, const float* A,
                      const Blocks<float>& B) {
  Blocks<float> a;
  a.p[0] = A;
  a.cols = m;
  a.count = 1;
  return gram_tc_pairs_eligible(N, m, a, B);
}

bool gram_tc_pairs_eligible(int64_t N, int m, const Blocks<float>& A,
                            const Blocks<float>& B) {
  // (m >= 32: a 128 x 128 tile at least a quarter used; below that the
  // SIMT kernel is as fast)
  if (N % 4 != 0 || N < BK || m < 32) return false;
  if (B.count > 4) return false;
  if (A.count > 1 && A.count != B.count) return false;
  for (int s = 0; s < A.count; ++s)
    if (reinterpret_cast<uintptr_t>(A.p[s]) % 16 != 0) return false;
  for (int s = 0; s < B.count; ++s)
    if (reinterpret_cast<uintptr_t>(B.p[s]) % 16 != 0) return false;
  return tc::encode_fn() != nullptr;
}

// Row slices for a launch of `tiles` output tiles: among the counts that
// keep at least kMinStages stages per slice, launch at most 8 waves of CTAs
// and stay within max_splits, the one whose CTAs fill the SMs most evenly,
// less 1 % per extra wave (each wave refills the pipelines). Every CTA of a
// launch does the same work, so with one slice per tile a launch of 164
// tiles would run a second wave of 12 CTAs as long as the first.
static int tc_splits(int64_t N, int tiles, int max_splits, int sms) {
  const int64_t by_rows = ceil_div(N, (int64_t)BK * kMinStages);
  const int smax = (int)std::max<int64_t>(
      1, std::min<int64_t>({by_rows, (int64_t)8 * sms / tiles,
                            (int64_t)max_splits}));
  int best = 1;
  double beff = 0.0;
  for (int sp = 1; sp <= smax; ++sp) {
    const int64_t ctas = (int64_t)tiles * sp;
    const int64_t waves = ceil_div(ctas, (int64_t)sms);
    const double eff =
        (double)ctas / ((double)sms * (double)waves) - 0.01 * (double)(waves - 1);
    if (eff > beff + 1e-3) {
      beff = eff;
      best = sp;
    }
  }
  return best;
}

// Autotuned row slices. The formula above fills the SMs in whole waves, but
// how many slices run best also depends on how the CTAs of a wave share
// their operand tiles in L2, which the formula does not model. The first
// launch of each (N, m, n, tiles, symmetric segment) in the process
// therefore times the formula's count and half of it (at least kMinStages
// stages per slice), twice each in turn with CUDA events on the stream, and
// keeps the faster for the process (never inside a stream capture: the
// formula's count is used there until a choice exists). No candidate
// exceeds the formula's count, which every caller's partials buffer holds,
// so the choice does not depend on which caller made it. Every count gives the same sum to the
// accumulation bound; the bytes depend on the count, so the choice is
// fixed per process and repeated solves agree bit for bit.
struct SliceKey {
  int64_t N;
  int m, n, tiles, sym;
  bool operator<(const SliceKey& o) const {
    return std::tie(N, m, n, tiles, sym) <
           std::tie(o.N, o.m, o.n, o.tiles, o.sym);
  }
};
std::mutex g_slice_mu;
std::map<SliceKey, int> g_slices;

template <typename Run>
int tuned_splits(int64_t N, int m, int n, int tiles, int sym, int smax,
                 cudaStream_t s, Run& run) {
  const int sms = sm_count();
  const int base = tc_splits(N, tiles, smax, sms);
  // TRM_GRAM_SLICES=formula (or a count) fixes the slices instead (for
  // profilers, whose serialised replay would distort the timing)
  if (const char* f = std::getenv("TRM_GRAM_SLICES")) {
    const int v = std::atoi(f);
    return v > 0 ? std::min(v, smax) : base;
  }
  const SliceKey key{N, m, n, tiles, sym};
  {
    std::lock_guard<std::mutex> lock(g_slice_mu);
    auto it = g_slices.find(key);
    if (it != g_slices.end()) return std::min(it->second, smax);
  }
  const int most = (int)std::max<int64_t>(
      1, std::min<int64_t>(smax, ceil_div(N, (int64_t)BK * kMinStages)));
  int cand[2], nc = 0;
  for (int c : {base, base / 2}) {
    c = std::max(1, std::min(c, most));
    bool dup = false;
    for (int k = 0; k < nc; ++k) dup |= cand[k] == c;
    if (!dup) cand[nc++] = c;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TRM_CUDA(cudaStreamIsCapturing(s, &cs));
  if (nc == 1 || cs != cudaStreamCaptureStatusNone) return base;
  constexpr int kRounds = 2;
  cudaEvent_t ev[1 + 2 * kRounds];
  for (auto& e : ev) TRM_CUDA(cudaEventCreate(&e));
  long long tuning = 0;
  capture_launches(&tuning);  // the timing launches are not the caller's
  for (int k = 0; k < nc; ++k) run(cand[k]);  // warm-up
  TRM_CUDA(cudaEventRecord(ev[0], s));
  int e = 1;
  for (int r = 0; r < kRounds; ++r)
    for (int k = 0; k < nc; ++k) {
      run(cand[k]);
      TRM_CUDA(cudaEventRecord(ev[e++], s));
    }
  capture_launches(nullptr);
  TRM_CUDA(cudaEventSynchronize(ev[e - 1]));
  float tot[2] = {0.f, 0.f}, t = 0.f;
  for (int i = 1; i < e; ++i) {
    TRM_CUDA(cudaEventElapsedTime(&t, ev[i - 1], ev[i]));
    tot[(i - 1) % nc] += t;
  }
  for (auto& ee : ev) cudaEventDestroy(ee);
  int best = 0;
  for (int k = 1; k < nc; ++k)
    if (tot[k] < tot[best]) best = k;
  std::lock_guard<std::mutex> lock(g_slice_mu);
  // the first decision for a key stands (another thread may have tuned it)
  return std::min(g_slices.emplace(key, cand[best]).first->second, smax);
}

size_t gram_tc_partials_doubles(int64_t N, int m, int n, int skipped_tiles) {
  const int tiles = ceil_div(m, BM) * ceil_div(n, BN) - skipped_tiles;
  return (size_t)tc_splits(N, std::max(1, tiles), 1 << 30, sm_count()) * m * n;
}

void gram_tc(int64_t N, int m, const float* A, const Blocks<float>& B,
             double* out, double* partials, size_t cap, int* err,
             cudaStream_t s, float* out32, int max_splits) {
  Blocks<float> a;
  a.p[0] = A;
  a.cols = m;
  a.count = 1;
  gram_tc_pairs(N, m, a, B, out, partials, cap, err, s, out32, -1,
                max_splits);
}

void gram_tc_pairs(int64_t N, int m, const Blocks<float>& A,
                   const Blocks<float>& B, double* out, double* partials,
                   size_t cap, int* err, cudaStream_t s, float* out32,
                   int sym_seg, int max_splits) {
  const int n = B.total();
  const int tiles_m = ceil_div(m, BM);
  const int segcols = B.count > 1 ? B.cols : n;
  const int nseg = B.count > 1 ? B.count : 1;
  const int tps = ceil_div(segcols, BN);  // a segment's last tile is ragged
  if (sym_seg >= 0 && (sym_seg >= B.count || B.cols != m))
    throw Error(-1, "gram_tc: a symmetric segment must be m x m");
  TcArgs a{};
  int tiles = 0;
  for (int tj = 0; tj < nseg * tps; ++tj) {
    const int seg = tj / tps;
    const int tjs = tj - seg * tps;  // column tile in its segment
    for (int ti = 0; ti < tiles_m; ++ti) {
      if (seg == sym_seg && ti > tjs) continue;  // mirrored from (tjs, ti)
      if (tiles == kMaxTiles) throw Error(-1, "gram_tc: too many output tiles");
      a.ti[tiles] = (uint8_t)ti;
      a.tj[tiles] = (uint8_t)tj;
      ++tiles;
    }
  }
  // (the partials buffer bounds the slices too)
  const size_t by_cap = cap / ((size_t)m * n);
  if (by_cap < 1) throw Error(-2, "gram_tc: partials buffer too small");
  int smax = max_splits > 0 ? max_splits : 1 << 30;
  if ((size_t)smax > by_cap) smax = (int)by_cap;
  TcMaps maps;
  for (int k = 0; k < 4; ++k) {
    const int kb = k < B.count ? k : 0;
    maps.a[k] = block_map(A.p[A.count > 1 ? kb : 0], N, m);
    maps.b[k] = block_map(B.p[kb], N, B.cols);
  }
  a.N = N;
  a.m = m;
  a.n = n;
  a.seg_cols = segcols;
  a.tps = tps;
  // TRM_GRAM_KC overrides the chunk length (measurements of the
  // accumulation error against the fold's cost)
  a.kc = KC;
  if (const char* f = std::getenv("TRM_GRAM_KC")) {
    const int v = std::atoi(f);
    if (v >= 1 && v <= kSingleChunk) a.kc = v;
  }
  a.part = partials;
  a.err = err;
  const size_t smem = sizeof(TcSmem) + 1024;
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  });
  const size_t count = (size_t)m * n;
  // one launch with about `want` row slices (rounded to whole stages)
  auto run = [&](int want) {
    int64_t rows = (N + want - 1) / want;
    rows = ((rows + BK - 1) / BK) * BK;
    const int splits = (int)((N + rows - 1) / rows);
    if ((size_t)splits * count > cap)
      throw Error(-2, "gram_tc: partials buffer too small");
    a.rows_per_split = rows;
    k_gram_tc<<<dim3(splits, tiles), THREADS, smem, s>>>(maps, a);
    TRM_CHECK_LAUNCH();
    sum_splits_pairs(reinterpret_cast<const float*>(partials), splits, count,
                     out, s, out32, SymSeg{sym_seg, m, segcols, BM});
  };
  run(tuned_splits(N, m, n, tiles, sym_seg, smax, s, run));
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
  int br, bc, sw;
  bool operator==(const MapKey& o) const {
    return p == o.p && rows == o.rows && cols == o.cols && ld == o.ld &&
           br == o.br && bc == o.bc && sw == o.sw;
  }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    size_t h = std::hash<const void*>()(k.p);
    for (int64_t v : {k.rows, k.cols, k.ld, (int64_t)k.br, (int64_t)k.bc,
                      (int64_t)k.sw})
      h = h * 1000003u ^ std::hash<int64_t>()(v);
    return h;
  }
};
std::mutex g_map_mu;
std::unordered_map<MapKey, CUtensorMap, MapKeyHash> g_maps;
}  // namespace

CUtensorMap f32_map(const float* p, int64_t rows, int64_t cols, int64_t ld,
                    int box_rows, int box_cols, bool swizzle) {
  std::lock_guard<std::mutex> lock(g_map_mu);
  MapKey key{p, rows, cols, ld, box_rows, box_cols, swizzle ? 1 : 0};
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
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw Error(-5, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  g_maps.emplace(key, map);
  return map;
}

namespace {
struct GridKey {
  const void* p;
  int nx, ny, nz, nc, by;
  bool operator==(const GridKey& o) const {
    return p == o.p && nx == o.nx && ny == o.ny && nz == o.nz && nc == o.nc &&
           by == o.by;
  }
};
struct GridKeyHash {
  size_t operator()(const GridKey& k) const {
    size_t h = std::hash<const void*>()(k.p);
    for (int v : {k.nx, k.ny, k.nz, k.nc, k.by})
      h = h * 1000003u ^ std::hash<int>()(v);
    return h;
  }
};
std::unordered_map<GridKey, CUtensorMap, GridKeyHash> g_grid_maps;
}  // namespace

CUtensorMap f32_grid_map(const float* p, int nx, int ny, int nz, int ncols,
                         int box_y) {
  std::lock_guard<std::mutex> lock(g_map_mu);
  GridKey key{p, nx, ny, nz, ncols, box_y};
  auto it = g_grid_maps.find(key);
  if (it != g_grid_maps.end()) return it->second;
  if (g_grid_maps.size() > 512) g_grid_maps.clear();
  EncodeFn fn = encode_fn();
  if (!fn) throw Error(-5, "cuTensorMapEncodeTiled is not available");
  CUtensorMap map;
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz,
                              (cuuint64_t)ncols};
  const cuuint64_t plane = (cuuint64_t)nx * ny * sizeof(float);
  const cuuint64_t strides[3] = {(cuuint64_t)nx * sizeof(float), plane,
                                 plane * (cuuint64_t)nz};
  const cuuint32_t box[4] = {(cuuint32_t)nx, (cuuint32_t)box_y, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                  const_cast<float*>(p), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw Error(-5, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  g_grid_maps.emplace(key, map);
  return map;
}

}  // namespace tc
}  // namespace trm
