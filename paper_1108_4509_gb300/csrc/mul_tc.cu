// Products of a tall FP32 block with a small matrix, Y M (Y: N x k, M: k x n),
// on the 5th-generation tensor cores: the O(N m^2) products of the gradient
// G = -2 (X' - C H') (Fig. EGFIG step (7)) and of the update
// (C + alpha P) L^{-T} (Fig. TMFIG with the orthonormalisation of Fig. ONFIG).
//
// Precision: as in the Gram kernel, each FP32 value of Y is split in shared
// memory into two TF32 terms (hi = rna_tf32(y), lo = rna_tf32(y - hi)), M is
// split the same way from FP64 by k_split_small, and hi.hi + hi.lo + lo.hi is
// accumulated in FP32 in tensor memory (FP32-class accuracy, ~2^-22 relative
// per term).
//
// Layout: Y is column-major (rows contiguous), so a TMA box of 32 rows x 32
// columns with the 128-byte swizzle holds 32 lines of 32 rows each (the
// contraction index k is the strided one). The TF32 MMA reads both operands
// K-major, so the converter warps transpose while they split: they read Y
// (and P) from the staging ring and write hi and lo as 128 rows of 128 bytes
// (32 k values), the layout of the Gram kernel's operands. M (hi and lo, k
// contiguous) is loaded K-major by TMA directly.
//
// Rings: staging (TMA -> converters; raw Y and P tiles), operand (converters
// and TMA -> MMA; hi, lo and the M tiles), accumulator (MMA -> epilogue; two
// 128-column TMEM buffers, so the epilogue of one tile overlaps the next).
// Persistent CTAs (one per SM) walk (128-row, 128-column) tiles. Warp roles
// (512 threads): warp 0 TMA for Y/P, warp 1 TMEM allocation and MMA issue
// (one thread), warp 2 TMA for M, warp 3 TMA for the gradient's epilogue
// operands, warps 4-7 form Y = C (+ alpha P), split and transpose (one row
// per thread), warps 8-15 read the accumulator and run the fused epilogue
// (two warps per TMEM lane quarter, one column half each: the epilogue
// streams most of the kernel's bytes, so it gets the warps). Every wait is
// bounded (bit 2 of *err).
//
// The gradient's epilogue reads X', G_prev and P_prev (three of its five
// N x m streams). With plain loads each thread had a few hundred bytes in
// flight and then waited on DRAM; instead warp 3 stages them by TMA, 8
// columns x 128 rows of each per slot, into the P ring that the gradient
// does not use (4 slots, two per column half, so the loads of the next
// 8 columns are in flight while the epilogue works on these).
#include <atomic>
#include <numeric>

#include "dfmath.cuh"
#include "ops.cuh"
#include "tc.cuh"

namespace trm {

namespace {

using namespace tc;

constexpr int BM = 128;  // rows per tile (MMA M)
constexpr int NC = 128;  // output columns per tile (MMA N)
constexpr int BK = 32;   // columns of Y per stage
constexpr int RS = 3;    // staging stages
constexpr int CS = 2;    // operand stages
constexpr int THREADS = 512;
constexpr int CONV0 = 4, NCONV = 4, EPI0 = 8, NEPI = 8;

enum Mode { kStore = 0, kGrad = 1, kSplit64 = 2, kSplitDf = 3 };

constexpr int EC = 8;                // columns per epilogue slot
constexpr int ESLOT = 3 * EC * BM;   // X', G_prev, P_prev: EC columns each
constexpr int NSLOT = 4;             // two per column half

struct MulSmem {
  float raw[RS][BM * BK];   // Y tile as loaded (32 lines of 32 rows each)
  float rawp[RS][BM * BK];  // P tile as loaded; kGrad: the epilogue slots
  float ah[CS][BM * BK];    // Y hi, K-major (128 rows of 32 k values)
  float al[CS][BM * BK];    // Y lo
  float bh[CS][NC * BK];    // M hi, K-major
  float bl[CS][NC * BK];    // M lo
  uint64_t raw_full[RS], raw_empty[RS];
  uint64_t conv_done[CS], b_full[CS], op_empty[CS];
  uint64_t accfull[2], accempty[2], mmadone;
  uint64_t efull[NSLOT], eempty[NSLOT];  // kGrad epilogue slots
  uint32_t tmem_base;
  int failed;
  double red[NEPI][4];
  int last;  // kGrad: this CTA finished last
};

struct MulArgs {
  int64_t N;
  int k, n;        // Y: N x k, M: k x n
  int ntr, nch;    // row tiles, column chunks of 128
  int has_p;       // Y = A + alpha P
  int tri;         // M upper triangular: column j of Y M needs rows k <= j
  const IterScalars* sc;
  float* out;      // kStore: Y M; kGrad: G (N x n, ld N)
  const float* xp; // kGrad
  const float* gprev;
  const float* pprev;
  const float* minv;
  double* part;    // kGrad: 4 sums per CTA
  IterScalars* scw;  // kGrad: the CG scalars (formed by the last CTA)
  const double* c64;  // kSplit64: Cn = (C64 + alpha P) diag(R) + Y M
  const float* p32;
  const double* R;
  double* out64;
  const float* ch;     // kSplitDf: C as FP32 pairs, Cn written as pairs
  const float* cl;
  float* outh;
  float* outl;
  const float* rdiag;  // kSplitDf: diag(R) as pairs (hi[0..n), lo[n..2n))
  int* err;
};
static_assert(NSLOT * ESLOT <= RS * BM * BK,
              "the epilogue slots overlay the P staging ring");

// Converter thread (row i, half h) reads the 16 values of row i in the
// column groups q = 2j + h (j = 0..3) of a staged tile: element (i, k) of a
// staged 32 x 32 box sits in line k at 16-byte chunk ((i % 32) / 4) ^ (k % 8).
__device__ __forceinline__ float staged(const float* t, int i, int k) {
  return t[(i >> 5) * 1024 + k * 32 + (((((i & 31) >> 2) ^ (k & 7))) << 2) +
           (i & 3)];
}

// Tile t of a launch: row tile t / nch, so the nch column chunks of a row
// tile are taken by neighbouring CTAs at about the same time and the
// chunks after the first find the Y (and P) tile in L2 instead of reading
// it again from DRAM; its chunk rotates with the row so that a persistent
// CTA cycles through the chunks (with a triangular M the chunks differ in
// work: chunk c needs the K blocks below (c + 1) NC only).
__device__ __forceinline__ void tile_rc(const MulArgs& a, int t, int& r0,
                                        int& c0) {
  const int row = t / a.nch;
  r0 = row * BM;
  c0 = ((t - row * a.nch + row) % a.nch) * NC;
}
__device__ __forceinline__ int tile_nk(const MulArgs& a, int c0, int nk) {
  return a.tri ? min(nk, (c0 + NC + BK - 1) / BK) : nk;
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
    k_mul_tc(const __grid_constant__ CUtensorMap mapA,
             const __grid_constant__ CUtensorMap mapP,
             const __grid_constant__ CUtensorMap mapBh,
             const __grid_constant__ CUtensorMap mapBl,
             const __grid_constant__ CUtensorMap mapX,
             const __grid_constant__ CUtensorMap mapGp,
             const __grid_constant__ CUtensorMap mapPp, MulArgs args) {
  extern __shared__ unsigned char smem_raw[];
  MulSmem* sm = reinterpret_cast<MulSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = args.ntr * args.nch;
  const int nk = (args.k + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RS; ++s) {
      mbar_init(&sm->raw_full[s], 1);
      mbar_init(&sm->raw_empty[s], NCONV * 32);
    }
    for (int s = 0; s < CS; ++s) {
      mbar_init(&sm->conv_done[s], NCONV * 32);
      mbar_init(&sm->b_full[s], 1);
      mbar_init(&sm->op_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm->accfull[b], 1);
      mbar_init(&sm->accempty[b], NEPI * 32);
    }
    for (int e = 0; e < NSLOT; ++e) {
      mbar_init(&sm->efull[e], 1);
      mbar_init(&sm->eempty[e], NEPI * 16);  // the four warps of one half
    }
    mbar_init(&sm->mmadone, 1);
    sm->failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(&sm->tmem_base, 2 * NC);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp == 0) {
    // ---------------- TMA: Y (and P) into the staging ring ----------------
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)(BM * BK * 4 * (args.has_p ? 2 : 1));
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int r0, c0;
        tile_rc(args, t, r0, c0);
        const int nkt = tile_nk(args, c0, nk);
        for (int kb = 0; kb < nkt; ++kb, ++it) {
          const int s = it % RS;
          if (it >= RS &&
              !mbar_wait(&sm->raw_empty[s], ((it / RS) - 1) & 1, args.err,
                         &sm->failed)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&sm->raw_full[s], bytes);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            tma_load_2d(sm->raw[s] + c * 1024, &mapA, r0 + 32 * c, kb * BK,
                        &sm->raw_full[s]);
            if (args.has_p)
              tma_load_2d(sm->rawp[s] + c * 1024, &mapP, r0 + 32 * c,
                          kb * BK, &sm->raw_full[s]);
          }
        }
      }
      // the copies in flight must land before the CTA may exit
      for (int j = it > RS ? it - RS : 0; j < it; ++j)
        mbar_wait_own(&sm->raw_full[j % RS], (j / RS) & 1, args.err);
    }
  } else if (warp == 2) {
    // ---------------- TMA: M hi/lo into the operand ring ----------------
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int r0, c0;
        tile_rc(args, t, r0, c0);
        const int nkt = tile_nk(args, c0, nk);
        for (int kb = 0; kb < nkt; ++kb, ++it) {
          const int s = it % CS;
          if (it >= CS &&
              !mbar_wait(&sm->op_empty[s], ((it / CS) - 1) & 1, args.err,
                         &sm->failed)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&sm->b_full[s], 2 * NC * BK * 4);
          tma_load_2d(sm->bh[s], &mapBh, kb * BK, c0, &sm->b_full[s]);
          tma_load_2d(sm->bl[s], &mapBl, kb * BK, c0, &sm->b_full[s]);
        }
      }
      for (int j = it > CS ? it - CS : 0; j < it; ++j)
        mbar_wait_own(&sm->b_full[j % CS], (j / CS) & 1, args.err);
    }
  } else if (warp == 3) {
    // ------- TMA: the gradient's epilogue operands into the slots -------
    // Slot sequence: tile tl, column half g, 8-column group q (0..7) is
    // number j = 8 tl + q of half g and lands in slot 2 g + (j & 1).
    if (MODE == kGrad && lane == 0) {
      const bool hg = args.gprev != nullptr, hp = args.pprev != nullptr;
      const uint32_t bytes = (uint32_t)(EC * BM * 4) * (1 + hg + hp);
      float* slots = &sm->rawp[0][0];
      int last[NSLOT] = {-1, -1, -1, -1};  // the number last loaded per slot
      int j = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int r0, c0;
        tile_rc(args, t, r0, c0);
        for (int q = 0; q < 8 && ok; ++q, ++j)
          for (int g = 0; g < 2 && ok; ++g) {
            const int e = 2 * g + (j & 1);
            if (j >= 2 && !mbar_wait(&sm->eempty[e], ((j >> 1) - 1) & 1,
                                     args.err, &sm->failed)) {
              ok = false;
              break;
            }
            float* d = slots + e * ESLOT;
            const int c = c0 + g * (NC / 2) + q * EC;
            mbar_expect_tx(&sm->efull[e], bytes);
            tma_load_2d(d, &mapX, r0, c, &sm->efull[e]);
            if (hg) tma_load_2d(d + EC * BM, &mapGp, r0, c, &sm->efull[e]);
            if (hp) tma_load_2d(d + 2 * EC * BM, &mapPp, r0, c, &sm->efull[e]);
            last[e] = j;
          }
      }
      // the copies in flight must land before the CTA may exit
      for (int e = 0; e < NSLOT; ++e)
        if (last[e] >= 0)
          mbar_wait_own(&sm->efull[e], (last[e] >> 1) & 1, args.err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(BM, NC, false, false);
      int it = 0, tl = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
        const int b = tl & 1;
        if (tl >= 2 && !mbar_wait(&sm->accempty[b], ((tl / 2) - 1) & 1,
                                  args.err, &sm->failed)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(b * NC);
        int r0, c0;
        tile_rc(args, t, r0, c0);
        const int nkt = tile_nk(args, c0, nk);
        for (int kb = 0; kb < nkt; ++kb, ++it) {
          const int s = it % CS;
          const uint32_t par = (it / CS) & 1;
          if (!mbar_wait(&sm->conv_done[s], par, args.err, &sm->failed) ||
              !mbar_wait(&sm->b_full[s], par, args.err, &sm->failed)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t aH = smem_u32(sm->ah[s]), aL = smem_u32(sm->al[s]);
          const uint32_t bH = smem_u32(sm->bh[s]), bL = smem_u32(sm->bl[s]);
          const uint32_t pa[3] = {aH, aH, aL};
          const uint32_t pb[3] = {bH, bL, bH};
#pragma unroll
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk)  // K = 8 per MMA (32 bytes)
              mma_tf32(d, smem_desc(pa[p] + kk * 32, 16, 1024),
                       smem_desc(pb[p] + kk * 32, 16, 1024), idesc,
                       (kb > 0 || p > 0 || kk > 0) ? 1u : 0u);
          mma_commit(&sm->op_empty[s]);
        }
        if (ok) mma_commit(&sm->accfull[b]);
      }
      // every MMA of this thread completes before the TMEM is released
      mma_commit(&sm->mmadone);
      mbar_wait_own(&sm->mmadone, 0, args.err);
    }
  } else if (warp >= CONV0 && warp < EPI0) {
    // ------------- form Y, split it and write it K-major -------------
    const int i = threadIdx.x - CONV0 * 32;  // 0..127: row of the tile
    const bool axpy = args.has_p != 0;
    const float alpha = (axpy && args.sc) ? (float)args.sc->alpha : 0.f;
    int it = 0;
    bool ok = true;
    for (int tt = blockIdx.x; tt < ntiles && ok; tt += gridDim.x) {
      int r0, c0;
      tile_rc(args, tt, r0, c0);
      const int nkt = tile_nk(args, c0, nk);
      for (int kb = 0; kb < nkt; ++kb, ++it) {
        const int rs = it % RS, cs = it % CS;
        if (!mbar_wait(&sm->raw_full[rs], (it / RS) & 1, args.err,
                       &sm->failed)) {
          ok = false;
          break;
        }
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          float y = staged(sm->raw[rs], i, k);
          if (axpy) y = fmaf(alpha, staged(sm->rawp[rs], i, k), y);
          v[k] = y;
        }
        // The staged tile is overwritten next by TMA (async proxy): order
        // these generic-proxy reads before that write.
        fence_proxy_async();
        mbar_arrive(&sm->raw_empty[rs]);
        if (it >= CS && !mbar_wait(&sm->op_empty[cs], ((it / CS) - 1) & 1,
                                   args.err, &sm->failed)) {
          ok = false;
          break;
        }
        float4* hi = reinterpret_cast<float4*>(sm->ah[cs] + i * 32);
        float4* lo = reinterpret_cast<float4*>(sm->al[cs] + i * 32);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int q = j ^ (i & 7);  // 128-byte swizzle
          float4 a, o;
          a.x = tf32_rna(v[4 * j + 0]); o.x = tf32_rna(v[4 * j + 0] - a.x);
          a.y = tf32_rna(v[4 * j + 1]); o.y = tf32_rna(v[4 * j + 1] - a.y);
          a.z = tf32_rna(v[4 * j + 2]); o.z = tf32_rna(v[4 * j + 2] - a.z);
          a.w = tf32_rna(v[4 * j + 3]); o.w = tf32_rna(v[4 * j + 3] - a.w);
          hi[q] = a;
          lo[q] = o;
        }
        fence_proxy_async();
        mbar_arrive(&sm->conv_done[cs]);
      }
    }
  } else if (warp >= EPI0) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;                  // TMEM lane quarter
    const int cbeg = ((warp - EPI0) >> 2) * (NC / 2);  // column half
    const int rr = 32 * q + lane;
    const int64_t N = args.N;
    // Polak-Ribiere sums as double-float pairs (no FP64 instruction per
    // batch: GB300's FP64 pipe is 1/64 of its FP32 rate)
    F2 s_sum[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    double alpha64 = 0.0;
    if (MODE == kSplit64 && args.sc) alpha64 = args.sc->alpha;
    F2 alpha2 = {0.f, 0.f};
    if (MODE == kSplitDf && args.sc) alpha2 = df_of(args.sc->alpha);
    const float* slots = &sm->rawp[0][0];
    const int half = cbeg ? 1 : 0;
    const bool hg = args.gprev != nullptr, hp = args.pprev != nullptr;
    bool dead = false;
    int tl = 0;
    for (int t = blockIdx.x; t < ntiles && !dead; t += gridDim.x, ++tl) {
      const int b = tl & 1;
      // warp-uniform outcome: the TMEM loads below are .sync.aligned
      const bool got =
          mbar_wait(&sm->accfull[b], (tl / 2) & 1, args.err, &sm->failed);
      if (!__all_sync(0xffffffffu, got)) break;
      fence_after();
      int r0, c0;
      tile_rc(args, t, r0, c0);
      const int64_t row = (int64_t)r0 + rr;
      const bool rin = row < N;
      float mi = 1.f;
      if (MODE == kGrad && rin && args.minv) mi = args.minv[row];
#pragma unroll 1
      for (int cb = cbeg; cb < cbeg + NC / 2; cb += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * NC + cb), r);
        if (MODE == kGrad) {
          // the two slots of these 16 columns: wait, read, release (every
          // thread of the half arrives, rows past N included)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = 8 * tl + (cb - cbeg) / EC + h;
            const int e = 2 * half + (j & 1);
            const bool in_slot =
                mbar_wait(&sm->efull[e], (j >> 1) & 1, args.err, &sm->failed);
            if (!__all_sync(0xffffffffu, in_slot)) {
              dead = true;
              break;
            }
            const float* d = slots + e * ESLOT + rr;
            float gg = 0.f, gmg = 0.f, pmg = 0.f, gpp = 0.f;
            if (rin) {
#pragma unroll
              for (int u = 0; u < EC; ++u) {
                const int col = c0 + cb + h * EC + u;
                if (col < args.n) {
                  const float x = d[u * BM];
                  const float gp = hg ? d[(EC + u) * BM] : 0.f;
                  const float pp = hp ? d[(2 * EC + u) * BM] : 0.f;
                  const float g = -2.f * (x - __uint_as_float(r[h * EC + u]));
                  args.out[row + (int64_t)col * N] = g;
                  const float mg = mi * g;
                  gg = fmaf(g, g, gg);
                  gmg = fmaf(g, mg, gmg);
                  pmg = fmaf(gp, mg, pmg);
                  gpp = fmaf(g, pp, gpp);
                }
              }
            }
            // the slot is overwritten next by TMA (async proxy)
            fence_proxy_async();
            mbar_arrive(&sm->eempty[e]);
            s_sum[0] = df_add(s_sum[0], F2{gg, 0.f});
            s_sum[1] = df_add(s_sum[1], F2{gmg, 0.f});
            s_sum[2] = df_add(s_sum[2], F2{pmg, 0.f});
            s_sum[3] = df_add(s_sum[3], F2{gpp, 0.f});
          }
          if (dead) break;
          continue;
        }
        if (!rin) continue;
        if (MODE == kStore) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int col = c0 + cb + e;
            if (col < args.n)
              args.out[row + (int64_t)col * N] = __uint_as_float(r[e]);
          }
        } else if (MODE == kSplitDf) {
#pragma unroll
          for (int h = 0; h < 16; h += 8) {
            float hv[8], lv[8], pv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int col = c0 + cb + h + e;
              const int64_t idx = row + (int64_t)col * N;
              const bool in = col < args.n;
              hv[e] = in ? args.ch[idx] : 0.f;
              lv[e] = in ? args.cl[idx] : 0.f;
              pv[e] = in ? args.p32[idx] : 0.f;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int col = c0 + cb + h + e;
              if (col < args.n) {
                const F2 y = df_add(F2{hv[e], lv[e]},
                                    df_mul(alpha2, F2{pv[e], 0.f}));
                const F2 rd = {args.rdiag[col], args.rdiag[args.n + col]};
                const F2 t = df_add(df_mul(y, rd),
                                    F2{__uint_as_float(r[h + e]), 0.f});
                const int64_t idx = row + (int64_t)col * N;
                args.outh[idx] = t.h;
                args.outl[idx] = t.l;
              }
            }
          }
        } else {
#pragma unroll
          for (int h = 0; h < 16; h += 8) {
            double cv[8];
            float pv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int col = c0 + cb + h + e;
              const int64_t idx = row + (int64_t)col * N;
              const bool in = col < args.n;
              cv[e] = in ? args.c64[idx] : 0.0;
              pv[e] = in ? args.p32[idx] : 0.f;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int col = c0 + cb + h + e;
              if (col < args.n) {
                const double y = fma(alpha64, (double)pv[e], cv[e]);
                args.out64[row + (int64_t)col * N] =
                    fma(y, args.R[col + (int64_t)col * args.k],
                        (double)__uint_as_float(r[h + e]));
              }
            }
          }
        }
      }
      fence_before();
      mbar_arrive(&sm->accempty[b]);
    }
    if (MODE == kGrad) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          s_sum[j] = df_add(s_sum[j],
                            F2{__shfl_xor_sync(0xffffffffu, s_sum[j].h, o),
                               __shfl_xor_sync(0xffffffffu, s_sum[j].l, o)});
      if (lane == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          sm->red[warp - EPI0][j] = (double)s_sum[j].h + (double)s_sum[j].l;
      asm volatile("bar.sync 1, %0;" ::"n"(NEPI * 32) : "memory");
      if (threadIdx.x == EPI0 * 32) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          double t = sm->red[0][j];
#pragma unroll
          for (int w = 1; w < NEPI; ++w) t += sm->red[w][j];
          args.part[(size_t)blockIdx.x * 4 + j] = t;
        }
        // the last CTA to finish forms the CG scalars (the fence orders
        // this CTA's sums before its count)
        __threadfence();
        const unsigned prev = atomicAdd(&args.scw->grad_done, 1u);
        sm->last = prev == gridDim.x - 1;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(NEPI * 32) : "memory");
      if (sm->last) {
        __threadfence();
        // fixed order: thread t sums the CTAs t, t + 256, ..., then warps
        // by shuffles, then the warps in order (whichever CTA is last)
        const int t = threadIdx.x - EPI0 * 32;
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = t; c < (int)gridDim.x; c += NEPI * 32)
#pragma unroll
          for (int j = 0; j < 4; ++j) v[j] += __ldcg(&args.part[(size_t)c * 4 + j]);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
            v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
        asm volatile("bar.sync 1, %0;" ::"n"(NEPI * 32) : "memory");
        if (lane == 0)
#pragma unroll
          for (int j = 0; j < 4; ++j) sm->red[warp - EPI0][j] = v[j];
        asm volatile("bar.sync 1, %0;" ::"n"(NEPI * 32) : "memory");
        if (t == 0) {
          double tot[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            tot[j] = sm->red[0][j];
#pragma unroll
            for (int w = 1; w < NEPI; ++w) tot[j] += sm->red[w][j];
          }
          cg_scalars(tot, args.k, args.scw);
          args.scw->grad_done = 0u;  // ready for the next launch
        }
      }
    }
  }
  __syncwarp();
  fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    tmem_dealloc(tmem, 2 * NC);
  }
}

// hi + lo = M (FP64 k x n, ld k) to ~2^-22 relative, as TF32 values stored in
// FP32 with leading dimension ldm; zero_diag leaves the diagonal out.
__global__ void k_split_small(int k, int n, int ldm, const double* __restrict__ M,
                              float* __restrict__ hi, float* __restrict__ lo,
                              int zero_diag, float* __restrict__ diag2) {
  const int total = ldm * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += gridDim.x * blockDim.x) {
    const int i = e % ldm, j = e / ldm;
    double x = 0.0;
    if (i < k && !(zero_diag && i == j)) x = M[i + (size_t)j * k];
    const float h = tf32_rna((float)x);
    hi[e] = h;
    lo[e] = tf32_rna((float)(x - (double)h));
    if (diag2 && i == j && i < k) {  // the left-out diagonal as FP32 pairs
      const F2 d = df_of(M[i + (size_t)j * k]);
      diag2[j] = d.h;
      diag2[n + j] = d.l;
    }
  }
}

int ldm_of(int k) { return (k + 3) & ~3; }

// Persistent grid of a product with a triangular M: nch x q CTAs with q
// coprime to the chunk count nch, so that each CTA steps through every
// column chunk (tile_rc) and the CTAs share the uneven chunks evenly.
int tri_grid(int64_t N, int n) {
  const int nch = ceil_div(n, NC);
  const int g = mul_tc_parts(N, n);
  if (nch == 1 || g < sm_count()) return g;
  int q = g / nch;
  while (q > 1 && std::gcd(q, nch) != 1) --q;
  return q * nch;
}

template <int MODE>
void launch(const MulArgs& a0, const float* A, const float* P,
            const double* M, int zero_diag, float* ws, cudaStream_t s,
            int* grid_out) {
  MulArgs a = a0;
  const int ldm = ldm_of(a.k);
  float* hi = ws;
  float* lo = ws + (size_t)ldm * a.n;
  float* diag2 = MODE == kSplitDf ? lo + (size_t)ldm * a.n : nullptr;
  if (diag2) a.rdiag = diag2;
  k_split_small<<<ceil_div((int64_t)ldm * a.n, 256), 256, 0, s>>>(
      a.k, a.n, ldm, M, hi, lo, zero_diag, diag2);
  TRM_CHECK_LAUNCH();
  CUtensorMap mA = f32_map(A, a.N, a.k, a.N, 32, BK);
  CUtensorMap mP = f32_map(P ? P : A, a.N, a.k, a.N, 32, BK);
  CUtensorMap mBh = f32_map(hi, a.k, a.n, ldm, BK, NC);
  CUtensorMap mBl = f32_map(lo, a.k, a.n, ldm, BK, NC);
  // the gradient's epilogue operands, 128 rows x EC columns per box
  CUtensorMap mX = mA, mGp = mA, mPp = mA;
  if (MODE == kGrad) {
    mX = f32_map(a.xp, a.N, a.n, a.N, BM, EC, false);
    if (a.gprev) mGp = f32_map(a.gprev, a.N, a.n, a.N, BM, EC, false);
    if (a.pprev) mPp = f32_map(a.pprev, a.N, a.n, a.N, BM, EC, false);
  }
  a.ntr = (int)ceil_div(a.N, (int64_t)BM);
  a.nch = ceil_div(a.n, NC);
  a.has_p = P ? 1 : 0;
  const int grid = a.tri ? tri_grid(a.N, a.n) : mul_tc_parts(a.N, a.n);
  const size_t smem = sizeof(MulSmem) + 1024;
  static std::atomic<int> attr_dev{-1};  // launches may come from several threads
  int dev = 0;
  TRM_CUDA(cudaGetDevice(&dev));
  if (attr_dev.load(std::memory_order_relaxed) != dev) {
    TRM_CUDA(cudaFuncSetAttribute(k_mul_tc<MODE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    attr_dev.store(dev, std::memory_order_relaxed);
  }
  k_mul_tc<MODE><<<grid, THREADS, smem, s>>>(mA, mP, mBh, mBl, mX, mGp, mPp,
                                              a);
  TRM_CHECK_LAUNCH();
  if (grid_out) *grid_out = grid;
}

}  // namespace

bool mul_tc_eligible(int64_t N, int k, int n, const TcWork* tw) {
  if (!tw || !tw->msplit || !tw->err) return false;
  if (N % 4 != 0 || N < BM || k < 32 || n < 32) return false;
  if (tw->msplit_floats < mul_tc_work_floats(k, n)) return false;
  return encode_fn() != nullptr;
}

size_t mul_tc_work_floats(int k, int n) {
  return 2 * (size_t)ldm_of(k) * n + 2 * (size_t)n;
}

int mul_tc_parts(int64_t N, int n) {
  const int64_t tiles = (int64_t)ceil_div(N, (int64_t)BM) * ceil_div(n, NC);
  // persistent CTAs, one per SM at most, and at least two tiles each below
  // 2 x SMs tiles (each CTA holds a whole SM: a small problem leaves the
  // rest of the GPU to concurrent solves)
  const int64_t two = (tiles + 1) / 2;
  return (int)(tiles >= 2 * sm_count() ? sm_count() : (two < 1 ? 1 : two));
}

void mul_tc_store(int64_t N, int k, int n, const float* A, const float* P,
                  const IterScalars* sc, const double* M, float* out,
                  const TcWork& tw, cudaStream_t s) {
  MulArgs a{};
  a.N = N; a.k = k; a.n = n; a.sc = sc; a.out = out; a.err = tw.err;
  a.tri = 1;  // the rotation's L^{-T}
  launch<kStore>(a, A, P, M, 0, tw.msplit, s, nullptr);
}

int mul_tc_grad(int64_t N, int m, const float* C, const double* Hp,
                const float* Xp, float* G, const float* Gprev,
                const float* Pprev, const float* minv, double* part,
                IterScalars* sc, const TcWork& tw, cudaStream_t s) {
  MulArgs a{};
  a.N = N; a.k = m; a.n = m; a.out = G; a.xp = Xp; a.gprev = Gprev;
  a.pprev = Pprev; a.minv = minv; a.part = part; a.scw = sc; a.err = tw.err;
  int grid = 0;
  launch<kGrad>(a, C, nullptr, Hp, 0, tw.msplit, s, &grid);
  return grid;
}

void mul_tc_splitdf(int64_t N, int m, const float* Ch, const float* Cl,
                    const float* P, const IterScalars* sc, const double* R,
                    float* Cnh, float* Cnl, const TcWork& tw, cudaStream_t s) {
  MulArgs a{};
  a.N = N; a.k = m; a.n = m; a.sc = sc; a.ch = Ch; a.cl = Cl; a.p32 = P;
  a.R = R; a.outh = Cnh; a.outl = Cnl; a.err = tw.err;
  a.tri = 1;
  launch<kSplitDf>(a, Ch, P, R, 1, tw.msplit, s, nullptr);
}

void mul_tc_split64(int64_t N, int m, const float* C32, const float* P,
                    const double* C64, const IterScalars* sc, const double* R,
                    double* Cn, const TcWork& tw, cudaStream_t s) {
  MulArgs a{};
  a.N = N; a.k = m; a.n = m; a.sc = sc; a.c64 = C64; a.p32 = P; a.R = R;
  a.out64 = Cn; a.err = tw.err;
  a.tri = 1;
  launch<kSplit64>(a, C32, P, R, 1, tw.msplit, s, nullptr);
}

}  // namespace trm
