// Persistent warp-specialised tcgen05 GEMM (see tc_gemm.cuh).
//
// Roles per CTA (320 threads, one CTA per SM):
//   warp 0      one thread issues TMA loads into an S-stage shared ring
//   warp 1      allocates TMEM; one thread issues tcgen05.mma (K = 16 each)
//   warps 2..9  epilogue: TMEM -> registers -> fused op -> global memory;
//               two warps per TMEM lane quadrant take alternate 32-column
//               chunks
// Accumulators are double-buffered in TMEM when they fit, so the epilogue
// of one tile overlaps the MMAs of the next. Every mbarrier wait is bounded
// in time; a timeout sets *err and the roles wind down without hanging.
//
// Pair mode (k_tc_gemm_pair, clusters of two CTAs on two SMs; the weight
// gradients dW = delta^T h with MN-major operands): a tile is 256 rows
// (output neurons) x N; the even CTA's MMA thread issues
// tcgen05.mma.cta_group::2 with M = 256, each CTA loading its own 128 rows
// of A (delta columns) and half of the N columns of B (h), and each CTA's
// epilogue reads its own 128 rows of D from its TMEM. Per SM this halves the
// B operand streamed through TMA and read by the tensor core, and the h
// block of a K step is fetched once per pair instead of once per CTA. Both
// CTAs' loads of a stage count on the even CTA's stage barrier; MMA
// completions are multicast to both CTAs' barriers; the odd CTA's epilogue
// releases an accumulator to the even CTA remotely.
#include "tc_gemm.cuh"
#include "tc_pair.cuh"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>

#include <cstring>

namespace dinr {

using namespace tc;

namespace {
constexpr int BM = 128, BK = 64;
constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int kOnesBytes = 1024;

constexpr int kStageBytes = 32 * 32 * 2;  // one warp's 32 x 32 BF16 output block

struct Smem {
  uint8_t *a, *b, *ones;
  uint8_t *stage;  // [8 epilogue warps][2] output blocks (stage_out)
  float *dot;  // [2 tile parities][2 halves][128 rows]
  uint64_t *full, *empty, *tfull, *tempty, *drain, *dotbar;
  uint32_t *tslot;
};

__device__ __forceinline__ Smem carve(uint8_t *base, const TcGemmArgs &p) {
  Smem s;
  s.a = base;
  s.b = base + (size_t)p.stages * p.a_bytes;
  s.ones = s.b + (size_t)p.stages * p.b_bytes;
  s.stage = s.ones + kOnesBytes;
  s.dot = reinterpret_cast<float *>(s.stage + (p.stage_out ? kEpiWarps * 2 * kStageBytes : 0));
  s.full = reinterpret_cast<uint64_t *>(s.dot + 2 * 2 * 128);
  s.empty = s.full + p.stages;
  s.tfull = s.empty + p.stages;
  s.tempty = s.tfull + 2;
  s.drain = s.tempty + 2;
  s.dotbar = s.drain + 1;
  s.tslot = reinterpret_cast<uint32_t *>(s.dotbar + 2);
  return s;
}

__device__ __forceinline__ int acc_stride(const TcGemmArgs &p) {
  int cols = p.N + (p.with_db ? 16 : 0);
  return (cols + 31) / 32 * 32;
}

__device__ __forceinline__ int n_tn(const TcGemmArgs &p) { return p.n_tn > 1 ? p.n_tn : 1; }

// M units a tile index runs over: 128-row tiles, or pairs of them.
__device__ __forceinline__ int m_units(const TcGemmArgs &p) {
  return p.pair ? (p.m_tiles + 1) / 2 : p.m_tiles;
}
__device__ __forceinline__ int n_tiles_of(const TcGemmArgs &p) {
  return m_units(p) * (p.n_tn > 1 ? p.n_tn : 1) * p.splits;
}
// This CTA's first tile and tile stride (a pair shares its tiles).
__device__ __forceinline__ int first_tile(const TcGemmArgs &p) {
  return p.pair ? (int)blockIdx.x / 2 : (int)blockIdx.x;
}
__device__ __forceinline__ int tile_stride(const TcGemmArgs &p) {
  return p.pair ? (int)gridDim.x / 2 : (int)gridDim.x;
}

// Tile t -> M tile (of this CTA of a pair: rank), N tile, K split and the
// K range of the split.
__device__ __forceinline__ void tile_range(const TcGemmArgs &p, int t, int &mt, int &nt, int &sp,
                                           long long &k0, int &nk, int rank = 0) {
  const int mu = m_units(p);
  if (p.splits <= 1) {
    // no K split (forward, input gradients): the N tiles of one M tile (or
    // pair of M tiles) are consecutive, so CTAs that run at the same time
    // read the same rows of A, which then come from HBM once and from L2
    // for the other N tiles
    nt = t % n_tn(p);
    mt = p.pair ? 2 * (t / n_tn(p)) + rank : t / n_tn(p);
    sp = 0;
  } else {
    mt = p.pair ? 2 * (t % mu) + rank : t % mu;
    const int rest = t / mu;
    nt = rest % n_tn(p);
    sp = rest / n_tn(p);
  }
  k0 = (long long)sp * p.k_per_split;
  long long k1 = k0 + p.k_per_split < p.K ? k0 + p.k_per_split : p.K;
  const int bk = tc_k_block(p);
  nk = (int)((k1 - k0 + bk - 1) / bk);
}

// Four E4M3 bytes (a in the lowest), round to nearest even, saturating.
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  uint16_t lo, hi;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

// BF16 pair (lo, hi) of max(x, 0), rounded to nearest even.
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// 0xFFFF in each half of a BF16 pair whose value is > 0.
__device__ __forceinline__ uint32_t bf16x2_positive(uint32_t w) {
  uint32_t m;
  asm("set.gt.u32.bf16x2 %0, %1, %2;" : "=r"(m) : "r"(w), "r"(0u));
  return m;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

template <bool kPair>
__device__ void producer(const CUtensorMap *ta, const CUtensorMap *tb, const TcGemmArgs &p,
                         const Smem &s) {
  prefetch_tmap(ta);
  prefetch_tmap(tb);
  const int S = p.stages;
  const uint32_t nb_mn = (uint32_t)(((kPair ? p.N / 2 : p.N) + 63) / 64);
  const uint32_t tx = (uint32_t)p.a_bytes + (uint32_t)p.b_bytes;
  const int kblk = tc_k_block(p);
  const int mn_box = kblk * 128;  // bytes of one 64-column MN-major box
  uint32_t it = 0;
  const int rank = kPair ? (int)cluster_ctarank() : 0;
  const int n_tiles = n_tiles_of(p);
  for (int t = first_tile(p); t < n_tiles; t += tile_stride(p)) {
    int mt, nt, sp, nk;
    long long k0;
    tile_range(p, t, mt, nt, sp, k0, nk, rank);
    // a pair's B tile: this CTA's half of the N rows
    const int n0 = nt * p.N + (kPair ? rank * (p.N / 2) : 0);
    for (int kb = 0; kb < nk; ++kb, ++it) {
      uint32_t st = it % S, rd = it / S;
      if (!mbar_wait(&s.empty[st], (rd & 1) ^ 1, p.err, 1)) return;
      int kx = (int)(k0 + (long long)kb * kblk);
      uint8_t *da = s.a + (size_t)st * p.a_bytes;
      uint8_t *db = s.b + (size_t)st * p.b_bytes;
      if constexpr (kPair) {
        // both CTAs' loads count on the even CTA's barrier, which expects
        // the bytes of both (its MMA thread reads both halves)
        if (rank == 0) mbar_expect_tx(&s.full[st], 2 * tx);
        const uint32_t bar = mapa_shared(smem_u32(&s.full[st]), 0);
        // this CTA's 128 rows of A and its half of the N rows of B
        if (!p.a_mn) {
          tma_load_2d_pair(ta, bar, da, kx, mt * BM);
        } else {
          tma_load_2d_pair(ta, bar, da, mt * BM, kx);
          tma_load_2d_pair(ta, bar, da + mn_box, mt * BM + 64, kx);
        }
        if (!p.b_mn) {
          tma_load_2d_pair(tb, bar, db, kx, n0);
        } else {
          for (uint32_t j = 0; j < nb_mn; ++j)
            tma_load_2d_pair(tb, bar, db + mn_box * j, n0 + 64 * (int)j, kx);
        }
        continue;
      }
      mbar_expect_tx(&s.full[st], tx);
      if (!p.a_mn) {
        tma_load_2d(ta, &s.full[st], da, kx, mt * BM);
      } else {
        tma_load_2d(ta, &s.full[st], da, mt * BM, kx);
        tma_load_2d(ta, &s.full[st], da + mn_box, mt * BM + 64, kx);
      }
      if (!p.b_mn) {
        tma_load_2d(tb, &s.full[st], db, kx, n0);
      } else {
        for (uint32_t j = 0; j < nb_mn; ++j)
          tma_load_2d(tb, &s.full[st], db + mn_box * j, n0 + 64 * (int)j, kx);
      }
    }
  }
  // Before the CTA can exit, every load issued must have landed (a pair's
  // loads are counted on the even CTA's barriers: the odd CTA's landed
  // before the even CTA's MMAs read them, and the final cluster barrier
  // keeps the odd CTA alive until then).
  if (kPair && rank != 0) return;
  uint32_t n = it < (uint32_t)S ? it : (uint32_t)S;
  for (uint32_t q = it - n; q < it; ++q) {
    uint32_t st = q % S, rd = q / S;
    if (!mbar_wait(&s.full[st], rd & 1, p.err, 6)) break;
  }
}

template <bool kPair>
__device__ void mma_issuer(const TcGemmArgs &p, const Smem &s, uint32_t tbase) {
  const int S = p.stages;
  const int n_acc = 2 * acc_stride(p) <= 512 ? 2 : 1;
  const uint32_t idesc = p.fp8 ? idesc_e4m3(BM, p.N)
                               : idesc_bf16(p.pair ? 2 * BM : BM, p.N, p.a_mn, p.b_mn);
  const uint32_t idesc_db = idesc_bf16(BM, 16, p.a_mn, false);
  const uint32_t idesc_db2 = idesc_bf16(2 * BM, 16, p.a_mn, false);
  // an all-ones 16 x 16 BF16 block, no swizzle: every layout reads ones
  const uint64_t ones = smem_desc(smem_u32(s.ones), 128, 256, 0);
  // instructions per stage, each over 32 bytes of K (16 BF16 or 32 E4M3)
  const int n_k16 = p.a_mn ? tc_k_block(p) / 16 : BK / 16;
  const uint32_t mn_box = (uint32_t)tc_k_block(p) * 128;
  uint32_t it = 0, lt = 0;
  const int n_tiles = n_tiles_of(p);
  bool ok = true;
  for (int t = first_tile(p); t < n_tiles && ok; t += tile_stride(p), ++lt) {
    int mt, nt, sp, nk;
    long long k0;
    tile_range(p, t, mt, nt, sp, k0, nk);
    const bool db_tile = p.with_db && nt == 0;
    uint32_t ab = lt % n_acc, ar = lt / n_acc;
    if (!mbar_wait(&s.tempty[ab], (ar & 1) ^ 1, p.err, 2)) break;
    tc_fence_after();
    uint32_t d = tbase + ab * (uint32_t)acc_stride(p);
    for (int kb = 0; kb < nk; ++kb, ++it) {
      uint32_t st = it % S, rd = it / S;
      if (!mbar_wait(&s.full[st], rd & 1, p.err, 3)) {
        ok = false;
        break;
      }
      tc_fence_after();
      uint32_t aa = smem_u32(s.a + (size_t)st * p.a_bytes);
      uint32_t ba = smem_u32(s.b + (size_t)st * p.b_bytes);
#pragma unroll
      for (int k = 0; k < n_k16; ++k) {
        // K-major: the next 16 elements of K are 32 bytes further along
        // each swizzled 128-byte row; MN-major: 16 more rows of 128 bytes.
        uint64_t adesc = p.a_mn ? smem_desc(aa + 2048 * k, mn_box, 1024, kSwizzle128)
                                : smem_desc(aa + 32 * k, 16, 1024, kSwizzle128);
        uint64_t bdesc = p.b_mn ? smem_desc(ba + 2048 * k, mn_box, 1024, kSwizzle128)
                                : smem_desc(ba + 32 * k, 16, 1024, kSwizzle128);
        uint32_t acc = (kb | k) != 0;
        // both kinds take 32 bytes of K per instruction (16 BF16 or 32 E4M3)
        if constexpr (kPair) {
          mma_bf16_pair(d, adesc, bdesc, idesc, acc);
          if (db_tile) mma_bf16_pair(d + p.N, adesc, ones, idesc_db2, acc);
        } else {
          if (p.fp8)
            mma_fp8(d, adesc, bdesc, idesc, acc);
          else
            mma_bf16(d, adesc, bdesc, idesc, acc);
          if (db_tile) mma_bf16(d + p.N, adesc, ones, idesc_db, acc);
        }
      }
      if constexpr (kPair)
        mma_commit_pair_both(&s.empty[st]);
      else
        mma_commit(&s.empty[st]);
    }
    if (ok) {
      if constexpr (kPair)
        mma_commit_pair_both(&s.tfull[ab]);
      else
        mma_commit(&s.tfull[ab]);
    }
  }
  // all MMAs of this thread must have completed before TMEM is freed (a
  // pair's commit arrives on the drain barrier of both CTAs; only this
  // one waits)
  if constexpr (kPair)
    mma_commit_pair_both(s.drain);
  else
    mma_commit(s.drain);
  mbar_wait(s.drain, 0, p.err, 4);
}

__device__ __forceinline__ void load_h32(const __nv_bfloat16 *p, uint4 (&h)[4]) {
  const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
  for (int j = 0; j < 4; ++j) h[j] = q[j];
}

__device__ __forceinline__ bool bf16_positive(uint32_t b) { return b != 0 && (b & 0x8000u) == 0; }

// d/dz of z sigmoid(z) = sigmoid(z) (1 + z (1 - sigmoid(z))).
__device__ __forceinline__ float swish_grad(float z) {
  const float s = __frcp_rn(1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// kEpi, kAct (ReLU 0, Swish 1) and kFp8 are fixed per kernel, so that an
// epilogue carries no work of the other kinds (a runtime switch left the
// Swish and FP8 arithmetic in the BF16 ReLU epilogue: 13 % of the wide
// network's forward GEMM time).
template <int kEpi, int kAct, bool kFp8>
__device__ void epilogue(const TcGemmArgs &p, const Smem &s, uint32_t tbase,
                         const CUtensorMap *tout) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int q = warp & 3;              // TMEM lane quadrant this warp may access
  const int half = (warp - 2) / 4;     // which alternate 32-column chunks
  const int n_acc = 2 * acc_stride(p) <= 512 ? 2 : 1;
  const int n_tiles = n_tiles_of(p);
  const int n_chunks = (p.N + 31) / 32;
  const int rank = p.pair ? (int)cluster_ctarank() : 0;
  uint32_t lt = 0, staged = 0;
  for (int t = first_tile(p); t < n_tiles; t += tile_stride(p), ++lt) {
    int mt, nt, sp, nk;
    long long k0;
    tile_range(p, t, mt, nt, sp, k0, nk, rank);
    const int n0 = nt * p.N;
    uint32_t ab = lt % n_acc, ar = lt / n_acc;
    const int r_in = q * 32 + lane;
    const int row = mt * BM + r_in;
    const bool live = row < p.M;
    // prefetch the mask operand of this warp's first chunk
    uint4 hcur[4], hnext[4];
    if (kEpi == kTcDx && live && half < n_chunks)
      load_h32(p.hprev + (long long)row * p.ldh + n0 + half * 32, hcur);
    if (!warp_wait(&s.tfull[ab], ar & 1, p.err, 5)) return;
    tc_fence_after();
    const uint32_t trow = tbase + ((uint32_t)(q * 32) << 16) + ab * (uint32_t)acc_stride(p);
    float dot = 0.0f;
    const float descale = kFp8 ? *p.scale_a * *p.scale_b : 1.0f;
    const float inv_out = kFp8 && p.out8 ? 1.0f / *p.scale_out : 0.0f;
    float amax = 0.0f;
    for (int ch = half; ch < n_chunks; ch += 2) {
      const int c0 = n0 + ch * 32;  // output column of the chunk
      if (kEpi == kTcDx && live && ch + 2 < n_chunks)
        load_h32(p.hprev + (long long)row * p.ldh + c0 + 64, hnext);
      // forward: the chunk's bias first, so that its load overlaps the TMEM load
      float4 bb[8];
      if (kEpi == kTcFwd) {
        const float4 *b4 = reinterpret_cast<const float4 *>(p.bias + c0);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          bb[j] = c0 + 4 * j < p.n_store ? __ldg(b4 + j) : make_float4(0, 0, 0, 0);
      }
      float v[32];
      tmem_ld32(trow + ch * 32, v);
      // the chunk's BF16 output pairs (forward and input gradients; rows past
      // M stay zero and are clipped by the staged store's tensor map)
      uint32_t ow[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) ow[k] = 0u;
      // BF16 ReLU forward: z stays in v and the ReLU is taken in the packing
      constexpr bool kReluPack = kEpi == kTcFwd && kAct == 0 && !kFp8;
      if (live) {
        if (kEpi == kTcFwd) {
          // z = descale * acc + bias; x = act(z). Swish uses a fast
          // exponential and reciprocal (relative error about 1e-6, far below
          // the BF16 rounding of x).
          float x[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float4 b = bb[i / 4];
            const float bi = (i & 3) == 0 ? b.x : (i & 3) == 1 ? b.y : (i & 3) == 2 ? b.z : b.w;
            const float z = kFp8 ? fmaf(v[i], descale, bi) : v[i] + bi;
            x[i] = kAct ? z * __frcp_rn(1.0f + __expf(-z)) : fmaxf(z, 0.0f);
            v[i] = z;
            if (kFp8) amax = fmaxf(amax, fabsf(x[i]));
          }
          if (p.w_out) {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (c0 + i < p.n_store) dot = fmaf(x[i], __ldg(p.w_out + c0 + i), dot);
          }
          if (kAct && p.zpre && c0 + 32 <= p.n_store) {
            uint4 *oz = reinterpret_cast<uint4 *>(p.zpre + (long long)row * p.ldz + c0);
#pragma unroll
            for (int j = 0; j < 4; ++j)
              oz[j] = make_uint4(pack_bf16(v[8 * j], v[8 * j + 1]),
                                 pack_bf16(v[8 * j + 2], v[8 * j + 3]),
                                 pack_bf16(v[8 * j + 4], v[8 * j + 5]),
                                 pack_bf16(v[8 * j + 6], v[8 * j + 7]));
          }
          if (!kReluPack) {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = x[i];
          }
          if (kFp8 && p.out8 && c0 + 32 <= p.n_store) {
            uint32_t q8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
              q8[j] = pack_e4m3x4(v[4 * j] * inv_out, v[4 * j + 1] * inv_out,
                                  v[4 * j + 2] * inv_out, v[4 * j + 3] * inv_out);
            uint4 *o8 = reinterpret_cast<uint4 *>(p.out8 + (long long)row * p.ldo8 + c0);
            o8[0] = make_uint4(q8[0], q8[1], q8[2], q8[3]);
            o8[1] = make_uint4(q8[4], q8[5], q8[6], q8[7]);
          }
#pragma unroll
          for (int k = 0; k < 16; ++k)
            ow[k] = kReluPack ? pack_bf16_relu(v[2 * k], v[2 * k + 1])
                              : pack_bf16(v[2 * k], v[2 * k + 1]);
        } else if (kEpi == kTcDx) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint32_t w[4] = {hcur[j].x, hcur[j].y, hcur[j].z, hcur[j].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (kAct) {
                ow[4 * j + e] =
                    pack_bf16(v[8 * j + 2 * e] * swish_grad(__uint_as_float(w[e] << 16)),
                              v[8 * j + 2 * e + 1] * swish_grad(__uint_as_float(w[e] & 0xFFFF0000u)));
              } else {
                // the ReLU mask of the pair from one packed compare
                ow[4 * j + e] = pack_bf16(v[8 * j + 2 * e], v[8 * j + 2 * e + 1]) &
                                bf16x2_positive(w[e]);
              }
            }
          }
        }
        if ((kEpi == kTcFwd || kEpi == kTcDx) && !p.stage_out) {
          if (c0 + 32 <= p.n_store) {
            uint4 *o = reinterpret_cast<uint4 *>(p.out + (long long)row * p.ldo + c0);
#pragma unroll
            for (int j = 0; j < 4; ++j)
              o[j] = make_uint4(ow[4 * j], ow[4 * j + 1], ow[4 * j + 2], ow[4 * j + 3]);
          } else {
            uint16_t *o = reinterpret_cast<uint16_t *>(p.out + (long long)row * p.ldo + c0);
            for (int i = 0; i < 32 && c0 + i < p.n_store; ++i)
              o[i] = (uint16_t)(ow[i >> 1] >> (16 * (i & 1)));
          }
        } else if (kEpi == kTcDw) {
          float *o = p.part + ((long long)sp * p.M + row) * p.part_ld + c0;
          for (int i = 0; i < 32 && c0 + i < p.n_store; ++i) o[i] = v[i];
        }
      }
      if (p.stage_out) {
        // the warp's 32 x 32 block through shared memory and one TMA store
        // (rows past M are clipped by the tensor map)
        uint8_t *stg = s.stage + (size_t)((warp - 2) * 2 + (staged & 1)) * kStageBytes;
        ++staged;
        if (lane == 0) bulk_wait_read1();  // this buffer's store of two chunks ago has read it
        __syncwarp();
        uint4 *o = reinterpret_cast<uint4 *>(stg + lane * 64);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          o[j] = make_uint4(ow[4 * j], ow[4 * j + 1], ow[4 * j + 2], ow[4 * j + 3]);
        fence_async_smem();
        __syncwarp();
        const int row0 = mt * BM + q * 32;
        if (lane == 0 && row0 < p.M) {
          tma_store_2d(tout, stg, c0, row0);
          bulk_commit();
        }
      }
      if (kEpi == kTcDx) {
#pragma unroll
        for (int j = 0; j < 4; ++j) hcur[j] = hnext[j];
      }
    }
    if (kFp8 && p.amax) {
      // activations are non-negative: their float bits order like integers
      const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(amax));
      if (lane == 0 && m != 0u) atomicMax(p.amax, m);
    }
    if (kEpi == kTcDw && p.with_db && nt == 0 && half == 0) {
      float v[32];
      tmem_ld32(trow + p.N, v);  // 16 db columns (all equal) + padding
      if (live) p.part_db[(long long)sp * p.M + row] = v[0];
    }
    if (kEpi == kTcFwd && p.z_out) {
      // the second half hands its partial dot products to the first half
      float *db = s.dot + (ab & 1) * 256;
      if (half == 1) {
        db[r_in] = dot;
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.dotbar[ab]);
      } else {
        if (!warp_wait(&s.dotbar[ab], ar & 1, p.err, 7)) return;
        if (live) {
          if (n_tn(p) > 1)
            p.z_out[(long long)nt * p.M + row] = dot + db[r_in];
          else
            p.z_out[row] = dot + db[r_in] + p.b_out[0];
        }
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
      // the accumulator is free again: tell the CTA whose thread issues the MMAs
      if (rank == 0)
        mbar_arrive(&s.tempty[ab]);
      else
        mbar_arrive_remote(mapa_shared(smem_u32(&s.tempty[ab]), 0));
    }
  }
  if (p.stage_out && lane == 0) bulk_wait_all();  // stores done before the CTA exits
  __syncwarp();
}

// The body of both kernels (kPair: a cluster of two CTAs, see the header).
template <bool kPair, int kEpi, int kAct, bool kFp8>
__device__ __forceinline__ void gemm_cta(const CUtensorMap *ta, const CUtensorMap *tb,
                                         const CUtensorMap *tout, const TcGemmArgs &p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  Smem s = carve(base, p);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int rank = kPair ? (int)cluster_ctarank() : 0;
  const int n_acc = 2 * acc_stride(p) <= 512 ? 2 : 1;
  uint32_t cols = 32;
  while (cols < (uint32_t)(n_acc * acc_stride(p))) cols <<= 1;

  if (threadIdx.x == 0) {
    for (int i = 0; i < p.stages; ++i) {
      // (a pair's loads all count on the even CTA's barriers)
      mbar_init(&s.full[i], 1);
      mbar_init(&s.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s.tfull[i], 1);
      // a pair's accumulator is released by the epilogue warps of both CTAs
      mbar_init(&s.tempty[i], kPair ? 2 * kEpiWarps : kEpiWarps);
    }
    mbar_init(s.drain, 1);
    for (int i = 0; i < 2; ++i) mbar_init(&s.dotbar[i], kEpiWarps / 2);
    fence_mbar_init();
  }
  if (p.with_db) {
    uint32_t *o = reinterpret_cast<uint32_t *>(s.ones);
    for (int i = threadIdx.x; i < kOnesBytes / 4; i += blockDim.x) o[i] = 0x3F803F80u;  // 1.0, 1.0
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    if (kPair)
      tmem_alloc_pair(s.tslot, cols);
    else
      tmem_alloc(s.tslot, cols);
  }
  tc_fence_before();
  __syncthreads();
  if (kPair) cluster_sync();  // both CTAs' barriers exist before either touches the other's
  tc_fence_after();
  const uint32_t tbase = *s.tslot;

  if (warp == 0) {
    if (lane == 0) producer<kPair>(ta, tb, p, s);
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) mma_issuer<kPair>(p, s, tbase);
  } else {
    epilogue<kEpi, kAct, kFp8>(p, s, tbase, tout);
  }
  tc_fence_before();
  __syncthreads();
  if (kPair) cluster_sync();  // no CTA frees TMEM or exits while its pair still signals it
  if (warp == 1) {
    tc_fence_after();
    if (kPair)
      tmem_dealloc_pair(tbase, cols);
    else
      tmem_dealloc(tbase, cols);
  }
}

template <int kEpi, int kAct, bool kFp8>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
              const __grid_constant__ CUtensorMap tout, const TcGemmArgs p) {
  gemm_cta<false, kEpi, kAct, kFp8>(&ta, &tb, &tout, p);
}

template <int kEpi, int kAct>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_tc_gemm_pair(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                   const __grid_constant__ CUtensorMap tout, const TcGemmArgs p) {
  gemm_cta<true, kEpi, kAct, false>(&ta, &tb, &tout, p);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}
}  // namespace

bool make_tmap_bf16(CUtensorMap *tm, const void *ptr, long long rows, long long cols,
                    long long ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_tmap_u8(CUtensorMap *tm, const void *ptr, long long rows, long long cols, long long ld,
                  int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld};
  cuuint32_t box[2] = {128, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(ptr), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_tmap_bf16_plain(CUtensorMap *tm, const void *ptr, long long rows, long long cols,
                          long long ld, int box_cols, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int kEpi, int kAct, bool kFp8>
static int launch_one(const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap &tout,
                      const TcGemmArgs &a, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<kEpi, kAct, kFp8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  k_tc_gemm<kEpi, kAct, kFp8><<<grid, kThreads, smem, st>>>(ta, tb, tout, a);
  return (int)cudaGetLastError();
}

// The same on clusters of two CTAs: as many clusters as can be resident at
// once (a persistent launch with clusters that would wait for others to
// finish runs a tail); if the query fails, one per SM pair (extra clusters
// then run in a later wave, which costs time but nothing else).
template <int kEpi, int kAct>
static int launch_pair(const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap &tout,
                       const TcGemmArgs &a, int num_sms, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm_pair<kEpi, kAct>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * (num_sms / 2), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  int max_clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&max_clusters, k_tc_gemm_pair<kEpi, kAct>, &cfg) !=
          cudaSuccess ||
      max_clusters < 1) {
    cudaGetLastError();
    max_clusters = num_sms / 2 > 0 ? num_sms / 2 : 1;
  }
  const int pair_tiles = (a.m_tiles + 1) / 2 * (a.n_tn > 1 ? a.n_tn : 1) * a.splits;
  const int clusters = pair_tiles < max_clusters ? pair_tiles : max_clusters;
  k_tc_gemm_pair<kEpi, kAct><<<2 * clusters, kThreads, smem, st>>>(ta, tb, tout, a);
  return (int)cudaGetLastError();
}

int launch_tc_gemm(const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap *tout,
                   TcGemmArgs a, int num_sms, cudaStream_t st) {
  if (a.stage_out && (!tout || a.epi == kTcDw || a.n_store % 32 != 0))
    return (int)cudaErrorInvalidValue;
  if (a.fp8 && (a.epi != kTcFwd || a.a_mn || a.b_mn || a.with_db))
    return (int)cudaErrorInvalidValue;
  // pair mode: BF16, an even number of 128-row M tiles; weight gradients
  // (MN-major A and B, each CTA's half of N a whole number of 64-column
  // boxes) or forward / input gradients (K-major A and B, N = 256)
  // an MN-major A sets the stage's K block for both operands
  if (a.a_mn && !a.b_mn) return (int)cudaErrorInvalidValue;
  if (a.k_per_split % tc_k_block(a) != 0) return (int)cudaErrorInvalidValue;
  if (a.pair && (a.fp8 || a.m_tiles % 2 != 0 ||
                 (a.epi == kTcDw ? (!a.a_mn || !a.b_mn || (a.N != 128 && a.N != 256))
                                 : (a.a_mn || a.b_mn || a.N != 256))))
    return (int)cudaErrorInvalidValue;
  // MN-major operands come in 64-column boxes of k_block rows x 128 bytes
  // (a pair CTA holds half of N); K-major ones in rows of 128 bytes
  const int mn_box = tc_k_block(a) * 128;
  a.a_bytes = a.a_mn ? 2 * mn_box : BM * BK * 2;
  a.b_bytes = a.b_mn ? (((a.pair ? a.N / 2 : a.N) + 63) / 64) * mn_box
                      : (a.pair ? a.N / 2 : a.N) * BK * 2;
  const int fixed = kOnesBytes + 2048 /*dot buffer*/ + 1024 /*alignment*/ + 256 /*barriers*/ +
                    (a.stage_out ? kEpiWarps * 2 * kStageBytes : 0);
  const int budget = 220 * 1024;
  int stages = (budget - fixed) / (a.a_bytes + a.b_bytes);
  a.stages = stages > 8 ? 8 : stages;
  if (a.stages < 2) return (int)cudaErrorInvalidValue;
  size_t smem = (size_t)a.stages * (a.a_bytes + a.b_bytes) + fixed;
  CUtensorMap none;
  memset(&none, 0, sizeof(none));
  const CUtensorMap &to = tout ? *tout : none;
  if (a.pair) {
    if (a.epi == kTcDw) return launch_pair<kTcDw, 0>(ta, tb, to, a, num_sms, smem, st);
    if (a.epi == kTcDx)
      return a.act ? launch_pair<kTcDx, 1>(ta, tb, to, a, num_sms, smem, st)
                   : launch_pair<kTcDx, 0>(ta, tb, to, a, num_sms, smem, st);
    return a.act ? launch_pair<kTcFwd, 1>(ta, tb, to, a, num_sms, smem, st)
                 : launch_pair<kTcFwd, 0>(ta, tb, to, a, num_sms, smem, st);
  }
  int tiles = a.m_tiles * (a.n_tn > 1 ? a.n_tn : 1) * a.splits;
  int grid = tiles < num_sms ? tiles : num_sms;
  if (a.epi == kTcDw) return launch_one<kTcDw, 0, false>(ta, tb, to, a, grid, smem, st);
  if (a.epi == kTcDx)
    return a.act ? launch_one<kTcDx, 1, false>(ta, tb, to, a, grid, smem, st)
                 : launch_one<kTcDx, 0, false>(ta, tb, to, a, grid, smem, st);
  if (a.epi != kTcFwd) return (int)cudaErrorInvalidValue;
  if (a.fp8)
    return a.act ? launch_one<kTcFwd, 1, true>(ta, tb, to, a, grid, smem, st)
                 : launch_one<kTcFwd, 0, true>(ta, tb, to, a, grid, smem, st);
  return a.act ? launch_one<kTcFwd, 1, false>(ta, tb, to, a, grid, smem, st)
               : launch_one<kTcFwd, 0, false>(ta, tb, to, a, grid, smem, st);
}

}  // namespace dinr
