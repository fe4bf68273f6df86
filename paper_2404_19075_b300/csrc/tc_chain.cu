// Fused forward and backward chains (see tc_chain.cuh).
//
// One persistent CTA per SM, 320 threads (576 in the ReLU backward):
//   warp 0      one thread streams the weight K-chunks of every layer by TMA
//               into an S-stage ring (each chunk once per tile)
//   warp 1      TMEM owner; one thread issues tcgen05.mma (M = 128, N = W,
//               K = 16) for every layer of two 128-sample tiles in turn
//   warps 2..9  two per TMEM lane quadrant (the ReLU backward: warps 2..17,
//               four per quadrant, one 64-column chunk each): build the layer-0 input of a
//               tile in shared memory (ray generation + Fourier features,
//               Sec. III, App. A, App. B), then after each layer read the
//               accumulator, add the bias, apply ReLU, write the BF16
//               activations back into the tile's shared buffer (the next
//               layer's A operand) and TMA-store them to HBM for the
//               backward; after the last layer they form
//               z_out = h . w_out + b_out.
// The two tiles ping-pong: while the epilogue warps work on one, the tensor
// cores run the other. Activations of a tile never leave the SM between
// layers. All mbarrier waits are bounded (see tc_ptx.cuh).
#include "tc_chain.cuh"
#include "tc_ptx.cuh"

namespace dinr {

using namespace tc;

namespace {

// Epilogue warps per TMEM lane quadrant ("parts"; part p owns the 64-column
// chunks jc with jc % parts == p): two, or four in the ReLU backward chain,
// whose epilogue is short enough for the 96 registers a thread of 18 warps
// gets (the forward's and the Swish epilogues need more).
template <bool kBwd, int kAct>
constexpr int parts_of() { return (kBwd && kAct == kActRelu) ? 4 : 2; }
template <bool kBwd, int kAct>
constexpr int threads_of() { return 64 + 128 * parts_of<kBwd, kAct>(); }
constexpr int kEpiWarps = 8;  // forward chains (the dot-product exchange)
constexpr int kChunkBytes = 128 * 128;  // 128 rows x 64 BF16 (one K-chunk, 128B swizzle)
constexpr int kSmemLimit = 232448;

struct Smem {
  uint8_t *A[2];      // two tile slots, K-chunks of kChunkBytes each
  uint8_t *ring;      // weight stages, W rows x 128 bytes each
  float *dot;         // [2 slots][128] partial output dot products
  uint64_t *full, *empty, *aready, *tfull, *dotbar, *drain;
  uint32_t *tslot;
};

__host__ __device__ inline int a_chunks(int W, int k0) { return (W > k0 ? W : k0) / 64; }

__device__ __forceinline__ Smem carve(uint8_t *base, const ChainArgs &p) {
  Smem s;
  const size_t a_bytes = (size_t)a_chunks(p.W, p.k0) * kChunkBytes;
  s.A[0] = base;
  s.A[1] = base + a_bytes;
  s.ring = base + 2 * a_bytes;
  s.dot = reinterpret_cast<float *>(s.ring + (size_t)p.stages * p.W * 128);
  s.full = reinterpret_cast<uint64_t *>(s.dot + 2 * 128);
  s.empty = s.full + p.stages;
  s.aready = s.empty + p.stages;
  s.tfull = s.aready + 2;
  s.dotbar = s.tfull + 2;
  s.drain = s.dotbar + 2;
  s.tslot = reinterpret_cast<uint32_t *>(s.drain + 1);
  return s;
}

// Byte offset of 16-byte unit c16 of row r in a 128B-swizzled K-chunk.
__device__ __forceinline__ uint32_t swz(int r, int c16) {
  return (uint32_t)(r * 128 + ((c16 ^ (r & 7)) << 4));
}

// TMEM store of 32 consecutive columns of this warp's 32 lanes (one value
// per lane and column), and the wait for this thread's TMEM stores.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&v);
}

// Packed FP32 add, multiply and fused multiply-add of two pairs (one
// instruction each on sm_100 and later; the compiler's builtins, so that
// the pairs stay in registers without packing moves).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// BF16 pair (lo, hi) of max(x, 0), rounded to nearest even.
__device__ __forceinline__ uint32_t pack2_relu(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// L1 policy. With nearly all of the SM's shared memory in use the L1 cache
// is small: the per-layer vectors every tile reads (biases, output weights)
// are loaded with evict_last, and the per-sample streams (ReLU bits, ray
// records) bypass L1 so that they do not evict them.
__device__ __forceinline__ float4 ld_keep(const float *p) {
  float4 v;
  asm("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}
// Eight consecutive floats (32-byte aligned) with the evict_last policy.
__device__ __forceinline__ void ld_keep8(const float *p, float4 &a, float4 &b) {
  asm("ld.global.nc.L1::evict_last.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}
__device__ __forceinline__ float4 ld_stream4(const float *p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ld_stream2(const uint32_t *p) {
  uint2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];"
               : "=r"(v.x), "=r"(v.y)
               : "l"(p));
  return v;
}
// 32-byte streaming load / store (sm_100 and later), as two 16-byte halves.
__device__ __forceinline__ void ld_stream32(const void *p, uint4 &a, uint4 &b) {
  asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z),
                 "=r"(b.w)
               : "l"(p));
}
__device__ __forceinline__ void st_stream32(void *p, uint4 a, uint4 b) {
  asm volatile("st.global.L1::no_allocate.v8.u32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p),
               "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
               : "memory");
}
// Swish derivatives of layer L in HBM, tile-interleaved so that a warp's 32
// rows of one 32-byte column unit (16 columns) are 1 KB contiguous
// (coalesced in both chains): unit (row, chunk jc, unit m) at
// (((row / 128) * (W / 64) + jc) * 4 + m) * 4096 + (row % 128) * 32.
__device__ __forceinline__ uint8_t *gact_unit(const ChainArgs &p, int L, long long row, int jc,
                                              int m) {
  return reinterpret_cast<uint8_t *>(p.gact[L]) +
         ((((row >> 7) * (p.W / 64) + jc) * 4 + m) << 12) + ((row & 127) << 5);
}
// The 64 derivatives of chunk jc of a row (zeros if not live): 16-byte
// column unit c16 in g[c16].
__device__ __forceinline__ void load_gact(const ChainArgs &p, int L, long long row, int jc,
                                          bool live, uint4 (&g)[8]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if (live)
      ld_stream32(gact_unit(p, L, row, jc, m), g[2 * m], g[2 * m + 1]);
    else
      g[2 * m] = g[2 * m + 1] = make_uint4(0, 0, 0, 0);
  }
}

// ReLU bits of layer L in HBM, tile-interleaved the same way: the two
// words of (row, 64-column chunk jc) at
// ((row / 128) * (W / 64) + jc) * 256 + (row % 128) * 2, so that a warp's 32
// rows are 256 contiguous bytes.
__device__ __forceinline__ uint32_t *mask_unit(const ChainArgs &p, int L, long long row, int jc) {
  return p.masks[L] + (((row >> 7) * (p.W / 64) + jc) << 8) + ((row & 127) << 1);
}

// lo += low BF16 half of w, hi += high half, each in FP32 with one rounding
// (the mixed-precision add of sm_100 and later; the halves are register
// halves, so no unpacking).
__device__ __forceinline__ void add_bf16x2(float &lo, float &hi, uint32_t w) {
  asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
      "add.rn.f32.bf16 %0, l, %0;\n\tadd.rn.f32.bf16 %1, h, %1;\n\t}"
      : "+f"(lo), "+f"(hi)
      : "r"(w));
}

// Low / high BF16 half of a packed pair, as FP32.
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Swish h = z sigmoid(z) and its derivative g = sigmoid(z)(1 + z(1 - sigmoid(z)))
// for a pair, in packed FP32, with sigmoid(z) = 1 / (1 + 2^(-z log2 e)) from
// the hardware exp2 and reciprocal (relative error about 2^-22 for every z;
// a tanh-based sigmoid loses relative accuracy for negative z, where
// 1/2 + tanh/2 cancels). g is formed as s + h (1 - s); h and g are returned
// as BF16 pairs, h also in FP32.
__device__ __forceinline__ void swish_pair(float2 z, float2 &h, uint32_t &wh, uint32_t &wg) {
  const float2 t = mul2(z, make_float2(-1.4426950408889634f, -1.4426950408889634f));
  float2 e, sg;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(t.x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(t.y));
  const float2 d = add2(e, make_float2(1.0f, 1.0f));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(sg.x) : "f"(d.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(sg.y) : "f"(d.y));
  h = mul2(z, sg);
  const float2 u = fma2(sg, make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));
  const float2 g = fma2(h, u, sg);
  wh = pack2(h.x, h.y);
  wg = pack2(g.x, g.y);
}

__device__ __forceinline__ void st_stream2(uint32_t *p, uint2 v) {
  asm volatile("st.global.L1::no_allocate.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(v.x), "r"(v.y)
               : "memory");
}

// ReLU bits. Of the 32 columns of a mask word, the pair (2k, 2k+1) sits at
// bits 15-k and 31-k. A packed BF16 compare against zero gives 0xFFFF in
// each half that is > 0, so one AND with the pair's two bit positions picks
// its flags with no shift.
__device__ __forceinline__ uint32_t pair_flags(uint32_t w, int k) {
  uint32_t m;
  asm("set.gt.u32.bf16x2 %0, %1, %2;" : "=r"(m) : "r"(w), "r"(0u));
  return m & (0x80008000u >> k);
}
// 0xFFFF in each half of a BF16 pair whose bit is set in mask word m (pair k).
__device__ __forceinline__ uint32_t pair_mask(uint32_t m, int k) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %1, 0xBB99;" : "=r"(d) : "r"(m << k));
  return d;
}
// The same from ms = m << (k % 8): pairs k and k + 8 share the shift, their
// bits landing at the top of bytes 1 and 3 (k < 8) or bytes 0 and 2.
__device__ __forceinline__ uint32_t pair_mask_sh(uint32_t ms, int k) {
  uint32_t d;
  if (k < 8)
    asm("prmt.b32 %0, %1, %1, 0xBB99;" : "=r"(d) : "r"(ms));
  else
    asm("prmt.b32 %0, %1, %1, 0xAA88;" : "=r"(d) : "r"(ms));
  return d;
}

// Tiles of this CTA: blockIdx.x + k * gridDim.x, processed in pairs.
__device__ __forceinline__ long long tile_of(const ChainArgs &p, int pair, int slot) {
  return (long long)blockIdx.x + (long long)(2 * pair + slot) * gridDim.x;
}
__device__ __forceinline__ int n_pairs(const ChainArgs &p) {
  int nt = (p.m_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  return (nt + 1) / 2;
}

// MMA steps of a tile: forward layers L = 0..H-1 (K = k0 for L = 0, else W);
// backward input gradients through layers L = H-1..1 (K = W).
template <bool kBwd>
__device__ __forceinline__ int n_steps(const ChainArgs &p) { return kBwd ? p.H - 1 : p.H; }
template <bool kBwd>
__device__ __forceinline__ int step_layer(const ChainArgs &p, int i) {
  return kBwd ? p.H - 1 - i : i;
}
template <bool kBwd>
__device__ __forceinline__ int step_k(const ChainArgs &p, int i) {
  return (!kBwd && i == 0) ? p.k0 : p.W;
}

// ---------------------------------------------------------------- roles

template <bool kBwd>
__device__ void producer(const ChainMaps &maps, const ChainArgs &p, const Smem &s) {
  for (int i = 0; i < n_steps<kBwd>(p); ++i) prefetch_tmap(&maps.w[step_layer<kBwd>(p, i)]);
  const uint32_t S = p.stages, tx = (uint32_t)p.W * 128;
  uint32_t it = 0;
  const int np = n_pairs(p);
  for (int pr = 0; pr < np; ++pr)
    for (int i = 0; i < n_steps<kBwd>(p); ++i)
      for (int slot = 0; slot < 2; ++slot)
        for (int kc = 0; kc < step_k<kBwd>(p, i) / 64; ++kc, ++it) {
          uint32_t st = it % S, rd = it / S;
          if (!mbar_wait(&s.empty[st], (rd & 1) ^ 1, p.err, 11)) goto drain;
          mbar_expect_tx(&s.full[st], tx);
          tma_load_2d(&maps.w[step_layer<kBwd>(p, i)], &s.full[st],
                      s.ring + (size_t)st * p.W * 128, 64 * kc, 0);
        }
drain:
  uint32_t n = it < S ? it : S;
  for (uint32_t q = it - n; q < it; ++q)
    if (!mbar_wait(&s.full[q % S], (q / S) & 1, p.err, 16)) break;
}

template <bool kBwd>
__device__ void mma_issuer(const ChainArgs &p, const Smem &s, uint32_t tbase) {
  const uint32_t S = p.stages;
  const uint32_t idesc = idesc_bf16(128, p.W, false, false);
  uint32_t it = 0, waits[2] = {0, 0};
  const int np = n_pairs(p);
  bool ok = true;
  for (int pr = 0; pr < np && ok; ++pr)
    for (int i = 0; i < n_steps<kBwd>(p) && ok; ++i)
      for (int slot = 0; slot < 2 && ok; ++slot) {
        if (!mbar_wait(&s.aready[slot], waits[slot]++ & 1, p.err, 12)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tbase + (uint32_t)(slot * p.W);
        const uint32_t a0 = smem_u32(s.A[slot]);
        const int nk = step_k<kBwd>(p, i) / 64;
        for (int kc = 0; kc < nk; ++kc, ++it) {
          uint32_t st = it % S, rd = it / S;
          if (!mbar_wait(&s.full[st], rd & 1, p.err, 13)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t b0 = smem_u32(s.ring + (size_t)st * p.W * 128);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            uint64_t ad = smem_desc(a0 + kc * kChunkBytes + 32 * k, 16, 1024, kSwizzle128);
            uint64_t bd = smem_desc(b0 + 32 * k, 16, 1024, kSwizzle128);
            // forward: the accumulator already holds the layer's bias
            mma_bf16(d, ad, bd, idesc, !kBwd || (kc | k) != 0);
          }
          mma_commit(&s.empty[st]);
        }
        if (ok) mma_commit(&s.tfull[slot]);
      }
  mma_commit(s.drain);
  mbar_wait(s.drain, 0, p.err, 14);
}

// The features of a sample with normalised coordinates c (FP32) into the
// K-chunks this warp owns, in the 128B-swizzled layout the MMA reads.
template <int F>
__device__ __forceinline__ void write_features(uint8_t *A, const float (&c)[4], bool live,
                                               int r_in, int half, const float (*B)[4]) {
  if constexpr (F == kGrffChain) {
    // GRFF (App. B item 2): frequencies 64 half .. 64 half + 63; cosines go
    // to chunk `half` (columns k), sines to chunk `half + 2` (columns C + k).
    // The phase u = B[k] . r is reduced to [-1/2, 1/2] turns, then one fast
    // sincos (absolute error about 1e-6, far below BF16 resolution).
    uint32_t wc[32], ws[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      float cv[2], sv[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float *b = B[64 * half + 2 * i + e];
        const float u = fmaf(b[0], c[0], fmaf(b[1], c[1], fmaf(b[2], c[2], b[3] * c[3])));
        __sincosf(6.28318530717958648f * (u - rintf(u)), &sv[e], &cv[e]);
      }
      wc[i] = live ? pack2(cv[0], cv[1]) : 0u;
      ws[i] = live ? pack2(sv[0], sv[1]) : 0u;
    }
    uint8_t *chc = A + (size_t)half * kChunkBytes;
    uint8_t *chs = A + (size_t)(half + 2) * kChunkBytes;
#pragma unroll
    for (int c16 = 0; c16 < 8; ++c16) {
      *reinterpret_cast<uint4 *>(chc + swz(r_in, c16)) =
          make_uint4(wc[4 * c16], wc[4 * c16 + 1], wc[4 * c16 + 2], wc[4 * c16 + 3]);
      *reinterpret_cast<uint4 *>(chs + swz(r_in, c16)) =
          make_uint4(ws[4 * c16], ws[4 * c16 + 1], ws[4 * c16 + 2], ws[4 * c16 + 3]);
    }
    return;
  }
  constexpr int kDin = 4 + 8 * F;
  constexpr int kChunks = (kDin + 63) / 64;
#pragma unroll
  for (int jc = 0; jc < kChunks; ++jc) {
    if ((jc & 1) != half) continue;
    uint32_t w[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) w[i] = 0u;
    if (jc == 0) {
      w[0] = pack2(c[0], c[1]);
      w[1] = pack2(c[2], c[3]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int lo_col = 4 + 2 * F * k;
      if (lo_col + 2 * F <= 64 * jc || lo_col >= 64 * (jc + 1)) continue;
      const float hi = c[k];
      float sp = 0.0f, cp = 1.0f, scale = 1.0f;
#pragma unroll
      for (int l = 0; l < F; ++l) {
        if ((l & 3) == 0) {
          const float x = hi * scale;
          const float y = x - 2.0f * rintf(0.5f * x);
          // the hardware sine and cosine of pi y, |y| <= 1 (absolute error
          // about 1e-6, at most about 1e-5 after three doublings; BF16
          // resolution is 4e-3 relative)
          __sincosf(3.14159265358979f * y, &sp, &cp);
        } else {
          const float s2 = 2.0f * sp * cp;
          cp = (cp - sp) * (cp + sp);
          sp = s2;
        }
        scale *= 2.0f;
        const int col = lo_col + 2 * l;
        if (col >= 64 * jc && col < 64 * (jc + 1)) w[(col - 64 * jc) / 2] = pack2(sp, cp);
      }
    }
    if (!live) {
#pragma unroll
      for (int i = 0; i < 32; ++i) w[i] = 0u;
    }
    uint8_t *chunk = A + (size_t)jc * kChunkBytes;
#pragma unroll
    for (int c16 = 0; c16 < 8; ++c16)
      *reinterpret_cast<uint4 *>(chunk + swz(r_in, c16)) =
          make_uint4(w[4 * c16], w[4 * c16 + 1], w[4 * c16 + 2], w[4 * c16 + 3]);
  }
}

// Coordinates of one training / re-projection / point sample (single source).
template <int F>
__device__ __forceinline__ void tile_features(const ChainArgs &p, uint8_t *A, long long tile,
                                              long long smp, bool live, int r_in, int q,
                                              int half, int lane) {
  const bool ray_src = p.src.kind == kSrcTrainRays || p.src.kind == kSrcVirtualView ||
                       p.src.kind == kSrcSubRays;
  // Normalised (t, z, y, x) in FP32. A ray is set up once in FP64 (chord,
  // normalised start point of its first sample and normalised step); its
  // samples are then start + j * step in FP32, whose rounding (about 1e-7)
  // moves the phase of the highest octave by under 1e-3 rad, below BF16
  // resolution of the features.
  float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (ray_src) {
    const long long s0 = live ? smp : 0;
    long long r;
    int j;
    if (p.owner) {  // App. A: ragged rays
      r = live ? p.owner[s0] : 0;
      j = (int)(s0 - p.sfirst[r]);
    } else {
      r = s0 / p.S;
      j = (int)(s0 - r * p.S);
    }
    if (live) {
      // tbar, start (z, y, x), step (z, y, x), chord length
      const float4 a = ld_stream4(p.rays + 8 * r);
      const float4 b = ld_stream4(p.rays + 8 * r + 4);
      c[0] = a.x;
      c[1] = fmaf((float)j, b.x, a.y);
      c[2] = fmaf((float)j, b.y, a.z);
      c[3] = fmaf((float)j, b.z, a.w);
    }
  } else if (live) {
    double cd[4];
    float len;
    source_coords(p.g, p.src, smp, 0, 1, cd, &len);
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = (float)cd[k];
    if (half == 0 && p.ray_l) p.ray_l[smp] = 1.0f;
  }
  write_features<F>(A, c, live, r_in, half, p.grff_B);
}


// Layer-0 input of one tile: the Fourier features of its 128 samples, in
// the K-chunks this warp owns (chunks half, half + 2, ...). F is a template
// parameter so that every feature lands in a register by static index.
// Octave features use the hardware sincos of the reduced phase at octaves
// 0, 4, 8, ... and angle doubling in between (error below about 1e-5, far
// below BF16 resolution).
template <int F>
__device__ void encode_tile(const ChainMaps &maps, const ChainArgs &p, uint8_t *A,
                            long long tile, int q, int half, int lane) {
  const int r_in = q * 32 + lane;
  long long smp = tile * 128 + r_in;
  bool live = smp < p.ns;
  if (p.items && live) {
    // serving batch: the tile's work item decides what its samples are
    const WorkItem &wi = p.items[p.tile_item[tile]];
    const long long local = (tile - wi.tile0) * 128 + r_in;
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (local < wi.n) {
      if (wi.kind == kSrcVirtualView) {
        const long long r = wi.rec0 + local / wi.S;
        const int j = (int)(local % wi.S);
        const float4 a = ld_stream4(p.rays + 8 * r);
        const float4 b = ld_stream4(p.rays + 8 * r + 4);
        c[0] = a.x;
        c[1] = fmaf((float)j, b.x, a.y);
        c[2] = fmaf((float)j, b.y, a.z);
        c[3] = fmaf((float)j, b.z, a.w);
      } else {
        double cd[4];
        float len;
        source_coords(p.g, wi.src, local, 0, 1, cd, &len);
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = (float)cd[k];
        if (half == 0 && p.ray_l) p.ray_l[smp] = 1.0f;
      }
    } else {
      live = false;
    }
    write_features<F>(A, c, live, r_in, half, p.grff_B);
  } else {
    tile_features<F>(p, A, tile, smp, live, r_in, q, half, lane);
  }
  fence_async_smem();
  __syncwarp();
  if (lane == 0 && p.store_h && tile * 128 + q * 32 < p.ns) {
    for (int jc = half; jc < (p.d_in + 63) / 64; jc += 2)
      tma_store_2d(&maps.e, A + (size_t)jc * kChunkBytes + q * 32 * 128, 64 * jc,
                   (int)(tile * 128 + q * 32));
    bulk_commit();
  }
}

// Swish part of the forward epilogue for the 32 columns c0 .. c0 + 31 whose
// pre-activations z (the accumulator started from the bias) are in r:
// h = swish(z) into the tile buffer, the derivative g into gact[L] (the
// backward's factor in place of the ReLU mask), and on the last layer the
// output dot product.
__device__ __forceinline__ void swish_group(const ChainArgs &p, uint8_t *A, int L, int c0,
                                            const uint32_t (&r)[32], int r_in, uint8_t *gbase,
                                            bool last, float &dot) {
  uint32_t wh[16], wg[16];
#pragma unroll
  for (int i4 = 0; i4 < 8; ++i4) {
    const float2 z0 = make_float2(__uint_as_float(r[4 * i4]), __uint_as_float(r[4 * i4 + 1]));
    const float2 z1 = make_float2(__uint_as_float(r[4 * i4 + 2]), __uint_as_float(r[4 * i4 + 3]));
    float2 h0, h1;
    swish_pair(z0, h0, wh[2 * i4], wg[2 * i4]);
    swish_pair(z1, h1, wh[2 * i4 + 1], wg[2 * i4 + 1]);
    if (last) {
      const float4 o = ld_keep(p.w_out + c0 + 4 * i4);
      dot = fmaf(h0.x, o.x, dot);
      dot = fmaf(h0.y, o.y, dot);
      dot = fmaf(h1.x, o.z, dot);
      dot = fmaf(h1.y, o.w, dot);
    }
  }
  const int jc = c0 >> 6, hh = (c0 >> 5) & 1;
  uint8_t *chunk = A + (size_t)jc * kChunkBytes;
#pragma unroll
  for (int u = 0; u < 4; ++u)
    *reinterpret_cast<uint4 *>(chunk + swz(r_in, 4 * hh + u)) =
        make_uint4(wh[4 * u], wh[4 * u + 1], wh[4 * u + 2], wh[4 * u + 3]);
  if (gbase) {
#pragma unroll
    for (int v = 0; v < 2; ++v)
      st_stream32(gbase + ((size_t)(jc * 4 + 2 * hh + v) << 12),
                  make_uint4(wg[8 * v], wg[8 * v + 1], wg[8 * v + 2], wg[8 * v + 3]),
                  make_uint4(wg[8 * v + 4], wg[8 * v + 5], wg[8 * v + 6], wg[8 * v + 7]));
  }
}

// Swish epilogue of layer L over this warp's 32-column groups (columns
// 64 (half + 2 m) + 32 hh). The TMEM load of the next group is in flight
// while the current one is processed.
__device__ __forceinline__ void swish_layer(const ChainArgs &p, uint8_t *A, int L,
                                            uint32_t trow, int r_in, long long row, bool live,
                                            bool last, int half, float &dot) {
  const int ng = 2 * ((p.W / 64 - half + 1) / 2);
  if (ng == 0) return;
  // gact_unit(row, 0, 0) of layer L; unit (jc, m) is 4096 (4 jc + m) further
  uint8_t *gbase = live && p.gact[L] ? gact_unit(p, L, row, 0, 0) : nullptr;
  auto col = [&](int g) { return 64 * (half + 2 * (g >> 1)) + 32 * (g & 1); };
  uint32_t ra[32], rb[32];
  tmem_ld32_issue(trow + col(0), ra);
  tmem_wait_ld32(ra);
  for (int g = 0; g < ng; g += 2) {
    tmem_ld32_issue(trow + col(g + 1), rb);
    swish_group(p, A, L, col(g), ra, r_in, gbase, last, dot);
    tmem_wait_ld32(rb);
    const bool more = g + 2 < ng;
    if (more) tmem_ld32_issue(trow + col(g + 2), ra);
    swish_group(p, A, L, col(g + 1), rb, r_in, gbase, last, dot);
    if (more) tmem_wait_ld32(ra);
  }
}

// Column sums of this warp's 32 rows of the last hidden layer (the BF16
// values it has just written to the tile buffer) over its 64-column chunks
// jc = half, half + 2, ...: lane l sums columns 64 jc + 2 l and 2 l + 1 over
// the live rows, in FP32, into hsum (see ChainArgs::hsum).
__device__ __forceinline__ void warp_column_sums(const ChainArgs &p, const uint8_t *A,
                                                 long long tile, int q, int half, int lane) {
  if (tile >= p.m_tiles) return;  // a slot with no tile (its rows are all past ns)
  const long long row0 = tile * 128 + q * 32;
  const long long left = p.ns - row0;
  const int n = left <= 0 ? 0 : (left >= 32 ? 32 : (int)left);
  for (int jc = half; jc < p.W / 64; jc += 2) {
    const uint8_t *chunk = A + (size_t)jc * kChunkBytes + (lane & 3) * 4;
    float2 acc = make_float2(0.0f, 0.0f);
    if (n == 32) {
      // all 32 rows' words in flight together, summed in four independent
      // chains per column (the sum sits on the path to the slot's next tile)
      uint32_t w[32];
#pragma unroll
      for (int i = 0; i < 32; ++i)
        w[i] = *reinterpret_cast<const uint32_t *>(chunk + swz(q * 32 + i, lane >> 2));
      float lo[4] = {0.0f, 0.0f, 0.0f, 0.0f}, hi[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int i = 0; i < 32; ++i) add_bf16x2(lo[i & 3], hi[i & 3], w[i]);
      acc = make_float2((lo[0] + lo[1]) + (lo[2] + lo[3]), (hi[0] + hi[1]) + (hi[2] + hi[3]));
    } else {
      for (int i = 0; i < n; ++i) {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(chunk + swz(q * 32 + i, lane >> 2));
        add_bf16x2(acc.x, acc.y, w);
      }
    }
    *reinterpret_cast<float2 *>(p.hsum + (tile * 4 + q) * p.W + 64 * jc + 2 * lane) = acc;
  }
}

// The bias of the next MMA into this warp's TMEM lanes and 64-column chunks
// (half, half + 2, ...) of a tile slot, whose accumulator the epilogue has
// just read: the next layer's MMAs then accumulate onto it, so the epilogue
// adds no bias.
__device__ __forceinline__ void tmem_put_bias(const float *bias, uint32_t trow, int half, int W) {
  for (int jc = half; jc < W / 64; jc += 2) {
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      uint32_t r[32];
#pragma unroll
      for (int i8 = 0; i8 < 4; ++i8) {
        float4 b0, b1;
        ld_keep8(bias + 64 * jc + 32 * hh + 8 * i8, b0, b1);
        r[8 * i8] = __float_as_uint(b0.x);
        r[8 * i8 + 1] = __float_as_uint(b0.y);
        r[8 * i8 + 2] = __float_as_uint(b0.z);
        r[8 * i8 + 3] = __float_as_uint(b0.w);
        r[8 * i8 + 4] = __float_as_uint(b1.x);
        r[8 * i8 + 5] = __float_as_uint(b1.y);
        r[8 * i8 + 6] = __float_as_uint(b1.z);
        r[8 * i8 + 7] = __float_as_uint(b1.w);
      }
      tmem_st32(trow + 64 * jc + 32 * hh, r);
    }
  }
  tmem_wait_st();
}

// After layer L of one tile: activation of the accumulator (which started
// from the bias), BF16 back into the tile buffer, ReLU bits (or the Swish
// derivative), TMA store of h_L (on the last layer with hsum set, the column
// sums instead), on the last layer the output dot product; then next_bias
// (the slot's next layer, or layer 0 of its next tile; null if none) into
// the accumulator.
template <int kAct>
__device__ bool epilogue_layer(const ChainMaps &maps, const ChainArgs &p, const Smem &s,
                               int slot, uint32_t tcol, int L, long long tile, int q, int half,
                               int lane, uint32_t dot_phase, const float *next_bias) {
  const int r_in = q * 32 + lane;
  const long long row = tile * 128 + r_in;
  const bool live = row < p.ns;
  const bool last = L == p.H - 1;
  const uint32_t trow = tcol + ((uint32_t)(q * 32) << 16);
  uint8_t *A = s.A[slot];
  float dot = 0.0f;
  if constexpr (kAct == kActSwish) swish_layer(p, A, L, trow, r_in, row, live, last, half, dot);
  for (int jc = half; kAct != kActSwish && jc < p.W / 64; jc += 2) {
    float v[64];
    tmem_ld64(trow + 64 * jc, v);
    uint32_t w[32];
#pragma unroll
    for (int i4 = 0; i4 < 16; ++i4) {
      const float2 s0 = make_float2(v[4 * i4], v[4 * i4 + 1]);
      const float2 s1 = make_float2(v[4 * i4 + 2], v[4 * i4 + 3]);
      w[2 * i4] = pack2_relu(s0.x, s0.y);
      w[2 * i4 + 1] = pack2_relu(s1.x, s1.y);
      if (last) {
        const float4 o = ld_keep(p.w_out + 64 * jc + 4 * i4);
        dot = fmaf(fmaxf(s0.x, 0.0f), o.x, dot);
        dot = fmaf(fmaxf(s0.y, 0.0f), o.y, dot);
        dot = fmaf(fmaxf(s1.x, 0.0f), o.z, dot);
        dot = fmaf(fmaxf(s1.y, 0.0f), o.w, dot);
      }
    }
    uint8_t *chunk = A + (size_t)jc * kChunkBytes;
#pragma unroll
    for (int c16 = 0; c16 < 8; ++c16)
      *reinterpret_cast<uint4 *>(chunk + swz(r_in, c16)) =
          make_uint4(w[4 * c16], w[4 * c16 + 1], w[4 * c16 + 2], w[4 * c16 + 3]);
    if (p.masks[L]) {  // bits only for a backward (not for queries)
      uint32_t bits[2] = {0u, 0u};
#pragma unroll
      for (int i = 0; i < 32; ++i) bits[i >> 4] |= pair_flags(w[i], i & 15);
      if (live) st_stream2(mask_unit(p, L, row, jc), make_uint2(bits[0], bits[1]));
    }
  }
  if (next_bias) tmem_put_bias(next_bias, trow, half, p.W);
  fence_async_smem();
  __syncwarp();
  const bool sums = last && p.hsum;
  if (lane == 0 && p.store_h && !sums && tile * 128 + q * 32 < p.ns) {
    for (int jc = half; jc < p.W / 64; jc += 2)
      tma_store_2d(&maps.h[L], A + (size_t)jc * kChunkBytes + q * 32 * 128, 64 * jc,
                   (int)(tile * 128 + q * 32));
    bulk_commit();
  }
  if (sums) warp_column_sums(p, A, tile, q, half, lane);
  if (last) {
    float *db = s.dot + slot * 128;
    if (half == 1) {
      db[r_in] = dot;
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.dotbar[slot]);
    } else {
      if (!warp_wait(&s.dotbar[slot], dot_phase & 1, p.err, 15)) return false;
      if (live) p.z_out[row] = dot + db[r_in] + p.b_out[0];
    }
  }
  return true;
}

// ------------------------------------------------------ backward chain



// Store this warp's chunks of the tile buffer through maps.h[L].
template <int kP>
__device__ __forceinline__ void store_chunks(const ChainMaps &maps, const ChainArgs &p,
                                             uint8_t *A, int L, long long tile, int q, int half,
                                             int lane) {
  fence_async_smem();
  __syncwarp();
  if (lane == 0 && p.store_h && tile * 128 + q * 32 < p.ns) {
    for (int jc = half; jc < p.W / 64; jc += kP)
      tma_store_2d(&maps.h[L], A + (size_t)jc * kChunkBytes + q * 32 * 128, 64 * jc,
                   (int)(tile * 128 + q * 32));
    bulk_commit();
  }
}

// delta_{H-1}[s][c] = dz[s] * w_out[c] * act'(.) into the tile buffer: the
// ReLU bit of h_{H-1}, or the stored Swish derivative.
template <int kAct, int kP>
__device__ void bwd_prologue(const ChainMaps &maps, const ChainArgs &p, uint8_t *A,
                             long long tile, int q, int half, int lane) {
  const int r_in = q * 32 + lane;
  const long long row = tile * 128 + r_in;
  const bool live = row < p.ns;
  const float dzr = live ? p.dz[row] : 0.0f;
  if constexpr (kAct == kActSwish) {
    for (int jc = half; jc < p.W / 64; jc += kP) {
      uint8_t *chunk = A + (size_t)jc * kChunkBytes;
      uint4 gq[8];  // the chunk's derivatives, all loads in flight together
      load_gact(p, p.H - 1, row, jc, live, gq);
#pragma unroll
      for (int c16 = 0; c16 < 8; ++c16) {
        const uint32_t gw[4] = {gq[c16].x, gq[c16].y, gq[c16].z, gq[c16].w};
        float4 oa, ob;
        ld_keep8(p.w_out + 64 * jc + 8 * c16, oa, ob);
        const float o[8] = {oa.x, oa.y, oa.z, oa.w, ob.x, ob.y, ob.z, ob.w};
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          w[e] = pack2(dzr * o[2 * e] * bf_lo(gw[e]), dzr * o[2 * e + 1] * bf_hi(gw[e]));
        *reinterpret_cast<uint4 *>(chunk + swz(r_in, c16)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    store_chunks<kP>(maps, p, A, p.H - 1, tile, q, half, lane);
    return;
  }
  for (int jc = half; jc < p.W / 64; jc += kP) {
    const uint2 mb = live ? ld_stream2(mask_unit(p, p.H - 1, row, jc)) : make_uint2(0u, 0u);
    uint8_t *chunk = A + (size_t)jc * kChunkBytes;
#pragma unroll
    for (int c16 = 0; c16 < 8; ++c16) {
      float4 oa, ob;
      ld_keep8(p.w_out + 64 * jc + 8 * c16, oa, ob);
      const float o[8] = {oa.x, oa.y, oa.z, oa.w, ob.x, ob.y, ob.z, ob.w};
      const uint32_t m = c16 < 4 ? mb.x : mb.y;
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e)
        w[e] = pack2(dzr * o[2 * e], dzr * o[2 * e + 1]) & pair_mask(m, (4 * c16 + e) & 15);
      *reinterpret_cast<uint4 *>(chunk + swz(r_in, c16)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  store_chunks<kP>(maps, p, A, p.H - 1, tile, q, half, lane);
}

// Swish: delta_{L-1} = acc * g_{L-1} with the derivative the forward stored;
// the first chunk's factors are loaded before the wait.
__device__ bool bwd_epilogue_swish(const ChainMaps &maps, const ChainArgs &p, const Smem &s,
                                   int slot, uint32_t tcol, int L, long long tile, int q, int half,
                                   int lane, uint32_t tfull_phase) {
  const int r_in = q * 32 + lane;
  const long long row = tile * 128 + r_in;
  const bool live = row < p.ns;
  uint4 gq[8];
  load_gact(p, L - 1, row, half, live && half < p.W / 64, gq);
  if (!warp_wait(&s.tfull[slot], tfull_phase & 1, p.err, 18)) return false;
  tc_fence_after();
  if (lane == 0) bulk_wait_read();
  __syncwarp();
  const uint32_t trow = tcol + ((uint32_t)(q * 32) << 16);
  uint8_t *A = s.A[slot];
  // the next chunk's derivatives are requested before this chunk is
  // processed, so their latency overlaps it
  uint4 gn[8];
  for (int jc = half; jc < p.W / 64; jc += 2) {
    const bool more = jc + 2 < p.W / 64;
    if (more) load_gact(p, L - 1, row, jc + 2, live, gn);
    float v[64];
    tmem_ld64(trow + 64 * jc, v);
    uint8_t *chunk = A + (size_t)jc * kChunkBytes;
#pragma unroll
    for (int c16 = 0; c16 < 8; ++c16) {
      const uint32_t gw[4] = {gq[c16].x, gq[c16].y, gq[c16].z, gq[c16].w};
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 8 * c16 + 2 * e;
        w[e] = pack2(v[i] * bf_lo(gw[e]), v[i + 1] * bf_hi(gw[e]));
      }
      *reinterpret_cast<uint4 *>(chunk + swz(r_in, c16)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (more) {
#pragma unroll
      for (int c16 = 0; c16 < 8; ++c16) gq[c16] = gn[c16];
    }
  }
  store_chunks<2>(maps, p, A, L - 1, tile, q, half, lane);
  return true;
}

// delta = acc * [h > 0] for the 32 columns c0 .. c0 + 31 whose accumulators
// are in r, with the group's mask word m (pair k at bits 15 - k and
// 31 - k), in BF16 into the tile buffer.
__device__ __forceinline__ void bwd_relu_group(uint8_t *A, int c0, const uint32_t (&r)[32],
                                               uint32_t m, int r_in) {
  uint32_t ms[8];  // the mask word shifted by 0..7 (pairs k and k + 8 share one)
#pragma unroll
  for (int j = 0; j < 8; ++j) ms[j] = m << j;
  uint32_t w[16];
#pragma unroll
  for (int k = 0; k < 16; ++k)
    w[k] = pack2(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1])) &
           pair_mask_sh(ms[k & 7], k);
  const int jc = c0 >> 6, hh = (c0 >> 5) & 1;
  uint8_t *chunk = A + (size_t)jc * kChunkBytes;
#pragma unroll
  for (int u = 0; u < 4; ++u)
    *reinterpret_cast<uint4 *>(chunk + swz(r_in, 4 * hh + u)) =
        make_uint4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
}

// After the input-gradient GEMM through layer L: delta_{L-1} = acc * [h_{L-1} > 0].
template <int kAct, int kP>
__device__ bool bwd_epilogue(const ChainMaps &maps, const ChainArgs &p, const Smem &s, int slot,
                             uint32_t tcol, int L, long long tile, int q, int half, int lane,
                             uint32_t tfull_phase) {
  if constexpr (kAct == kActSwish)
    return bwd_epilogue_swish(maps, p, s, slot, tcol, L, tile, q, half, lane, tfull_phase);
  const int r_in = q * 32 + lane;
  const long long row = tile * 128 + r_in;
  const bool live = row < p.ns;

  uint2 mb[2] = {make_uint2(0u, 0u), make_uint2(0u, 0u)};
  if (live)  // before the wait: the ReLU bits of this warp's (at most two) chunks
    for (int k = 0; k < 2 && half + kP * k < p.W / 64; ++k)
      mb[k] = ld_stream2(mask_unit(p, L - 1, row, half + kP * k));
  if (!warp_wait(&s.tfull[slot], tfull_phase & 1, p.err, 18)) return false;
  tc_fence_after();
  if (lane == 0) bulk_wait_read();
  __syncwarp();
  const uint32_t trow = tcol + ((uint32_t)(q * 32) << 16);
  uint8_t *A = s.A[slot];
  if constexpr (kP > 2) {
    // one chunk per warp, 32 columns at a time (the register budget of 18 warps)
    for (int k = 0, jc = half; jc < p.W / 64; ++k, jc += kP) {
      const uint2 m2 = k == 0 ? mb[0] : mb[1];
      uint32_t r[32];
      tmem_ld32_issue(trow + 64 * jc, r);
      tmem_wait_ld32(r);
      bwd_relu_group(A, 64 * jc, r, m2.x, r_in);
      tmem_ld32_issue(trow + 64 * jc + 32, r);
      tmem_wait_ld32(r);
      bwd_relu_group(A, 64 * jc + 32, r, m2.y, r_in);
    }
    store_chunks<kP>(maps, p, A, L - 1, tile, q, half, lane);
    return true;
  }
  for (int k = 0, jc = half; jc < p.W / 64; ++k, jc += 2) {
    float v[64];
    tmem_ld64(trow + 64 * jc, v);
    const uint2 m2 = k == 0 ? mb[0] : mb[1];
    uint32_t msx[8], msy[8];  // the mask words shifted by 0..7
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      msx[j] = m2.x << j;
      msy[j] = m2.y << j;
    }
    uint8_t *chunk = A + (size_t)jc * kChunkBytes;
#pragma unroll
    for (int c16 = 0; c16 < 8; ++c16) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 8 * c16 + 2 * e;
        const int pk = (4 * c16 + e) & 15;
        const uint32_t ms = c16 < 4 ? msx[pk & 7] : msy[pk & 7];
        w[e] = pack2(v[i], v[i + 1]) & pair_mask_sh(ms, pk);
      }
      *reinterpret_cast<uint4 *>(chunk + swz(r_in, c16)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  store_chunks<2>(maps, p, A, L - 1, tile, q, half, lane);
  return true;
}

// ------------------------------------------------------- epilogue warps

template <int F, bool kBwd, int kAct>
__device__ void epilogue_warps(const ChainMaps &maps, const ChainArgs &p, const Smem &s,
                               uint32_t tbase) {
  constexpr int kP = parts_of<kBwd, kAct>();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int q = warp & 3, half = (warp - 2) / 4;  // half: this warp's part (0 .. kP - 1)
  const int np = n_pairs(p);
  const int ns = n_steps<kBwd>(p);
  uint32_t waits[2] = {0, 0}, dots[2] = {0, 0};
  auto wait_stores = [&]() {
    if (lane == 0) bulk_wait_read();  // earlier stores of this warp have read the buffer
    __syncwarp();
  };
  auto start_tile = [&](int slot, long long tile) {
    if (kBwd)
      bwd_prologue<kAct, kP>(maps, p, s.A[slot], tile, q, half, lane);
    else
      encode_tile<F>(maps, p, s.A[slot], tile, q, half, lane);
  };
  if (np == 0) return;
  for (int slot = 0; slot < 2; ++slot) {
    start_tile(slot, tile_of(p, 0, slot));
    if (!kBwd) {
      // the first layer's bias into the slot's accumulator
      tmem_put_bias(p.bias[0], tbase + (uint32_t)(slot * p.W) + ((uint32_t)(q * 32) << 16), half,
                    p.W);
      tc_fence_before();
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&s.aready[slot]);
  }
  for (int pr = 0; pr < np; ++pr)
    for (int i = 0; i < ns; ++i)
      for (int slot = 0; slot < 2; ++slot) {
        const long long tile = tile_of(p, pr, slot);
        const bool last = i == ns - 1;
        const uint32_t tcol = tbase + (uint32_t)(slot * p.W);
        if (kBwd) {
          if (!bwd_epilogue<kAct, kP>(maps, p, s, slot, tcol, step_layer<true>(p, i), tile, q,
                                      half, lane, waits[slot]++))
            return;
        } else {
          if (!warp_wait(&s.tfull[slot], waits[slot]++ & 1, p.err, 17)) return;
          tc_fence_after();
          wait_stores();
          const float *nb = i + 1 < ns ? p.bias[i + 1] : (pr + 1 < np ? p.bias[0] : nullptr);
          if (!epilogue_layer<kAct>(maps, p, s, slot, tcol, i, tile, q, half, lane,
                              last ? dots[slot]++ : 0, nb))
            return;
        }
        tc_fence_before();
        if (last) {
          if (pr + 1 == np) continue;
          wait_stores();
          start_tile(slot, tile_of(p, pr + 1, slot));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.aready[slot]);
      }
}

template <int F, bool kBwd, int kAct>
__global__ void __launch_bounds__(threads_of<kBwd, kAct>(), 1)
    k_chain(const __grid_constant__ ChainMaps maps, const __grid_constant__ ChainArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  Smem s = carve(base, p);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * p.W)) cols <<= 1;
  if (threadIdx.x == 0) {
    for (int i = 0; i < p.stages; ++i) {
      mbar_init(&s.full[i], 1);
      mbar_init(&s.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s.aready[i], 4 * parts_of<kBwd, kAct>());
      mbar_init(&s.tfull[i], 1);
      mbar_init(&s.dotbar[i], kEpiWarps / 2);
    }
    mbar_init(s.drain, 1);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(s.tslot, cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *s.tslot;
  if (warp == 0) {
    if (lane == 0) producer<kBwd>(maps, p, s);
  } else if (warp == 1) {
    if (lane == 0) mma_issuer<kBwd>(p, s, tbase);
  } else {
    epilogue_warps<F, kBwd, kAct>(maps, p, s, tbase);
    if (lane == 0) bulk_wait_all();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, cols);
  }
}

}  // namespace

size_t chain_smem_bytes(int W, int k0, int stages) {
  return 2 * (size_t)a_chunks(W, k0) * kChunkBytes + (size_t)stages * W * 128 +
         2 * 128 * sizeof(float) + 256 /*barriers*/ + 1024 /*alignment*/;
}

int chain_stages(int W, int k0) {
  for (int st = 4; st >= 2; --st)
    if (chain_smem_bytes(W, k0, st) <= (size_t)kSmemLimit) return st;
  return 0;
}

bool chain_supports_freq(int F) { return F == 6 || F == 8 || F == 10 || F == 12 || F == 16; }
bool chain_supports_grff(int C) { return C == kGrffChain; }

template <int F, bool kBwd, int kAct>
static int launch_fa(const ChainMaps &maps, const ChainArgs &a, int num_sms, cudaStream_t st) {
  size_t smem = chain_smem_bytes(a.W, a.k0, a.stages);
  cudaError_t e = cudaFuncSetAttribute(k_chain<F, kBwd, kAct>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  int grid = a.m_tiles < num_sms ? a.m_tiles : num_sms;
  k_chain<F, kBwd, kAct><<<grid, threads_of<kBwd, kAct>(), smem, st>>>(maps, a);
  return (int)cudaGetLastError();
}

template <int F, bool kBwd>
static int launch_f(const ChainMaps &maps, const ChainArgs &a, int num_sms, cudaStream_t st) {
  return a.act == kActSwish ? launch_fa<F, kBwd, kActSwish>(maps, a, num_sms, st)
                            : launch_fa<F, kBwd, kActRelu>(maps, a, num_sms, st);
}

int launch_fwd_chain(const ChainMaps &maps, const ChainArgs &a, int num_sms, cudaStream_t st) {
  if (a.grff_c == kGrffChain) return launch_f<kGrffChain, false>(maps, a, num_sms, st);
  if (a.grff_c != 0) return (int)cudaErrorInvalidValue;
  switch (a.F) {
    case 6: return launch_f<6, false>(maps, a, num_sms, st);
    case 8: return launch_f<8, false>(maps, a, num_sms, st);
    case 10: return launch_f<10, false>(maps, a, num_sms, st);
    case 12: return launch_f<12, false>(maps, a, num_sms, st);
    case 16: return launch_f<16, false>(maps, a, num_sms, st);
    default: return (int)cudaErrorInvalidValue;
  }
}

__global__ void k_ray_records(GeoDev g, SourceArgs src, long long n_rays, int S, float *rec,
                              float *ray_l, const float *proj, float *ray_p) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= n_rays) return;
  const Ray ray = source_ray(g, src, r);
  const double step = ray.l / S;
  const double s = ray.s0 + 0.5 * step;
  float4 a = make_float4((float)ray.tbar, (float)((ray.oz + s * ray.dz) * g.zs + g.zb),
                         (float)((ray.oy + s * ray.dy) * g.inv_R),
                         (float)((ray.ox + s * ray.dx) * g.inv_R));
  float4 b = make_float4((float)(step * ray.dz * g.zs), (float)(step * ray.dy * g.inv_R),
                         (float)(step * ray.dx * g.inv_R), (float)ray.l);
  reinterpret_cast<float4 *>(rec + 8 * r)[0] = a;
  reinterpret_cast<float4 *>(rec + 8 * r)[1] = b;
  if (ray_l) ray_l[r] = (float)ray.l;
  if (ray_p) ray_p[r] = proj ? proj[src.idx[r]] : 0.0f;
}

void launch_ray_records(const GeoDev &g, const SourceArgs &src, long long n_rays, int S,
                        float *rec, float *ray_l, const float *proj, float *ray_p,
                        cudaStream_t st) {
  k_ray_records<<<(int)((n_rays + 127) / 128), 128, 0, st>>>(g, src, n_rays, S, rec, ray_l, proj,
                                                             ray_p);
}

int launch_bwd_chain(const ChainMaps &maps, const ChainArgs &a, int num_sms, cudaStream_t st) {
  if (a.H < 2) return (int)cudaErrorInvalidValue;
  return launch_f<0, true>(maps, a, num_sms, st);
}

}  // namespace dinr
