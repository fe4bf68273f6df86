// BF16 tensor-core pipeline of the training step and the queries.
//
// Per pass of rays: encode (BF16 features) -> H forward GEMMs with fused
// bias + ReLU (the last one also forms z_out = h . w_out + b_out) ->
// warp-segmented forward model + loss -> output-layer delta -> per layer
// from the last: split-K weight-gradient GEMM (bias gradient from an
// all-ones MMA in the same kernel) and the input-gradient GEMM with the ReLU
// mask fused. Master weights, gradients, segment sums and loss stay FP32.
// Widths up to 256 run the fused chains (tc_chain.cu) for the forward and
// the input gradients; wider layers run as N-tiled GEMMs, optionally with
// activation recomputation (only checkpoint layers kept, the others
// recomputed by the same forward GEMM in the backward).
#include "subpixel.cuh"
#include "tc.cuh"
#include "tc_chain.cuh"
#include "tc_gemm.cuh"

#include <cstring>
#include <vector>

using namespace dinr;

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "%s: %s (%s:%d)", #call,        \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);      \
  } while (0)
#define CKL()            \
  do {                   \
    ++c->launches;       \
    CK(cudaGetLastError()); \
  } while (0)

namespace {

constexpr int kMaxSplits = 148;

struct TcState {
  int num_sms = 148;
  std::vector<__nv_bfloat16 *> Wb, WbT;  // per hidden layer: [fan_out][kpad], [fan_in][W]
  std::vector<int> kpad;
  __nv_bfloat16 *E = nullptr, *H = nullptr, *D0 = nullptr, *D1 = nullptr;
  __nv_bfloat16 *Z = nullptr;     // Swish: pre-activations, one buffer per activation buffer
  __nv_bfloat16 *Dall = nullptr;  // [H][samples][W] deltas of every layer (chain path)
  uint32_t *masks = nullptr;      // [H][samples][W/32] ReLU bits (chain path)
  __nv_bfloat16 *G = nullptr;     // [H][samples][W] Swish derivatives (chain path)
  float *rec = nullptr;           // per-ray records [samples][8] (chain path)
  float *ones = nullptr;          // 1.0 [samples], allocated when serving starts
  bool chain = false;
  float *zpart = nullptr;         // [N tiles][samples] partial output dots (W > 256)
  // [tiles][4][W] column sums of h_{H-1} per TMEM lane quadrant (chain path,
  // see ChainArgs::hsum); hsum_used: the last training forward wrote them
  // in place of h_{H-1}
  float *hsum = nullptr;
  bool hsum_used = false;
  // FP8 forward (DINR_PREC_FP8): E4M3 copies of the features, of two
  // consecutive hidden outputs and of the weights, and per-tensor scales
  // fscale = [1 (features), s_w[H], s_h[H]] with amax records.
  bool fp8 = false;
  uint8_t *E8 = nullptr, *H8[2] = {nullptr, nullptr};
  std::vector<uint8_t *> W8;
  float *fscale = nullptr;
  unsigned int *amax_w = nullptr, *amax_h = nullptr;
  std::vector<int> owner;         // layer whose output each activation buffer holds
  float *zout = nullptr, *dz = nullptr, *ray_l = nullptr, *ray_p = nullptr, *pbar = nullptr,
        *sq = nullptr, *part = nullptr, *part_db = nullptr;
  long long part_floats = 0;
  int *err = nullptr;
};

TcState *S_(dinr_ctx *c) { return static_cast<TcState *>(c->tc); }

// ------------------------------------------------------------ small kernels

__global__ void k_to_bf16(const float *W, int rows, int cols, int kpad, __nv_bfloat16 *Wb,
                          __nv_bfloat16 *WbT) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)rows * kpad) return;
  int r = (int)(q / kpad), k = (int)(q - (long long)r * kpad);
  float x = k < cols ? W[(long long)r * cols + k] : 0.0f;
  __nv_bfloat16 b = __float2bfloat16_rn(x);
  Wb[q] = b;
  if (WbT && k < cols) WbT[(long long)k * rows + r] = b;
}

// delta_H[s][c] = dz[s] * w_out[c] * act'(.): with ReLU [h_H[s][c] > 0] from
// the activations, with Swish sigmoid(z)(1 + z(1 - sigmoid(z))) from the
// pre-activations z passed in h.
__global__ void k_out_delta_bf16(const float *dz, const float *w_out, const __nv_bfloat16 *h,
                                 int W, long long n, int swish, __nv_bfloat16 *D) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n * W) return;
  long long s = q / W;
  int col = (int)(q - s * W);
  float x = __bfloat162float(h[q]);
  float g;
  if (swish) {
    const float sg = 1.0f / (1.0f + expf(-x));
    g = sg * (1.0f + x * (1.0f - sg));
  } else {
    g = x > 0.0f ? 1.0f : 0.0f;
  }
  D[q] = __float2bfloat16_rn(dz[s] * w_out[col] * g);
}

// ---------------------------------------------------------------- FP8 (E4M3)
// Per-tensor scaling: a tensor x is stored as e4m3(x / s) with s = amax / 448
// (448 = the largest finite E4M3 value), so its largest magnitude lands on
// the top of the format's range.
constexpr float kE4M3Max = 448.0f;

__device__ __forceinline__ uint16_t e4m3x2(float lo, float hi) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
  return r;
}

// *out = max |x| (as float bits; non-negative floats order like integers).
__global__ void k_amax_abs(const float *x, long long n, unsigned int *out) {
  float m = 0.0f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[i]));
  const unsigned int b = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
  if ((threadIdx.x & 31) == 0 && b != 0u) atomicMax(out, b);
}

// Wq[r][k] = e4m3(W[r][k] / s), zero for k >= cols, s = amax / 448 (1 if 0).
__global__ void k_to_e4m3(const float *W, int rows, int cols, int kpad, const unsigned int *amax,
                          float *scale, uint8_t *Wq) {
  const float a = __uint_as_float(*amax);
  const float s = a > 0.0f ? a / kE4M3Max : 1.0f;
  long long q = 2 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  if (q == 0) *scale = s;
  if (q >= (long long)rows * kpad) return;
  int r = (int)(q / kpad), k = (int)(q - (long long)r * kpad);  // kpad is even
  float x0 = k < cols ? W[(long long)r * cols + k] / s : 0.0f;
  float x1 = k + 1 < cols ? W[(long long)r * cols + k + 1] / s : 0.0f;
  *reinterpret_cast<uint16_t *>(Wq + q) = e4m3x2(x0, x1);
}

// E4M3 copy of BF16 features (scale 1: features lie in [-1, 1]).
__global__ void k_bf16_to_e4m3(const __nv_bfloat16 *x, long long n, uint8_t *y) {
  long long q = 2 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  if (q >= n) return;
  *reinterpret_cast<uint16_t *>(y + q) =
      e4m3x2(__bfloat162float(x[q]), q + 1 < n ? __bfloat162float(x[q + 1]) : 0.0f);
}

// Delayed scaling: the activation scales of the next step from this step's
// amax records, which are then cleared.
__global__ void k_fp8_scales(unsigned int *amax_h, float *s_h, int H) {
  int L = threadIdx.x;
  if (L >= H) return;
  const float a = __uint_as_float(amax_h[L]);
  if (a > 0.0f) s_h[L] = a / kE4M3Max;
  amax_h[L] = 0u;
}

// z_out[s] = b_out + sum over N tiles of the partial dots, in tile order.
__global__ void k_sum_parts(const float *part, int n_parts, long long n, const float *b_out,
                            float *z_out) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  float z = part[s];
  for (int k = 1; k < n_parts; ++k) z += part[(long long)k * n + s];
  z_out[s] = z + b_out[0];
}

// part[z][c] = sum over rows of split z of w[s] * X[s][c] for BF16 X with C
// columns (C a multiple of 8). A block of 256 threads reads whole rows as
// 16-byte streaming loads (C/8 threads per row, 256/(C/8) rows at a time,
// eight rows in flight per thread), keeps eight column sums per thread
// (blocked summation every 256 rows) and combines the row lanes in shared
// memory.
__global__ void __launch_bounds__(256)
    k_colsum_bf16(const __nv_bfloat16 *X, int C, long long rows, const float *w, int splits,
                  float *part) {
  __shared__ float red[256][9];
  const int z = blockIdx.x;
  const int vpr = C / 8;                 // 16-byte vectors per row
  const int lanes = 256 / vpr;           // rows read at a time
  const int cv = threadIdx.x % vpr, rl = threadIdx.x / vpr;
  const long long per = (rows + splits - 1) / splits;
  const long long r0 = z * per, r1 = r0 + per < rows ? r0 + per : rows;
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0}, blk[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (rl < lanes) {
    int n = 0;
    long long r = r0 + rl;
    // eight rows per step: their loads are in flight together
    for (; r + 7 * (long long)lanes < r1; r += 8 * (long long)lanes) {
      uint4 u[8];
      float wr[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        u[k] = __ldcs(reinterpret_cast<const uint4 *>(X + (r + k * lanes) * C + 8 * cv));
        wr[k] = w[r + k * lanes];
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t v[4] = {u[k].x, u[k].y, u[k].z, u[k].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          blk[2 * e] += wr[k] * __uint_as_float(v[e] << 16);
          blk[2 * e + 1] += wr[k] * __uint_as_float(v[e] & 0xFFFF0000u);
        }
      }
      if ((n += 8) == 256) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          acc[k] += blk[k];
          blk[k] = 0.0f;
        }
        n = 0;
      }
    }
    for (; r < r1; r += lanes) {
      const uint4 u = *reinterpret_cast<const uint4 *>(X + r * C + 8 * cv);
      const float wr = w[r];
      const uint32_t v[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        blk[2 * e] += wr * __uint_as_float(v[e] << 16);
        blk[2 * e + 1] += wr * __uint_as_float(v[e] & 0xFFFF0000u);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) red[threadIdx.x][k] = acc[k] + blk[k];
  __syncthreads();
  if (threadIdx.x < vpr) {
    for (int k = 0; k < 8; ++k) {
      float s = 0.0f;
      for (int l = 0; l < lanes; ++l) s += red[l * vpr + threadIdx.x][k];
      part[(long long)z * C + 8 * threadIdx.x + k] = s;
    }
  }
}

// part[z][c] = sum over the rows r of split z of dz[128 (r / 4)] hsum[r][c]
// (r = 4 tile + quadrant): the output-layer weight gradient from the forward
// chain's column sums of h_{H-1} per tile quadrant, when dz is constant over
// every tile. One thread per column; eight rows in flight per thread.
__global__ void __launch_bounds__(256)
    k_tilesum_grad(const float *hsum, int W, long long rows, const float *dz, int splits,
                   float *part) {
  const int z = blockIdx.x, c = threadIdx.x;
  const long long per = (rows + splits - 1) / splits;
  const long long r0 = z * per, r1 = r0 + per < rows ? r0 + per : rows;
  float acc = 0.0f;
  long long r = r0;
  for (; r + 8 <= r1; r += 8) {
    float h[8], d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      h[k] = __ldcs(hsum + (r + k) * W + c);
      d[k] = dz[((r + k) >> 2) * 128];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) acc = fmaf(d[k], h[k], acc);
  }
  for (; r < r1; ++r) acc = fmaf(dz[(r >> 2) * 128], hsum[r * W + c], acc);
  part[(long long)z * W + c] = acc;
}

// Blocks of the output-layer column sum: at most one full wave (SMs x the
// blocks an SM holds), so that no partial second wave trails the sum, and
// no more than colsum_splits (the size of the partials buffer).
int colsum_bf16_splits(int num_sms, long long rows) {
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_colsum_bf16, 256, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  const long long wave = (long long)num_sms * per_sm;
  const long long cap = colsum_splits(rows);
  return (int)(cap < wave ? cap : wave);
}

int splits_for(long long rows, int m_tiles, int num_sms) {
  long long s = num_sms / m_tiles;
  long long by_rows = (rows + 4095) / 4096;  // at least 4096 samples per split
  if (s > by_rows) s = by_rows;
  if (s > kMaxSplits) s = kMaxSplits;
  return (int)(s < 1 ? 1 : s);
}

dinr_status gemm(dinr_ctx *c, const char *name, double flops, double bytes, TcGemmArgs a,
                 const void *A, long long a_rows, long long a_cols, const void *B,
                 long long b_rows, long long b_cols) {
  CUtensorMap ta, tb;
  // MN-major operands: boxes of one stage's K rows; K-major: the tile's
  // rows (a pair CTA loads half of N)
  int a_box = a.a_mn ? tc_k_block(a) : 128;
  int b_box = a.b_mn ? tc_k_block(a) : (a.pair ? a.N / 2 : a.N);
  if (!make_tmap_bf16(&ta, A, a_rows, a_cols, a_cols, a_box) ||
      !make_tmap_bf16(&tb, B, b_rows, b_cols, b_cols, b_box))
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "tensor map encoding failed (%s)", name);
  a.err = S_(c)->err;
  ProfScope ps(c, name, flops, bytes);
  // forward and input-gradient outputs go out through staged TMA stores
  CUtensorMap to;
  const bool staged = a.epi != kTcDw && a.out && a.n_store % 32 == 0 &&
                      make_tmap_bf16_plain(&to, a.out, a.M, a.n_store, a.ldo, 32, 32);
  a.stage_out = staged ? 1 : 0;
  int e = launch_tc_gemm(ta, tb, staged ? &to : nullptr, a, S_(c)->num_sms, c->st);
  ++c->launches;
  if (e != 0)
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "%s launch: %s", name,
                                  cudaGetErrorString((cudaError_t)e));
  return DINR_OK;
}

// N tiles of a W-wide output: one tile up to 256 columns, else 256-wide tiles.
int tile_w(int W) { return W <= 256 ? W : 256; }

// Forward / input-gradient GEMMs on two-SM tiles (256 rows over a CTA pair,
// each SM loading half of the weight rows): BF16, 256-column N tiles and an
// even number of 128-row M tiles.
static bool pair_ok(const TcGemmArgs &a) {
  return !a.fp8 && a.N == 256 && a.m_tiles % 2 == 0 && !a.a_mn && !a.b_mn;
}
int tiles_n(int W) { return W <= 256 ? 1 : W / 256; }

// Activation buffers of the unfused path. Without recomputation layer L has
// buffer L. With it, h_L is kept only for checkpoint layers (L % k == k - 1
// and the last layer, k = ceil(sqrt(H))); the other layers share k - 1
// segment buffers (layer L uses L % k) and are recomputed when the backward
// needs them. Consecutive layers never share a buffer.
int rc_k(const dinr_ctx *c) {
  int k = 1;
  while (k * k < c->H) ++k;
  return k;
}
bool is_ckpt(const dinr_ctx *c, int L) {
  if (!c->recompute) return true;
  const int k = rc_k(c);
  return L == c->H - 1 || L % k == k - 1;
}
int n_ckpt(const dinr_ctx *c) {
  int n = 0;
  for (int L = 0; L < c->H; ++L) n += is_ckpt(c, L);
  return n;
}
int h_slot(const dinr_ctx *c, int L) {
  if (!c->recompute) return L;
  if (is_ckpt(c, L)) {
    int n = 0;
    for (int j = 0; j < L; ++j) n += is_ckpt(c, j);
    return n;
  }
  return n_ckpt(c) + L % rc_k(c);
}
int n_hbuf(const dinr_ctx *c) { return c->recompute ? n_ckpt(c) + rc_k(c) - 1 : c->H; }

// The FP8 forward GEMM of one layer (E4M3 A [ns][acols], B [W][K]).
dinr_status gemm8(dinr_ctx *c, const char *name, double flops, double bytes, TcGemmArgs a,
                  const void *A, long long a_rows, long long a_cols, const void *B,
                  long long b_rows, long long b_cols) {
  CUtensorMap ta, tb;
  if (!make_tmap_u8(&ta, A, a_rows, a_cols, a_cols, 128) ||
      !make_tmap_u8(&tb, B, b_rows, b_cols, b_cols, a.N))
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "tensor map encoding failed (%s)", name);
  a.err = S_(c)->err;
  ProfScope ps(c, name, flops, bytes);
  // forward and input-gradient outputs go out through staged TMA stores
  CUtensorMap to;
  const bool staged = a.epi != kTcDw && a.out && a.n_store % 32 == 0 &&
                      make_tmap_bf16_plain(&to, a.out, a.M, a.n_store, a.ldo, 32, 32);
  a.stage_out = staged ? 1 : 0;
  int e = launch_tc_gemm(ta, tb, staged ? &to : nullptr, a, S_(c)->num_sms, c->st);
  ++c->launches;
  if (e != 0)
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "%s launch: %s", name,
                                  cudaGetErrorString((cudaError_t)e));
  return DINR_OK;
}

__nv_bfloat16 *hid(dinr_ctx *c, int L, long long ns) {
  return S_(c)->H + (long long)h_slot(c, L) * ns * c->W;
}
// Swish pre-activations of layer L (same buffer slots as hid).
__nv_bfloat16 *zid(dinr_ctx *c, int L, long long ns) {
  return S_(c)->Z + (long long)h_slot(c, L) * ns * c->W;
}

// Forward GEMMs of layers [L0, L1) over ns samples whose features are in E
// (the last layer also forms z_out).
dinr_status forward_layers(dinr_ctx *c, long long ns, int L0, int L1) {
  TcState *t = S_(c);
  if (t->fp8 && L0 == 0) {
    const long long n = ns * c->ldE;
    k_bf16_to_e4m3<<<ceil_div((n + 1) / 2, 256), 256, 0, c->st>>>(t->E, n, t->E8);
    CKL();
  }
  for (int L = L0; L < L1; ++L) {
    const bool last = L == c->H - 1;
    TcGemmArgs a{};
    a.epi = kTcFwd;
    a.M = (int)ns;
    a.N = tile_w(c->W);
    a.n_tn = tiles_n(c->W);
    a.K = t->kpad[L];
    a.m_tiles = (int)((ns + 127) / 128);
    a.splits = 1;
    a.k_per_split = (a.K + 63) / 64 * 64;
    a.n_store = c->W;
    a.bias = c->d_params + c->offb[L];
    a.out = hid(c, L, ns);
    a.ldo = c->W;
    if (c->act == DINR_ACT_SWISH) {
      a.act = 1;
      a.zpre = zid(c, L, ns);
      a.ldz = c->W;
    }
    if (last) {
      a.w_out = c->d_params + c->offW[c->H];
      a.b_out = c->d_params + c->offb[c->H];
      a.z_out = a.n_tn > 1 ? t->zpart : t->zout;
    }
    long long acols = L == 0 ? c->ldE : c->W;
    dinr_status s;
    if (t->fp8) {
      const float *s_w = t->fscale + 1, *s_h = t->fscale + 1 + c->H;
      a.fp8 = 1;
      a.k_per_split = (a.K + 127) / 128 * 128;
      a.scale_a = L == 0 ? t->fscale : s_h + (L - 1);
      a.scale_b = s_w + L;
      a.amax = t->amax_h + L;
      if (!last) {
        a.out8 = t->H8[L & 1];
        a.ldo8 = c->W;
        a.scale_out = s_h + L;
      }
      const void *A8 = L == 0 ? (const void *)t->E8 : (const void *)t->H8[(L - 1) & 1];
      s = gemm8(c, "tc_fwd_fp8", 2.0 * ns * c->W * c->fan_in[L],
                ns * (acols + 3.0 * c->W), a, A8, ns, acols, t->W8[L], c->W, t->kpad[L]);
    } else {
      const void *A = L == 0 ? (const void *)t->E : (const void *)hid(c, L - 1, ns);
      a.pair = pair_ok(a) ? 1 : 0;
      s = gemm(c, L0 > 0 || L1 < c->H ? "tc_fwd_recompute" : "tc_fwd",
               2.0 * ns * c->W * c->fan_in[L], 2.0 * ns * (acols + c->W), a, A, ns, acols,
               t->Wb[L], c->W, t->kpad[L]);
    }
    if (s != DINR_OK) return s;
    t->owner[h_slot(c, L)] = L;
    if (last && a.n_tn > 1) {
      k_sum_parts<<<ceil_div(ns, 256), 256, 0, c->st>>>(t->zpart, a.n_tn, ns, a.b_out, t->zout);
      CKL();
    }
  }
  return DINR_OK;
}

dinr_status forward(dinr_ctx *c, long long ns) { return forward_layers(c, ns, 0, c->H); }

// Makes h_L available: recomputes the segment from the checkpoint below it
// (or from E) when its buffer holds another layer.
dinr_status ensure_hidden(dinr_ctx *c, long long ns, int L) {
  TcState *t = S_(c);
  if (t->owner[h_slot(c, L)] == L) return DINR_OK;
  int c0 = L - 1;
  while (c0 >= 0 && !is_ckpt(c, c0)) --c0;
  return forward_layers(c, ns, c0 + 1, L + 1);
}

int chain_k0(const dinr_ctx *c) { return (c->d_in + 63) / 64 * 64; }

// Activation of the chains and the buffers carrying it to the backward:
// ReLU bits or Swish derivatives of every hidden layer.
void set_act_buffers(dinr_ctx *c, ChainArgs &a, long long ns) {
  TcState *t = S_(c);
  a.act = c->act == DINR_ACT_SWISH ? kActSwish : kActRelu;
  for (int L = 0; L < c->H; ++L) {
    if (t->masks) a.masks[L] = t->masks + (long long)L * ((ns + 127) / 128 * 128) * (c->W / 32);
    if (t->G) a.gact[L] = t->G + (long long)L * ((ns + 127) / 128 * 128) * c->W;
  }
}

// GRFF matrix of the context into the chain's parameters (C = 128 only).
void set_grff(const dinr_ctx *c, ChainArgs &a) {
  a.grff_c = c->grff_c;
  if (c->grff_c == kGrffChain) memcpy(a.grff_B, c->grff_B.data(), sizeof(a.grff_B));
}

bool chain_ok(const dinr_ctx *c) {
  if (c->prec != DINR_PREC_BF16) return false;  // the chains compute in BF16
  if (c->act != DINR_ACT_RELU && c->act != DINR_ACT_SWISH) return false;
  const bool enc = c->grff_c > 0 ? chain_supports_grff(c->grff_c) : chain_supports_freq(c->F);
  if (!(c->W % 64 == 0 && c->W <= 256 && c->H <= kChainMaxLayers && chain_k0(c) <= 256 && enc &&
        chain_stages(c->W, chain_k0(c)) >= 2))
    return false;
  // biases and output weights are read eight floats (32 bytes) at a time
  for (int L = 0; L <= c->H; ++L)
    if (c->offb[L] % 8 != 0) return false;
  return c->offW[c->H] % 8 == 0;
}

// The fused forward chain over a pass: rays of `src` (or points), encoding
// in shared memory, all hidden layers, z_out; with store_h it also writes E
// and every h_L for the backward.
dinr_status chain(dinr_ctx *c, const SourceArgs &src, long long n_rays, int S, bool store_h,
                  const float *proj) {
  TcState *t = S_(c);
  const long long ns = n_rays * S;
  ChainMaps maps;
  memset(&maps, 0, sizeof(maps));
  bool ok = true;
  for (int L = 0; L < c->H; ++L) {
    ok = ok && make_tmap_bf16(&maps.w[L], t->Wb[L], c->W, t->kpad[L], t->kpad[L], c->W);
    ok = ok && make_tmap_bf16(&maps.h[L], hid(c, L, ns), ns, c->W, c->W, 32);
  }
  ok = ok && make_tmap_bf16(&maps.e, t->E, ns, c->ldE, c->ldE, 32);
  if (!ok) return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "tensor map encoding failed (chain)");
  ChainArgs a{};
  a.g = c->geo;
  a.src = src;
  a.n_rays = n_rays;
  a.S = S;
  a.F = c->F;
  set_grff(c, a);
  a.d_in = c->d_in;
  a.k0 = chain_k0(c);
  a.W = c->W;
  a.H = c->H;
  a.ns = ns;
  a.m_tiles = (int)((ns + 127) / 128);
  a.stages = chain_stages(c->W, a.k0);
  a.store_h = store_h ? 1 : 0;
  // training rays whose samples fill whole tiles and an identity output: dz
  // is constant over each tile, so the output-layer weight gradient needs
  // only the column sums of h_{H-1} per tile
  const bool sums = store_h && t->hsum && src.kind == kSrcTrainRays && S % 128 == 0 &&
                    c->out_act == DINR_OUT_IDENTITY;
  a.hsum = sums ? t->hsum : nullptr;
  if (store_h) t->hsum_used = sums;
  for (int L = 0; L < c->H; ++L) a.bias[L] = c->d_params + c->offb[L];
  a.w_out = c->d_params + c->offW[c->H];
  a.b_out = c->d_params + c->offb[c->H];
  a.z_out = t->zout;
  a.ray_l = t->ray_l;
  a.ray_p = proj ? t->ray_p : nullptr;
  a.proj = proj;
  a.err = t->err;
  set_act_buffers(c, a, ns);
  if (src.kind == kSrcTrainRays || src.kind == kSrcVirtualView) {
    launch_ray_records(c->geo, src, n_rays, S, t->rec, t->ray_l, proj, a.ray_p, c->st);
    CKL();
    a.rays = t->rec;
  } else if (src.kind == kSrcSubRays) {  // App. A records from subpix_setup
    a.rays = src.srec32;
    a.owner = src.owner;
    a.sfirst = src.sfirst;
    a.ray_l = nullptr;
  }
  double pw = (double)c->W * c->d_in + (double)(c->H - 1) * c->W * c->W + c->W;
  ProfScope ps(c, "tc_fwd_chain", 2.0 * ns * pw,
               store_h ? 2.0 * ns * (c->ldE + (double)(sums ? c->H - 1 : c->H) * c->W) +
                             (sums ? 16.0 * a.m_tiles * c->W : 0.0)
                       : 4.0 * ns);
  int e = launch_fwd_chain(maps, a, t->num_sms, c->st);
  ++c->launches;
  if (e != 0)
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "chain launch: %s",
                                  cudaGetErrorString((cudaError_t)e));
  return DINR_OK;
}

// Backward chain over a pass: every delta_L into Dall.
dinr_status bwd_chain(dinr_ctx *c, long long ns) {
  TcState *t = S_(c);
  ChainMaps maps;
  memset(&maps, 0, sizeof(maps));
  bool ok = true;
  for (int L = 0; L < c->H; ++L) {
    if (L > 0) ok = ok && make_tmap_bf16(&maps.w[L], t->WbT[L], c->W, c->W, c->W, c->W);
    ok = ok && make_tmap_bf16(&maps.h[L], t->Dall + (long long)L * ns * c->W, ns, c->W, c->W, 32);
  }
  if (!ok) return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "tensor map encoding failed (bwd)");
  ChainArgs a{};
  a.g = c->geo;
  a.W = c->W;
  a.H = c->H;
  a.k0 = chain_k0(c);
  a.ns = ns;
  a.m_tiles = (int)((ns + 127) / 128);
  a.stages = chain_stages(c->W, a.k0);
  a.store_h = 1;
  a.w_out = c->d_params + c->offW[c->H];
  a.dz = t->dz;
  set_act_buffers(c, a, ns);
  a.err = t->err;
  ProfScope ps(c, "tc_bwd_chain", 2.0 * ns * (double)(c->H - 1) * c->W * c->W,
               2.0 * ns * c->W * c->H + ns * (c->W / 8.0) * c->H + 4.0 * ns);
  int e = launch_bwd_chain(maps, a, t->num_sms, c->st);
  ++c->launches;
  if (e != 0)
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "backward chain launch: %s",
                                  cudaGetErrorString((cudaError_t)e));
  return DINR_OK;
}

dinr_status reduce_into(dinr_ctx *c, const float *part, int splits, long long C, long long off,
                        bool acc) {
  launch_reduce_partials(part, splits, C, c->d_grad + off, acc, c->st);
  CKL();
  return DINR_OK;
}

dinr_status backward(dinr_ctx *c, long long ns, bool acc) {
  TcState *t = S_(c);
  const int W = c->W;
  __nv_bfloat16 *hH = hid(c, c->H - 1, ns);
  // output layer: delta_H, grad w_out = sum dz h_H, grad b_out = sum dz
  const bool swish = c->act == DINR_ACT_SWISH;
  if (!t->chain) {
    k_out_delta_bf16<<<ceil_div(ns * W, 256), 256, 0, c->st>>>(
        t->dz, c->d_params + c->offW[c->H], swish ? zid(c, c->H - 1, ns) : hH, W, ns, swish,
        t->D0);
    CKL();
  }
  int cs = colsum_bf16_splits(t->num_sms, ns);
  dinr_status s;
  if (t->chain && t->hsum_used) {
    // from the forward chain's column sums of h_{H-1}: dz is constant over a tile
    const long long rows = (ns + 127) / 128 * 4;
    const int ts = t->num_sms * 2;
    ProfScope ps(c, "dw_out", 2.0 * rows * W, 4.0 * rows * W + 4.0 * rows / 4);
    k_tilesum_grad<<<ts, W, 0, c->st>>>(t->hsum, W, rows, t->dz, ts, t->part);
    CKL();
    s = reduce_into(c, t->part, ts, W, c->offW[c->H], acc);
    if (s != DINR_OK) return s;
    launch_colsum(t->dz, 1, 1, ns, nullptr, false, 0, cs, t->part, c->st);
    CKL();
    s = reduce_into(c, t->part, cs, 1, c->offb[c->H], acc);
    if (s != DINR_OK) return s;
  } else {
    ProfScope ps(c, "dw_out", 2.0 * ns * W, 2.0 * ns * W + 4.0 * ns);
    k_colsum_bf16<<<cs, 256, 0, c->st>>>(hH, W, ns, t->dz, cs, t->part);
    CKL();
    s = reduce_into(c, t->part, cs, W, c->offW[c->H], acc);
    if (s != DINR_OK) return s;
    launch_colsum(t->dz, 1, 1, ns, nullptr, false, 0, cs, t->part, c->st);
    CKL();
    s = reduce_into(c, t->part, cs, 1, c->offb[c->H], acc);
    if (s != DINR_OK) return s;
  }

  if (t->chain) {
    s = bwd_chain(c, ns);
    if (s != DINR_OK) return s;
  }
  __nv_bfloat16 *D = t->chain ? t->Dall + (long long)(c->H - 1) * ns * W : t->D0;
  __nv_bfloat16 *Dn = t->D1;
  for (int L = c->H - 1; L >= 0; --L) {
    if (t->chain) D = t->Dall + (long long)L * ns * W;
    if (L > 0 && !t->chain) {
      s = ensure_hidden(c, ns, L - 1);
      if (s != DINR_OK) return s;
    }
    const void *In = L == 0 ? (const void *)t->E : (const void *)hid(c, L - 1, ns);
    int in_cols = L == 0 ? c->ldE : W;
    int fan_in = c->fan_in[L];
    TcGemmArgs a{};
    a.epi = kTcDw;
    a.M = W;
    a.N = tile_w(in_cols);
    a.n_tn = tiles_n(in_cols);
    a.K = ns;
    a.a_mn = 1;
    a.b_mn = 1;
    a.m_tiles = (W + 127) / 128;
    // two-SM tiles (256 neurons) where the layer has an even number of
    // 128-neuron tiles and its input splits into whole 64-column boxes per
    // CTA: N = 256 tiles, or one N = 128 tile for inputs of up to 128
    // columns (the layer-0 encoding; columns past in_cols read as zeros)
    if (a.m_tiles % 2 == 0 && (in_cols <= 128 || in_cols % 256 == 0)) {
      a.pair = 1;
      if (in_cols <= 128) a.N = 128;
    }
    a.splits = splits_for(ns, a.m_tiles * a.n_tn, t->num_sms);
    a.k_per_split = ((ns + a.splits - 1) / a.splits + 127) / 128 * 128;  // tc_k_block
    a.splits = (int)((ns + a.k_per_split - 1) / a.k_per_split);
    a.n_store = fan_in;
    a.part = t->part;
    a.part_ld = fan_in;
    a.part_db = t->part_db;
    a.with_db = 1;
    s = gemm(c, "tc_dw", 2.0 * ns * W * fan_in, 2.0 * ns * (W + in_cols), a, D, ns, W, In, ns,
             in_cols);
    if (s != DINR_OK) return s;
    s = reduce_into(c, t->part, a.splits, (long long)W * fan_in, c->offW[L], acc);
    if (s != DINR_OK) return s;
    s = reduce_into(c, t->part_db, a.splits, W, c->offb[L], acc);
    if (s != DINR_OK) return s;
    if (L > 0 && !t->chain) {
      TcGemmArgs b{};
      b.epi = kTcDx;
      b.M = (int)ns;
      b.N = tile_w(W);
      b.n_tn = tiles_n(W);
      b.K = W;
      b.m_tiles = (int)((ns + 127) / 128);
      b.splits = 1;
      b.k_per_split = (W + 63) / 64 * 64;
      b.n_store = W;
      b.out = Dn;
      b.ldo = W;
      b.act = swish ? 1 : 0;
      b.hprev = swish ? zid(c, L - 1, ns) : hid(c, L - 1, ns);
      b.ldh = W;
      b.pair = pair_ok(b) ? 1 : 0;
      s = gemm(c, "tc_dx", 2.0 * ns * W * W, 2.0 * ns * 3 * W, b, D, ns, W, t->WbT[L], W, W);
      if (s != DINR_OK) return s;
      __nv_bfloat16 *tmp = D;
      D = Dn;
      Dn = tmp;
    }
  }
  return DINR_OK;
}

dinr_status check_err(dinr_ctx *c) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, S_(c)->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (e) {
    CK(cudaMemsetAsync(S_(c)->err, 0, sizeof(int), c->st));
    return (dinr_status)dinr_fail(c, DINR_ERR_TIMEOUT,
                                  "a tensor-core kernel gave up waiting (code %d)", e);
  }
  return DINR_OK;
}

}  // namespace

static bool chains_used(const dinr_ctx *c);

bool tc_supported(const dinr_net *net) {
  // ReLU hidden layers; widths in [32, 256] in multiples of 32 (one N tile,
  // whole 32-column TMEM loads) or 512, 768, 1024 (256-wide N tiles); at
  // most 16 octaves (<= 144 padded inputs, one N tile of the first layer's
  // weight gradient).
  // Swish runs on the unfused GEMMs; the first layer's input width (d_in
  // padded to 16) must be one N tile (<= 256) of its weight gradient or whole
  // 256-wide tiles.
  const int W = net->width;
  const int d_in = net->encoding == DINR_ENC_GRFF ? 2 * net->grff_c : 4 + 8 * net->n_freq;
  const int ld = (d_in + 15) / 16 * 16;
  return (net->act == DINR_ACT_RELU || net->act == DINR_ACT_SWISH) && W % 32 == 0 && W >= 32 &&
         (W <= 256 || (W % 256 == 0 && W <= 1024)) && net->n_freq <= 16 &&
         (ld <= 256 || ld % 256 == 0);
}

static bool chains_used(const dinr_ctx *c) { return chain_ok(c) && c->H >= 2; }

bool tc_recompute_applies(const dinr_ctx *c) {
  return !chains_used(c) && c->prec == DINR_PREC_BF16;
}

long long tc_bytes_per_sample(const dinr_ctx *c) {
  if (chains_used(c))
    return 2LL * (c->ldE + 2LL * c->H * c->W) + 32 + 8 + 16 + c->W / 8 /*hsum*/ +
           (c->act == DINR_ACT_SWISH ? 2LL * c->H * c->W : (long long)c->H * c->W / 8);
  return 2LL * (c->ldE + (long long)(n_hbuf(c) * (c->act == DINR_ACT_SWISH ? 2 : 1) + 2) * c->W) +
         8 + 16 +
         (tiles_n(c->W) > 1 ? 4LL * tiles_n(c->W) : 0) +
         (c->prec == DINR_PREC_FP8 ? c->ldE + 2LL * c->W : 0);
}

dinr_status tc_alloc(dinr_ctx *c) {
  TcState *t = new TcState();
  c->tc = t;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, dev));
  long long ns = (long long)c->chunk_rays * c->S;
  auto grab = [&](void **p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    c->allocs.push_back(*p);
    return true;
  };
  bool ok = true;
  for (int L = 0; L < c->H; ++L) {
    int kp = L == 0 ? c->ldE : c->W;
    t->kpad.push_back(kp);
    void *wb = nullptr, *wt = nullptr;
    ok = ok && grab(&wb, sizeof(__nv_bfloat16) * (size_t)c->W * kp);
    ok = ok && grab(&wt, sizeof(__nv_bfloat16) * (size_t)c->fan_in[L] * c->W);
    t->Wb.push_back((__nv_bfloat16 *)wb);
    t->WbT.push_back((__nv_bfloat16 *)wt);
  }
  int maxN = c->ldE > c->W ? c->ldE : c->W;
  long long pf = (long long)kMaxSplits * c->W * maxN;
  long long pc = (long long)colsum_splits(ns) * c->W;
  t->part_floats = pf > pc ? pf : pc;
  t->chain = chains_used(c);
  const long long ns_tiles = (ns + 127) / 128 * 128;  // the side streams hold whole tiles
  if (t->chain)
    ok = ok && grab((void **)&t->Dall, 2ull * ns * c->W * c->H) &&
         (c->act == DINR_ACT_SWISH
              ? grab((void **)&t->G, 2ull * ns_tiles * c->W * c->H)
              : grab((void **)&t->masks, 4ull * ns_tiles * (c->W / 32) * c->H)) &&
         grab((void **)&t->rec, 32ull * ns) &&
         grab((void **)&t->hsum, 4ull * (ns_tiles / 128) * 4 * c->W);
  else
    ok = ok && grab((void **)&t->D0, 2ull * ns * c->W) && grab((void **)&t->D1, 2ull * ns * c->W);
  t->owner.assign(n_hbuf(c), -1);
  t->fp8 = c->prec == DINR_PREC_FP8;
  if (t->fp8) {
    for (int L = 0; L < c->H; ++L) {
      void *w8 = nullptr;
      ok = ok && grab(&w8, (size_t)c->W * t->kpad[L]);
      t->W8.push_back((uint8_t *)w8);
    }
    ok = ok && grab((void **)&t->E8, (size_t)ns * c->ldE) &&
         grab((void **)&t->H8[0], (size_t)ns * c->W) &&
         grab((void **)&t->H8[1], (size_t)ns * c->W) &&
         grab((void **)&t->fscale, 4ull * (1 + 2 * c->H)) &&
         grab((void **)&t->amax_w, 4ull * c->H) && grab((void **)&t->amax_h, 4ull * c->H);
    if (ok) {
      // features at scale 1; first-step activation scales 1/32 (values up to 14)
      std::vector<float> f(1 + 2 * c->H, 1.0f);
      for (int L = 0; L < c->H; ++L) f[1 + c->H + L] = 1.0f / 32.0f;
      CK(cudaMemcpyAsync(t->fscale, f.data(), 4 * f.size(), cudaMemcpyHostToDevice, c->st));
      CK(cudaMemsetAsync(t->amax_h, 0, 4ull * c->H, c->st));
      CK(cudaStreamSynchronize(c->st));
    }
  }
  if (tiles_n(c->W) > 1) ok = ok && grab((void **)&t->zpart, 4ull * ns * tiles_n(c->W));
  if (c->act == DINR_ACT_SWISH && !t->chain)
    ok = ok && grab((void **)&t->Z, 2ull * ns * c->W * n_hbuf(c));
  ok = ok && grab((void **)&t->E, 2ull * ns * c->ldE) &&
       grab((void **)&t->H, 2ull * ns * c->W * n_hbuf(c)) && grab((void **)&t->zout, 4ull * ns) &&
       grab((void **)&t->dz, 4ull * ns) && grab((void **)&t->ray_l, 4ull * ns) &&
       grab((void **)&t->ray_p, 4ull * ns) && grab((void **)&t->pbar, 4ull * ns) &&
       grab((void **)&t->sq, 4ull * ns) && grab((void **)&t->part, 4ull * t->part_floats) &&
       grab((void **)&t->part_db, 4ull * kMaxSplits * c->W) && grab((void **)&t->err, 16);
  if (!ok) return (dinr_status)dinr_fail(c, DINR_ERR_OOM, "BF16 workspace allocation failed");
  CK(cudaMemsetAsync(t->err, 0, 16, c->st));
  return tc_params_changed(c);
}

void tc_destroy(dinr_ctx *c) {
  delete S_(c);
  c->tc = nullptr;
}

dinr_status tc_params_changed(dinr_ctx *c) {
  TcState *t = S_(c);
  if (!t) return DINR_OK;
  for (int L = 0; L < c->H; ++L) {
    int rows = c->W, cols = c->fan_in[L], kp = t->kpad[L];
    k_to_bf16<<<ceil_div((long long)rows * kp, 256), 256, 0, c->st>>>(
        c->d_params + c->offW[L], rows, cols, kp, t->Wb[L], t->WbT[L]);
    CKL();
    if (t->fp8) {
      CK(cudaMemsetAsync(t->amax_w + L, 0, 4, c->st));
      k_amax_abs<<<148, 256, 0, c->st>>>(c->d_params + c->offW[L], (long long)rows * cols,
                                         t->amax_w + L);
      CKL();
      k_to_e4m3<<<ceil_div((long long)rows * kp / 2, 256), 256, 0, c->st>>>(
          c->d_params + c->offW[L], rows, cols, kp, t->amax_w + L, t->fscale + 1 + L, t->W8[L]);
      CKL();
    }
  }
  return DINR_OK;
}

// Outputs z_out of the samples of the last sub-ray setup (App. A): fused
// chain or encode + forward GEMMs.
static dinr_status subpix_outputs(dinr_ctx *c, long long ns, bool store_h) {
  TcState *t = S_(c);
  SourceArgs src = subpix_source(c);
  if (chain_ok(c)) return chain(c, src, ns, 1, store_h, nullptr);
  {
    ProfScope ps(c, "encode", 0.0, 2.0 * ns * c->ldE);
    launch_encode_bf16(c->geo, src, ns, 1, c->F, c->grff_c, c->d_grff_B, c->ldE, t->E, nullptr,
                       nullptr, nullptr, c->st);
    CKL();
  }
  return forward(c, ns);
}

dinr_status tc_loss_grad(dinr_ctx *c, int n, RunMode mode) {
  TcState *t = S_(c);
  if (mode == kGradOnly) {
    dinr_status s = backward(c, c->fwd_ns, false);
    c->fwd_kept = false;
    if (s == DINR_OK && t->fp8) {
      k_fp8_scales<<<1, 32, 0, c->st>>>(t->amax_h, t->fscale + 1 + c->H, c->H);
      CKL();
    }
    return s;
  }
  const bool one_pass = n <= c->chunk_rays;
  // a forward whose backward comes later stores its activations only when
  // they stay in the workspace (one pass); otherwise the backward recomputes
  const bool store = mode == kLossGrad || one_pass;
  float inv_B = 1.0f / (float)n;
  for (int r0 = 0, pass = 0; r0 < n; r0 += c->chunk_rays, ++pass) {
    int nr = n - r0 < c->chunk_rays ? n - r0 : c->chunk_rays;
    long long ns = (long long)nr * c->S;
    if (c->geo.D > 0) {
      dinr_status s = subpix_setup(c, c->d_idx + r0, nr, c->d_proj, &ns);
      if (s == DINR_OK) s = subpix_outputs(c, ns, store);
      if (s == DINR_OK) s = subpix_segsum(c, t->zout, nr, inv_B, true, t->pbar, t->sq, t->dz);
      if (s != DINR_OK) return s;
    } else {
      SourceArgs src{};
      src.kind = kSrcTrainRays;
      src.idx = c->d_idx + r0;
      dinr_status s;
      if (chain_ok(c)) {
        s = chain(c, src, nr, c->S, store, c->d_proj);
      } else {
        {
          ProfScope ps(c, "encode", 0.0, 2.0 * ns * c->ldE);
          launch_encode_bf16(c->geo, src, nr, c->S, c->F, c->grff_c, c->d_grff_B, c->ldE, t->E,
                             t->ray_l, c->d_proj, t->ray_p, c->st);
          CKL();
        }
        s = forward(c, ns);
      }
      if (s != DINR_OK) return s;
      launch_segsum(t->zout, c->out_act, nr, c->S, c->mu0, t->ray_l, t->ray_p, inv_B, true,
                    t->pbar, t->sq, t->dz, c->st);
      CKL();
    }
    launch_loss_sum(t->sq, nr, inv_B, c->d_loss, pass > 0, c->st);
    CKL();
    if (c->prof) c->samples_done += ns;
    if (mode == kLossOnly) {
      if (one_pass) {
        c->fwd_kept = true;
        c->fwd_ns = ns;
      }
      continue;
    }
    dinr_status s = backward(c, ns, pass > 0);
    if (s != DINR_OK) return s;
  }
  if (t->fp8 && mode == kLossGrad) {
    k_fp8_scales<<<1, 32, 0, c->st>>>(t->amax_h, t->fscale + 1 + c->H, c->H);
    CKL();
  }
  return DINR_OK;
}

static dinr_status tc_forward(dinr_ctx *c, const SourceArgs &src0, long long n_rays, int S,
                              float *out) {
  TcState *t = S_(c);
  if (src0.kind == kSrcTrainRays && c->geo.D > 0) {  // App. A model of minibatch pixels
    for (long long r0 = 0; r0 < n_rays; r0 += c->chunk_rays) {
      int nr = (int)(n_rays - r0 < c->chunk_rays ? n_rays - r0 : c->chunk_rays);
      long long ns = 0;
      dinr_status s = subpix_setup(c, src0.idx + r0, nr, nullptr, &ns);
      if (s == DINR_OK) s = subpix_outputs(c, ns, false);
      if (s == DINR_OK) s = subpix_segsum(c, t->zout, nr, 1.0f, false, out + r0, nullptr, nullptr);
      if (s != DINR_OK) return s;
    }
    return DINR_OK;
  }
  long long per = (long long)c->chunk_rays * c->S / S;
  if (per < 1) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "S larger than the workspace");
  for (long long r0 = 0; r0 < n_rays; r0 += per) {
    long long nr = n_rays - r0 < per ? n_rays - r0 : per;
    SourceArgs src = src0;
    if (src.kind == kSrcTrainRays)
      src.idx = src0.idx + r0;
    else
      src.first = src0.first + r0;
    long long ns = nr * S;
    dinr_status s;
    if (chain_ok(c)) {
      s = chain(c, src, nr, S, false, nullptr);
    } else {
      launch_encode_bf16(c->geo, src, nr, S, c->F, c->grff_c, c->d_grff_B, c->ldE, t->E,
                         t->ray_l, nullptr, nullptr, c->st);
      CKL();
      s = forward(c, ns);
    }
    if (s != DINR_OK) return s;
    launch_segsum(t->zout, c->out_act, nr, S, c->mu0, t->ray_l, nullptr, 1.0f, false, out + r0,
                  nullptr, nullptr, c->st);
    CKL();
  }
  return DINR_OK;
}

dinr_status tc_poll(dinr_ctx *c) { return S_(c) ? check_err(c) : DINR_OK; }

dinr_status tc_forward_rays(dinr_ctx *c, const SourceArgs &src, long long n_rays, int S,
                            float *out) {
  return tc_forward(c, src, n_rays, S, out);
}

dinr_status tc_forward_points(dinr_ctx *c, const SourceArgs &src, long long n, float *out) {
  return tc_forward(c, src, n, 1, out);
}

// ------------------------------------------------------------------ serving

struct ServeBackend {
  float *zout, *rec, *ray_l;
  const float *ones;
  long long capacity;
};

__global__ void k_fill(float *p, long long n, float v) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

bool tc_serve_backend(dinr_ctx *c, ServeBackend *b) {
  TcState *t = S_(c);
  if (!t || !t->chain) return false;
  long long ns = (long long)c->chunk_rays * c->S;
  if (!t->ones) {
    void *p = nullptr;
    if (cudaMalloc(&p, sizeof(float) * ns) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    c->allocs.push_back(p);
    t->ones = (float *)p;
    k_fill<<<ceil_div(ns, 256), 256, 0, c->st>>>(t->ones, ns, 1.0f);
  }
  b->zout = t->zout;
  b->rec = t->rec;
  b->ray_l = t->ray_l;
  b->ones = t->ones;
  b->capacity = ns;
  return true;
}

dinr_status tc_serve_chain(dinr_ctx *c, const WorkItem *items, const int *tile_item,
                           long long m_tiles) {
  c->fwd_kept = false;  // the batch overwrites the workspace
  TcState *t = S_(c);
  ChainMaps maps;
  memset(&maps, 0, sizeof(maps));
  bool ok = true;
  for (int L = 0; L < c->H; ++L)
    ok = ok && make_tmap_bf16(&maps.w[L], t->Wb[L], c->W, t->kpad[L], t->kpad[L], c->W);
  if (!ok) return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "tensor map encoding failed (serve)");
  ChainArgs a{};
  a.g = c->geo;
  a.F = c->F;
  set_grff(c, a);
  a.d_in = c->d_in;
  a.k0 = chain_k0(c);
  a.W = c->W;
  a.H = c->H;
  a.ns = m_tiles * 128;
  a.m_tiles = (int)m_tiles;
  a.stages = chain_stages(c->W, a.k0);
  a.store_h = 0;
  a.act = c->act == DINR_ACT_SWISH ? kActSwish : kActRelu;
  for (int L = 0; L < c->H; ++L) a.bias[L] = c->d_params + c->offb[L];
  a.w_out = c->d_params + c->offW[c->H];
  a.b_out = c->d_params + c->offb[c->H];
  a.z_out = t->zout;
  a.rays = t->rec;
  a.items = items;
  a.tile_item = tile_item;
  a.err = t->err;
  double pw = (double)c->W * c->d_in + (double)(c->H - 1) * c->W * c->W + c->W;
  ProfScope ps(c, "tc_serve_chain", 2.0 * a.ns * pw, 4.0 * a.ns);
  int e = launch_fwd_chain(maps, a, t->num_sms, c->st);
  ++c->launches;
  if (e != 0)
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "serving chain launch: %s",
                                  cudaGetErrorString((cudaError_t)e));
  return DINR_OK;
}
