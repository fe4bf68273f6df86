// Persistent tcgen05 BF16 GEMM with the MLP's fused epilogues.
//
// D[M x N] = sum_k A(m, k) B(n, k) with BF16 operands fetched by TMA into
// 128-byte-swizzled shared memory and FP32 accumulation in TMEM.
//   A K-major: A(m, k) = A[m][k] (rows of samples), tile 128 x 64
//   A MN-major: A(m, k) = A[k][m] (e.g. delta^T for weight gradients)
//   B K-major: B(n, k) = B[n][k]; B MN-major: B(n, k) = B[k][n]
// N (the tile width) <= 256 and a multiple of 16; the output has n_tn tiles
// of N columns (column offset nt * N), M tiles of 128 rows, K in blocks of
// 64 (TMA zero-fills past the tensor's extent).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace dinr {

enum TcEpi {
  kTcFwd = 0,  // out = bf16(act(acc + bias)); optional z_out = out . w_out + b_out
               // (with n_tn > 1: z_out[nt][row] = the N-tile's part of out . w_out)
  kTcDx = 1,   // out = bf16(acc * [hprev > 0])
  kTcDw = 2    // part[split][m][n] = acc (FP32); optional part_db[split][m] = sum over k of A
};

struct TcGemmArgs {
  int epi;
  int M, N;              // output rows / columns of one N tile (MMA N)
  int n_tn;              // N tiles (0 or 1: one)
  long long K;           // reduction extent
  int a_mn, b_mn;
  int m_tiles, splits;
  long long k_per_split; // multiple of tc_k_block
  int n_store;           // columns written (<= N * n_tn)
  // kTcFwd
  const float *bias;
  __nv_bfloat16 *out;
  long long ldo;
  const float *w_out, *b_out;
  float *z_out;
  // activation of the hidden layers: 0 ReLU, 1 Swish z sigmoid(z). With
  // Swish, kTcFwd also stores the pre-activations z (BF16) in zpre, and
  // kTcDx reads pre-activations from hprev and multiplies by the Swish
  // derivative sigmoid(z) (1 + z (1 - sigmoid(z))) instead of the ReLU mask.
  int act;
  __nv_bfloat16 *zpre;
  long long ldz;
  // kTcDx
  const __nv_bfloat16 *hprev;
  long long ldh;
  // kTcDw
  float *part, *part_db;
  long long part_ld;
  int with_db;
  // FP8 forward (kTcFwd only): E4M3 A and B, K-major, K blocks of 128; the
  // accumulator is multiplied by *scale_a * *scale_b before the bias; when
  // out8 is set the activations are also written as E4M3 of x / *scale_out
  // (saturating), and the largest activation goes to *amax (float bits).
  int fp8;
  const float *scale_a, *scale_b, *scale_out;
  uint8_t *out8;
  long long ldo8;
  unsigned int *amax;
  // kTcFwd / kTcDx: write out through shared memory and TMA stores (a map
  // of out with box {32, 32}, no swizzle, passed to launch_tc_gemm), so
  // that every HBM write is a contiguous run; otherwise per-row stores.
  int stage_out;
  // launch geometry (filled by the launcher)
  int stages, a_bytes, b_bytes;
  int *err;              // device flag: nonzero when a bounded wait gave up
  // Run on clusters of two CTAs (two SMs) whose tensor cores share one
  // M = 256 MMA (tcgen05 .cta_group::2); needs BF16 and an even m_tiles, and
  // either kTcDw with MN-major A and B and N of 128 or 256, or kTcFwd / kTcDx
  // with K-major A and B and N = 256. Results are bitwise those of the
  // single-CTA kernel (the same products summed in the same order).
  int pair;
};

// K elements a pipeline stage holds. K-major operands take one 128-byte
// swizzled row per M/N row: 64 BF16 or 128 E4M3 values. MN-major operands
// (the weight gradients, K = samples; A and B both MN-major) take 128 rows
// of K per stage, which halves the stages per tile and so the barrier round
// trips between the loader and the MMA issuer. k_per_split is a multiple.
__host__ __device__ __forceinline__ int tc_k_block(const TcGemmArgs &p) {
  return p.fp8 || p.a_mn ? 128 : 64;
}

// 2D BF16 tensor map over a row-major [rows][cols] array with row stride
// ld (elements), box {64, box_rows}, 128-byte swizzle, zero fill.
bool make_tmap_bf16(CUtensorMap *tm, const void *ptr, long long rows, long long cols,
                    long long ld, int box_rows);
// The same for a byte-element (E4M3) array, box {128, box_rows}.
bool make_tmap_u8(CUtensorMap *tm, const void *ptr, long long rows, long long cols, long long ld,
                  int box_rows);

// 2D BF16 tensor map with box {box_cols, box_rows} and no swizzle.
bool make_tmap_bf16_plain(CUtensorMap *tm, const void *ptr, long long rows, long long cols,
                          long long ld, int box_cols, int box_rows);

// Launches over min(tiles, SMs) persistent CTAs (pair mode: min(tiles,
// resident two-CTA clusters) clusters). tout: the map of out for
// stage_out (else null). Returns a cudaError_t.
int launch_tc_gemm(const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap *tout,
                   TcGemmArgs a, int num_sms, cudaStream_t st);

}  // namespace dinr
