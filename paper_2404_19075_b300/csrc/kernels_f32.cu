// The plain FP32 path: a register-blocked SIMT SGEMM (no tensor cores, no
// TF32) with the MLP's epilogues. Activations live in HBM between layers.
//
// Tile 128 x 128 x 8, 256 threads, 8 x 8 outputs per thread arranged as
// two 4 x 4 blocks 64 apart in each direction; the next K slice is fetched
// into registers while the current one is multiplied out of shared memory.
#include "internal.cuh"

namespace dinr {

namespace {
constexpr int BM = 128, BN = 128, BK = 8;

// KC: element (r, k) at P[r*ld + k]; thread t owns row t/2, k (t%2)*4..+3.
// else: element (r, k) at P[k*ld + r]; thread t owns k t/32, rows (t%32)*4..+3.
template <bool KC>
__device__ __forceinline__ void tile_pos(int t, int q, int &r, int &kk) {
  if (KC) {
    r = t >> 1;
    kk = (t & 1) * 4 + q;
  } else {
    kk = t >> 5;
    r = (t & 31) * 4 + q;
  }
}

template <bool KC>
__device__ __forceinline__ void load_tile(const float *P, long long ld, int rows_total,
                                          long long k0, long long k1, int r0, bool apply_act,
                                          int act, float (&reg)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int r, kk;
    tile_pos<KC>(threadIdx.x, q, r, kk);
    long long k = k0 + kk;
    int rr = r0 + r;
    float x = 0.0f;
    if (rr < rows_total && k < k1) {
      x = KC ? P[(long long)rr * ld + k] : P[k * ld + rr];
      if (apply_act) x = act_f(x, act);
    }
    reg[q] = x;
  }
}

template <bool KC>
__device__ __forceinline__ void store_tile(float (*S)[BM + 4], const float (&reg)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int r, kk;
    tile_pos<KC>(threadIdx.x, q, r, kk);
    S[kk][r] = reg[q];
  }
}

template <bool A_KC, bool B_KC, bool A_ACT, bool B_ACT, int EPI>
__global__ void __launch_bounds__(256) k_sgemm(SgemmArgs a) {
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  long long kb = (long long)blockIdx.z * a.k_per_split;
  long long ke = kb + a.k_per_split < a.K ? kb + a.k_per_split : a.K;
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  // Blocked summation: products are accumulated in blocks of kBlockK terms
  // and each block is added into the total, which keeps the rounding growth
  // near kBlockK + K/kBlockK instead of K (K is 256 for hidden layers and
  // thousands of samples for weight gradients).
  constexpr bool kBlocked = true;
  constexpr int kBlockK = 32;
  float tot[kBlocked ? 8 : 1][kBlocked ? 8 : 1];
#pragma unroll
  for (int i = 0; i < (kBlocked ? 8 : 1); ++i)
#pragma unroll
    for (int j = 0; j < (kBlocked ? 8 : 1); ++j) tot[i][j] = 0.0f;

  float ra[4], rb[4];
  load_tile<A_KC>(a.A, a.lda, a.M, kb, ke, m0, A_ACT, a.act, ra);
  load_tile<B_KC>(a.B, a.ldb, a.N, kb, ke, n0, B_ACT, a.act, rb);
  for (long long k0 = kb; k0 < ke; k0 += BK) {
    __syncthreads();
    store_tile<A_KC>(As, ra);
    store_tile<B_KC>(Bs, rb);
    __syncthreads();
    if (k0 + BK < ke) {
      load_tile<A_KC>(a.A, a.lda, a.M, k0 + BK, ke, m0, A_ACT, a.act, ra);
      load_tile<B_KC>(a.B, a.ldb, a.N, k0 + BK, ke, n0, B_ACT, a.act, rb);
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float4 a0 = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4 *>(&As[k][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4 *>(&Bs[k][64 + tx * 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if constexpr (kBlocked) {
      if (((k0 - kb) / BK + 1) % (kBlockK / BK) == 0 || k0 + BK >= ke) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            tot[i][j] += acc[i][j];
            acc[i][j] = 0.0f;
          }
      }
    }
  }
  if constexpr (kBlocked) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = tot[i][j];
  }

  float *C = a.C;
  if (EPI == kEpiPartial) C += (long long)blockIdx.z * a.split_stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (m >= a.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (n >= a.N) continue;
      float v = acc[i][j];
      if (EPI == kEpiBias) v += a.bias[n];
      if (EPI == kEpiMask) v *= act_grad_f(a.Zp[(long long)m * a.ldz + n], a.act);
      C[(long long)m * a.ldc + n] = v;
    }
  }
}
}  // namespace

int launch_sgemm(const SgemmArgs &a, bool a_kc, bool b_kc, bool a_act, bool b_act, int epi,
                 int splits, cudaStream_t st) {
  dim3 grid(ceil_div(a.M, BM), ceil_div(a.N, BN), splits);
  dim3 block(256);
  // The combinations the MLP uses:
  //   forward:  A = inputs (k-contiguous, act on hidden inputs), B = W (k-contiguous)
  //   backward: A = delta (k-contiguous), B = W (n-contiguous), mask epilogue
  //   weights:  A = delta^T (m-contiguous), B = inputs^T (n-contiguous, act)
  if (a_kc && b_kc && !a_act && !b_act && epi == kEpiBias)
    k_sgemm<true, true, false, false, kEpiBias><<<grid, block, 0, st>>>(a);
  else if (a_kc && b_kc && a_act && !b_act && epi == kEpiBias)
    k_sgemm<true, true, true, false, kEpiBias><<<grid, block, 0, st>>>(a);
  else if (a_kc && !b_kc && !a_act && !b_act && epi == kEpiMask)
    k_sgemm<true, false, false, false, kEpiMask><<<grid, block, 0, st>>>(a);
  else if (!a_kc && !b_kc && !a_act && !b_act && epi == kEpiPartial)
    k_sgemm<false, false, false, false, kEpiPartial><<<grid, block, 0, st>>>(a);
  else if (!a_kc && !b_kc && !a_act && b_act && epi == kEpiPartial)
    k_sgemm<false, false, false, true, kEpiPartial><<<grid, block, 0, st>>>(a);
  else
    return -1;
  return 0;
}

}  // namespace dinr
