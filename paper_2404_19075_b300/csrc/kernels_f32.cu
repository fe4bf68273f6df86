// The plain FP32 path: a register-blocked SIMT SGEMM (no tensor cores, no
// TF32) with the MLP's epilogues. Activations live in HBM between layers.
//
// Tile 128 x 128 x 16, 256 threads, 8 x 8 outputs per thread arranged as
// two 4 x 4 blocks 64 apart in each direction. Shared memory holds two K
// slices: while one is multiplied out, the next is fetched from global
// memory into registers (16-byte loads where the layout allows) and then
// stored into the other, so there is one barrier per slice.
#include "internal.cuh"

namespace dinr {

namespace {
constexpr int BM = 128, BN = 128, BK = 16;

// The 8 elements of a 128 x 16 slice a thread fetches (2048 / 256 threads).
// KC (element (r, k) at P[r*ld + k]): row t/2, k (t%2)*8 .. +7.
// else (element (r, k) at P[k*ld + r]): k t/16, rows (t%16)*8 .. +7.
template <bool KC>
__device__ __forceinline__ void tile_pos(int t, int q, int &r, int &kk) {
  if (KC) {
    r = t >> 1;
    kk = (t & 1) * 8 + q;
  } else {
    kk = t >> 4;
    r = (t & 15) * 8 + q;
  }
}

template <bool KC>
__device__ __forceinline__ void load_tile(const float *P, long long ld, int rows_total,
                                          long long k0, long long k1, int r0, bool apply_act,
                                          int act, float (&reg)[8]) {
  int r, kk;
  tile_pos<KC>(threadIdx.x, 0, r, kk);
  const long long k = k0 + kk;
  const int rr = r0 + r;
  // the thread's 8 elements are contiguous in memory: two 16-byte loads
  // when they are all in range and the address is 16-byte aligned
  const float *src = KC ? P + (long long)rr * ld + k : P + k * ld + rr;
  const bool full = KC ? (rr < rows_total && k + 8 <= k1) : (k < k1 && rr + 8 <= rows_total);
  if (full && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const float4 v0 = reinterpret_cast<const float4 *>(src)[0];
    const float4 v1 = reinterpret_cast<const float4 *>(src)[1];
    reg[0] = v0.x; reg[1] = v0.y; reg[2] = v0.z; reg[3] = v0.w;
    reg[4] = v1.x; reg[5] = v1.y; reg[6] = v1.z; reg[7] = v1.w;
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int r2, k2;
      tile_pos<KC>(threadIdx.x, q, r2, k2);
      const long long kq = k0 + k2;
      const int rq = r0 + r2;
      reg[q] = (rq < rows_total && kq < k1) ? (KC ? P[(long long)rq * ld + kq] : P[kq * ld + rq])
                                            : 0.0f;
    }
  }
  if (apply_act) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int r2, k2;
      tile_pos<KC>(threadIdx.x, q, r2, k2);
      // only elements inside the matrix are transformed (zero fill stays 0)
      if (r0 + r2 < rows_total && k0 + k2 < k1) reg[q] = act_f(reg[q], act);
    }
  }
}

template <bool KC>
__device__ __forceinline__ void store_tile(float (*S)[BM + 4], const float (&reg)[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    int r, kk;
    tile_pos<KC>(threadIdx.x, q, r, kk);
    S[kk][r] = reg[q];
  }
}

// Blocked summation (below) in the forward and weight-gradient GEMMs; the
// input-gradient GEMMs (K = layer width) sum straight into the accumulators
// and keep two blocks per SM resident. (Without blocking in the forward as
// well, the layer-0 weight gradient of a 128-ray parallel-beam subset left
// the 1e-5 bound against the FP64 oracle: 2.3e-5 norm-wise.)
template <bool A_KC, bool B_KC, bool A_ACT, bool B_ACT, int EPI>
__global__ void __launch_bounds__(256, EPI != kEpiMask ? 1 : 2) k_sgemm(SgemmArgs a) {
  constexpr bool kBlocked = EPI != kEpiMask;
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
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
  // near kBlockK + K/kBlockK instead of K (thousands of samples for weight
  // gradients).
  constexpr int kBlockK = 32;
  float tot[8][8];  // (unused, and removed, without blocking)
  if constexpr (kBlocked) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) tot[i][j] = 0.0f;
  }

  float ra[8], rb[8];
  load_tile<A_KC>(a.A, a.lda, a.M, kb, ke, m0, A_ACT, a.act, ra);
  load_tile<B_KC>(a.B, a.ldb, a.N, kb, ke, n0, B_ACT, a.act, rb);
  store_tile<A_KC>(As[0], ra);
  store_tile<B_KC>(Bs[0], rb);
  __syncthreads();
  int buf = 0;
  for (long long k0 = kb; k0 < ke; k0 += BK) {
    const bool more = k0 + BK < ke;
    if (more) {
      load_tile<A_KC>(a.A, a.lda, a.M, k0 + BK, ke, m0, A_ACT, a.act, ra);
      load_tile<B_KC>(a.B, a.ldb, a.N, k0 + BK, ke, n0, B_ACT, a.act, rb);
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 + tx * 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if constexpr (kBlocked) {
      if (((k0 - kb) / BK + 1) % (kBlockK / BK) == 0 || !more) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            tot[i][j] += acc[i][j];
            acc[i][j] = 0.0f;
          }
      }
    }
    if (more) {
      // the other buffer was last read before the previous barrier
      store_tile<A_KC>(As[buf ^ 1], ra);
      store_tile<B_KC>(Bs[buf ^ 1], rb);
      __syncthreads();
      buf ^= 1;
    }
  }

  float *C = a.C;
  if (EPI == kEpiPartial) C += (long long)blockIdx.z * a.split_stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (m >= a.M) continue;
#pragma unroll
    for (int jh = 0; jh < 2; ++jh) {
      // four consecutive columns of the row: 16-byte loads and stores when
      // they are all inside and aligned
      const int n = n0 + jh * 64 + tx * 4;
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = kBlocked ? tot[i][4 * jh + e] : acc[i][4 * jh + e];
      float *dst = C + (long long)m * a.ldc + n;
      const float *zp = EPI == kEpiMask ? a.Zp + (long long)m * a.ldz + n : nullptr;
      const bool vec = n + 4 <= a.N && (reinterpret_cast<uintptr_t>(dst) & 15) == 0 &&
                       (EPI != kEpiMask || (reinterpret_cast<uintptr_t>(zp) & 15) == 0) &&
                       (EPI != kEpiBias || ((reinterpret_cast<uintptr_t>(a.bias + n) & 15) == 0));
      if (vec) {
        if (EPI == kEpiBias) {
          const float4 b = *reinterpret_cast<const float4 *>(a.bias + n);
          v[0] += b.x; v[1] += b.y; v[2] += b.z; v[3] += b.w;
        }
        if (EPI == kEpiMask) {
          const float4 z = *reinterpret_cast<const float4 *>(zp);
          v[0] *= act_grad_f(z.x, a.act);
          v[1] *= act_grad_f(z.y, a.act);
          v[2] *= act_grad_f(z.z, a.act);
          v[3] *= act_grad_f(z.w, a.act);
        }
        *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (n + j >= a.N) continue;
          float x = v[j];
          if (EPI == kEpiBias) x += a.bias[n + j];
          if (EPI == kEpiMask) x *= act_grad_f(zp[j], a.act);
          dst[j] = x;
        }
      }
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
