// 4D export (C ABI dinr_export): the reconstruction mu0 * M on a voxel grid
// at a sequence of times, streamed to the host (Sec. V: the 4D
// reconstruction at every view time).
//
// Two device volumes and two pinned host volumes are used in turn: volume k
// is computed on the context stream while volume k-1 is copied to the host
// on a second stream and volume k-2 is handed to the caller's sink. A
// device volume is reused only after its copy has completed (event), a host
// volume only after the sink has returned, so computation, the device-to-host
// copy and the caller's consumption of the data overlap.
#include "context.cuh"

#include <vector>

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      st = (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "%s: %s (%s:%d)", #call,          \
                                  cudaGetErrorString(e_), __FILE__, __LINE__);        \
      goto done;                                                                      \
    }                                                                                 \
  } while (0)

dinr_status dinr_export(dinr_ctx *c, const double *times, int n_times, const double *lo,
                        const double *hi, const int *dims, dinr_volume_sink sink, void *user) {
  if (!c) return DINR_ERR_ARG;
  if (c->failed) return DINR_ERR_CUDA;
  if (!times || n_times < 0 || !lo || !hi || !dims || !sink || dims[0] < 1 || dims[1] < 1 ||
      dims[2] < 1)
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "invalid export request");
  const long long n = (long long)dims[0] * dims[1] * dims[2];
  const size_t bytes = sizeof(float) * (size_t)n;
  dinr_status st = DINR_OK;
  float *dvol[2] = {nullptr, nullptr}, *hvol[2] = {nullptr, nullptr};
  cudaEvent_t computed[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
  cudaStream_t copy_st = nullptr;
  int delivered = 0;
  // hands volume k (already being copied) to the sink once its copy is done
  auto deliver = [&](int k) -> dinr_status {
    const int b = k & 1;
    cudaError_t e = cudaEventSynchronize(copied[b]);
    if (e != cudaSuccess)
      return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "export copy: %s", cudaGetErrorString(e));
    if (sink(user, k, times[k], hvol[b], (int64_t)n) != 0)
      return (dinr_status)dinr_fail(c, DINR_ERR_STATE, "export stopped by the sink at volume %d",
                                    k);
    ++delivered;
    return DINR_OK;
  };
  if (n_times == 0) return DINR_OK;
  for (int b = 0; b < 2; ++b) {
    CK(cudaMalloc(&dvol[b], bytes));
    CK(cudaMallocHost(&hvol[b], bytes));
    CK(cudaEventCreateWithFlags(&computed[b], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming));
  }
  CK(cudaStreamCreateWithFlags(&copy_st, cudaStreamNonBlocking));
  for (int k = 0; k < n_times; ++k) {
    const int b = k & 1;
    // device volume b last held volume k-2: its copy must be complete
    CK(cudaStreamWaitEvent(c->st, copied[b], 0));
    st = dinr_query_grid(c, times[k], lo, hi, dims, dvol[b]);
    if (st != DINR_OK) goto done;
    CK(cudaEventRecord(computed[b], c->st));
    CK(cudaStreamWaitEvent(copy_st, computed[b], 0));
    // host volume b last held volume k-2, handed to the sink already
    CK(cudaMemcpyAsync(hvol[b], dvol[b], bytes, cudaMemcpyDeviceToHost, copy_st));
    CK(cudaEventRecord(copied[b], copy_st));
    if (k >= 1) {
      st = deliver(k - 1);
      if (st != DINR_OK) goto done;
    }
  }
  st = deliver(n_times - 1);
done:
  if (copy_st) cudaStreamSynchronize(copy_st);
  cudaStreamSynchronize(c->st);
  for (int b = 0; b < 2; ++b) {
    if (computed[b]) cudaEventDestroy(computed[b]);
    if (copied[b]) cudaEventDestroy(copied[b]);
    if (dvol[b]) cudaFree(dvol[b]);
    if (hvol[b]) cudaFreeHost(hvol[b]);
  }
  if (copy_st) cudaStreamDestroy(copy_st);
  cudaGetLastError();
  (void)delivered;
  return st;
}
