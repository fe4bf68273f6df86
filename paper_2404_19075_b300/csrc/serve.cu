// Query server of a trained network (C ABI dinr_serve_*): continuous
// batching of voxel-point, grid and re-projection queries into persistent
// forward-chain launches.
//
// Requests are admitted while their outputs fit a budget of in-flight bytes.
// Every dinr_serve_step builds one batch from the in-flight requests (whole
// 128-sample tiles, whole rays for re-projections), so a large request is
// spread over several launches and requests that arrive meanwhile join the
// next one. The order is the arrival order, or (least-work policy) the
// requests with the least work left first, so that a small request is not
// queued behind a large one; there a request passed over for kMaxSkips
// batches in a row goes first, so none waits without bound. A batch is one
// launch of the forward chain over a device work list, followed by the
// per-item forward model (segment sums of re-projection rays, mu0 * M of
// voxels). Networks the fused chain does not take (FP32 contexts, BF16
// widths above 256) run the pieces of a batch one after another through the
// single-query path instead, with the same scheduling. A request is complete
// when the event recorded after the launch holding its last work has
// completed.
#include "context.cuh"
#include "tc_chain.cuh"

#include <algorithm>
#include <cmath>
#include <deque>
#include <vector>

using namespace dinr;

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "%s: %s (%s:%d)", #call,        \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);      \
  } while (0)

// Backend hooks of the BF16 pipeline (tc_pipeline.cu).
struct ServeBackend {
  float *zout;         // per-sample outputs of a batch [capacity]
  float *rec;          // ray records [capacity][8]
  float *ray_l;        // chord lengths of the batch's re-projection rays [capacity]
  const float *ones;   // 1.0 [capacity] (forward model of voxels: l = S = 1)
  long long capacity;  // samples per batch
};
bool tc_serve_backend(dinr_ctx *c, ServeBackend *b);
dinr_status tc_serve_chain(dinr_ctx *c, const WorkItem *items_dev, const int *tile_item_dev,
                           long long m_tiles);

namespace {

struct Request {
  long long id;
  dinr_request q;
  long long samples;   // total samples of the query
  long long unit;      // samples per scheduling unit (S for rays, 1 otherwise)
  long long next = 0;  // next sample to schedule
  long long bytes;     // output bytes (admission)
  cudaEvent_t done_event = nullptr;
  int skips = 0;           // batches in a row that gave this request no work
};

constexpr int kMaxSkips = 16;

struct Server {
  long long max_batch = 0, max_inflight = 1LL << 32, inflight = 0;
  int policy = DINR_SERVE_ARRIVAL;
  bool chain = true;  // one fused-chain launch per batch, else piece by piece
  long long next_id = 1;
  std::deque<Request> active;          // not yet completely launched
  std::vector<Request> launched;       // completely launched, not yet seen done
  std::vector<long long> done_ids;     // completed (reported by poll)
  std::vector<cudaEvent_t> pool;
  WorkItem *items_dev = nullptr;
  int *tile_item_dev = nullptr;
  // pinned staging of the work list, a ring of slots: a slot is rewritten
  // only after the copy that read it has run (its event)
  static constexpr int kSlots = 4;
  WorkItem *items_host = nullptr;      // [kSlots][max_items]
  int *tile_item_host = nullptr;       // [kSlots][max_tiles]
  cudaEvent_t slot_event[kSlots] = {};
  int slot = 0;
  long long max_items = 0, max_tiles = 0;
  ServeBackend be{};
};

Server *server(dinr_ctx *c) { return static_cast<Server *>(c->serve); }

long long outputs_of(const dinr_request &q) {
  if (q.kind == DINR_QUERY_POINTS) return q.n;
  if (q.kind == DINR_QUERY_GRID) return (long long)q.dims[0] * q.dims[1] * q.dims[2];
  return (long long)q.rows * q.cols;
}

SourceArgs source_of(const dinr_ctx *c, const dinr_request &q) {
  SourceArgs s{};
  if (q.kind == DINR_QUERY_POINTS) {
    s.kind = kSrcPoints;
    s.points = q.coords_dev;
    s.t_scale = 2.0 / (c->t1 - c->t0);
    s.t_bias = -2.0 * c->t0 / (c->t1 - c->t0) - 1.0;
  } else if (q.kind == DINR_QUERY_GRID) {
    s.kind = kSrcGrid;
    for (int d = 0; d < 3; ++d) {
      s.glo[d] = q.lo[d];
      s.gstep[d] = (q.hi[d] - q.lo[d]) / q.dims[d];
      s.gdims[d] = q.dims[d];
    }
    s.gtbar = 2.0 * (q.t - c->t0) / (c->t1 - c->t0) - 1.0;
  } else {
    s.kind = kSrcVirtualView;
    s.vc = std::cos(q.theta);
    s.vs = std::sin(q.theta);
    s.vtbar = 2.0 * (q.t - c->t0) / (c->t1 - c->t0) - 1.0;
    s.vpu = c->geo.pu * c->det_cols / q.cols;
    s.vpv = c->geo.pv * c->det_rows / q.rows;
    s.vrows = q.rows;
    s.vcols = q.cols;
  }
  return s;
}

void reap(dinr_ctx *c, Server *sv) {
  for (size_t i = 0; i < sv->launched.size();) {
    Request &r = sv->launched[i];
    if (cudaEventQuery(r.done_event) == cudaSuccess) {
      sv->done_ids.push_back(r.id);
      sv->inflight -= r.bytes;
      sv->pool.push_back(r.done_event);
      sv->launched[i] = sv->launched.back();
      sv->launched.pop_back();
    } else {
      ++i;
    }
  }
  cudaGetLastError();  // cudaErrorNotReady is not an error
}

}  // namespace

dinr_status dinr_serve_config(dinr_ctx *c, int64_t max_batch_samples, int64_t max_inflight_bytes) {
  if (!c) return DINR_ERR_ARG;
  if (c->failed) return DINR_ERR_CUDA;
  Server *sv = server(c);
  if (!sv) {
    ServeBackend be{};
    const bool chain = tc_serve_backend(c, &be);
    if (!chain) be.capacity = (long long)c->chunk_rays * c->S;  // the single-query passes
    sv = new Server();
    sv->be = be;
    sv->chain = chain;
    sv->max_items = 4096;
    sv->max_tiles = be.capacity / 128 + sv->max_items;
    void *p = nullptr;
    bool ok = cudaMalloc(&p, sizeof(WorkItem) * sv->max_items) == cudaSuccess;
    sv->items_dev = (WorkItem *)p;
    ok = ok && cudaMalloc(&p, sizeof(int) * sv->max_tiles) == cudaSuccess;
    sv->tile_item_dev = (int *)p;
    ok = ok && cudaMallocHost(&p, sizeof(WorkItem) * sv->max_items * Server::kSlots) ==
                   cudaSuccess;
    sv->items_host = (WorkItem *)p;
    ok = ok && cudaMallocHost(&p, sizeof(int) * sv->max_tiles * Server::kSlots) == cudaSuccess;
    sv->tile_item_host = (int *)p;
    for (int i = 0; i < Server::kSlots; ++i)
      ok = ok && cudaEventCreateWithFlags(&sv->slot_event[i], cudaEventDisableTiming) ==
                     cudaSuccess;
    c->serve = sv;
    if (!ok) {
      cudaGetLastError();
      return (dinr_status)dinr_fail(c, DINR_ERR_OOM, "serving buffers");
    }
  }
  // whole tiles only, so that a batch never outgrows the workspace
  long long cap = sv->be.capacity / 128 * 128;
  long long mb = max_batch_samples > 0 && max_batch_samples < cap ? max_batch_samples : cap;
  sv->max_batch = mb / 128 * 128 > 0 ? mb / 128 * 128 : 128;
  if (max_inflight_bytes > 0) sv->max_inflight = max_inflight_bytes;
  return DINR_OK;
}

void dinr_serve_release(dinr_ctx *c) {
  Server *sv = c ? server(c) : nullptr;
  if (!sv) return;
  cudaStreamSynchronize(c->st);
  for (auto &r : sv->launched) cudaEventDestroy(r.done_event);
  for (auto e : sv->pool) cudaEventDestroy(e);
  for (auto e : sv->slot_event)
    if (e) cudaEventDestroy(e);
  cudaFree(sv->items_dev);
  cudaFree(sv->tile_item_dev);
  cudaFreeHost(sv->items_host);
  cudaFreeHost(sv->tile_item_host);
  delete sv;
  c->serve = nullptr;
}

dinr_status dinr_serve_policy(dinr_ctx *c, int policy) {
  if (!c) return DINR_ERR_ARG;
  if (policy != DINR_SERVE_ARRIVAL && policy != DINR_SERVE_LEAST_WORK)
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "unknown serving policy %d", policy);
  if (!server(c)) {
    dinr_status s = dinr_serve_config(c, 0, 0);
    if (s != DINR_OK) return s;
  }
  server(c)->policy = policy;
  return DINR_OK;
}

dinr_status dinr_serve_submit(dinr_ctx *c, const dinr_request *q, int64_t *id) {
  if (!c || !q || !id) return DINR_ERR_ARG;
  if (c->failed) return DINR_ERR_CUDA;
  if (!server(c)) {
    dinr_status s = dinr_serve_config(c, 0, 0);
    if (s != DINR_OK) return s;
  }
  Server *sv = server(c);
  const dinr_request &r = *q;
  bool ok = r.out_dev != nullptr;
  if (r.kind == DINR_QUERY_POINTS) ok = ok && r.coords_dev && r.n > 0;
  else if (r.kind == DINR_QUERY_GRID) ok = ok && r.dims[0] > 0 && r.dims[1] > 0 && r.dims[2] > 0;
  else if (r.kind == DINR_QUERY_PROJECT)
    ok = ok && r.rows > 0 && r.cols > 0 && r.S > 0 && r.S <= 4096 && r.S <= sv->max_batch;
  else ok = false;
  if (!ok) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "invalid request");
  reap(c, sv);
  Request rq;
  rq.q = r;
  rq.unit = r.kind == DINR_QUERY_PROJECT ? r.S : 1;
  rq.samples = outputs_of(r) * rq.unit;
  rq.bytes = 4 * outputs_of(r);
  if (sv->inflight + rq.bytes > sv->max_inflight)
    return (dinr_status)dinr_fail(c, DINR_ERR_BUSY, "in-flight budget full; retry later");
  rq.id = sv->next_id++;
  sv->inflight += rq.bytes;
  sv->active.push_back(rq);
  *id = rq.id;
  return DINR_OK;
}

dinr_status dinr_serve_step(dinr_ctx *c, int *in_flight) {
  if (!c) return DINR_ERR_ARG;
  if (c->failed) return DINR_ERR_CUDA;
  Server *sv = server(c);
  if (!sv) return (dinr_status)dinr_fail(c, DINR_ERR_STATE, "no request submitted");
  reap(c, sv);
  if (!sv->active.empty()) {
    // one batch: whole tiles, whole rays; in arrival order, or requests
    // passed over kMaxSkips times first (in arrival order), then least
    // remaining work first
    const size_t na = sv->active.size();
    std::vector<size_t> ord(na);
    for (size_t k = 0; k < na; ++k) ord[k] = k;
    if (sv->policy == DINR_SERVE_LEAST_WORK)
      std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) {
        const Request &ra = sv->active[a], &rb = sv->active[b];
        const bool sa = ra.skips >= kMaxSkips, sb = rb.skips >= kMaxSkips;
        if (sa != sb) return sa;
        return !sa && ra.samples - ra.next < rb.samples - rb.next;
      });
    long long tiles = 0, rec = 0;
    int n_items = 0;
    std::vector<size_t> finished, item_req;
    std::vector<long long> first_unit(na);
    std::vector<char> served(na, 0);
    // the staging slot's previous copy must have run before it is rewritten
    const int slot = sv->slot;
    sv->slot = (slot + 1) % Server::kSlots;
    CK(cudaEventSynchronize(sv->slot_event[slot]));
    WorkItem *items_host = sv->items_host + (size_t)slot * sv->max_items;
    int *tile_item_host = sv->tile_item_host + (size_t)slot * sv->max_tiles;
    for (size_t j = 0; j < na && n_items < sv->max_items; ++j) {
      const size_t k = ord[j];
      Request &r = sv->active[k];
      long long room = sv->max_batch - tiles * 128;
      long long units = (r.samples - r.next) / r.unit;
      long long fit = room / r.unit;
      if (room <= 0) break;
      if (fit <= 0) continue;  // a whole ray does not fit; smaller units may
      if (units > fit) units = fit;
      long long n = units * r.unit;
      WorkItem &w = items_host[n_items];
      w = WorkItem{};
      w.kind = r.q.kind == DINR_QUERY_PROJECT ? kSrcVirtualView : source_of(c, r.q).kind;
      w.S = (int)r.unit;
      w.tile0 = tiles;
      w.n = n;
      w.rec0 = rec;
      w.src = source_of(c, r.q);
      w.src.first = r.next / r.unit;  // first ray / point of this piece
      long long nt = (n + 127) / 128;
      for (long long t = 0; t < nt; ++t) tile_item_host[tiles + t] = n_items;
      first_unit[k] = r.next / r.unit;
      tiles += nt;
      if (w.kind == kSrcVirtualView) rec += units;
      r.next += n;
      ++n_items;
      item_req.push_back(k);
      served[k] = 1;
      if (r.next >= r.samples) finished.push_back(k);
    }
    for (size_t k = 0; k < na; ++k) sv->active[k].skips = served[k] ? 0 : sv->active[k].skips + 1;
    if (n_items > 0) {
      if (!sv->chain) {
        // piece by piece through the single-query path (bitwise the same
        // results as the single queries)
        for (int i = 0; i < n_items; ++i) {
          const WorkItem &w = items_host[i];
          const size_t k = item_req[i];
          float *out = sv->active[k].q.out_dev + first_unit[k];
          dinr_status s = w.kind == kSrcVirtualView
                              ? run_forward_rays(c, w.src, w.n / w.S, w.S, out)
                              : run_forward_points(c, w.src, w.n, out);
          if (s != DINR_OK) return s;
        }
      } else {
        CK(cudaMemcpyAsync(sv->items_dev, items_host, sizeof(WorkItem) * n_items,
                           cudaMemcpyHostToDevice, c->st));
        CK(cudaMemcpyAsync(sv->tile_item_dev, tile_item_host, sizeof(int) * tiles,
                           cudaMemcpyHostToDevice, c->st));
        CK(cudaEventRecord(sv->slot_event[slot], c->st));
        // ray records of the re-projection pieces
        for (int i = 0; i < n_items; ++i) {
          const WorkItem &w = items_host[i];
          if (w.kind != kSrcVirtualView) continue;
          launch_ray_records(c->geo, w.src, w.n / w.S, w.S, sv->be.rec + 8 * w.rec0,
                             sv->be.ray_l + w.rec0, nullptr, nullptr, c->st);
          ++c->launches;
        }
        dinr_status s = tc_serve_chain(c, sv->items_dev, sv->tile_item_dev, tiles);
        if (s != DINR_OK) return s;
        // forward model of each piece into the request's output
        for (int i = 0; i < n_items; ++i) {
          const WorkItem &w = items_host[i];
          const size_t k = item_req[i];
          Request &r = sv->active[k];
          const float *z = sv->be.zout + w.tile0 * 128;
          if (w.kind == kSrcVirtualView) {
            launch_segsum(z, c->out_act, w.n / w.S, w.S, c->mu0, sv->be.ray_l + w.rec0, nullptr,
                          1.0f, false, r.q.out_dev + first_unit[k], nullptr, nullptr, c->st);
          } else {
            launch_segsum(z, c->out_act, w.n, 1, c->mu0, sv->be.ones, nullptr, 1.0f, false,
                          r.q.out_dev + first_unit[k], nullptr, nullptr, c->st);
          }
          ++c->launches;
        }
        CK(cudaGetLastError());
      }
      // completely launched requests leave the active list, highest position
      // first; each owns one event recorded after this batch
      std::sort(finished.begin(), finished.end());
      for (size_t f = finished.size(); f-- > 0;) {
        cudaEvent_t ev;
        if (!sv->pool.empty()) {
          ev = sv->pool.back();
          sv->pool.pop_back();
        } else {
          CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        }
        CK(cudaEventRecord(ev, c->st));
        Request r = sv->active[finished[f]];
        r.done_event = ev;
        sv->launched.push_back(r);
        sv->active.erase(sv->active.begin() + (long)finished[f]);
      }
    }
  }
  if (in_flight) *in_flight = (int)(sv->active.size() + sv->launched.size());
  return DINR_OK;
}

dinr_status dinr_serve_poll(dinr_ctx *c, int64_t id, int *done) {
  if (!c || !done) return DINR_ERR_ARG;
  if (c->failed) return DINR_ERR_CUDA;
  Server *sv = server(c);
  if (!sv) return (dinr_status)dinr_fail(c, DINR_ERR_STATE, "no request submitted");
  reap(c, sv);
  *done = 0;
  for (size_t i = 0; i < sv->done_ids.size(); ++i)
    if (sv->done_ids[i] == id) {
      *done = 1;
      sv->done_ids[i] = sv->done_ids.back();
      sv->done_ids.pop_back();
      return DINR_OK;
    }
  for (auto &r : sv->active)
    if (r.id == id) return DINR_OK;
  for (auto &r : sv->launched)
    if (r.id == id) return DINR_OK;
  return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "unknown request id %lld", (long long)id);
}
