// server.cu -- continuous-batching request loop over the iontrap C ABI (host code).
//
// A request is one trap simulation (species, initial state, parameters, step budget).
// Requests wait in arrival order until a slot and enough of the device-memory budget are
// free; admitted requests stay resident on the device until their last step.  Every
// scheduling round (iontrap_server_poll):
//   1. requests whose enqueued chunk has finished (CUDA event) advance their count; a
//      request at its budget is retired: its final state is copied out and its device
//      memory returned to the budget;
//   2. waiting requests are admitted, first come first served, while they fit; a handle
//      is created on the server's own admission stream (so admission never waits for a
//      chunk in flight) and then moved to the stream it is stepped on, and its device
//      buffers come from the library's stream-ordered pool (no device-wide
//      synchronisation at admission or retirement);
//   3. the next chunks: requests the batched kernel accepts (FP32 form, N <= 2048) go
//      into one iontrap_step_many per size class (up to 64, 256, 512, 1024 and 2048
//      ions), each class on a stream of its own -- smaller classes at higher stream
//      priority -- so that a small request's chunk does not wait for a large one's; the
//      others share max_parallel streams, each idle one taking the request with the least
//      remaining pair work (N^2 x steps left: shortest remaining work first, preempting at
//      chunk boundaries), in chunks of at most chunk_steps x (4096 / N)^2 steps, so that
//      every chunk is short and no stream queues a large one ahead of the others.
// A request's trajectory does not depend on what else is resident: batched requests are
// bitwise independent of the mix, the others run one chunk at a time on one stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "iontrap.h"

namespace it {
int use_nonpersistent_default(iontrap_t* h);       // iontrap_api.cu
int rebind_stream(iontrap_t* h, cudaStream_t st);  // iontrap_api.cu
}

namespace {

struct Event {
  cudaEvent_t ev = nullptr;
  Event() { cudaEventCreateWithFlags(&ev, cudaEventDisableTiming); }
  ~Event() {
    if (ev) cudaEventDestroy(ev);
  }
};

struct Request {
  int64_t id = 0;
  int64_t n = 0;
  std::vector<iontrap_species> species;
  std::vector<uint8_t> soi;
  std::vector<double> x0, v0;
  bool has_v0 = false;
  iontrap_params p{};
  int64_t steps = 0, done = 0, inflight = 0;
  iontrap_t* h = nullptr;
  int solo = -1;  // the shared stream its chunk in flight runs on (requests stepped alone)
  bool batched = false;
  int lane = 0;  // batched size class
  int64_t bytes = 0;
  int status = IONTRAP_OK;
  std::vector<double> xo, vo;
  int64_t final_step = 0;
};

// Device bytes a request will hold before its handle exists (for admission).
int64_t estimate_bytes(int64_t n, int precision) {
  int64_t b = 0;
  if (iontrap_estimate_bytes(n, precision, &b) != IONTRAP_OK) b = n * (3 * 3 * 8 + 1 + 2 * 32 + 32 * 64) + 4096;
  return b;
}

}  // namespace

// Batched size classes: the largest ensemble of each (ions).
constexpr int kLanes = 5;
constexpr int64_t kLaneMax[kLanes] = {64, 256, 512, 1024, 2048};

struct Lane {
  cudaStream_t stream = nullptr;
  std::shared_ptr<Event> ev;  // the class's batch in flight
  bool inflight = false;
};

// Chunks of a request stepped alone: at most chunk_steps x (kSoloChunkIons / N)^2 steps.
constexpr int64_t kSoloChunkIons = 4096;

struct iontrap_server {
  iontrap_server_config cfg{};
  Lane lanes[kLanes];
  std::vector<Lane> solo;        // the shared streams of the requests stepped alone
  cudaStream_t admit = nullptr;  // where handles are created
  std::deque<std::unique_ptr<Request>> waiting;
  std::vector<std::unique_ptr<Request>> resident;
  std::map<int64_t, std::unique_ptr<Request>> completed;
  int64_t next_id = 1;
  int64_t bytes_in_use = 0;
  int64_t completed_total = 0;
};

static void retire(iontrap_server* s, std::unique_ptr<Request>& r) {
  r->xo.resize(3 * r->n);
  r->vo.resize(3 * r->n);
  int64_t step = 0;
  const int st = iontrap_state(r->h, r->xo.data(), r->vo.data(), &step, nullptr);
  r->final_step = step;
  if (st && !r->status) r->status = st;
  iontrap_destroy(r->h);
  r->h = nullptr;
  s->bytes_in_use -= r->bytes;
  r->x0.clear();
  r->v0.clear();
  r->x0.shrink_to_fit();
  r->v0.shrink_to_fit();
  ++s->completed_total;
}

extern "C" {

int iontrap_server_create(const iontrap_server_config* cfg, iontrap_server_t** out) {
  if (!out) return IONTRAP_EINVAL;
  *out = nullptr;
  iontrap_server* s = new (std::nothrow) iontrap_server();
  if (!s) return IONTRAP_ENOMEM;
  if (cfg) s->cfg = *cfg;
  if (s->cfg.mem_budget_bytes <= 0) s->cfg.mem_budget_bytes = (int64_t)2 << 30;
  if (s->cfg.max_resident <= 0) s->cfg.max_resident = 4096;
  if (s->cfg.chunk_steps <= 0) s->cfg.chunk_steps = 100;
  if (s->cfg.max_parallel <= 0) s->cfg.max_parallel = 3;
  // stream priorities: the smallest class highest (lower numbers are higher priorities),
  // the requests stepped alone lowest
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
  bool ok = cudaStreamCreateWithFlags(&s->admit, cudaStreamNonBlocking) == cudaSuccess;
  for (int c = 0; c < kLanes && ok; ++c)
    ok = cudaStreamCreateWithPriority(&s->lanes[c].stream, cudaStreamNonBlocking, std::min(least, greatest + c)) ==
         cudaSuccess;
  s->solo.resize((size_t)s->cfg.max_parallel);
  for (Lane& l : s->solo)
    if (ok) ok = cudaStreamCreateWithPriority(&l.stream, cudaStreamNonBlocking, least) == cudaSuccess;
  if (!ok) {
    iontrap_server_destroy(s);
    return IONTRAP_ECUDA;
  }
  *out = s;
  return IONTRAP_OK;
}

int iontrap_server_submit(iontrap_server_t* s, const iontrap_species* species, int n_species,
                          const uint8_t* species_of_ion, const double* x0, const double* v0, int64_t n,
                          const iontrap_params* p, int64_t n_steps, int64_t* id) {
  if (!s || !species || n_species < 1 || n_species > IONTRAP_MAX_SPECIES || !species_of_ion || !x0 || !p ||
      n < 1 || n_steps < 0 || !id)
    return IONTRAP_EINVAL;
  auto r = std::make_unique<Request>();
  r->id = s->next_id++;
  r->n = n;
  r->species.assign(species, species + n_species);
  r->soi.assign(species_of_ion, species_of_ion + n);
  r->x0.assign(x0, x0 + 3 * n);
  if (v0) {
    r->v0.assign(v0, v0 + 3 * n);
    r->has_v0 = true;
  }
  r->p = *p;
  r->steps = n_steps;
  r->batched = p->precision == IONTRAP_PREC_FP32 && n <= kLaneMax[kLanes - 1];
  while (r->lane + 1 < kLanes && n > kLaneMax[r->lane]) ++r->lane;
  r->bytes = estimate_bytes(n, p->precision);
  *id = r->id;
  s->waiting.push_back(std::move(r));
  return IONTRAP_OK;
}

int iontrap_server_poll(iontrap_server_t* s, int64_t* completed_ids, int64_t cap, int64_t* n_completed) {
  if (!s || !n_completed || (cap > 0 && !completed_ids)) return IONTRAP_EINVAL;
  *n_completed = 0;
  auto report = [&](int64_t rid) {
    if (*n_completed < cap) completed_ids[*n_completed] = rid;
    ++*n_completed;
  };
  // 1. finished chunks
  for (Lane& l : s->lanes)
    if (l.inflight && cudaEventQuery(l.ev->ev) == cudaSuccess) l.inflight = false;
  for (Lane& l : s->solo)
    if (l.inflight && cudaEventQuery(l.ev->ev) == cudaSuccess) l.inflight = false;
  for (size_t k = 0; k < s->resident.size();) {
    auto& r = s->resident[k];
    if (r->inflight) {
      const bool fin = r->batched ? !s->lanes[r->lane].inflight : !s->solo[r->solo].inflight;
      if (fin) {
        r->done += r->inflight;
        r->inflight = 0;
        r->solo = -1;
      }
    }
    if (!r->inflight && (r->done >= r->steps || r->status)) {
      const int64_t rid = r->id;
      retire(s, r);
      report(rid);
      s->completed[rid] = std::move(r);
      s->resident.erase(s->resident.begin() + k);
      continue;
    }
    ++k;
  }
  // 2. admission, first come first served
  // (a request larger than the whole budget is admitted when nothing else is resident)
  while (!s->waiting.empty() && (int64_t)s->resident.size() < s->cfg.max_resident &&
         (s->bytes_in_use + s->waiting.front()->bytes <= s->cfg.mem_budget_bytes || s->resident.empty())) {
    auto r = std::move(s->waiting.front());
    s->waiting.pop_front();
    r->status = iontrap_create(r->species.data(), (int)r->species.size(), r->soi.data(), r->x0.data(),
                               r->has_v0 ? r->v0.data() : nullptr, r->n, &r->p, 0, (void*)s->admit, &r->h);
    if (!r->status && !r->batched) r->status = it::use_nonpersistent_default(r->h);
    // the batched ones live on their class's stream; the others move at each chunk
    if (!r->status && r->batched) r->status = it::rebind_stream(r->h, s->lanes[r->lane].stream);
    if (r->status) {  // rejected (unstable trap, bad input, no memory): completes at once
      if (r->h) iontrap_destroy(r->h);
      r->h = nullptr;
      ++s->completed_total;
      const int64_t rid = r->id;
      report(rid);
      s->completed[rid] = std::move(r);
      continue;
    }
    int64_t bytes = 0;
    if (iontrap_device_bytes(r->h, &bytes) == IONTRAP_OK) r->bytes = bytes;
    s->bytes_in_use += r->bytes;
    s->resident.push_back(std::move(r));
  }
  // 3. next chunks: each batched size class together on its stream, then the shared
  // streams of the others, least remaining work first
  for (int c = 0; c < kLanes; ++c) {
    Lane& l = s->lanes[c];
    if (l.inflight) continue;
    std::vector<iontrap_t*> hs;
    std::vector<int64_t> ns;
    std::vector<Request*> rs;
    for (auto& r : s->resident)
      if (r->batched && r->lane == c && !r->inflight && r->done < r->steps) {
        hs.push_back(r->h);
        ns.push_back(std::min<int64_t>(s->cfg.chunk_steps, r->steps - r->done));
        rs.push_back(r.get());
      }
    if (!hs.empty()) {
      const int st = iontrap_step_many(hs.data(), ns.data(), (int)hs.size());
      auto ev = std::make_shared<Event>();
      cudaEventRecord(ev->ev, l.stream);
      l.ev = ev;
      l.inflight = true;
      for (size_t k = 0; k < rs.size(); ++k) {
        rs[k]->inflight = ns[k];
        if (st && !rs[k]->status) rs[k]->status = st;
      }
    }
  }
  for (size_t q = 0; q < s->solo.size(); ++q) {
    Lane& l = s->solo[q];
    while (!l.inflight) {  // a request whose launch fails is retired; the stream goes to the next
      Request* best = nullptr;
      double best_work = 0.0;
      for (auto& r : s->resident)
        if (!r->batched && !r->inflight && r->done < r->steps && !r->status) {
          const double work = (double)r->n * (double)r->n * (double)(r->steps - r->done);
          if (!best || work < best_work) best = r.get(), best_work = work;
        }
      if (!best) return IONTRAP_OK;
      const double scale = (double)kSoloChunkIons / (double)best->n;
      const int64_t chunk = std::max<int64_t>(
          1, std::min<int64_t>(s->cfg.chunk_steps, (int64_t)(s->cfg.chunk_steps * scale * scale)));
      const int64_t k = std::min<int64_t>(chunk, best->steps - best->done);
      int st = it::rebind_stream(best->h, l.stream);
      if (!st) st = iontrap_step(best->h, k);
      if (st) {
        best->status = st;
        continue;
      }
      l.ev = std::make_shared<Event>();
      cudaEventRecord(l.ev->ev, l.stream);
      l.inflight = true;
      best->inflight = k;
      best->solo = (int)q;
    }
  }
  return IONTRAP_OK;
}

int iontrap_server_result(iontrap_server_t* s, int64_t id, double* x, double* v, int64_t* step, int* status) {
  if (!s) return IONTRAP_EINVAL;
  auto it = s->completed.find(id);
  if (it == s->completed.end()) return IONTRAP_EINVAL;
  Request& r = *it->second;
  if (x && !r.xo.empty()) std::memcpy(x, r.xo.data(), r.xo.size() * sizeof(double));
  if (v && !r.vo.empty()) std::memcpy(v, r.vo.data(), r.vo.size() * sizeof(double));
  if (step) *step = r.final_step;
  if (status) *status = r.status;
  s->completed.erase(it);
  return IONTRAP_OK;
}

int iontrap_server_stats(const iontrap_server_t* s, iontrap_server_counters* out) {
  if (!s || !out) return IONTRAP_EINVAL;
  out->waiting = (int64_t)s->waiting.size();
  out->resident = (int64_t)s->resident.size();
  out->completed = s->completed_total;
  out->device_bytes = s->bytes_in_use;
  return IONTRAP_OK;
}

void iontrap_server_destroy(iontrap_server_t* s) {
  if (!s) return;
  for (Lane& l : s->lanes)
    if (l.stream) cudaStreamSynchronize(l.stream);
  for (Lane& l : s->solo)
    if (l.stream) cudaStreamSynchronize(l.stream);
  for (auto& r : s->resident)
    if (r->h) iontrap_destroy(r->h);
  for (Lane& l : s->lanes) {
    l.ev.reset();
    if (l.stream) cudaStreamDestroy(l.stream);
  }
  for (Lane& l : s->solo) {
    l.ev.reset();
    if (l.stream) cudaStreamDestroy(l.stream);
  }
  if (s->admit) {
    cudaStreamSynchronize(s->admit);
    cudaStreamDestroy(s->admit);
  }
  delete s;
}

}  // extern "C"
