// pdd_server.cu -- serving runtime: continuous batching of estimate requests.
//
// A request (nodes, n_paths, dt, control grid, seed, tag) is admitted when a
// slot of the running batch and room in the device arena are free.  Every
// scheduler iteration issues ONE multi-segment launch of the path kernel that
// carries slices of paths (path indices p0 .. p0+m-1 of every node) of the
// admitted requests -- equal shares of the launch's path-steps, or (policy
// PDD_SERVE_SHORTEST) the requests with the least remaining work first -- so
// requests that arrive while others run join the next launch, and long
// requests progress while short ones come and go.  Launches
// alternate between two streams, so the next launch's blocks fill SMs while
// the previous launch drains.  A request's node records accumulate exact
// integer sums across its slices, so its result is bit-identical to running
// it alone (pdd_estimate_nodes).  When its last slice has been issued, its
// finalisation and the copy of its results to page-locked host memory follow
// on the same stream; the scheduler polls CUDA events (host side) and
// pdd_poll hands the results over.  No device code waits on anything.
//
// Admission by predicted work: a request's work is predicted as n_nodes x
// n_paths x the expected exit index of its (problem, dt), measured by a
// pilot launch the first time the pair is seen and refined by every
// completed request; with a deadline set, pdd_submit refuses a request whose
// work, after the predicted remaining work of everything queued and running,
// would not finish within 80 % of the deadline at the measured rate
// (path-steps of retired launches over the time they took).  Under the earliest-deadline
// policy (every request has the same relative deadline, so it serves them in
// submission order) the admitted work finishes in time as far as the
// prediction holds, and no executed work is thrown away under overload;
// under fair shares or shortest-first a request admitted earlier can be
// slowed by later ones.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pdd.h"
#include "pdd_internal.h"

namespace pdd {
void set_error(const char* fmt, ...);
}

using namespace pdd;

namespace {

using Clock = std::chrono::steady_clock;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// First-fit allocator over [0, size) with coalescing of free ranges.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align256(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

enum class RState { kPending, kActive, kFinishing, kDone, kFailed, kCancelled };

struct Request {
  uint64_t ticket = 0;
  pdd_problem* prob = nullptr;
  ProblemView pv{};
  int cv = 0;  // 0 none, 1 grid, 2 exact
  const void* table = nullptr;
  int grid_n = 0;
  int64_t n_nodes = 0;
  uint64_t n_paths = 0;
  double dt = 0, kappa = 1;
  uint64_t seed = 0;
  uint32_t tag = 0;
  int max_steps = 0;
  std::vector<float> coords[3];
  RState state = RState::kPending;
  int status = PDD_OK;
  uint64_t next_path = 0;  // paths per node already issued
  uint64_t retired_paths = 0;  // paths per node whose launches have completed
  size_t dev_off = 0, dev_bytes = 0, host_off = 0, host_bytes = 0;
  bool has_mem = false;
  int inflight = 0;  // in-flight launches that reference this request
  bool in_active = false;  // in the running batch (until the scheduler drops it)
  cudaEvent_t ready = nullptr;  // inputs copied and records cleared
  cudaEvent_t done = nullptr;   // results in host memory
  Clock::time_point t_submit, t_done;
  double est_steps = 0;  // expected steps per path (for slicing)
  int group = 0;         // requests that can share a launch (problem, CV class)
};

struct Launch {
  cudaEvent_t ev = nullptr;
  int stream = 0;
  std::vector<uint64_t> tickets;
  std::vector<uint64_t> paths;  // paths per node of each ticket's slice
  Clock::time_point t_issue;
};

// Expected exit index of the paths of one (problem, dt): a weighted mean over
// the pilot's and the completed requests' paths.
struct StepsEst {
  double steps = 0.0;
  double weight = 0.0;
};

constexpr int kPilotNodes = 128;        // nodes of a request the pilot samples
constexpr uint64_t kPilotPaths = 64;    // paths per pilot node
constexpr double kDefaultRate = 1e11;   // path-steps/s before any launch has retired

}  // namespace

struct pdd_server {
  pdd_ctx* ctx = nullptr;
  int device = 0, num_sms = 0;
  pdd_server_desc desc{};
  cudaStream_t stream[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  int next_stream = 0;
  char* dev_arena = nullptr;
  char* host_arena = nullptr;  // page-locked results
  char* hdr = nullptr;         // per-launch header slots (cursor, err, trunc, steps): 2 x 256 B
  unsigned long long* hdr_host = nullptr;  // page-locked copies of the 2 headers (4 words each)
  cudaStream_t pilot_stream = nullptr;
  char* pilot_dev = nullptr;   // pilot scratch: header | records | coordinates | mean steps
  double* pilot_host = nullptr;  // page-locked mean exit index of the pilot nodes
  std::mutex pilot_mu;
  std::map<std::pair<pdd_problem*, double>, StepsEst> steps_est;
  double busy_steps = 0.0;     // path-steps of all retired launches
  double busy_s = 0.0;         // time the GPU was busy with them
  Clock::time_point last_retire;
  bool busy_since_retire = false;
  Arena dmem, hmem;
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::deque<uint64_t> pending;
  std::vector<uint64_t> active;
  std::deque<Launch> inflight;
  uint64_t next_ticket = 1;
  std::thread worker;
  std::atomic<bool> stop{false};
  pdd_server_stats st{};
  int inject = 0;
  std::map<pdd_problem*, int> group_ids;
};

namespace {

int request_cv_class(const Request& r) { return r.cv == 2 ? 2 : 0; }

// Bytes of device arena a request needs: records, coordinates, outputs.
size_t dev_need(int64_t n, int dim) {
  return align256((size_t)n * kAccWords * 8) + dim * align256((size_t)n * 4) +
         14 * align256((size_t)n * 8);
}
size_t host_need(int64_t n) { return 14 * align256((size_t)n * 8); }

unsigned long long* req_acc(pdd_server* s, const Request& r) {
  return (unsigned long long*)(s->dev_arena + r.dev_off);
}
float* req_coord(pdd_server* s, const Request& r, int j) {
  return (float*)(s->dev_arena + r.dev_off + align256((size_t)r.n_nodes * kAccWords * 8) +
                  j * align256((size_t)r.n_nodes * 4));
}
char* req_out_dev(pdd_server* s, const Request& r) {
  return s->dev_arena + r.dev_off + align256((size_t)r.n_nodes * kAccWords * 8) +
         r.pv.dim * align256((size_t)r.n_nodes * 4);
}

void release_mem(pdd_server* s, Request& r) {
  if (!r.has_mem) return;
  s->dmem.release(r.dev_off, r.dev_bytes);
  s->hmem.release(r.host_off, r.host_bytes);
  r.has_mem = false;
}

void finish_request(pdd_server* s, Request& r, RState state, int status) {
  r.state = state;
  r.status = status;
  r.t_done = Clock::now();
  if (state == RState::kDone) s->st.completed++;
  else if (state == RState::kCancelled) s->st.cancelled++;
  else s->st.failed++;
  s->cv_done.notify_all();
}

// Predicted path-steps still to run for a queued or running request: the
// paths whose launches have not completed yet.
double remaining_work(const Request& r) {
  if (r.state != RState::kPending && r.state != RState::kActive &&
      r.state != RState::kFinishing)
    return 0.0;
  return (double)(r.n_paths - r.retired_paths) * (double)r.n_nodes * r.est_steps;
}

double backlog_work(pdd_server* s) {
  double b = 0.0;
  for (uint64_t t : s->pending) {
    auto it = s->reqs.find(t);
    if (it != s->reqs.end()) b += remaining_work(*it->second);
  }
  for (uint64_t t : s->active) {
    auto it = s->reqs.find(t);
    if (it != s->reqs.end()) b += remaining_work(*it->second);
  }
  return b;
}

// Share of the deadline that admission fills with predicted work; the rest
// is a margin for the error of the predicted work and rate: work is counted
// in path-steps and the rate is the average over the requests served, while
// a control-variate step costs ~1.3 plain ones and 10-step paths run at
// about half the path-step rate of 1,000-step ones, so a stretch of costly
// requests runs slower than the average (at 90 % the p99 latency under
// overload was 1-7 % above the deadline).
constexpr double kDeadlineShare = 0.8;

// Path-steps per second of GPU-busy time over every retired launch (launch
// overheads and the drain of small launches included), once 0.2 s of busy
// time has been seen; the hint (or 1e11) before.
double current_rate(const pdd_server* s) {
  if (s->busy_s >= 0.2 && s->busy_steps > 0.0) return s->busy_steps / s->busy_s;
  return s->desc.rate_hint > 0.0 ? s->desc.rate_hint : kDefaultRate;
}

size_t pilot_bytes() {
  return 256 + (size_t)kPilotNodes * kAccWords * 8 + 3 * align256(kPilotNodes * 4) +
         align256(kPilotNodes * 8);
}

// Expected exit index at r.dt from a pilot launch: kPilotPaths plain paths
// from each of up to kPilotNodes nodes of the request, on the server's pilot
// stream (synchronous; it queues behind launches already on the device).
int run_pilot(pdd_server* s, const Request& r, double* steps) {
  std::lock_guard<std::mutex> lk(s->pilot_mu);
  DeviceGuard guard(s->device);
  const int dim = r.pv.dim;
  const int64_t n = std::min<int64_t>(r.n_nodes, kPilotNodes);
  char* hdr = s->pilot_dev;
  unsigned long long* acc = (unsigned long long*)(hdr + 256);
  char* coords = hdr + 256 + (size_t)kPilotNodes * kAccWords * 8;
  double* mean_steps = (double*)(coords + 3 * align256(kPilotNodes * 4));
  float sample[3][kPilotNodes];
  for (int64_t i = 0; i < n; ++i) {
    const int64_t src = n == r.n_nodes ? i : i * r.n_nodes / n;  // evenly spread
    for (int j = 0; j < dim; ++j) sample[j][i] = r.coords[j][(size_t)src];
  }
  cudaStream_t st = s->pilot_stream;
  cudaError_t e = cudaMemsetAsync(hdr, 0, 256 + (size_t)n * kAccWords * 8, st);
  for (int j = 0; j < dim && e == cudaSuccess; ++j)
    e = cudaMemcpyAsync(coords + j * align256(kPilotNodes * 4), sample[j], (size_t)n * 4,
                        cudaMemcpyHostToDevice, st);
  PathArgs pa{};
  pa.cursor = (unsigned long long*)hdr;
  pa.err = (unsigned*)(hdr + 8);
  pa.trunc_total = (unsigned long long*)(hdr + 16);
  pa.y_exp = r.pv.y_rule == PDD_Y_EXP;
  pa.n_segs = 1;
  SegArgs& sg = pa.seg[0];
  sg.cx = (const float*)coords;
  sg.cy = (const float*)(coords + align256(kPilotNodes * 4));
  sg.cz = dim == 3 ? (const float*)(coords + 2 * align256(kPilotNodes * 4)) : sg.cx;
  sg.total = (unsigned long long)n * kPilotPaths;
  sg.n_paths = kPilotPaths;
  sg.n_nodes = (unsigned long long)n;
  sg.acc = acc;
  sg.emit_stride = kPilotPaths;
  sg.h = r.dt;
  sg.sqrt_h = std::sqrt(r.dt);
  sg.thr0 = (r.pv.exit_rule == PDD_EXIT_GOBET_MENOZZI ? 0.5826 : 0.0) * sg.sqrt_h;
  sg.key0 = 0x5eed1u;  // a stream of its own, apart from any request's
  sg.key1 = 0xFFFFFFF0u;
  sg.max_steps = r.max_steps;
  pa.total = sg.total;
  int blocks = 0;
  if (e == cudaSuccess) e = launch_paths(r.pv.kind, r.pv.precision, 0, pa, s->num_sms, st, &blocks);
  StatPtrs sp{};
  sp.mean_steps = mean_steps;
  if (e == cudaSuccess) e = launch_finalize(acc, (uint32_t)n, 1.0, sp, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->pilot_host, mean_steps, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error("pdd_submit: pilot launch: %s", cudaGetErrorString(e));
    return PDD_ERR_CUDA;
  }
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) m += s->pilot_host[i];
  *steps = n > 0 ? m / (double)n : 0.0;
  return PDD_OK;
}

// Admit pending requests while slots and arena room allow (FIFO, no overtaking).
void admit(pdd_server* s) {
  while (!s->pending.empty() && (int)s->active.size() < s->desc.max_active) {
    const uint64_t t = s->pending.front();
    auto it = s->reqs.find(t);
    if (it == s->reqs.end() || it->second->state != RState::kPending) {
      s->pending.pop_front();
      continue;
    }
    Request& r = *it->second;
    const size_t dneed = dev_need(r.n_nodes, r.pv.dim), hneed = host_need(r.n_nodes);
    size_t doff = 0, hoff = 0;
    if (s->inject == 1) {  // injected allocation failure (host side)
      s->inject = 0;
      s->pending.pop_front();
      finish_request(s, r, RState::kFailed, PDD_ERR_NOMEM);
      continue;
    }
    if (!s->dmem.alloc(dneed, &doff)) break;  // wait for room
    if (!s->hmem.alloc(hneed, &hoff)) {
      s->dmem.release(doff, dneed);
      break;
    }
    r.dev_off = doff;
    r.dev_bytes = dneed;
    r.host_off = hoff;
    r.host_bytes = hneed;
    r.has_mem = true;
    s->pending.pop_front();
    // inputs and cleared records, ordered before every launch by `ready`
    cudaError_t e = cudaMemsetAsync(req_acc(s, r), 0, (size_t)r.n_nodes * kAccWords * 8,
                                    s->copy_stream);
    for (int j = 0; j < r.pv.dim && e == cudaSuccess; ++j)
      e = cudaMemcpyAsync(req_coord(s, r, j), r.coords[j].data(), (size_t)r.n_nodes * 4,
                          cudaMemcpyHostToDevice, s->copy_stream);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r.ready, s->copy_stream);
    if (e != cudaSuccess) {
      release_mem(s, r);
      finish_request(s, r, RState::kFailed, PDD_ERR_CUDA);
      continue;
    }
    r.state = RState::kActive;
    r.in_active = true;
    s->active.push_back(t);
    s->st.admitted++;
  }
}

// Issue one launch with slices of the active requests of one group.
bool issue_launch(pdd_server* s) {
  // the group of the oldest active request that still has paths to issue
  int group = -1;
  for (uint64_t t : s->active) {
    Request& r = *s->reqs[t];
    if (r.state == RState::kActive && r.next_path < r.n_paths) {
      group = r.group;
      break;
    }
  }
  if (group < 0) return false;
  std::vector<Request*> batch;
  for (uint64_t t : s->active) {
    Request& r = *s->reqs[t];
    if (r.state == RState::kActive && r.next_path < r.n_paths && r.group == group)
      batch.push_back(&r);
    if ((int)batch.size() == kMaxSegments) break;
  }
  // paths of every request in this launch: equal shares of the quantum, or
  // the least remaining work first, each request up to all its paths
  auto per_path_of = [](const Request* r) {
    return std::max(1.0, r->est_steps) * (double)r->n_nodes;
  };
  const double quantum = (double)s->desc.quantum_path_steps;
  std::vector<uint64_t> take(batch.size(), 0);
  if (s->desc.policy == PDD_SERVE_SHORTEST || s->desc.policy == PDD_SERVE_EARLIEST_DEADLINE) {
    // shortest remaining work first; or, with one relative deadline for every
    // request, earliest deadline first = submission order, which is the order
    // of the running batch already
    if (s->desc.policy == PDD_SERVE_SHORTEST)
      std::stable_sort(batch.begin(), batch.end(), [&](const Request* x, const Request* y) {
        return (double)(x->n_paths - x->next_path) * per_path_of(x) <
               (double)(y->n_paths - y->next_path) * per_path_of(y);
      });
    double budget = quantum;
    for (size_t i = 0; i < batch.size() && budget > 0.0; ++i) {
      const double pp = per_path_of(batch[i]);
      const uint64_t m = (uint64_t)std::max(1.0, std::floor(budget / pp));
      take[i] = std::min<uint64_t>(m, batch[i]->n_paths - batch[i]->next_path);
      budget -= (double)take[i] * pp;
    }
  } else {
    const double share = quantum / (double)batch.size();
    for (size_t i = 0; i < batch.size(); ++i) {
      const uint64_t m = (uint64_t)std::max(1.0, std::floor(share / per_path_of(batch[i])));
      take[i] = std::min<uint64_t>(m, batch[i]->n_paths - batch[i]->next_path);
    }
  }
  size_t kept = 0;
  for (size_t i = 0; i < batch.size(); ++i)
    if (take[i] > 0) {
      batch[kept] = batch[i];
      take[kept] = take[i];
      ++kept;
    }
  batch.resize(kept);
  take.resize(kept);
  const ProblemView& pv = batch[0]->pv;
  int cv = 0;
  for (Request* r : batch) cv = std::max(cv, r->cv);
  const int sidx = s->next_stream;
  s->next_stream ^= 1;
  cudaStream_t st = s->stream[sidx];
  PathArgs pa{};
  char* hdr = s->hdr + 256 * sidx;
  // The header slot of this stream is reused every other launch; the previous
  // launch on this stream is ordered before this one.
  cudaError_t e = cudaMemsetAsync(hdr, 0, 256, st);
  pa.cursor = (unsigned long long*)hdr;
  pa.err = (unsigned*)(hdr + 8);
  pa.trunc_total = (unsigned long long*)(hdr + 16);
  pa.steps_total = (unsigned long long*)(hdr + 24);
  pa.y_exp = pv.y_rule == PDD_Y_EXP;
  int bt = 0, mb = 0, dev = 0, sms = 0;
  ctx_view(s->ctx, &dev, &sms, &bt, &mb);
  pa.block_threads = bt;
  pa.max_blocks = mb;
  pa.claim = ctx_claim(s->ctx);
  unsigned long long begin = 0;
  int ns = 0;
  Launch L;
  for (size_t bi = 0; bi < batch.size(); ++bi) {
    Request* r = batch[bi];
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, r->ready, 0);
    const uint64_t m = take[bi];
    SegArgs& sg = pa.seg[ns++];
    sg.cx = req_coord(s, *r, 0);
    sg.cy = req_coord(s, *r, 1);
    sg.cz = r->pv.dim == 3 ? req_coord(s, *r, 2) : sg.cx;
    sg.begin = begin;
    sg.total = (unsigned long long)r->n_nodes * m;
    sg.n_paths = m;
    sg.n_nodes = (unsigned long long)r->n_nodes;
    sg.acc = req_acc(s, *r);
    sg.grad = r->table;
    sg.emit_phi = nullptr;
    sg.emit_xi = nullptr;
    sg.emit_steps = nullptr;
    sg.emit_stride = r->n_paths;
    sg.h = r->dt;
    sg.sqrt_h = std::sqrt(r->dt);
    const double c0 = r->pv.exit_rule == PDD_EXIT_GOBET_MENOZZI ? 0.5826 : 0.0;
    sg.thr0 = c0 * sg.sqrt_h;
    sg.path_off = (uint32_t)r->next_path;
    sg.key0 = (uint32_t)r->seed;
    sg.key1 = r->tag;
    sg.seed_hi = (uint32_t)(r->seed >> 32);
    sg.grid_n = r->grid_n;
    sg.max_steps = r->max_steps;
    begin += sg.total;
    r->next_path += m;
    r->inflight += 1;
    L.tickets.push_back(r->ticket);
    L.paths.push_back(m);
  }
  pa.n_segs = ns;
  pa.total = begin;
  int blocks = 0;
  if (e == cudaSuccess) e = launch_paths(pv.kind, pv.precision, cv, pa, s->num_sms, st, &blocks);
  // the launch's header (error word, executed path-steps), read when its event
  // has completed; the slot is not reused before then (the next launch on this
  // stream is issued after this one retires)
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->hdr_host + 4 * sidx, hdr, 32, cudaMemcpyDeviceToHost, st);
  L.stream = sidx;
  L.t_issue = Clock::now();
  s->st.launches++;
  // requests whose last slice is in this launch: finalise and copy out
  const cudaEvent_t prev = s->inflight.empty() ? nullptr : s->inflight.back().ev;
  for (Request* r : batch) {
    if (r->next_path < r->n_paths || e != cudaSuccess) continue;
    // earlier slices may be in the launch on the other stream
    if (prev) e = cudaStreamWaitEvent(st, prev, 0);
    StatPtrs sp{};
    char* o = req_out_dev(s, *r);
    const size_t n8 = align256((size_t)r->n_nodes * 8);
    double* d[12];
    for (int i = 0; i < 12; ++i) d[i] = (double*)(o + i * n8);
    sp = StatPtrs{d[0], d[1], d[2], d[3], d[4], d[5], d[6], d[7], d[8], d[9], d[10], d[11],
                  (unsigned long long*)(o + 12 * n8), (unsigned long long*)(o + 13 * n8)};
    if (e == cudaSuccess)
      e = launch_finalize(req_acc(s, *r), (uint32_t)r->n_nodes, r->kappa, sp, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->host_arena + r->host_off, o, 14 * n8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r->done, st);
    r->state = RState::kFinishing;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(L.ev, st);
  if (e != cudaSuccess) {
    set_error("pdd server: launch failed: %s", cudaGetErrorString(e));
    for (Request* r : batch) {
      r->inflight -= 1;
      if (r->state != RState::kFailed) finish_request(s, *r, RState::kFailed, PDD_ERR_CUDA);
    }
    if (L.ev) cudaEventDestroy(L.ev);
    return false;
  }
  if (s->inject == 2 && !batch.empty()) {  // injected loss of one request mid-flight
    s->inject = 0;
    Request* r = batch.back();
    r->next_path = r->n_paths;
    finish_request(s, *r, RState::kFailed, PDD_ERR_CANCELLED);
  }
  s->inflight.push_back(std::move(L));
  return true;
}

// Retire completed launches and requests (host-side event polling).
void retire(pdd_server* s) {
  while (!s->inflight.empty() && cudaEventQuery(s->inflight.front().ev) == cudaSuccess) {
    Launch& L = s->inflight.front();
    const unsigned long long* h = s->hdr_host + 4 * L.stream;
    const double steps = (double)h[3];
    s->st.path_steps += (int64_t)h[3];
    const unsigned err = (unsigned)(h[1] & 0xFFFFFFFFull);
    // measured rate: this launch's path-steps over the time since the GPU last
    // became busy with it (the previous retirement, or this launch's issue)
    const Clock::time_point now = Clock::now();
    const Clock::time_point from =
        s->busy_since_retire && s->last_retire > L.t_issue ? s->last_retire : L.t_issue;
    const double secs = std::chrono::duration<double>(now - from).count();
    if (secs > 0.0) {
      s->busy_steps += steps;
      s->busy_s += secs;
    }
    s->last_retire = now;
    s->busy_since_retire = s->inflight.size() > 1;
    const int fail_status = err != 0u ? error_word_status(err, "pdd server launch") : PDD_OK;
    for (size_t k = 0; k < L.tickets.size(); ++k) {
      auto it = s->reqs.find(L.tickets[k]);
      if (it == s->reqs.end()) continue;
      Request& r = *it->second;
      r.inflight -= 1;
      r.retired_paths += L.paths[k];
      if (fail_status != PDD_OK &&
          (r.state == RState::kActive || r.state == RState::kFinishing)) {
        r.next_path = r.n_paths;
        finish_request(s, r, RState::kFailed, fail_status);
      }
    }
    cudaEventDestroy(L.ev);
    s->inflight.pop_front();
  }
  for (size_t i = 0; i < s->active.size();) {
    Request& r = *s->reqs[s->active[i]];
    bool drop = false;
    if (r.state == RState::kFinishing && r.done && cudaEventQuery(r.done) == cudaSuccess) {
      // exit indices of the completed request: goodput and the (problem, dt) estimate
      const size_t n8 = align256((size_t)r.n_nodes * 8);
      const double* ms = (const double*)(s->host_arena + r.host_off + 11 * n8);
      double m = 0.0;
      for (int64_t i = 0; i < r.n_nodes; ++i) m += ms[i];
      m /= (double)r.n_nodes;
      s->st.completed_path_steps += (int64_t)(m * (double)r.n_nodes * (double)r.n_paths);
      StepsEst& est = s->steps_est[{r.prob, r.dt}];
      const double w = (double)r.n_nodes * (double)r.n_paths;
      est.steps = (est.steps * est.weight + m * w) / (est.weight + w);
      est.weight += w;
      finish_request(s, r, RState::kDone, PDD_OK);
      drop = true;
    } else if ((r.state == RState::kCancelled || r.state == RState::kFailed) && r.inflight == 0 &&
               (!r.done || cudaEventQuery(r.done) == cudaSuccess)) {
      drop = true;
    }
    if (drop) {
      if (r.state != RState::kDone) release_mem(s, r);  // done: freed when polled
      r.in_active = false;
      s->active.erase(s->active.begin() + i);
      s->cv_done.notify_all();
    } else {
      ++i;
    }
  }
}

void worker_loop(pdd_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    retire(s);
    admit(s);
    bool issued = false;
    if ((int)s->inflight.size() < 2) issued = issue_launch(s);
    if (s->stop && s->inflight.empty()) break;
    if (!issued) {
      // nothing to issue now: wait for a submission or for running work
      const auto wait = s->inflight.empty() && s->pending.empty() ? std::chrono::milliseconds(5)
                                                                   : std::chrono::milliseconds(0);
      if (wait.count() > 0) {
        s->cv_work.wait_for(lk, wait);
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(100));
        lk.lock();
      }
    }
  }
}

}  // namespace

extern "C" {

int pdd_server_create(pdd_ctx* ctx, const pdd_server_desc* desc, pdd_server** out) {
  if (!ctx || !out) {
    set_error("pdd_server_create: NULL argument");
    return PDD_ERR_INVALID;
  }
  *out = nullptr;
  pdd_server_desc d{};
  if (desc) d = *desc;
  if (d.max_active <= 0) d.max_active = 32;
  if (d.max_active > kMaxSegments) {
    set_error("pdd_server_create: max_active %d > %d", d.max_active, kMaxSegments);
    return PDD_ERR_INVALID;
  }
  if (d.max_queue <= 0) d.max_queue = 256;
  if (d.quantum_path_steps <= 0) d.quantum_path_steps = 8000000000ll;
  if (d.device_arena_bytes == 0) d.device_arena_bytes = (size_t)256 << 20;
  if (!(d.deadline_s >= 0.0) || !(d.rate_hint >= 0.0)) {
    set_error("pdd_server_create: deadline_s and rate_hint must be >= 0");
    return PDD_ERR_INVALID;
  }
  if (d.policy != PDD_SERVE_FAIR && d.policy != PDD_SERVE_SHORTEST &&
      d.policy != PDD_SERVE_EARLIEST_DEADLINE) {
    set_error("pdd_server_create: policy %d is not PDD_SERVE_FAIR, PDD_SERVE_SHORTEST or "
              "PDD_SERVE_EARLIEST_DEADLINE", d.policy);
    return PDD_ERR_INVALID;
  }
  auto s = std::make_unique<pdd_server>();
  s->ctx = ctx;
  s->desc = d;
  int bt = 0, mb = 0;
  ctx_view(ctx, &s->device, &s->num_sms, &bt, &mb);
  DeviceGuard guard(s->device);  // restores the caller's device on return
  if (!guard.ok) {
    set_error("pdd_server_create: cannot select device %d", s->device);
    return PDD_ERR_CUDA;
  }
  // host results need 112 of every 252 device bytes per node
  const size_t host_bytes = d.device_arena_bytes / 2 + (1 << 20);
  cudaError_t e = cudaMalloc((void**)&s->dev_arena, d.device_arena_bytes);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s->host_arena, host_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->hdr, 512);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s->hdr_host, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->pilot_dev, pilot_bytes());
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s->pilot_host, kPilotNodes * sizeof(double));
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&s->stream[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->pilot_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    set_error("pdd_server_create: %s", cudaGetErrorString(e));
    if (s->dev_arena) cudaFree(s->dev_arena);
    if (s->host_arena) cudaFreeHost(s->host_arena);
    if (s->hdr) cudaFree(s->hdr);
    if (s->hdr_host) cudaFreeHost(s->hdr_host);
    if (s->pilot_dev) cudaFree(s->pilot_dev);
    if (s->pilot_host) cudaFreeHost(s->pilot_host);
    for (auto& x : s->stream)
      if (x) cudaStreamDestroy(x);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->pilot_stream) cudaStreamDestroy(s->pilot_stream);
    return e == cudaErrorMemoryAllocation ? PDD_ERR_NOMEM : PDD_ERR_CUDA;
  }
  s->dmem.reset(d.device_arena_bytes);
  s->hmem.reset(host_bytes);
  pdd_server* raw = s.release();
  raw->worker = std::thread(worker_loop, raw);
  *out = raw;
  return PDD_OK;
}

int pdd_submit(pdd_server* s, pdd_problem* p, const pdd_estimate_args* a, uint64_t* ticket) {
  if (!s || !p || !a || !ticket) {
    set_error("pdd_submit: NULL argument");
    return PDD_ERR_INVALID;
  }
  auto r = std::make_unique<Request>();
  if (!problem_view(p, &r->pv) || problem_ctx(p) != s->ctx) {
    set_error("pdd_submit: the problem belongs to another context");
    return PDD_ERR_INVALID;
  }
  const int dim = r->pv.dim;
  std::string why;
  if (a->n_nodes < 0 || a->n_nodes > ((int64_t)1 << 31)) why = "n_nodes out of range";
  else if (a->n_paths < 1 || a->n_paths >= ((int64_t)1 << 32)) why = "n_paths outside [1, 2^32)";
  else if (!(a->dt > 0.0) || !std::isfinite(a->dt)) why = "dt must be finite and > 0";
  else if (a->flags & ~PDD_FLAG_ASYNC) why = "serving takes no per-path output";
  if (why.empty() && a->n_nodes > 0)
    for (int j = 0; j < dim; ++j)
      if (!a->coords[j]) why = "NULL coordinates";
  if (why.empty()) {
    if (a->grid_id == PDD_CV_NONE) {
      r->cv = 0;
    } else if (a->grid_id == PDD_CV_EXACT) {
      r->cv = 2;
    } else if (a->grid_id >= 0 && a->grid_id < PDD_MAX_GRIDS && r->pv.grid_table[a->grid_id]) {
      r->cv = 1;
      r->table = r->pv.grid_table[a->grid_id];
      r->grid_n = r->pv.grid_n[a->grid_id];
    } else {
      why = "grid_id is not a loaded grid";
    }
  }
  if (!why.empty()) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.rejected_invalid++;
    set_error("pdd_submit: %s", why.c_str());
    return PDD_ERR_INVALID;
  }
  if (dev_need(a->n_nodes, dim) > s->desc.device_arena_bytes) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.rejected_nomem++;
    set_error("pdd_submit: request needs %zu bytes, the arena has %zu", dev_need(a->n_nodes, dim),
              s->desc.device_arena_bytes);
    return PDD_ERR_NOMEM;
  }
  r->prob = p;
  r->n_nodes = a->n_nodes;
  r->n_paths = (uint64_t)a->n_paths;
  r->dt = a->dt;
  r->kappa = a->kappa > 0.0 ? a->kappa : 1.0;
  r->seed = a->seed;
  r->tag = a->stream_tag;
  int64_t ms = r->pv.max_steps;
  if (ms <= 0) ms = (int64_t)std::min(2.0e9, std::ceil(100.0 / a->dt));
  r->max_steps = (int)std::min<int64_t>(ms, 2000000000ll);
  // copy the inputs now: the caller may reuse its buffers on return
  for (int j = 0; j < dim; ++j) {
    r->coords[j].resize((size_t)a->n_nodes);
    if (a->n_nodes == 0) continue;
    if (a->coords_on_device) {
      DeviceGuard guard(s->device);
      cudaError_t e = cudaMemcpy(r->coords[j].data(), a->coords[j], (size_t)a->n_nodes * 4,
                                 cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        set_error("pdd_submit: reading coordinates: %s", cudaGetErrorString(e));
        return PDD_ERR_CUDA;
      }
    } else {
      std::memcpy(r->coords[j].data(), a->coords[j], (size_t)a->n_nodes * 4);
    }
  }
  // expected exit index of this (problem, dt): cached, else a pilot launch
  double est = 0.0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->steps_est.find({p, a->dt});
    if (it != s->steps_est.end()) est = it->second.steps;
  }
  if (est <= 0.0 && r->n_nodes > 0) {
    const int rc = run_pilot(s, *r, &est);
    if (rc != PDD_OK) return rc;
    std::lock_guard<std::mutex> lk(s->mu);
    StepsEst& e = s->steps_est[{p, a->dt}];
    if (e.weight == 0.0) {
      e.steps = est;
      e.weight = (double)std::min<int64_t>(r->n_nodes, kPilotNodes) * (double)kPilotPaths;
    }
  }
  r->est_steps = std::max(1.0, est);
  std::lock_guard<std::mutex> lk(s->mu);
  s->st.submitted++;
  if ((int64_t)s->pending.size() >= s->desc.max_queue) {
    s->st.rejected_busy++;
    set_error("pdd_submit: admission queue full (%d requests)", s->desc.max_queue);
    return PDD_ERR_BUSY;
  }
  if (s->desc.deadline_s > 0.0) {
    const double work = (double)r->n_nodes * (double)r->n_paths * r->est_steps;
    const double backlog = backlog_work(s);
    const double rate = current_rate(s);
    if ((backlog + work) / rate > kDeadlineShare * s->desc.deadline_s) {
      s->st.rejected_deadline++;
      set_error("pdd_submit: predicted %.3g path-steps after a backlog of %.3g do not finish "
                "within the %.3g s deadline at %.3g path-steps/s",
                work, backlog, s->desc.deadline_s, rate);
      return PDD_ERR_DEADLINE;
    }
  }
  auto git = s->group_ids.find(p);
  int gid = (int)s->group_ids.size() * 3;
  if (git == s->group_ids.end()) s->group_ids[p] = gid;
  else gid = git->second;
  r->group = gid + request_cv_class(*r);
  r->ticket = s->next_ticket++;
  r->t_submit = Clock::now();
  *ticket = r->ticket;
  if (r->n_nodes == 0) {
    r->state = RState::kDone;
    r->t_done = r->t_submit;
    s->st.completed++;
    s->reqs[r->ticket] = std::move(r);
    return PDD_OK;
  }
  s->pending.push_back(r->ticket);
  s->reqs[r->ticket] = std::move(r);
  s->cv_work.notify_all();
  return PDD_OK;
}

int pdd_poll(pdd_server* s, uint64_t ticket, pdd_node_stats* out, int timeout_us) {
  if (!s || !out) {
    set_error("pdd_poll: NULL argument");
    return PDD_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("pdd_poll: unknown ticket %llu", (unsigned long long)ticket);
    return PDD_ERR_INVALID;
  }
  // a cancelled or failed request is handed back only once the scheduler has
  // let go of it (no launch in flight references its memory)
  auto finished = [&] {
    const Request& q = *s->reqs[ticket];
    return q.state == RState::kDone ||
           ((q.state == RState::kCancelled || q.state == RState::kFailed) && q.inflight == 0 &&
            !q.in_active);
  };
  if (!finished()) {
    if (timeout_us <= 0) return PDD_ERR_NOT_READY;
    if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), finished)) {
      set_error("pdd_poll: ticket %llu not finished within %d us", (unsigned long long)ticket,
                timeout_us);
      return PDD_ERR_TIMEOUT;
    }
  }
  Request& r = *s->reqs[ticket];
  int status = r.status;
  if (r.state == RState::kCancelled) status = PDD_ERR_CANCELLED;
  if (r.state == RState::kDone && r.n_nodes > 0) {
    const size_t n = (size_t)r.n_nodes, n8 = align256(n * 8);
    const char* src = s->host_arena + r.host_off;
    double* const user_d[12] = {out->mean_phi, out->var_phi, out->mean_cv, out->var_cv,
                                out->cov_phi_xi, out->var_xi, out->rho, out->se_phi,
                                out->se_cv, out->vr, out->pred_speedup, out->mean_steps};
    uint64_t* const user_u[2] = {out->n_paths, out->n_truncated};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 14 && e == cudaSuccess; ++i) {
      void* dst = i < 12 ? (void*)user_d[i] : (void*)user_u[i - 12];
      if (!dst) continue;
      if (out->on_device) e = cudaMemcpy(dst, src + i * n8, n * 8, cudaMemcpyHostToDevice);
      else std::memcpy(dst, src + i * n8, n * 8);
    }
    if (e != cudaSuccess) {
      set_error("pdd_poll: copying results: %s", cudaGetErrorString(e));
      status = PDD_ERR_CUDA;
    }
    release_mem(s, r);
  }
  if (r.ready) cudaEventDestroy(r.ready);
  if (r.done) cudaEventDestroy(r.done);
  s->reqs.erase(it);
  if (status < 0 && status != PDD_ERR_CANCELLED) set_error("pdd_poll: request failed (%d)", status);
  if (status == PDD_ERR_CANCELLED) set_error("pdd_poll: request was cancelled");
  return status;
}

int pdd_cancel(pdd_server* s, uint64_t ticket) {
  if (!s) {
    set_error("pdd_cancel: NULL argument");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("pdd_cancel: unknown ticket %llu", (unsigned long long)ticket);
    return PDD_ERR_INVALID;
  }
  Request& r = *it->second;
  if (r.state == RState::kPending || r.state == RState::kActive) {
    r.next_path = r.n_paths;  // no further slices
    finish_request(s, r, RState::kCancelled, PDD_ERR_CANCELLED);
  }
  return PDD_OK;
}

int pdd_server_get_stats(pdd_server* s, pdd_server_stats* out) {
  if (!s || !out) {
    set_error("pdd_server_get_stats: NULL argument");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->pending = (int64_t)s->pending.size();
  out->active = (int64_t)s->active.size();
  out->backlog_path_steps = (int64_t)backlog_work(s);
  out->rate_path_steps_per_s = (int64_t)current_rate(s);
  return PDD_OK;
}

int pdd_server_inject_fault(pdd_server* s, int fault) {
  if (!s || fault < 0 || fault > 2) {
    set_error("pdd_server_inject_fault: bad arguments");
    return PDD_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->inject = fault;
  return PDD_OK;
}

void pdd_server_destroy(pdd_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->reqs) {
      Request& r = *kv.second;
      if (r.state == RState::kPending || r.state == RState::kActive) {
        r.next_path = r.n_paths;
        finish_request(s, r, RState::kCancelled, PDD_ERR_CANCELLED);
      }
    }
    s->pending.clear();
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  DeviceGuard guard(s->device);
  for (auto& x : s->stream) cudaStreamSynchronize(x);
  cudaStreamSynchronize(s->copy_stream);
  cudaStreamSynchronize(s->pilot_stream);
  for (auto& kv : s->reqs) {
    if (kv.second->ready) cudaEventDestroy(kv.second->ready);
    if (kv.second->done) cudaEventDestroy(kv.second->done);
  }
  for (auto& L : s->inflight)
    if (L.ev) cudaEventDestroy(L.ev);
  cudaFree(s->dev_arena);
  cudaFreeHost(s->host_arena);
  cudaFree(s->hdr);
  cudaFreeHost(s->hdr_host);
  cudaFree(s->pilot_dev);
  cudaFreeHost(s->pilot_host);
  for (auto& x : s->stream) cudaStreamDestroy(x);
  cudaStreamDestroy(s->copy_stream);
  cudaStreamDestroy(s->pilot_stream);
  delete s;
}

}  // extern "C"
