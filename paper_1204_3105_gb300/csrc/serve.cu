// serve.cu - a continuous-batching server for FMM solves (fmm2d_serve_*).
//
// Requests (points, strengths and output in host memory) are queued on
// submit and admitted, oldest first, as soon as an execution slot is free and
// the request's device-memory estimate fits in the HBM budget next to the
// requests already running (a request that does not fit lets smaller,
// later requests go first).  Each slot is a host thread with its own CUDA
// stream and its own plans (one per tiling and precision, reused across
// requests), so the work of several requests overlaps on the device.  When a
// slot takes a small adaptive request, the queued requests that can share its
// solve (same tiling, eps, p, flags and domain) come along and the batch runs
// as one forest: one build and one evaluation for all of them.
// Completion is reported through fmm2d_serve_poll / fmm2d_serve_wait.
// The paper has no serving layer; the evaluation each request runs is the
// FMM of fmm2d_build + fmm2d_evaluate.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "plan.h"

namespace fmm2d {
namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket = 0;
  fmm2d_request req;
  size_t est_bytes = 0;
  Clock::time_point t_submit, t_start, t_end;
  fmm2d_result res;
  bool done = false;
};

struct SlotBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaError_t reserve(size_t b) {
    if (b <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, b);
    if (e == cudaSuccess) bytes = b;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  ~SlotBuf() { release(); }
};

struct Slot {
  int id = 0;
  cudaStream_t stream = nullptr;
  // plans keyed by (tiling, flags, levels, p): a plan keeps its operator
  // tables and device memory for requests with the same parameters; the
  // cache is trimmed, least recently used first, to cache_bytes
  std::map<std::tuple<int, unsigned, int, int>, fmm2d_plan *> plans;
  std::map<std::tuple<int, unsigned, int, int>, uint64_t> last_use;
  uint64_t tick = 0;
  size_t cache_bytes = 0;
  SlotBuf src, tgt, u, out;
};

// Drop the slot's cached plans, least recently used first, until the device
// memory they hold is at most `cap` bytes.  cap = 0 drops every plan and
// frees the slot's input and output buffers too.
void trim_plans(Slot &sl, size_t cap) {
  for (;;) {
    size_t tot = 0;
    bool found = false;
    std::tuple<int, unsigned, int, int> victim;
    uint64_t oldest = UINT64_MAX;
    for (auto &kv : sl.plans) {
      if (!kv.second) continue;
      tot += plan_device_bytes(kv.second);
      const uint64_t t = sl.last_use[kv.first];
      if (t < oldest) {
        oldest = t;
        victim = kv.first;
        found = true;
      }
    }
    if (tot <= cap || !found) break;
    fmm2d_plan_destroy(sl.plans[victim]);
    sl.plans.erase(victim);
    sl.last_use.erase(victim);
  }
  if (cap == 0) {
    sl.src.release();
    sl.tgt.release();
    sl.u.release();
    sl.out.release();
  }
}

// Device-memory estimate of one request: inputs and outputs, the plan's
// per-point arrays, and its tree (about 1 KB per cell, cells <= points).
size_t estimate_bytes(const fmm2d_request &r) {
  const size_t esz = (r.flags & FMM2D_IN_F32) ? 4 : 8;
  const size_t ns = (size_t)r.n_src, nt = r.tgt_xy ? (size_t)r.n_tgt : 0;
  const size_t io = ns * 3 * esz + nt * 2 * esz + (r.tgt_xy ? nt : ns) * 8;
  const size_t pts = (ns + nt) * 96;
  const size_t tree = (ns + nt) * 1024 / 16 + (32u << 20);
  return io + pts + tree;
}

// Continuous batching: small adaptive requests with targets = sources that
// wait together with equal tiling, eps, p, flags and domain are solved as one
// forest (fmm2d_build_forest), so the launches and level read-backs of one
// solve serve them all.
constexpr int64_t MERGE_MAX_POINTS = (int64_t)1 << 19;     // requests up to this size merge
constexpr int64_t MERGE_BATCH_POINTS = (int64_t)1 << 22;   // points per forest at most
constexpr int MERGE_MAX = 256;                              // requests per forest at most

bool mergeable(const fmm2d_request &r) {
  return (r.flags & FMM2D_ADAPTIVE) && r.tgt_xy == nullptr && r.levels == 0 && r.n_src > 0 &&
         r.n_src <= MERGE_MAX_POINTS;
}

bool same_solve(const fmm2d_request &a, const fmm2d_request &b) {
  return a.tiling == b.tiling && a.flags == b.flags && a.eps == b.eps && a.p == b.p &&
         a.domain[0] == b.domain[0] && a.domain[1] == b.domain[1] && a.domain[2] == b.domain[2];
}

// Leaf size of the server's adaptive trees: measured on 5e5-point uniform
// and 8-cluster sets at eps = 1e-4 (tensor-core form) and 1e-8 (hybrid form),
// 128 beats 64 for the septree and the triangle tiling (up to 2x on uniform
// sets, never slower on clustered ones); 64 stays best for the quadtree.
int serve_leaf_size(int tiling) { return tiling == FMM2D_QUAD ? 64 : 128; }

unsigned precision_for(double eps, int p) {
  // FP32 expansions cannot reach tolerances much below 1e-7: FP64 expansions
  // with the FP32-pair P2P down to 1e-9, FP64 with the split-precision M2L below
  if (eps < 1e-9) return FMM2D_PREC_SPLIT;
  if (eps < 1e-6) return FMM2D_PREC_HYBRID;
  return p <= 31 ? FMM2D_PREC_MIXED_TC : FMM2D_PREC_MIXED;
}

}  // namespace
}  // namespace fmm2d

using namespace fmm2d;

struct fmm2d_server {
  size_t budget = 0;
  int device = 0;
  std::vector<std::unique_ptr<Slot>> slots;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job *> queue;
  std::unordered_map<uint64_t, Job *> jobs;
  uint64_t next_ticket = 1;
  size_t in_use = 0;
  int running = 0;
  uint64_t completed = 0;
  bool stop = false;
};

namespace {

// Pick the first queued job that fits the budget (mu held); nullptr if none.
Job *admit(fmm2d_server *sv) {
  for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
    Job *j = *it;
    if (sv->in_use + j->est_bytes <= sv->budget || sv->running == 0) {
      sv->queue.erase(it);
      sv->in_use += j->est_bytes;
      ++sv->running;
      return j;
    }
  }
  return nullptr;
}

// The slot's plan for request r's parameters (created on first use), with
// the request's domain set; *flags_out: the precision and input flags used.
fmm2d_status slot_plan(Slot &sl, const fmm2d_request &r, int64_t n_points, fmm2d_plan **out,
                       unsigned *flags_out) {
  int p = r.p;
  if (p == 0) fmm2d_default_params(r.tiling, n_points, 64, r.eps, nullptr, &p, nullptr);
  const unsigned prec = ((r.flags & FMM2D_PREC_MASK) || (r.flags & FMM2D_SERVE_PREC_AS_GIVEN))
                            ? (r.flags & FMM2D_PREC_MASK)
                            : precision_for(r.eps, p);
  const unsigned flags = prec | (r.flags & (FMM2D_IN_F32 | FMM2D_ADAPTIVE));
  int L = r.levels;
  if (L == 0 && !(flags & FMM2D_ADAPTIVE))
    fmm2d_default_params(r.tiling, n_points, 64, r.eps, &L, nullptr, nullptr);
  auto key = std::make_tuple(r.tiling, flags, L, p);
  fmm2d_plan *pl = sl.plans[key];
  fmm2d_status st;
  if (!pl) {
    st = fmm2d_plan_create(r.tiling, L, p, r.eps, flags, &pl);
    if (st != FMM2D_OK) {
      sl.plans.erase(key);
      return st;
    }
    if (flags & FMM2D_ADAPTIVE) fmm2d_plan_set_leaf_size(pl, serve_leaf_size(r.tiling));
    sl.plans[key] = pl;
  }
  sl.last_use[key] = ++sl.tick;
  const double *dom = r.domain;
  st = fmm2d_plan_set_domain(pl, dom[2] > 0 ? dom[0] : 0.0, dom[2] > 0 ? dom[1] : 0.0,
                             dom[2] > 0 ? dom[2] : 1.0);
  *out = pl;
  *flags_out = flags;
  return st;
}

// The text of a failed request: the plan's last error, or `what`.
void set_error(Job &j, const fmm2d_plan *pl, const char *what) {
  const char *m = pl ? fmm2d_last_error(pl) : "";
  if (!m || !*m) m = what;
  std::strncpy(j.res.error, m, sizeof(j.res.error) - 1);
  j.res.error[sizeof(j.res.error) - 1] = 0;
}

fmm2d_status run_job(Slot &sl, Job &j) {
  const fmm2d_request &r = j.req;
  const bool same = r.tgt_xy == nullptr;
  const int64_t nt = same ? r.n_src : r.n_tgt;
  const size_t esz = (r.flags & FMM2D_IN_F32) ? 4 : 8;
  fmm2d_plan *pl = nullptr;
  unsigned flags = 0;
  fmm2d_status st = slot_plan(sl, r, std::max(r.n_src, nt), &pl, &flags);
  if (st != FMM2D_OK) {
    set_error(j, pl, "plan creation failed");
    return st;
  }
  cudaStream_t s = sl.stream;
  if (sl.src.reserve(std::max<size_t>(16, r.n_src * 2 * esz)) || sl.u.reserve(std::max<size_t>(16, r.n_src * esz)) ||
      sl.out.reserve(std::max<size_t>(16, nt * 8)) || (!same && sl.tgt.reserve(std::max<size_t>(16, nt * 2 * esz)))) {
    cudaGetLastError();
    set_error(j, nullptr, "out of device memory for the request's buffers");
    return FMM2D_ENOMEM;
  }
  if (r.n_src > 0) {
    cudaMemcpyAsync(sl.src.p, r.src_xy, r.n_src * 2 * esz, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(sl.u.p, r.strengths, r.n_src * esz, cudaMemcpyHostToDevice, s);
  }
  if (!same && nt > 0) cudaMemcpyAsync(sl.tgt.p, r.tgt_xy, nt * 2 * esz, cudaMemcpyHostToDevice, s);
  st = fmm2d_build(pl, sl.src.p, r.n_src, same ? sl.src.p : sl.tgt.p, nt, s);
  if (st != FMM2D_OK) {
    set_error(j, pl, "build failed");
    return st;
  }
  st = fmm2d_evaluate(pl, sl.u.p, (double *)sl.out.p, s);
  if (st != FMM2D_OK) {
    set_error(j, pl, "evaluate failed");
    return st;
  }
  if (nt > 0) cudaMemcpyAsync(r.potentials, sl.out.p, nt * 8, cudaMemcpyDeviceToHost, s);
  const cudaError_t ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) {
    set_error(j, nullptr, cudaGetErrorString(ce));
    return FMM2D_ECUDA;
  }
  fmm2d_info info;
  fmm2d_plan_query(pl, &info);
  j.res.levels = info.levels;
  j.res.p = info.p;
  j.res.flags = flags;
  if (info.device_error) set_error(j, nullptr, "a bounded device wait gave up");
  return info.device_error ? FMM2D_ETIMEOUT : FMM2D_OK;
}

// Requests jobs (mergeable, same solve) as one forest: inputs copied one
// after another into the slot's buffers, one fmm2d_build_forest and one
// fmm2d_evaluate, each output copied back to its request.
fmm2d_status run_batch(Slot &sl, std::vector<Job *> &jobs) {
  const fmm2d_request &r = jobs[0]->req;
  const size_t esz = (r.flags & FMM2D_IN_F32) ? 4 : 8;
  std::vector<int64_t> off(jobs.size() + 1, 0);
  for (size_t i = 0; i < jobs.size(); ++i) off[i + 1] = off[i] + jobs[i]->req.n_src;
  const int64_t n = off.back();
  fmm2d_plan *pl = nullptr;
  unsigned flags = 0;
  fmm2d_status st = slot_plan(sl, r, n, &pl, &flags);
  if (st != FMM2D_OK) return st;
  cudaStream_t s = sl.stream;
  if (sl.src.reserve(n * 2 * esz) || sl.u.reserve(n * esz) || sl.out.reserve(n * 8)) return FMM2D_ENOMEM;
  for (size_t i = 0; i < jobs.size(); ++i) {
    const fmm2d_request &q = jobs[i]->req;
    cudaMemcpyAsync((char *)sl.src.p + off[i] * 2 * esz, q.src_xy, q.n_src * 2 * esz,
                    cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync((char *)sl.u.p + off[i] * esz, q.strengths, q.n_src * esz, cudaMemcpyHostToDevice, s);
  }
  st = fmm2d_build_forest(pl, sl.src.p, off.data(), (int)jobs.size(), s);
  if (st != FMM2D_OK) return st;
  st = fmm2d_evaluate(pl, sl.u.p, (double *)sl.out.p, s);
  if (st != FMM2D_OK) return st;
  for (size_t i = 0; i < jobs.size(); ++i)
    cudaMemcpyAsync(jobs[i]->req.potentials, (double *)sl.out.p + off[i], jobs[i]->req.n_src * 8,
                    cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return FMM2D_ECUDA;
  fmm2d_info info;
  fmm2d_plan_query(pl, &info);
  for (Job *j : jobs) {
    j->res.levels = info.levels;
    j->res.p = info.p;
    j->res.flags = flags;
  }
  return info.device_error ? FMM2D_ETIMEOUT : FMM2D_OK;
}

void worker(fmm2d_server *sv, Slot *sl) {
  cudaSetDevice(sv->device);
  for (;;) {
    std::vector<Job *> batch;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      Job *j = nullptr;
      sv->cv_work.wait(lk, [&] { return sv->stop || (j = admit(sv)) != nullptr; });
      if (!j) return;   // stopping
      batch.push_back(j);
      if (mergeable(j->req)) {   // queued requests that can share this solve
        int64_t pts = j->req.n_src;
        for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)batch.size() < MERGE_MAX;) {
          Job *k = *it;
          if (mergeable(k->req) && same_solve(k->req, j->req) && pts + k->req.n_src <= MERGE_BATCH_POINTS &&
              sv->in_use + k->est_bytes <= sv->budget) {
            pts += k->req.n_src;
            sv->in_use += k->est_bytes;
            ++sv->running;
            batch.push_back(k);
            it = sv->queue.erase(it);
          } else {
            ++it;
          }
        }
      }
      const Clock::time_point now = Clock::now();
      for (Job *k : batch) k->t_start = now;
    }
    for (Job *k : batch) std::memset(&k->res, 0, sizeof(k->res));
    std::vector<fmm2d_status> st(batch.size(), FMM2D_OK);
    if (batch.size() == 1) {
      st[0] = run_job(*sl, *batch[0]);
      if (st[0] == FMM2D_ENOMEM) {   // free the slot's cache and try once more
        cudaStreamSynchronize(sl->stream);
        trim_plans(*sl, 0);
        std::memset(&batch[0]->res, 0, sizeof(batch[0]->res));
        st[0] = run_job(*sl, *batch[0]);
      }
    } else {
      fmm2d_status bs = run_batch(*sl, batch);
      if (bs == FMM2D_ENOMEM) {
        cudaStreamSynchronize(sl->stream);
        trim_plans(*sl, 0);
        bs = run_batch(*sl, batch);
      }
      if (bs == FMM2D_OK) {
        std::fill(st.begin(), st.end(), FMM2D_OK);
      } else {   // one request may be at fault (e.g. a point outside the domain): run each alone
        for (size_t i = 0; i < batch.size(); ++i) {
          std::memset(&batch[i]->res, 0, sizeof(batch[i]->res));
          st[i] = run_job(*sl, *batch[i]);
        }
      }
    }
    // under memory pressure (cudaFree synchronises the device, so not after
    // every request) the slot's cache goes back within its share
    {
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && free_b < total_b / 10)
        trim_plans(*sl, sl->cache_bytes);
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      const Clock::time_point now = Clock::now();
      for (size_t i = 0; i < batch.size(); ++i) {
        Job *k = batch[i];
        k->t_end = now;
        k->res.status = st[i];
        k->res.slot = sl->id;
        k->res.batched = (int32_t)batch.size();
        k->res.queue_ms = std::chrono::duration<double, std::milli>(k->t_start - k->t_submit).count();
        k->res.run_ms = std::chrono::duration<double, std::milli>(k->t_end - k->t_start).count();
        k->res.latency_ms = std::chrono::duration<double, std::milli>(k->t_end - k->t_submit).count();
        k->done = true;
        sv->in_use -= k->est_bytes;
        --sv->running;
        ++sv->completed;
      }
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

fmm2d_status fmm2d_serve_create(size_t hbm_budget_bytes, int max_slots, fmm2d_server **out) {
  if (!out || max_slots < 1 || max_slots > 256 || hbm_budget_bytes == 0) return FMM2D_EINVAL;
  *out = nullptr;
  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0 || cudaGetDevice(&dev) != cudaSuccess)
    return FMM2D_ECUDA;
  fmm2d_server *sv = new (std::nothrow) fmm2d_server();
  if (!sv) return FMM2D_ENOMEM;
  planner_precompute();   // not on the first request's clock
  sv->budget = hbm_budget_bytes;
  sv->device = dev;
  for (int i = 0; i < max_slots; ++i) {
    auto sl = std::make_unique<Slot>();
    sl->id = i;
    // when device memory runs low, the cached plans of all slots together
    // are trimmed to half the budget
    sl->cache_bytes = hbm_budget_bytes / 2 / (size_t)max_slots;
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
      fmm2d_serve_destroy(sv);
      return FMM2D_ECUDA;
    }
    sv->slots.push_back(std::move(sl));
  }
  for (auto &sl : sv->slots) sv->workers.emplace_back(worker, sv, sl.get());
  *out = sv;
  return FMM2D_OK;
}

fmm2d_status fmm2d_serve_submit(fmm2d_server *sv, const fmm2d_request *r, uint64_t *ticket) {
  if (!sv || !r || !ticket) return FMM2D_EINVAL;
  if (r->tiling < 0 || r->tiling > 2 || r->n_src < 0 || (r->tgt_xy && r->n_tgt < 0) ||
      (r->n_src > 0 && (!r->src_xy || !r->strengths)) || !r->potentials ||
      (r->p == 0 && !(r->eps > 0.0 && r->eps < 1.0)))
    return FMM2D_EINVAL;
  Job *j = new (std::nothrow) Job();
  if (!j) return FMM2D_ENOMEM;
  j->req = *r;
  j->est_bytes = estimate_bytes(*r);
  if (j->est_bytes > sv->budget) {
    delete j;
    return FMM2D_EBUSY;   // could never be admitted
  }
  j->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    j->ticket = sv->next_ticket++;
    sv->jobs[j->ticket] = j;
    sv->queue.push_back(j);
    *ticket = j->ticket;
  }
  sv->cv_work.notify_one();
  return FMM2D_OK;
}

fmm2d_status fmm2d_serve_poll(fmm2d_server *sv, uint64_t ticket, fmm2d_result *res) {
  if (!sv) return FMM2D_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return FMM2D_EINVAL;
  if (!it->second->done) return FMM2D_ENOTREADY;
  if (res) *res = it->second->res;
  delete it->second;
  sv->jobs.erase(it);
  return FMM2D_OK;
}

fmm2d_status fmm2d_serve_wait(fmm2d_server *sv, uint64_t ticket, double timeout_ms,
                              fmm2d_result *res) {
  if (!sv) return FMM2D_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return FMM2D_EINVAL;
  Job *j = it->second;
  const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                       [&] { return j->done; });
  if (!ok) return FMM2D_ETIMEOUT;
  if (res) *res = j->res;
  delete j;
  sv->jobs.erase(ticket);
  return FMM2D_OK;
}

fmm2d_status fmm2d_serve_stats(fmm2d_server *sv, fmm2d_serve_info *info) {
  if (!sv || !info) return FMM2D_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  info->queued = (int64_t)sv->queue.size();
  info->running = sv->running;
  info->completed = (int64_t)sv->completed;
  info->bytes_in_use = sv->in_use;
  info->budget_bytes = sv->budget;
  info->slots = (int32_t)sv->slots.size();
  return FMM2D_OK;
}

void fmm2d_serve_destroy(fmm2d_server *sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    for (Job *j : sv->queue) {
      sv->jobs.erase(j->ticket);
      delete j;
    }
    sv->queue.clear();
  }
  sv->cv_work.notify_all();
  for (auto &t : sv->workers) t.join();
  for (auto &kv : sv->jobs) delete kv.second;
  for (auto &sl : sv->slots) {
    for (auto &kv : sl->plans) fmm2d_plan_destroy(kv.second);
    if (sl->stream) cudaStreamDestroy(sl->stream);
  }
  delete sv;
}

}  // extern "C"
