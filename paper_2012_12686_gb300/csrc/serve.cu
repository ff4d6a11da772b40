// Serving loop: continuous batching of loss/gradient requests over several CUDA streams.
//
// A request is queued by adorym_submit.  A worker thread admits queued requests whenever a slot
// (stream) is free and the request's workspace fits the footprint budget; the workspace is carved
// from one device arena with a first-fit allocator.  Admission is in arrival order, except that
// when the oldest request does not fit, later requests that do fit may go ahead of it -- at most
// kMaxOvertakes admissions past one waiting request, after which nothing overtakes it, so a large
// request is never starved.  Half of the slots (rounded down) are short-request slots: their
// streams have the highest scheduling priority and only requests with a small amount of work
// (kShortWork) are admitted to them, so a short request neither waits for a slot behind long
// ones nor waits on the device for long requests' queued thread blocks.  Long requests take the
// other slots, at normal priority; short ones take any free slot, short-request slots first.
// Admitted requests are recorded by stream capture into a CUDA graph
// and launched; the executable graph of each (slot, problem shape) is kept and updated in place
// (cudaGraphExecUpdate) for the next request of that shape, so steady-state launches cost one
// graph launch.  Completion is event driven: each slot has a waiter thread blocked in
// cudaEventSynchronize on the slot's blocking-sync event, which retires the request and wakes the
// admission worker and adorym_poll (no polling loop).  No device-side waiting is involved: a
// request that never completes shows up as ETIMEDOUT on the host, never as a spinning kernel.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "engine.h"

namespace adorym {

struct Arena {
  // first-fit free list over [0, cap) of one device allocation
  char* base = nullptr;
  size_t cap = 0;
  std::map<size_t, size_t> free_;   // offset -> size
  size_t used = 0;
  bool init(size_t bytes) {
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
      cudaGetLastError();
      base = nullptr;
      return false;
    }
    cap = bytes;
    free_.clear();
    free_[0] = bytes;
    used = 0;
    return true;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, o2 = it->first + bytes;
        free_.erase(it);
        if (rest) free_[o2] = rest;
        used += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    used -= bytes;
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
};

using Clock = std::chrono::steady_clock;

struct Ticket {
  adorym_request req{};
  Plan plan;
  bool is_short = false;  // work below kShortWork: may use the high-priority slots
  int state = 0;          // 0 queued, 1 running, 2 done
  int rc = ADORYM_OK;
  int slot = -1;
  size_t ws_off = 0;
  bool waited = false;
  int overtaken = 0;      // admissions of later requests while this one waited at the head
  Clock::time_point t_submit, t_admit, t_done;
};

struct Slot {
  bool fast = false;      // short-request slot: highest-priority stream, short requests only
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int* status = nullptr;  // mapped pinned host word: the running ticket's status (kernels write it
                          // only on bad input; zeroed by the host before each launch)
  int* status_dev = nullptr;
  uint64_t ticket = 0;    // 0 = free
  bool launched = false;  // the ticket's graph and completion event are enqueued (waiter may wait)
  std::map<std::string, cudaGraphExec_t> graphs;
  std::thread waiter;     // blocks on `done` and retires the slot's ticket
};

// admissions of later requests allowed past a request that waits at the head of the queue
constexpr int kMaxOvertakes = 8;

// A request is short when its work, B * M * L * N^2 pixel-slices (doubled for the two-pass path at
// N >= 256, whose fields make HBM round trips), is at most 2^26: about a millisecond of device time
// on this part (a 128 x 128 batch of 4096 position-slices is 2^26 and takes ~1.4 ms).
constexpr double kShortWork = 67108864.0;
static bool short_request(const adorym_problem& p) {
  const double w = (double)p.B * p.M * p.L * (double)p.N * p.N * (two_pass(p.N) ? 2.0 : 1.0);
  return w <= kShortWork;
}

struct Serve {
  int nslots = 4;
  size_t budget = 0;      // bytes; 0 = arena default
  Arena arena;
  std::vector<Slot> slots;
  std::deque<uint64_t> queue;
  std::map<uint64_t, Ticket> tickets;
  uint64_t next = 1;
  uint64_t completed = 0, waits = 0;
  bool stop = false;
  uint64_t epoch = 0;     // bumped by every submission, completion and cancellation
  Clock::time_point t_start = Clock::now();
  std::thread worker;
  std::condition_variable cv_work, cv_done, cv_slot;
};

static std::string shape_key(const Plan& pl, const adorym_request& r) {
  char buf[320];
  const adorym_problem& p = pl.p;
  snprintf(buf, sizeof buf, "%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d%d%d%d|%d%d%d", p.N, p.L, p.M, p.B, p.Ly, p.Lx,
           p.Lz, p.farfield, p.n_dist, p.loss, p.tomo, pl.cp, pl.ncp, r.g_delta != nullptr, r.g_probe != nullptr,
           r.g_pos != nullptr, r.loss_out != nullptr, r.I_out != nullptr, 0, 0);
  return std::string(buf);
}

// launch one admitted ticket on its slot (ctx->mu held)
static int launch_ticket(adorym_ctx* ctx, Serve& S, uint64_t id) {
  Ticket& t = S.tickets[id];
  Slot& sl = S.slots[t.slot];
  const adorym_request& r = t.req;
  auto it = ctx->objects.find(r.obj_id);
  if (it == ctx->objects.end()) {
    ctx->err = "unknown object id";
    return ADORYM_ENOENT;
  }
  Tables tab;
  int rc = get_tables(ctx, r.problem, &tab);
  if (rc) return rc;
  CallPtrs c;
  c.probe = reinterpret_cast<const float2*>(r.probe);
  c.pos = r.pos;
  c.I_meas = r.I_meas;
  c.loss = r.loss_out;
  c.gd = r.g_delta;
  c.gb = r.g_beta;
  c.g_probe = reinterpret_cast<float2*>(r.g_probe);
  c.g_pos = r.g_pos;
  c.I_out = r.I_out;
  std::string err;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    ctx->err = std::string("begin capture: ") + cudaGetErrorString(e);
    return ADORYM_EDEVICE;
  }
  c.status = sl.status_dev;
  rc = enqueue(t.plan, it->second, tab, c, S.arena.base + t.ws_off, sl.stream, &err);
  e = cudaStreamEndCapture(sl.stream, &g);
  if (rc || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    ctx->err = rc ? err : std::string("end capture: ") + cudaGetErrorString(e);
    return rc ? rc : ADORYM_EDEVICE;
  }
  const std::string key = shape_key(t.plan, r);
  auto git = sl.graphs.find(key);
  bool ok = false;
  if (git != sl.graphs.end()) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(git->second, g, &info) == cudaSuccess) ok = true;
    else {
      cudaGetLastError();
      cudaGraphExecDestroy(git->second);
      sl.graphs.erase(git);
    }
  }
  if (!ok) {
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      ctx->err = std::string("graph instantiate: ") + cudaGetErrorString(e);
      return ADORYM_EDEVICE;
    }
    sl.graphs[key] = ex;
  }
  cudaGraphDestroy(g);
  if (sl.status) *sl.status = 0;   // the slot's previous ticket has finished
  e = cudaGraphLaunch(sl.graphs[key], sl.stream);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
  if (e != cudaSuccess) {
    ctx->err = std::string("graph launch: ") + cudaGetErrorString(e);
    return ADORYM_EDEVICE;
  }
  sl.launched = true;
  S.cv_slot.notify_all();
  return ADORYM_OK;
}

static void finish(Serve& S, uint64_t id, int rc) {
  Ticket& t = S.tickets[id];
  if (t.slot >= 0) {
    S.slots[t.slot].ticket = 0;
    S.slots[t.slot].launched = false;
    S.arena.release(t.ws_off, t.plan.total);
  }
  t.state = 2;
  t.rc = rc;
  t.t_done = Clock::now();
  S.completed++;
  S.epoch++;
}

// waiter of slot i: sleeps until the slot's ticket is launched, blocks (without the context lock)
// until its completion event, then retires it and wakes the admission worker and pollers
static void slot_waiter(adorym_ctx* ctx, int i) {
  Serve& S = *ctx->serve;
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(ctx->mu);
  for (;;) {
    S.cv_slot.wait(lk, [&] { return S.stop || (S.slots[i].ticket && S.slots[i].launched); });
    if (S.stop && !(S.slots[i].ticket && S.slots[i].launched)) return;
    Slot& sl = S.slots[i];
    const uint64_t id = sl.ticket;
    const cudaEvent_t ev = sl.done;
    lk.unlock();
    const cudaError_t q = cudaEventSynchronize(ev);
    lk.lock();
    const bool bad_data = q == cudaSuccess && sl.status && *sl.status != 0;
    if (q != cudaSuccess) {
      cudaGetLastError();
      ctx->err = std::string("request failed: ") + cudaGetErrorString(q);
    }
    if (bad_data) ctx->err = std::string("request failed: ") + status_message(*sl.status);
    finish(S, id, q != cudaSuccess ? ADORYM_EDEVICE : bad_data ? ADORYM_EDATA : ADORYM_OK);
    S.cv_done.notify_all();
    S.cv_work.notify_all();
  }
}

// a free slot for ticket t: short requests take a short-request slot first, then a normal one;
// long requests only normal slots (-1: none)
static int free_slot_for(const Serve& S, const Ticket& t) {
  int normal = -1;
  for (int i = 0; i < (int)S.slots.size(); ++i) {
    if (S.slots[i].ticket) continue;
    if (S.slots[i].fast) {
      if (t.is_short) return i;
    } else if (normal < 0) {
      normal = i;
    }
  }
  return normal;
}

// admit one queued request if one may go now: the head if a slot and memory are free for it;
// else, unless the head has been overtaken kMaxOvertakes times already, the oldest later request
// for which they are.  A later request that takes a short-request slot while a long head waits
// for a normal slot does not compete with it: it is always allowed and does not count as an
// overtake (a long request can never use that slot).
static bool admit_one(adorym_ctx* ctx, Serve& S) {
  bool head_closed = false;      // the head has been overtaken kMaxOvertakes times
  bool head_wants_slot = false;  // the head is long and waits for a normal slot (memory not tried)
  for (size_t i = 0; i < S.queue.size(); ++i) {
    const uint64_t id = S.queue[i];
    Ticket& t = S.tickets[id];
    const int slot = free_slot_for(S, t);
    const bool beside_head = i > 0 && head_wants_slot && slot >= 0 && S.slots[slot].fast;
    size_t off = 0;
    if (slot < 0 || (head_closed && !beside_head) || !S.arena.alloc(t.plan.total, &off)) {
      if (!t.waited) S.waits++;
      t.waited = true;
      if (i == 0) {
        head_closed = t.overtaken >= kMaxOvertakes;
        head_wants_slot = slot < 0 && !t.is_short;
      }
      continue;
    }
    if (i > 0 && !beside_head) S.tickets[S.queue.front()].overtaken++;
    S.queue.erase(S.queue.begin() + (std::ptrdiff_t)i);
    t.slot = slot;
    t.ws_off = off;
    t.state = 1;
    t.t_admit = Clock::now();
    S.slots[slot].ticket = id;
    S.slots[slot].launched = false;
    const int rc = launch_ticket(ctx, S, id);
    if (rc) {
      finish(S, id, rc);
      S.cv_done.notify_all();
    }
    return true;
  }
  return false;
}

static void worker_main(adorym_ctx* ctx) {
  Serve& S = *ctx->serve;
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(ctx->mu);
  uint64_t seen = ~(uint64_t)0;
  while (!S.stop) {
    if (seen != S.epoch) {
      seen = S.epoch;
      // admit while a queued request may go
      while (!S.queue.empty() && admit_one(ctx, S)) {
      }
    }
    S.cv_work.wait(lk, [&] { return S.stop || S.epoch != seen; });
  }
}

// create the serving state of ctx (ctx->mu held): arena, slots, worker and slot waiters
static int serve_create(adorym_ctx* ctx, int nslots, size_t budget_bytes) {
  auto S = std::make_unique<Serve>();
  S->nslots = nslots;
  S->budget = budget_bytes;
  size_t freeb = 0, totalb = 0;
  cudaSetDevice(ctx->device);
  cudaMemGetInfo(&freeb, &totalb);
  const size_t bytes = budget_bytes ? budget_bytes : std::min(freeb / 2, (size_t)8 << 30);
  if (!S->arena.init(bytes)) {
    ctx->err = "serving arena allocation failed";
    return ADORYM_ENOMEM;
  }
  S->slots.resize(nslots);
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);   // (least, greatest)
  for (int i = 0; i < nslots; ++i) {
    Slot& sl = S->slots[i];
    sl.fast = i < nslots / 2;
    cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, sl.fast ? prio_hi : prio_lo);
    // blocking sync: the slot's waiter thread sleeps in cudaEventSynchronize instead of spinning
    cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming | cudaEventBlockingSync);
    void* h = nullptr;
    void* hd = nullptr;
    if (cudaHostAlloc(&h, sizeof(int), cudaHostAllocMapped) == cudaSuccess &&
        cudaHostGetDevicePointer(&hd, h, 0) == cudaSuccess) {
      sl.status = static_cast<int*>(h);
      sl.status_dev = static_cast<int*>(hd);
      *sl.status = 0;
    } else {
      cudaGetLastError();
    }
  }
  ctx->serve = S.release();
  ctx->serve->worker = std::thread(worker_main, ctx);
  for (int i = 0; i < nslots; ++i) ctx->serve->slots[i].waiter = std::thread(slot_waiter, ctx, i);
  return ADORYM_OK;
}

static int serve_start(adorym_ctx* ctx) {
  if (ctx->serve) return ADORYM_OK;
  return serve_create(ctx, 4, 0);
}

void serve_shutdown(adorym_ctx* ctx) {
  if (!ctx->serve) return;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->serve->stop = true;
  }
  ctx->serve->cv_work.notify_all();
  ctx->serve->cv_slot.notify_all();
  if (ctx->serve->worker.joinable()) ctx->serve->worker.join();
  Serve& S = *ctx->serve;
  for (auto& sl : S.slots)   // a waiter retires its launched ticket (the GPU work completes) first
    if (sl.waiter.joinable()) sl.waiter.join();
  for (auto& sl : S.slots) {
    cudaStreamSynchronize(sl.stream);
    for (auto& kv : sl.graphs) cudaGraphExecDestroy(kv.second);
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
    if (sl.status) cudaFreeHost(sl.status);
  }
  if (S.arena.base) cudaFree(S.arena.base);
  delete ctx->serve;
  ctx->serve = nullptr;
}

}  // namespace adorym

using namespace adorym;

extern "C" {

int adorym_serve_config(adorym_ctx* ctx, int slots, uint64_t budget_bytes) {
  if (!ctx) return ADORYM_EINVAL;
  if (slots < 1 || slots > 16) {
    ctx->err = "slots must be in 1..16";
    return ADORYM_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serve) {
      for (auto& kv : ctx->serve->tickets)
        if (kv.second.state != 2) {
          ctx->err = "requests in flight";
          return ADORYM_EINVAL;
        }
    }
  }
  serve_shutdown(ctx);
  std::lock_guard<std::mutex> lk(ctx->mu);
  return serve_create(ctx, slots, budget_bytes);
}

int adorym_submit(adorym_ctx* ctx, const adorym_request* req, uint64_t* ticket) {
  if (!ctx || !req || !ticket) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->serve) {
    int rc = serve_start(ctx);
    if (rc) return rc;
  }
  Serve& S = *ctx->serve;
  const adorym_request& r = *req;
  if (!r.probe || !r.pos || !r.I_meas) {
    ctx->err = "probe, pos and I_meas are required";
    return ADORYM_EINVAL;
  }
  const void* ptrs[] = {r.probe, r.pos, r.I_meas, r.loss_out, r.g_delta, r.g_beta, r.g_probe, r.g_pos, r.I_out};
  for (const void* q : ptrs) {
    if (!q) continue;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      ctx->err = "serving requests take device pointers only";
      return ADORYM_EINVAL;
    }
  }
  if ((r.g_delta == nullptr) != (r.g_beta == nullptr)) {
    ctx->err = "g_delta and g_beta must both be given or both be NULL";
    return ADORYM_EINVAL;
  }
  auto it = ctx->objects.find(r.obj_id);
  if (it == ctx->objects.end()) {
    ctx->err = "unknown object id";
    return ADORYM_ENOENT;
  }
  const Object& obj = it->second;
  if (obj.Lz != r.problem.Lz || obj.Ly != r.problem.Ly || obj.Lx != r.problem.Lx) {
    ctx->err = "problem Lz/Ly/Lx differ from the registered object";
    return ADORYM_EINVAL;
  }
  Ticket t;
  t.req = r;
  const int grads = (r.g_delta ? 1 : 0) | (r.g_probe ? 2 : 0) | (r.g_pos ? 4 : 0);
  const char* msg = "";
  int rc = make_plan(r.problem, true, grads, r.loss_out != nullptr, &t.plan, &msg);
  if (rc) {
    ctx->err = msg;
    return rc;
  }
  if (t.plan.total > S.arena.cap) {
    ctx->err = "request workspace exceeds the serving footprint budget";
    return ADORYM_ENOMEM;
  }
  // set kernel attributes and build tables outside of any capture
  Tables tab;
  if ((rc = get_tables(ctx, r.problem, &tab))) return rc;
  if ((rc = prepare_kernels(r.problem, &msg))) {
    ctx->err = msg;
    return rc;
  }
  const uint64_t id = S.next++;
  t.is_short = short_request(r.problem);
  t.t_submit = Clock::now();
  S.tickets[id] = t;
  S.queue.push_back(id);
  *ticket = id;
  S.epoch++;
  S.cv_work.notify_all();
  return ADORYM_OK;
}

int adorym_poll(adorym_ctx* ctx, uint64_t ticket, int64_t timeout_us) {
  return adorym_poll_times(ctx, ticket, timeout_us, nullptr);
}

int adorym_poll_times(adorym_ctx* ctx, uint64_t ticket, int64_t timeout_us, double* times_us) {
  if (!ctx) return ADORYM_EINVAL;
  std::unique_lock<std::mutex> lk(ctx->mu);
  if (!ctx->serve) return ADORYM_ENOENT;
  Serve& S = *ctx->serve;
  auto it = S.tickets.find(ticket);
  if (it == S.tickets.end()) return ADORYM_ENOENT;
  auto ready = [&] { return S.tickets[ticket].state == 2; };
  if (timeout_us < 0) S.cv_done.wait(lk, ready);
  else if (timeout_us > 0) S.cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
  if (!ready()) return ADORYM_ETIMEDOUT;
  const Ticket& t = S.tickets[ticket];
  const int rc = t.rc;
  if (times_us) {
    const bool ran = t.slot >= 0;
    auto us = [](Clock::duration d) { return std::chrono::duration<double, std::micro>(d).count(); };
    times_us[0] = us((ran ? t.t_admit : t.t_done) - t.t_submit);   // waiting for admission
    times_us[1] = ran ? us(t.t_done - t.t_admit) : 0.0;             // admitted until retired
    times_us[2] = ran ? us(t.t_admit - S.t_start) : -1.0;           // admission instant
  }
  S.tickets.erase(ticket);
  return rc;
}

int adorym_cancel(adorym_ctx* ctx, uint64_t ticket) {
  if (!ctx) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->serve) return ADORYM_ENOENT;
  Serve& S = *ctx->serve;
  auto it = S.tickets.find(ticket);
  if (it == S.tickets.end()) return ADORYM_ENOENT;
  if (it->second.state != 0) {
    ctx->err = "request already admitted or finished";
    return ADORYM_EINVAL;
  }
  for (auto q = S.queue.begin(); q != S.queue.end(); ++q)
    if (*q == ticket) {
      S.queue.erase(q);
      break;
    }
  it->second.state = 2;
  it->second.rc = ADORYM_ECANCELED;
  it->second.t_done = Clock::now();
  S.epoch++;
  S.cv_done.notify_all();
  S.cv_work.notify_all();   // the request behind it may now fit
  return ADORYM_OK;
}

int adorym_serve_stats(adorym_ctx* ctx, uint64_t* completed, uint64_t* admission_waits) {
  if (!ctx) return ADORYM_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (completed) *completed = ctx->serve ? ctx->serve->completed : 0;
  if (admission_waits) *admission_waits = ctx->serve ? ctx->serve->waits : 0;
  return ADORYM_OK;
}

}  // extern "C"
