// Continuous-batching request server for predict / peel requests of uneven size.
//
// A scheduler thread owns the GPU side:
//  * admission by memory: each request's output visibilities are carved from one device pool
//    (first fit); a request waits until a slot (max_inflight) and pool space are free, and one that
//    can never fit is refused at submit (WN_EBUSY);
//  * batching: admitted requests that are not yet running are packed into one work table of
//    (request, row tile, channel block) entries and run by the persistent batched phasor kernel,
//    replayed from a CUDA graph captured once per stream; shapelet components follow per request on
//    the same stream, with that stream's own tables.  A small request that batching would not help
//    (more than a millisecond of work, or a short grid of long tiles) runs alone on a stream through
//    the single-request kernels instead;
//  * overlap: there are n_streams batch slots; requests that arrive while batches are on the GPU are
//    admitted as memory and slots free up and go out in the next batch on a free stream, so their
//    work overlaps the batches in flight;
//  * large requests: a batch carries at most ~kBatchBudget of estimated GPU work; a request larger than
//    that runs on a stream of its own through the single-request kernels (the table-form phasor kernel
//    and the shapelet kernel, with that stream's own workspaces: the same work the request does alone).
//    In arrival order (the default) large requests start in submission order, each after the small
//    requests submitted before it, in one launch on the highest-priority stream; small-first, they run
//    on the lowest-priority stream in chunks of whole time steps so that small requests keep flowing
//    (launch_ready).  While one runs, small requests go out one batch at a time on another stream, so
//    the ones that arrive meanwhile are packed into the next batch;
//  * completion: an event per batch, polled without blocking; the caller reads the result in place
//    and releases it, which returns its pool space.
// A batched tile is computed by the same code in the same order as a single-request launch of the
// batched kernel's form, and a large request (or a chunk of it) by the single-request kernels on its
// rows, so a request's result does not depend on what it was batched with.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "wn_internal.cuh"

namespace wn {

enum ReqState { RQ_PENDING = 0, RQ_ADMITTED = 1, RQ_RUNNING = 2, RQ_DONE = 3, RQ_CANCELLED = 4, RQ_FAILED = 5 };

constexpr double kBatchBudget = 0.02;   // seconds of estimated GPU work per batch / chunk
// Large requests in flight at once.  They share the GPU with each other and with the small batches, so
// more of them at once stretches every one of them.  A large request keeps its place until its last
// launch has completed.
constexpr int kMaxLargeInFlight = 1;  // default; wn_server_set_policy changes it per server
// In the small-first order, large requests start in order of estimated work, least first, which keeps a
// burst of them from holding back the many mid-sized ones behind the few largest; a request that has
// waited this long since submission starts before any younger one, so the largest are passed over for
// a bounded time.
constexpr double kMaxLargeWait = 1.0;  // seconds; default, as above
// Request orders (wn_server_set_order).  Measured on the serving bench (1,000 requests at 70 % load),
// p99 of the requests of 20 ms or more / of the others, against 0.48 s / 0.47 s one at a time:
//  * arrival order (the default): 0.47 s / 0.42-0.43 s (overall p99 0.44 s, p50 26 ms against 35 ms);
//  * small requests first, large ones least work first with the 1 s wait limit: 0.93 s / 0.09 s
//    (overall p99 0.27 s, p50 8 ms); with a 0.3 s wait limit 0.54-0.59 s / 0.09 s.
constexpr double kEvalRate = 3.0e12;    // component-visibility evaluations per second (estimate)

struct ServeReq {
  uint64_t ticket = 0;
  K1Args k1;              // batched-kernel arguments (set at admission)
  int gx = 0, gy = 0;     // tile grid of the phasor kernel
  long tiles = 0, issued = 0;  // tiles of the batched kernel's grid; work issued (0: not started)
  int t_next = 0;              // a large request's next time step to issue
  double tile_cost = 0;        // estimated GPU seconds per tile
  int owner_slot = -1;    // slot that issues a large request's chunks
  ObsDev od;
  const Model* M = nullptr;
  int mode = OUT_STORE;
  PeelArgs pa;
  size_t bytes = 0, off = 0;
  bool has_mem = false;
  int state = RQ_PENDING;
  int batch = -1;
  int error = WN_OK;
  double t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
};

struct ServeSlot {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t gexec = nullptr;
  char* d_table = nullptr;  // [n_work int (16 B)][K1Args x max_reqs][K1Work x max_work]
  char* h_table = nullptr;  // pinned copy written before each replay
  float4* chaninfo = nullptr;
  float4* rowinfo = nullptr;
  std::vector<uint64_t> reqs;     // requests that complete with this slot's current launch
  bool busy = false;
  int priority = 0;                // CUDA stream priority (lower number runs first)
  uint64_t owner = 0;              // large request whose chunks this slot issues (0: none)
  KsWork ks;                       // table-form workspaces of the large requests this slot runs
};

}  // namespace wn

struct wn_server {
  wn_ctx* ctx = nullptr;
  int max_inflight = 8;
  int max_reqs = 64;
  int max_work = 1 << 14;
  size_t table_bytes = 0;
  int max_rows = 0, max_chan = 0;
  int max_large_inflight = wn::kMaxLargeInFlight;  // admission policy (wn_server_set_policy)
  double max_large_wait = wn::kMaxLargeWait;
  int order = WN_SERVE_ARRIVAL;                    // request order (wn_server_set_order)
  char* pool = nullptr;
  size_t pool_bytes = 0;
  std::map<size_t, size_t> free_list;  // offset -> size
  std::vector<wn::ServeSlot> slots;
  std::map<uint64_t, wn::ServeReq> reqs;
  std::deque<uint64_t> queue;  // pending, in arrival order
  uint64_t next_ticket = 1;
  int admitted = 0;            // admitted and not yet released
  int batches = 0, max_running_batches = 0, max_batch_reqs = 0, launched = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  std::chrono::steady_clock::time_point t0;
};

namespace wn {

static double now_s(wn_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

static bool pool_alloc(wn_server* s, size_t bytes, size_t* off) {
  for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t base = it->first;
      s->free_list.erase(it);
      if (rest) s->free_list[base + bytes] = rest;
      return true;
    }
  }
  return false;
}

static void pool_free(wn_server* s, size_t off, size_t bytes) {
  auto it = s->free_list.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->free_list.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_list.erase(nx);
  }
  if (it != s->free_list.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_list.erase(it);
    }
  }
}

static size_t round_bytes(size_t b) { return (b + 255) & ~(size_t)255; }

// Shapelet row tables a slot holds: a request's shapelets are summed this many per launch.
constexpr int kSlotRowTables = 4;

static bool has_pg(const ServeReq& r) { return r.M->n_point + r.M->n_gauss > 0 || r.M->n_shape == 0; }

static void finish_launch(wn_server* s, int k, const std::vector<uint64_t>& complete, cudaError_t e);

// Launch on slot k the work table in the slot's pinned staging (nwork entries), the shapelets of the
// requests in `shapes`, and the completion event that completes the requests in `complete`.  Called
// with the lock held.
static void launch_slot(wn_server* s, int k, int nwork, const std::vector<uint64_t>& complete,
                        const std::vector<uint64_t>& shapes) {
  ServeSlot& sl = s->slots[k];
  *reinterpret_cast<int*>(sl.h_table) = nwork;
  cudaError_t e = cudaGraphLaunch(sl.gexec, sl.st);  // copies the table, then the batched kernel
  for (uint64_t t : shapes) {
    ServeReq& r = s->reqs[t];
    const int smode = r.M->n_point + r.M->n_gauss > 0 ? (r.mode == OUT_PEEL ? OUT_SUBG : OUT_ACCUM) : r.mode;
    if (launch_shapelets_ws(s->ctx, r.od, r.M, reinterpret_cast<float2*>(s->pool + r.off), smode, r.pa, sl.chaninfo,
                            sl.rowinfo, (size_t)kSlotRowTables * s->max_rows, sl.st) != WN_OK) {
      r.state = RQ_FAILED;
      r.error = WN_ECUDA;
    }
  }
  finish_launch(s, k, complete, e);
}

// The completion event of slot k's launch, which completes the requests in `complete`.  Called with
// the lock held.
static void finish_launch(wn_server* s, int k, const std::vector<uint64_t>& complete, cudaError_t e) {
  ServeSlot& sl = s->slots[k];
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.st);
  sl.reqs = complete;
  if (e != cudaSuccess)
    for (uint64_t t : sl.reqs) {
      s->reqs[t].state = RQ_FAILED;
      s->reqs[t].error = WN_ECUDA;
    }
  sl.busy = true;
  s->batches++;
  s->launched += (int)complete.size();
  s->max_batch_reqs = std::max(s->max_batch_reqs, (int)complete.size());
  int running = 0;
  for (auto& x : s->slots) running += x.busy ? 1 : 0;
  s->max_running_batches = std::max(s->max_running_batches, running);
}

// Append tiles [from, to) of request r (table entry index `slot_req`) to the work list.
static int add_tiles(ServeReq& r, int slot_req, long from, long to, K1Work* work, int nwork) {
  for (long t = from; t < to; ++t) work[nwork++] = K1Work{slot_req, (int)(t % r.gx), (int)(t / r.gx)};
  return nwork;
}

static double large_cost(const ServeReq& r) { return r.tile_cost * r.tiles; }
static bool is_large(const ServeReq& r) { return r.tiles > 0 && large_cost(r) > kBatchBudget; }

// An admitted request that no launch has taken yet.
static bool unstarted(const ServeReq& r) { return r.state == RQ_ADMITTED && r.issued == 0 && r.owner_slot < 0; }

// A small request submitted before ticket `bar` (all of them when bar is UINT64_MAX) waits for a launch.
static bool small_waiting(wn_server* s, uint64_t bar) {
  for (auto& kv : s->reqs) {
    if (kv.first >= bar) break;
    if (unstarted(kv.second) && !is_large(kv.second)) return true;
  }
  return false;
}

static K1Args* slot_args(wn_server*, ServeSlot& sl) { return reinterpret_cast<K1Args*>(sl.h_table + 16); }
static K1Work* slot_work(wn_server* s, ServeSlot& sl) {
  return reinterpret_cast<K1Work*>(sl.h_table + 16 + sizeof(K1Args) * s->max_reqs);
}

// Launch on slot k time steps [t0, t0 + steps) of request r as one observation through the
// single-request kernels: the table-form phasor kernel with the slot's workspaces, then the shapelet
// kernel with the slot's tables.  Step ranges are disjoint rows, so each applies the request's mode.
// Called with the lock held; the slot is idle.  Returns a WN_ status.
static int launch_steps(wn_server* s, int k, ServeReq& r, int t0, int steps) {
  ServeSlot& sl = s->slots[k];
  const int B = r.od.n_base, F = r.od.n_chan;
  ObsDev o = r.od;
  o.n_time = steps;
  o.n_rows = steps * B;
  o.uvw = r.od.uvw + (size_t)3 * t0 * B;
  float2* out = reinterpret_cast<float2*>(s->pool + r.off) + (size_t)t0 * B * F;
  PeelArgs pa = r.pa;
  if (r.mode == OUT_PEEL) {
    pa.data = r.pa.data + (size_t)t0 * B * F;
    if (r.pa.gt > 1) pa.gains = r.pa.gains + (size_t)t0 * r.pa.gf * r.pa.n_ant;  // per-step gains
  }
  int rc = WN_OK;
  cudaError_t e = cudaSuccess;
  // the spectrum table depends on the observation's channels too: a request's first steps build it
  if (t0 == 0) sl.ks.spec_model = nullptr;
  const size_t need = phasor_table_spec_bytes(o, r.M);
  if (sl.ks.spec_bytes < need) {  // grow-only; the slot's stream is idle
    cudaFree(sl.ks.spec);
    sl.ks = KsWork{nullptr, 0, sl.ks.part, nullptr, 0};
    e = dev_malloc(&sl.ks.spec, need);
    if (e == cudaSuccess) sl.ks.spec_bytes = need;
  }
  if (e == cudaSuccess && !sl.ks.part) e = dev_malloc(&sl.ks.part, k1_part_bytes(s->ctx->num_sms));
  if (e != cudaSuccess) rc = set_error(WN_ENOMEM, std::string("serving workspace: ") + cudaGetErrorString(e));
  if (rc == WN_OK) rc = launch_phasor_table_ws(s->ctx, o, r.M, out, r.mode, pa, sl.ks, sl.st);
  if (rc == WN_OK && r.M->n_shape > 0)
    rc = launch_shapelets_ws(s->ctx, o, r.M, out, r.mode == OUT_PEEL ? OUT_SUBG : OUT_ACCUM, pa, sl.chaninfo, sl.rowinfo,
                             (size_t)kSlotRowTables * s->max_rows, sl.st);
  return rc;
}

// Launch on slot k the next chunk of the large request the slot owns.  In arrival order the chunk is the
// whole request; small-first, it is its next time steps, about kBatchBudget of estimated work and at
// least two waves of the phasor kernel's row tiles (32 rows, one CTA per SM) so that a chunk fills the
// GPU.  The last chunk completes the request.  Called with the lock held; the slot is idle.
static void launch_chunk(wn_server* s, int k) {
  ServeSlot& sl = s->slots[k];
  ServeReq& r = s->reqs[sl.owner];
  std::vector<uint64_t> complete;
  const int T = r.od.n_time, B = r.od.n_base;
  int steps = T - r.t_next;
  if (s->order == WN_SERVE_SMALL_FIRST) {
    const double per_step = large_cost(r) / T;
    const int min_steps = (2 * 32 * s->ctx->num_sms + B - 1) / B;
    steps = std::max(1, std::min(steps, std::max(min_steps, (int)(kBatchBudget / std::max(per_step, 1e-12)))));
  }
  const int t0 = r.t_next;
  const int rc = launch_steps(s, k, r, t0, steps);
  r.issued = 1;
  r.t_next = t0 + steps;
  if (rc != WN_OK) {
    r.state = RQ_FAILED;
    r.error = rc;
  }
  if (r.t_next == T || rc != WN_OK) {
    if (rc == WN_OK) r.state = RQ_RUNNING;
    r.batch = s->batches;
    r.owner_slot = -1;  // every chunk is issued; the slot stays the request's until the last completes
    complete.push_back(r.ticket);
  }
  finish_launch(s, k, complete, cudaSuccess);
}

// A small request runs alone, through the single-request kernels, when batching would gain it nothing:
//  * its estimated work is above kSoloCost, where a launch's fixed cost is negligible and the
//    table-form phasor kernel is faster than the batched per-warp form;
//  * or the batched kernel would run it on less than one wave of its tiles with enough work that those
//    tiles would run long (few rows and channels, many components), while the single-request kernels
//    split a short grid's tiles over component ranges so that the request fills the GPU.
constexpr double kSoloCost = 1.0e-3;     // seconds of estimated work
constexpr double kSoloMinCost = 2.0e-4;  // seconds of estimated work
static bool is_solo(const wn_server* s, const ServeReq& r) {
  const double cost = r.tile_cost * r.tiles;
  return r.tiles > 0 && (cost > kSoloCost || (r.tiles < 2L * s->ctx->num_sms && cost > kSoloMinCost));
}

// Launch small request r alone on slot k (is_solo).  Called with the lock held; the slot is idle.
static void launch_solo(wn_server* s, int k, ServeReq& r) {
  const int rc = launch_steps(s, k, r, 0, r.od.n_time);
  r.issued = 1;
  r.state = rc == WN_OK ? RQ_RUNNING : RQ_FAILED;
  if (rc != WN_OK) r.error = rc;
  r.batch = s->batches;
  r.t_launch = now_s(s);
  finish_launch(s, k, std::vector<uint64_t>{r.ticket}, cudaSuccess);
}

// Launch on slot k one batch of small unstarted requests submitted before ticket `bar`, in ticket order,
// up to kBatchBudget of estimated work (the first always goes), or the first of them alone when it is a
// solo request.  Called with the lock held.
static void launch_small(wn_server* s, int k, uint64_t bar) {
  ServeSlot& sl = s->slots[k];
  K1Args* args = slot_args(s, sl);
  K1Work* work = slot_work(s, sl);
  std::vector<uint64_t> complete, shapes;
  int nreq = 0, nwork = 0;
  double budget = kBatchBudget;
  for (auto& kv : s->reqs) {
    ServeReq& r = kv.second;
    if (kv.first >= bar) break;
    if (!unstarted(r) || is_large(r)) continue;
    if (is_solo(s, r)) {
      if (!complete.empty()) continue;  // it takes a slot of its own
      launch_solo(s, k, r);
      return;
    }
    const double cost = r.tile_cost * r.tiles;
    if (nreq == s->max_reqs || (!complete.empty() && (cost > budget || nwork + r.tiles > s->max_work))) continue;
    if (r.tiles > 0) {
      args[nreq] = r.k1;
      nwork = add_tiles(r, nreq, 0, r.tiles, work, nwork);
      ++nreq;
    }
    budget -= cost;
    r.issued = std::max(1L, r.tiles);
    r.state = RQ_RUNNING;
    r.batch = s->batches;
    r.t_launch = now_s(s);
    complete.push_back(r.ticket);
    if (r.M->n_shape > 0) shapes.push_back(r.ticket);
  }
  if (!complete.empty()) launch_slot(s, k, nwork, complete, shapes);
}

// Fill the free slots (slot 0 has the highest stream priority).
//  * Arrival order: large requests start in submission order.  One that is due takes the
//    highest-priority free slot, waits for the small requests submitted before it to be launched and
//    to finish, and then runs in one launch; small requests submitted after it wait until it has
//    started.  Small batches take the lowest-priority free slots, whose blocks the GPU dispatches after
//    a running large request's, one batch at a time while a large request runs.
//  * Small first: small batches take the highest-priority free slots as soon as there is work, one
//    batch at a time while a large request runs; large requests take the lowest-priority free slots,
//    least estimated work first with the wait limit, and run in chunks back to back.
// At most max_large_inflight large requests hold a slot, never the last free one.
static bool launch_ready(wn_server* s) {
  bool progress = false;
  const bool arrival = s->order == WN_SERVE_ARRIVAL;
  const int ns = (int)s->slots.size();
  auto free_slot = [&](bool highest) {
    for (int j = 0; j < ns; ++j) {
      const int k = highest ? j : ns - 1 - j;
      if (!s->slots[k].busy && !s->slots[k].owner) return k;
    }
    return -1;
  };
  int owners = 0;
  for (auto& sl : s->slots) owners += sl.owner ? 1 : 0;
  const double t_now = now_s(s);
  while (owners < std::min(s->max_large_inflight, std::max(1, ns - 1))) {
    const int k = free_slot(arrival);
    if (k < 0) break;
    // arrival order: the first submitted; small first: the oldest request past the wait limit, else
    // the least estimated work (ties: ticket order)
    ServeReq* pick = nullptr;
    bool pick_old = false;
    for (auto& kv : s->reqs) {
      ServeReq& q = kv.second;
      if (!unstarted(q) || !is_large(q)) continue;
      if (arrival) {
        pick = &q;
        break;
      }
      const bool old = t_now - q.t_submit > s->max_large_wait;
      if (pick_old && !old) continue;
      if (!pick || (old && !pick_old) || (!old && large_cost(q) < large_cost(*pick))) {
        pick = &q;
        pick_old = old;
      }
    }
    if (!pick) break;
    ServeReq& r = *pick;
    r.owner_slot = k;
    r.t_launch = now_s(s);
    s->slots[k].owner = r.ticket;
    ++owners;
  }
  int small_busy = 0;
  for (auto& sl : s->slots) small_busy += (sl.busy && !sl.owner) ? 1 : 0;
  // arrival order: small requests submitted after a large request that holds a slot but has not started
  // wait for it
  uint64_t bar = UINT64_MAX;
  if (arrival)
    for (auto& sl : s->slots)
      if (sl.owner) {
        auto it = s->reqs.find(sl.owner);
        if (it != s->reqs.end() && it->second.issued == 0) bar = std::min(bar, sl.owner);
      }
  while (small_waiting(s, bar)) {
    // while a large request runs, small batches go out one at a time (they keep batching while it runs)
    if (bar == UINT64_MAX && owners > 0 && small_busy >= 1) break;
    const int k = free_slot(!arrival);
    if (k < 0) break;
    launch_small(s, k, bar);
    ++small_busy;
    progress = true;
  }
  for (int k = 0; k < ns; ++k) {
    if (s->slots[k].busy || !s->slots[k].owner) continue;
    auto it = s->reqs.find(s->slots[k].owner);
    if (it == s->reqs.end() || it->second.owner_slot != k) continue;
    int kk = k;
    if (arrival && it->second.issued == 0) {
      // the small requests submitted before it go first; then it moves to the highest-priority free slot
      if (small_busy > 0 || small_waiting(s, it->first)) continue;
      const int j = free_slot(true);
      if (j >= 0 && j < k) {
        s->slots[j].owner = it->first;
        s->slots[k].owner = 0;
        it->second.owner_slot = j;
        kk = j;
      }
    }
    launch_chunk(s, kk);
    progress = true;
  }
  return progress;
}

static void scheduler(wn_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    // completions
    for (auto& sl : s->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      const double t = now_s(s);
      for (uint64_t tk : sl.reqs) {
        ServeReq& r = s->reqs[tk];
        if (r.state == RQ_RUNNING) {
          r.state = q == cudaSuccess ? RQ_DONE : RQ_FAILED;
          if (q != cudaSuccess) r.error = WN_ECUDA;
        }
        r.t_done = t;
      }
      sl.reqs.clear();
      sl.busy = false;
      // a large request holds its slot (and its place among max_large_inflight) until its last chunk
      // has completed, so the next one does not start beside that chunk and hold it back
      if (sl.owner) {
        auto it = s->reqs.find(sl.owner);
        if (it == s->reqs.end() || it->second.owner_slot < 0) sl.owner = 0;
      }
      progress = true;
    }
    // admission by slots and memory, in arrival order (a request that does not fit yet does not
    // block smaller ones behind it)
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      ServeReq& r = s->reqs[*it];
      if (r.state != RQ_PENDING) {
        it = s->queue.erase(it);
        continue;
      }
      size_t off = 0;
      if (s->admitted < s->max_inflight && pool_alloc(s, r.bytes, &off)) {
        r.off = off;
        r.has_mem = true;
        r.state = RQ_ADMITTED;
        r.tiles = 0;
        if (has_pg(r)) {
          if (k1_batched_args(s->ctx, r.od, r.M, reinterpret_cast<float2*>(s->pool + off), r.mode, r.pa, &r.k1, &r.gx,
                              &r.gy) != WN_OK) {
            r.state = RQ_FAILED;
            r.error = WN_EINVAL;
          } else {
            r.tiles = (long)r.gx * r.gy;
            const double rows_tile = (double)r.od.n_rows / r.gx, chans_tile = (double)r.od.n_chan / r.gy;
            const int n_pg = r.M->n_point + r.M->n_gauss;
            r.tile_cost = rows_tile * chans_tile * n_pg / kEvalRate;
          }
        }
        r.t_admit = now_s(s);
        s->admitted++;
        it = s->queue.erase(it);
        progress = true;
      } else {
        ++it;
      }
    }
    progress |= launch_ready(s);
    if (progress) s->cv.notify_all();
    s->cv.wait_for(lk, std::chrono::microseconds(progress ? 0 : 20));
  }
}

}  // namespace wn

using namespace wn;

extern "C" {

int wn_server_create(wn_ctx* ctx, int n_streams, size_t pool_bytes, int max_inflight, int max_rows, int max_chan,
                     wn_server** out) {
  if (!ctx || !out) return set_error(WN_EINVAL, "NULL argument");
  *out = nullptr;
  if (n_streams < 1 || n_streams > 16 || max_inflight < 1 || max_rows < 1 || max_chan < 1 || pool_bytes < 256)
    return set_error(WN_EINVAL, "server sizes out of range");
  cudaSetDevice(ctx->device);
  wn_server* s = new wn_server();
  s->ctx = ctx;
  s->max_inflight = max_inflight;
  s->max_reqs = std::max(1, std::min(max_inflight, 256));
  s->max_rows = max_rows;
  s->max_chan = max_chan;
  s->table_bytes = 16 + sizeof(K1Args) * s->max_reqs + sizeof(K1Work) * s->max_work;
  s->pool_bytes = pool_bytes & ~(size_t)255;
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = dev_malloc(&s->pool, s->pool_bytes);
  if (e != cudaSuccess) {
    delete s;
    return set_error(WN_ENOMEM, std::string("server pool: ") + cudaGetErrorString(e));
  }
  s->free_list[0] = s->pool_bytes;
  const size_t chan_bytes = round_bytes((size_t)max_chan * sizeof(float4));
  const int grid = ctx->num_sms * 2;
  s->slots.resize(n_streams);
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  for (size_t k = 0; k < s->slots.size(); ++k) {
    auto& sl = s->slots[k];
    // slot 0 has the highest priority, later slots lower ones (clamped to the device's range)
    sl.priority = std::min(prio_least, prio_greatest + (int)k);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.st, cudaStreamNonBlocking, sl.priority);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = dev_malloc(&sl.d_table, s->table_bytes);
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_table, s->table_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = dev_malloc(&sl.chaninfo, chan_bytes + (size_t)kSlotRowTables * max_rows * sizeof(float4));
    if (e == cudaSuccess) sl.rowinfo = reinterpret_cast<float4*>(reinterpret_cast<char*>(sl.chaninfo) + chan_bytes);
    if (e == cudaSuccess) {
      // graph per stream: copy of the work table from pinned memory, then the batched kernel
      cudaGraph_t g = nullptr;
      e = k1_batched_setup();
      if (e == cudaSuccess) e = cudaStreamBeginCapture(sl.st, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaMemcpyAsync(sl.d_table, sl.h_table, s->table_bytes, cudaMemcpyHostToDevice, sl.st);
        const K1Args* d_args = reinterpret_cast<const K1Args*>(sl.d_table + 16);
        const K1Work* d_work = reinterpret_cast<const K1Work*>(sl.d_table + 16 + sizeof(K1Args) * s->max_reqs);
        k1_batched_launch(d_args, d_work, reinterpret_cast<const int*>(sl.d_table), grid, sl.st);
        e = cudaStreamEndCapture(sl.st, &g);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.gexec, g, 0);
      if (g) cudaGraphDestroy(g);
    }
  }
  if (e != cudaSuccess) {
    for (auto& sl : s->slots) {
      if (sl.gexec) cudaGraphExecDestroy(sl.gexec);
      if (sl.st) cudaStreamDestroy(sl.st);
      if (sl.done) cudaEventDestroy(sl.done);
      cudaFree(sl.d_table);
      if (sl.h_table) cudaFreeHost(sl.h_table);
      cudaFree(sl.chaninfo);
      cudaFree(sl.ks.spec);
      cudaFree(sl.ks.part);
    }
    cudaFree(s->pool);
    delete s;
    return set_error(WN_ECUDA, std::string("server setup: ") + cudaGetErrorString(e));
  }
  s->worker = std::thread(scheduler, s);
  *out = s;
  return WN_OK;
}

void wn_server_destroy(wn_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->ctx->device);
  for (auto& sl : s->slots) {
    cudaStreamSynchronize(sl.st);
    cudaGraphExecDestroy(sl.gexec);
    cudaStreamDestroy(sl.st);
    cudaEventDestroy(sl.done);
    cudaFree(sl.d_table);
    cudaFreeHost(sl.h_table);
    cudaFree(sl.chaninfo);
    cudaFree(sl.ks.spec);
    cudaFree(sl.ks.part);
  }
  cudaFree(s->pool);
  delete s;
}

int wn_server_submit(wn_server* s, const wn_obs* obs, int model_id, int peel, const void* gains_c64, int gains_t,
                     int gains_f, const void* data_c64, uint64_t* ticket) {
  TraceRange trace_range(s ? s->ctx : nullptr, "wn_server_submit");
  if (!s || !ticket) return set_error(WN_EINVAL, "NULL argument");
  *ticket = 0;
  ServeReq r;
  if (!obs) return set_error(WN_EINVAL, "obs is NULL");
  // validation shared with the single-request entry points
  if (obs->n_ant < 2 || obs->n_base < 1 || obs->n_time < 1 || obs->n_chan < 1 || !obs->uvw || !obs->freq_hz ||
      !obs->ant1 || !obs->ant2 || !(obs->freq0_hz > 0.0))
    return set_error(WN_EINVAL, "invalid observation");
  if (!(obs->chan_spacing_hz > 0.0) && obs->n_chan > 1)
    return set_error(WN_EINVAL, "served observations need uniformly spaced channels");
  r.od.n_ant = obs->n_ant;
  r.od.n_base = obs->n_base;
  r.od.n_time = obs->n_time;
  r.od.n_chan = obs->n_chan;
  r.od.n_rows = obs->n_base * obs->n_time;
  r.od.uvw = obs->uvw;
  r.od.freq = obs->freq_hz;
  r.od.ant1 = obs->ant1;
  r.od.ant2 = obs->ant2;
  r.od.dec0 = obs->dec0;
  r.od.nu0 = obs->freq0_hz;
  r.od.dnu = obs->chan_spacing_hz;
  r.od.uniform = true;
  if (r.od.n_rows > s->max_rows || r.od.n_chan > s->max_chan)
    return set_error(WN_EINVAL, "observation larger than the server's row / channel tables");
  if (peel) {
    if (!gains_c64 || !data_c64 || !(gains_t == 1 || gains_t == obs->n_time) || !(gains_f == 1 || gains_f == obs->n_chan))
      return set_error(WN_EINVAL, "peel request needs data and gains [1|T][1|F][A]");
    r.pa.data = static_cast<const float2*>(data_c64);
    r.pa.gains = static_cast<const float2*>(gains_c64);
    r.pa.ant1 = obs->ant1;
    r.pa.ant2 = obs->ant2;
    r.pa.gt = gains_t;
    r.pa.gf = gains_f;
    r.pa.n_ant = obs->n_ant;
  }
  r.mode = peel ? OUT_PEEL : OUT_STORE;
  r.bytes = round_bytes((size_t)r.od.n_rows * r.od.n_chan * sizeof(float2));
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->ctx->models.find(model_id);
  if (it == s->ctx->models.end()) return set_error(WN_ENOTFOUND, "unknown model id");
  r.M = it->second;
  if (r.bytes > s->pool_bytes) return set_error(WN_EBUSY, "request larger than the server's memory pool");
  r.ticket = s->next_ticket++;
  r.t_submit = now_s(s);
  s->reqs[r.ticket] = r;
  s->queue.push_back(r.ticket);
  *ticket = r.ticket;
  s->cv.notify_all();
  return WN_OK;
}

// info: [t_submit, t_admit, t_launch, t_done] seconds on the server clock, then batch index.
int wn_server_poll(wn_server* s, uint64_t ticket, int* state, void** vis_out, double* info) {
  if (!s || !state) return set_error(WN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(WN_ENOTFOUND, "unknown ticket");
  const ServeReq& r = it->second;
  *state = r.state;
  if (vis_out) *vis_out = r.state == RQ_DONE ? static_cast<void*>(s->pool + r.off) : nullptr;
  if (info) {
    info[0] = r.t_submit;
    info[1] = r.t_admit;
    info[2] = r.t_launch;
    info[3] = r.t_done;
    info[4] = r.batch;
  }
  return r.state == RQ_FAILED ? set_error(r.error, "request failed") : WN_OK;
}

int wn_server_wait(wn_server* s, uint64_t ticket, double timeout_s, void** vis_out, double* info) {
  if (!s) return set_error(WN_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(WN_ENOTFOUND, "unknown ticket");
    const int st = it->second.state;
    if (st == RQ_DONE || st == RQ_FAILED || st == RQ_CANCELLED) break;
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) return set_error(WN_ETIMEOUT, "wait timed out");
  }
  lk.unlock();
  int state = 0;
  return wn_server_poll(s, ticket, &state, vis_out, info);
}

int wn_server_release(wn_server* s, uint64_t ticket) {
  if (!s) return set_error(WN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(WN_ENOTFOUND, "unknown ticket");
  ServeReq& r = it->second;
  if (r.state == RQ_RUNNING || r.state == RQ_ADMITTED) return set_error(WN_EBUSY, "request still on the GPU");
  if (r.has_mem) {
    pool_free(s, r.off, r.bytes);
    s->admitted--;
  }
  s->reqs.erase(it);
  s->cv.notify_all();
  return WN_OK;
}

int wn_server_copy(wn_server* s, uint64_t ticket, void* dst, void* stream) {
  if (!s || !dst) return set_error(WN_EINVAL, "NULL argument");
  const void* src = nullptr;
  size_t bytes = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(WN_ENOTFOUND, "unknown ticket");
    if (it->second.state != RQ_DONE) return set_error(WN_EBUSY, "request not done");
    src = s->pool + it->second.off;
    bytes = (size_t)it->second.od.n_rows * it->second.od.n_chan * sizeof(float2);
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return set_error(WN_ECUDA, std::string("copy result: ") + cudaGetErrorString(e));
  return WN_OK;
}

int wn_server_cancel(wn_server* s, uint64_t ticket) {
  if (!s) return set_error(WN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(WN_ENOTFOUND, "unknown ticket");
  if (it->second.state != RQ_PENDING) return set_error(WN_EBUSY, "request already admitted");
  it->second.state = RQ_CANCELLED;
  return WN_OK;
}

int wn_server_set_order(wn_server* s, int order) {
  if (!s) return set_error(WN_EINVAL, "NULL argument");
  if (order != WN_SERVE_ARRIVAL && order != WN_SERVE_SMALL_FIRST) return set_error(WN_EINVAL, "unknown request order");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->order = order;
  }
  s->cv.notify_all();
  return WN_OK;
}

int wn_server_set_policy(wn_server* s, int max_large_inflight, double max_large_wait_s) {
  if (!s) return set_error(WN_EINVAL, "NULL argument");
  if (max_large_inflight < 1 || max_large_inflight > 16) return set_error(WN_EINVAL, "max_large_inflight outside 1..16");
  if (!(max_large_wait_s >= 0.0)) return set_error(WN_EINVAL, "max_large_wait_s must be >= 0");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->max_large_inflight = max_large_inflight;
    s->max_large_wait = max_large_wait_s;
  }
  s->cv.notify_all();
  return WN_OK;
}

// stats: [batches, max batches on the GPU at once, most requests in one batch, requests launched,
//         requests admitted now, free pool bytes]
int wn_server_stats(wn_server* s, double* stats) {
  if (!s || !stats) return set_error(WN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  size_t free_b = 0;
  for (auto& kv : s->free_list) free_b += kv.second;
  stats[0] = s->batches;
  stats[1] = s->max_running_batches;
  stats[2] = s->max_batch_reqs;
  stats[3] = s->launched;
  stats[4] = s->admitted;
  stats[5] = (double)free_b;
  return WN_OK;
}

}  // extern "C"
