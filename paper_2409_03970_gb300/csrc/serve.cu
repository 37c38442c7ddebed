// Sort server: continuous batching of sort requests on one GPU.
//
// A context owns a scheduler thread, `streams` CUDA streams (slots), one
// device arena of mem_budget_bytes for scratch, and pinned host buffers for
// batch descriptors.  Requests wait in a FIFO queue; whenever a slot is
// free and the arena can hold the scratch of the request at the head, it is
// admitted (while a request of LARGE_MIN_KEYS keys or more runs, the next
// such request waits and the first smaller one is admitted ahead of it; the
// next large one is enqueued behind the running one on the GPU, through a
// completion event, once no smaller request waits):
// large requests run alone as nsort_keys / nsort_pairs; small ones
// (n <= batch_max_keys) are co-batched with the other waiting small requests
// of the same kind and dtype into one segmented sort (a gather kernel packs
// their keys, nsort_segmented sorts every request as its own segment, a
// scatter kernel writes each result back).  Admitted work on different slots
// overlaps on the device.  Completion is signalled from the stream by a host
// function; the scheduler then frees the scratch and wakes waiters.  Each
// result is bit-identical to the plain call on the same input, batched or
// not.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nsort.h"
#include "nsort_internal.h"
#include "serve_policy.h"

namespace nsort {
namespace serve {

constexpr size_t MAX_BATCH = 4096;                 // requests per co-batch
constexpr uint64_t MAX_BATCH_KEYS = uint64_t(1) << 24;
// Requests of at least this many keys run one at a time (their sorts'
// persistent merge grids fill every SM); smaller ones may pass them.
constexpr uint64_t LARGE_MIN_KEYS = uint64_t(1) << 22;

struct BatchItem {
  const uint32_t *kin;
  uint32_t *kout;
  const uint32_t *vin;
  uint32_t *vout;
  int64_t off;   // position in the packed batch
  int64_t n;
};

// Packs every request of a batch into one array (keys and values).
__global__ void batch_gather_kernel(const BatchItem *items, int count, uint32_t *sk, uint32_t *sv) {
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const BatchItem it = items[i];
    for (int64_t e = threadIdx.x; e < it.n; e += blockDim.x) {
      sk[it.off + e] = it.kin[e];
      if (sv) sv[it.off + e] = it.vin[e];
    }
  }
}

// Writes each request's sorted segment back to its own output.
__global__ void batch_scatter_kernel(const BatchItem *items, int count, const uint32_t *sk,
                                     const uint32_t *sv) {
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const BatchItem it = items[i];
    for (int64_t e = threadIdx.x; e < it.n; e += blockDim.x) {
      it.kout[e] = sk[it.off + e];
      if (sv) it.vout[e] = sv[it.off + e];
    }
  }
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
  nsort_request r;
  int status = NSORT_OK;
  bool done = false;
  int batched = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Ctx;

struct Job {
  Ctx *ctx = nullptr;
  int slot = -1;
  std::vector<uint64_t> tickets;
  std::vector<std::pair<size_t, size_t>> allocs;   // arena blocks
  std::atomic<int> finished{0};
  double t_finish = 0;
  int status = NSORT_OK;     // launch status, reported to every request of the job
  bool large = false;        // a request of at least LARGE_MIN_KEYS keys
  cudaEvent_t done_ev = nullptr;   // large jobs: recorded after their work
  ~Job() {
    if (done_ev) cudaEventDestroy(done_ev);
  }
};

struct Slot {
  cudaStream_t stream = nullptr;
  bool busy = false;
  void *pinned = nullptr;    // batch descriptor staging
  size_t pinned_bytes = 0;
};

struct Ctx {
  int device = 0;
  size_t budget = 0;
  uint64_t batch_max_keys = 0;
  char *arena_base = nullptr;
  Arena arena;
  std::vector<Slot> slots;
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<Pending> queue;
  std::list<std::unique_ptr<Job>> jobs;
  std::mutex mu;
  std::condition_variable cv;        // wakes the scheduler
  std::condition_variable cv_done;   // wakes nsort_wait
  std::thread th;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::atomic<uint64_t> epoch{0};    // bumped by every completion callback
};

// Runs on the driver's callback thread when the stream reaches the end of
// a job.  Takes no lock (the scheduler may hold it while it enqueues work):
// it publishes the completion and bumps the epoch the scheduler waits on.
void CUDART_CB job_done(void *p) {
  Job *j = static_cast<Job *>(p);
  j->t_finish = now_s();
  Ctx *c = j->ctx;
  j->finished.store(1);
  c->epoch.fetch_add(1);
  c->cv.notify_all();
}

size_t single_need(const Req &q) {
  return nsort_temp_bytes(q.r.kind, q.r.n, 0, q.r.dtype);
}

// Arena bytes of a co-batch of `total` keys in `count` requests.
size_t batch_need(int kind, uint64_t total, size_t count) {
  const bool pairs = kind == NSORT_KIND_PAIRS;
  size_t b = align_up(total * 4, 256) * (pairs ? 2 : 1);
  b += align_up((count + 1) * sizeof(int64_t), 256);
  b += align_up(count * sizeof(BatchItem), 256);
  b += nsort_temp_bytes(pairs ? NSORT_KIND_SEGMENTED_PAIRS : NSORT_KIND_SEGMENTED, total, count, 0);
  return b;
}

void finish_now(Ctx *c, uint64_t t, int status) {
  Req &q = c->reqs[t];
  q.status = status;
  q.done = true;
  q.t_done = now_s();
}

// Launches one job on slot s (the caller holds c->mu).  On a launch error
// the requests complete at once with that status.  after: the completion
// event of a large job this one must follow on the GPU (or null).
void launch(Ctx *c, int s, std::vector<Pending> &picked, std::vector<std::pair<size_t, size_t>> &allocs,
            cudaEvent_t after = nullptr) {
  Slot &slot = c->slots[s];
  auto job = std::make_unique<Job>();
  job->ctx = c;
  job->slot = s;
  for (auto &p : picked) job->tickets.push_back(p.ticket);
  job->allocs = allocs;
  job->large = picked.size() == 1 && picked[0].n >= LARGE_MIN_KEYS;
  const double t = now_s();
  for (auto &p : picked) c->reqs[p.ticket].t_admit = t;
  int rc = NSORT_OK;
  if (after && cudaStreamWaitEvent(slot.stream, after, 0) != cudaSuccess) rc = NSORT_ECUDA;
  if (picked.size() == 1 && c->reqs[picked[0].ticket].batched == 0) {
    const Req &q = c->reqs[picked[0].ticket];
    void *tmp = allocs.empty() ? nullptr : c->arena_base + allocs[0].first;
    const size_t tb = allocs.empty() ? 0 : allocs[0].second;
    if (q.r.kind == NSORT_KIND_KEYS)
      rc = nsort_keys(q.r.d_keys_in, q.r.d_keys_out, q.r.n, q.r.dtype, tmp, tb, slot.stream);
    else
      rc = nsort_pairs(q.r.d_keys_in, q.r.d_vals_in, q.r.d_keys_out, q.r.d_vals_out, q.r.n,
                       q.r.dtype, tmp, tb, slot.stream);
  } else {
    const int kind = picked[0].kind;
    const bool pairs = kind == NSORT_KIND_PAIRS;
    const size_t count = picked.size();
    uint64_t total = 0, longest = 0;
    for (auto &p : picked) {
      total += p.n;
      longest = p.n > longest ? p.n : longest;
    }
    char *base = c->arena_base + allocs[0].first;
    size_t o = 0;
    uint32_t *sk = reinterpret_cast<uint32_t *>(base + o);
    o += align_up(total * 4, 256);
    uint32_t *sv = nullptr;
    if (pairs) {
      sv = reinterpret_cast<uint32_t *>(base + o);
      o += align_up(total * 4, 256);
    }
    int64_t *offs = reinterpret_cast<int64_t *>(base + o);
    o += align_up((count + 1) * sizeof(int64_t), 256);
    BatchItem *items = reinterpret_cast<BatchItem *>(base + o);
    o += align_up(count * sizeof(BatchItem), 256);
    void *segtmp = base + o;
    const size_t segbytes = allocs[0].second - o;
    // descriptors: offsets then items, staged in the slot's pinned buffer
    int64_t *h_offs = static_cast<int64_t *>(slot.pinned);
    BatchItem *h_items = reinterpret_cast<BatchItem *>(
        static_cast<char *>(slot.pinned) + align_up((count + 1) * sizeof(int64_t), 256));
    int64_t acc = 0;
    for (size_t i = 0; i < count; ++i) {
      const Req &q = c->reqs[picked[i].ticket];
      h_offs[i] = acc;
      h_items[i] = {static_cast<const uint32_t *>(q.r.d_keys_in), static_cast<uint32_t *>(q.r.d_keys_out),
                    q.r.d_vals_in, q.r.d_vals_out, acc, (int64_t)q.r.n};
      acc += (int64_t)q.r.n;
    }
    h_offs[count] = acc;
    const size_t desc_bytes = align_up((count + 1) * sizeof(int64_t), 256) + count * sizeof(BatchItem);
    // the device copy of [offsets | items] has the same layout as the pinned one
    if (cudaMemcpyAsync(offs, slot.pinned, desc_bytes, cudaMemcpyHostToDevice, slot.stream) !=
        cudaSuccess)
      rc = NSORT_ECUDA;
    if (rc == NSORT_OK) {
      const unsigned g = (unsigned)(count < 2048 ? count : 2048);
      batch_gather_kernel<<<g, 256, 0, slot.stream>>>(items, (int)count, sk, sv);
      // no segment is longer than the longest request: launch only the
      // merge levels it needs
      rc = segmented_impl(sk, sk, sv, sv, offs, count, total, picked[0].dtype, segtmp, segbytes,
                          slot.stream, longest);
      if (rc == NSORT_OK) {
        batch_scatter_kernel<<<g, 256, 0, slot.stream>>>(items, (int)count, sk, sv);
        if (cudaGetLastError() != cudaSuccess) rc = NSORT_ECUDA;
      }
    }
  }
  if (job->large && cudaEventCreateWithFlags(&job->done_ev, cudaEventDisableTiming) == cudaSuccess &&
      cudaEventRecord(job->done_ev, slot.stream) != cudaSuccess) {
    cudaEventDestroy(job->done_ev);
    job->done_ev = nullptr;
  }
  // the job completes through the stream even when a launch failed, so its
  // scratch is released only after everything enqueued so far has run
  job->status = rc;
  if (cudaLaunchHostFunc(slot.stream, job_done, job.get()) != cudaSuccess) {
    job->status = NSORT_ECUDA;
    job->t_finish = now_s();
    job->finished.store(1);   // nothing will signal it; the scheduler syncs the slot
    job->slot = -1 - s;       // marks "synchronise before releasing"
  }
  slot.busy = true;
  c->jobs.push_back(std::move(job));
}

void scheduler(Ctx *c) {
  cudaSetDevice(c->device);
  std::unique_lock<std::mutex> lk(c->mu);
  for (;;) {
    const uint64_t seen = c->epoch.load();
    bool completed = false;
    for (auto it = c->jobs.begin(); it != c->jobs.end();) {
      Job *j = it->get();
      if (!j->finished.load()) {
        ++it;
        continue;
      }
      int slot = j->slot;
      if (slot < 0) {   // no callback could be enqueued: wait for the stream here
        slot = -1 - slot;
        lk.unlock();
        cudaStreamSynchronize(c->slots[slot].stream);
        lk.lock();
      }
      for (uint64_t t : j->tickets) {
        Req &q = c->reqs[t];
        q.done = true;
        q.status = j->status;
        q.t_done = j->t_finish;
      }
      for (auto &a : j->allocs) c->arena.release(a.first, a.second);
      c->slots[slot].busy = false;
      it = c->jobs.erase(it);
      completed = true;
    }
    if (completed) c->cv_done.notify_all();
    if (c->stop) {
      // cancel what was never admitted
      for (auto &p : c->queue) finish_now(c, p.ticket, NSORT_EBUSY);
      if (!c->queue.empty()) c->cv_done.notify_all();
      c->queue.clear();
      if (c->jobs.empty()) break;
    }
    // admission: FIFO, except that while a large request runs the next
    // one waits and smaller requests go ahead; the batch must fit in the arena
    for (int s = 0; s < (int)c->slots.size() && !c->queue.empty(); ++s) {
      if (c->slots[s].busy) continue;
      int large_live = 0;          // large jobs enqueued and not finished
      Job *large_last = nullptr;   // the latest of them
      for (auto &j : c->jobs)
        if (j->large && !j->finished.load()) {
          ++large_live;
          large_last = j.get();
        }
      std::vector<size_t> pos = pick_batch(c->queue, c->batch_max_keys, MAX_BATCH, MAX_BATCH_KEYS,
                                           LARGE_MIN_KEYS, large_live > 0);
      cudaEvent_t after = nullptr;
      if (pos.empty()) {
        // only large requests wait and one runs: enqueue the next one behind
        // it on the GPU (its stream waits for the running job's completion
        // event), so that it starts without a round trip through this thread;
        // at most one waits so
        if (large_live != 1 || !large_last->done_ev) break;
        pos = pick_batch(c->queue, c->batch_max_keys, MAX_BATCH, MAX_BATCH_KEYS);
        after = large_last->done_ev;
      }
      const Pending &head = c->queue[pos[0]];
      const bool batch = c->batch_max_keys > 0 && head.n <= c->batch_max_keys;
      size_t need;
      if (batch) {
        uint64_t total = 0;
        for (size_t i : pos) total += c->queue[i].n;
        need = batch_need(head.kind, total, pos.size());
      } else {
        need = single_need(c->reqs[head.ticket]);
      }
      size_t off = 0;
      std::vector<std::pair<size_t, size_t>> allocs;
      if (need > 0) {
        if (!c->arena.alloc(need, &off)) break;   // wait for memory (FIFO)
        allocs.push_back({off, need});
      }
      std::vector<Pending> picked = take(c->queue, pos);
      if (batch)
        for (auto &p : picked) c->reqs[p.ticket].batched = 1;
      launch(c, s, picked, allocs, after);
    }
    // sleep until a submission, a completion or destruction; the short
    // time-out covers a completion notified between the scan and the wait
    c->cv.wait_for(lk, std::chrono::microseconds(200),
                   [&] { return c->epoch.load() != seen || c->stop; });
  }
}

}  // namespace serve
}  // namespace nsort

using namespace nsort;

struct nsort_ctx {
  serve::Ctx c;
};

extern "C" int nsort_ctx_create(int device, size_t mem_budget_bytes, int streams,
                                uint64_t batch_max_keys, nsort_ctx **out) {
  if (!out || streams < 1 || streams > 64) return NSORT_EINVAL;
  *out = nullptr;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    set_last_error("nsort_ctx_create: bad device");
    return NSORT_EINVAL;
  }
  auto ctx = std::make_unique<nsort_ctx>();
  serve::Ctx &c = ctx->c;
  c.device = device;
  c.budget = mem_budget_bytes;
  c.batch_max_keys = batch_max_keys;
  int rc = NSORT_OK;
  if (mem_budget_bytes) {
    if (cudaMalloc(&c.arena_base, mem_budget_bytes) != cudaSuccess) {
      set_last_error("nsort_ctx_create: cannot allocate the scratch arena");
      rc = NSORT_ENOMEM;
    }
  }
  c.arena.reset(rc == NSORT_OK ? mem_budget_bytes : 0, 256);
  const size_t pinned_bytes =
      align_up((serve::MAX_BATCH + 1) * sizeof(int64_t), 256) + serve::MAX_BATCH * sizeof(serve::BatchItem);
  c.slots.resize(streams);
  for (auto &s : c.slots) {
    if (rc != NSORT_OK) break;
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&s.pinned, pinned_bytes) != cudaSuccess) {
      set_last_error("nsort_ctx_create: stream or pinned buffer");
      rc = NSORT_ECUDA;
    }
    s.pinned_bytes = pinned_bytes;
  }
  if (rc != NSORT_OK) {
    for (auto &s : c.slots) {
      if (s.stream) cudaStreamDestroy(s.stream);
      if (s.pinned) cudaFreeHost(s.pinned);
    }
    if (c.arena_base) cudaFree(c.arena_base);
    cudaSetDevice(prev);
    return rc;
  }
  c.th = std::thread(serve::scheduler, &c);
  cudaSetDevice(prev);
  *out = ctx.release();
  return NSORT_OK;
}

extern "C" void nsort_ctx_destroy(nsort_ctx *ctx) {
  if (!ctx) return;
  serve::Ctx &c = ctx->c;
  {
    std::lock_guard<std::mutex> lk(c.mu);
    c.stop = true;
  }
  c.cv.notify_all();
  if (c.th.joinable()) c.th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c.device);
  for (auto &s : c.slots) {
    if (s.stream) {
      cudaStreamSynchronize(s.stream);
      cudaStreamDestroy(s.stream);
    }
    if (s.pinned) cudaFreeHost(s.pinned);
  }
  if (c.arena_base) cudaFree(c.arena_base);
  cudaSetDevice(prev);
  delete ctx;
}

extern "C" int nsort_submit(nsort_ctx *ctx, const nsort_request *req, uint64_t *ticket) {
  if (!ctx || !req || !ticket) return NSORT_EINVAL;
  const nsort_request &r = *req;
  if (r.kind != NSORT_KIND_KEYS && r.kind != NSORT_KIND_PAIRS) return NSORT_EINVAL;
  if (r.dtype != NSORT_U32 && r.dtype != NSORT_I32 && r.dtype != NSORT_F32) return NSORT_EINVAL;
  if (r.n > MAX_KEYS) return NSORT_EINVAL;
  if (r.n > 0 && (!r.d_keys_in || !r.d_keys_out)) return NSORT_EINVAL;
  if (r.kind == NSORT_KIND_PAIRS && r.n > 0 && (!r.d_vals_in || !r.d_vals_out)) return NSORT_EINVAL;
  serve::Ctx &c = ctx->c;
  const bool batch = c.batch_max_keys > 0 && r.n <= c.batch_max_keys;
  const size_t need = batch ? serve::batch_need(r.kind, r.n, 1)
                            : nsort_temp_bytes(r.kind, r.n, 0, r.dtype);
  if (need > c.arena.capacity() && need > 0) return NSORT_ENOMEM;   // can never be admitted
  {
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.stop) return NSORT_EBUSY;
    const uint64_t t = c.next_ticket++;
    serve::Req q;
    q.r = r;
    q.t_submit = serve::now_s();
    if (r.n == 0) {
      q.done = true;
      q.t_admit = q.t_done = q.t_submit;
      c.reqs[t] = q;
      *ticket = t;
      c.cv_done.notify_all();
      return NSORT_OK;
    }
    c.reqs[t] = q;
    c.queue.push_back({t, r.kind, r.dtype, r.n});
    *ticket = t;
    c.epoch.fetch_add(1);
  }
  c.cv.notify_all();
  return NSORT_OK;
}

extern "C" int nsort_poll(nsort_ctx *ctx, uint64_t ticket, int *done, nsort_timing *timing) {
  if (!ctx || !done) return NSORT_EINVAL;
  serve::Ctx &c = ctx->c;
  std::lock_guard<std::mutex> lk(c.mu);
  auto it = c.reqs.find(ticket);
  if (it == c.reqs.end()) return NSORT_ENOTFOUND;
  const serve::Req &q = it->second;
  *done = q.done ? 1 : 0;
  if (timing && q.done) {
    timing->t_submit = q.t_submit;
    timing->t_admit = q.t_admit;
    timing->t_done = q.t_done;
    timing->status = q.status;
    timing->batched = q.batched;
  }
  return NSORT_OK;
}

extern "C" int nsort_wait(nsort_ctx *ctx, uint64_t ticket, uint32_t timeout_ms) {
  if (!ctx) return NSORT_EINVAL;
  serve::Ctx &c = ctx->c;
  std::unique_lock<std::mutex> lk(c.mu);
  auto it = c.reqs.find(ticket);
  if (it == c.reqs.end()) return NSORT_ENOTFOUND;
  const bool ok = c.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
    return c.reqs[ticket].done;
  });
  if (!ok) return NSORT_ETIMEOUT;
  return c.reqs[ticket].status;
}

// ---- policy hooks for CPU tests (no CUDA calls) --------------------------

extern "C" int nsort_policy_pick_batch(const uint64_t *tickets, const int *kinds, const int *dtypes,
                                       const uint64_t *ns, int count, uint64_t batch_max_keys,
                                       int max_batch, uint64_t max_batch_keys,
                                       uint64_t large_min_keys, int large_running, uint64_t *out,
                                       int *out_count) {
  if (count < 0 || !out || !out_count || max_batch < 1) return NSORT_EINVAL;
  std::deque<serve::Pending> q;
  for (int i = 0; i < count; ++i) q.push_back({tickets[i], kinds[i], dtypes[i], ns[i]});
  const std::vector<size_t> pos = serve::pick_batch(q, batch_max_keys, (size_t)max_batch,
                                                    max_batch_keys, large_min_keys,
                                                    large_running != 0);
  const std::vector<serve::Pending> got = serve::take(q, pos);
  for (size_t i = 0; i < got.size(); ++i) out[i] = got[i].ticket;
  *out_count = (int)got.size();
  return NSORT_OK;
}

extern "C" int nsort_policy_arena_replay(uint64_t capacity, const int64_t *ops, int nops,
                                         int64_t *offsets) {
  // ops[i] > 0: allocate ops[i] bytes (offsets[i] = offset or -1);
  // ops[i] < 0: release the block allocated by op number -ops[i]-1 (offsets[i] = 0).
  if (!ops || !offsets || nops < 0) return NSORT_EINVAL;
  serve::Arena a(capacity, 256);
  std::vector<int64_t> sizes(nops, 0);
  for (int i = 0; i < nops; ++i) {
    if (ops[i] > 0) {
      size_t off = 0;
      if (a.alloc((size_t)ops[i], &off)) {
        offsets[i] = (int64_t)off;
        sizes[i] = ops[i];
      } else {
        offsets[i] = -1;
      }
    } else {
      const int64_t k = -ops[i] - 1;
      if (k < 0 || k >= i || offsets[k] < 0 || sizes[k] == 0) return NSORT_EINVAL;
      a.release((size_t)offsets[k], (size_t)sizes[k]);
      sizes[k] = 0;
      offsets[i] = 0;
    }
  }
  return NSORT_OK;
}
