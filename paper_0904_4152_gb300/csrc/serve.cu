// Continuous-batching solve server.  Requests go to one of two lanes by size (levels below
// kLargeLevel, and the rest); each lane has its own FIFO queue, worker thread, engine and streams,
// so that small requests' iterations run at their own cadence beside the large requests' ones
// instead of waiting for their finest-level steps.  A request is admitted when a slot is free and
// its hierarchy fits the device-memory budget (slots and budget shared by the lanes).  Every pass
// of a lane's worker runs one launch sequence of the V-cycle schedule (engine.cu) over the lane's
// active requests at once; requests that finish leave between passes, free their memory and let
// queued requests in.  The hierarchy of a request stays resident on the device from admission to
// completion.
#include <algorithm>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "engine.h"

using namespace hn;

namespace {

// Page-locked host buffers, recycled by size: a request's inputs and result live in them, so
// the copies to and from the device are plain DMA and no fresh host pages are touched per request.
struct HostPool {
  std::mutex mu;
  std::multimap<size_t, void*> blocks;
  size_t cached = 0;
  static constexpr size_t kCap = size_t(4) << 30;   // cached bytes kept at most
  void* take(size_t bytes) {
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = blocks.find(bytes);
      if (it != blocks.end()) {
        void* p = it->second;
        blocks.erase(it);
        cached -= bytes;
        return p;
      }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void give(void* p, size_t bytes) {
    if (!p) return;
    {
      std::lock_guard<std::mutex> lk(mu);
      if (cached + bytes <= kCap) {
        blocks.emplace(bytes, p);
        cached += bytes;
        return;
      }
    }
    cudaFreeHost(p);
  }
  ~HostPool() {
    for (auto& kv : blocks) cudaFreeHost(kv.second);
  }
};

// n doubles in a HostPool block, returned to the pool on release / destruction
struct HostBuf {
  HostPool* pool = nullptr;
  double* p = nullptr;
  size_t n = 0;
  HostBuf() = default;
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  ~HostBuf() { release(); }
  bool alloc(HostPool* pl, size_t count) {
    release();
    pool = pl;
    p = static_cast<double*>(pl->take(count * 8));
    n = p ? count : 0;
    return p != nullptr;
  }
  void release() {
    if (p) pool->give(p, n * 8);
    p = nullptr;
    n = 0;
  }
};

struct Request {
  unsigned long long ticket = 0;
  int L = 0;
  unsigned bc = 15u;                 // Dirichlet sides of its operator
  HostBuf coef, b, x;                // coef empty for a = 1
  hn_mg* mg = nullptr;
  int slot = -1;
  int lane = 0;                      // 0: levels below kLargeLevel, 1: the others
  size_t bytes = 0;
  bool done = false;
  int status = HN_PENDING;
  hn_mg_stats stats{};
  long long t_submit = 0, t_admit = 0, t_done = 0;
};

// Device blocks of retired requests (hierarchies, transient operators), kept for the next
// request that needs a block of the same size: cudaMalloc / cudaFree of these sizes take
// milliseconds and synchronize the device, on the worker's critical path.
struct BlockCache {
  std::multimap<size_t, void*> blocks;
  size_t bytes = 0;
  void* take(size_t b) {
    auto it = blocks.find(b);
    if (it == blocks.end()) return nullptr;
    void* p = it->second;
    blocks.erase(it);
    bytes -= b;
    return p;
  }
  void give(void* p, size_t b) {
    if (!p) return;
    blocks.emplace(b, p);
    bytes += b;
  }
  void clear() {
    for (auto& kv : blocks) cudaFree(kv.second);
    blocks.clear();
    bytes = 0;
  }
  // free cached blocks, largest first, until at most `target` bytes stay cached; one block of
  // each size in `keep` (the blocks the next request will take) is freed last
  void release_to(size_t target, size_t keep0, size_t keep1) {
    bool kept0 = false, kept1 = false;
    std::vector<std::pair<size_t, void*>> spared;
    while (bytes > target && !blocks.empty()) {
      auto it = std::prev(blocks.end());
      if ((!kept0 && it->first == keep0) || (!kept1 && it->first == keep1)) {
        if (it->first == keep0 && !kept0) kept0 = true; else kept1 = true;
        spared.emplace_back(*it);
        bytes -= it->first;                         // set aside, counted again below
        blocks.erase(it);
        continue;
      }
      cudaFree(it->second);
      bytes -= it->first;
      blocks.erase(it);
    }
    for (auto& kv : spared) { blocks.emplace(kv.first, kv.second); bytes += kv.first; }
    while (bytes > target && !blocks.empty()) {    // still above: the spared blocks too
      auto it = std::prev(blocks.end());
      cudaFree(it->second);
      bytes -= it->first;
      blocks.erase(it);
    }
  }
};

}  // namespace

struct hn_server {
  HostPool host;                     // first member: outlives the requests' buffers
  size_t budget = 0;
  int max_active = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  static constexpr int kLanes = 2;
  static constexpr int kLargeLevel = 10;
  std::deque<Request*> queue[kLanes];   // FIFO per lane
  std::map<unsigned long long, std::unique_ptr<Request>> all;
  unsigned long long next_ticket = 1;
  bool stop = false;
  bool have_opts = false;
  hn_mg_opts opts{};
  size_t in_use = 0;
  long long submitted = 0, completed = 0, iterations = 0;
  long long admit_ns = 0, schedule_ns = 0, iterate_ns = 0, retire_ns = 0;   // worker time
  std::vector<Request*> slots;
  // Admitted requests go to the builder threads, which assemble their operators and hierarchies
  // on their own streams while the workers keep iterating the running requests; built requests
  // join their lane's schedule at its worker's next pass.
  std::deque<Request*> to_build;     // admitted, waiting for the builder (under mu)
  std::vector<Request*> built[kLanes];   // built (or failed), not yet in the schedule (under mu)
  int building = 0;                  // requests the builders hold (under mu)
  bool builder_stop = false;         // (under mu)
  std::condition_variable cv_build;
  std::mutex cache_mu;               // the block cache and the builders' scratch bytes
  BlockCache cache;
  size_t scratch_bytes = 0;          // the builders' setup temporaries, together
  static constexpr int kBuilders = 2;  // a small request need not wait for a large one's setup
  std::thread workers[kLanes], builders[kBuilders];
  std::string worker_error;          // the first worker failure (under mu)
  void run(int lane);
  void build_loop();
};

namespace {

// Detach a device block from its owner for the block cache.  A block the server supplied (no
// base) or one the library allocated without guards (base == block) moves to the cache and its
// owner forgets it; a guarded block of the checked build (base != block) stays with its owner,
// which frees it.  Returns the block for the cache, or nullptr.
void* detach_block(void*& mem, void*& base) {
  if (!mem || (base && base != mem)) return nullptr;
  void* b = mem;
  mem = nullptr;
  base = nullptr;
  return b;
}

size_t request_bytes(int L, const hn_mg_opts& o) {
  const Params p = params_from(o);
  // resident hierarchy + the transient fine operator built during admission
  return hierarchy_bytes(L, o.coarse_L, p.prec, p.solver) + (size_t)9 * pitch_of(L) * 8 +
         (size_t)(1LL << L) * (1LL << L) * 8 + 4096;
}

}  // namespace

void hn_server::build_loop() {
  cudaSetDevice(device);
  void* scratch = nullptr;           // this builder's setup temporaries, grown on demand
  size_t my_scratch = 0;
  cudaStream_t sb = nullptr;
  const bool stream_ok = cudaStreamCreateWithFlags(&sb, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_build.wait(lk, [&] { return builder_stop || !to_build.empty(); });
      if (to_build.empty()) break;
      r = to_build.front();
      to_build.pop_front();
      ++building;
    }
    // the operator and hierarchy (explicit copies of the inputs, checked at submit; device blocks
    // from the cache when it has one), the right-hand side and a zero iterate
    const long long t0 = now_ns();
    const bool has_coef = r->coef.p != nullptr;
    const size_t bb = band_bytes(r->L, has_coef);
    hn_mg_opts o = opts;
    o.stream = sb;
    const Params prm = params_from(o);
    const size_t hb = hierarchy_bytes(r->L, o.coarse_L, prm.prec, prm.solver);
    void* band_blk = nullptr;
    void* hier_blk = nullptr;
    {
      std::lock_guard<std::mutex> lk(cache_mu);
      band_blk = cache.take(bb);
      hier_blk = cache.take(hb);
      const size_t tmp = hierarchy_tmp_bytes(r->L, o.coarse_L, prm.prec, has_coef);
      if (tmp > my_scratch) {
        if (scratch) cudaFree(scratch);
        scratch = nullptr;
        scratch_bytes -= my_scratch;
        my_scratch = 0;
        if (cudaMalloc(&scratch, tmp) == cudaSuccess) my_scratch = tmp;
        else cudaGetLastError();                    // build_hierarchy allocates its own then
        scratch_bytes += my_scratch;
      }
    }
    hn_status st = stream_ok ? HN_OK : HN_ERR_CUDA;
    hn_band* A = nullptr;
    if (st == HN_OK) st = build_band(r->L, has_coef ? r->coef.p : nullptr, r->bc, sb, band_blk, &A);
    else if (band_blk) { std::lock_guard<std::mutex> lk(cache_mu); cache.give(band_blk, bb); }
    std::unique_ptr<hn_mg> h;
    if (st == HN_OK) {
      h.reset(new hn_mg());
      h->stream = sb;
      st = build_hierarchy(A, o, sb, h.get(), hier_blk, scratch, my_scratch);
      hier_blk = nullptr;
    }
    if (hier_blk) { std::lock_guard<std::mutex> lk(cache_mu); cache.give(hier_blk, hb); }
    if (st == HN_OK) {
      const long long N = N_of(r->L);
      if (cudaMemcpyAsync(h->host.b64, r->b.p, (size_t)N * 8, cudaMemcpyHostToDevice, sb) != cudaSuccess ||
          cudaMemsetAsync(h->host.x64, 0, (size_t)N * 8, sb) != cudaSuccess ||
          cudaStreamSynchronize(sb) != cudaSuccess)
        st = HN_ERR_CUDA;
    }
    if (A) {                                        // its block: free again once sb got here
      cudaStreamSynchronize(sb);
      void* blk = detach_block(A->mem, A->mem_base);
      hn_band_destroy(A);
      if (blk) { std::lock_guard<std::mutex> lk(cache_mu); cache.give(blk, bb); }
    }
    hn_mg* mg = nullptr;
    if (h) {
      h->stream = nullptr;                          // built: later users run on the worker's streams
      h->setup_ns = now_ns() - t0;
      mg = h.release();
    }
    if (st != HN_OK && mg) {
      hn_mg_destroy(mg);
      mg = nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    r->mg = mg;
    if (st != HN_OK) r->status = st;
    else r->stats.setup_ns = mg->setup_ns;
    admit_ns += now_ns() - t0;
    built[r->lane].push_back(r);
    --building;
    cv_work.notify_all();
  }
  {
    std::lock_guard<std::mutex> lk(cache_mu);
    if (scratch) cudaFree(scratch);
    scratch_bytes -= my_scratch;
  }
  if (sb) cudaStreamDestroy(sb);
}

void hn_server::run(int lane) {
  cudaSetDevice(device);
  // s: the lane's iterations (the small requests' lane at the greatest stream priority, so that
  // its short kernels are not queued behind the large requests' blocks); s3: copying finished
  // requests' results back while the next iteration runs (the builders have their own streams)
  cudaStream_t s = nullptr, s3 = nullptr;
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
    cudaGetLastError();
    prio_least = prio_greatest = 0;
  }
  if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, lane == 0 ? prio_greatest : prio_least) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s3, cudaStreamNonBlocking) != cudaSuccess) {
    std::lock_guard<std::mutex> lk(mu);
    if (worker_error.empty()) worker_error = "stream creation failed";
    stop = true;
    for (std::deque<Request*>& q : queue) {
      for (Request* r : q) { r->status = HN_ERR_CUDA; r->done = true; }
      q.clear();
    }
    cv_work.notify_all();
    cv_done.notify_all();
    if (s) cudaStreamDestroy(s);
    return;
  }
  // Finished requests whose results are being copied back on s3: their slot is free for the
  // schedule already, their hierarchy and budget share are released once the copy has landed.
  struct Retiring {
    Request* r;
    ProbState st;
    cudaEvent_t ev;            // recorded on s3 after the request's copy
  };
  std::vector<Retiring> retiring;
  std::unique_ptr<Engine> engine;
  int engine_lmax = 0;
  bool members_dirty = false;
  std::vector<int> fresh;
  std::vector<hn_mg*> running(max_active, nullptr);   // members of the schedule the engine runs
  auto any_running = [&] { return std::any_of(running.begin(), running.end(), [](hn_mg* m) { return m != nullptr; }); };
  // release the requests whose copies have landed (all of them, waiting, with `wait`)
  auto finish_retiring = [&](bool wait) {
    size_t k = 0;
    for (; k < retiring.size(); ++k) {
      Retiring& e = retiring[k];
      if (wait) cudaEventSynchronize(e.ev);
      else if (cudaEventQuery(e.ev) != cudaSuccess) break;      // in order of recording
    }
    for (size_t i = 0; i < k; ++i) {
      Retiring& e = retiring[i];
      Request* r = e.r;
      cudaEventDestroy(e.ev);
      r->b.release();                               // the inputs were consumed at admission
      r->coef.release();
      const size_t hbytes = r->mg->bytes;           // kept for the next request of its size
      void* hmem = detach_block(r->mg->mem, r->mg->mem_base);
      hn_mg_destroy(r->mg);
      if (hmem) { std::lock_guard<std::mutex> lk(cache_mu); cache.give(hmem, hbytes); }
      std::lock_guard<std::mutex> lk(mu);
      r->mg = nullptr;
      r->status = e.st.status;
      r->stats.cycles = e.st.cycles;
      r->stats.outer_iters = e.st.outer_iters;
      r->stats.inner_cycles = e.st.inner_cycles;
      r->stats.status = e.st.status;
      r->stats.relres = e.st.relres;
      r->t_done = now_ns();
      r->stats.solve_ns = r->t_done - r->t_submit;
      r->done = true;
      in_use -= r->bytes;
      ++completed;
      cv_done.notify_all();
      cv_work.notify_all();                         // (memory for the other lane's queue head)
    }
    retiring.erase(retiring.begin(), retiring.begin() + k);
  };
  // A failure stops the server: this lane's requests, the queued ones and those admitted but not
  // yet built fail; the other lane fails its own at the end of its pass.
  auto fail_all = [&](const char* why) {
    cudaStreamSynchronize(s3);
    std::unique_lock<std::mutex> lk(mu);
    // the builders first finish the requests they hold (a failed request may be forgotten by
    // hn_mg_poll at once)
    builder_stop = true;
    for (Request* r : to_build) {
      slots[r->slot] = nullptr;
      r->status = HN_ERR_CUDA;
      r->done = true;
    }
    to_build.clear();
    cv_build.notify_all();
    cv_work.wait(lk, [&] { return building == 0; });
    if (worker_error.empty()) worker_error = why;
    for (Retiring& e : retiring) { e.r->status = HN_ERR_CUDA; e.r->done = true; cudaEventDestroy(e.ev); }
    retiring.clear();
    for (Request* r : built[lane]) {
      if (r->mg) hn_mg_destroy(r->mg);
      r->mg = nullptr;
    }
    built[lane].clear();
    for (Request*& r : slots)
      if (r && r->lane == lane) { r->status = HN_ERR_CUDA; r->done = true; r = nullptr; }
    for (std::deque<Request*>& q : queue) {
      for (Request* r : q) { r->status = HN_ERR_CUDA; r->done = true; }
      q.clear();
    }
    stop = true;
    cv_done.notify_all();
    cv_work.notify_all();
  };
  for (;;) {
    bool admitted_any = false;
    {
      std::unique_lock<std::mutex> lk(mu);
      auto occupied = [&] {
        return std::any_of(slots.begin(), slots.end(), [&](Request* r) { return r != nullptr && r->lane == lane; });
      };
      std::deque<Request*>& q = queue[lane];
      // wake for: the end, an admission that can happen now (a free slot and budget room for the
      // head of the lane's queue), built requests, copies in flight, or running requests
      auto admissible = [&] {
        return !stop && !q.empty() && std::find(slots.begin(), slots.end(), nullptr) != slots.end() &&
               in_use + q.front()->bytes <= budget;
      };
      cv_work.wait(lk, [&] {
        return (stop && !occupied() && retiring.empty()) || admissible() || !built[lane].empty() ||
               !retiring.empty() || any_running();
      });
      if (stop && !occupied() && retiring.empty()) break;
      if (!stop) {
        while (!q.empty()) {
          auto free_slot = std::find(slots.begin(), slots.end(), nullptr);
          if (free_slot == slots.end()) break;
          Request* r = q.front();
          {
            std::lock_guard<std::mutex> ck(cache_mu);
            if (in_use + r->bytes + cache.bytes + scratch_bytes > budget) {
              // cached blocks count against the budget: give back only as many as the head of
              // the queue needs (largest first, the blocks it will reuse last); freeing every
              // cached block would make the next requests of each size allocate anew
              const Params hp = params_from(opts);
              const size_t hb = hierarchy_bytes(r->L, opts.coarse_L, hp.prec, hp.solver);
              const size_t bb = band_bytes(r->L, r->coef.p != nullptr);
              const size_t need = in_use + r->bytes + scratch_bytes;
              cache.release_to(need < budget ? budget - need : 0, hb, bb);
            }
          }
          if (in_use + r->bytes > budget) break;    // FIFO: the head waits for memory
          q.pop_front();
          in_use += r->bytes;
          r->slot = (int)(free_slot - slots.begin());
          *free_slot = r;
          r->t_admit = now_ns();
          to_build.push_back(r);
          admitted_any = true;
        }
        if (admitted_any) cv_build.notify_all();
      }
    }
    // the next iteration of the running requests (the builder assembles admitted requests
    // meanwhile)
    const bool launched = engine && any_running();
    if (launched && engine->launch_iteration() != HN_OK) { fail_all(hn_last_error()); break; }
    const long long t_wait0 = now_ns();
    std::vector<ProbState> st;
    if (launched && (engine->finish_iteration(nullptr) != HN_OK || engine->read_states(st) != HN_OK)) {
      fail_all(hn_last_error());
      break;
    }
    const long long t_ret0 = now_ns();
    {
      std::lock_guard<std::mutex> lk(mu);
      if (launched) ++iterations;
      iterate_ns += t_ret0 - t_wait0;
    }
    // the requests the iteration finished: results back on s3 (the iteration is complete); they
    // leave the schedule now and are released once their copies have landed
    std::vector<std::pair<int, Request*>> done_now;
    if (launched) {
      std::lock_guard<std::mutex> lk(mu);
      for (int q = 0; q < max_active; ++q)
        if (running[q] && st[q].phase == PH_DONE) done_now.emplace_back(q, slots[q]);
    }
    bool copy_failed = false;
    if (!done_now.empty()) {
      for (auto& [q, r] : done_now) {
        const long long N = N_of(r->L);
        if (!r->x.alloc(&host, (size_t)N)) { copy_failed = true; break; }
        if (st[q].status == HN_OK && st[q].bnorm == 0.0) std::fill(r->x.p, r->x.p + N, 0.0);
        else if (cudaMemcpyAsync(r->x.p, r->mg->host.x64, (size_t)N * 8, cudaMemcpyDeviceToHost, s3) != cudaSuccess)
          copy_failed = true;
      }
      if (copy_failed) { fail_all("result copy failed"); break; }
      for (auto& [q, r] : done_now) {
        Retiring e{r, st[q], nullptr};              // an event per request, after all the copies
        if (cudaEventCreateWithFlags(&e.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(e.ev, s3) != cudaSuccess) {
          if (e.ev) cudaEventDestroy(e.ev);
          copy_failed = true;
          break;
        }
        running[q] = nullptr;
        retiring.push_back(e);
        std::lock_guard<std::mutex> lk(mu);
        slots[q] = nullptr;
        members_dirty = true;
        cv_work.notify_all();                       // (a free slot for the other lane)
      }
      if (copy_failed) { fail_all("result copy failed"); break; }
    }
    // with nothing iterating, wait for the copies in flight (their memory may be what the head
    // of the queue waits for)
    finish_retiring(!launched && !retiring.empty());
    const long long t_sched0 = now_ns();
    {
      std::lock_guard<std::mutex> lk(mu);
      retire_ns += t_sched0 - t_ret0;
    }
    // built requests join the schedule (or leave, if their setup failed)
    {
      std::lock_guard<std::mutex> lk(mu);
      for (Request* r : built[lane]) {
        if (!r->mg) {
          r->done = true;
          r->t_done = now_ns();
          in_use -= r->bytes;
          slots[r->slot] = nullptr;
          cv_done.notify_all();
          cv_work.notify_all();                     // (a slot and memory for the other lane)
          continue;
        }
        fresh.push_back(r->slot);
        members_dirty = true;
      }
      built[lane].clear();
    }
    // the schedule of the next iteration: (re)build the engine for the current highest level,
    // refresh its work lists, start the new requests
    int lmax = 0;
    std::vector<hn_mg*> members(max_active, nullptr);
    {
      std::lock_guard<std::mutex> lk(mu);
      for (int q = 0; q < max_active; ++q)
        if (slots[q] && slots[q]->mg && (running[q] || std::find(fresh.begin(), fresh.end(), q) != fresh.end())) {
          members[q] = slots[q]->mg;
          lmax = std::max(lmax, slots[q]->L);
        }
    }
    if (lmax == 0) {
      running = members;
      continue;
    }
    if (!engine || lmax > engine_lmax) {
      // a larger level than the schedule covers: wait until the running requests drain
      bool running_old = false;
      if (engine)
        for (int q = 0; q < max_active; ++q)
          if (members[q] && std::find(fresh.begin(), fresh.end(), q) == fresh.end()) running_old = true;
      if (!engine || !running_old) {
        const int Lcap = std::max(lmax, 8);
        std::vector<long long> caps(kMaxLevel + 1, 0);
        const long long budget_tiles = (long long)(budget / (64 * kTile)) + max_active;
        for (int l = opts.coarse_L; l <= Lcap; ++l)
          caps[l] = std::min<long long>((long long)max_active * (pitch_of(l) / kTile), budget_tiles);
        const long long fine_cap = std::min<long long>((long long)max_active * (pitch_of(Lcap) / kTile), budget_tiles);
        engine.reset(new Engine());
        if (engine->create(params_from(opts), max_active, Lcap, caps, fine_cap, s) != HN_OK) {
          fail_all(hn_last_error());
          break;
        }
        engine->set_iter_limit(UINT_MAX - 1);
        engine->set_top_mask_all();
        engine_lmax = Lcap;
        members_dirty = true;
        // every admitted request (re)starts on the new engine
        fresh.clear();
        for (int q = 0; q < max_active; ++q) if (members[q]) fresh.push_back(q);
      } else {
        // keep the too-large requests out of this iteration
        for (int q = 0; q < max_active; ++q)
          if (members[q] && members[q]->L > engine_lmax) members[q] = nullptr;
      }
    }
    if (members_dirty) {
      if (engine->set_members(members) != HN_OK) { fail_all(hn_last_error()); break; }
      members_dirty = false;
    }
    std::vector<int> start_now;
    for (int q : fresh) if (members[q]) start_now.push_back(q);
    if (!start_now.empty()) {
      if (engine->start(start_now, std::vector<int>(start_now.size(), 0)) != HN_OK ||
          engine->run_init() != HN_OK) { fail_all(hn_last_error()); break; }
      fresh.erase(std::remove_if(fresh.begin(), fresh.end(), [&](int q) { return members[q] != nullptr; }), fresh.end());
    }
    running = members;
    {
      std::lock_guard<std::mutex> lk(mu);
      schedule_ns += now_ns() - t_sched0;
    }
    bool failed_elsewhere = false;                   // the other lane's worker failed
    {
      std::lock_guard<std::mutex> lk(mu);
      failed_elsewhere = stop && !worker_error.empty();
    }
    if (failed_elsewhere) {
      cudaStreamSynchronize(s);
      fail_all("stopped by the other lane's failure");
      break;
    }
  }
  engine.reset();
  cudaStreamSynchronize(s);
  finish_retiring(true);
  cudaStreamDestroy(s3);
  cudaStreamDestroy(s);
}

extern "C" {

hn_status hn_server_create(size_t budget_bytes, int max_active, hn_server** out) {
  clear_error();
  if (!out || budget_bytes == 0 || max_active < 1 || max_active > 4096)
    return set_error(HN_ERR_ARG, "bad server arguments");
  std::unique_ptr<hn_server> srv(new hn_server());
  srv->budget = budget_bytes;
  srv->max_active = max_active;
  srv->slots.assign(max_active, nullptr);
  HN_CUDA(cudaGetDevice(&srv->device));
  hn_server* raw = srv.get();
  for (std::thread& t : srv->builders) t = std::thread([raw] { raw->build_loop(); });
  for (int lane = 0; lane < hn_server::kLanes; ++lane)
    srv->workers[lane] = std::thread([raw, lane] { raw->run(lane); });
  *out = srv.release();
  return HN_OK;
}

hn_status hn_mg_submit(hn_server* srv, int L, const double* cell_coef, const double* b,
                       const hn_mg_opts* opts, unsigned long long* ticket) {
  clear_error();
  if (!srv || !b || !ticket) return set_error(HN_ERR_ARG, "null argument");
  if (L < HN_MIN_LEVEL || L > HN_MAX_LEVEL) return set_error(HN_ERR_ARG, "level %d out of range", L);
  hn_mg_opts o;
  if (opts) o = *opts; else hn_mg_opts_default(&o);
  HN_TRY(validate_opts(o, L));
  HN_TRY(check_band_inputs(L, cell_coef, o.dirichlet_sides));   // here, not on the worker
  std::unique_ptr<Request> r(new Request());
  r->L = L;
  r->lane = L >= hn_server::kLargeLevel ? 1 : 0;
  r->bc = o.dirichlet_sides;
  const long long N = N_of(L), cells = (1LL << L) * (1LL << L);
  if (cell_coef) {
    if (!r->coef.alloc(&srv->host, (size_t)cells)) return set_error(HN_ERR_OOM, "pinned host memory for the coefficients");
    std::memcpy(r->coef.p, cell_coef, (size_t)cells * 8);
  }
  if (!r->b.alloc(&srv->host, (size_t)N)) return set_error(HN_ERR_OOM, "pinned host memory for b");
  std::memcpy(r->b.p, b, (size_t)N * 8);
  r->bytes = request_bytes(L, o);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stop) return set_error(HN_ERR_STATE, "server stopped: %s", srv->worker_error.c_str());
  if (!srv->have_opts) {
    srv->opts = o;
    srv->have_opts = true;
  } else {
    const hn_mg_opts& a = srv->opts;
    if (a.prec != o.prec || a.pre != o.pre || a.post != o.post || a.omega != o.omega ||
        a.coarse_L != o.coarse_L || a.tol != o.tol || a.inner_tol != o.inner_tol ||
        a.max_cycles != o.max_cycles || a.max_outer != o.max_outer || a.inner_max != o.inner_max ||
        a.solver != o.solver || a.coarse_solver != o.coarse_solver)
      return set_error(HN_ERR_ARG, "options differ from the server's (first submit)");
  }
  if (r->bytes > srv->budget) return set_error(HN_ERR_BUDGET, "request needs %zu bytes, budget %zu", r->bytes, srv->budget);
  r->ticket = srv->next_ticket++;
  r->t_submit = now_ns();
  *ticket = r->ticket;
  srv->queue[r->lane].push_back(r.get());
  srv->all[r->ticket] = std::move(r);
  ++srv->submitted;
  srv->cv_work.notify_all();                        // (the workers share the condition)
  return HN_OK;
}

hn_status hn_mg_poll(hn_server* srv, unsigned long long ticket, long long timeout_ns, double* x_out,
                     hn_mg_stats* stats) {
  clear_error();
  if (!srv) return set_error(HN_ERR_ARG, "null server");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->all.find(ticket);
  if (it == srv->all.end()) return set_error(HN_ERR_ARG, "unknown ticket %llu", ticket);
  Request* r = it->second.get();
  if (!r->done) {
    if (timeout_ns == 0) return HN_PENDING;
    if (timeout_ns < 0) {
      srv->cv_done.wait(lk, [&] { return r->done; });
    } else {
      const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns);
      if (!srv->cv_done.wait_until(lk, deadline, [&] { return r->done; }))
        return set_error(HN_ERR_TIMEOUT, "request %llu not finished before the deadline", ticket);
    }
  }
  if (x_out && r->x.p) std::memcpy(x_out, r->x.p, r->x.n * 8);
  if (stats) *stats = r->stats;
  const hn_status st = (hn_status)r->status;
  srv->all.erase(it);
  if (st != HN_OK) set_error(st, "request %llu finished with status %d", ticket, (int)st);
  return st;
}

hn_status hn_server_query(hn_server* srv, hn_server_info* info) {
  clear_error();
  if (!srv || !info) return set_error(HN_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  info->submitted = srv->submitted;
  info->completed = srv->completed;
  info->active = std::count_if(srv->slots.begin(), srv->slots.end(), [](Request* r) { return r != nullptr; });
  info->queued = (long long)(srv->queue[0].size() + srv->queue[1].size());
  info->iterations = srv->iterations;
  info->bytes_in_use = srv->in_use;
  info->budget = srv->budget;
  info->admit_ns = srv->admit_ns;
  info->schedule_ns = srv->schedule_ns;
  info->iterate_ns = srv->iterate_ns;
  info->retire_ns = srv->retire_ns;
  return HN_OK;
}

void hn_server_destroy(hn_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    for (std::deque<Request*>& q : srv->queue) {
      for (Request* r : q) { r->status = HN_ERR_STATE; r->done = true; }
      q.clear();
    }
    srv->cv_work.notify_all();
  }
  for (std::thread& t : srv->workers)
    if (t.joinable()) t.join();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->builder_stop = true;
    srv->cv_build.notify_all();
  }
  for (std::thread& t : srv->builders)
    if (t.joinable()) t.join();
  {
    // the retired requests' device blocks (on the server's device)
    int prev = -1;
    const bool switched = cudaGetDevice(&prev) == cudaSuccess && prev != srv->device &&
                          cudaSetDevice(srv->device) == cudaSuccess;
    std::lock_guard<std::mutex> lk(srv->cache_mu);
    srv->cache.clear();
    if (switched) cudaSetDevice(prev);
  }
  delete srv;
}

}  // extern "C"
