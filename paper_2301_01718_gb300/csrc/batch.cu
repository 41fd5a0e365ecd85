// Batching form: many independent instances of Algorithm 1 stepped together
// by a pool of host threads.  Each instance is a context with its own
// stream; a thread takes one instance at a time and runs its steps, so the
// GPU holds the kernels of up to `threads` instances at once.  Small
// instances cannot fill 152 SMs alone and spend much of a step in launch
// latency and host round trips; overlapping them fills the gaps.  The
// instances are handed out largest first (longest-processing-time order by
// device footprint, which grows with dofs x window), so the last ones to
// finish are the short ones.  Per instance nothing changes: the same kernels
// run in the same order on its stream, so its results are the same bits as
// stepping it alone.  Instances that share a stream form one group, stepped
// by one thread in turn: a stream being captured into an instance's CUDA
// graph must see no other instance's work.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/hyrom.h"
#include "internal.h"

struct hyrom_batch {
  std::vector<hyrom_ctx*> ctx;
  // contexts and streams made by hyrom_init_batch, released with the batch
  std::vector<hyrom_ctx*> owned_ctx;
  std::vector<cudaStream_t> owned_streams;
  std::vector<std::vector<int>> groups;  // instances sharing a stream, largest groups first
  int device = 0;
  std::vector<std::thread> pool;

  std::mutex mu;
  std::condition_variable cv_go, cv_done;
  uint64_t gen = 0;  // bumped per hyrom_batch_step call
  int busy = 0;      // threads still working on the current call
  bool quit = false;

  // the current call
  std::atomic<int> next{0};
  int nsteps = 0;
  hyrom_step_info* infos = nullptr;
  std::vector<int32_t> status;
};

namespace {

// One instance: nsteps steps in order; a failure other than a Newton solve
// that hit its cap (whose state is still advanced) ends the instance's run.
// The rank information HYROM_ERANK (a complete step with m_eff < m) is not a
// failure and is not reported (m_eff is in the step info).
void run_instance(hyrom_batch* b, int i) {
  hyrom_step_info info{};
  int32_t first = HYROM_OK;
  for (int s = 0; s < b->nsteps; ++s) {
    hyrom_status st = hyrom_step(b->ctx[i], &info);
    if (st == HYROM_ERANK) st = HYROM_OK;
    if (st != HYROM_OK && first == HYROM_OK) first = st;
    if (st != HYROM_OK && st != HYROM_ENOTCONV) break;
  }
  b->status[i] = first;
  if (b->infos) b->infos[i] = info;
}

void worker(hyrom_batch* b) {
  cudaSetDevice(b->device);
  uint64_t seen = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(b->mu);
      b->cv_go.wait(lk, [&] { return b->quit || b->gen != seen; });
      if (b->quit) return;
      seen = b->gen;
    }
    const int ng = (int)b->groups.size();
    for (int j; (j = b->next.fetch_add(1, std::memory_order_relaxed)) < ng;)
      for (int i : b->groups[j]) run_instance(b, i);
    std::lock_guard<std::mutex> lk(b->mu);
    if (--b->busy == 0) b->cv_done.notify_all();
  }
}

}  // namespace

extern "C" hyrom_status hyrom_batch_create(hyrom_ctx* const* ctxs, int32_t n, int32_t threads,
                                           hyrom_batch** out) {
  if (!out || !ctxs || n <= 0 || threads < 0) return HYROM_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return HYROM_EINVAL;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j)
      if (ctxs[i] == ctxs[j]) return HYROM_EINVAL;
  hyrom_batch* b = new (std::nothrow) hyrom_batch;
  if (!b) return HYROM_ENOMEM;
  b->ctx.assign(ctxs, ctxs + n);
  b->status.assign(n, HYROM_OK);
  // group by stream (first appearance order), then largest groups first
  std::vector<void*> streams;
  std::vector<size_t> gbytes;
  for (int i = 0; i < n; ++i) {
    void* st = hy::ctx_stream(ctxs[i]);
    size_t g = 0;
    while (g < streams.size() && streams[g] != st) ++g;
    if (g == streams.size()) {
      streams.push_back(st);
      b->groups.emplace_back();
      gbytes.push_back(0);
    }
    b->groups[g].push_back(i);
    gbytes[g] += hyrom_device_bytes(ctxs[i]);
  }
  std::vector<int> perm(b->groups.size());
  for (size_t g = 0; g < perm.size(); ++g) perm[g] = (int)g;
  std::stable_sort(perm.begin(), perm.end(),
                   [&](int x, int y) { return gbytes[x] > gbytes[y]; });
  std::vector<std::vector<int>> sorted;
  for (int g : perm) sorted.push_back(b->groups[g]);
  b->groups.swap(sorted);
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return HYROM_ECUDA;
  }
  // default: half the host's hardware threads, at most 8 (a thread spins on
  // the CPU while its instance's stream drains; more threads than half the
  // cores starved the launching ones)
  const int hw = (int)std::thread::hardware_concurrency();
  const int ng = (int)b->groups.size();
  const int nt = std::min(ng, threads == 0 ? std::max(1, std::min(8, hw / 2)) : (int)threads);
  try {
    for (int t = 0; t < nt; ++t) b->pool.emplace_back(worker, b);
  } catch (...) {
    hyrom_batch_destroy(b);
    return HYROM_ENOMEM;
  }
  *out = b;
  return HYROM_OK;
}

extern "C" hyrom_status hyrom_batch_step(hyrom_batch* b, int32_t nsteps, hyrom_step_info* infos,
                                         int32_t* status) {
  if (!b || nsteps < 0) return HYROM_EINVAL;
  const int n = (int)b->ctx.size();
  {
    std::unique_lock<std::mutex> lk(b->mu);
    b->nsteps = nsteps;
    b->infos = infos;
    std::fill(b->status.begin(), b->status.end(), (int32_t)HYROM_OK);
    b->next.store(0, std::memory_order_relaxed);
    b->busy = (int)b->pool.size();
    ++b->gen;
    b->cv_go.notify_all();
    b->cv_done.wait(lk, [&] { return b->busy == 0; });
    b->infos = nullptr;
  }
  hyrom_status first = HYROM_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = b->status[i];
    if (first == HYROM_OK && b->status[i] != HYROM_OK) first = (hyrom_status)b->status[i];
  }
  return first;
}

extern "C" int32_t hyrom_batch_threads(const hyrom_batch* b) {
  return b ? (int32_t)b->pool.size() : 0;
}

extern "C" void hyrom_batch_destroy(hyrom_batch* b) {
  if (!b) return;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->quit = true;
  }
  b->cv_go.notify_all();
  for (auto& t : b->pool)
    if (t.joinable()) t.join();
  for (hyrom_ctx* c : b->owned_ctx) hyrom_destroy(c);
  for (cudaStream_t st : b->owned_streams) cudaStreamDestroy(st);
  delete b;
}

// n instances in one call: each context on a stream of its own, made here
// and owned by the batch with the contexts (hyrom_batch_destroy releases
// both).  The scope table's hyrom_init_batch.
extern "C" hyrom_status hyrom_init_batch(const hyrom_config* cfgs, const double* const* q0,
                                         int32_t q0_on_host, int32_t n, int32_t threads,
                                         hyrom_ctx** ctxs_out, hyrom_batch** out) {
  if (!cfgs || !q0 || !out || n <= 0 || threads < 0) return HYROM_EINVAL;
  std::vector<hyrom_ctx*> ctxs;
  std::vector<cudaStream_t> streams;
  auto undo = [&](hyrom_status s) {
    for (hyrom_ctx* c : ctxs) hyrom_destroy(c);
    for (cudaStream_t st : streams) cudaStreamDestroy(st);
    return s;
  };
  for (int i = 0; i < n; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return undo(HYROM_ECUDA);
    }
    streams.push_back(st);
    hyrom_ctx* c = nullptr;
    const hyrom_status s = hyrom_init(&cfgs[i], q0[i], q0_on_host, (void*)st, &c);
    if (s != HYROM_OK) return undo(s);
    ctxs.push_back(c);
  }
  hyrom_batch* b = nullptr;
  const hyrom_status s = hyrom_batch_create(ctxs.data(), n, threads, &b);
  if (s != HYROM_OK) return undo(s);
  b->owned_ctx = ctxs;
  b->owned_streams = streams;
  if (ctxs_out)
    for (int i = 0; i < n; ++i) ctxs_out[i] = ctxs[i];
  *out = b;
  return HYROM_OK;
}
