// Batching form: many independent instances of Algorithm 1 stepped together
// by a pool of host threads, in one of two forms.  In the fused form (the
// default) the instances advance one step at a time: the threads run every
// instance's step up to its ODEIM oversampling loop, the loops of all
// instances then run as one launch per pass (launch_odeim_multi, replayed
// from a CUDA graph), and the threads finish the steps.  In the streams form
// each thread runs whole instances, as follows.  Each instance is a context with its own
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
  void (*job)(hyrom_batch*, int) = nullptr;  // what the threads run per instance

  // fused form (HYROM_BATCH_FUSED): the step in two phases around one
  // multi-instance launch of all instances' oversampling loops
  int mode = HYROM_BATCH_FUSED;
  std::vector<int32_t> s_adv;  // the advance's status of the current step
  std::vector<hyrom_step_info> inf;
  std::vector<char> stopped;  // ended by a failure in this call
  std::vector<cudaEvent_t> ev;  // instance i's stream reached its loop
  cudaStream_t sb = nullptr;   // the multi-instance launches
  cudaEvent_t ev_done = nullptr;
  hy::OdeimMulti* mu32 = nullptr;
  hy::OdeimMulti* mu64 = nullptr;
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

// hyrom_step's order of statuses: a failure of the rebuild first, then the
// advance's own condition, then the rebuild's rank information
hyrom_status step_status(hyrom_status sa, hyrom_status su) {
  if (su != HYROM_OK && su != HYROM_ERANK) return su;
  if (sa != HYROM_OK) return sa;
  return su;
}

// the end of instance i's step in the fused form (run_instance's rules)
void end_step(hyrom_batch* b, int i, hyrom_status st) {
  if (st == HYROM_ERANK) st = HYROM_OK;
  if (st != HYROM_OK && b->status[i] == HYROM_OK) b->status[i] = st;
  if (st != HYROM_OK && st != HYROM_ENOTCONV) b->stopped[i] = 1;
  if (b->infos) b->infos[i] = b->inf[i];
}

// Fused form, phase 1: the advance and the rebuild up to the oversampling
// loop, which is left described in the context.
void phase_begin(hyrom_batch* b, int i) {
  if (b->stopped[i]) return;
  hyrom_ctx* c = b->ctx[i];
  hy::ctx_set_defer(c, true);
  hyrom_step_info inf{};
  const hyrom_status sa = hyrom_advance(c, &inf);
  b->s_adv[i] = sa;
  b->inf[i] = inf;
  if (sa != HYROM_OK && sa != HYROM_ENOTCONV && sa != HYROM_ENONPHYS) {
    end_step(b, i, sa);
    return;
  }
  const hyrom_status su = hyrom_update_basis(c, &inf);
  b->inf[i] = inf;
  if (hy::ctx_pending_over(c)) return;
  end_step(b, i, step_status(sa, su));
}

// Fused form, phase 2: after the loops, the rest of the rebuild.
void phase_finish(hyrom_batch* b, int i) {
  hyrom_ctx* c = b->ctx[i];
  if (b->stopped[i] || !hy::ctx_pending_over(c)) return;
  hyrom_status su = HYROM_OK;
  if (cudaStreamWaitEvent((cudaStream_t)hy::ctx_stream(c), b->ev_done, 0) != cudaSuccess) {
    cudaGetLastError();
    su = HYROM_ECUDA;
    hy::ctx_drop_pending(c);
  } else {
    su = hy::ctx_finish_rebuild(c, &b->inf[i]);
  }
  end_step(b, i, step_status((hyrom_status)b->s_adv[i], su));
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
      for (int i : b->groups[j]) b->job(b, i);
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
  b->s_adv.assign(n, HYROM_OK);
  b->inf.assign(n, hyrom_step_info{});
  b->stopped.assign(n, 0);
  b->ev.assign(n, nullptr);
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
  bool ok = cudaGetDevice(&b->device) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->sb, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < n; ++i)
    ok = cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    hyrom_batch_destroy(b);
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

namespace {

// Every thread runs b->job on the groups it takes; returns when all are done.
void run_phase(hyrom_batch* b, void (*job)(hyrom_batch*, int)) {
  std::unique_lock<std::mutex> lk(b->mu);
  b->job = job;
  b->next.store(0, std::memory_order_relaxed);
  b->busy = (int)b->pool.size();
  ++b->gen;
  b->cv_go.notify_all();
  b->cv_done.wait(lk, [&] { return b->busy == 0; });
}

// The fused form's multi-instance launch: the batch stream waits for every
// instance that left a loop, runs the loops (FP32 and FP64 instances apart)
// and records ev_done, which phase_finish makes each instance wait for.
// Returns false on a CUDA error (the pending instances then fail).
bool launch_loops(hyrom_batch* b) {
  std::vector<const hy::OdeimOver*> f32, f64;
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; ++i) {
    if (b->stopped[i]) continue;
    const hy::OdeimOver* o = hy::ctx_pending_over(b->ctx[i]);
    if (!o) continue;
    if (cudaEventRecord(b->ev[i], (cudaStream_t)hy::ctx_stream(b->ctx[i])) != cudaSuccess ||
        cudaStreamWaitEvent(b->sb, b->ev[i], 0) != cudaSuccess)
      return false;
    (hy::ctx_is_f32(b->ctx[i]) ? f32 : f64).push_back(o);
  }
  if (f32.empty() && f64.empty()) return true;
  if (!f32.empty() && !b->mu32 && !(b->mu32 = hy::odeim_multi_create())) return false;
  if (!f64.empty() && !b->mu64 && !(b->mu64 = hy::odeim_multi_create())) return false;
  if (!f32.empty() &&
      hy::launch_odeim_multi<float>(b->mu32, f32.data(), (int)f32.size(), b->sb) < 0)
    return false;
  if (!f64.empty() &&
      hy::launch_odeim_multi<double>(b->mu64, f64.data(), (int)f64.size(), b->sb) < 0)
    return false;
  return cudaEventRecord(b->ev_done, b->sb) == cudaSuccess;
}

}  // namespace

extern "C" hyrom_status hyrom_batch_step(hyrom_batch* b, int32_t nsteps, hyrom_step_info* infos,
                                         int32_t* status) {
  if (!b || nsteps < 0) return HYROM_EINVAL;
  const int n = (int)b->ctx.size();
  b->nsteps = nsteps;
  b->infos = infos;
  std::fill(b->status.begin(), b->status.end(), (int32_t)HYROM_OK);
  if (b->mode == HYROM_BATCH_FUSED) {
    std::fill(b->stopped.begin(), b->stopped.end(), (char)0);
    for (int s = 0; s < nsteps; ++s) {
      run_phase(b, phase_begin);
      if (!launch_loops(b)) {
        cudaGetLastError();
        for (int i = 0; i < n; ++i)
          if (!b->stopped[i] && hy::ctx_pending_over(b->ctx[i])) {
            hy::ctx_drop_pending(b->ctx[i]);
            end_step(b, i, HYROM_ECUDA);
          }
      }
      run_phase(b, phase_finish);
    }
    for (int i = 0; i < n; ++i) hy::ctx_set_defer(b->ctx[i], false);
  } else {
    run_phase(b, run_instance);
  }
  b->infos = nullptr;
  hyrom_status first = HYROM_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = b->status[i];
    if (first == HYROM_OK && b->status[i] != HYROM_OK) first = (hyrom_status)b->status[i];
  }
  return first;
}

extern "C" hyrom_status hyrom_batch_set_mode(hyrom_batch* b, int32_t mode) {
  if (!b || (mode != HYROM_BATCH_STREAMS && mode != HYROM_BATCH_FUSED)) return HYROM_EINVAL;
  b->mode = mode;
  return HYROM_OK;
}

extern "C" int32_t hyrom_batch_tuning(const hyrom_batch* b, int32_t* rows_per_cta,
                                      float* ms_per_step, int32_t n) {
  if (!b) return -1;
  const hy::OdeimMulti* mu = b->mu32 ? b->mu32 : b->mu64;
  if (!mu) {
    if (rows_per_cta) *rows_per_cta = 0;
    for (int c = 0; ms_per_step && c < n; ++c) ms_per_step[c] = -1.f;
    return 0;
  }
  float ms[8];
  int got = hy::odeim_multi_tuning(mu, rows_per_cta, ms, 8);
  for (int c = 0; ms_per_step && c < n && c < got; ++c) ms_per_step[c] = ms[c];
  return got;
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
  if (b->sb) cudaStreamSynchronize(b->sb);
  hy::odeim_multi_free(b->mu32);
  hy::odeim_multi_free(b->mu64);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  if (b->sb) cudaStreamDestroy(b->sb);
  for (hyrom_ctx* c : b->owned_ctx) hyrom_destroy(c);
  for (cudaStream_t st : b->owned_streams) cudaStreamDestroy(st);
  delete b;
}

// n instances in one call: each context on a stream of its own, made here
// and owned by the batch with the contexts (hyrom_batch_destroy releases
// both): the batching form's one-call constructor.
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
