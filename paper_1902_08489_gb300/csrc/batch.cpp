// Instance batch: many independent time evolutions (different orbitals,
// electrons, bond dimensions and Hamiltonians) advanced together.
//
// Every instance runs the same integrator code as a single evolution, on one
// of n_workers worker contexts; each worker owns a CUDA stream, a staging
// ring and its caches, and is driven by one host thread that takes the next
// unfinished instance from a shared counter, so uneven instances keep all
// workers busy.  The kernels of different workers overlap on the GPU, which
// fills the device with the many small block contractions that one small
// instance alone cannot.  The calling context's stream is ordered before and
// after the whole batch by events.
#include <atomic>
#include <exception>
#include <thread>

#include "engine.hpp"

namespace tdmps {

Worker::Worker(int precision, size_t ring_bytes) {
  TD_CHECK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  try {
    c = std::make_unique<Context>(st, precision, ring_bytes);
  } catch (...) {
    cudaStreamDestroy(st);
    throw;
  }
}

Worker::~Worker() {
  c.reset();
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
}

namespace {

// Future stream-ordered frees of the state's blocks go to `st`.
void rehome(MPSd& m, cudaStream_t st) {
  for (auto& s : m.sites)
    if (s.data) s.data->st = st;
}

}  // namespace

void evolve_batch(Context& c, const std::vector<BatchItem>& items, int method, int m, bool orth,
                  int n_workers, int* status, std::vector<std::string>& msgs) {
  const int n = (int)items.size();
  msgs.assign(n, std::string());
  if (n == 0) return;
  if (method != 0 && method != 1) throw Error(TDMPS_ERR_INVALID_ARG, "method must be 0 (Krylov) or 1 (RK4)");
  if (n_workers <= 0) n_workers = 8;
  n_workers = std::min(n_workers, n);
  while ((int)c.workers.size() < n_workers)
    c.workers.push_back(std::make_unique<Worker>(c.precision, (size_t)32 << 20));
  for (int w = 0; w < n_workers; ++w) {
    Context& wc = *c.workers[w]->c;
    wc.precision = c.precision;
    wc.n_two_site = c.n_two_site;
    wc.n_one_site = c.n_one_site;
    wc.krylov_fp64 = c.krylov_fp64;
    wc.stats = c.stats;
  }
  // inputs and MPO tables were written on the caller's stream
  cudaEvent_t ready;
  TD_CHECK_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  TD_CHECK_CUDA(cudaEventRecord(ready, c.st));
  for (int w = 0; w < n_workers; ++w) TD_CHECK_CUDA(cudaStreamWaitEvent(c.workers[w]->st, ready, 0));
  TD_CHECK_CUDA(cudaEventDestroy(ready));

  std::vector<MPSd> result(n);
  std::atomic<int> next{0};
  const int device = c.device;
  auto run = [&](int w) {
    Context& wc = *c.workers[w]->c;
    if (cudaSetDevice(device) != cudaSuccess) {
      for (int k; (k = next.fetch_add(1)) < n;) { status[k] = TDMPS_ERR_CUDA; msgs[k] = "cudaSetDevice failed"; }
      return;
    }
    for (int k; (k = next.fetch_add(1)) < n;) {
      const BatchItem& it = items[k];
      try {
        FitOpts o;
        o.D = it.D;
        o.eps = it.eps;
        o.n_two_site = wc.n_two_site;
        o.n_one_site = wc.n_one_site;
        MPSd cur = *it.state;   // shares the input blocks; they stay alive until the join
        for (int s = 0; s < it.n_steps; ++s)
          cur = method == 0 ? krylov_step(wc, *it.H, cur, it.dt, m, orth, o)
                            : rk4_step(wc, *it.H, cur, it.dt, o);
        wc.sync();
        result[k] = std::move(cur);
        status[k] = TDMPS_OK;
      } catch (const Error& e) {
        status[k] = e.code;
        msgs[k] = e.what();
      } catch (const std::bad_alloc&) {
        status[k] = TDMPS_ERR_OOM;
        msgs[k] = "host allocation failed";
      } catch (const std::exception& e) {
        status[k] = TDMPS_ERR_INVALID_ARG;
        msgs[k] = e.what();
      }
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < n_workers; ++w) th.emplace_back(run, w);
  run(0);
  for (auto& t : th) t.join();
  // order the caller's stream after every worker, then hand over the results
  for (int w = 0; w < n_workers; ++w) {
    cudaEvent_t done;
    TD_CHECK_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    TD_CHECK_CUDA(cudaEventRecord(done, c.workers[w]->st));
    TD_CHECK_CUDA(cudaStreamWaitEvent(c.st, done, 0));
    TD_CHECK_CUDA(cudaEventDestroy(done));
    Context& wc = *c.workers[w]->c;
    if (c.stats) {
      wc.collect_stats();
      for (int k = 0; k < TDMPS_KSTAT_COUNT; ++k) {
        c.kstat[k].launches += wc.kstat[k].launches;
        c.kstat[k].ms += wc.kstat[k].ms;
        c.kstat[k].flops += wc.kstat[k].flops;
        c.kstat[k].bytes += wc.kstat[k].bytes;
        wc.kstat[k] = KStat();
      }
    }
  }
  for (int k = 0; k < n; ++k) {
    if (status[k] != TDMPS_OK) continue;
    rehome(result[k], c.st);
    *items[k].state = std::move(result[k]);   // the old blocks are freed on their own stream
  }
}

}  // namespace tdmps
