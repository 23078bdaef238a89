// batch.cu -- many independent registration problems on one GPU.
//
// Serving-style workloads register many image pairs of uneven size. A single
// small pair cannot fill the GPU: its kernels are short and its Krylov loop
// waits on the host for every inner product. reg_solve_batched therefore runs
// the pairs concurrently: worker threads, each driving its own CUDA stream,
// take pairs from a shared queue (largest first) and solve them with contexts
// cached per configuration. Contexts with their own stream replay the Hessian
// matvec as a captured CUDA graph, so a small pair's matvec costs one graph
// launch instead of a few hundred kernel launches.
#include <algorithm>
#include <cstring>
#include <string>
#include <atomic>
#include <map>
#include <numeric>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/reg.h"
#include "internal.h"

using namespace reg;

namespace {

using Key = std::tuple<int, int64_t, int64_t, int64_t, int, int, double, int, int, int>;

Key key_of(const reg_problem& p, int precision) {
  return Key(p.d, p.n[0], p.n[1], p.d == 3 ? p.n[2] : 1, p.n_t, p.n_c, p.beta, p.reg_type, p.stokes, precision);
}

}  // namespace

extern "C" reg_status reg_solve_batched(const reg_problem* problems, int count, int precision,
                                        const reg_solve_opts* opts, reg_solve_report* reports, int workers) {
  if (!problems || count < 0) {
    set_thread_error("reg_solve_batched: bad arguments");
    return REG_EINVAL;
  }
  if (count == 0) return REG_OK;
  if (workers < 1) workers = 1;
  if (workers > count) workers = count;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    set_thread_error("reg_solve_batched: no CUDA device");
    return REG_ECUDA;
  }
  // largest problems first, so the tail of the queue is short work
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  auto size_of = [&](int i) {
    const reg_problem& p = problems[i];
    int64_t N = 1;
    for (int a = 0; a < p.d && a < 3; ++a) N *= p.n[a];
    return N * (int64_t)p.n_t;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return size_of(a) > size_of(b); });
  std::vector<int> status(count, REG_OK);
  std::vector<std::string> errors(count);
  std::atomic<int> next{0};
  auto work = [&]() {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      st = nullptr;
    }
    std::map<Key, reg_ctx*> cache;
    for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
      const int idx = order[i];
      const reg_problem& p = problems[idx];
      Key k = key_of(p, precision);
      reg_ctx* ctx = nullptr;
      auto it = cache.find(k);
      if (it != cache.end()) {
        ctx = it->second;
      } else {
        reg_status s = reg_create(&ctx, p.d, p.n, p.n_t, p.n_c, p.beta, p.reg_type, p.stokes, precision, 0, st);
        if (s != REG_OK) {
          status[idx] = s;
          errors[idx] = reg_last_error(nullptr);
          continue;
        }
        cache[k] = ctx;
      }
      reg_status s = reg_set_images(ctx, p.m_T, p.m_R);
      reg_solve_report rep;
      std::memset(&rep, 0, sizeof(rep));
      if (s == REG_OK) s = reg_solve(ctx, p.v, opts, &rep);
      if (s != REG_OK) errors[idx] = reg_last_error(ctx);
      status[idx] = s;
      rep.status = s;
      if (reports) reports[idx] = rep;
    }
    for (auto& kv : cache) reg_destroy(kv.second);
    if (st) cudaStreamDestroy(st);
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < workers; ++w) pool.emplace_back(work);
  for (auto& t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (status[i] != REG_OK && status[i] != REG_EMAXIT) {
      set_thread_error("reg_solve_batched: problem " + std::to_string(i) + ": " + errors[i]);
      return (reg_status)status[i];
    }
  return REG_OK;
}
