// batch.cu: many reconstructions of uneven mesh and catalogue sizes in one call (recon_batch_run).
//
// Mocks are grouped by mesh side.  Each size class gets one persistent handle (its buffers,
// twiddle tables and smoothing taps are reused; only the per-mock parameters are re-uploaded), and
// its mocks run back to back on the caller's stream, each iteration loop as one CUDA graph with a
// device-side convergence test.  Before the first mock of a size class, an autotuner times the
// candidate schedules of that class — the x-line FFT tile width, the deposit path and the shift
// path — on that mock and keeps the fastest; the choice is cached for the process.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/recon.h"

namespace {

struct Plan {
  int line_tile = 0;
  int deposit_path = RECON_PATH_DIRECT;
  int shift_path = RECON_PATH_SORTED;
};

std::mutex g_plan_mu;
std::map<int, Plan> g_plans;   // mesh side -> tuned schedule

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  void start() { cudaEventRecord(a, st); }
  float stop() {
    float ms = 0.f;
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
};

// Tune the deposit path of one size class on one mock.  Leaves the handle deposited.
recon_status tune(recon_handle* h, recon_batch_item& it, cudaStream_t st, Plan* plan) {
  Timer t(st);
  float best = 1e30f;
  // deposit path
  for (int path : {RECON_PATH_DIRECT, RECON_PATH_SORTED}) {
    recon_set_option(h, RECON_OPT_DEPOSIT_PATH, path);
    recon_status s = recon_deposit(h, &it.gal, &it.ran);   // warm
    if (s != RECON_OK) return s;
    t.start();
    s = recon_deposit(h, &it.gal, &it.ran);
    const float ms = t.stop();
    if (s != RECON_OK) return s;
    if (ms < best) {
      best = ms;
      plan->deposit_path = path;
    }
  }
  recon_set_option(h, RECON_OPT_DEPOSIT_PATH, plan->deposit_path);
  return recon_deposit(h, &it.gal, &it.ran);
}

}  // namespace

extern "C" recon_status recon_batch_run(recon_batch_item* items, int n_items, void* stream, int autotune) {
  if (n_items < 0 || (n_items > 0 && !items)) return RECON_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> order(n_items);
  for (int i = 0; i < n_items; ++i) {
    order[i] = i;
    items[i].status = RECON_ERR_STATE;
    items[i].n_iter = 0;
    items[i].rel = 0.0;
    items[i].ms = 0.f;
  }
  // size classes in order of first appearance
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return items[a].params.nmesh[0] < items[b].params.nmesh[0];
  });
  recon_status first_error = RECON_OK;
  size_t i = 0;
  while (i < order.size()) {
    const int n = items[order[i]].params.nmesh[0];
    size_t j = i;
    while (j < order.size() && items[order[j]].params.nmesh[0] == n) ++j;
    recon_handle* h = nullptr;
    recon_status s = recon_create(&items[order[i]].params, st, nullptr, 0, &h);
    if (s != RECON_OK) {
      for (size_t k = i; k < j; ++k) items[order[k]].status = s;
      if (first_error == RECON_OK) first_error = s;
      i = j;
      continue;
    }
    Plan plan;
    bool have_plan = false;
    {
      std::lock_guard<std::mutex> lock(g_plan_mu);
      auto f = g_plans.find(n);
      if (f != g_plans.end()) {
        plan = f->second;
        have_plan = true;
      }
    }
    Timer timer(st);
    for (size_t k = i; k < j; ++k) {
      recon_batch_item& it = items[order[k]];
      timer.start();
      s = recon_reconfigure(h, &it.params);
      bool tuned_now = false;
      if (s == RECON_OK && autotune && !have_plan) {
        s = tune(h, it, st, &plan);
        tuned_now = (s == RECON_OK);
      }
      if (s == RECON_OK) {
        recon_set_option(h, RECON_OPT_LINE_TILE, plan.line_tile);
        recon_set_option(h, RECON_OPT_DEPOSIT_PATH, plan.deposit_path);
        recon_set_option(h, RECON_OPT_SHIFT_PATH, plan.shift_path);
        if (!tuned_now) s = recon_deposit(h, &it.gal, &it.ran);
      }
      if (s == RECON_OK) s = recon_smooth(h);
      if (s == RECON_OK) {
        // the x-line tile width is tuned on the iteration of the class's first mock: the first
        // iteration loop runs with each width in turn from the same delta(k)
        if (tuned_now) {
          float best = 1e30f;
          int n_it = 0;
          double rel = 0.0;
          for (int tile : {0, 1}) {
            recon_set_option(h, RECON_OPT_LINE_TILE, tile);
            Timer t(st);
            t.start();
            recon_status si = recon_iterate(h, it.start, it.tol, it.max_iter, &n_it, &rel);
            const float ms = t.stop();
            if (si != RECON_OK && si != RECON_ERR_NOT_CONVERGED) {
              s = si;
              break;
            }
            if (ms < best) {
              best = ms;
              plan.line_tile = tile;
            }
          }
          recon_set_option(h, RECON_OPT_LINE_TILE, plan.line_tile);
        }
      }
      recon_status si = RECON_OK;
      if (s == RECON_OK) {
        si = recon_iterate(h, it.start, it.tol, it.max_iter, &it.n_iter, &it.rel);
        if (si != RECON_OK && si != RECON_ERR_NOT_CONVERGED) s = si;
      }
      if (s == RECON_OK && tuned_now) {
        float best = 1e30f;
        for (int path : {RECON_PATH_DIRECT, RECON_PATH_SORTED}) {
          if (!it.shift_ran) break;
          recon_set_option(h, RECON_OPT_SHIFT_PATH, path);
          Timer t(st);
          t.start();
          recon_status ss = recon_shift(h, &it.ran, 0, it.shift_ran, nullptr, it.out_on_device);
          const float ms = t.stop();
          if (ss != RECON_OK) {
            s = ss;
            break;
          }
          if (ms < best) {
            best = ms;
            plan.shift_path = path;
          }
        }
        recon_set_option(h, RECON_OPT_SHIFT_PATH, plan.shift_path);
        std::lock_guard<std::mutex> lock(g_plan_mu);
        g_plans[n] = plan;
        have_plan = true;
      }
      if (s == RECON_OK && it.shift_gal) s = recon_shift(h, &it.gal, 1, it.shift_gal, nullptr, it.out_on_device);
      if (s == RECON_OK && it.shift_ran) s = recon_shift(h, &it.ran, 0, it.shift_ran, nullptr, it.out_on_device);
      it.ms = timer.stop();
      it.status = (s == RECON_OK) ? si : s;
      if (s != RECON_OK && first_error == RECON_OK) first_error = s;
    }
    recon_destroy(h);
    i = j;
  }
  return first_error;
}

extern "C" recon_status recon_batch_plan(int nmesh, int* line_tile, int* deposit_path, int* shift_path) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto f = g_plans.find(nmesh);
  if (f == g_plans.end()) return RECON_ERR_STATE;
  if (line_tile) *line_tile = f->second.line_tile;
  if (deposit_path) *deposit_path = f->second.deposit_path;
  if (shift_path) *shift_path = f->second.shift_path;
  return RECON_OK;
}
