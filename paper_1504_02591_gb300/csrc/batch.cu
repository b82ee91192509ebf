// batch.cu: many reconstructions of uneven mesh and catalogue sizes in one call (recon_batch_run).
//
// Mocks are grouped by mesh side.  Each size class gets one persistent handle (its buffers and
// twiddle tables are reused; each mock's smoothing and line-of-sight tables are uploaded once, for
// the whole batch).  When every catalogue and output is in device memory, each mock is one CUDA
// graph (its deposit, smoothing, start, the iteration as a conditional WHILE node with the
// device-side stopping test, and its shifts), and the graphs go onto the stream back to back,
// smallest mesh first: the host builds and instantiates mock i + 1's graph while the device runs
// the mocks before it, and waits once, for the whole batch.  Per-mock results and globaltimer stamps
// are written on the device.  With RECON_BATCH_ONE_GRAPH the whole batch is instead one graph built
// before anything runs, with one chain per size class, the chains side by side.  With any catalogue
// or output in host memory the mocks run one after another through the handle API.
//
// Before the first mock of a size class not seen before in this process, the autotuner times the
// class's candidate schedules on that mock (outside the items' times) and keeps the fastest for the
// process: the deposit path (direct atomics or brick-sorted), the x-line FFT tile width (16 or 8
// columns), for N = 512 the k-space kernel family (register-fused or generic staged), for N = 256
// and 384 the FFT radix order (largest or smallest radix first) and the shift path.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/recon.h"
#include "batch_graph.h"

namespace {

struct Plan {
  int line_tile = 0;
  int deposit_path = RECON_PATH_DIRECT;
  int shift_path = RECON_PATH_SORTED;
  int kspace_generic = 0;
  int fft_radix = 0;
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

void apply_plan(recon_handle* h, const Plan& p) {
  recon_set_option(h, RECON_OPT_LINE_TILE, p.line_tile);
  recon_set_option(h, RECON_OPT_DEPOSIT_PATH, p.deposit_path);
  recon_set_option(h, RECON_OPT_SHIFT_PATH, p.shift_path);
  recon_set_option(h, RECON_OPT_KSPACE_GENERIC, p.kspace_generic);
  recon_set_option(h, RECON_OPT_FFT_RADIX, p.fft_radix);
}

// Time the candidate schedules of one size class on one mock (each timed run after a warm run).
recon_status tune(recon_handle* h, recon_batch_item& it, cudaStream_t st, Plan* plan) {
  Timer t(st);
  recon_status s = recon_reconfigure(h, &it.params);
  if (s != RECON_OK) return s;
  const bool uniform = it.params.mean_density_mode == RECON_MEAN_UNIFORM;
  const recon_catalog* ran = uniform ? nullptr : &it.ran;
  float best = 1e30f;
  for (int path : {RECON_PATH_DIRECT, RECON_PATH_SORTED}) {
    recon_set_option(h, RECON_OPT_DEPOSIT_PATH, path);
    if ((s = recon_deposit(h, &it.gal, ran)) != RECON_OK) return s;
    t.start();
    s = recon_deposit(h, &it.gal, ran);
    const float ms = t.stop();
    if (s != RECON_OK) return s;
    if (ms < best) {
      best = ms;
      plan->deposit_path = path;
    }
  }
  recon_set_option(h, RECON_OPT_DEPOSIT_PATH, plan->deposit_path);
  if ((s = recon_deposit(h, &it.gal, ran)) != RECON_OK) return s;
  if ((s = recon_smooth(h)) != RECON_OK) return s;
  // iteration schedules, each on the same delta(k) for a fixed number of updates
  best = 1e30f;
  const int fams = it.params.nmesh[0] == 512 ? 2 : 1;   // the register-fused family exists at N = 512
  // the alternative radix order exists where the option accepts it
  const int orders = recon_set_option(h, RECON_OPT_FFT_RADIX, 1) == RECON_OK ? 2 : 1;
  int n_it = 0;
  double rel = 0.0;
  for (int order = 0; order < orders; ++order) {
    if ((s = recon_set_option(h, RECON_OPT_FFT_RADIX, order)) != RECON_OK) return s;
    for (int fam = 0; fam < fams; ++fam) {
      for (int tile : {0, 1}) {
        recon_set_option(h, RECON_OPT_KSPACE_GENERIC, fam);
        recon_set_option(h, RECON_OPT_LINE_TILE, tile);
        recon_status si = recon_iterate(h, it.start, 0.0, 4, &n_it, &rel);   // warm (and graph build)
        if (si != RECON_OK) return si;
        t.start();
        si = recon_iterate(h, it.start, 0.0, 4, &n_it, &rel);
        const float ms = t.stop();
        if (si != RECON_OK) return si;
        if (ms < best) {
          best = ms;
          plan->line_tile = tile;
          plan->kspace_generic = fam;
          plan->fft_radix = order;
        }
      }
    }
  }
  if ((s = recon_set_option(h, RECON_OPT_FFT_RADIX, plan->fft_radix)) != RECON_OK) return s;
  recon_set_option(h, RECON_OPT_KSPACE_GENERIC, plan->kspace_generic);
  recon_set_option(h, RECON_OPT_LINE_TILE, plan->line_tile);
  // shift path, on the randoms (or the galaxies when there are none)
  const recon_catalog* cat = ran ? ran : &it.gal;
  float* out = ran ? it.shift_ran : it.shift_gal;
  if (out && cat->n > 0) {
    best = 1e30f;
    for (int path : {RECON_PATH_DIRECT, RECON_PATH_SORTED}) {
      recon_set_option(h, RECON_OPT_SHIFT_PATH, path);
      if ((s = recon_shift(h, cat, ran ? 0 : 1, out, nullptr, it.out_on_device)) != RECON_OK) return s;
      t.start();
      s = recon_shift(h, cat, ran ? 0 : 1, out, nullptr, it.out_on_device);
      const float ms = t.stop();
      if (s != RECON_OK) return s;
      if (ms < best) {
        best = ms;
        plan->shift_path = path;
      }
    }
  }
  return RECON_OK;
}

// Mocks of one class one after another through the handle API (host memory allowed).
recon_status run_eager(recon_handle* h, recon_batch_item& it, cudaStream_t st) {
  Timer timer(st);
  timer.start();
  const bool uniform = it.params.mean_density_mode == RECON_MEAN_UNIFORM;
  recon_status s = recon_reconfigure(h, &it.params);
  if (s == RECON_OK) s = recon_deposit(h, &it.gal, uniform ? nullptr : &it.ran);
  if (s == RECON_OK) s = recon_smooth(h);
  recon_status si = RECON_OK;
  if (s == RECON_OK) {
    si = recon_iterate(h, it.start, it.tol, it.max_iter, &it.n_iter, &it.rel);
    if (si != RECON_OK && si != RECON_ERR_NOT_CONVERGED) s = si;
  }
  if (s == RECON_OK && it.shift_gal) s = recon_shift(h, &it.gal, 1, it.shift_gal, nullptr, it.out_on_device);
  if (s == RECON_OK && it.shift_ran && !uniform) s = recon_shift(h, &it.ran, 0, it.shift_ran, nullptr, it.out_on_device);
  it.ms = timer.stop();
  it.status = (s == RECON_OK) ? si : s;
  return s;
}

bool graph_eligible(const recon_batch_item& it) {
  const bool uniform = it.params.mean_density_mode == RECON_MEAN_UNIFORM;
  if (!it.gal.on_device) return false;
  if (!uniform && it.ran.n > 0 && !it.ran.on_device) return false;
  if ((it.shift_gal || it.shift_ran) && !it.out_on_device) return false;
  return it.max_iter >= 1 && it.max_iter <= 1024;
}

struct SizeClass {
  int n = 0;
  std::vector<int> idx;
  recon_handle* h = nullptr;
  recon_status status = RECON_OK;
};

}  // namespace

extern "C" recon_status recon_batch_run(recon_batch_item* items, int n_items, void* stream, int flags) {
  if (n_items < 0 || (n_items > 0 && !items)) return RECON_ERR_INVALID_ARG;
  if (flags & ~(RECON_BATCH_TUNE | RECON_BATCH_ONE_GRAPH)) return RECON_ERR_INVALID_ARG;
  const bool autotune = flags & RECON_BATCH_TUNE, one_graph = flags & RECON_BATCH_ONE_GRAPH;
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < n_items; ++i) {
    items[i].status = RECON_ERR_STATE;
    items[i].n_iter = 0;
    items[i].rel = 0.0;
    items[i].ms = 0.f;
  }
  // size classes in order of mesh side
  std::vector<SizeClass> classes;
  for (int i = 0; i < n_items; ++i) {
    const int n = items[i].params.nmesh[0];
    auto c = std::find_if(classes.begin(), classes.end(), [&](const SizeClass& k) { return k.n == n; });
    if (c == classes.end()) {
      classes.push_back(SizeClass{});
      classes.back().n = n;
      c = classes.end() - 1;
    }
    c->idx.push_back(i);
  }
  std::sort(classes.begin(), classes.end(), [](const SizeClass& a, const SizeClass& b) { return a.n < b.n; });
  recon_status first_error = RECON_OK;
  auto fail = [&](recon_status s) {
    if (first_error == RECON_OK) first_error = s;
  };
  bool all_graph = true;
  for (auto& c : classes) {
    c.status = recon_create(&items[c.idx[0]].params, st, nullptr, 0, &c.h);
    if (c.status != RECON_OK) {
      for (int k : c.idx) items[k].status = c.status;
      fail(c.status);
      c.h = nullptr;
      continue;
    }
    Plan plan;
    bool have = false;
    {
      std::lock_guard<std::mutex> lock(g_plan_mu);
      auto f = g_plans.find(c.n);
      if (f != g_plans.end()) {
        plan = f->second;
        have = true;
      }
    }
    if (autotune && !have) {   // tuning runs before the batch and is charged to no item
      recon_status s = tune(c.h, items[c.idx[0]], st, &plan);
      if (s == RECON_OK) {
        std::lock_guard<std::mutex> lock(g_plan_mu);
        g_plans[c.n] = plan;
      }
    }
    apply_plan(c.h, plan);
    for (int k : c.idx) all_graph = all_graph && graph_eligible(items[k]);
  }

  if (all_graph) {
    // per-mock tables (smoothing taps, node offsets) in one device buffer, uploaded once
    std::vector<float> host;
    struct Tab { size_t taps, off; int t0, ntap; };
    std::vector<Tab> tabs(n_items);
    for (auto& c : classes) {
      if (!c.h) continue;
      for (int k : c.idx) {
        std::vector<float> taps, off;
        rg::config_tables(c.n, &items[k].params, taps, &tabs[k].t0, &tabs[k].ntap, off);
        tabs[k].taps = host.size();
        host.insert(host.end(), taps.begin(), taps.end());
        host.resize((host.size() + 63) & ~size_t(63), 0.f);
        tabs[k].off = host.size();
        host.insert(host.end(), off.begin(), off.end());
        host.resize((host.size() + 63) & ~size_t(63), 0.f);
      }
    }
    float* dtab = nullptr;
    rg::BatchSlot* slots = nullptr;
    cudaGraph_t top = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphExec_t> execs;   // one per mock, launched back to back
    recon_status s = RECON_OK;
    do {
      if (cudaMalloc(&dtab, std::max<size_t>(host.size(), 1) * sizeof(float)) != cudaSuccess ||
          cudaMalloc(&slots, std::max(n_items, 1) * sizeof(rg::BatchSlot)) != cudaSuccess) {
        s = RECON_ERR_OOM;
        break;
      }
      if (cudaMemcpyAsync(dtab, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemsetAsync(slots, 0, n_items * sizeof(rg::BatchSlot), st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        s = RECON_ERR_CUDA;
        break;
      }
      if (one_graph && cudaGraphCreate(&top, 0) != cudaSuccess) {
        s = RECON_ERR_CUDA;
        break;
      }
      for (auto& c : classes) {
        if (!c.h) continue;
        cudaGraphNode_t last = nullptr;
        for (int k : c.idx) {
          rg::BatchJob job{&items[k], dtab + tabs[k].taps, tabs[k].t0, tabs[k].ntap, dtab + tabs[k].off, slots + k};
          if (one_graph) {
            const recon_status sj = rg::batch_append(c.h, top, &last, job);
            if (sj != RECON_OK) {
              items[k].status = sj;
              fail(sj);
            }
            continue;
          }
          // this mock's own graph, on the stream behind the mocks already launched
          cudaGraph_t g = nullptr;
          cudaGraphExec_t ex = nullptr;
          cudaGraphNode_t none = nullptr;
          if (cudaGraphCreate(&g, 0) != cudaSuccess) {
            s = RECON_ERR_CUDA;
            break;
          }
          const recon_status sj = rg::batch_append(c.h, g, &none, job);
          if (sj != RECON_OK) {
            items[k].status = sj;
            fail(sj);
          } else if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess || cudaGraphLaunch(ex, st) != cudaSuccess) {
            s = RECON_ERR_CUDA;
          }
          cudaGraphDestroy(g);
          if (ex) execs.push_back(ex);
          if (s != RECON_OK) break;
        }
        rg::batch_restore(c.h);
        if (s != RECON_OK) break;
      }
      if (s != RECON_OK) {
        cudaStreamSynchronize(st);   // the mocks already launched finish before their buffers go
        break;
      }
      if (one_graph && (cudaGraphInstantiate(&exec, top, 0) != cudaSuccess || cudaGraphLaunch(exec, st) != cudaSuccess)) {
        s = RECON_ERR_CUDA;
        break;
      }
      if (cudaStreamSynchronize(st) != cudaSuccess) {
        s = RECON_ERR_CUDA;
        break;
      }
      std::vector<rg::BatchSlot> res(n_items);
      if (cudaMemcpy(res.data(), slots, n_items * sizeof(rg::BatchSlot), cudaMemcpyDeviceToHost) != cudaSuccess) {
        s = RECON_ERR_CUDA;
        break;
      }
      for (auto& c : classes) {
        if (!c.h) continue;
        for (int k : c.idx) {
          recon_batch_item& it = items[k];
          if (it.status != RECON_ERR_STATE) continue;   // failed while building the graph
          it.n_iter = res[k].it;
          it.rel = res[k].rel;
          it.ms = (float)((double)(res[k].t1 - res[k].t0) * 1e-6);
          if (res[k].flag == 2) it.status = RECON_ERR_NONFINITE;
          else if (it.tol > 0 && it.rel >= it.tol) it.status = RECON_ERR_NOT_CONVERGED;
          else it.status = RECON_OK;
          if (it.status == RECON_ERR_NONFINITE) fail(RECON_ERR_NONFINITE);
        }
      }
    } while (0);
    for (cudaGraphExec_t ex : execs) cudaGraphExecDestroy(ex);
    if (exec) cudaGraphExecDestroy(exec);
    if (top) cudaGraphDestroy(top);
    if (slots) cudaFree(slots);
    if (dtab) cudaFree(dtab);
    if (s != RECON_OK) {
      for (auto& c : classes)
        for (int k : c.idx)
          if (items[k].status == RECON_ERR_STATE) items[k].status = s;
      fail(s);
    }
  } else {
    for (auto& c : classes) {
      if (!c.h) continue;
      for (int k : c.idx) {
        const recon_status s = run_eager(c.h, items[k], st);
        if (s != RECON_OK) fail(s);
      }
    }
  }
  for (auto& c : classes)
    if (c.h) recon_destroy(c.h);
  return first_error;
}

extern "C" recon_status recon_batch_plan(int nmesh, int* line_tile, int* deposit_path, int* shift_path,
                                         int* fft_radix) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto f = g_plans.find(nmesh);
  if (f == g_plans.end()) return RECON_ERR_STATE;
  if (line_tile) *line_tile = f->second.line_tile;
  if (deposit_path) *deposit_path = f->second.deposit_path;
  if (shift_path) *shift_path = f->second.shift_path;
  if (fft_radix) *fft_radix = f->second.fft_radix;
  return RECON_OK;
}
