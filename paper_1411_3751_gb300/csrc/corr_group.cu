// Groups of sub-arrays of the C ABI (corr_group_*): several contexts of different N and C with one
// block length, correlated by one persistent tensor-core launch over all their work items.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "corr_ctx.cuh"
#include "corr_internal.cuh"

using namespace corr;
using namespace corr::host;

// =============================================================================================
// Groups of sub-arrays (different N and C, one block length): one persistent tensor-core launch
// covers the work items of every sub-array; per-array tile plans come from a small autotuner.
// =============================================================================================

struct corr_group {
  int n;
  corr_ctx* ctx[kMaxGroupArrays];
  WorkItem* d_items;
  long long n_items;
  cudaGraphExec_t graph;
  int T;
};

namespace {

// autotuner cache: (N, C, T, n_pol, SMs) -> tile plan; optionally mirrored in the file named by the
// CORR_AUTOTUNE_CACHE environment variable (lines "N C T n_pol SMs plan")
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tune;
bool g_tune_loaded = false;

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("CORR_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* fh = std::fopen(path, "r");
  if (!fh) return;
  // lines "N C T n_pol SMs plan" (other lines in the file belong to other tuners)
  char line[256];
  int a, b, c, d, e, p;
  while (std::fgets(line, sizeof line, fh))
    if (std::sscanf(line, "%d %d %d %d %d %d", &a, &b, &c, &d, &e, &p) == 6) g_tune[std::make_tuple(a, b, c, d, e)] = p;
  std::fclose(fh);
}

void tune_store(const std::tuple<int, int, int, int, int>& k, int plan) {
  g_tune[k] = plan;
  const char* path = std::getenv("CORR_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* fh = std::fopen(path, "a");
  if (!fh) return;
  std::fprintf(fh, "%d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
               std::get<4>(k), plan);
  std::fclose(fh);
}

// Group work list: arrays in order of decreasing N (largest tiles first, the short items of small
// arrays last, where they even out the tail), each channel-major. (Merging the arrays in proportion
// to their channel counts, so that HBM-bound small-array items run beside tensor-bound large ones,
// measured the same: 0.638 against 0.641 ms for 32-512 inputs x 2400-109 channels x 4096 samples,
// whose X-engine time is the MMA issue of the 200-512-input members.)
int group_build_items(corr_group* g) {
  std::vector<int> order(g->n);
  for (int i = 0; i < g->n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return g->ctx[x]->L.s.N > g->ctx[y]->L.s.N; });
  std::vector<WorkItem> items;
  for (int i : order) {
    corr_ctx* c = g->ctx[i];
    // group launches run the one-SM mode: a member on plan 2 or 3 joins with plan 0; members of at
    // most 32 inputs as channel groups
    if (channel_group(c->L) > 0) {
      for (int f = 0; f < c->L.s.C; f += channel_group(c->L)) items.push_back(WorkItem{i, f, 0, 0, 128, 0});
      continue;
    }
    const std::vector<F8Tile> t8 = f8_tile_plan(c->L.s.N, c->L.R, c->tile_plan >= 2 ? 0 : c->tile_plan);
    for (int f = 0; f < c->L.s.C; ++f)
      for (const F8Tile& t : t8) items.push_back(WorkItem{i, f, t.c0, t.a0, t.nb, 0});
  }
  WorkItem* d = nullptr;
  if (cudaMalloc(&d, items.size() * sizeof(WorkItem)) != cudaSuccess) {
    cudaGetLastError();
    return fail(CORR_ERR_OOM, "group work list allocation failed");
  }
  cudaError_t e = cudaMemcpy(d, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "group work list upload");
  }
  cudaFree(g->d_items);
  g->d_items = d;
  g->n_items = (long long)items.size();
  return CORR_OK;
}

// One grouped accumulate: one operand-build launch over all arrays, then one persistent X-engine launch.
int group_enqueue(corr_group* g, const uint8_t* const* in, cudaStream_t st) {
  corr_ctx* c0 = g->ctx[0];
  const int T_pad = c0->L.T_pad;
  XengArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int i = 0; i < g->n; ++i)
    if (!g->ctx[i]->d_op)
      return fail(CORR_ERR_STATE, "group member " + std::to_string(i) +
                                      " has no operand scratch (its path was set to FP32 or int8; set a tensor path)");
  // every member's operand build in one launch
  PrepJobDesc jobs[kMaxGroupArrays];
  for (int i = 0; i < g->n; ++i) {
    corr_ctx* c = g->ctx[i];
    jobs[i].s = c->L.s;
    jobs[i].in = in[i];
    jobs[i].T_stride = c->L.T_pad * c->L.K_batch;
    jobs[i].t_base = 0;
    jobs[i].R = c->L.R_buf;
    jobs[i].op = c->d_op;
    jobs[i].s1 = c->d_soff;
    jobs[i].s2 = c->d_soff_auto;
  }
  {
    const bool tb = timer_begin(c0, CORR_KERNEL_UNPACK, st);
    const cudaError_t e = launch_f8_prep_group(jobs, g->n, c0->L.s.T, T_pad, st);
    timer_end(c0, CORR_KERNEL_UNPACK, st, tb);
    if (e != cudaSuccess) return cuda_fail(e, "group operand build");
  }
  for (int i = 0; i < g->n; ++i) {
    corr_ctx* c = g->ctx[i];
    a.a[i].tmap = channel_group(c->L) > 0 ? c->tmap_cp : c->tmap;
    a.a[i].cgroup = channel_group(c->L);
    a.a[i].C = c->L.s.C;
    a.a[i].cross = c->d_cross;
    a.a[i].autos = c->d_autos;
    a.a[i].Bs = c->L.s.Bs;
    a.a[i].N = c->L.s.N;
    a.a[i].npol = c->L.s.npol;
  }
  a.items = g->d_items;
  a.n_items = g->n_items;
  a.T_run = T_pad;
  a.flush_len = flush_for(c0, CORR_PATH_FP8TC);
  a.err = c0->d_err;
  const bool tb = timer_begin(c0, CORR_KERNEL_XENG, st);
  cudaError_t e = launch_f8_xeng(a, c0->num_sms, st);
  timer_end(c0, CORR_KERNEL_XENG, st, tb);
  if (e != cudaSuccess) return cuda_fail(e, "group x-engine launch");
  return CORR_OK;
}

void group_count(corr_group* g) {
  for (int i = 0; i < g->n; ++i) {
    corr_ctx* c = g->ctx[i];
    c->n_cross += c->L.s.T;
    c->n_auto += c->L.s.T;
    c->n_off += c->L.s.T;
    c->n_off_auto += c->L.s.T;
  }
}

}  // namespace

extern "C" {

corr_group* corr_group_create(int n_arrays, const int* n_inputs, const int* n_chans, int n_time_per_block, int n_pol) {
  if (n_arrays < 1 || n_arrays > kMaxGroupArrays || !n_inputs || !n_chans) {
    fail(CORR_ERR_ARG, "corr_group_create: need 1.." + std::to_string(kMaxGroupArrays) + " sub-arrays");
    return nullptr;
  }
  corr_group* g = new (std::nothrow) corr_group{};
  if (!g) {
    fail(CORR_ERR_OOM, "corr_group_create: host allocation");
    return nullptr;
  }
  g->n = n_arrays;
  g->T = n_time_per_block;
  for (int i = 0; i < n_arrays; ++i) {
    g->ctx[i] = corr_create(n_inputs[i], n_chans[i], n_time_per_block, n_pol);
    if (!g->ctx[i]) {
      const std::string msg = corr_last_error();
      corr_group_destroy(g);
      fail(CORR_ERR_ARG, "corr_group_create: sub-array " + std::to_string(i) + ": " + msg);
      return nullptr;
    }
  }
  if (group_build_items(g) != CORR_OK) {
    const std::string msg = corr_last_error();
    corr_group_destroy(g);
    fail(CORR_ERR_OOM, "corr_group_create: " + msg);
    return nullptr;
  }
  return g;
}

corr_ctx* corr_group_member(corr_group* g, int i) {
  if (!g || i < 0 || i >= g->n) {
    fail(CORR_ERR_ARG, "corr_group_member: bad index");
    return nullptr;
  }
  return g->ctx[i];
}

int corr_group_accumulate(corr_group* g, const void* const* d_samples, int mode, void* stream) {
  if (!g || !d_samples) return fail(CORR_ERR_ARG, "corr_group_accumulate: NULL argument");
  for (int i = 0; i < g->n; ++i)
    if (!d_samples[i]) return fail(CORR_ERR_ARG, "corr_group_accumulate: NULL block " + std::to_string(i));
  cudaStream_t st = (cudaStream_t)stream;
  const uint8_t* const* in = reinterpret_cast<const uint8_t* const*>(d_samples);
  if (mode == 1) {
    for (int i = 0; i < g->n; ++i) {
      const int rc = corr_accumulate(g->ctx[i], d_samples[i], stream);
      if (rc != CORR_OK) return rc;
    }
    return CORR_OK;
  }
  if (mode != 0) return fail(CORR_ERR_ARG, "corr_group_accumulate: mode must be 0 (grouped) or 1 (separate)");
  const int rc = group_enqueue(g, in, st);
  if (rc != CORR_OK) return rc;
  group_count(g);
  return CORR_OK;
}

int corr_group_autotune(corr_group* g, const void* const* d_samples, int* plans_out, void* stream) {
  if (!g || !d_samples) return fail(CORR_ERR_ARG, "corr_group_autotune: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load();
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "corr_group_autotune: events");
  int rc = CORR_OK;
  for (int i = 0; i < g->n && rc == CORR_OK; ++i) {
    corr_ctx* c = g->ctx[i];
    const auto key = std::make_tuple(c->L.s.N, c->L.s.C, c->L.s.T, c->L.s.npol, c->num_sms);
    auto it = g_tune.find(key);
    int best = 0;
    if (it != g_tune.end()) {
      best = it->second;
    } else {
      float best_ms = 1e30f;
      for (int plan = 0; plan < 2 && rc == CORR_OK; ++plan) {
        rc = set_tile_plan(c, plan);
        if (rc != CORR_OK) break;
        // one warm-up block, then three timed blocks through the tensor path of this array alone
        for (int rep = 0; rep < 4 && rc == CORR_OK; ++rep) {
          if (rep == 1) cudaEventRecord(e0, st);
          rc = accumulate_device(c, static_cast<const uint8_t*>(d_samples[i]), c->L.s.T, st);
        }
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "corr_group_autotune");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best = plan;
        }
      }
      if (rc == CORR_OK) tune_store(key, best);
    }
    if (rc == CORR_OK) rc = set_tile_plan(c, best);
    if (rc == CORR_OK) rc = corr_reset(c, CORR_WHAT_CROSS | CORR_WHAT_AUTO, stream);
    if (plans_out) plans_out[i] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CORR_OK) return rc;
  // a captured graph refers to the old work list: drop it (corr_group_capture records a new one)
  if (g->graph) {
    cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
  return group_build_items(g);
}

int corr_group_capture(corr_group* g, const void* const* d_samples, void* stream) {
  if (!g || !d_samples) return fail(CORR_ERR_ARG, "corr_group_capture: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return fail(CORR_ERR_ARG, "corr_group_capture: needs a non-default stream");
  bool prof[kMaxGroupArrays];
  for (int i = 0; i < g->n; ++i) {
    prof[i] = g->ctx[i]->profiling;
    g->ctx[i]->profiling = false;  // no timing events inside the graph
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  int rc = CORR_OK;
  if (e == cudaSuccess) {
    rc = group_enqueue(g, reinterpret_cast<const uint8_t* const*>(d_samples), st);
    e = cudaStreamEndCapture(st, &graph);
  }
  for (int i = 0; i < g->n; ++i) g->ctx[i]->profiling = prof[i];
  if (rc != CORR_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "corr_group_capture: capture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "corr_group_capture: instantiate");
  if (g->graph) cudaGraphExecDestroy(g->graph);
  g->graph = exec;
  return CORR_OK;
}

int corr_group_launch(corr_group* g, void* stream) {
  if (!g) return fail(CORR_ERR_ARG, "corr_group_launch: NULL group");
  if (!g->graph) return fail(CORR_ERR_STATE, "corr_group_launch: no captured graph (call corr_group_capture)");
  cudaError_t e = cudaGraphLaunch(g->graph, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "corr_group_launch");
  group_count(g);
  return CORR_OK;
}

int corr_group_destroy(corr_group* g) {
  if (!g) return CORR_OK;
  int rc = CORR_OK;
  if (g->graph) cudaGraphExecDestroy(g->graph);
  cudaFree(g->d_items);
  for (int i = 0; i < g->n; ++i)
    if (g->ctx[i] && corr_destroy(g->ctx[i]) != CORR_OK) rc = CORR_ERR_CUDA;
  delete g;
  return rc;
}

}  // extern "C"
