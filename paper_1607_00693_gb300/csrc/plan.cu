// Plans: the Monte Carlo step of one batch shape (sample the coefficient of
// S samples, upscale every (sample, cell) unit, assemble and solve the
// coarse systems and merge the moments) as a reusable object.  A plan owns
// the step's intermediate device buffers and workspaces, picks its launch
// shapes by timing them on the caller's batch (blocks per SM of the
// persistent upscaling launch; for the FP32 forms, the factorisation engine
// (tensor-core or FMA); for the FP32 form, the separate forward-only launch
// for unoversampled cells or a single launch), and
// replays the whole step as one CUDA graph captured on first use.
#include <vector>

#include "common.cuh"

using namespace stomsfem;

struct stomsfem_plan {
  stomsfem_grid grid;
  stomsfem_field field;
  int S = 0, precision = 0, max_o = 0, refine = 0;
  const int8_t* oversample = nullptr;  // device, owned by the caller
  double *a = nullptr, *Ke = nullptr, *be = nullptr;
  void* wsu = nullptr;
  size_t wsu_bytes = 0;
  void* wsc = nullptr;
  size_t wsc_bytes = 0;
  int blocks_per_sm = 0, split = 1, engine = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // xi, u, mean, m2, count of the graph
  cudaStream_t key_stream = nullptr;
};

static void plan_drop_graph(stomsfem_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
}

static void plan_free(stomsfem_plan* p) {
  if (!p) return;
  plan_drop_graph(p);
  cudaFree(p->a);
  cudaFree(p->Ke);
  cudaFree(p->be);
  cudaFree(p->wsu);
  cudaFree(p->wsc);
  delete p;
}

// One step, stream-ordered (also the body of the captured graph).
static int plan_launch(stomsfem_plan* p, const double* xi, double* u, double* mean, double* m2, double* count,
                       cudaStream_t st) {
  stomsfem_stream_t s = reinterpret_cast<stomsfem_stream_t>(st);
  int rc = stomsfem_sample_coef_precision(&p->grid, &p->field, xi, p->S,
                                          p->precision == STOMSFEM_FP32 ? STOMSFEM_FP32 : STOMSFEM_FP64, p->a, s);
  if (rc) return rc;
  rc = upscale_tuned(&p->grid, p->a, p->oversample, p->max_o, p->S, p->precision, p->refine, p->Ke, p->be, p->wsu,
                     p->wsu_bytes, st, p->blocks_per_sm, p->split, p->engine);
  if (rc) return rc;
  return stomsfem_coarse_solve(&p->grid, p->Ke, p->be, p->S, u, mean, m2, count, p->wsc, p->wsc_bytes, s);
}

extern "C" int stomsfem_plan_create(const stomsfem_grid* grid, const stomsfem_field* field, const int8_t* oversample,
                                    int32_t max_oversample, int32_t S, int32_t precision, int32_t refine_iters,
                                    stomsfem_plan** out) {
  if (!grid || !field || !out) return set_error(STOMSFEM_EINVAL, "NULL argument");
  *out = nullptr;
  if (grid->nf <= 0 || grid->nc <= 0 || grid->nf % grid->nc) return set_error(STOMSFEM_EINVAL, "bad grid");
  if (S < 1) return set_error(STOMSFEM_EINVAL, "S must be >= 1");
  if (precision < 0 || precision > 2) return set_error(STOMSFEM_EINVAL, "bad precision %d", precision);
  if (max_oversample < 0) return set_error(STOMSFEM_EINVAL, "bad max_oversample");
  auto* p = new stomsfem_plan();
  p->grid = *grid;
  p->field = *field;
  p->S = S;
  p->precision = precision;
  p->max_o = oversample ? max_oversample : 0;
  p->refine = refine_iters;
  p->oversample = oversample;
  size_t sb = 0;
  int rc = stomsfem_upscale_workspace_size(grid, p->max_o, precision, &sb, &p->wsu_bytes);
  if (rc == STOMSFEM_OK) rc = stomsfem_coarse_workspace_size(grid, S, &p->wsc_bytes);
  if (rc) {
    delete p;
    return rc;
  }
  const size_t ncell = (size_t)grid->nc * grid->nc;
#define TRY(x)                                   \
  if ((rc = check_cuda((x), #x)) != STOMSFEM_OK) { \
    plan_free(p);                                \
    return rc;                                   \
  }
  TRY(cudaMalloc(&p->a, sizeof(double) * S * (size_t)grid->nf * grid->nf));
  TRY(cudaMalloc(&p->Ke, sizeof(double) * S * ncell * 10));
  TRY(cudaMalloc(&p->be, sizeof(double) * S * ncell * 4));
  TRY(cudaMalloc(&p->wsu, p->wsu_bytes));
  TRY(cudaMalloc(&p->wsc, p->wsc_bytes));
#undef TRY
  *out = p;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_plan_destroy(stomsfem_plan* plan) {
  plan_free(plan);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_plan_tune(stomsfem_plan* p, const double* xi, double* u, int32_t* blocks_per_sm,
                                  int32_t* split_fp32, float* ms_best, stomsfem_stream_t stream) {
  if (!p || !xi || !u) return set_error(STOMSFEM_EINVAL, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  struct Cand {
    int bps, split, engine;
  };
  // FP32 forms: the exact tensor-core factorisation and the FMA one (the
  // two-part split is left out: its rounding exceeds the FP32 form's)
  std::vector<int> engines = {STOMSFEM_ENGINE_AUTO};
  if (upscale_tc_ok(&p->grid, p->max_o, p->precision)) engines = {STOMSFEM_ENGINE_TC3, STOMSFEM_ENGINE_BLOCKED};
  std::vector<Cand> cands;
  for (int eng : engines)
    for (int bps : {0, 2, 1}) {
      cands.push_back({bps, 1, eng});
      if (p->precision == STOMSFEM_FP32 && p->oversample) cands.push_back({bps, 0, eng});
    }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  STOMSFEM_TRY_CUDA(cudaEventCreate(&e0));
  int rc = check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
  float best = -1.f;
  Cand pick{0, 1, STOMSFEM_ENGINE_AUTO};
  for (const Cand& c : cands) {
    if (rc) break;
    p->blocks_per_sm = c.bps;
    p->split = c.split;
    p->engine = c.engine;
    // one untimed run, then two timed
    rc = plan_launch(p, xi, u, nullptr, nullptr, nullptr, st);
    if (rc) break;
    if ((rc = check_cuda(cudaEventRecord(e0, st), "cudaEventRecord"))) break;
    for (int r = 0; r < 2 && !rc; ++r) rc = plan_launch(p, xi, u, nullptr, nullptr, nullptr, st);
    if (rc) break;
    if ((rc = check_cuda(cudaEventRecord(e1, st), "cudaEventRecord"))) break;
    if ((rc = check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize"))) break;
    float ms = 0.f;
    if ((rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime"))) break;
    ms *= 0.5f;
    if (best < 0.f || ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  p->blocks_per_sm = pick.bps;
  p->split = pick.split;
  p->engine = pick.engine;
  plan_drop_graph(p);
  if (rc) return rc;
  if (blocks_per_sm) *blocks_per_sm = pick.bps;
  if (split_fp32) *split_fp32 = pick.split;
  if (ms_best) *ms_best = best;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_plan_step(stomsfem_plan* p, const double* xi, double* u, double* mean, double* m2,
                                  double* count, int32_t use_graph, stomsfem_stream_t stream) {
  if (!p || !xi || !u) return set_error(STOMSFEM_EINVAL, "NULL argument");
  const bool mom = mean || m2 || count;
  if (mom && !(mean && m2 && count)) return set_error(STOMSFEM_EINVAL, "mean, m2 and count must be given together");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the legacy and per-thread default streams cannot be captured
  if (!use_graph || st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread)
    return plan_launch(p, xi, u, mean, m2, count, st);
  const void* key[5] = {xi, u, mean, m2, count};
  bool same = p->exec && p->key_stream == st;
  for (int k = 0; k < 5 && same; ++k) same = p->key[k] == key[k];
  if (!same) {
    plan_drop_graph(p);
    STOMSFEM_TRY_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int rc = plan_launch(p, xi, u, mean, m2, count, st);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    STOMSFEM_TRY_CUDA(ce);
    p->graph = g;
    const int rc2 = check_cuda(cudaGraphInstantiate(&p->exec, p->graph, 0), "cudaGraphInstantiate");
    if (rc2) {
      plan_drop_graph(p);
      return rc2;
    }
    for (int k = 0; k < 5; ++k) p->key[k] = key[k];
    p->key_stream = st;
  }
  STOMSFEM_TRY_CUDA(cudaGraphLaunch(p->exec, st));
  return STOMSFEM_OK;
}

extern "C" int stomsfem_plan_set_choice(stomsfem_plan* p, int32_t blocks_per_sm, int32_t split_fp32,
                                        int32_t engine) {
  if (!p) return set_error(STOMSFEM_EINVAL, "plan is NULL");
  if (blocks_per_sm < 0 || split_fp32 < 0 || split_fp32 > 1 || engine < STOMSFEM_ENGINE_AUTO ||
      engine > STOMSFEM_ENGINE_TC2)
    return set_error(STOMSFEM_EINVAL, "bad launch choice (%d, %d, %d)", blocks_per_sm, split_fp32, engine);
  if (engine != STOMSFEM_ENGINE_AUTO && engine != STOMSFEM_ENGINE_BLOCKED &&
      !upscale_tc_ok(&p->grid, p->max_o, p->precision))
    return set_error(STOMSFEM_EINVAL, "the tensor-core engines need an FP32 form, 4 <= nf/nc and a half bandwidth <= 40");
  p->blocks_per_sm = blocks_per_sm;
  p->split = split_fp32;
  p->engine = engine;
  plan_drop_graph(p);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_plan_info(const stomsfem_plan* p, int32_t* blocks_per_sm, int32_t* split_fp32,
                                  int32_t* engine, int32_t* graph_ready, size_t* device_bytes) {
  if (!p) return set_error(STOMSFEM_EINVAL, "plan is NULL");
  if (blocks_per_sm) *blocks_per_sm = p->blocks_per_sm;
  if (split_fp32) *split_fp32 = p->split;
  if (engine) *engine = upscale_engine_of(&p->grid, p->max_o, p->precision, p->engine);
  if (graph_ready) *graph_ready = p->exec ? 1 : 0;
  if (device_bytes) {
    const size_t ncell = (size_t)p->grid.nc * p->grid.nc;
    *device_bytes = sizeof(double) * p->S * ((size_t)p->grid.nf * p->grid.nf + ncell * 14) + p->wsu_bytes +
                    p->wsc_bytes;
  }
  return STOMSFEM_OK;
}
