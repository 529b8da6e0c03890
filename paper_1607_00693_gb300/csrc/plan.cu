// Plans: the Monte Carlo step of one batch shape (sample the coefficient of
// S samples, upscale every (sample, cell) unit, assemble and solve the
// coarse systems and merge the moments) as a reusable object.  A plan owns
// the step's intermediate device buffers and workspaces, picks its launch
// shapes by timing them on the caller's batch (for the FP32 forms the
// factorisation engine: two units per warp in column blocks of 8, one unit
// per warp in blocks of 16, or the tensor-core one; the unit order, cells
// fastest or by patch size; for the FP32 form, the separate forward-only
// launch for unoversampled cells or a single launch; blocks per SM of the
// persistent upscaling launch), and replays the whole step as one CUDA
// graph captured on first use, with two timing events around the
// upscaling inside it.
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
  int blocks_per_sm = 0, split = 1, engine = 0, order = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};  // around the upscaling launches of each step
  bool stepped = false;                    // ev recorded at least once
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
  for (cudaEvent_t e : p->ev)
    if (e) cudaEventDestroy(e);
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
  // the timing events: external event nodes when the step is captured, so
  // that every replay records them
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  STOMSFEM_TRY_CUDA(cudaStreamIsCapturing(st, &cs));
  const unsigned evf = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  STOMSFEM_TRY_CUDA(cudaEventRecordWithFlags(p->ev[0], st, evf));
  rc = upscale_tuned(&p->grid, p->a, p->oversample, p->max_o, p->S, p->precision, p->refine, p->Ke, p->be, p->wsu,
                     p->wsu_bytes, st, p->blocks_per_sm, p->split, p->engine, p->order);
  if (rc) return rc;
  STOMSFEM_TRY_CUDA(cudaEventRecordWithFlags(p->ev[1], st, evf));
  p->stepped = true;
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
  TRY(cudaEventCreate(&p->ev[0]));
  TRY(cudaEventCreate(&p->ev[1]));
#undef TRY
  *out = p;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_plan_destroy(stomsfem_plan* plan) {
  plan_free(plan);
  return STOMSFEM_OK;
}

// Time of one step under the plan's current choice: one untimed run, then
// the mean of two timed ones (CUDA events on the stream).
static int plan_time(stomsfem_plan* p, const double* xi, double* u, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                     float* ms) {
  int rc = plan_launch(p, xi, u, nullptr, nullptr, nullptr, st);
  if (rc) return rc;
  STOMSFEM_TRY_CUDA(cudaEventRecord(e0, st));
  for (int r = 0; r < 2; ++r)
    if ((rc = plan_launch(p, xi, u, nullptr, nullptr, nullptr, st))) return rc;
  STOMSFEM_TRY_CUDA(cudaEventRecord(e1, st));
  STOMSFEM_TRY_CUDA(cudaEventSynchronize(e1));
  STOMSFEM_TRY_CUDA(cudaEventElapsedTime(ms, e0, e1));
  *ms *= 0.5f;
  return STOMSFEM_OK;
}

extern "C" int stomsfem_plan_tune(stomsfem_plan* p, const double* xi, double* u, int32_t* blocks_per_sm,
                                  int32_t* split_fp32, float* ms_best, stomsfem_stream_t stream) {
  if (!p || !xi || !u) return set_error(STOMSFEM_EINVAL, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool fp32_forms = p->precision != STOMSFEM_FP64;
  // the candidate values of each choice, the first being the start point
  // (the two-part tensor-core engine is left out: its rounding exceeds the
  // FP32 form's)
  std::vector<int> engines = {STOMSFEM_ENGINE_BLOCKED};
  if (fp32_forms) {
    engines.push_back(STOMSFEM_ENGINE_WIDE);
    if (upscale_engine_ok(&p->grid, p->max_o, p->precision, STOMSFEM_ENGINE_TC3))
      engines.push_back(STOMSFEM_ENGINE_TC3);
  }
  std::vector<int> orders = {STOMSFEM_ORDER_CELL};
  if (p->oversample) orders.push_back(STOMSFEM_ORDER_PATCH);
  std::vector<int> splits = {1};
  if (p->precision == STOMSFEM_FP32 && p->oversample) splits.push_back(0);
  const std::vector<int> bpss = {0, 2, 1};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  STOMSFEM_TRY_CUDA(cudaEventCreate(&e0));
  int rc = check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
  int* field[4] = {&p->engine, &p->order, &p->split, &p->blocks_per_sm};
  const std::vector<int>* vals[4] = {&engines, &orders, &splits, &bpss};
  for (int d = 0; d < 4; ++d) *field[d] = (*vals[d])[0];
  float best = -1.f;
  if (!rc) rc = plan_time(p, xi, u, st, e0, e1, &best);
  // one pass of coordinate descent: each choice in turn, the others fixed
  for (int d = 0; d < 4 && !rc; ++d) {
    const int keep = *field[d];
    int pick = keep;
    for (size_t k = 1; k < vals[d]->size() && !rc; ++k) {
      *field[d] = (*vals[d])[k];
      float ms = 0.f;
      rc = plan_time(p, xi, u, st, e0, e1, &ms);
      if (!rc && ms < best) {
        best = ms;
        pick = *field[d];
      }
    }
    *field[d] = pick;
  }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  plan_drop_graph(p);
  if (rc) return rc;
  if (blocks_per_sm) *blocks_per_sm = p->blocks_per_sm;
  if (split_fp32) *split_fp32 = p->split;
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
                                        int32_t engine, int32_t order) {
  if (!p) return set_error(STOMSFEM_EINVAL, "plan is NULL");
  if (blocks_per_sm < 0 || split_fp32 < 0 || split_fp32 > 1 || engine < STOMSFEM_ENGINE_AUTO ||
      engine > STOMSFEM_ENGINE_WIDE || (order != STOMSFEM_ORDER_CELL && order != STOMSFEM_ORDER_PATCH))
    return set_error(STOMSFEM_EINVAL, "bad launch choice (%d, %d, %d, %d)", blocks_per_sm, split_fp32, engine,
                     order);
  if (engine != STOMSFEM_ENGINE_AUTO && !upscale_engine_ok(&p->grid, p->max_o, p->precision, engine))
    return set_error(STOMSFEM_EINVAL,
                     "engine %d is not offered here (WIDE and the tensor-core engines: FP32 forms; tensor-core: "
                     "4 <= nf/nc and a half bandwidth <= 40)", engine);
  p->blocks_per_sm = blocks_per_sm;
  p->split = split_fp32;
  p->engine = engine;
  p->order = order;
  plan_drop_graph(p);
  return STOMSFEM_OK;
}

extern "C" int stomsfem_plan_info(const stomsfem_plan* p, int32_t* blocks_per_sm, int32_t* split_fp32,
                                  int32_t* engine, int32_t* order, int32_t* graph_ready, size_t* device_bytes) {
  if (!p) return set_error(STOMSFEM_EINVAL, "plan is NULL");
  if (blocks_per_sm) *blocks_per_sm = p->blocks_per_sm;
  if (split_fp32) *split_fp32 = p->split;
  if (engine) *engine = upscale_engine_of(&p->grid, p->max_o, p->precision, p->engine);
  if (order) *order = p->order;
  if (graph_ready) *graph_ready = p->exec ? 1 : 0;
  if (device_bytes) {
    const size_t ncell = (size_t)p->grid.nc * p->grid.nc;
    *device_bytes = sizeof(double) * p->S * ((size_t)p->grid.nf * p->grid.nf + ncell * 14) + p->wsu_bytes +
                    p->wsc_bytes;
  }
  return STOMSFEM_OK;
}

extern "C" int stomsfem_plan_upscale_ms(stomsfem_plan* p, float* ms) {
  if (!p || !ms) return set_error(STOMSFEM_EINVAL, "NULL argument");
  if (!p->stepped) return set_error(STOMSFEM_EINVAL, "the plan has not run a step");
  STOMSFEM_TRY_CUDA(cudaEventSynchronize(p->ev[1]));
  STOMSFEM_TRY_CUDA(cudaEventElapsedTime(ms, p->ev[0], p->ev[1]));
  return STOMSFEM_OK;
}
