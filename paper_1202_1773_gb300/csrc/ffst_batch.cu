// Batched transforms over images of uneven sizes, and CUDA-graph capture.
//
// A batch holds one plan per (image size, lane).  Images are spread over
// `lanes` streams by longest-processing-time scheduling (largest eta*M*N
// first, each to the least loaded lane), so transforms of different images
// overlap on the GPU; two images of the same size on the same lane share a
// plan and run one after the other.  Every call forks the lanes from the
// caller's stream with an event and joins them back, so a whole batch can
// be captured into one CUDA graph and replayed.
#include <algorithm>
#include <array>
#include <numeric>

#include "ffst_internal.cuh"

struct ffst_batch_s {
  int n = 0, lanes = 1;
  std::vector<int> rows, cols, scales, eta;  // per image
  std::vector<int> lane;                     // per image
  std::vector<int> plan_of;                  // per image: index into plans
  std::vector<ffst_plan_t> plans;
  std::vector<cudaStream_t> lane_streams;
  std::vector<cudaEvent_t> lane_done;
  cudaEvent_t fork = nullptr;
};

using namespace ffst;

static void free_batch(ffst_batch_s* b) {
  if (!b) return;
  for (auto p : b->plans) ffst_destroy(p);
  for (auto s : b->lane_streams) cudaStreamDestroy(s);
  for (auto e : b->lane_done) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

extern "C" ffst_status ffst_plan_batched(int n, const int* rows, const int* cols, const int* scales, int lanes,
                                         ffst_batch_t* out) {
  if (!out) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_batched: out is NULL");
  *out = nullptr;
  if (n <= 0 || !rows || !cols) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_batched: need n > 0 images with sizes");
  if (lanes < 1 || lanes > 16) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_batched: lanes must be in 1..16");
  ffst_batch_s* b = new ffst_batch_s;
  b->n = n;
  b->lanes = lanes;
  b->rows.assign(rows, rows + n);
  b->cols.assign(cols, cols + n);
  b->scales.resize(n);
  b->eta.resize(n);
  for (int i = 0; i < n; ++i) {
    const int mx = std::max(rows[i], cols[i]);
    int lg = 0;
    while ((1 << (lg + 1)) <= mx) ++lg;
    b->scales[i] = (scales && scales[i] > 0) ? scales[i] : lg / 2;
    b->eta[i] = (1 << (b->scales[i] + 2)) - 3;
  }
  // longest processing time first onto the least loaded lane
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  auto work = [&](int i) { return (double)b->eta[i] * b->rows[i] * b->cols[i]; };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
  std::vector<double> load(lanes, 0.0);
  b->lane.assign(n, 0);
  for (int i : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->lane[i] = l;
    load[l] += work(i);
  }
  // one plan per (rows, cols, scales, lane)
  std::vector<std::array<int, 4>> keys;
  b->plan_of.assign(n, -1);
  for (int i = 0; i < n; ++i) {
    const std::array<int, 4> key{b->rows[i], b->cols[i], b->scales[i], b->lane[i]};
    auto it = std::find(keys.begin(), keys.end(), key);
    if (it != keys.end()) {
      b->plan_of[i] = (int)(it - keys.begin());
      continue;
    }
    ffst_plan_t p = nullptr;
    const ffst_status st = ffst_plan(b->rows[i], b->cols[i], b->scales[i], &p);
    if (st != FFST_OK) {
      free_batch(b);
      return st;
    }
    keys.push_back(key);
    b->plans.push_back(p);
    b->plan_of[i] = (int)b->plans.size() - 1;
  }
  b->lane_streams.resize(lanes);
  b->lane_done.resize(lanes);
  for (int l = 0; l < lanes; ++l) {
    cudaStreamCreateWithFlags(&b->lane_streams[l], cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&b->lane_done[l], cudaEventDisableTiming);
  }
  cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "ffst_plan_batched streams");
  }
  *out = b;
  return FFST_OK;
}

extern "C" ffst_status ffst_batch_autotune(ffst_batch_t b, int storage, int reps) {
  if (!b) return fail(FFST_ERR_INVALID_ARG, "ffst_batch_autotune: batch is NULL");
  // one tuning run per distinct shape, then its configuration on every plan of that shape
  std::vector<int> tuned(b->plans.size(), -1);  // plan index -> index of the tuned plan of its shape
  for (int i = 0; i < b->n; ++i) {
    const int pi = b->plan_of[i];
    if (tuned[pi] >= 0) continue;
    int src = -1;
    for (size_t q = 0; q < b->plans.size() && src < 0; ++q)
      if (tuned[q] == (int)q && b->plans[q]->M == b->rows[i] && b->plans[q]->N == b->cols[i] &&
          b->plans[q]->j0 == b->scales[i])
        src = (int)q;
    if (src < 0) {
      const ffst_status st = ffst_plan_autotune(b->plans[pi], storage, reps, nullptr, nullptr);
      if (st != FFST_OK) return st;
      tuned[pi] = pi;
    } else {
      const ffst_status st = copy_tuning(b->plans[src], b->plans[pi]);
      if (st != FFST_OK) return st;
      tuned[pi] = src;
    }
  }
  return FFST_OK;
}

extern "C" ffst_status ffst_batch_info(ffst_batch_t b, int i, int* rows, int* cols, int* scales, int* num_planes,
                                       int* lane) {
  if (!b) return fail(FFST_ERR_INVALID_ARG, "ffst_batch_info: batch is NULL");
  if (i < 0 || i >= b->n) return fail(FFST_ERR_INVALID_ARG, "ffst_batch_info: image index out of range");
  if (rows) *rows = b->rows[i];
  if (cols) *cols = b->cols[i];
  if (scales) *scales = b->scales[i];
  if (num_planes) *num_planes = b->eta[i];
  if (lane) *lane = b->lane[i];
  return FFST_OK;
}

// mode 0: forward (a = images, b = stacks), 1: inverse, 2: adjoint (a = stacks, b = images)
static ffst_status run_batch(ffst_batch_t bt, int mode, const void* const* a, void* const* b, int storage,
                             float* const* scales, cudaStream_t s) {
  if (!bt || !a || !b) return fail(FFST_ERR_INVALID_ARG, "batched transform: NULL argument");
  if (storage != FFST_STORE_F32 && !scales)
    return fail(FFST_ERR_INVALID_ARG, "batched transform: plane_scales are required for F16/BF16 storage");
  cudaError_t e = cudaEventRecord(bt->fork, s);
  for (int l = 0; l < bt->lanes && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(bt->lane_streams[l], bt->fork, 0);
  if (e != cudaSuccess) return cuda_fail(e, "batched transform fork");
  for (int i = 0; i < bt->n; ++i) {
    ffst_plan_t p = bt->plans[bt->plan_of[i]];
    cudaStream_t ls = bt->lane_streams[bt->lane[i]];
    float* sc = scales ? scales[i] : nullptr;
    ffst_status st;
    if (mode == 0) st = ffst_forward(p, static_cast<const float*>(a[i]), b[i], storage, sc, ls);
    else if (mode == 1) st = ffst_inverse(p, a[i], storage, sc, static_cast<float*>(b[i]), ls);
    else st = ffst_adjoint(p, a[i], storage, sc, static_cast<float*>(b[i]), ls);
    if (st != FFST_OK) return st;
  }
  for (int l = 0; l < bt->lanes && e == cudaSuccess; ++l) {
    e = cudaEventRecord(bt->lane_done[l], bt->lane_streams[l]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, bt->lane_done[l], 0);
  }
  if (e != cudaSuccess) return cuda_fail(e, "batched transform join");
  return FFST_OK;
}

extern "C" ffst_status ffst_forward_batched(ffst_batch_t b, const float* const* imgs, void* const* coeffs, int storage,
                                            float* const* plane_scales, void* stream) {
  return run_batch(b, 0, reinterpret_cast<const void* const*>(imgs), coeffs, storage, plane_scales,
                   static_cast<cudaStream_t>(stream));
}

extern "C" ffst_status ffst_inverse_batched(ffst_batch_t b, const void* const* coeffs, int storage,
                                            float* const* plane_scales, float* const* imgs, void* stream) {
  return run_batch(b, 1, coeffs, reinterpret_cast<void* const*>(imgs), storage, plane_scales,
                   static_cast<cudaStream_t>(stream));
}

extern "C" void ffst_batch_destroy(ffst_batch_t b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_batch(b);
}

extern "C" ffst_status ffst_graph_capture_batched(ffst_batch_t b, int what, const float* const* imgs,
                                                  void* const* coeffs, int storage, float* const* plane_scales,
                                                  float* const* out_imgs, void** graph_exec) {
  if (!b || !graph_exec || (what & 3) == 0) return fail(FFST_ERR_INVALID_ARG, "ffst_graph_capture_batched: bad argument");
  if ((what & 1) && !imgs) return fail(FFST_ERR_INVALID_ARG, "ffst_graph_capture_batched: forward needs imgs");
  if ((what & 2) && !out_imgs) return fail(FFST_ERR_INVALID_ARG, "ffst_graph_capture_batched: inverse needs out_imgs");
  *graph_exec = nullptr;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "ffst_graph_capture_batched stream");
  auto body = [&]() -> ffst_status {
    if (what & 1) {
      const ffst_status st = ffst_forward_batched(b, imgs, coeffs, storage, plane_scales, cs);
      if (st != FFST_OK) return st;
    }
    if (what & 2)
      return ffst_inverse_batched(b, const_cast<const void* const*>(coeffs), storage, plane_scales, out_imgs, cs);
    return FFST_OK;
  };
  // one eager run first: loads modules and sets kernel attributes outside the capture
  ffst_status st = body();
  if (st == FFST_OK && (e = cudaStreamSynchronize(cs)) != cudaSuccess) st = cuda_fail(e, "graph warm-up");
  cudaGraph_t graph = nullptr;
  if (st == FFST_OK) {
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "cudaStreamBeginCapture");
    } else {
      st = body();
      const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (st == FFST_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
    }
  }
  if (st == FFST_OK) {
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
    else *graph_exec = exec;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  return st;
}

extern "C" ffst_status ffst_graph_launch(void* graph_exec, void* stream) {
  if (!graph_exec) return fail(FFST_ERR_INVALID_ARG, "ffst_graph_launch: NULL graph");
  const cudaError_t e = cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return FFST_OK;
}

extern "C" void ffst_graph_destroy(void* graph_exec) {
  if (graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec));
}
