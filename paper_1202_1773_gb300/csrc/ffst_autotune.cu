// Autotuner of a plan's launch configuration.
//
// The knob with the largest measured effect is the plane-group budget (how
// many planes' column-pass intermediates one fused launch holds): larger
// groups mean fewer launches and shorter tails, smaller groups keep more of
// the intermediates in L2.  ffst_plan_autotune times a forward + inverse
// round trip for each candidate budget on the plan's own shape and keeps the
// fastest.  With FFST_AUTOTUNE_CACHE set, results are appended to that text
// file ("<device> <rows> <cols> <scales> <storage> <MB>" per line) and
// ffst_plan reads them back, so a shape is tuned once per machine.
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <mutex>
#include <sstream>

#include "ffst_internal.cuh"

namespace ffst {

static const double kCandidatesMB[] = {32.0, 64.0, 96.0, 128.0, 192.0};
static std::mutex g_cache_mutex;

static std::string cache_path() {
  const char* e = std::getenv("FFST_AUTOTUNE_CACHE");
  return e ? std::string(e) : std::string();
}

static std::string plan_key(const ffst_plan_s* p, int storage) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, p->device);
  std::string name(prop.name);
  for (auto& ch : name)
    if (ch == ' ') ch = '_';
  std::ostringstream os;
  os << name << ' ' << p->M << ' ' << p->N << ' ' << p->j0 << ' ' << storage;
  return os.str();
}

bool autotune_lookup(const ffst_plan_s* p, int storage, double* mb) {
  const std::string path = cache_path();
  if (path.empty()) return false;
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  std::ifstream in(path);
  if (!in) return false;
  const std::string key = plan_key(p, storage);
  std::string line;
  bool found = false;
  while (std::getline(in, line)) {
    const size_t cut = line.rfind(' ');
    if (cut == std::string::npos || line.substr(0, cut) != key) continue;
    const double v = std::atof(line.c_str() + cut + 1);
    if (v > 0.0) {
      *mb = v;  // the last entry for a key wins
      found = true;
    }
  }
  return found;
}

static void autotune_store(const ffst_plan_s* p, int storage, double mb) {
  const std::string path = cache_path();
  if (path.empty()) return;
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  std::ofstream out(path, std::ios::app);
  if (out) out << plan_key(p, storage) << ' ' << mb << '\n';
}

}  // namespace ffst

using namespace ffst;

extern "C" ffst_status ffst_plan_autotune(ffst_plan_t plan, int storage, int reps, double* chosen_mb) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_autotune: plan is NULL");
  if (storage < FFST_STORE_F32 || storage > FFST_STORE_BF16)
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_autotune: unknown storage code");
  if (reps < 1) reps = 3;
  ffst_plan_s* p = plan;
  const size_t plane = (size_t)p->M * p->N;
  const size_t esz = storage == FFST_STORE_F32 ? 4 : 2;
  float* img = nullptr;
  float* out = nullptr;
  float* scale = nullptr;
  void* coeffs = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  auto cleanup = [&] {
    cudaFree(img);
    cudaFree(out);
    cudaFree(scale);
    cudaFree(coeffs);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&img, plane * 4)) != cudaSuccess || (e = cudaMalloc(&out, plane * 4)) != cudaSuccess ||
      (e = cudaMalloc(&scale, p->eta * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&coeffs, plane * esz * p->eta)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "ffst_plan_autotune buffers");
  }
  cudaMemset(img, 0, plane * 4);
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const bool was_timing = p->timer.enabled;
  p->timer.enabled = false;
  const double before = p->group_mb;
  double best_mb = before, best_ms = 1e30;
  for (double mb : kCandidatesMB) {
    if (plan_regroup(p, mb) != FFST_OK) continue;
    bool ok = true;
    for (int q = 0; q < 1 + reps && ok; ++q) {
      if (q == 1) cudaEventRecord(a, s);
      ok = ffst_forward(p, img, coeffs, storage, scale, s) == FFST_OK &&
           ffst_inverse(p, coeffs, storage, scale, out, s) == FFST_OK;
    }
    cudaEventRecord(b, s);
    if (!ok || cudaEventSynchronize(b) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best_ms) {
      best_ms = ms;
      best_mb = mb;
    }
  }
  p->timer.enabled = was_timing;
  const ffst_status st = plan_regroup(p, best_mb);
  cleanup();
  if (st != FFST_OK) return st;
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "ffst_plan_autotune");
  autotune_store(p, storage, best_mb);
  if (chosen_mb) *chosen_mb = best_mb;
  return FFST_OK;
}

extern "C" ffst_status ffst_plan_group_mb(ffst_plan_t plan, double* mb) {
  if (!plan || !mb) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_group_mb: NULL argument");
  *mb = plan->group_mb;
  return FFST_OK;
}
