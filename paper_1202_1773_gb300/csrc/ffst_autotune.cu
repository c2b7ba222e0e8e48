// Autotuner of a plan's launch configuration, per shape and storage type.
//
// Stage 1, the plane-group budget (how many planes' column-pass
// intermediates one fused launch holds): larger groups mean fewer launches
// and shorter tails, smaller groups keep more of the intermediates in L2.
// Stage 2, at those budgets, the kernel configuration of each direction:
// fused plane-pass launches or separate row and column launches, and for
// separate launches the row-FFT tile and radix schedule (ffst_rows.cu
// variants: 16 elements per thread with radix 16 x 16 x 4 at length 1024,
// two rows per team in packed FP32 pairs, or 32 elements per thread with
// radix 32 x 32 and one exchange); for the inverse also the number of plane
// chunks of its sum (1, 2, 4, 8, 16 or the plan's default).  Every candidate is timed on the plan's own shape, the
// forward and the inverse apart, and the fastest kept.  With
// FFST_AUTOTUNE_CACHE set, results are appended to that text file, one line
// "<device> <rows> <cols> <scales> <storage> <forward MB> <inverse MB>
// <fuse fwd> <row fwd> <fuse inv> <row inv> <inverse chunks>", and
// ffst_plan reads them back, so a shape is tuned once per machine (lines
// with only the two budgets are read as well).
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

bool autotune_lookup(const ffst_plan_s* p, int storage, TuneConfig* cfg) {
  const std::string path = cache_path();
  if (path.empty()) return false;
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  std::ifstream in(path);
  if (!in) return false;
  const std::string key = plan_key(p, storage);
  std::string line;
  bool found = false;
  while (std::getline(in, line)) {
    if (line.compare(0, key.size() + 1, key + " ") != 0) continue;
    std::istringstream rest(line.substr(key.size() + 1));
    TuneConfig c;
    if (!(rest >> c.fwd_mb >> c.inv_mb) || c.fwd_mb <= 0.0 || c.inv_mb <= 0.0) continue;
    int ff = -1, rf = -1, fi = -1, ri = -1, ns = -1;
    if (rest >> ff >> rf >> fi >> ri >> ns) {
      c.fuse_fwd = ff;
      c.row_fwd = rf;
      c.fuse_inv = fi;
      c.row_inv = ri;
      c.inv_split = ns;
    }
    *cfg = c;  // the last entry for a key wins
    found = true;
  }
  return found;
}

static void autotune_store(const ffst_plan_s* p, int storage, double fwd_mb, double inv_mb) {
  const std::string path = cache_path();
  if (path.empty()) return;
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  std::ofstream out(path, std::ios::app);
  if (out)
    out << plan_key(p, storage) << ' ' << fwd_mb << ' ' << inv_mb << ' ' << p->fuse_fwd << ' ' << p->row_fwd << ' '
        << p->fuse_inv << ' ' << p->row_inv << ' ' << p->inv_split << '\n';
}

}  // namespace ffst

using namespace ffst;

extern "C" ffst_status ffst_plan_autotune(ffst_plan_t plan, int storage, int reps, double* fwd_mb, double* inv_mb) {
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
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  auto cleanup = [&] {
    cudaFree(img);
    cudaFree(out);
    cudaFree(scale);
    cudaFree(coeffs);
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
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
  for (auto& x : ev) cudaEventCreate(&x);
  const bool was_timing = p->timer.enabled;
  p->timer.enabled = false;
  // forward and inverse are timed apart: each direction keeps its own best budget
  double best_f = p->group_mb, best_i = p->group_mb_inv, tf = 1e30, ti = 1e30;
  for (double mb : kCandidatesMB) {
    if (plan_regroup(p, mb, mb) != FFST_OK) continue;
    bool ok = true;
    float f_ms = 0.f, i_ms = 0.f;
    for (int q = 0; q < 1 + reps && ok; ++q) {
      cudaEventRecord(ev[0], s);
      ok = ffst_forward(p, img, coeffs, storage, scale, s) == FFST_OK;
      cudaEventRecord(ev[1], s);
      ok = ok && ffst_inverse(p, coeffs, storage, scale, out, s) == FFST_OK;
      cudaEventRecord(ev[2], s);
      if (!ok || cudaEventSynchronize(ev[2]) != cudaSuccess) {
        ok = false;
        break;
      }
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, ev[0], ev[1]);
      cudaEventElapsedTime(&b, ev[1], ev[2]);
      if (q > 0) {  // the first round trip is the warm-up
        f_ms += a;
        i_ms += b;
      }
    }
    if (!ok) continue;
    if (f_ms < tf) {
      tf = f_ms;
      best_f = mb;
    }
    if (i_ms < ti) {
      ti = i_ms;
      best_i = mb;
    }
  }
  ffst_status st = plan_regroup(p, best_f, best_i);
  if (st != FFST_OK) {
    p->timer.enabled = was_timing;
    cleanup();
    return st;
  }

  // stage 2: kernel configuration of each direction at the chosen budgets
  auto time_dir = [&](bool fwd) -> float {  // summed ms of reps calls after one warm-up; < 0 on failure
    float tot = 0.f;
    for (int q = 0; q < 1 + reps; ++q) {
      cudaEventRecord(ev[0], s);
      const bool ok = fwd ? ffst_forward(p, img, coeffs, storage, scale, s) == FFST_OK
                          : ffst_inverse(p, coeffs, storage, scale, out, s) == FFST_OK;
      cudaEventRecord(ev[1], s);
      if (!ok || cudaEventSynchronize(ev[1]) != cudaSuccess) return -1.f;
      float a = 0.f;
      cudaEventElapsedTime(&a, ev[0], ev[1]);
      if (q > 0) tot += a;
    }
    return tot;
  };
  const int L = p->N / 2;
  const bool native = p->bl_rows.n == 0;
  const bool fusable = fused_supported(p->M, p->N);
  struct Cand {
    int fuse, row, split;
  };
  std::vector<Cand> fc;
  if (fusable) fc.push_back({1, 0, 0});
  for (int v = 0; v <= kRowVariants - 1; ++v)
    if (v == 0 || (native && row_variant_ok(L, v, true))) fc.push_back({0, v, 0});
  Cand bf = {p->fuse_fwd, p->row_fwd, 0};
  float tb = 1e30f;
  for (const Cand& c : fc) {
    p->fuse_fwd = c.fuse;
    p->row_fwd = c.row;
    const float t = time_dir(true);
    if (t >= 0.f && t < tb) {
      tb = t;
      bf = c;
    }
  }
  p->fuse_fwd = bf.fuse;
  p->row_fwd = bf.row;
  std::vector<int> splits = {p->inv_split_default};
  for (int n : {1, 2, 4, 8, 16})
    if (n != p->inv_split_default) splits.push_back(n);
  std::vector<Cand> ic;
  for (int n : splits) {
    if (fusable) ic.push_back({1, 0, n});
    for (int v = 0; v <= kRowVariants - 1; ++v)
      if (v == 0 || (native && row_variant_ok(L, v, false))) ic.push_back({0, v, n});
  }
  Cand bi = {p->fuse_inv, p->row_inv, p->inv_split};
  tb = 1e30f;
  for (const Cand& c : ic) {
    p->fuse_inv = c.fuse;
    p->row_inv = c.row;
    if (plan_set_inv_split(p, c.split) != FFST_OK) continue;
    const float t = time_dir(false);
    if (t >= 0.f && t < tb) {
      tb = t;
      bi = c;
    }
  }
  p->fuse_inv = bi.fuse;
  p->row_inv = bi.row;
  st = plan_set_inv_split(p, bi.split);
  p->timer.enabled = was_timing;
  cleanup();
  if (st != FFST_OK) return st;
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "ffst_plan_autotune");
  autotune_store(p, storage, best_f, best_i);
  if (fwd_mb) *fwd_mb = best_f;
  if (inv_mb) *inv_mb = best_i;
  return FFST_OK;
}

namespace ffst {

// Give plan q the launch configuration of plan p (same shape).
ffst_status copy_tuning(const ffst_plan_s* p, ffst_plan_s* q) {
  if (p == q) return FFST_OK;
  ffst_status st = plan_regroup(q, p->group_mb, p->group_mb_inv);
  if (st != FFST_OK) return st;
  q->fuse_fwd = p->fuse_fwd;
  q->fuse_inv = p->fuse_inv;
  q->row_fwd = p->row_fwd;
  q->row_inv = p->row_inv;
  return plan_set_inv_split(q, p->inv_split);
}

}  // namespace ffst

extern "C" ffst_status ffst_plan_group_mb(ffst_plan_t plan, double* fwd_mb, double* inv_mb) {
  if (!plan || !fwd_mb || !inv_mb) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_group_mb: NULL argument");
  *fwd_mb = plan->group_mb;
  *inv_mb = plan->group_mb_inv;
  return FFST_OK;
}
