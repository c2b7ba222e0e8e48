// Transforms (forward / inverse / adjoint / spectra export) and kernel timers.
#include <cstring>

#include "ffst_internal.cuh"

namespace ffst {

static cudaEvent_t take_event(ffst_plan_s* p) {
  if (!p->timer.pool.empty()) {
    cudaEvent_t e = p->timer.pool.back();
    p->timer.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Enqueue one launch; with timing on, bracket it with events on its stream.
template <class F>
static cudaError_t timed(ffst_plan_s* p, int kind, double bytes, cudaStream_t s, F&& launch) {
  if (!p->timer.enabled) return launch();
  cudaEvent_t a = take_event(p), b = take_event(p);
  cudaEventRecord(a, s);
  const cudaError_t e = launch();
  cudaEventRecord(b, s);
  p->timer.pending.push_back(Timer::Rec{kind, a, b, bytes});
  return e;
}

static const char* kKindNames[kTimeKinds] = {"img_rows_r2c", "img_cols_fft", "fwd_cols", "fwd_rows_c2r",
                                             "inv_rows_r2c", "inv_cols",     "out_cols_ifft", "out_rows_c2r",
                                             "other"};

static ffst_status check_storage(int storage, const float* scale, const char* fn) {
  if (storage != FFST_STORE_F32 && storage != FFST_STORE_F16 && storage != FFST_STORE_BF16)
    return fail(FFST_ERR_INVALID_ARG, std::string(fn) + ": unknown storage code " + std::to_string(storage));
  if (storage != FFST_STORE_F32 && !scale)
    return fail(FFST_ERR_INVALID_ARG, std::string(fn) + ": plane_scale is required for F16/BF16 storage");
  return FFST_OK;
}

static ffst_status synthesis(ffst_plan_s* p, const void* coeffs, int storage, const float* plane_scale, float* img,
                             cudaStream_t s, bool normalise) {
  const long long plane = (long long)p->M * p->N;
  const int esz = storage == FFST_STORE_F32 ? 4 : 2;
  cudaError_t e;
  for (size_t gi = 0; gi < p->groups.size(); ++gi) {
    const Group& g = p->groups[gi];
    const int n = g.p1 - g.p0;
    e = timed(p, kTimeInvRows, (double)n * plane * esz, s, [&] {
      return launch_rows_r2c(p, p->N, static_cast<const char*>(coeffs) + (long long)g.p0 * plane * esz, storage,
                             plane_scale, g.p0, n, plane, p->d_H, true, 0, 0, 0, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "inverse row pass");
    e = timed(p, kTimeInvCols, 0.0, s, [&] { return launch_inv_cols(p, p->M, g, gi == 0, s); });
    if (e != cudaSuccess) return cuda_fail(e, "inverse column pass");
  }
  e = timed(p, kTimeOutCols, 0.0, s,
            [&] { return launch_cols_fft(p, p->M, p->d_S, p->Hc, p->Hc, true, normalise ? p->d_D : nullptr, s); });
  if (e != cudaSuccess) return cuda_fail(e, "inverse final column pass");
  e = timed(p, kTimeOutRows, 4.0 * plane, s, [&] {
    return launch_rows_c2r(p, p->N, p->d_S, false, p->Hc, p->Hc, 0, 1, img, FFST_STORE_F32, nullptr, 0,
                           1.0f / (float)plane, s);
  });
  if (e != cudaSuccess) return cuda_fail(e, "inverse final row pass");
  return FFST_OK;
}

}  // namespace ffst

using namespace ffst;

extern "C" ffst_status ffst_spectra(ffst_plan_t plan, float* psi, void* stream) {
  if (!plan || !psi) return fail(FFST_ERR_INVALID_ARG, "ffst_spectra: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = timed(plan, kTimeOther, 0.0, s, [&] { return launch_spectra(plan, psi, s); });
  if (e != cudaSuccess) return cuda_fail(e, "ffst_spectra");
  return FFST_OK;
}

extern "C" ffst_status ffst_forward(ffst_plan_t plan, const float* img, void* coeffs, int storage,
                                    float* plane_scale, void* stream) {
  if (!plan || !img || !coeffs) return fail(FFST_ERR_INVALID_ARG, "ffst_forward: NULL argument");
  ffst_status st = check_storage(storage, plane_scale, "ffst_forward");
  if (st != FFST_OK) return st;
  ffst_plan_s* p = plan;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long plane = (long long)p->M * p->N;
  const int esz = storage == FFST_STORE_F32 ? 4 : 2;
  cudaError_t e;
  // fft2 of the image: row R2C into F, then column FFT in place
  e = timed(p, kTimeImgRows, 4.0 * plane, s, [&] {
    return launch_rows_r2c(p, p->N, img, FFST_STORE_F32, nullptr, 0, 1, 0, p->d_F, false, 0, p->Hc, p->Hc, s);
  });
  if (e != cudaSuccess) return cuda_fail(e, "forward image row pass");
  e = timed(p, kTimeImgCols, 0.0, s, [&] { return launch_cols_fft(p, p->M, p->d_F, p->Hc, p->Hc, false, nullptr, s); });
  if (e != cudaSuccess) return cuda_fail(e, "forward image column pass");
  float* partials = storage == FFST_STORE_F32 ? nullptr : p->d_partials;
  // F16 stores c_i * s_i with max |c_i s_i| <= 2^15 < 65504; BF16 normalises to <= 1
  const float target = storage == FFST_STORE_F16 ? 32768.0f : 1.0f;
  for (const Group& g : p->groups) {
    const int n = g.p1 - g.p0;
    e = timed(p, kTimeFwdCols, 0.0, s, [&] { return launch_fwd_cols(p, p->M, g, partials, s); });
    if (e != cudaSuccess) return cuda_fail(e, "forward column pass");
    if (partials) {
      e = timed(p, kTimeOther, 0.0, s, [&] { return launch_plane_scales(p, g, partials, target, plane_scale, s); });
      if (e != cudaSuccess) return cuda_fail(e, "forward plane scales");
    }
    e = timed(p, kTimeFwdRows, (double)n * plane * esz, s, [&] {
      return launch_rows_c2r(p, p->N, p->d_H, true, 0, 0, g.p0, n,
                             static_cast<char*>(coeffs) + (long long)g.p0 * plane * esz, storage, plane_scale, plane,
                             1.0f / (float)plane, s);
    });
    if (e != cudaSuccess) return cuda_fail(e, "forward row pass");
  }
  return FFST_OK;
}

extern "C" ffst_status ffst_inverse(ffst_plan_t plan, const void* coeffs, int storage, const float* plane_scale,
                                    float* img, void* stream) {
  if (!plan || !coeffs || !img) return fail(FFST_ERR_INVALID_ARG, "ffst_inverse: NULL argument");
  ffst_status st = check_storage(storage, plane_scale, "ffst_inverse");
  if (st != FFST_OK) return st;
  return synthesis(plan, coeffs, storage, plane_scale, img, static_cast<cudaStream_t>(stream), true);
}

extern "C" ffst_status ffst_adjoint(ffst_plan_t plan, const void* coeffs, int storage, const float* plane_scale,
                                    float* img, void* stream) {
  if (!plan || !coeffs || !img) return fail(FFST_ERR_INVALID_ARG, "ffst_adjoint: NULL argument");
  ffst_status st = check_storage(storage, plane_scale, "ffst_adjoint");
  if (st != FFST_OK) return st;
  return synthesis(plan, coeffs, storage, plane_scale, img, static_cast<cudaStream_t>(stream), false);
}

extern "C" ffst_status ffst_timing_enable(ffst_plan_t plan, int enable) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_timing_enable: plan is NULL");
  plan->timer.enabled = enable != 0;
  return FFST_OK;
}

static void drain(ffst_plan_s* p) {
  for (auto& r : p->timer.pending) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      p->timer.total_ms[r.kind] += ms;
      p->timer.launches[r.kind] += 1;
      p->timer.bytes[r.kind] += r.bytes;
    }
    p->timer.pool.push_back(r.a);
    p->timer.pool.push_back(r.b);
  }
  p->timer.pending.clear();
}

extern "C" ffst_status ffst_timing_reset(ffst_plan_t plan) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_timing_reset: plan is NULL");
  drain(plan);
  for (int k = 0; k < kTimeKinds; ++k) {
    plan->timer.total_ms[k] = 0.0;
    plan->timer.launches[k] = 0;
    plan->timer.bytes[k] = 0.0;
  }
  return FFST_OK;
}

extern "C" int ffst_timing_kinds(void) { return kTimeKinds; }

extern "C" ffst_status ffst_timing_read(ffst_plan_t plan, int kind, const char** name, double* total_ms,
                                        long long* launches, double* algorithmic_bytes) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_timing_read: plan is NULL");
  if (kind < 0 || kind >= kTimeKinds) return fail(FFST_ERR_INVALID_ARG, "ffst_timing_read: bad kind");
  drain(plan);
  if (name) *name = kKindNames[kind];
  if (total_ms) *total_ms = plan->timer.total_ms[kind];
  if (launches) *launches = plan->timer.launches[kind];
  if (algorithmic_bytes) *algorithmic_bytes = plan->timer.bytes[kind];
  return FFST_OK;
}
