// Transforms (forward / inverse / adjoint / spectra export) and kernel timers.
//
// Schedule of one transform on a plan with plane groups g = 0..G-1 (each
// group's column-pass intermediate fits in L2; two buffers alternate):
//   forward:  fft2(img) -> F;  cols(0);  [cols(g) | rows(g-1)] for g = 1..G-1;  rows(G-1)
//   inverse:  S = 0;  rows(0);  [rows(g) | cols(g-1)] for g = 1..G-1;  cols(G-1);  ifft2(S)
// where [a | b] is one fused launch whose blocks interleave both passes
// (square images); other sizes run the same passes as separate launches.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "ffst_blue.cuh"

namespace ffst {

// NVTX range around one launch (profilers show the kernel kind and, as the
// payload, its plane group; -1 outside the group loops).  Header-only NVTX:
// without an attached tool each call is a null check.
struct NvtxRange {
  NvtxRange(const char* name, int group) {
    nvtxEventAttributes_t a{};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    a.payloadType = NVTX_PAYLOAD_TYPE_INT32;
    a.payload.iValue = group;
    nvtxRangePushEx(&a);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

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

static const char* kKindNames[kTimeKinds] = {"img_rows_r2c", "img_cols_fft", "fwd_cols",      "fwd_rows_c2r",
                                             "inv_rows_r2c", "inv_cols",     "out_cols_ifft", "out_rows_c2r",
                                             "fwd_fused",    "inv_fused",    "fwd_sched",     "inv_sched",
                                             "other"};

// Enqueue one launch inside an NVTX range named for its kind (payload: the
// plane group); with timing on, bracket it with events on its stream.
template <class F>
static cudaError_t timed(ffst_plan_s* p, int kind, double bytes, cudaStream_t s, F&& launch, int group = -1) {
  NvtxRange range(kKindNames[kind], group);
  if (!p->timer.enabled) return launch();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone) return launch();
  cudaEvent_t a = take_event(p), b = take_event(p);
  cudaEventRecord(a, s);
  const cudaError_t e = launch();
  cudaEventRecord(b, s);
  p->timer.pending.push_back(Timer::Rec{kind, a, b, bytes});
  return e;
}

static ffst_status check_storage(int storage, const float* scale, const char* fn) {
  if (storage != FFST_STORE_F32 && storage != FFST_STORE_F16 && storage != FFST_STORE_BF16)
    return fail(FFST_ERR_INVALID_ARG, std::string(fn) + ": unknown storage code " + std::to_string(storage));
  if (storage != FFST_STORE_F32 && !scale)
    return fail(FFST_ERR_INVALID_ARG, std::string(fn) + ": plane_scale is required for F16/BF16 storage");
  return FFST_OK;
}

static float2* hbuf(const ffst_plan_s* p, size_t g) { return p->d_H + (g % 2) * p->h_elems; }

// Fused plane-pass launches (square powers of two) per direction, as the
// plan's kernel configuration selects (ffst_plan_set_kernels).
static bool use_fused(const ffst_plan_s* p) { return p->fuse_inv && fused_supported(p->M, p->N); }
static bool use_fused_fwd(const ffst_plan_s* p) { return p->fuse_fwd && fused_supported(p->M, p->N); }



// Persistent schedule when the plan has one and its mode selects it.
static bool use_sched(const ffst_plan_s* p) { return p->sched.on && p->sched_mode != 0; }

// Row kernel variant of a direction's standalone plane row passes; the fused
// and persistent launches (and so the standalone edge groups of a fused
// schedule) use 0.
static int fwd_row_variant(const ffst_plan_s* p) {
  return use_fused_fwd(p) || use_sched(p) || p->bl_rows.n ? 0 : p->row_fwd;
}
static int inv_row_variant(const ffst_plan_s* p) {
  return use_fused(p) || use_sched(p) || p->bl_rows.n ? 0 : p->row_inv;
}
static const float2* row_table(const ffst_plan_s* p, int variant) {
  return variant >= 2 ? p->d_tw_rows32 : p->d_tw_rows;  // 2 and 3: the (L, 32) pass table
}

static Group all_planes(const ffst_plan_s* p) { return Group{p->pr0, p->pr1, 0, 0, p->total_items}; }

// Fused per-plane statistics and shrinkage of a forward (ffst_forward_stats).
struct StatsOpts {
  int shrink = 0;               // 0 none, 1 soft, 2 hard
  const float* thresh = nullptr;
  bool stats = false;           // accumulate sum |c| per (plane, row block)
  int cplx_part = -1;           // one-sided complex stack (Sec. 3.8.2): 0 real parts, 1 imaginary parts
};

// Line passes at the plan's sizes: native FFT lines, or generic (Bluestein)
// lines for a dimension without them (ffst_blue.cuh).  Generic sizes never
// take the fused or persistent launches (fused_supported).
static cudaError_t rows_r2c(const ffst_plan_s* p, const R2CArgs& a, int nplanes, cudaStream_t s, int variant = 0) {
  return p->bl_rows.n ? launch_blue_rows_r2c(p->bl_rows, a, nplanes, s)
                      : launch_rows_r2c(p->N / 2, a, nplanes, s, variant);
}

static cudaError_t rows_c2r(const ffst_plan_s* p, const C2RArgs& a, int nplanes, cudaStream_t s, int variant = 0) {
  return p->bl_rows.n ? launch_blue_rows_c2r(p->bl_rows, a, nplanes, s)
                      : launch_rows_c2r(p->N / 2, a, nplanes, s, variant);
}

static cudaError_t cols_fft(const ffst_plan_s* p, float2* buf, bool inverse, const float* scale_tab, cudaStream_t s,
                            int nsum = 1, long long sstride = 0) {
  return p->bl_cols.n
             ? launch_blue_cols_fft(p->bl_cols, buf, p->Hc, p->Hc, inverse, scale_tab, s, nsum, sstride)
             : launch_cols_fft(p->M, buf, p->Hc, p->Hc, inverse, scale_tab, p->d_tw_cols, s, nsum, sstride,
                               (long long)(nsum > 1 ? nsum : 1) * p->M * p->Hc * (long long)sizeof(float2), p->d_err);
}

static cudaError_t fwd_cols(const ffst_plan_s* p, const FwdColsArgs& a, int nitems, cudaStream_t s) {
  return p->bl_cols.n ? launch_blue_fwd_cols(p->bl_cols, a, nitems, s) : launch_fwd_cols(p->M, a, nitems, s);
}

static cudaError_t inv_cols(const ffst_plan_s* p, const InvColsArgs& a, cudaStream_t s) {
  return p->bl_cols.n ? launch_blue_inv_cols(p->bl_cols, a, s) : launch_inv_cols(p->M, a, s);
}

static FwdColsArgs fwd_cols_args(const ffst_plan_s* p, const Group& g, float2* H, float* partials,
                                 const StatsOpts* so = nullptr) {
  FwdColsArgs a;
  a.F = p->d_F;
  a.Hc = p->Hc;
  a.planes = p->d_planes;
  a.items = p->d_items + g.item0;
  a.rng = p->d_rng;
  a.H = H;
  a.w = p->win;
  a.tw = p->d_tw_cols;
  a.partials = partials ? partials + g.item0 : nullptr;
  a.gain = 1.0f / (kR2CGain * (float)p->M * (float)p->N);
  a.tmaps = p->d_tmaps;
  a.odd = (so && so->cplx_part == 1) ? 1 : 0;
  a.F_bytes = (long long)p->M * p->Hc * (long long)sizeof(float2);
  a.H_bytes = p->h_elems * (long long)sizeof(float2);
  a.err = p->d_err;
  return a;
}


static C2RArgs plane_c2r_args(const ffst_plan_s* p, const Group& g, const float2* H, void* coeffs, int storage,
                              const float* plane_scale, const StatsOpts* so = nullptr) {
  const long long plane = (long long)p->M * p->N;
  C2RArgs a;
  a.src = H;
  a.planes = p->d_planes;
  a.c0 = 0;
  a.W = 0;
  a.ld = 0;
  a.M = p->M;
  a.plane0 = g.p0;
  // the caller's stack holds the active planes [pr0, pr1)
  a.dst = static_cast<char*>(coeffs) + (long long)(g.p0 - p->pr0) * plane * (storage == FFST_STORE_F32 ? 4 : 2);
  a.dst_plane_stride = plane;
  a.st = storage;
  a.plane_scale = plane_scale;
  a.scale = 1.0f;  // fwd_cols already applied 1/(M N) (and the R2C gain)
  a.tw = row_table(p, fwd_row_variant(p));
  a.rtw = p->d_rtw;
  a.shrink = so ? so->shrink : 0;
  a.thresh = so ? so->thresh : nullptr;
  a.abs_partials = (so && so->stats) ? p->d_abs_partials : nullptr;
  a.rbx = p->row_blocks;
  a.cplx = 0;
  if (so && so->cplx_part >= 0) {  // planar complex stack [eta][2][M][N]: this part of each plane
    a.cplx = 1;
    a.dst = static_cast<char*>(coeffs) + ((long long)(g.p0 - p->pr0) * 2 + so->cplx_part) * plane * sizeof(float);
    a.dst_plane_stride = 2 * plane;
  }
  a.src_bytes = p->h_elems * (long long)sizeof(float2);
  {  // the planes [g.p0, g.p1) of the caller's stack from a.dst
    const long long es = a.cplx ? 4 : (storage == FFST_STORE_F32 ? 4 : 2);
    a.dst_bytes = g.p1 > g.p0 ? ((long long)(g.p1 - g.p0 - 1) * a.dst_plane_stride + plane) * es : 0;
  }
  a.err = p->d_err;
  return a;
}

static R2CArgs plane_r2c_args(const ffst_plan_s* p, const Group& g, const void* coeffs, int storage,
                              const float* plane_scale, float2* H, bool cplx = false) {
  const long long plane = (long long)p->M * p->N;
  R2CArgs a;
  a.src = static_cast<const char*>(coeffs) + (long long)(g.p0 - p->pr0) * plane * (storage == FFST_STORE_F32 ? 4 : 2);
  a.src_plane_stride = plane;
  a.st = storage;
  a.plane_scale = plane_scale;
  a.cplx = cplx ? 1 : 0;
  if (cplx) {  // real parts of the planar complex stack [eta][2][M][N]
    a.src = static_cast<const char*>(coeffs) + (long long)(g.p0 - p->pr0) * 2 * plane * sizeof(float);
    a.src_plane_stride = 2 * plane;
  }
  a.plane0 = g.p0;
  a.M = p->M;
  a.dst = H;
  a.planes = p->d_planes_inv;
  a.c0 = 0;
  a.W = 0;
  a.ld = 0;
  a.tw = row_table(p, inv_row_variant(p));
  a.rtw = p->d_rtw;
  {  // the planes [g.p0, g.p1) of the caller's stack from a.src
    const long long es = cplx ? 4 : (storage == FFST_STORE_F32 ? 4 : 2);
    a.src_bytes = g.p1 > g.p0 ? ((long long)(g.p1 - g.p0 - 1) * a.src_plane_stride + plane) * es : 0;
  }
  a.dst_bytes = p->h_elems * (long long)sizeof(float2);
  a.err = p->d_err;
  return a;
}

static InvColsArgs inv_cols_args(const ffst_plan_s* p, const Group& g, const float2* H) {
  InvColsArgs a;
  a.H = H;
  a.Hc = p->Hc;
  a.planes = p->d_planes_inv;
  a.p0 = g.p0;
  a.p1 = g.p1;
  a.rng = p->d_rng;
  a.S = p->d_S;
  a.sstride = (long long)p->M * p->Hc;
  a.npanels = (p->Hc + p->P - 1) / p->P;
  a.eta = p->eta;
  a.nsplit = p->inv_split;
  a.k0 = g.p1 > g.p0 ? inv_part(p, g.p0) : 0;
  a.nchunks = g.p1 > g.p0 ? inv_part(p, g.p1 - 1) - a.k0 + 1 : 0;
  a.w = p->win;
  a.tw = p->d_tw_cols;
  a.tmaps = p->d_tmaps_inv;
  a.err = p->d_err;
  a.H_bytes = p->h_elems * (long long)sizeof(float2);
  a.S_bytes = (long long)p->inv_split * p->M * p->Hc * (long long)sizeof(float2);
  return a;
}

static ffst_status analysis(ffst_plan_s* p, const float* img, void* coeffs, int storage, float* plane_scale,
                            cudaStream_t s, const StatsOpts* so = nullptr) {
  const long long plane = (long long)p->M * p->N;
  const int esz = storage == FFST_STORE_F32 ? 4 : 2;
  cudaError_t e;
  // fft2 of the image: row R2C into F, then column FFT in place
  R2CArgs ia;
  std::memset(&ia, 0, sizeof(ia));
  ia.src = img;
  ia.st = FFST_STORE_F32;
  ia.M = p->M;
  ia.dst = p->d_F;
  ia.c0 = 0;
  ia.W = p->Hc;
  ia.ld = p->Hc;
  ia.tw = p->d_tw_rows;
  ia.rtw = p->d_rtw;
  ia.src_bytes = plane * (long long)sizeof(float);
  ia.dst_bytes = (long long)p->M * p->Hc * (long long)sizeof(float2);
  ia.err = p->d_err;
  e = timed(p, kTimeImgRows, 4.0 * plane, s, [&] { return rows_r2c(p, ia, 1, s); });
  if (e != cudaSuccess) return cuda_fail(e, "forward image row pass");
  e = timed(p, kTimeImgCols, 0.0, s,
            [&] { return cols_fft(p, p->d_F, false, nullptr, s); });
  if (e != cudaSuccess) return cuda_fail(e, "forward image column pass");

  float* partials = storage == FFST_STORE_F32 ? nullptr : p->d_partials;
  // F16 stores c_i * s_i with max |c_i s_i| <= 2^15 < 65504; BF16 normalises to <= 1
  const float target = storage == FFST_STORE_F16 ? 32768.0f : 1.0f;
  auto scales = [&](size_t gi) -> cudaError_t {
    if (!partials) return cudaSuccess;
    return timed(p, kTimeOther, 0.0, s,
                 [&] { return launch_plane_scales(p, p->groups[gi], partials, target, plane_scale, s); });
  };
  const size_t G = p->groups.size();
  if (use_sched(p)) {
    const Group all = all_planes(p);
    e = timed(p, kTimeFwdSched, (double)p->eta * plane * esz, s, [&] {
      return launch_fwd_sched(p, fwd_cols_args(p, all, nullptr, partials, so),
                              plane_c2r_args(p, all, nullptr, coeffs, storage, nullptr, so), target,
                              partials ? plane_scale : nullptr, s);
    });
  } else if (use_fused_fwd(p)) {
    e = timed(p, kTimeFwdCols, 0.0, s, [&] {
      return fwd_cols(p, fwd_cols_args(p, p->groups[0], hbuf(p, 0), partials, so), p->groups[0].nitems, s);
    });
    if (e == cudaSuccess) e = scales(0);
    for (size_t g = 1; g < G && e == cudaSuccess; ++g) {
      const Group& cg = p->groups[g];
      const Group& rg = p->groups[g - 1];
      const double by = (double)(rg.p1 - rg.p0) * plane * esz;
      e = timed(p, kTimeFwdFused, by, s, [&] {
        return launch_fwd_fused(p->M, fwd_cols_args(p, cg, hbuf(p, g), partials, so), cg.nitems,
                                plane_c2r_args(p, rg, hbuf(p, g - 1), coeffs, storage, plane_scale, so), rg.p1 - rg.p0,
                                s);
      }, (int)g);
      if (e == cudaSuccess) e = scales(g);
    }
    if (e == cudaSuccess) {
      const Group& rg = p->groups[G - 1];
      e = timed(p, kTimeFwdRows, (double)(rg.p1 - rg.p0) * plane * esz, s, [&] {
        return rows_c2r(p, plane_c2r_args(p, rg, hbuf(p, G - 1), coeffs, storage, plane_scale, so),
                               rg.p1 - rg.p0, s, fwd_row_variant(p));
      });
    }
  } else {
    for (size_t g = 0; g < G && e == cudaSuccess; ++g) {
      const Group& gr = p->groups[g];
      // group g's buffer is hbuf(g) as in the fused schedule (the TMA maps point there)
      e = timed(p, kTimeFwdCols, 0.0, s, [&] {
        return fwd_cols(p, fwd_cols_args(p, gr, hbuf(p, g), partials, so), gr.nitems, s);
      });
      if (e == cudaSuccess) e = scales(g);
      if (e == cudaSuccess)
        e = timed(p, kTimeFwdRows, (double)(gr.p1 - gr.p0) * plane * esz, s, [&] {
          return rows_c2r(p, plane_c2r_args(p, gr, hbuf(p, g), coeffs, storage, plane_scale, so), gr.p1 - gr.p0,
                                 s, fwd_row_variant(p));
        });
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "forward plane passes");
  return FFST_OK;
}

// Plane passes of the inverse (Sec. 3.3): S_k = sum over the active planes of
// chunk k of psi_i * fft2(c_i), the half spectrum in the plan's partial
// accumulators.
static ffst_status synthesis_planes(ffst_plan_s* p, const void* coeffs, int storage, const float* plane_scale,
                                    cudaStream_t s, bool cplx) {
  const long long plane = (long long)p->M * p->N;
  const int esz = storage == FFST_STORE_F32 ? 4 : 2;
  const long long spec = (long long)p->M * p->Hc;
  cudaError_t e = cudaMemsetAsync(p->d_S, 0, sizeof(float2) * (size_t)(p->inv_split * spec), s);
  if (e != cudaSuccess) return cuda_fail(e, "inverse accumulator clear");
  const size_t G = p->groups_inv.size();
  if (use_sched(p)) {
    const Group all = all_planes(p);
    e = timed(p, kTimeInvSched, (double)p->eta * plane * esz, s, [&] {
      return launch_inv_sched(p, plane_r2c_args(p, all, coeffs, storage, plane_scale, nullptr, cplx),
                              inv_cols_args(p, all, nullptr), s);
    });
  } else if (use_fused(p)) {
    {
      const Group& rg = p->groups_inv[0];
      e = timed(p, kTimeInvRows, (double)(rg.p1 - rg.p0) * plane * esz, s, [&] {
        return rows_r2c(p, plane_r2c_args(p, rg, coeffs, storage, plane_scale, hbuf(p, 0), cplx), rg.p1 - rg.p0,
                               s, inv_row_variant(p));
      });
    }
    for (size_t g = 1; g < G && e == cudaSuccess; ++g) {
      const Group& rg = p->groups_inv[g];
      const Group& cg = p->groups_inv[g - 1];
      e = timed(p, kTimeInvFused, (double)(rg.p1 - rg.p0) * plane * esz, s, [&] {
        return launch_inv_fused(p->M, plane_r2c_args(p, rg, coeffs, storage, plane_scale, hbuf(p, g), cplx), rg.p1 - rg.p0,
                                inv_cols_args(p, cg, hbuf(p, g - 1)), s);
      }, (int)g);
    }
    if (e == cudaSuccess)
      e = timed(p, kTimeInvCols, 0.0, s, [&] {
        return inv_cols(p, inv_cols_args(p, p->groups_inv[G - 1], hbuf(p, G - 1)), s);
      });
  } else {
    for (size_t g = 0; g < G && e == cudaSuccess; ++g) {
      const Group& gr = p->groups_inv[g];
      e = timed(p, kTimeInvRows, (double)(gr.p1 - gr.p0) * plane * esz, s, [&] {
        return rows_r2c(p, plane_r2c_args(p, gr, coeffs, storage, plane_scale, hbuf(p, g), cplx), gr.p1 - gr.p0,
                               s, inv_row_variant(p));
      });
      if (e == cudaSuccess)
        e = timed(p, kTimeInvCols, 0.0, s,
                  [&] { return inv_cols(p, inv_cols_args(p, gr, hbuf(p, g)), s); });
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "inverse plane passes");
  return FFST_OK;
}

// ifft2 of a half spectrum held as nsum partial sums (M x Hc apart) in buf,
// added in index order, times 1/sum_i psi_i^2 when `normalise`; the column
// pass works in place in buf.
static ffst_status synthesis_finish(ffst_plan_s* p, float2* buf, int nsum, bool normalise, float* img,
                                    cudaStream_t s) {
  const long long plane = (long long)p->M * p->N;
  const long long spec = (long long)p->M * p->Hc;
  cudaError_t e = timed(p, kTimeOutCols, 0.0, s, [&] {
    return cols_fft(p, buf, true, normalise ? p->d_invD : nullptr, s, nsum, spec);
  });
  if (e != cudaSuccess) return cuda_fail(e, "inverse final column pass");
  C2RArgs oa;
  std::memset(&oa, 0, sizeof(oa));
  oa.src = buf;
  oa.c0 = 0;
  oa.W = p->Hc;
  oa.ld = p->Hc;
  oa.M = p->M;
  oa.dst = img;
  oa.st = FFST_STORE_F32;
  oa.scale = 1.0f / (kR2CGain * (float)plane);
  oa.cplx = 0;
  oa.tw = p->d_tw_rows;
  oa.rtw = p->d_rtw;
  oa.src_bytes = spec * (long long)sizeof(float2);
  oa.dst_bytes = plane * (long long)sizeof(float);
  oa.err = p->d_err;
  e = timed(p, kTimeOutRows, 4.0 * plane, s, [&] { return rows_c2r(p, oa, 1, s); });
  if (e != cudaSuccess) return cuda_fail(e, "inverse final row pass");
  return FFST_OK;
}

static ffst_status synthesis(ffst_plan_s* p, const void* coeffs, int storage, const float* plane_scale, float* img,
                             cudaStream_t s, bool normalise, bool cplx = false) {
  const ffst_status st = synthesis_planes(p, coeffs, storage, plane_scale, s, cplx);
  if (st != FFST_OK) return st;
  return synthesis_finish(p, p->d_S, p->inv_split, normalise, img, s);
}

// out = sum_k S_k (k = 0 .. nsum-1 in order), n complex values per sum.
__global__ void k_sum_partials(const float2* __restrict__ S, int nsum, long long n, float2* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float2 acc = __ldcs(&S[i]);
    for (int k = 1; k < nsum; ++k) {
      const float2 y = __ldcs(&S[i + k * n]);
      acc = make_float2(acc.x + y.x, acc.y + y.y);
    }
    out[i] = acc;
  }
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
  NvtxRange range("ffst_forward", -1);
  return analysis(plan, img, coeffs, storage, plane_scale, static_cast<cudaStream_t>(stream));
}

extern "C" ffst_status ffst_forward_stats(ffst_plan_t plan, const float* img, void* coeffs, int storage,
                                          float* plane_scale, int shrink, const float* thresh, float* mean_abs,
                                          void* stream) {
  if (!plan || !img || !coeffs) return fail(FFST_ERR_INVALID_ARG, "ffst_forward_stats: NULL argument");
  ffst_status st = check_storage(storage, plane_scale, "ffst_forward_stats");
  if (st != FFST_OK) return st;
  if (shrink < 0 || shrink > 2) return fail(FFST_ERR_INVALID_ARG, "ffst_forward_stats: shrink must be 0, 1 or 2");
  if (shrink && !thresh) return fail(FFST_ERR_INVALID_ARG, "ffst_forward_stats: thresh is required for shrinkage");
  StatsOpts so;
  so.shrink = shrink;
  so.thresh = thresh;
  so.stats = mean_abs != nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = analysis(plan, img, coeffs, storage, plane_scale, s, &so);
  if (st != FFST_OK || !mean_abs) return st;
  const cudaError_t e = timed(plan, kTimeOther, 0.0, s, [&] { return launch_mean_abs(plan, mean_abs, s); });
  if (e != cudaSuccess) return cuda_fail(e, "ffst_forward_stats mean |c|");
  return FFST_OK;
}

extern "C" ffst_status ffst_forward_complex(ffst_plan_t plan, const float* img, float* coeffs, void* stream) {
  if (!plan || !img || !coeffs) return fail(FFST_ERR_INVALID_ARG, "ffst_forward_complex: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StatsOpts re, im;
  re.cplx_part = 0;
  im.cplx_part = 1;
  ffst_status st = analysis(plan, img, coeffs, FFST_STORE_F32, nullptr, s, &re);
  if (st == FFST_OK) st = analysis(plan, img, coeffs, FFST_STORE_F32, nullptr, s, &im);
  return st;
}

extern "C" ffst_status ffst_inverse_complex(ffst_plan_t plan, const float* coeffs, float* img, void* stream) {
  if (!plan || !coeffs || !img) return fail(FFST_ERR_INVALID_ARG, "ffst_inverse_complex: NULL argument");
  return synthesis(plan, coeffs, FFST_STORE_F32, nullptr, img, static_cast<cudaStream_t>(stream), true, true);
}

extern "C" ffst_status ffst_inverse(ffst_plan_t plan, const void* coeffs, int storage, const float* plane_scale,
                                    float* img, void* stream) {
  if (!plan || !coeffs || !img) return fail(FFST_ERR_INVALID_ARG, "ffst_inverse: NULL argument");
  ffst_status st = check_storage(storage, plane_scale, "ffst_inverse");
  if (st != FFST_OK) return st;
  NvtxRange range("ffst_inverse", -1);
  return synthesis(plan, coeffs, storage, plane_scale, img, static_cast<cudaStream_t>(stream), true);
}

extern "C" ffst_status ffst_adjoint(ffst_plan_t plan, const void* coeffs, int storage, const float* plane_scale,
                                    float* img, void* stream) {
  if (!plan || !coeffs || !img) return fail(FFST_ERR_INVALID_ARG, "ffst_adjoint: NULL argument");
  ffst_status st = check_storage(storage, plane_scale, "ffst_adjoint");
  if (st != FFST_OK) return st;
  NvtxRange range("ffst_adjoint", -1);
  return synthesis(plan, coeffs, storage, plane_scale, img, static_cast<cudaStream_t>(stream), false);
}

extern "C" ffst_status ffst_plan_set_kernels(ffst_plan_t plan, int fuse_fwd, int fuse_inv, int row_fwd, int row_inv) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_kernels: plan is NULL");
  if ((fuse_fwd | fuse_inv) & ~1) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_kernels: fuse flags are 0 or 1");
  const int L = plan->N / 2;
  const bool native = plan->bl_rows.n == 0;
  if (!(row_fwd == 0 || (native && row_variant_ok(L, row_fwd, true))))
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_kernels: row variant " + std::to_string(row_fwd) +
                                          " does not exist for forward rows of length " + std::to_string(plan->N));
  if (!(row_inv == 0 || (native && row_variant_ok(L, row_inv, false))))
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_kernels: row variant " + std::to_string(row_inv) +
                                          " does not exist for inverse rows of length " + std::to_string(plan->N));
  plan->fuse_fwd = fuse_fwd;
  plan->fuse_inv = fuse_inv;
  plan->row_fwd = row_fwd;
  plan->row_inv = row_inv;
  return FFST_OK;
}

extern "C" ffst_status ffst_plan_get_kernels(ffst_plan_t plan, int* fuse_fwd, int* fuse_inv, int* row_fwd,
                                             int* row_inv) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_get_kernels: plan is NULL");
  if (fuse_fwd) *fuse_fwd = plan->fuse_fwd;
  if (fuse_inv) *fuse_inv = plan->fuse_inv;
  if (row_fwd) *row_fwd = plan->row_fwd;
  if (row_inv) *row_inv = plan->row_inv;
  return FFST_OK;
}

extern "C" ffst_status ffst_plan_set_planes(ffst_plan_t plan, int p0, int p1) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_planes: plan is NULL");
  if (p0 < 0 || p1 > plan->eta || p0 >= p1)
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_planes: need 0 <= p0 < p1 <= eta, got [" + std::to_string(p0) +
                                          ", " + std::to_string(p1) + ")");
  if (plan->sched_mode != 0 && (p0 != 0 || p1 != plan->eta))
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_planes: the persistent schedule runs every plane");
  if (p0 == plan->pr0 && p1 == plan->pr1) return FFST_OK;
  cudaError_t e = cudaDeviceSynchronize();  // in-flight transforms use the groups and buffers
  if (e != cudaSuccess) return cuda_fail(e, "ffst_plan_set_planes");
  plan->pr0 = p0;
  plan->pr1 = p1;
  return plan_regroup(plan, plan->group_mb, plan->group_mb_inv);
}

extern "C" ffst_status ffst_plan_get_planes(ffst_plan_t plan, int* p0, int* p1) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_get_planes: plan is NULL");
  if (p0) *p0 = plan->pr0;
  if (p1) *p1 = plan->pr1;
  return FFST_OK;
}

extern "C" ffst_status ffst_inverse_partial(ffst_plan_t plan, const void* coeffs, int storage,
                                            const float* plane_scale, float* spectrum, void* stream) {
  if (!plan || !coeffs || !spectrum) return fail(FFST_ERR_INVALID_ARG, "ffst_inverse_partial: NULL argument");
  ffst_status st = check_storage(storage, plane_scale, "ffst_inverse_partial");
  if (st != FFST_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = synthesis_planes(plan, coeffs, storage, plane_scale, s, false);
  if (st != FFST_OK) return st;
  const long long n = (long long)plan->M * plan->Hc;
  k_sum_partials<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(
      plan->d_S, plan->inv_split, n, reinterpret_cast<float2*>(spectrum));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "ffst_inverse_partial");
  return FFST_OK;
}

extern "C" ffst_status ffst_inverse_finish(ffst_plan_t plan, float* spectrum, int normalise, float* img,
                                           void* stream) {
  if (!plan || !spectrum || !img) return fail(FFST_ERR_INVALID_ARG, "ffst_inverse_finish: NULL argument");
  return synthesis_finish(plan, reinterpret_cast<float2*>(spectrum), 1, normalise != 0, img,
                          static_cast<cudaStream_t>(stream));
}

extern "C" ffst_status ffst_plan_set_schedule(ffst_plan_t plan, int mode) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_schedule: plan is NULL");
  if (mode < 0 || mode > 2) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_schedule: mode must be 0, 1 or 2");
  if (mode != 0 && (plan->pr0 != 0 || plan->pr1 != plan->eta))
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_schedule: the persistent schedule runs every plane");
  if (mode != 0 && !plan->sched.on && fused_supported(plan->M, plan->N)) {  // built on first use
    const ffst_status st = sched_build(plan, default_ring_mb());
    if (st != FFST_OK) return st;
  }
  plan->sched_mode = mode;
  return FFST_OK;
}

extern "C" ffst_status ffst_plan_set_inverse_split(ffst_plan_t plan, int nsplit) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_inverse_split: plan is NULL");
  if (nsplit < 0 || nsplit > kMaxInvSplit)
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_set_inverse_split: nsplit must be in 0..16");
  if (nsplit == 0) nsplit = plan->inv_split_default;
  return plan_set_inv_split(plan, nsplit);
}

extern "C" ffst_status ffst_plan_get_inverse_split(ffst_plan_t plan, int* nsplit) {
  if (!plan || !nsplit) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_get_inverse_split: NULL argument");
  *nsplit = plan->inv_split;
  return FFST_OK;
}

extern "C" ffst_status ffst_plan_get_schedule(ffst_plan_t plan, int* mode) {
  if (!plan || !mode) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_get_schedule: NULL argument");
  *mode = use_sched(plan) ? plan->sched_mode : 0;
  return FFST_OK;
}

extern "C" ffst_status ffst_plan_check(ffst_plan_t plan, void* stream) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_check: plan is NULL");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ffst_plan_check");
  int err = 0;
  e = cudaMemcpy(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && err) e = cudaMemset(plan->d_err, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "ffst_plan_check");
  if (err & kErrBounds)
    return fail(FFST_ERR_BOUNDS, "an index outside its buffer was caught and skipped (FFST_CHECK build); the "
                                 "transform output is unspecified");
  if (err) return fail(FFST_ERR_TIMEOUT, "a bounded device-side wait ran out; the transform output is unspecified");
  return FFST_OK;
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
