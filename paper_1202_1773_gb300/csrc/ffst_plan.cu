// Plan construction: FP64 host tables, plane indexing, spectral supports,
// plane grouping and workspace; plus the spectra export kernel.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>

#include "ffst_blue.cuh"

namespace ffst {

// ---------------------------------------------------------------------------
// FP64 window functions for the once-per-plan tables (host only)
// ---------------------------------------------------------------------------
// The plan's auxiliary function v: eq. (v) of Sec. 2.1 or one of its
// variants (Sec. 2.1, Sec. 3.4 remark construction_v).
struct VSpec {
  int kind = FFST_V_MEYER;
  int deg = 0;     // FFST_V_POLY: degree of v on [0, 1] (2k + 1)
  double c[16]{};  // FFST_V_POLY: coefficients of v on [0, 1]
};
// v'(x) = c x^k (x - 1)^k, v(1) = 1: the binomial expansion integrated term
// by term, c = (-1)^k (2k + 1)! / (k!)^2.
static VSpec v_poly_spec(int k) {
  VSpec s;
  s.kind = FFST_V_POLY;
  s.deg = 2 * k + 1;
  double c = (k % 2 ? -1.0 : 1.0);
  for (int q = k + 2; q <= 2 * k + 1; ++q) c *= q;  // (2k+1)!/(k+1)! ...
  for (int q = 2; q <= k; ++q) c /= q;               // ... / k! = (2k+1)!/(k! k!) with the (k+1) below
  c *= (k + 1);
  double binom = 1.0;  // C(k, m)
  for (int m = 0; m <= k; ++m) {
    s.c[k + m + 1] = c * binom * (((k - m) % 2) ? -1.0 : 1.0) / (k + m + 1);
    binom = binom * (k - m) / (m + 1);
  }
  return s;
}

// v on [0, 1/2]; v(x) = 1 - v(1 - x) gives the rest (Lemma, Sec. 2.1).
static double vhalf64(double x, const VSpec& vs) {
  switch (vs.kind) {
    case FFST_V_QUADRATIC:
      return 2.0 * x * x;
    case FFST_V_POLY: {
      double acc = vs.c[vs.deg];
      for (int n = vs.deg - 1; n >= 0; --n) acc = acc * x + vs.c[n];
      return acc;
    }
    case FFST_V_CINF: {
      if (x <= 0.0) return 0.0;
      const double s0 = std::exp(-(1.0 / (x * x) + 1.0 / ((2.0 - x) * (2.0 - x))));
      const double s1 = std::exp(-(1.0 / ((1.0 + x) * (1.0 + x)) + 1.0 / ((1.0 - x) * (1.0 - x))));
      return s0 / (s0 + s1);
    }
    default: {
      const double y2 = x * x;
      return y2 * y2 * (35.0 + x * (-84.0 + x * (70.0 - 20.0 * x)));
    }
  }
}

static double v64(double x, const VSpec& vs) {
  if (x <= 0.0) return 0.0;
  if (x >= 1.0) return 1.0;
  return x <= 0.5 ? vhalf64(x, vs) : 1.0 - vhalf64(1.0 - x, vs);
}

// psi1_hat in the closed form of Sec. 3.4 (equal to eq. (Psi1) of Sec. 2.1).
static double psi1_64(double w, const VSpec& vs) {
  w = std::fabs(w);
  if (w <= 0.5) return 0.0;
  if (w < 1.0) return std::sin(0.5 * kPi * v64(2.0 * w - 1.0, vs));
  if (w <= 2.0) return 1.0;
  if (w < 4.0) return std::cos(0.5 * kPi * v64(0.5 * w - 1.0, vs));
  return 0.0;
}

// varphi of Sec. 2.4.
static double varphi64(double w, const VSpec& vs) {
  w = std::fabs(w);
  if (w <= 0.5) return 1.0;
  if (w < 1.0) return std::cos(0.5 * kPi * v64(2.0 * w - 1.0, vs));
  return 0.0;
}

// 1 - varphi(w)^2, written as a sine square so it keeps full precision
// where varphi is close to 1.
static double varphi_sig64(double w, const VSpec& vs) {
  w = std::fabs(w);
  if (w <= 0.5) return 0.0;
  if (w < 1.0) {
    const double s = std::sin(0.5 * kPi * v64(2.0 * w - 1.0, vs));
    return s * s;
  }
  return 1.0;
}

// ---------------------------------------------------------------------------
// device kernels used at plan time / for export
// ---------------------------------------------------------------------------

// For every plane, the smallest and largest half-spectrum column where the
// spectrum is nonzero (minmax[2i], minmax[2i+1]).  Block (plane i, row
// chunk): each thread keeps its own extremes over its elements, a block
// reduction leaves one atomic pair per block.
__global__ void k_support(WinParams w, const PlaneDesc* __restrict__ planes, int Hc, int rows_per_block,
                          int* minmax) {
  __shared__ int smin[32], smax[32];
  const int i = blockIdx.y;
  const PlaneDesc d = planes[i];
  const int r0 = blockIdx.x * rows_per_block;
  const int r1 = min(w.M, r0 + rows_per_block);
  int lo = 0x7fffffff, hi = -1;
  // A classic h-cone plane is zero wherever its radial factor psi1(4^-j |xi1|)
  // is (column pc, |omega1| = pc or N - pc), a v-cone plane wherever
  // psi1(4^-j |xi2|) is (row pr); the Sec. 3.8.1 mirror keeps |omega|, so
  // skipping those columns or rows finds the same extremes.
  const bool radial = !w.smooth && (d.kappa == kH || d.kappa == kV);
  if (radial && d.kappa == kH) {
    for (int pc = threadIdx.x; pc < Hc; pc += blockDim.x) {
      const int a1 = (2 * pc < w.N) ? pc : w.N - pc;
      if (__ldg(&w.psi1_col[d.j * (w.hn + 1) + a1]) == 0.0f) continue;
      for (int pr = r0; pr < r1; ++pr)
        if (win_at(w, d, pr, pc) != 0.0f) {
          lo = min(lo, pc);
          hi = max(hi, pc);
        }
    }
  } else {
    for (int pr = r0; pr < r1; ++pr) {  // rows of the chunk, the threads across the columns
      if (radial) {
        const int a2 = (2 * pr < w.M) ? pr : w.M - pr;
        if (__ldg(&w.psi1_row[d.j * (w.hm + 1) + a2]) == 0.0f) continue;  // uniform over the block
      }
      for (int pc = threadIdx.x; pc < Hc; pc += blockDim.x)
        if (win_at(w, d, pr, pc) != 0.0f) {
          lo = min(lo, pc);
          hi = max(hi, pc);
        }
    }
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    smin[wid] = lo;
    smax[wid] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < nw; ++q) {
      lo = min(lo, smin[q]);
      hi = max(hi, smax[q]);
    }
    if (hi >= 0) {
      atomicMin(&minmax[2 * i], lo);
      atomicMax(&minmax[2 * i + 1], hi);
    }
  }
}

// psi[i][pr][pc] on the full grid in FFT order; columns beyond N/2 use the
// point symmetry psi(-omega) = psi(omega) that the Sec. 3.8.1 fix guarantees.
__global__ void k_spectra(WinParams w, const PlaneDesc* __restrict__ planes, int eta, float* __restrict__ psi) {
  const long long per_plane = (long long)w.M * w.N;
  const long long total = per_plane * eta;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / per_plane);
    const long long rem = idx - (long long)i * per_plane;
    const int pr = (int)(rem / w.N), pc = (int)(rem % w.N);
    const PlaneDesc d = planes[i];
    float val;
    if (2 * pc <= w.N) val = win_at(w, d, pr, pc);
    else val = win_at(w, d, (w.M - pr) % w.M, w.N - pc);
    psi[idx] = val;
  }
}

cudaError_t launch_spectra(const ffst_plan_s* p, float* psi, cudaStream_t s) {
  k_spectra<<<152 * 8, 256, 0, s>>>(p->win, p->d_planes, p->eta, psi);
  return cudaGetLastError();
}

cudaError_t launch_support(const ffst_plan_s* p, int* d_minmax, cudaStream_t s) {
  // about 64K window values per block
  const int rpb = std::max(1, (1 << 16) / p->Hc);
  const dim3 grid((p->M + rpb - 1) / rpb, p->eta);
  k_support<<<grid, 256, 0, s>>>(p->win, p->d_planes, p->Hc, rpb, d_minmax);
  return cudaGetLastError();
}

// For every plane and support column, the shortest cyclic row interval
// (start, len) that holds all nonzero rows: the complement of the largest
// cyclic gap between consecutive nonzero rows.  One warp per (plane, support
// column) (blockIdx.y = plane): lane l scans the rows [l M/32, (l+1) M/32) in
// order (first and last nonzero row, largest inner gap), then lane 0 joins
// the 32 chunks in row order, as one sequential scan over all rows would.
__global__ void k_ranges(WinParams w, const PlaneDesc* __restrict__ planes, int2* __restrict__ rng) {
  const PlaneDesc d = planes[blockIdx.y];
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= d.W) return;  // whole warps
  const int lane = threadIdx.x & 31;
  const int c = d.c0 + q;
  const int chunk = (w.M + 31) / 32;
  const int ra = lane * chunk, rb = min(w.M, ra + chunk);
  int first = -1, prev = -1, maxgap = -1, after = 0;
  for (int r = ra; r < rb; ++r) {
    if (win_at(w, d, r, c) != 0.0f) {
      if (first < 0) {
        first = r;
      } else if (r - prev - 1 > maxgap) {
        maxgap = r - prev - 1;
        after = r;
      }
      prev = r;
    }
  }
  // join the chunks in order on lane 0 (same result as one scan over 0..M-1)
  int gfirst = -1, gprev = -1, gmax = -1, gafter = 0;
  for (int l = 0; l < 32; ++l) {
    const int f = __shfl_sync(0xffffffffu, first, l);
    const int p = __shfl_sync(0xffffffffu, prev, l);
    const int g = __shfl_sync(0xffffffffu, maxgap, l);
    const int a = __shfl_sync(0xffffffffu, after, l);
    if (f < 0) continue;
    if (gfirst < 0) {
      gfirst = f;
    } else if (f - gprev - 1 > gmax) {
      gmax = f - gprev - 1;
      gafter = f;
    }
    if (g > gmax) {
      gmax = g;
      gafter = a;
    }
    gprev = p;
  }
  if (lane == 0) {
    int2 out = make_int2(0, 0);
    if (gfirst >= 0) {
      const int wrap = gfirst + w.M - gprev - 1;
      out = (wrap >= gmax) ? make_int2(gfirst, gprev - gfirst + 1) : make_int2(gafter, w.M - gmax);
    }
    rng[d.rng_off + q] = out;
  }
}

// 1 / sum_i psi_i^2 on the half spectrum, from the same FP32 generator the
// transforms use (the inverse's normalisation, Sec. 3.3).
__global__ void k_inv_norm(WinParams w, const PlaneDesc* __restrict__ planes, int eta, int Hc,
                           const int2* __restrict__ rng, float* __restrict__ inv_d) {
  extern __shared__ PlaneDesc sp[];
  for (int i = threadIdx.x; i < eta; i += blockDim.x) sp[i] = planes[i];
  __syncthreads();
  const long long total = (long long)w.M * Hc;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int pr = (int)(idx / Hc), pc = (int)(idx % Hc);
    float sum = 0.0f;
    for (int i = 0; i < eta; ++i) {
      const PlaneDesc& d = sp[i];
      const int q = pc - d.c0;
      if (q < 0 || q >= d.W) continue;
      const int2 rg = rng[d.rng_off + q];
      int off = pr - rg.x;
      if (off < 0) off += w.M;
      if (off >= rg.y) continue;
      const float psi = win_at(w, d, pr, pc);
      sum = fmaf(psi, psi, sum);
    }
    inv_d[idx] = sum > 0.0f ? 1.0f / sum : 1.0f;
  }
}

cudaError_t launch_ranges(const ffst_plan_s* p, cudaStream_t s) {
  int wmax = 1;
  for (const PlaneDesc& d : p->planes) wmax = std::max(wmax, d.W);
  const dim3 grid((wmax + 7) / 8, p->eta);  // 8 warps per block, one per support column
  k_ranges<<<grid, 256, 0, s>>>(p->win, p->d_planes, p->d_rng);
  return cudaGetLastError();
}

cudaError_t launch_inv_norm(const ffst_plan_s* p, cudaStream_t s) {
  const size_t smem = sizeof(PlaneDesc) * p->eta;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_inv_norm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_inv_norm<<<152 * 8, 256, smem, s>>>(p->win, p->d_planes, p->eta, p->Hc, p->d_rng, p->d_invD);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

ffst_status fail(ffst_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

ffst_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? FFST_ERR_OUT_OF_MEMORY : FFST_ERR_CUDA;
}

static void free_plan(ffst_plan_s* p) {
  if (!p) return;
  cudaFree(p->d_planes);
  cudaFree(p->d_planes_inv);
  cudaFree(p->d_tables);
  cudaFree(p->d_tw_rows);
  cudaFree(p->d_tw_rows32);
  cudaFree(p->d_tw_cols);
  cudaFree(p->d_rtw);
  cudaFree(p->d_blue);
  cudaFree(p->d_rng);
  cudaFree(p->d_F);
  cudaFree(p->d_S);
  cudaFree(p->d_invD);
  cudaFree(p->d_H);
  cudaFree(p->d_partials);
  cudaFree(p->d_items);
  cudaFree(p->d_err);
  cudaFree(p->d_abs_partials);
  tma_free(p);
  sched_free(p);
  for (auto& r : p->timer.pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : p->timer.pool) cudaEventDestroy(e);
  delete p;
}

// Intermediate budgets per plane group of the forward and of the inverse.
// The column pass writes a group's intermediates and the row pass reads
// them back (two groups in flight, double-buffered); the stack streams past
// L2 with evict-first hints.  Larger groups mean fewer launches and shorter
// tails, smaller ones keep more of the intermediates in L2; the two
// directions weigh this differently (2048x2048 J=5, ms: forward 1.07 at
// 96 MB, 1.12 at 128, 1.16 at 192; inverse 1.17 at 96, 1.10 at 128, 1.07 at
// 192).  FFST_GROUP_MB sets both, FFST_GROUP_MB_INV the inverse;
// ffst_plan_autotune measures the candidates instead.
void default_group_mb(double* fwd_mb, double* inv_mb) {
  double f = 96.0, i = 192.0;
  if (const char* e = std::getenv("FFST_GROUP_MB")) {
    const double v = std::atof(e);
    if (v > 0.0) f = i = v;
  }
  if (const char* e = std::getenv("FFST_GROUP_MB_INV")) {
    const double v = std::atof(e);
    if (v > 0.0) i = v;
  }
  *fwd_mb = f;
  *inv_mb = i;
}

// Size of the first and the last plane group relative to the budget
// (measured at 2048x2048 J=5, 128 MB: 0.5 -> 2.54 ms fwd+inv, 1 -> 2.61 ms).
#ifndef FFST_GROUP_RAMP
#define FFST_GROUP_RAMP 0.5
#endif
constexpr double kGroupRamp = FFST_GROUP_RAMP;

// Plane groups for a budget of `mb` megabytes: runs of consecutive planes
// cut at targets of the cumulative intermediate size (a plane goes to the
// group its midpoint falls in).  The first and the last group aim at
// kGroupRamp times the budget (they run in launches of their own: one pass
// alone before the first fused launch, the other alone after the last), the
// others split the rest evenly into the fewest groups of at most about the
// budget.  Writes each plane's slot offset inside its group to off[] and
// returns the largest group size (float2 elements).
static long long build_groups(const ffst_plan_s* p, double mb, std::vector<Group>& groups,
                              std::vector<long long>& off) {
  const double budget = mb * 1024.0 * 1024.0 / sizeof(float2);
  groups.clear();
  off.assign(p->eta, 0);
  auto elems_of = [&](int i) { return (long long)p->M * p->planes[i].ldw; };
  double total = 0.0;
  for (int i = p->pr0; i < p->pr1; ++i) total += (double)elems_of(i);
  std::vector<double> cuts;  // group k holds the planes whose midpoint lies in [cuts[k-1], cuts[k])
  if (total > budget) {
    const bool ramp = kGroupRamp < 1.0;
    const double e = ramp ? std::min(kGroupRamp * budget, total / 3.0) : budget;
    const double rest = total - (ramp ? 2.0 : 1.0) * e;
    const int k = std::max(1, (int)std::ceil(rest / budget - 1e-9));
    cuts.push_back(e);
    for (int j = 1; j < (ramp ? k + 1 : k); ++j) cuts.push_back(e + rest * j / k);
  }
  Group g{p->pr0, p->pr0, 0, p->planes[p->pr0].item0, 0};
  long long maxg = 0;
  double acc = 0.0;
  size_t gk = 0;  // group index of the open group
  for (int i = p->pr0; i < p->pr1; ++i) {
    const long long el = elems_of(i);
    const double mid = acc + 0.5 * (double)el;
    acc += (double)el;
    size_t k = 0;
    while (k < cuts.size() && cuts[k] <= mid) ++k;
    if (g.p1 > g.p0 && k != gk) {
      g.nitems = p->planes[i].item0 - g.item0;
      groups.push_back(g);
      maxg = std::max(maxg, g.elems);
      g = Group{i, i, 0, p->planes[i].item0, 0};
    }
    gk = k;
    off[i] = g.elems;
    g.elems += el;
    g.p1 = i + 1;
  }
  g.nitems = p->total_items - g.item0;
  groups.push_back(g);
  return std::max(maxg, g.elems);
}

// (Re)build the forward column work items, the plane groups of both
// directions and the double-buffered intermediate (sized for the larger
// group of either direction).
ffst_status plan_regroup(ffst_plan_s* p, double fwd_mb, double inv_mb) {
  const int P = p->P;
  cudaFree(p->d_items);
  cudaFree(p->d_partials);
  cudaFree(p->d_H);
  p->d_items = nullptr;
  p->d_partials = nullptr;
  p->d_H = nullptr;
  // forward column items: the panels of every active plane's slot, in plane order
  std::vector<ColItem> items;
  for (int i = 0; i < p->eta; ++i) {
    p->planes[i].item0 = (int)items.size();
    if (i >= p->pr0 && i < p->pr1)
      for (int c = p->planes[i].c0al; c < p->planes[i].c0 + p->planes[i].W; c += P) items.push_back(ColItem{i, c});
    p->planes[i].nitems = (int)items.size() - p->planes[i].item0;
  }
  p->total_items = (int)items.size();
  std::vector<long long> off_f, off_i;
  const long long hf = build_groups(p, fwd_mb, p->groups, off_f);
  const long long hi = build_groups(p, inv_mb, p->groups_inv, off_i);
  p->h_elems = std::max(hf, hi);
  p->group_mb = fwd_mb;
  p->group_mb_inv = inv_mb;
  std::vector<PlaneDesc> pi = p->planes;
  for (int i = 0; i < p->eta; ++i) {
    p->planes[i].off = off_f[i];
    pi[i].off = off_i[i];
  }
  cudaError_t e = cudaMemcpy(p->d_planes, p->planes.data(), p->planes.size() * sizeof(PlaneDesc),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !p->d_planes_inv) e = cudaMalloc(&p->d_planes_inv, pi.size() * sizeof(PlaneDesc));
  if (e == cudaSuccess) e = cudaMemcpy(p->d_planes_inv, pi.data(), pi.size() * sizeof(PlaneDesc), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "plane descriptors");
  if (!items.empty()) {
    if ((e = cudaMalloc(&p->d_items, items.size() * sizeof(ColItem))) != cudaSuccess) return cuda_fail(e, "items");
    if ((e = cudaMemcpy(p->d_items, items.data(), items.size() * sizeof(ColItem), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return cuda_fail(e, "items");
    if ((e = cudaMalloc(&p->d_partials, items.size() * sizeof(float))) != cudaSuccess) return cuda_fail(e, "partials");
  }
  if (p->h_elems > 0 && (e = cudaMalloc(&p->d_H, 2 * (size_t)p->h_elems * sizeof(float2))) != cudaSuccess)
    return cuda_fail(e, "workspace H");
  return tma_build(p, off_f, off_i);
}

int inv_part(const ffst_plan_s* p, int plane) {
  for (int k = 0; k < p->inv_split; ++k)
    if (plane < (int)((long long)p->eta * (k + 1) / p->inv_split)) return k;
  return p->inv_split - 1;
}

// Default plane chunks of the inverse column pass: enough column blocks
// (panels x chunks) for about four resident blocks per SM, at most
// kMaxInvSplit; FFST_INV_SPLIT overrides.  At 2048x2048 the 513 panels
// already fill the GPU (one chunk); at 512x512 there are only 33.
static int default_inv_split(const ffst_plan_s* p) {
  if (const char* s = std::getenv("FFST_INV_SPLIT")) {
    const int n = std::atoi(s);
    if (n >= 1) return std::min(n, kMaxInvSplit);
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess || sms < 1) sms = 1;
  const int P = p->P;
  const int npanels = (p->Hc + P - 1) / P;
  return std::max(1, std::min(kMaxInvSplit, 4 * sms / npanels));
}

ffst_status plan_set_inv_split(ffst_plan_s* p, int n) {
  if (n < 1 || n > kMaxInvSplit) return fail(FFST_ERR_INVALID_ARG, "inverse split must be in 1..16");
  if (n > p->inv_split_cap) {
    float2* d = nullptr;
    const cudaError_t e = cudaMalloc(&d, (size_t)n * p->M * p->Hc * sizeof(float2));
    if (e != cudaSuccess) return cuda_fail(e, "inverse partial accumulators");
    cudaFree(p->d_S);
    p->d_S = d;
    p->inv_split_cap = n;
  }
  p->inv_split = n;
  return p->sched.on ? sched_build(p, p->sched.ring_mb) : FFST_OK;
}

// Pass twiddle table of a line (L, E) (layout in ffst_fft.cuh), FP64 -> FP32.
static std::vector<float2> pass_table(int L, int E) {
  std::vector<float2> t(L > 1 ? L : 1, make_float2(1.0f, 0.0f));
  for (int idx = 0; idx < L - 1; ++idx) {
    int m = 0, n = 1;
    pass_entry(L, E, idx, &m, &n);
    const double a = 2.0 * kPi * (double)m / (double)n;
    t[idx] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  return t;
}

// exp(-2 pi i k / N), k = 0..N/2: the split twiddles of the real-row FFTs.
static std::vector<float2> real_twiddles(int N) {
  std::vector<float2> t(N / 2 + 1);
  for (int k = 0; k <= N / 2; ++k) {
    const double a = 2.0 * kPi * (double)k / (double)N;
    t[k] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  return t;
}

static cudaError_t upload(float2** dst, const std::vector<float2>& v) {
  cudaError_t e = cudaMalloc(dst, v.size() * sizeof(float2));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(float2), cudaMemcpyHostToDevice);
}

}  // namespace ffst

using namespace ffst;

extern "C" ffst_status ffst_plan(int rows, int cols, int scales, ffst_plan_t* out) {
  return ffst_plan_ex(rows, cols, scales, FFST_VARIANT_CLASSIC, FFST_V_MEYER, 0, FFST_MAXSCALE_MAX,
                      FFST_SPACING_COMMON, out);
}

// FFST_PLAN_TIMES=1: wall time of each phase of plan creation on stderr
// (the device is synchronised at every mark, so the marks add a little).
namespace {
struct PhaseTimer {
  bool on = false;
  std::chrono::steady_clock::time_point t0, last;
  std::string line;
  PhaseTimer() {
    const char* e = std::getenv("FFST_PLAN_TIMES");
    on = e && e[0] == '1';
    t0 = last = std::chrono::steady_clock::now();
  }
  void mark(const char* what) {
    if (!on) return;
    cudaDeviceSynchronize();
    const auto now = std::chrono::steady_clock::now();
    char b[96];
    std::snprintf(b, sizeof b, " %s %.3f", what, std::chrono::duration<double, std::milli>(now - last).count());
    line += b;
    last = now;
  }
  ~PhaseTimer() {
    if (on)
      std::fprintf(stderr, "ffst_plan ms:%s | total %.3f\n", line.c_str(),
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
  }
};
}  // namespace

extern "C" ffst_status ffst_plan_ex(int rows, int cols, int scales, int variant, int vfun, int vorder, int max_scale,
                                    int spacing, ffst_plan_t* out) {
  if (!out) return fail(FFST_ERR_INVALID_ARG, "ffst_plan: out is NULL");
  PhaseTimer ptime;
  *out = nullptr;
  if (variant != FFST_VARIANT_CLASSIC && variant != FFST_VARIANT_SMOOTH)
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_ex: variant must be FFST_VARIANT_CLASSIC or FFST_VARIANT_SMOOTH");
  if (vfun < FFST_V_MEYER || vfun > FFST_V_CINF)
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_ex: vfun must be one of FFST_V_MEYER .. FFST_V_CINF");
  if (vfun == FFST_V_POLY && (vorder < 1 || vorder > 7))
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_ex: FFST_V_POLY needs an order in 1..7");
  if (max_scale != FFST_MAXSCALE_MAX && max_scale != FFST_MAXSCALE_MIN)
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_ex: max_scale must be FFST_MAXSCALE_MAX or FFST_MAXSCALE_MIN");
  if (spacing != FFST_SPACING_COMMON && spacing != FFST_SPACING_PER_AXIS)
    return fail(FFST_ERR_INVALID_ARG, "ffst_plan_ex: spacing must be FFST_SPACING_COMMON or FFST_SPACING_PER_AXIS");
  VSpec vs;
  if (vfun == FFST_V_POLY) vs = v_poly_spec(vorder);
  vs.kind = vfun;
  // native FFT lines: columns of length rows, rows as half-length complex
  // lines of cols/2; any other length runs generic lines: mixed-radix for
  // lengths with no prime factor above 7 (up to 4096 points), Bluestein for
  // the others (up to 2048; FFST_BLUESTEIN=1: for every generic length)
  const char* fb = std::getenv("FFST_BLUESTEIN");
  const bool all_blue = fb && fb[0] == '1';
  auto smooth7 = [](int n) {
    for (int q : {2, 3, 5, 7})
      while (n % q == 0) n /= q;
    return n == 1;
  };
  auto generic_ok = [&](int n) { return n <= kBlueMaxL2 / 2 || (!all_blue && smooth7(n)); };
  const bool nat_cols = rows >= 8 && rows <= 4096 && supported_line(rows);
  const bool nat_rows = cols >= 8 && cols <= 4096 && cols % 2 == 0 && supported_line(cols / 2);
  if (rows < 8 || cols < 8 || rows > 4096 || cols > 4096 || (!nat_cols && !generic_ok(rows)) ||
      (!nat_rows && !generic_ok(cols)))
    return fail(FFST_ERR_UNSUPPORTED_SIZE,
                "ffst_plan: rows and cols must be in [8, 4096], and at most 2048 unless they have no prime factor "
                "above 7, rows is a power of two or one of 240, 320, 384, 480, 640, 768 (cols: twice one of "
                "those), got " +
                    std::to_string(rows) + "x" + std::to_string(cols));
  const int mx = rows > cols ? rows : cols;
  int lg = 0;
  while ((1 << (lg + 1)) <= mx) ++lg;
  const int j0 = scales > 0 ? scales : lg / 2;  // Sec. 3.1: floor(1/2 log2 max(M, N))
  if (j0 < 1 || j0 > 8)
    return fail(FFST_ERR_UNSUPPORTED_SIZE, "ffst_plan: scales must be in 1..8, got " + std::to_string(j0));

  std::unique_ptr<ffst_plan_s, void (*)(ffst_plan_s*)> p(new ffst_plan_s, free_plan);
  cudaGetDevice(&p->device);
  p->M = rows;
  p->N = cols;
  p->j0 = j0;
  p->eta = (1 << (j0 + 2)) - 3;  // Sec. 3.5.2
  p->pr0 = 0;
  p->pr1 = p->eta;
  p->Hc = cols / 2 + 1;
  p->hm = rows / 2;
  p->hn = cols / 2;
  p->variant = variant;

  // plane table, Sec. 3.5.2: low-pass, then per scale counter-clockwise
  p->planes.clear();
  auto add = [&](int kappa, int j, int k) {
    PlaneDesc d{};
    d.kappa = kappa;
    d.j = j;
    d.k = k;
    p->planes.push_back(d);
  };
  add(kLowpass, -1, 0);
  for (int j = 0; j < j0; ++j) {
    const int J = 1 << j;
    add(kH, j, 0);
    for (int k = -1; k > -J; --k) add(kH, j, k);
    add(kSeam, j, -J);
    for (int k = -J + 1; k < J; ++k) add(kV, j, k);
    add(kSeam, j, J);
    for (int k = J - 1; k > 0; --k) add(kH, j, k);
  }
  if ((int)p->planes.size() != p->eta) return fail(FFST_ERR_INVALID_ARG, "ffst_plan: internal plane count mismatch");

  // FP64 window tables (Sec. 3.5.1 grid: xi = a * X / g, X = 2^{2 j0 - 1}, or
  // X = 2^{2 j0 - 2} for max_scale = FFST_MAXSCALE_MIN; one step g =
  // floor(max(M, N)/2) for both axes, or g = floor(L/2) per axis)
  const double X = std::ldexp(1.0, 2 * j0 - (max_scale == FFST_MAXSCALE_MAX ? 1 : 2));
  const int gm = spacing == FFST_SPACING_COMMON ? mx / 2 : p->hm;
  const int gn = spacing == FFST_SPACING_COMMON ? mx / 2 : p->hn;
  const double dc = X / gn, dr = X / gm;
  const int ncol = p->hn + 1, nrow = p->hm + 1;
  // layout: psi1 col [j0][ncol] | psi1 row [j0][nrow] | phi col | phi row |
  //         smooth: sig col [j0][ncol] | sig row [j0][nrow] | alp col [j0][ncol] | alp row [j0][nrow]
  const size_t per_scale = (size_t)j0 * (ncol + nrow);
  std::vector<float> tab(per_scale + ncol + nrow + 2 * per_scale);
  float* psi1_col = tab.data();
  float* psi1_row = psi1_col + (size_t)j0 * ncol;
  float* phi_col = psi1_row + (size_t)j0 * nrow;
  float* phi_row = phi_col + ncol;
  float* sig_col = phi_row + nrow;
  float* sig_row = sig_col + (size_t)j0 * ncol;
  float* alp_col = sig_row + (size_t)j0 * nrow;
  float* alp_row = alp_col + (size_t)j0 * ncol;
  for (int j = 0; j < j0; ++j) {
    const double a = std::ldexp(1.0, -2 * j);  // a_j = 4^-j
    for (int q = 0; q < ncol; ++q) {
      psi1_col[(size_t)j * ncol + q] = (float)psi1_64(a * q * dc, vs);
      sig_col[(size_t)j * ncol + q] = (float)varphi_sig64(a * q * dc, vs);
      const double f = varphi64(0.25 * a * q * dc, vs);
      alp_col[(size_t)j * ncol + q] = (float)(f * f);
    }
    for (int q = 0; q < nrow; ++q) {
      psi1_row[(size_t)j * nrow + q] = (float)psi1_64(a * q * dr, vs);
      sig_row[(size_t)j * nrow + q] = (float)varphi_sig64(a * q * dr, vs);
      const double f = varphi64(0.25 * a * q * dr, vs);
      alp_row[(size_t)j * nrow + q] = (float)(f * f);
    }
  }
  for (int q = 0; q < ncol; ++q) phi_col[q] = (float)varphi64(q * dc, vs);
  for (int q = 0; q < nrow; ++q) phi_row[q] = (float)varphi64(q * dr, vs);

  cudaError_t e;
  if ((e = cudaMalloc(&p->d_tables, tab.size() * sizeof(float))) != cudaSuccess) return cuda_fail(e, "ffst_plan tables");
  if ((e = cudaMemcpy(p->d_tables, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "ffst_plan tables upload");
  p->win.M = rows;
  p->win.N = cols;
  p->win.hm = p->hm;
  p->win.hn = p->hn;
  p->win.gm = gm;
  p->win.gn = gn;
  p->win.psi1_col = p->d_tables;
  p->win.psi1_row = p->d_tables + (size_t)j0 * ncol;
  p->win.phi_col = p->win.psi1_row + (size_t)j0 * nrow;
  p->win.phi_row = p->win.phi_col + ncol;
  p->win.smooth = variant == FFST_VARIANT_SMOOTH;
  p->win.vkind = vfun;
  p->win.vdeg = vfun == FFST_V_POLY ? vs.deg : 0;
  for (int n = 0; n < 16; ++n) p->win.vc[n] = (float)vs.c[n];
  p->win.sig_col = p->win.phi_row + nrow;
  p->win.sig_row = p->win.sig_col + (size_t)j0 * ncol;
  p->win.alp_col = p->win.sig_row + (size_t)j0 * nrow;
  p->win.alp_row = p->win.alp_col + (size_t)j0 * ncol;
  ptime.mark("tables");

  // twiddles (FP64 -> FP32): row lines of length N/2, their real split, column lines of length M
  if (nat_rows) {
    if ((e = upload(&p->d_tw_rows, pass_table(cols / 2, row_E(cols / 2)))) != cudaSuccess) return cuda_fail(e, "twiddles");
    if (row_variant_ok(cols / 2, 2, true) &&
        (e = upload(&p->d_tw_rows32, pass_table(cols / 2, 32))) != cudaSuccess)
      return cuda_fail(e, "twiddles");
    if ((e = upload(&p->d_rtw, real_twiddles(cols))) != cudaSuccess) return cuda_fail(e, "twiddles");
  }
  if (nat_cols) {
    if ((e = upload(&p->d_tw_cols, pass_table(rows, col_E(rows)))) != cudaSuccess) return cuda_fail(e, "twiddles");
  }
  // generic lines, per generic dimension: mixed-radix pass table (lengths
  // with no prime factor above 7), else chirp | filter spectrum | pass table
  {
    std::vector<float2> tab;
    size_t off[2][3] = {};
    const int lens[2] = {nat_rows ? 0 : cols, nat_cols ? 0 : rows};
    int L2s[2] = {0, 0};
    int nrads[2] = {0, 0};
    unsigned long long rcodes[2] = {0, 0};
    for (int q = 0; q < 2; ++q) {
      if (!lens[q]) continue;
      std::vector<float2> mtw;
      if (!all_blue && smooth_line(lens[q], &nrads[q], &rcodes[q], &mtw)) {
        L2s[q] = smooth_L2(lens[q]);
        off[q][0] = tab.size();
        tab.insert(tab.end(), mtw.begin(), mtw.end());
        continue;
      }
      std::vector<float2> chirp, bhat;
      blue_tables(lens[q], &L2s[q], &chirp, &bhat);
      const std::vector<float2> tw = pass_table(L2s[q], blue_E(L2s[q]));
      off[q][0] = tab.size();
      tab.insert(tab.end(), chirp.begin(), chirp.end());
      off[q][1] = tab.size();
      tab.insert(tab.end(), bhat.begin(), bhat.end());
      off[q][2] = tab.size();
      tab.insert(tab.end(), tw.begin(), tw.end());
    }
    if (!tab.empty()) {
      if ((e = upload(&p->d_blue, tab)) != cudaSuccess) return cuda_fail(e, "generic line tables");
      BlueLine* bl[2] = {&p->bl_rows, &p->bl_cols};
      for (int q = 0; q < 2; ++q) {
        if (!lens[q]) continue;
        bl[q]->n = lens[q];
        bl[q]->L2 = L2s[q];
        if (nrads[q] > 0) {
          bl[q]->nrad = nrads[q];
          bl[q]->radices = rcodes[q];
          bl[q]->mtw = p->d_blue + off[q][0];
        } else {
          bl[q]->chirp = p->d_blue + off[q][0];
          bl[q]->bhat = p->d_blue + off[q][1];
          bl[q]->tw = p->d_blue + off[q][2];
        }
      }
    }
  }
  p->P = nat_cols ? cols_per_cta(rows) : blue_lines_per_block(p->bl_cols.L2);
  ptime.mark("twiddles");

  // supports
  if ((e = cudaMalloc(&p->d_planes, p->planes.size() * sizeof(PlaneDesc))) != cudaSuccess)
    return cuda_fail(e, "plane descriptors");
  cudaMemcpy(p->d_planes, p->planes.data(), p->planes.size() * sizeof(PlaneDesc), cudaMemcpyHostToDevice);
  {
    std::vector<int> mm(2 * p->eta);
    for (int i = 0; i < p->eta; ++i) {
      mm[2 * i] = INT_MAX;
      mm[2 * i + 1] = -1;
    }
    int* d_mm = nullptr;
    if ((e = cudaMalloc(&d_mm, mm.size() * sizeof(int))) != cudaSuccess) return cuda_fail(e, "support scratch");
    cudaMemcpy(d_mm, mm.data(), mm.size() * sizeof(int), cudaMemcpyHostToDevice);
    e = launch_support(p.get(), d_mm, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(mm.data(), d_mm, mm.size() * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d_mm);
    if (e != cudaSuccess) return cuda_fail(e, "ffst_plan support kernel");
    int rng_total = 0;
    for (int i = 0; i < p->eta; ++i) {
      if (mm[2 * i + 1] < 0) {
        p->planes[i].c0 = 0;
        p->planes[i].W = 0;
      } else {
        p->planes[i].c0 = mm[2 * i];
        p->planes[i].W = mm[2 * i + 1] - mm[2 * i] + 1;
      }
      set_slot(p->planes[i]);
      p->planes[i].rng_off = rng_total;
      rng_total += p->planes[i].W;
    }
    // per-column row ranges of every plane's support
    if ((e = cudaMalloc(&p->d_rng, (size_t)(rng_total > 0 ? rng_total : 1) * sizeof(int2))) != cudaSuccess)
      return cuda_fail(e, "row ranges");
    cudaMemcpy(p->d_planes, p->planes.data(), p->planes.size() * sizeof(PlaneDesc), cudaMemcpyHostToDevice);
    e = launch_ranges(p.get(), 0);
    if (e != cudaSuccess) return cuda_fail(e, "ffst_plan row ranges");
  }
  ptime.mark("support+ranges");

  // kernel configuration and groups (autotune cache, else FFST_GROUP_MB* and defaults)
  TuneConfig tc;
  const bool tuned = autotune_lookup(p.get(), FFST_STORE_F32, &tc);
  {
    double fmb = tc.fwd_mb, imb = tc.inv_mb;
    if (!tuned) default_group_mb(&fmb, &imb);
    const ffst_status st = plan_regroup(p.get(), fmb, imb);
    if (st != FFST_OK) return st;
    const int L = cols / 2;
    if (tc.fuse_fwd >= 0) p->fuse_fwd = tc.fuse_fwd;
    if (tc.fuse_inv >= 0) p->fuse_inv = tc.fuse_inv;
    if (nat_rows && tc.row_fwd >= 0 && row_variant_ok(L, tc.row_fwd, true)) p->row_fwd = tc.row_fwd;
    if (nat_rows && tc.row_inv >= 0 && row_variant_ok(L, tc.row_inv, false)) p->row_inv = tc.row_inv;
    // FFST_FUSE=0 (both directions) and FFST_FUSE_FWD=0/1 override the fused launches (A/B timing)
    if (const char* f = std::getenv("FFST_FUSE"))
      if (f[0] == '0') p->fuse_fwd = p->fuse_inv = 0;
    if (const char* f = std::getenv("FFST_FUSE_FWD")) p->fuse_fwd = f[0] == '0' ? 0 : 1;
  }
  ptime.mark("groups");

  // workspace
  const size_t spec = (size_t)rows * p->Hc;
  if ((e = cudaMalloc(&p->d_F, spec * sizeof(float2))) != cudaSuccess) return cuda_fail(e, "workspace F");
  if ((e = cudaMalloc(&p->d_err, sizeof(int))) != cudaSuccess || (e = cudaMemset(p->d_err, 0, sizeof(int))) != cudaSuccess)
    return cuda_fail(e, "error word");
  {
    if (nat_rows) {
      const int L = cols / 2, teams = kThreads / (L / row_E(L));
      p->row_blocks = (rows + teams - 1) / teams;
    } else {  // generic row blocks take two rows per line
      const int lines = blue_lines_per_block(p->bl_rows.L2);
      p->row_blocks = ((rows + 1) / 2 + lines - 1) / lines;
    }
    if ((e = cudaMalloc(&p->d_abs_partials, sizeof(float) * (size_t)p->eta * p->row_blocks)) != cudaSuccess)
      return cuda_fail(e, "statistics partials");
  }
  ptime.mark("workspace");
  {
    p->inv_split_default = default_inv_split(p.get());
    const int ns = (tuned && tc.inv_split >= 1 && tc.inv_split <= kMaxInvSplit) ? tc.inv_split : p->inv_split_default;
    const ffst_status st = plan_set_inv_split(p.get(), ns);
    if (st != FFST_OK) return st;
  }
  ptime.mark("accumulators");
  if ((e = cudaMalloc(&p->d_invD, spec * sizeof(float))) != cudaSuccess) return cuda_fail(e, "normalisation");
  if ((e = launch_inv_norm(p.get(), 0)) != cudaSuccess) return cuda_fail(e, "ffst_plan normalisation");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "ffst_plan");
  ptime.mark("normalisation");
  *out = p.release();
  return FFST_OK;
}

extern "C" ffst_status ffst_plan_info(ffst_plan_t plan, int* rows, int* cols, int* scales, int* num_planes) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plan_info: plan is NULL");
  if (rows) *rows = plan->M;
  if (cols) *cols = plan->N;
  if (scales) *scales = plan->j0;
  if (num_planes) *num_planes = plan->eta;
  return FFST_OK;
}

extern "C" ffst_status ffst_plane_index(ffst_plan_t plan, int i, int* cone, int* j, int* k) {
  if (!plan) return fail(FFST_ERR_INVALID_ARG, "ffst_plane_index: plan is NULL");
  if (i < 0 || i >= plan->eta) return fail(FFST_ERR_INVALID_ARG, "ffst_plane_index: index out of range");
  const PlaneDesc& d = plan->planes[i];
  if (cone) *cone = d.kappa;
  if (j) *j = d.j;
  if (k) *k = d.k;
  return FFST_OK;
}

extern "C" void ffst_destroy(ffst_plan_t plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  free_plan(plan);
}

extern "C" const char* ffst_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* ffst_status_string(int status) {
  switch (status) {
    case FFST_OK: return "FFST_OK";
    case FFST_ERR_INVALID_ARG: return "FFST_ERR_INVALID_ARG";
    case FFST_ERR_UNSUPPORTED_SIZE: return "FFST_ERR_UNSUPPORTED_SIZE";
    case FFST_ERR_OUT_OF_MEMORY: return "FFST_ERR_OUT_OF_MEMORY";
    case FFST_ERR_CUDA: return "FFST_ERR_CUDA";
    case FFST_ERR_TIMEOUT: return "FFST_ERR_TIMEOUT";
    case FFST_ERR_BOUNDS: return "FFST_ERR_BOUNDS";
    default: return "FFST_ERR_UNKNOWN";
  }
}
