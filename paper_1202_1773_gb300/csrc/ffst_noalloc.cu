// ffst_forward_noalloc: a forward transform for small images that allocates
// no memory at all.
//
// Who needs it: callers that cannot call cudaMalloc.  Examples are
// processes whose framework has already reserved nearly all device memory
// for its own pool, plug-ins running inside a host application that owns
// the device's allocator and hands out buffers but no right to allocate,
// and real-time or embedded hosts whose rules forbid allocation after
// start-up.  ffst_plan allocates its tables and workspace, so these callers
// cannot build a plan.
//
// How: every table and every intermediate of this entry point lives in the
// file-scope device array g_noalloc_scratch below (kNoallocBytes, about
// 2.5 MB), which the CUDA module reserves once on every GPU that loads the
// library and keeps until the process exits.  The caller passes the input
// image and the output stack only.  Host code cannot use the array's name
// as a device address, so every call looks the address up with
// cudaGetSymbolAddress on the current device (a host-side lookup that
// allocates nothing; after a context reset the module reloads and the
// array may move, so the address is never cached).  The first call on a
// device loads the library's device code there and sets the array up, so
// make that first call before any stream capture begins.  Every call shares the one array and leaves its contents
// behind; each call writes every scratch word it later reads, so nothing
// needs clearing, but two calls whose work overlaps on the GPU (different
// streams, or different host threads on the same device) race on the
// scratch and corrupt each other's results.
//
// Limits: rows and cols powers of two in [8, 256], scales in 1..4 (or <= 0
// for the default).  Larger requests return FFST_ERR_UNSUPPORTED_SIZE
// before anything is enqueued.  Spectral supports are not pruned here (every
// column of every plane is transformed); results equal ffst_forward's to
// FP32 rounding.
#include <cstring>

#include "ffst_kernels.cuh"

namespace ffst {
namespace {

constexpr int kNaMaxSide = 256;
constexpr int kNaMaxScales = 4;
constexpr int kNaMaxPlanes = (1 << (kNaMaxScales + 2)) - 3;  // 61
constexpr int kNaGroup = 8;                                  // planes per column/row pass pair
constexpr long long kNaSpec = (long long)kNaMaxSide * (kNaMaxSide / 2 + 1);  // M x (N/2+1) complex
constexpr long long kNaSlot = (long long)kNaMaxSide * (kNaMaxSide / 2 + 2);  // one plane's intermediate (even pitch)
// Column panels per plane: ceil((N/2 + 1) / P) with P columns per column block
// (ColCfg); P shrinks as the column length grows, so the tallest image has the
// most panels (16 x 256 columns per block at the default 256 threads).
constexpr int kNaMinP = ColCfg<kNaMaxSide>::P;
constexpr int kNaMaxPanels = (kNaMaxSide / 2 + 1 + kNaMinP - 1) / kNaMinP;
constexpr long long kNaMaxItems = (long long)kNaMaxPlanes * kNaMaxPanels;
constexpr long long kNaTabFloats = 2LL * kNaMaxScales * (kNaMaxSide / 2 + 1) + 2 * (kNaMaxSide / 2 + 1);

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr long long align256(long long b) { return (b + 255) / 256 * 256; }
constexpr long long kOffF = 0;
constexpr long long kOffH = align256(kOffF + kNaSpec * 8);
constexpr long long kOffPlanes = align256(kOffH + kNaGroup * kNaSlot * 8);
constexpr long long kOffItems = align256(kOffPlanes + kNaMaxPlanes * (long long)sizeof(PlaneDesc));
constexpr long long kOffTab = align256(kOffItems + kNaMaxItems * (long long)sizeof(ColItem));
constexpr long long kOffTwR = align256(kOffTab + kNaTabFloats * 4);            // row pass table, N/2 entries
constexpr long long kOffRtw = align256(kOffTwR + (kNaMaxSide / 2) * 8);          // real split, N/2 + 1 entries
constexpr long long kOffTwC = align256(kOffRtw + (kNaMaxSide / 2 + 1) * 8);      // column pass table, M entries
constexpr long long kOffRng = align256(kOffTwC + kNaMaxSide * 8);                // row ranges, eta x (N/2 + 1)
constexpr long long kNoallocBytes = align256(kOffRng + kNaMaxPlanes * (kNaMaxSide / 2 + 1) * 8LL);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// FP64 window values on the device, for the tables only (Sec. 2.1, 2.4, 3.4).
__device__ double na_v(double x) {
  if (x <= 0.0) return 0.0;
  if (x >= 1.0) return 1.0;
  const double y = x <= 0.5 ? x : 1.0 - x;
  const double y2 = y * y;
  const double p = y2 * y2 * (35.0 + y * (-84.0 + y * (70.0 - 20.0 * y)));
  return x <= 0.5 ? p : 1.0 - p;
}
__device__ double na_psi1(double w) {
  w = fabs(w);
  if (w <= 0.5) return 0.0;
  if (w < 1.0) return sinpi(0.5 * na_v(2.0 * w - 1.0));
  if (w <= 2.0) return 1.0;
  if (w < 4.0) return cospi(0.5 * na_v(0.5 * w - 1.0));
  return 0.0;
}
__device__ double na_varphi(double w) {
  w = fabs(w);
  if (w <= 0.5) return 1.0;
  if (w < 1.0) return cospi(0.5 * na_v(2.0 * w - 1.0));
  return 0.0;
}

struct NaSetup {
  int M, N, j0, eta, Hc, P, ipp;  // ipp: column panels per plane
  float* tab;                      // psi1_col | psi1_row | phi_col | phi_row
  float2* twr;                     // pass table of the row lines (N/2, row_E)
  float2* rtw;                     // e^{-2 pi i k/N}, k = 0..N/2
  float2* twc;                     // pass table of the column lines (M, col_E)
  int2* rng;                       // row ranges: the full column for every (plane, column)
  PlaneDesc* planes;
  ColItem* items;
};

__device__ float2 na_root(int m, int n) {
  double sn, cs;
  sincospi(2.0 * m / n, &sn, &cs);
  return make_float2((float)cs, (float)-sn);
}

// Plane index -> (kappa, j, k) in the order of Sec. 3.5.2.
__device__ void na_plane(int i, int* kappa, int* j, int* k) {
  if (i == 0) {
    *kappa = kLowpass;
    *j = -1;
    *k = 0;
    return;
  }
  int jj = 0, base = 1;
  while (i >= base + (4 << jj)) {
    base += 4 << jj;
    ++jj;
  }
  const int J = 1 << jj, l = i - base;
  *j = jj;
  if (l == 0) { *kappa = kH; *k = 0; }
  else if (l < J) { *kappa = kH; *k = -l; }
  else if (l == J) { *kappa = kSeam; *k = -J; }
  else if (l < 3 * J) { *kappa = kV; *k = l - 2 * J; }
  else if (l == 3 * J) { *kappa = kSeam; *k = J; }
  else { *kappa = kH; *k = 4 * J - l; }
}

__global__ void k_na_setup(NaSetup s) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  const int hn = s.N / 2, hm = s.M / 2;
  const double X = ldexp(1.0, 2 * s.j0 - 1);
  const double dc = X / (s.M > s.N ? hm : hn), dr = dc;  // one step for both axes (Sec. 3.5.1)
  float* psi1_col = s.tab;
  float* psi1_row = psi1_col + s.j0 * (hn + 1);
  float* phi_col = psi1_row + s.j0 * (hm + 1);
  float* phi_row = phi_col + (hn + 1);
  for (int q = tid; q < s.j0 * (hn + 1); q += stride) {
    const int j = q / (hn + 1), a = q % (hn + 1);
    psi1_col[q] = (float)na_psi1(ldexp(1.0, -2 * j) * a * dc);
  }
  for (int q = tid; q < s.j0 * (hm + 1); q += stride) {
    const int j = q / (hm + 1), a = q % (hm + 1);
    psi1_row[q] = (float)na_psi1(ldexp(1.0, -2 * j) * a * dr);
  }
  for (int q = tid; q <= hn; q += stride) phi_col[q] = (float)na_varphi(q * dc);
  for (int q = tid; q <= hm; q += stride) phi_row[q] = (float)na_varphi(q * dr);
  const int Lr = s.N / 2;
  for (int q = tid; q < Lr; q += stride) {
    int m = 0, n = 1;
    if (q < Lr - 1) pass_entry(Lr, row_E(Lr), q, &m, &n);
    s.twr[q] = na_root(m, n);
  }
  for (int q = tid; q <= Lr; q += stride) s.rtw[q] = na_root(q, s.N);
  for (int q = tid; q < s.M; q += stride) {
    int m = 0, n = 1;
    if (q < s.M - 1) pass_entry(s.M, col_E(s.M), q, &m, &n);
    s.twc[q] = na_root(m, n);
  }
  for (int q = tid; q < s.eta * s.Hc; q += stride) s.rng[q] = make_int2(0, s.M);
  for (int i = tid; i < s.eta; i += stride) {
    PlaneDesc d{};
    na_plane(i, &d.kappa, &d.j, &d.k);
    d.c0 = 0;
    d.W = s.Hc;
    set_slot(d);
    d.item0 = i * s.ipp;
    d.nitems = s.ipp;
    d.rng_off = i * s.Hc;
    d.off = (long long)(i % kNaGroup) * s.M * d.ldw;
    s.planes[i] = d;
  }
  for (int q = tid; q < s.eta * s.ipp; q += stride) s.items[q] = ColItem{q / s.ipp, (q % s.ipp) * s.P};
}

// Device address of the scratch array on the current device, looked up on
// every call with that device current (never cached: a context reset reloads
// the module and may move the array).
ffst_status na_scratch(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "ffst_forward_noalloc: cudaGetSymbolAddress");
  *out = static_cast<unsigned char*>(p);
  return FFST_OK;
}

}  // namespace
}  // namespace ffst

using namespace ffst;

extern "C" ffst_status ffst_forward_noalloc(int rows, int cols, int scales, const float* img, float* coeffs,
                                            void* stream) {
  if (!img || !coeffs) return fail(FFST_ERR_INVALID_ARG, "ffst_forward_noalloc: NULL argument");
  auto pow2 = [](int n) { return n > 0 && (n & (n - 1)) == 0; };
  if (!pow2(rows) || !pow2(cols) || rows < 8 || cols < 8 || rows > kNaMaxSide || cols > kNaMaxSide)
    return fail(FFST_ERR_UNSUPPORTED_SIZE, "ffst_forward_noalloc: rows and cols must be powers of two in [8, " +
                                               std::to_string(kNaMaxSide) + "] (the static scratch limit), got " +
                                               std::to_string(rows) + "x" + std::to_string(cols));
  const int mx = rows > cols ? rows : cols;
  int lg = 0;
  while ((1 << (lg + 1)) <= mx) ++lg;
  const int j0 = scales > 0 ? scales : lg / 2;
  if (j0 < 1 || j0 > kNaMaxScales)
    return fail(FFST_ERR_UNSUPPORTED_SIZE, "ffst_forward_noalloc: scales must be in 1.." +
                                               std::to_string(kNaMaxScales) + ", got " + std::to_string(j0));
  unsigned char* base = nullptr;
  ffst_status st = na_scratch(&base);
  if (st != FFST_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // A plan object that only points into the scratch array (no allocation).
  ffst_plan_s P;
  P.M = rows;
  P.N = cols;
  P.j0 = j0;
  P.eta = (1 << (j0 + 2)) - 3;
  P.Hc = cols / 2 + 1;
  P.hm = rows / 2;
  P.hn = cols / 2;
  P.d_F = reinterpret_cast<float2*>(base + kOffF);
  P.d_H = reinterpret_cast<float2*>(base + kOffH);
  P.d_planes = reinterpret_cast<PlaneDesc*>(base + kOffPlanes);
  P.d_items = reinterpret_cast<ColItem*>(base + kOffItems);
  P.d_tw_rows = reinterpret_cast<float2*>(base + kOffTwR);
  P.d_rtw = reinterpret_cast<float2*>(base + kOffRtw);
  P.d_tw_cols = reinterpret_cast<float2*>(base + kOffTwC);
  P.d_rng = reinterpret_cast<int2*>(base + kOffRng);
  float* tab = reinterpret_cast<float*>(base + kOffTab);
  P.win.M = rows;
  P.win.N = cols;
  P.win.hm = P.hm;
  P.win.hn = P.hn;
  P.win.gm = P.win.gn = (rows > cols ? rows : cols) / 2;
  P.win.psi1_col = tab;
  P.win.psi1_row = tab + j0 * (P.hn + 1);
  P.win.phi_col = P.win.psi1_row + j0 * (P.hm + 1);
  P.win.phi_row = P.win.phi_col + (P.hn + 1);
  P.win.smooth = 0;  // the classic construction, eq. (v), X = 2^{2 j0 - 1} only
  P.win.vkind = FFST_V_MEYER;
  P.win.vdeg = 0;
  P.win.sig_col = P.win.sig_row = P.win.alp_col = P.win.alp_row = nullptr;

  NaSetup su;
  su.M = rows;
  su.N = cols;
  su.j0 = j0;
  su.eta = P.eta;
  su.Hc = P.Hc;
  su.P = cols_per_cta(rows);
  su.ipp = (P.Hc + su.P - 1) / su.P;
  if (su.P < 1 || (long long)su.ipp * P.eta > kNaMaxItems)  // kNaMaxItems covers kNaMaxSide; checked anyway
    return fail(FFST_ERR_UNSUPPORTED_SIZE, "ffst_forward_noalloc: column work items exceed the static scratch");
  su.tab = tab;
  su.twr = P.d_tw_rows;
  su.rtw = P.d_rtw;
  su.twc = P.d_tw_cols;
  su.rng = P.d_rng;
  su.planes = P.d_planes;
  su.items = P.d_items;
  k_na_setup<<<64, 256, 0, s>>>(su);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "ffst_forward_noalloc: setup");

  const long long plane = (long long)rows * cols;
  R2CArgs ia;
  std::memset(&ia, 0, sizeof(ia));
  ia.src = img;
  ia.st = FFST_STORE_F32;
  ia.M = rows;
  ia.dst = P.d_F;
  ia.W = P.Hc;
  ia.ld = P.Hc;
  ia.tw = P.d_tw_rows;
  ia.rtw = P.d_rtw;
  ia.src_bytes = plane * (long long)sizeof(float);
  ia.dst_bytes = (long long)rows * P.Hc * (long long)sizeof(float2);
  e = launch_rows_r2c(cols / 2, ia, 1, s);
  if (e == cudaSuccess)
    e = launch_cols_fft(rows, P.d_F, P.Hc, P.Hc, false, nullptr, P.d_tw_cols, s, 1, 0,
                        (long long)rows * P.Hc * (long long)sizeof(float2), nullptr);
  for (int p0 = 0; p0 < P.eta && e == cudaSuccess; p0 += kNaGroup) {
    const int p1 = p0 + kNaGroup < P.eta ? p0 + kNaGroup : P.eta;
    FwdColsArgs ca;
    ca.F = P.d_F;
    ca.Hc = P.Hc;
    ca.planes = P.d_planes;
    ca.items = P.d_items + p0 * su.ipp;
    ca.rng = P.d_rng;
    ca.H = P.d_H;
    ca.w = P.win;
    ca.tw = P.d_tw_cols;
    ca.partials = nullptr;
    ca.gain = 1.0f / (kR2CGain * (float)plane);
    ca.tmaps = nullptr;
    ca.odd = 0;
    ca.F_bytes = (long long)rows * P.Hc * (long long)sizeof(float2);
    ca.H_bytes = kNaGroup * kNaSlot * (long long)sizeof(float2);
    ca.err = nullptr;
    e = launch_fwd_cols(rows, ca, (p1 - p0) * su.ipp, s);
    if (e != cudaSuccess) break;
    C2RArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.src = P.d_H;
    ra.planes = P.d_planes;
    ra.M = rows;
    ra.plane0 = p0;
    ra.dst = coeffs + (long long)p0 * plane;
    ra.dst_plane_stride = plane;
    ra.st = FFST_STORE_F32;
    ra.scale = 1.0f;
    ra.tw = P.d_tw_rows;
    ra.rtw = P.d_rtw;
    ra.src_bytes = kNaGroup * kNaSlot * (long long)sizeof(float2);
    ra.dst_bytes = (long long)(p1 - p0) * plane * (long long)sizeof(float);
    e = launch_rows_c2r(cols / 2, ra, p1 - p0, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "ffst_forward_noalloc: transform");
  return FFST_OK;
}
