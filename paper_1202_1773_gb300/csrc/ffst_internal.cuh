// Internal declarations of the FFST CUDA library (not part of the C ABI).
#pragma once

#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime's entry-point query)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ffst.h"

namespace ffst {

// ---------------------------------------------------------------------------
// Complex helpers (float2 = re, im)
// ---------------------------------------------------------------------------
// Complex add and subtract.  With FFST_PACKED_ADD (the default), device
// code runs both components as one packed FP32 instruction (add.f32x2, and
// a - b as fma.f32x2(b, -1, a), which is exact before its one rounding): two
// round-to-nearest results in half the issue slots.  The packed add is never
// contracted with a preceding multiply, so results can differ from the
// scalar build (-DFFST_PACKED_ADD=0) by rounding where that build formed an
// FMA.  2048x2048 J=5 on a GB300: inverse 1.053 -> 1.028 ms, forward even.
#ifndef FFST_PACKED_ADD
#define FFST_PACKED_ADD 1
#endif
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && FFST_PACKED_ADD
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && FFST_PACKED_ADD
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Compile-time trigonometry for the constant twiddles inside radix-R DFTs.
// Plain Taylor series of sin and cos (double), after reducing the angle
// 2*pi*m/R to [-pi, pi]; 30 terms reach double precision there.  Only ever
// evaluated by the compiler to fold constants.
// ---------------------------------------------------------------------------
constexpr double kPi = 3.141592653589793238462643383279502884;

__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 30; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 30; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
// angle of the m-th R-th root of unity, reduced to [-pi, pi]
__host__ __device__ constexpr double root_angle(int m, int R) {
  int mm = ((m % R) + R) % R;
  if (2 * mm > R) mm -= R;
  return 2.0 * kPi * (double)mm / (double)R;
}
__host__ __device__ constexpr float root_cos(int m, int R) { return (float)taylor_cos(root_angle(m, R)); }
__host__ __device__ constexpr float root_sin(int m, int R) { return (float)taylor_sin(root_angle(m, R)); }

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// Elements per thread of the line FFTs.  Row kernels transform real rows of
// length N as complex lines of length L = N/2 (one warp per line at L =
// 1024); column kernels transform columns of length L = M.
// Build-time knobs (defaults are the tuned configuration): elements per
// thread of long row lines, and the minimum resident blocks per SM the
// compiler must allow for (caps registers per thread at 65536/(256*n)).
#ifndef FFST_ROW_E_LONG
#define FFST_ROW_E_LONG 16
#endif
#ifndef FFST_THREADS
#define FFST_THREADS 256
#endif
#ifndef FFST_MIN_BLOCKS
#define FFST_MIN_BLOCKS (1024 / FFST_THREADS)
#endif
__host__ __device__ constexpr bool is_pow2c(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Resident blocks per SM a column-length-L kernel's register budget is sized
// for: 4096-point columns hold 32 elements per thread (64 registers of data
// alone), so their kernels take the budget of two blocks instead of spilling.
__host__ __device__ constexpr int min_blocks_for(int L) { return L >= 4096 ? 2 : FFST_MIN_BLOCKS; }

// Line lengths with factors 3 or 5 (mixed radix) run 16 or 32 threads per
// line; powers of two use the register configuration below.
__host__ __device__ constexpr int mixed_E(int L) { return L / (L <= 256 ? 16 : 32); }
__host__ __device__ constexpr int row_E(int L) {
  return !is_pow2c(L) ? mixed_E(L) : (L >= 1024 ? FFST_ROW_E_LONG : (L >= 16 ? 16 : L));
}
__host__ __device__ constexpr int col_E(int L) {
  return !is_pow2c(L) ? mixed_E(L) : (L >= 4096 ? 32 : (L >= 16 ? 16 : L));
}

// Radix of the pass of a line of length L that starts at sub-transform
// length Ns: min(E, L/Ns) for powers of two; otherwise the largest of
// 16, 8, 4, 2 dividing what is left, then 3, then 5.
__host__ __device__ constexpr int next_radix(int L, int E, int Ns) {
  const int rem = L / Ns;
  if (is_pow2c(L)) return rem < E ? rem : E;
  if (rem % 16 == 0) return 16;
  if (rem % 8 == 0) return 8;
  if (rem % 4 == 0) return 4;
  if (rem % 2 == 0) return 2;
  if (rem % 3 == 0) return 3;
  return 5;
}

__host__ __device__ constexpr int num_passes(int L, int E) {
  int n = 0;
  for (int Ns = 1; Ns < L; Ns *= next_radix(L, E, Ns)) ++n;
  return n;
}

// Line lengths the kernels are built for: powers of two 4..4096 and
// 240, 320, 384, 480, 640, 768 (factors 2, 3, 5).
__host__ __device__ constexpr bool supported_line(int L) {
  return (is_pow2c(L) && L >= 4 && L <= 4096) || L == 240 || L == 320 || L == 384 || L == 480 || L == 640 ||
         L == 768;
}

// Every transform kernel runs blocks of kThreads threads, so a row-pass block
// and a column-pass block can share one fused launch.
constexpr int kThreads = FFST_THREADS;

// Entry idx of the pass twiddle table of a line (L, E) (see ffst_fft.cuh):
// pass with sub-transform length Ns and radix R = min(E, L/Ns) owns indices
// [Ns - 1, Ns R - 1); index Ns - 1 + (r - 1) Ns + kk holds W_{Ns R}^{kk r}.
// Returns the value as the root of unity exp(-2 pi i m / n).
__host__ __device__ inline void pass_entry(int L, int E, int idx, int* m, int* n) {
  int Ns = 1;
  while (Ns < L) {
    const int R = next_radix(L, E, Ns);
    if (idx < Ns * R - 1) {
      const int q = idx - (Ns - 1);
      *m = (q % Ns) * (q / Ns + 1);
      *n = Ns * R;
      return;
    }
    Ns *= R;
  }
  *m = 0;
  *n = 1;
}

// ---------------------------------------------------------------------------
// Plan data shared with the kernels
// ---------------------------------------------------------------------------

// Plane kinds (kappa of Sec. 3.1), same values as FFST_CONE_*.
enum : int { kLowpass = 0, kH = 1, kV = 2, kSeam = 3 };

// Per-plane descriptor, device resident.
struct PlaneDesc {
  int kappa;      // kLowpass / kH / kV / kSeam
  int j;          // scale 0..j0-1 (-1 for the low-pass)
  int k;          // shear, |k| <= 2^j
  int c0;         // first half-spectrum column with psi != 0
  int W;          // number of support columns (0: plane identically zero)
  int item0;      // first forward column work item of this plane (global index)
  int nitems;     // number of forward column work items
  int rng_off;    // offset of the plane's per-column row ranges (W entries)
  int c0al;       // first column of the plane's intermediate slot: c0 rounded down to even
  int ldw;        // row pitch of the slot: columns c0al .. c0 + W - 1, rounded up to even
  long long off;  // offset of the plane's column-pass intermediate inside its group (float2 units)
};

// Slot geometry of a plane's intermediate: rows of ldw complex values
// starting at column c0al, both even, so every row and every 2-column
// panel starts on a 16-byte boundary (what a TMA tile access needs).
__host__ __device__ inline void set_slot(PlaneDesc& d) {
  d.c0al = d.c0 & ~1;
  d.ldw = d.W ? ((d.c0 + d.W - d.c0al + 1) & ~1) : 0;
}

// Everything the in-register window generator needs (passed by value).
struct WinParams {
  int M, N;        // rows (omega_2 axis), cols (omega_1 axis)
  int hm, hn;      // floor(M/2), floor(N/2): table lengths - 1
  int gm, gn;      // grid denominators: xi2 = omega_2 X / gm, xi1 = omega_1 X / gn
                   // (one step: gm = gn = floor(max(M, N)/2); per axis: hm, hn)
  const float* psi1_col;  // [j0][hn+1]: psi1(4^-j * a * dc), a = |omega_1|
  const float* psi1_row;  // [j0][hm+1]: psi1(4^-j * a * dr), a = |omega_2|
  const float* phi_col;   // [hn+1]:     varphi(a * dc)
  const float* phi_row;   // [hm+1]:     varphi(a * dr)
  // auxiliary function v of psi2 (Sec. 2.1, Sec. 3.4 remark construction_v):
  // FFST_V_MEYER, FFST_V_QUADRATIC, FFST_V_POLY (coefficients vc[0..vdeg]
  // of v on [0, 1/2]) or FFST_V_CINF
  int vkind, vdeg;
  float vc[16];
  // smooth shearlets (Sec. 3.4): per scale j, with w = 4^-j a d (d = dc or dr)
  int smooth;
  const float* sig_col;   // [j0][hn+1]: 1 - varphi(w)^2
  const float* sig_row;   // [j0][hm+1]
  const float* alp_col;   // [j0][hn+1]: varphi(w / 4)^2
  const float* alp_row;   // [j0][hm+1]
};

// One column-panel work item of the forward column pass.
struct ColItem {
  int plane;  // plane index
  int col;    // first half-spectrum column of the panel
};

// Kernel kinds for the per-kernel timers.
enum TimingKind : int {
  kTimeImgRows = 0,   // image rows R2C
  kTimeImgCols,       // image column FFT
  kTimeFwdCols,       // forward plane column pass (generate psi, multiply, IFFT)
  kTimeFwdRows,       // forward plane row C2R + store of the stack
  kTimeInvRows,       // inverse plane row R2C (reads the stack)
  kTimeInvCols,       // inverse column FFT, multiply, accumulate
  kTimeOutCols,       // final column IFFT (with normalisation)
  kTimeOutRows,       // final row C2R to the image
  kTimeFwdFused,      // forward: column pass of group g fused with row pass of group g-1
  kTimeInvFused,      // inverse: row pass of group g fused with column pass of group g-1
  kTimeFwdSched,      // forward: all plane passes in one persistent launch
  kTimeInvSched,      // inverse: all plane passes in one persistent launch
  kTimeOther,         // spectra export, plane scales
  kTimeKinds
};

struct Group {
  int p0, p1;              // planes [p0, p1)
  long long elems;         // float2 elements of the group's intermediate
  int item0, nitems;       // forward column items
};

struct Timer {
  bool enabled = false;
  struct Rec { int kind; cudaEvent_t a, b; double bytes; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  double total_ms[kTimeKinds] = {0};
  long long launches[kTimeKinds] = {0};
  double bytes[kTimeKinds] = {0};
};

}  // namespace ffst

namespace ffst {

// Persistent schedule of the plane passes (square sizes, ffst_sched.cu).
// One launch per direction walks an ordered task queue; per-plane counters
// carry the dependencies (rows of a plane after its columns, reuse of the
// intermediate ring after its readers).
// Tables of the generic-length lines of one dimension (ffst_blue.cuh).
struct BlueLine {
  int n = 0;                      // line length; 0: the dimension runs native FFT lines
  int L2 = 0;                     // the power of two >= 2n - 1 (thread layout; Bluestein convolution length)
  const float2* chirp = nullptr;  // w_j = exp(-i pi j^2 / n), j < n (FP64-generated)
  const float2* bhat = nullptr;   // FFT_L2 of the filter conj(w_|m|), times 1/L2
  const float2* tw = nullptr;     // pass table (L2, blue_E(L2))
  // n with no prime factor above 7: the DFT runs as mixed-radix Stockham
  // passes in shared memory instead of Bluestein (nrad > 0)
  int nrad = 0;                   // number of passes
  unsigned long long radices = 0; // radix of pass s in bits [4s, 4s + 4): 2, 3, 4, 5, 7 or 8
  const float2* mtw = nullptr;    // pass twiddles W_{Ns R}^{kk r} at (Ns - 1) + (r - 1) Ns + kk
};

struct Sched {
  bool on = false;
  double ring_mb = 0.0;
  float2* d_ring = nullptr;             // intermediate ring
  long long ring_elems = 0;
  PlaneDesc* d_planes = nullptr;        // descriptors with ring offsets
  int4* d_fwd = nullptr;                // forward queue
  int n_fwd = 0;
  int4* d_inv = nullptr;                // inverse queue
  int n_inv = 0;
  int4* d_pdep = nullptr;               // per plane: ring predecessors [x, y], their batches [z, w]
  int2* d_batch = nullptr;              // per inverse batch: planes [x, y)
  int* d_batch_tasks = nullptr;         // per inverse batch: column tasks
  int* d_batch_part = nullptr;          // per inverse batch: partial accumulator
  int* d_ctl = nullptr;                 // per launch counters (zeroed before each launch)
  int ctl_ints = 0;
  int off_cols = 0, off_rows = 0, off_batch = 0, off_panel = 0;  // counter arrays inside d_ctl
  int nbatch = 0, npanels = 0, blocks = 0, rbx = 0;
};

}  // namespace ffst

struct ffst_plan_s {
  int M = 0, N = 0, j0 = 0, eta = 0, Hc = 0;
  int pr0 = 0, pr1 = 0;                 // active plane range [pr0, pr1) of the plane passes (default: all)
  int variant = 0;                      // FFST_VARIANT_CLASSIC or FFST_VARIANT_SMOOTH
  int hm = 0, hn = 0;
  int device = 0;
  std::vector<ffst::PlaneDesc> planes;  // host copy
  ffst::PlaneDesc* d_planes = nullptr;
  float* d_tables = nullptr;            // psi1_col | psi1_row | phi_col | phi_row
  ffst::WinParams win{};
  float2* d_tw_rows = nullptr;          // pass twiddles of the row lines (N/2, row_E)
  float2* d_tw_rows32 = nullptr;        // pass twiddles of 32-element row lines (N/2 = 1024, 2048 only)
  // kernel configuration (ffst_plan_set_kernels, ffst_plan_autotune): fused
  // plane-pass launches per direction, and the row kernel variant of the
  // standalone row passes (0 default, 1 paired rows, 2 32 elements per thread;
  // the fused launches always use variant 0)
  int fuse_fwd = 1, fuse_inv = 1;
  int row_fwd = 0, row_inv = 0;
  float2* d_rtw = nullptr;              // exp(-2 pi i k / N), k = 0..N/2 (real-FFT split)
  float2* d_tw_cols = nullptr;          // pass twiddles of the column lines (M, col_E)
  int2* d_rng = nullptr;                // per (plane, support column): cyclic row range (start, len)
  float2* d_F = nullptr;                // [M][Hc] image spectrum
  float2* d_S = nullptr;                // inv_split x [M][Hc] inverse partial accumulators
  int inv_split = 1;                    // plane chunks per inverse group (partial accumulators)
  int inv_split_cap = 0;                // partial accumulators allocated
  int inv_split_default = 1;            // the plan's choice at creation
  int P = 0;                            // columns per column-pass block (panel width)
  ffst::BlueLine bl_rows, bl_cols;      // generic-length lines (n = 0: native FFT lines)
  float2* d_blue = nullptr;             // their tables
  float* d_invD = nullptr;              // [M][Hc] 1 / sum_i psi_i^2 (FP32 psi), inverse normalisation
  float2* d_H = nullptr;                // two group intermediates (double buffer), h_elems each
  long long h_elems = 0;
  float* d_partials = nullptr;          // [total items] per-panel sums of |psi F| (low-precision storage)
  int total_items = 0;
  std::vector<ffst::Group> groups;      // forward plane groups (slot offsets in planes / d_planes)
  double group_mb = 0.0;                // budget the forward groups were built for
  std::vector<ffst::Group> groups_inv;  // inverse plane groups
  double group_mb_inv = 0.0;
  ffst::PlaneDesc* d_planes_inv = nullptr;  // descriptors with the inverse groups' slot offsets
  ffst::ColItem* d_items = nullptr;
  CUtensorMap* d_tmaps = nullptr;       // per plane: TMA map of its forward slot (or null)
  CUtensorMap* d_tmaps_inv = nullptr;   // per plane: TMA map of its inverse slot (or null)
  int* d_err = nullptr;                 // sticky device error word (bounded waits), read by ffst_plan_check
  float* d_abs_partials = nullptr;      // [eta][row_blocks] sum |c| per row block (ffst_forward_stats)
  int row_blocks = 0;                   // row-pass blocks per plane
  ffst::Sched sched;
  int sched_mode = 0;                   // 0: grouped launches, 1: persistent, 2: persistent with a stuck wait (test)
  ffst::Timer timer;
};

namespace ffst {

// thread-local error reporting
void set_error(const std::string& msg);
ffst_status fail(ffst_status st, const std::string& msg);
ffst_status cuda_fail(cudaError_t e, const char* what);

// plan grouping and autotuning (ffst_plan.cu, ffst_autotune.cu)
void default_group_mb(double* fwd_mb, double* inv_mb);
ffst_status plan_regroup(ffst_plan_s* p, double fwd_mb, double inv_mb);
// Plane chunks of the inverse column pass: chunk k of inv_split holds the
// planes [eta k / inv_split, eta (k + 1) / inv_split) (the device's
// inv_chunk boundaries) and is summed into partial accumulator k, whatever
// the plane groups; inv_part gives a plane's k.
constexpr int kMaxInvSplit = 16;
int inv_part(const ffst_plan_s* p, int plane);
ffst_status plan_set_inv_split(ffst_plan_s* p, int n);
// A tuned configuration of one plan shape (ffst_plan_autotune's cache entry).
struct TuneConfig {
  double fwd_mb = 0.0, inv_mb = 0.0;        // plane-group budgets
  int fuse_fwd = -1, fuse_inv = -1;         // -1: not in the entry (keep the defaults)
  int row_fwd = -1, row_inv = -1;
  int inv_split = -1;
};
bool autotune_lookup(const ffst_plan_s* p, int storage, TuneConfig* cfg);
// row kernel variant v (ffst_rows.cu) exists for half-length L
bool row_variant_ok(int L, int variant, bool c2r);
constexpr int kRowVariants = 4;  // row-FFT variants 0..3 (ffst_rows.cu)
// fused plane-pass launches exist for this shape (ffst_fused.cu)
bool fused_supported(int M, int N);
// give plan q the launch configuration (budgets, kernels, plane chunks) of plan p of the same shape
ffst_status copy_tuning(const ffst_plan_s* p, ffst_plan_s* q);

// timing helpers
void timer_begin(ffst_plan_s* p, int kind, cudaStream_t s, double bytes, cudaEvent_t* out_b);
void timer_end(ffst_plan_s* p, cudaStream_t s, cudaEvent_t b);

// plan-time kernels (ffst_plan.cu)
cudaError_t launch_spectra(const ffst_plan_s* p, float* psi, cudaStream_t s);
cudaError_t launch_support(const ffst_plan_s* p, int* d_minmax, cudaStream_t s);
cudaError_t launch_ranges(const ffst_plan_s* p, cudaStream_t s);
cudaError_t launch_inv_norm(const ffst_plan_s* p, cudaStream_t s);
cudaError_t launch_plane_scales(const ffst_plan_s* p, const Group& g, const float* partials, float target,
                                float* plane_scale, cudaStream_t s);
cudaError_t launch_mean_abs(const ffst_plan_s* p, float* mean_abs, cudaStream_t s);

// Opt a kernel into more than 48 KB of shared memory.  The kernels also
// hold up to 1 KB of static shared memory (reductions, barriers), which
// counts against the default 48 KB.
template <typename K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes + 1024 <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// per-length launch geometry of the column kernels (columns per CTA)
int cols_per_cta(int L);

// TMA panel maps (ffst_tma_maps.cu), rebuilt whenever the group buffers change
ffst_status tma_build(ffst_plan_s* p, const std::vector<long long>& off_fwd, const std::vector<long long>& off_inv);
void tma_free(ffst_plan_s* p);

// persistent schedule (ffst_sched.cu)
double default_ring_mb();
ffst_status sched_build(ffst_plan_s* p, double ring_mb);
void sched_free(ffst_plan_s* p);

}  // namespace ffst
