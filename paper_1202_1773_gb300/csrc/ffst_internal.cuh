// Internal declarations of the FFST CUDA library (not part of the C ABI).
#pragma once

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
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
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
  int pad_;
  long long off;  // offset of the plane's column-pass intermediate inside its group (float2 units)
};

// Everything the in-register window generator needs (passed by value).
struct WinParams {
  int M, N;        // rows (omega_2 axis), cols (omega_1 axis)
  int hm, hn;      // floor(M/2), floor(N/2)
  const float* psi1_col;  // [j0][hn+1]: psi1(4^-j * a * dc), a = |omega_1|
  const float* psi1_row;  // [j0][hm+1]: psi1(4^-j * a * dr), a = |omega_2|
  const float* phi_col;   // [hn+1]:     varphi(a * dc)
  const float* phi_row;   // [hm+1]:     varphi(a * dr)
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
  kTimeOther,         // spectra export, support, clears
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

struct ffst_plan_s {
  int M = 0, N = 0, j0 = 0, eta = 0, Hc = 0;
  int hm = 0, hn = 0;
  int device = 0;
  std::vector<ffst::PlaneDesc> planes;  // host copy
  ffst::PlaneDesc* d_planes = nullptr;
  float* d_tables = nullptr;            // psi1_col | psi1_row | phi_col | phi_row
  ffst::WinParams win{};
  float2* d_tw_rows = nullptr;          // twiddles of length N (row FFTs)
  float2* d_tw_cols = nullptr;          // twiddles of length M (column FFTs)
  float2* d_F = nullptr;                // [M][Hc] image spectrum
  float2* d_S = nullptr;                // [M][Hc] inverse accumulator
  float* d_D = nullptr;                 // [M][Hc] sum of psi^2
  float2* d_H = nullptr;                // group intermediate
  long long h_elems = 0;
  float* d_partials = nullptr;          // [total items] per-panel sums of |psi F| (low-precision storage)
  int total_items = 0;
  std::vector<ffst::Group> groups;
  ffst::ColItem* d_items = nullptr;
  ffst::Timer timer;
};

namespace ffst {

// thread-local error reporting
void set_error(const std::string& msg);
ffst_status fail(ffst_status st, const std::string& msg);
ffst_status cuda_fail(cudaError_t e, const char* what);

// timing helpers
void timer_begin(ffst_plan_s* p, int kind, cudaStream_t s, double bytes, cudaEvent_t* out_b);
void timer_end(ffst_plan_s* p, cudaStream_t s, cudaEvent_t b);

// kernel launchers (ffst_kernels_*.cu); all return cudaGetLastError() of the launch
cudaError_t launch_rows_r2c(const ffst_plan_s* p, int L, const void* src, int storage, const float* plane_scale,
                            int plane0, int nplanes, long long src_plane_stride, float2* dst, bool dst_grouped,
                            int full_c0, int full_W, int dst_ld, cudaStream_t s);
cudaError_t launch_rows_c2r(const ffst_plan_s* p, int L, const float2* src, bool src_grouped, int full_W, int src_ld,
                            int plane0, int nplanes, void* dst, int storage, const float* plane_scale,
                            long long dst_plane_stride, float scale, cudaStream_t s);
cudaError_t launch_cols_fft(const ffst_plan_s* p, int L, float2* buf, int width, int ld, bool inverse,
                            const float* divisor, cudaStream_t s);
cudaError_t launch_inv_cols(const ffst_plan_s* p, int L, const Group& g, bool first, cudaStream_t s);
cudaError_t launch_spectra(const ffst_plan_s* p, float* psi, cudaStream_t s);
cudaError_t launch_support(const ffst_plan_s* p, int* d_minmax, cudaStream_t s);
cudaError_t launch_fwd_cols(const ffst_plan_s* p, int L, const Group& g, float* partials, cudaStream_t s);
cudaError_t launch_plane_scales(const ffst_plan_s* p, const Group& g, const float* partials, float target,
                                float* plane_scale, cudaStream_t s);

// per-length launch geometry of the column kernels (columns per CTA)
int cols_per_cta(int L);

}  // namespace ffst
