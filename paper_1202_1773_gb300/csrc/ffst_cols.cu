// Column passes over half-spectrum buffers [M][ld] (complex, row-major).
//
// A CTA owns a panel of P adjacent columns; thread (t, c) of the panel is
// threadIdx.x = t * P + c, so at every step the P columns of one row are
// read or written by consecutive lanes (one 32-byte sector per 4 columns).
// Each column is transformed by the T threads with the same c; their
// shared-memory exchanges use CTA barriers.
#include "ffst_fft.cuh"
#include "ffst_window.cuh"

namespace ffst {

template <int L>
struct ColCfg {
  static constexpr int T = LCfg<L>::T;
  static constexpr int P = (256 / T) < 4 ? 4 : ((256 / T) > 64 ? 64 : 256 / T);  // columns per CTA
  static constexpr int THREADS = P * T;
  static constexpr size_t SMEM = sizeof(float2) * P * LCfg<L>::BUF;
};

int cols_per_cta(int L) {
  switch (L) {
    case 8: return ColCfg<8>::P;
    case 16: return ColCfg<16>::P;
    case 32: return ColCfg<32>::P;
    case 64: return ColCfg<64>::P;
    case 128: return ColCfg<128>::P;
    case 256: return ColCfg<256>::P;
    case 512: return ColCfg<512>::P;
    case 1024: return ColCfg<1024>::P;
    case 2048: return ColCfg<2048>::P;
    case 4096: return ColCfg<4096>::P;
    default: return 0;
  }
}

// In-place column FFTs of columns [0, width) of buf (row stride ld).  When
// `divisor` is given (same layout), each element is divided by it first.
template <int L, bool INV>
__global__ void __launch_bounds__(ColCfg<L>::THREADS)
    k_cols_fft(float2* __restrict__ buf, int width, int ld, const float* __restrict__ divisor,
               const float2* __restrict__ tw) {
  constexpr int E = LCfg<L>::E, T = LCfg<L>::T, P = ColCfg<L>::P;
  extern __shared__ float2 smem[];
  const int t = threadIdx.x / P, cl = threadIdx.x % P;
  const int c = blockIdx.x * P + cl;
  const bool act = c < width;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const long long at = (long long)(t + T * m) * ld + c;
    float2 x = act ? buf[at] : make_float2(0.f, 0.f);
    if (divisor && act) {
      const float r = 1.0f / __ldg(&divisor[at]);
      x = cscale(x, r);
    }
    v[m] = x;
  }
  line_fft<L, INV, false>(v, smem + cl * LCfg<L>::BUF, t, tw);
  if (act) {
#pragma unroll
    for (int m = 0; m < E; ++m) buf[(long long)(t + T * m) * ld + c] = v[m];
  }
}

// Forward column pass of one plane panel (Sec. 3.1 eq. shearletTransform):
// G = psi_hat_i * F on the panel's columns (psi generated in registers; F is
// only read where psi != 0), then the column IFFT; the result goes to the
// plane's slot of the group intermediate, [M][W_i] starting at column c0_i.
// With `partials` the CTA also writes sum |G| over its panel, each column
// counted once for itself and once for its conjugate partner (columns 0
// and N/2 are their own partners); a plane's partials add up to
// sum_omega |G(omega)| >= M N max_m |c_i(m)|.
template <int L>
__global__ void __launch_bounds__(ColCfg<L>::THREADS)
    k_fwd_cols(const float2* __restrict__ F, int Hc, const PlaneDesc* __restrict__ planes,
               const ColItem* __restrict__ items, float2* __restrict__ H, WinParams w,
               const float2* __restrict__ tw, float* __restrict__ partials) {
  constexpr int E = LCfg<L>::E, T = LCfg<L>::T, P = ColCfg<L>::P;
  extern __shared__ float2 smem[];
  __shared__ float red[32];
  const int t = threadIdx.x / P, cl = threadIdx.x % P;
  const ColItem it = items[blockIdx.x];
  const PlaneDesc d = planes[it.plane];
  const int c = it.col + cl;
  const bool act = c < d.c0 + d.W;
  float2 v[E];
  float mag = 0.0f;
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int row = t + T * m;
    const float psi = act ? win_at(w, d, row, c) : 0.0f;
    v[m] = (psi != 0.0f) ? cscale(F[(long long)row * Hc + c], psi) : make_float2(0.f, 0.f);
    if (partials) mag += sqrtf(v[m].x * v[m].x + v[m].y * v[m].y);
  }
  if (partials) {
    const bool self_partner = (c == 0) || (2 * c == w.N);
    mag *= self_partner ? 1.0f : 2.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mag += __shfl_xor_sync(0xffffffffu, mag, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mag;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.0f;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
      partials[blockIdx.x] = s;
    }
  }
  line_fft<L, true, false>(v, smem + cl * LCfg<L>::BUF, t, tw);
  if (act) {
    float2* out = H + d.off + (c - d.c0);
#pragma unroll
    for (int m = 0; m < E; ++m) out[(long long)(t + T * m) * d.W] = v[m];
  }
}

// Inverse column pass (Sec. 3.3 eq. inverseShearletTransform): for every plane
// of the group whose support meets this CTA's panel, column FFT of the
// plane's row spectra, times psi_hat_i, accumulated in registers in plane
// order; then S += acc and D += sum psi^2 (plain stores for the first group).
// Each CTA owns its columns, so the sums are deterministic.
template <int L>
__global__ void __launch_bounds__(ColCfg<L>::THREADS)
    k_inv_cols(const float2* __restrict__ H, int Hc, const PlaneDesc* __restrict__ planes, int p0, int p1,
               float2* __restrict__ S, float* __restrict__ D, int first, WinParams w,
               const float2* __restrict__ tw) {
  constexpr int E = LCfg<L>::E, T = LCfg<L>::T, P = ColCfg<L>::P;
  extern __shared__ float2 smem[];
  const int t = threadIdx.x / P, cl = threadIdx.x % P;
  const int cbase = blockIdx.x * P;
  const int c = cbase + cl;
  float2 acc[E];
  float den[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    acc[m] = make_float2(0.f, 0.f);
    den[m] = 0.f;
  }
  for (int p = p0; p < p1; ++p) {
    const PlaneDesc d = planes[p];
    if (d.W == 0 || d.c0 >= cbase + P || d.c0 + d.W <= cbase) continue;  // uniform over the CTA
    const bool act = c >= d.c0 && c < d.c0 + d.W;
    const float2* in = H + d.off + (c - d.c0);
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = act ? in[(long long)(t + T * m) * d.W] : make_float2(0.f, 0.f);
    line_fft<L, false, false>(v, smem + cl * LCfg<L>::BUF, t, tw);
    if (act) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const float psi = win_at(w, d, t + T * m, c);
        acc[m].x = fmaf(psi, v[m].x, acc[m].x);
        acc[m].y = fmaf(psi, v[m].y, acc[m].y);
        den[m] = fmaf(psi, psi, den[m]);
      }
    }
  }
  if (c < Hc) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const long long at = (long long)(t + T * m) * Hc + c;
      if (first) {
        S[at] = acc[m];
        D[at] = den[m];
      } else {
        S[at] = cadd(S[at], acc[m]);
        D[at] += den[m];
      }
    }
  }
}

// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t prepare(K kernel, size_t smem) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int L>
static cudaError_t cols_fft_L(const ffst_plan_s* p, float2* buf, int width, int ld, bool inverse,
                              const float* divisor, cudaStream_t s) {
  const int grid = (width + ColCfg<L>::P - 1) / ColCfg<L>::P;
  const size_t smem = ColCfg<L>::SMEM;
  cudaError_t e;
  if (inverse) {
    if ((e = prepare(k_cols_fft<L, true>, smem)) != cudaSuccess) return e;
    k_cols_fft<L, true><<<grid, ColCfg<L>::THREADS, smem, s>>>(buf, width, ld, divisor, p->d_tw_cols);
  } else {
    if ((e = prepare(k_cols_fft<L, false>, smem)) != cudaSuccess) return e;
    k_cols_fft<L, false><<<grid, ColCfg<L>::THREADS, smem, s>>>(buf, width, ld, divisor, p->d_tw_cols);
  }
  return cudaGetLastError();
}

template <int L>
static cudaError_t fwd_cols_L(const ffst_plan_s* p, const Group& g, float* partials, cudaStream_t s) {
  if (g.nitems == 0) return cudaSuccess;
  const size_t smem = ColCfg<L>::SMEM;
  cudaError_t e;
  if ((e = prepare(k_fwd_cols<L>, smem)) != cudaSuccess) return e;
  k_fwd_cols<L><<<g.nitems, ColCfg<L>::THREADS, smem, s>>>(p->d_F, p->Hc, p->d_planes, p->d_items + g.item0,
                                                             p->d_H, p->win, p->d_tw_cols,
                                                             partials ? partials + g.item0 : nullptr);
  return cudaGetLastError();
}

// s_i = 2^floor(log2(target / B_i)), B_i = (1/MN) sum of the plane's partials
// (summed in item order: deterministic); s_i = 1 for an all-zero plane.
__global__ void k_plane_scales(const PlaneDesc* __restrict__ planes, int p0, int p1,
                               const float* __restrict__ partials, float inv_mn, float target,
                               float* __restrict__ plane_scale) {
  const int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= p1) return;
  const PlaneDesc d = planes[p];
  float sum = 0.0f;
  for (int q = 0; q < d.nitems; ++q) sum += partials[d.item0 + q];
  const float B = sum * inv_mn;
  float s = 1.0f;
  if (B > 0.0f && isfinite(B)) {
    int e = (int)floorf(log2f(target / B));
    e = e < -100 ? -100 : (e > 100 ? 100 : e);
    s = ldexpf(1.0f, e);
  }
  plane_scale[p] = s;
}

cudaError_t launch_plane_scales(const ffst_plan_s* p, const Group& g, const float* partials, float target,
                                float* plane_scale, cudaStream_t s) {
  const int n = g.p1 - g.p0;
  if (n <= 0) return cudaSuccess;
  k_plane_scales<<<(n + 127) / 128, 128, 0, s>>>(p->d_planes, g.p0, g.p1, partials, 1.0f / ((float)p->M * p->N),
                                                 target, plane_scale);
  return cudaGetLastError();
}

template <int L>
static cudaError_t inv_cols_L(const ffst_plan_s* p, const Group& g, bool first, cudaStream_t s) {
  const int grid = (p->Hc + ColCfg<L>::P - 1) / ColCfg<L>::P;
  const size_t smem = ColCfg<L>::SMEM;
  cudaError_t e;
  if ((e = prepare(k_inv_cols<L>, smem)) != cudaSuccess) return e;
  k_inv_cols<L><<<grid, ColCfg<L>::THREADS, smem, s>>>(p->d_H, p->Hc, p->d_planes, g.p0, g.p1, p->d_S, p->d_D,
                                                        first ? 1 : 0, p->win, p->d_tw_cols);
  return cudaGetLastError();
}

#define FFST_DISPATCH_L(L, CALL)   \
  switch (L) {                     \
    case 8: return CALL(8);        \
    case 16: return CALL(16);      \
    case 32: return CALL(32);      \
    case 64: return CALL(64);      \
    case 128: return CALL(128);    \
    case 256: return CALL(256);    \
    case 512: return CALL(512);    \
    case 1024: return CALL(1024);  \
    case 2048: return CALL(2048);  \
    case 4096: return CALL(4096);  \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_cols_fft(const ffst_plan_s* p, int L, float2* buf, int width, int ld, bool inverse,
                            const float* divisor, cudaStream_t s) {
#define CALL_(LL) cols_fft_L<LL>(p, buf, width, ld, inverse, divisor, s)
  FFST_DISPATCH_L(L, CALL_)
#undef CALL_
}

cudaError_t launch_fwd_cols(const ffst_plan_s* p, int L, const Group& g, float* partials, cudaStream_t s) {
#define CALL_(LL) fwd_cols_L<LL>(p, g, partials, s)
  FFST_DISPATCH_L(L, CALL_)
#undef CALL_
}

cudaError_t launch_inv_cols(const ffst_plan_s* p, int L, const Group& g, bool first, cudaStream_t s) {
#define CALL_(LL) inv_cols_L<LL>(p, g, first, s)
  FFST_DISPATCH_L(L, CALL_)
#undef CALL_
}

}  // namespace ffst
