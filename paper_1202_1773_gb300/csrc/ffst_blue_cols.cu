// Generic-length column passes (Bluestein lines, ffst_blue.cuh): the same
// contracts as cols_fft_body, fwd_cols_body and inv_cols_body, with P
// columns per block interleaved across the warps (thread = t P + column).
#include "ffst_blue.cuh"

namespace ffst {

// In-place column DFTs (INV: unnormalised inverse) of columns [0, width) of
// buf, after summing nsum partial arrays and scaling by scale_tab (as
// cols_fft_body).
template <int L2, bool INV>
__global__ void __launch_bounds__(kThreads, 3)
    k_blue_cols(float2* __restrict__ buf, int width, int ld, const float* __restrict__ scale_tab, int nsum,
                long long sstride, BlueLine b) {
  constexpr int E = BlueCfg<L2>::E, T = BlueCfg<L2>::T, P = BlueCfg<L2>::P;
  extern __shared__ __align__(128) float2 smem[];
  const int t = threadIdx.x / P, cl = threadIdx.x % P;
  const int c = blockIdx.x * P + cl;
  const bool act = c < width;
  const int n = b.n;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int r = t + T * m;
    float2 x = make_float2(0.f, 0.f);
    if (act && r < n) {
      const long long i = (long long)r * ld + c;
      x = buf[i];
      for (int k = 1; k < nsum; ++k) {
        const float2 y = __ldcs(&buf[i + k * sstride]);
        x = make_float2(x.x + y.x, x.y + y.y);
      }
      if (scale_tab) x = cscale(x, __ldg(&scale_tab[i]));
    }
    v[m] = x;
  }
  blue_dft<L2, INV>(v, smem + cl * blue_stride<L2>(b), t, b);
  if (act) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int r = t + T * m;
      if (r < n) buf[(long long)r * ld + c] = v[m];
    }
  }
}

// Forward column pass of one item (P columns of one plane) per block:
// G = gain psi_hat_i F on the columns' support rows, the column IDFT into the
// plane's slot, and the item's sum |G| (each column counted for itself and
// its conjugate partner) as fwd_cols_body.
template <int L2>
__global__ void __launch_bounds__(kThreads, 3) k_blue_fwd_cols(FwdColsArgs a, BlueLine b) {
  constexpr int E = BlueCfg<L2>::E, T = BlueCfg<L2>::T, P = BlueCfg<L2>::P;
  extern __shared__ __align__(128) float2 smem[];
  __shared__ float red[kThreads / 32];
  const int t = threadIdx.x / P, cl = threadIdx.x % P;
  float2* buf = smem + cl * blue_stride<L2>(b);
  const int item = blockIdx.x;
  const int n = b.n;
  const ColItem it = a.items[item];
  const PlaneDesc d = a.planes[it.plane];
  const int c = it.col + cl;
  const bool act = c >= d.c0 && c < d.c0 + d.W;
  const int2 rg = act ? a.rng[d.rng_off + (c - d.c0)] : make_int2(0, 0);
  // G on the support rows (window evaluated in a rolled loop), through the
  // column's buffer into the register layout
  float mag = 0.0f;
  for (int q = t; q < rg.y; q += T) {
    int r = rg.x + q;
    if (r >= n) r -= n;
    float psi = win_at(a.w, d, r, c);
    if (a.odd) psi *= (float)half_sign(a.w, d.kappa, r, c);
    float2 g = make_float2(0.f, 0.f);
    if (psi != 0.0f) g = cscale(a.F[(long long)r * a.Hc + c], psi * a.gain);
    if (a.odd) g = make_float2(g.y, -g.x);  // -i g (the sign is in psi)
    buf[r] = g;
    mag += sqrtf(g.x * g.x + g.y * g.y);
  }
  __syncthreads();
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int r = t + T * m;
    v[m] = (r < n && in_cyclic(r, rg, n)) ? buf[r] : make_float2(0.f, 0.f);
  }
  __syncthreads();  // buffer reads done before the DFT reuses it
  if (a.partials) {  // uniform over the launch
    const bool self_partner = (c == 0) || (2 * c == a.w.N);
    mag *= self_partner ? 1.0f : 2.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mag += __shfl_xor_sync(0xffffffffu, mag, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mag;
    __syncthreads();
    if (threadIdx.x == 0) {
      float sum = 0.0f;
      for (int q = 0; q < kThreads / 32; ++q) sum += red[q];
      a.partials[item] = sum;
    }
  }
  blue_dft<L2, true>(v, buf, t, b);
  if (act) {
    float2* out = a.H + d.off + (c - d.c0al);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int r = t + T * m;
      if (r < n) __stcg(&out[(long long)r * d.ldw], v[m]);
    }
  }
}

// Inverse column pass of panel x plane chunk (inv_chunk): for every plane of
// the chunk whose support meets the panel, the column DFT of the plane's row
// spectra and S += psi_hat_i * (that) on the column's support rows, in plane
// order (each S element belongs to one thread: deterministic).
template <int L2>
__global__ void __launch_bounds__(kThreads, 3) k_blue_inv_cols(InvColsArgs a, BlueLine b) {
  constexpr int E = BlueCfg<L2>::E, T = BlueCfg<L2>::T, P = BlueCfg<L2>::P;
  extern __shared__ __align__(128) float2 smem[];
  const int t = threadIdx.x / P, cl = threadIdx.x % P;
  float2* buf = smem + cl * blue_stride<L2>(b);
  const int n = b.n;
  int q0, q1;
  float2* S;
  const int panel = inv_chunk(a, blockIdx.x, &q0, &q1, &S);
  const int cbase = panel * P, c = cbase + cl;
  for (int p = q0; p < q1; ++p) {
    const PlaneDesc d = a.planes[p];
    if (d.W == 0 || d.c0 >= cbase + P || d.c0 + d.W <= cbase) continue;  // uniform over the block
    const bool act = c >= d.c0 && c < d.c0 + d.W;
    const int2 rg = act ? a.rng[d.rng_off + (c - d.c0)] : make_int2(0, 0);
    const float2* in = a.H + d.off + (c - d.c0al);
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int r = t + T * m;
      v[m] = (act && r < n) ? __ldcg(&in[(long long)r * d.ldw]) : make_float2(0.f, 0.f);
    }
    blue_dft<L2, false>(v, buf, t, b);  // ends with a barrier after its last buffer read
    // the support rows through the column's buffer to a rolled loop (window
    // evaluated once per row)
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int r = t + T * m;
      if (r < n && in_cyclic(r, rg, n)) buf[r] = v[m];
    }
    __syncthreads();
    for (int q = t; q < rg.y; q += T) {
      int r = rg.x + q;
      if (r >= n) r -= n;
      const float psi = win_at(a.w, d, r, c);
      const float2 x = buf[r];
      float2* sp = S + (long long)r * a.Hc + c;
      const float2 old = __ldcg(sp);
      *sp = make_float2(fmaf(psi, x.x, old.x), fmaf(psi, x.y, old.y));
    }
    __syncthreads();  // buffer reads done before the next plane's DFT
  }
}

template <int L2>
static cudaError_t cols_L2(const BlueLine& b, float2* buf, int width, int ld, bool inverse, const float* scale_tab,
                           int nsum, long long sstride, cudaStream_t s) {
  constexpr int P = BlueCfg<L2>::P;
  const int grid = (width + P - 1) / P;
  if (grid <= 0) return cudaSuccess;
  cudaError_t e;
  if (inverse) {
    if ((e = set_smem(k_blue_cols<L2, true>, blue_smem<L2>(b))) != cudaSuccess) return e;
    k_blue_cols<L2, true><<<grid, kThreads, blue_smem<L2>(b), s>>>(buf, width, ld, scale_tab, nsum, sstride, b);
  } else {
    if ((e = set_smem(k_blue_cols<L2, false>, blue_smem<L2>(b))) != cudaSuccess) return e;
    k_blue_cols<L2, false><<<grid, kThreads, blue_smem<L2>(b), s>>>(buf, width, ld, scale_tab, nsum, sstride, b);
  }
  return cudaGetLastError();
}

template <int L2>
static cudaError_t fwd_cols_L2(const BlueLine& b, const FwdColsArgs& a, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  cudaError_t e = set_smem(k_blue_fwd_cols<L2>, blue_smem<L2>(b));
  if (e != cudaSuccess) return e;
  k_blue_fwd_cols<L2><<<nitems, kThreads, blue_smem<L2>(b), s>>>(a, b);
  return cudaGetLastError();
}

template <int L2>
static cudaError_t inv_cols_L2(const BlueLine& b, const InvColsArgs& a, cudaStream_t s) {
  const int nb = a.npanels * a.nchunks;
  if (nb <= 0) return cudaSuccess;
  cudaError_t e = set_smem(k_blue_inv_cols<L2>, blue_smem<L2>(b));
  if (e != cudaSuccess) return e;
  k_blue_inv_cols<L2><<<nb, kThreads, blue_smem<L2>(b), s>>>(a, b);
  return cudaGetLastError();
}

#define FFST_DISPATCH_BLUE(L2, CALL)       \
  switch (L2) {                            \
    case 16: return CALL(16);              \
    case 32: return CALL(32);              \
    case 64: return CALL(64);              \
    case 128: return CALL(128);            \
    case 256: return CALL(256);            \
    case 512: return CALL(512);            \
    case 1024: return CALL(1024);          \
    case 2048: return CALL(2048);          \
    case 4096: return CALL(4096);          \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_blue_cols_fft(const BlueLine& b, float2* buf, int width, int ld, bool inverse,
                                 const float* scale_tab, cudaStream_t s, int nsum, long long sstride) {
#define CALL_(LL) cols_L2<LL>(b, buf, width, ld, inverse, scale_tab, nsum, sstride, s)
  FFST_DISPATCH_BLUE(b.L2, CALL_)
#undef CALL_
}

cudaError_t launch_blue_fwd_cols(const BlueLine& b, const FwdColsArgs& a, int nitems, cudaStream_t s) {
#define CALL_(LL) fwd_cols_L2<LL>(b, a, nitems, s)
  FFST_DISPATCH_BLUE(b.L2, CALL_)
#undef CALL_
}

cudaError_t launch_blue_inv_cols(const BlueLine& b, const InvColsArgs& a, cudaStream_t s) {
#define CALL_(LL) inv_cols_L2<LL>(b, a, s)
  FFST_DISPATCH_BLUE(b.L2, CALL_)
#undef CALL_
}

}  // namespace ffst
