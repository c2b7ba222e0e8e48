// Lines of any length n (odd, prime, or even without a native FFT kernel):
// Bluestein's chirp-z form of the DFT (L. Bluestein, "A linear filtering
// approach to the computation of the discrete Fourier transform", 1970),
// run on the power-of-two register FFTs of ffst_fft.cuh.
//
// With the chirp w_j = exp(-i pi j^2 / n), jk = (j^2 + k^2 - (k - j)^2) / 2
// turns the DFT into a convolution:
//   X[k] = w_k sum_j (x_j w_j) conj(w_{k-j}),   0 <= j, k < n,
// evaluated as a cyclic convolution of length L2 (a power of two >= 2n - 1,
// so the filter's wrapped taps do not overlap) through two FFTs of length L2
// and a pointwise product with the filter's precomputed spectrum.  The
// inverse DFT (e^{+2 pi i jk/n}) is conj(DFT(conj x)).
//
// The generic passes below carry the same argument structs and the same
// contracts as the native ones of ffst_kernels.cuh (the Sec. 3.1 forward and
// Sec. 3.3 inverse of the shearlet transform on half spectra), with one
// line per team of T = L2/E threads:
//   rows: two real rows per complex line (z = x_a + i x_b), consecutive
//         threads on consecutive elements;
//   columns: P columns per block, interleaved across the warps.
#pragma once

#include "ffst_kernels.cuh"

namespace ffst {

// BlueLine (the tables of one dimension) is declared in ffst_internal.cuh.
constexpr int kBlueMinL2 = 16;
constexpr int kBlueMaxL2 = 4096;  // lines up to n = 2048

// Elements per thread of a generic line: as the native column lines, but at
// most 16, so that the two FFTs of a Bluestein line keep the register
// footprint of the native kernels (a 4096-point line is one team of 256
// threads).  The host builds the pass tables with the same E.
__host__ __device__ constexpr int blue_E(int L2) { return col_E(L2) < 16 ? col_E(L2) : 16; }

template <int L2>
struct BlueCfg {
  static constexpr int E = blue_E(L2);
  static constexpr int T = L2 / E;
  static constexpr int P = kThreads / T;  // lines per block
  static constexpr int BUF = team_stride(L2, E, P >= 16 ? 1 : 16 / P);
  static constexpr size_t SMEM = sizeof(float2) * P * BUF;
  static_assert(P * T == kThreads, "generic line teams must fill the block");
};

// Columns (lines) per block of the generic column (row) passes.
int blue_lines_per_block(int L2);

// Host tables of a line of length n (FP64, rounded to FP32).
void blue_tables(int n, int* L2, std::vector<float2>* chirp, std::vector<float2>* bhat);
// Lengths with no prime factor above 7: the radices of the mixed-radix
// passes (8s, then a 4 or 2, then 3s, 5s, 7s) packed 4 bits per pass, and
// the pass twiddle table (n - 1 entries).  False for other lengths.
bool smooth_line(int n, int* nrad, unsigned long long* radices, std::vector<float2>* tw);
// Line geometry of the generic kernels: the power of two >= 2n - 1 for
// Bluestein lines (their convolution length), >= n for smooth lines; at
// least kBlueMinL2.
int blue_L2(int n);
int smooth_L2(int n);

cudaError_t launch_blue_rows_r2c(const BlueLine& b, const R2CArgs& a, int nplanes, cudaStream_t s);
cudaError_t launch_blue_rows_c2r(const BlueLine& b, const C2RArgs& a, int nplanes, cudaStream_t s);
cudaError_t launch_blue_cols_fft(const BlueLine& b, float2* buf, int width, int ld, bool inverse,
                                 const float* scale_tab, cudaStream_t s, int nsum = 1, long long sstride = 0);
cudaError_t launch_blue_fwd_cols(const BlueLine& b, const FwdColsArgs& a, int nitems, cudaStream_t s);
cudaError_t launch_blue_inv_cols(const BlueLine& b, const InvColsArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// device side (included by ffst_blue_rows.cu and ffst_blue_cols.cu)
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

// One element of a stack (any storage code), streaming like load_pair.
__device__ __forceinline__ float load_one(const void* p, long long i, int st) {
  if (st == FFST_STORE_F32) return __ldcs(static_cast<const float*>(p) + i);
  if (st == FFST_STORE_F16) return __half2float(__ldcs(static_cast<const __half*>(p) + i));
  return __bfloat162float(__ldcs(static_cast<const __nv_bfloat16*>(p) + i));
}

__device__ __forceinline__ void store_one(void* p, long long i, float v, int st) {
  if (st == FFST_STORE_F32) __stcs(static_cast<float*>(p) + i, v);
  else if (st == FFST_STORE_F16) __stcs(static_cast<__half*>(p) + i, __float2half_rn(v));
  else __stcs(static_cast<__nv_bfloat16*>(p) + i, __float2bfloat16_rn(v));
}

// r in the cyclic row interval (start rg.x, length rg.y) of a column of height n.
__device__ __forceinline__ bool in_cyclic(int r, int2 rg, int n) {
  int q = r - rg.x;
  if (q < 0) q += n;
  return q < rg.y;
}

// One Stockham pass of radix R over a line of length n in shared memory
// (the autosort of ffst_fft.cuh with a runtime length): butterfly j < n/R
// takes a[j + r n/R], applies W_{Ns R}^{(j mod Ns) r} and the R-point DFT,
// and writes c[(j - j mod Ns) R + j mod Ns + r Ns].  Team threads t, t + T,
// ... share the butterflies.
// Buffer slot of element i of a smooth line: one pad slot per 32 elements,
// which spreads the radix-strided writes of the first passes over the banks
// (a half of the team buffer holds n + n/32 <= L2 + L2/E slots).
__device__ __forceinline__ int smooth_slot(int i) { return i + (i >> 5); }

template <int R, bool INV>
__device__ __forceinline__ void smooth_pass(const float2* a, float2* c, int n, int Ns, const float2* __restrict__ tw,
                                            int t, int T) {
  const int nb = n / R;
  for (int j = t; j < nb; j += T) {
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = a[smooth_slot(j + r * nb)];
    const int g = j / Ns, kk = j - g * Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = __ldg(&tw[(Ns - 1) + (r - 1) * Ns + kk]);
        if (INV) w.y = -w.y;
        x[r] = cmul(x[r], w);
      }
    }
    dft<R, INV>(x);
    const int base = g * Ns * R + kk;
#pragma unroll
    for (int r = 0; r < R; ++r) c[smooth_slot(base + r * Ns)] = x[r];
  }
}

// DFT (INV: unnormalised inverse) of length n, given as nrad > 0 radices,
// of the line in a[0, n), ping-ponging with c[0, n); returns the buffer that
// holds the result.  Every thread of the block calls it: a barrier follows
// each pass.  Not inlined: one copy serves every line geometry.
template <bool INV>
__device__ __noinline__ float2* smooth_dft(float2* a, float2* c, int n, int nrad, unsigned long long radices,
                                           const float2* __restrict__ tw, int t, int T) {
  int Ns = 1;
  for (int s = 0; s < nrad; ++s) {
    const int R = (int)((radices >> (4 * s)) & 15u);
    switch (R) {
      case 2: smooth_pass<2, INV>(a, c, n, Ns, tw, t, T); break;
      case 3: smooth_pass<3, INV>(a, c, n, Ns, tw, t, T); break;
      case 4: smooth_pass<4, INV>(a, c, n, Ns, tw, t, T); break;
      case 5: smooth_pass<5, INV>(a, c, n, Ns, tw, t, T); break;
      case 7: smooth_pass<7, INV>(a, c, n, Ns, tw, t, T); break;
      default: smooth_pass<8, INV>(a, c, n, Ns, tw, t, T); break;
    }
    __syncthreads();
    float2* x = a;
    a = c;
    c = x;
    Ns *= R;
  }
  return a;
}

// Team buffer stride (float2 slots) and dynamic shared memory of a generic
// line kernel: smooth lines ping-pong between two halves of BUF >= L2 >= n
// slots each, Bluestein lines use one.
template <int L2>
__host__ __device__ __forceinline__ int blue_stride(const BlueLine& b) {
  return b.nrad > 0 ? 2 * BlueCfg<L2>::BUF : BlueCfg<L2>::BUF;
}
template <int L2>
__host__ __device__ __forceinline__ size_t blue_smem(const BlueLine& b) {
  return sizeof(float2) * BlueCfg<L2>::P * (size_t)blue_stride<L2>(b);
}

// DFT (INV: unnormalised inverse DFT) of length b.n of the line whose
// element j = t + T m (j < b.n; the rest is ignored) thread t holds in v[m];
// on return v[m] holds output k = t + T m (zero for k >= b.n).  Every thread
// of the block calls it (block barriers); it ends with a barrier after its
// last read of `buf`.  Lengths with no prime factor above 7 run the
// mixed-radix passes (lines laid out with L2 >= n, a team buffer of two
// halves: blue_stride); the others Bluestein's convolution (L2 >= 2n - 1).
template <int L2, bool INV>
__device__ __forceinline__ void blue_dft(float2 (&v)[BlueCfg<L2>::E], float2* buf, int t, const BlueLine& b) {
  constexpr int E = BlueCfg<L2>::E, T = BlueCfg<L2>::T;
  static_assert(BlueCfg<L2>::BUF >= L2 + L2 / 32, "each half of a smooth line's team buffer holds n + n/32 slots");
  if (b.nrad > 0) {
    __syncthreads();  // earlier reads of buf by other threads of the team are done
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int j = t + T * m;
      if (j < b.n) buf[smooth_slot(j)] = v[m];
    }
    __syncthreads();
    const float2* res = smooth_dft<INV>(buf, buf + BlueCfg<L2>::BUF, b.n, b.nrad, b.radices, b.mtw, t, T);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + T * m;
      v[m] = k < b.n ? res[smooth_slot(k)] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int j = t + T * m;
    float2 x = v[m];
    if (INV) x.y = -x.y;
    v[m] = j < b.n ? cmul(x, __ldg(&b.chirp[j])) : make_float2(0.f, 0.f);
  }
  line_fft<L2, E, false, kSyncBlock>(v, buf, t, b.tw);
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = cmul(v[m], __ldg(&b.bhat[t + T * m]));
  line_fft<L2, E, true, kSyncBlock>(v, buf, t, b.tw);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = t + T * m;
    float2 x = k < b.n ? cmul(v[m], __ldg(&b.chirp[k])) : make_float2(0.f, 0.f);
    if (INV) x.y = -x.y;
    v[m] = x;
  }
}

#endif  // __CUDACC__

}  // namespace ffst
