// Standalone column-pass kernels (bodies in ffst_kernels.cuh), their
// launchers, and the per-plane scale kernel of low-precision storage.
#include "ffst_kernels.cuh"

namespace ffst {

template <int L, bool INV>
__global__ void __launch_bounds__(kThreads, min_blocks_for(L))
    k_cols_fft(float2* __restrict__ buf, int width, int ld, const float* __restrict__ scale_tab,
               const float2* __restrict__ tw, int nsum, long long sstride, long long buf_bytes, int* err) {
  extern __shared__ __align__(128) float2 smem[];
  cols_fft_body<L, INV>(buf, width, ld, scale_tab, tw, nsum, sstride, blockIdx.x, smem, buf_bytes, err);
}

template <int L>
__global__ void __launch_bounds__(kThreads, min_blocks_for(L)) k_fwd_cols(FwdColsArgs a) {
  extern __shared__ __align__(128) float2 smem[];
  fwd_cols_body<L>(a, blockIdx.x, smem);
}

template <int L>
__global__ void __launch_bounds__(kThreads, min_blocks_for(L)) k_inv_cols(InvColsArgs a) {
  extern __shared__ __align__(128) float2 smem[];
  int q0, q1;
  float2* S;
  const int panel = inv_chunk(a, blockIdx.x, &q0, &q1, &S);
  inv_cols_body<L>(a, panel, q0, q1, S, smem);
}

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
    case 240: return ColCfg<240>::P;
    case 320: return ColCfg<320>::P;
    case 384: return ColCfg<384>::P;
    case 480: return ColCfg<480>::P;
    case 640: return ColCfg<640>::P;
    case 768: return ColCfg<768>::P;
    default: return 0;
  }
}

template <int L>
static cudaError_t cols_fft_L(float2* buf, int width, int ld, bool inverse, const float* scale_tab,
                              const float2* tw, int nsum, long long sstride, long long buf_bytes, int* err,
                              cudaStream_t s) {
  const int grid = (width + ColCfg<L>::P - 1) / ColCfg<L>::P;
  cudaError_t e;
  if (inverse) {
    if ((e = set_smem(k_cols_fft<L, true>, ColCfg<L>::SMEM)) != cudaSuccess) return e;
    k_cols_fft<L, true><<<grid, kThreads, ColCfg<L>::SMEM, s>>>(buf, width, ld, scale_tab, tw, nsum, sstride,
                                                                  buf_bytes, err);
  } else {
    if ((e = set_smem(k_cols_fft<L, false>, ColCfg<L>::SMEM)) != cudaSuccess) return e;
    k_cols_fft<L, false><<<grid, kThreads, ColCfg<L>::SMEM, s>>>(buf, width, ld, scale_tab, tw, nsum, sstride,
                                                                   buf_bytes, err);
  }
  return cudaGetLastError();
}

template <int L>
static cudaError_t fwd_cols_L(const FwdColsArgs& a, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  cudaError_t e = set_smem(k_fwd_cols<L>, ColCfg<L>::SMEM);
  if (e != cudaSuccess) return e;
  FwdColsArgs b = a;
  b.nitems = nitems;
  k_fwd_cols<L><<<(nitems + kFwdItems - 1) / kFwdItems, kThreads, ColCfg<L>::SMEM, s>>>(b);
  return cudaGetLastError();
}

template <int L>
static cudaError_t inv_cols_L(const InvColsArgs& a, cudaStream_t s) {
  const int nb = a.npanels * a.nchunks;
  if (nb <= 0) return cudaSuccess;
  cudaError_t e = set_smem(k_inv_cols<L>, ColCfg<L>::SMEM);
  if (e != cudaSuccess) return e;
  k_inv_cols<L><<<nb, kThreads, ColCfg<L>::SMEM, s>>>(a);
  return cudaGetLastError();
}

#define FFST_DISPATCH_COL(L, CALL)         \
  switch (L) {                             \
    case 8: return CALL(8);                \
    case 16: return CALL(16);              \
    case 32: return CALL(32);              \
    case 64: return CALL(64);              \
    case 128: return CALL(128);            \
    case 256: return CALL(256);            \
    case 512: return CALL(512);            \
    case 1024: return CALL(1024);          \
    case 2048: return CALL(2048);          \
    case 4096: return CALL(4096);          \
    case 240: return CALL(240);            \
    case 320: return CALL(320);            \
    case 384: return CALL(384);            \
    case 480: return CALL(480);            \
    case 640: return CALL(640);            \
    case 768: return CALL(768);            \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_cols_fft(int L, float2* buf, int width, int ld, bool inverse, const float* scale_tab,
                            const float2* tw, cudaStream_t s, int nsum, long long sstride, long long buf_bytes,
                            int* err) {
#define CALL_(LL) cols_fft_L<LL>(buf, width, ld, inverse, scale_tab, tw, nsum, sstride, buf_bytes, err, s)
  FFST_DISPATCH_COL(L, CALL_)
#undef CALL_
}

cudaError_t launch_fwd_cols(int L, const FwdColsArgs& a, int nitems, cudaStream_t s) {
#define CALL_(LL) fwd_cols_L<LL>(a, nitems, s)
  FFST_DISPATCH_COL(L, CALL_)
#undef CALL_
}

cudaError_t launch_inv_cols(int L, const InvColsArgs& a, cudaStream_t s) {
#define CALL_(LL) inv_cols_L<LL>(a, s)
  FFST_DISPATCH_COL(L, CALL_)
#undef CALL_
}

// Per-plane scales of low-precision storage (plane_scale_of).
__global__ void k_plane_scales(const PlaneDesc* __restrict__ planes, int p0, int p1,
                               const float* __restrict__ partials, float target, float* __restrict__ plane_scale) {
  const int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= p1) return;
  plane_scale[p] = plane_scale_of(partials, planes[p].item0, planes[p].nitems, target);
}

// d(i) = 1/(MN) sum |c_i| from the row pass's per-block partial sums
// (Sec. 3.5.2 eq. shearlet_meanvalue), summed in block order.
__global__ void k_mean_abs(const float* __restrict__ partials, int rbx, int eta, float inv_mn, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= eta) return;
  float sum = 0.0f;
  for (int b = 0; b < rbx; ++b) sum += partials[(long long)i * rbx + b];
  out[i] = sum * inv_mn;
}

cudaError_t launch_mean_abs(const ffst_plan_s* p, float* mean_abs, cudaStream_t s) {
  k_mean_abs<<<(p->eta + 127) / 128, 128, 0, s>>>(p->d_abs_partials, p->row_blocks, p->eta,
                                                 1.0f / ((float)p->M * (float)p->N), mean_abs);
  return cudaGetLastError();
}

cudaError_t launch_plane_scales(const ffst_plan_s* p, const Group& g, const float* partials, float target,
                                float* plane_scale, cudaStream_t s) {
  const int n = g.p1 - g.p0;
  if (n <= 0) return cudaSuccess;
  // the forward column pass folds 1/(M N) into G, so its partials bound max |c_i| directly
  k_plane_scales<<<(n + 127) / 128, 128, 0, s>>>(p->d_planes, g.p0, g.p1, partials, target, plane_scale);
  return cudaGetLastError();
}

}  // namespace ffst
