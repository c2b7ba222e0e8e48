// Standalone row-pass kernels (bodies in ffst_kernels.cuh and
// ffst_rows_pair.cuh) and their launchers.
#include <cstdlib>

#include "ffst_rows_pair.cuh"

namespace ffst {

// Paired-row C2R (two rows per team, packed FP32 pairs) for power-of-two
// half lengths 256..2048 when FFST_PAIR_ROWS=1.  Off by default: at 2048x2048
// it measured 0.737 against 0.672 ms per forward's row passes (half the
// resident warps at 128 registers cost more than the halved FP instructions
// save).
static bool pair_rows_on(int L) {
  static const bool on = [] {
    const char* e = std::getenv("FFST_PAIR_ROWS");
    return e && e[0] == '1';
  }();
  return on && is_pow2c(L) && L >= 256 && L <= 2048;
}

template <int L>
__global__ void __launch_bounds__(kThreads, 2) k_rows_c2r_pair(C2RArgs a) {
  extern __shared__ __align__(128) float4 smem4[];
  rows_c2r_pair_body<L>(a, blockIdx.x, blockIdx.y, smem4, c2r_plane_factor(a, blockIdx.y));
}

template <int L>
static cudaError_t c2r_pair_L(const C2RArgs& a, int nplanes, cudaStream_t s) {
  if constexpr (is_pow2c(L) && L >= 256 && L <= 2048) {
    const dim3 grid((a.M + RowPairCfg<L>::ROWS - 1) / RowPairCfg<L>::ROWS, nplanes);
    cudaError_t e = set_smem(k_rows_c2r_pair<L>, RowPairCfg<L>::SMEM);
    if (e != cudaSuccess) return e;
    k_rows_c2r_pair<L><<<grid, kThreads, RowPairCfg<L>::SMEM, s>>>(a);
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidValue;
  }
}

template <int L>
__global__ void __launch_bounds__(kThreads, FFST_MIN_BLOCKS) k_rows_r2c(R2CArgs a) {
  extern __shared__ __align__(128) float2 smem[];
  rows_r2c_body<L>(a, blockIdx.x, blockIdx.y, smem);
}

template <int L>
__global__ void __launch_bounds__(kThreads, FFST_MIN_BLOCKS) k_rows_c2r(C2RArgs a) {
  extern __shared__ __align__(128) float2 smem[];
  rows_c2r_body<L>(a, blockIdx.x, blockIdx.y, smem, c2r_plane_factor(a, blockIdx.y));
}

template <int L>
static cudaError_t r2c_L(const R2CArgs& a, int nplanes, cudaStream_t s) {
  const dim3 grid((a.M + RowCfg<L>::TEAMS - 1) / RowCfg<L>::TEAMS, nplanes);
  cudaError_t e = set_smem(k_rows_r2c<L>, RowCfg<L>::SMEM);
  if (e != cudaSuccess) return e;
  k_rows_r2c<L><<<grid, kThreads, RowCfg<L>::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int L>
static cudaError_t c2r_L(const C2RArgs& a, int nplanes, cudaStream_t s) {
  if (pair_rows_on(L)) return c2r_pair_L<L>(a, nplanes, s);
  const dim3 grid((a.M + RowCfg<L>::TEAMS - 1) / RowCfg<L>::TEAMS, nplanes);
  cudaError_t e = set_smem(k_rows_c2r<L>, RowCfg<L>::SMEM);
  if (e != cudaSuccess) return e;
  k_rows_c2r<L><<<grid, kThreads, RowCfg<L>::SMEM, s>>>(a);
  return cudaGetLastError();
}

// Row line length L = N/2 for N = 8 .. 4096.
#define FFST_DISPATCH_ROW(L, CALL)         \
  switch (L) {                             \
    case 4: return CALL(4);                \
    case 8: return CALL(8);                \
    case 16: return CALL(16);              \
    case 32: return CALL(32);              \
    case 64: return CALL(64);              \
    case 128: return CALL(128);            \
    case 256: return CALL(256);            \
    case 512: return CALL(512);            \
    case 1024: return CALL(1024);          \
    case 2048: return CALL(2048);          \
    case 240: return CALL(240);            \
    case 320: return CALL(320);            \
    case 384: return CALL(384);            \
    case 480: return CALL(480);            \
    case 640: return CALL(640);            \
    case 768: return CALL(768);            \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_rows_r2c(int L, const R2CArgs& a, int nplanes, cudaStream_t s) {
#define CALL_(LL) r2c_L<LL>(a, nplanes, s)
  FFST_DISPATCH_ROW(L, CALL_)
#undef CALL_
}

cudaError_t launch_rows_c2r(int L, const C2RArgs& a, int nplanes, cudaStream_t s) {
#define CALL_(LL) c2r_L<LL>(a, nplanes, s)
  FFST_DISPATCH_ROW(L, CALL_)
#undef CALL_
}

}  // namespace ffst
