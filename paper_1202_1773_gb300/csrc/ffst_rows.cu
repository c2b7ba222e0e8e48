// Standalone row-pass kernels (bodies in ffst_kernels.cuh and
// ffst_rows_pair.cuh) and their launchers.
//
// Row kernel variants, a per-plan tuning choice (ffst_plan_set_kernels):
//  0  RowCfg<L>: 16 elements per thread for L >= 16 (radix 16 x 16 x 4 at
//     L = 1024; 64-register budget, 4 blocks per SM);
//  1  paired rows (C2R only): two rows per team in packed FP32 pairs,
//     power-of-two L in 256..2048 (ffst_rows_pair.cuh);
//  2  32 elements per thread, L = 1024 and 2048 (radix 32 x 32 at L = 1024:
//     one warp per line and one shared-memory exchange; budget of 3 blocks);
//  3  as 2 at L = 1024, with the exchange done by warp shuffles
//     (warp_transpose32; bitwise the results of 2; budget of 2 blocks for
//     the 32 extra registers of the transpose).
// Every variant computes the same transform; only the operation order of
// the FFT (and with it the rounding) differs.
#include "ffst_rows_pair.cuh"

namespace ffst {

bool row_variant_ok(int L, int variant, bool c2r) {
  if (variant == 0) return true;
  if (variant == 1) return c2r && is_pow2c(L) && L >= 256 && L <= 2048;
  if (variant == 2) return L == 1024 || L == 2048;
  if (variant == 3) return L == 1024;
  return false;
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

template <int EL, bool XSHFL>
constexpr int row_min_blocks() {
  return XSHFL ? 2 : (EL >= 32 ? 3 : FFST_MIN_BLOCKS);
}

template <int L, int EL, bool XSHFL = false>
__global__ void __launch_bounds__(kThreads, row_min_blocks<EL, XSHFL>()) k_rows_r2c(R2CArgs a) {
  extern __shared__ __align__(128) float2 smem[];
  rows_r2c_body<L, EL, XSHFL>(a, blockIdx.x, blockIdx.y, smem);
}

template <int L, int EL, bool XSHFL = false>
__global__ void __launch_bounds__(kThreads, row_min_blocks<EL, XSHFL>()) k_rows_c2r(C2RArgs a) {
  extern __shared__ __align__(128) float2 smem[];
  rows_c2r_body<L, EL, XSHFL>(a, blockIdx.x, blockIdx.y, smem, c2r_plane_factor(a, blockIdx.y));
}

template <int L, int EL, bool XSHFL = false>
static cudaError_t r2c_LE(const R2CArgs& a, int nplanes, cudaStream_t s) {
  using C = RowCfg<L, EL>;
  const dim3 grid((a.M + C::TEAMS - 1) / C::TEAMS, nplanes);
  cudaError_t e = set_smem(k_rows_r2c<L, EL, XSHFL>, C::SMEM);
  if (e != cudaSuccess) return e;
  k_rows_r2c<L, EL, XSHFL><<<grid, kThreads, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int L, int EL, bool XSHFL = false>
static cudaError_t c2r_LE(const C2RArgs& a, int nplanes, cudaStream_t s) {
  using C = RowCfg<L, EL>;
  const dim3 grid((a.M + C::TEAMS - 1) / C::TEAMS, nplanes);
  cudaError_t e = set_smem(k_rows_c2r<L, EL, XSHFL>, C::SMEM);
  if (e != cudaSuccess) return e;
  k_rows_c2r<L, EL, XSHFL><<<grid, kThreads, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int L>
static cudaError_t r2c_L(const R2CArgs& a, int nplanes, cudaStream_t s, int variant) {
  if (!row_variant_ok(L, variant, false)) return cudaErrorInvalidValue;
  if constexpr (L == 1024 || L == 2048) {
    if (variant == 2) return r2c_LE<L, 32>(a, nplanes, s);
  }
  if constexpr (L == 1024) {
    if (variant == 3) return r2c_LE<L, 32, true>(a, nplanes, s);
  }
  return r2c_LE<L, row_E(L)>(a, nplanes, s);
}

template <int L>
static cudaError_t c2r_L(const C2RArgs& a, int nplanes, cudaStream_t s, int variant) {
  if (!row_variant_ok(L, variant, true)) return cudaErrorInvalidValue;
  if (variant == 1) return c2r_pair_L<L>(a, nplanes, s);
  if constexpr (L == 1024 || L == 2048) {
    if (variant == 2) return c2r_LE<L, 32>(a, nplanes, s);
  }
  if constexpr (L == 1024) {
    if (variant == 3) return c2r_LE<L, 32, true>(a, nplanes, s);
  }
  return c2r_LE<L, row_E(L)>(a, nplanes, s);
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

cudaError_t launch_rows_r2c(int L, const R2CArgs& a, int nplanes, cudaStream_t s, int variant) {
#define CALL_(LL) r2c_L<LL>(a, nplanes, s, variant)
  FFST_DISPATCH_ROW(L, CALL_)
#undef CALL_
}

cudaError_t launch_rows_c2r(int L, const C2RArgs& a, int nplanes, cudaStream_t s, int variant) {
#define CALL_(LL) c2r_L<LL>(a, nplanes, s, variant)
  FFST_DISPATCH_ROW(L, CALL_)
#undef CALL_
}

}  // namespace ffst
