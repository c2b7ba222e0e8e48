// Row passes: real rows <-> half spectra, two real rows per complex line FFT.
//
// R2C: rows a, b of a real plane become z = a + i b; Z = FFT(z) gives
//   A(k) = (Z(k) + conj Z(L-k)) / 2,  B(k) = (Z(k) - conj Z(L-k)) / (2i)
// for the kept columns k in [c0, c0 + W) of the half spectrum [0, L/2].
// C2R: the Hermitian extensions of two half-spectrum rows A, B are packed as
// Z = A + i B; z = IFFT(Z) holds row a in Re z and row b in Im z.  Columns
// outside [c0, c0 + W) are zero (the plane's spectral support), and the
// imaginary parts at k = 0 and k = L/2 are dropped (Hermitian part).
#include "ffst_fft.cuh"

namespace ffst {

template <int ST>
__device__ __forceinline__ float load_st(const void* p, long long i) {
  if constexpr (ST == FFST_STORE_F32) return __ldg(static_cast<const float*>(p) + i);
  else if constexpr (ST == FFST_STORE_F16) return __half2float(static_cast<const __half*>(p)[i]);
  else return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
}

template <int ST>
__device__ __forceinline__ void store_st(void* p, long long i, float x) {
  if constexpr (ST == FFST_STORE_F32) static_cast<float*>(p)[i] = x;
  else if constexpr (ST == FFST_STORE_F16) static_cast<__half*>(p)[i] = __float2half_rn(x);
  else static_cast<__nv_bfloat16*>(p)[i] = __float2bfloat16_rn(x);
}

template <int L>
struct RowCfg {
  static constexpr int T = LCfg<L>::T;
  static constexpr int TEAMS = (T >= 256) ? 1 : 256 / T;  // row pairs per CTA
  static constexpr int THREADS = TEAMS * T;
  static constexpr bool WARP = T <= 32;
  static constexpr size_t SMEM = sizeof(float2) * TEAMS * LCfg<L>::BUF;
};

struct R2CArgs {
  const void* src;          // plane 0 of the batch (row-major rows x L)
  long long src_plane_stride;
  const float* plane_scale;  // per plane s_i (low-precision storage) or null
  int plane0;                // plane index of blockIdx.y == 0 (for descriptors/scales)
  int M;                     // rows
  float2* dst;
  const PlaneDesc* planes;   // non-null: grouped output (per-plane c0, W, off)
  int c0, W, ld;             // used when planes == null
  const float2* tw;
};

template <int L, int ST>
__global__ void __launch_bounds__(RowCfg<L>::THREADS) k_rows_r2c(R2CArgs a) {
  constexpr int E = LCfg<L>::E, T = LCfg<L>::T;
  extern __shared__ float2 smem[];
  const int team = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = smem + team * LCfg<L>::BUF;
  const int plane = a.plane0 + blockIdx.y;
  const int r0 = 2 * (blockIdx.x * RowCfg<L>::TEAMS + team), r1 = r0 + 1;
  const bool act0 = r0 < a.M, act1 = r1 < a.M;
  const void* src = static_cast<const char*>(a.src) +
                    (long long)blockIdx.y * a.src_plane_stride * (ST == FFST_STORE_F32 ? 4 : 2);
  const float us = (ST != FFST_STORE_F32 && a.plane_scale) ? 1.0f / __ldg(&a.plane_scale[plane]) : 1.0f;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int n = t + T * m;
    const float xa = act0 ? load_st<ST>(src, (long long)r0 * L + n) : 0.0f;
    const float xb = act1 ? load_st<ST>(src, (long long)r1 * L + n) : 0.0f;
    v[m] = make_float2(xa * us, xb * us);
  }
  line_fft<L, false, RowCfg<L>::WARP>(v, buf, t, a.tw);
#pragma unroll
  for (int m = 0; m < E; ++m) buf[LCfg<L>::pad(t + T * m)] = v[m];
  team_sync<RowCfg<L>::WARP>();
  int c0 = a.c0, W = a.W, ld = a.ld;
  float2* dst = a.dst;
  if (a.planes) {
    const PlaneDesc d = a.planes[plane];
    c0 = d.c0;
    W = d.W;
    ld = d.W;
    dst = a.dst + d.off;
  }
  for (int idx = t; idx < W; idx += T) {
    const int kx = c0 + idx;
    const float2 z = buf[LCfg<L>::pad(kx)];
    const float2 zn = buf[LCfg<L>::pad((L - kx) & (L - 1))];
    if (act0) dst[(long long)r0 * ld + idx] = make_float2(0.5f * (z.x + zn.x), 0.5f * (z.y - zn.y));
    if (act1) dst[(long long)r1 * ld + idx] = make_float2(0.5f * (z.y + zn.y), -0.5f * (z.x - zn.x));
  }
}

struct C2RArgs {
  const float2* src;
  const PlaneDesc* planes;  // non-null: grouped input (per-plane c0, W, off)
  int c0, W, ld;            // used when planes == null
  int M;
  int plane0;
  void* dst;                // plane 0 of the batch
  long long dst_plane_stride;
  const float* plane_scale;  // low-precision storage: multiply by s_i before rounding
  float scale;               // 1/(M N)
  const float2* tw;
};

template <int L, int ST>
__global__ void __launch_bounds__(RowCfg<L>::THREADS) k_rows_c2r(C2RArgs a) {
  constexpr int E = LCfg<L>::E, T = LCfg<L>::T;
  extern __shared__ float2 smem[];
  const int team = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = smem + team * LCfg<L>::BUF;
  const int plane = a.plane0 + blockIdx.y;
  const int r0 = 2 * (blockIdx.x * RowCfg<L>::TEAMS + team), r1 = r0 + 1;
  const bool act0 = r0 < a.M, act1 = r1 < a.M;
  int c0 = a.c0, W = a.W, ld = a.ld;
  const float2* src = a.src;
  if (a.planes) {
    const PlaneDesc d = a.planes[plane];
    c0 = d.c0;
    W = d.W;
    ld = d.W;
    src = a.src + d.off;
  }
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int kx = t + T * m;
    const bool upper = 2 * kx > L;
    const int kk = upper ? L - kx : kx;
    const int idx = kk - c0;
    const bool in = idx >= 0 && idx < W;
    float2 A = (in && act0) ? src[(long long)r0 * ld + idx] : make_float2(0.f, 0.f);
    float2 B = (in && act1) ? src[(long long)r1 * ld + idx] : make_float2(0.f, 0.f);
    if (kx == 0 || 2 * kx == L) {
      A.y = 0.f;
      B.y = 0.f;
    }
    if (upper) {
      A.y = -A.y;
      B.y = -B.y;
    }
    v[m] = make_float2(A.x - B.y, A.y + B.x);
  }
  line_fft<L, true, RowCfg<L>::WARP>(v, buf, t, a.tw);
  float s = a.scale;
  if (ST != FFST_STORE_F32 && a.plane_scale) s *= __ldg(&a.plane_scale[plane]);
  void* dst = static_cast<char*>(a.dst) + (long long)blockIdx.y * a.dst_plane_stride * (ST == FFST_STORE_F32 ? 4 : 2);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int n = t + T * m;
    if (act0) store_st<ST>(dst, (long long)r0 * L + n, v[m].x * s);
    if (act1) store_st<ST>(dst, (long long)r1 * L + n, v[m].y * s);
  }
}

// ---------------------------------------------------------------------------
// launchers
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
static cudaError_t r2c_L(const ffst_plan_s* p, const R2CArgs& a, int storage, int nplanes, cudaStream_t s) {
  const int pairs = (a.M + 1) / 2;
  dim3 grid((pairs + RowCfg<L>::TEAMS - 1) / RowCfg<L>::TEAMS, nplanes);
  const size_t smem = RowCfg<L>::SMEM;
  cudaError_t e;
  switch (storage) {
    case FFST_STORE_F32:
      if ((e = prepare(k_rows_r2c<L, FFST_STORE_F32>, smem)) != cudaSuccess) return e;
      k_rows_r2c<L, FFST_STORE_F32><<<grid, RowCfg<L>::THREADS, smem, s>>>(a);
      break;
    case FFST_STORE_F16:
      if ((e = prepare(k_rows_r2c<L, FFST_STORE_F16>, smem)) != cudaSuccess) return e;
      k_rows_r2c<L, FFST_STORE_F16><<<grid, RowCfg<L>::THREADS, smem, s>>>(a);
      break;
    default:
      if ((e = prepare(k_rows_r2c<L, FFST_STORE_BF16>, smem)) != cudaSuccess) return e;
      k_rows_r2c<L, FFST_STORE_BF16><<<grid, RowCfg<L>::THREADS, smem, s>>>(a);
      break;
  }
  return cudaGetLastError();
}

template <int L>
static cudaError_t c2r_L(const ffst_plan_s* p, const C2RArgs& a, int storage, int nplanes, cudaStream_t s) {
  const int pairs = (a.M + 1) / 2;
  dim3 grid((pairs + RowCfg<L>::TEAMS - 1) / RowCfg<L>::TEAMS, nplanes);
  const size_t smem = RowCfg<L>::SMEM;
  cudaError_t e;
  switch (storage) {
    case FFST_STORE_F32:
      if ((e = prepare(k_rows_c2r<L, FFST_STORE_F32>, smem)) != cudaSuccess) return e;
      k_rows_c2r<L, FFST_STORE_F32><<<grid, RowCfg<L>::THREADS, smem, s>>>(a);
      break;
    case FFST_STORE_F16:
      if ((e = prepare(k_rows_c2r<L, FFST_STORE_F16>, smem)) != cudaSuccess) return e;
      k_rows_c2r<L, FFST_STORE_F16><<<grid, RowCfg<L>::THREADS, smem, s>>>(a);
      break;
    default:
      if ((e = prepare(k_rows_c2r<L, FFST_STORE_BF16>, smem)) != cudaSuccess) return e;
      k_rows_c2r<L, FFST_STORE_BF16><<<grid, RowCfg<L>::THREADS, smem, s>>>(a);
      break;
  }
  return cudaGetLastError();
}

#define FFST_DISPATCH_L(L, CALL)                                   \
  switch (L) {                                                     \
    case 8: return CALL(8);                                        \
    case 16: return CALL(16);                                      \
    case 32: return CALL(32);                                      \
    case 64: return CALL(64);                                      \
    case 128: return CALL(128);                                    \
    case 256: return CALL(256);                                    \
    case 512: return CALL(512);                                    \
    case 1024: return CALL(1024);                                  \
    case 2048: return CALL(2048);                                  \
    case 4096: return CALL(4096);                                  \
    default: return cudaErrorInvalidValue;                         \
  }

cudaError_t launch_rows_r2c(const ffst_plan_s* p, int L, const void* src, int storage, const float* plane_scale,
                            int plane0, int nplanes, long long src_plane_stride, float2* dst, bool dst_grouped,
                            int full_c0, int full_W, int dst_ld, cudaStream_t s) {
  R2CArgs a;
  a.src = src;
  a.src_plane_stride = src_plane_stride;
  a.plane_scale = plane_scale;
  a.plane0 = plane0;
  a.M = p->M;
  a.dst = dst;
  a.planes = dst_grouped ? p->d_planes : nullptr;
  a.c0 = full_c0;
  a.W = full_W;
  a.ld = dst_ld;
  a.tw = p->d_tw_rows;
#define R2C_CALL(LL) r2c_L<LL>(p, a, storage, nplanes, s)
  FFST_DISPATCH_L(L, R2C_CALL)
#undef R2C_CALL
}

cudaError_t launch_rows_c2r(const ffst_plan_s* p, int L, const float2* src, bool src_grouped, int full_W, int src_ld,
                            int plane0, int nplanes, void* dst, int storage, const float* plane_scale,
                            long long dst_plane_stride, float scale, cudaStream_t s) {
  C2RArgs a;
  a.src = src;
  a.planes = src_grouped ? p->d_planes : nullptr;
  a.c0 = 0;
  a.W = full_W;
  a.ld = src_ld;
  a.M = p->M;
  a.plane0 = plane0;
  a.dst = dst;
  a.dst_plane_stride = dst_plane_stride;
  a.plane_scale = plane_scale;
  a.scale = scale;
  a.tw = p->d_tw_rows;
#define C2R_CALL(LL) c2r_L<LL>(p, a, storage, nplanes, s)
  FFST_DISPATCH_L(L, C2R_CALL)
#undef C2R_CALL
}

}  // namespace ffst
