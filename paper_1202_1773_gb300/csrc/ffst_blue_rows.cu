// Generic-length row passes (Bluestein lines, ffst_blue.cuh) and the
// Bluestein tables.
#include <cmath>
#include <vector>

#include "ffst_blue.cuh"

namespace ffst {

// ---------------------------------------------------------------------------
// host tables
// ---------------------------------------------------------------------------
int blue_L2(int n) {
  int L2 = kBlueMinL2;
  while (L2 < 2 * n - 1) L2 *= 2;
  return L2;
}

int smooth_L2(int n) {
  int L2 = kBlueMinL2;
  while (L2 < n) L2 *= 2;
  return L2;
}

bool smooth_line(int n, int* nrad, unsigned long long* radices, std::vector<float2>* tw) {
  std::vector<int> rs;
  int m = n;
  while (m % 8 == 0) {
    rs.push_back(8);
    m /= 8;
  }
  if (m % 4 == 0) {
    rs.push_back(4);
    m /= 4;
  } else if (m % 2 == 0) {
    rs.push_back(2);
    m /= 2;
  }
  for (int p : {3, 5, 7})
    while (m % p == 0) {
      rs.push_back(p);
      m /= p;
    }
  if (m != 1 || rs.empty() || rs.size() > 16) return false;
  *nrad = (int)rs.size();
  *radices = 0;
  for (size_t s = 0; s < rs.size(); ++s) *radices |= (unsigned long long)rs[s] << (4 * s);
  // pass s (sub-transform length Ns, radix R): W_{Ns R}^{kk r} = exp(-2 pi i kk r / (Ns R))
  // at (Ns - 1) + (r - 1) Ns + kk, the angle reduced exactly (kk r mod Ns R)
  tw->assign(n > 1 ? n - 1 : 1, make_float2(1.f, 0.f));
  const double pi = 3.14159265358979323846;
  long long Ns = 1;
  for (int R : rs) {
    for (int r = 1; r < R; ++r)
      for (long long kk = 0; kk < Ns; ++kk) {
        const long long q = (kk * r) % (Ns * R);
        const double ang = -2.0 * pi * (double)q / (double)(Ns * R);
        (*tw)[(Ns - 1) + (r - 1) * Ns + kk] = make_float2((float)std::cos(ang), (float)std::sin(ang));
      }
    Ns *= R;
  }
  return true;
}

void blue_tables(int n, int* L2out, std::vector<float2>* chirp, std::vector<float2>* bhat) {
  const int L2 = blue_L2(n);
  *L2out = L2;
  const double pi = 3.14159265358979323846;
  // w_j = exp(-i pi j^2 / n): j^2 reduced mod 2n exactly, so the angle stays small
  std::vector<double> wr(n), wi(n);
  for (int j = 0; j < n; ++j) {
    const long long q = ((long long)j * j) % (2LL * n);
    const double ang = -pi * (double)q / (double)n;
    wr[j] = std::cos(ang);
    wi[j] = std::sin(ang);
  }
  chirp->assign(n, make_float2(0.f, 0.f));
  for (int j = 0; j < n; ++j) (*chirp)[j] = make_float2((float)wr[j], (float)wi[j]);
  // filter b[m] = conj(w_|m|) on -n < m < n, wrapped to length L2
  std::vector<double> br(L2, 0.0), bi(L2, 0.0);
  for (int m = 0; m < n; ++m) {
    br[m] = wr[m];
    bi[m] = -wi[m];
    if (m > 0) {
      br[L2 - m] = wr[m];
      bi[L2 - m] = -wi[m];
    }
  }
  // its DFT by the definition (exact index reduction k m mod L2), times 1/L2
  std::vector<double> cr(L2), ci(L2);
  for (int q = 0; q < L2; ++q) {
    cr[q] = std::cos(2.0 * pi * q / L2);
    ci[q] = -std::sin(2.0 * pi * q / L2);
  }
  bhat->assign(L2, make_float2(0.f, 0.f));
  for (int k = 0; k < L2; ++k) {
    double sr = 0.0, si = 0.0;
    for (int m = 0; m < L2; ++m) {
      if (br[m] == 0.0 && bi[m] == 0.0) continue;
      const int q = (int)(((long long)k * m) & (L2 - 1));
      sr += br[m] * cr[q] - bi[m] * ci[q];
      si += br[m] * ci[q] + bi[m] * cr[q];
    }
    (*bhat)[k] = make_float2((float)(sr / L2), (float)(si / L2));
  }
}

int blue_lines_per_block(int L2) {
  switch (L2) {
    case 16: return BlueCfg<16>::P;
    case 32: return BlueCfg<32>::P;
    case 64: return BlueCfg<64>::P;
    case 128: return BlueCfg<128>::P;
    case 256: return BlueCfg<256>::P;
    case 512: return BlueCfg<512>::P;
    case 1024: return BlueCfg<1024>::P;
    case 2048: return BlueCfg<2048>::P;
    case 4096: return BlueCfg<4096>::P;
    default: return 0;
  }
}

// Elements j = t + T m (j < n) of rows r0 and r1 (when present) of a stack
// of storage type ST, times f, as the line z = x_a + i x_b.
template <int E, int T, int ST>
__device__ __forceinline__ void load_row_pair(float2 (&v)[E], const void* src, int r0, int r1, bool a0, bool a1,
                                              int n, int t, float f) {
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int j = t + T * m;
    const float x0 = (a0 && j < n) ? load_one(src, (long long)r0 * n + j, ST) * f : 0.0f;
    const float x1 = (a1 && j < n) ? load_one(src, (long long)r1 * n + j, ST) * f : 0.0f;
    v[m] = make_float2(x0, x1);
  }
}

// The line x_a + i x_b back to rows r0 and r1 (when present), elements
// j = t + T m < n, in storage type ST.
template <int E, int T, int ST>
__device__ __forceinline__ void store_row_pair(const float2 (&v)[E], void* dst, int r0, int r1, bool a0, bool a1,
                                               int n, int t) {
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int j = t + T * m;
    if (j >= n) continue;
    if (a0) store_one(dst, (long long)r0 * n + j, v[m].x, ST);
    if (a1) store_one(dst, (long long)r1 * n + j, v[m].y, ST);
  }
}

// ---------------------------------------------------------------------------
// row R2C: rows r0 = 2 (bx P + team) and r0 + 1 of plane plane0 + by as one
// complex line z = x_a + i x_b; Z = DFT_n(z) goes through the team buffer and
// 2 X_a[k] = Z[k] + conj Z[n-k], 2 X_b[k] = -i (Z[k] - conj Z[n-k]) are
// written for the half-spectrum columns k of the output (kR2CGain = 2, as
// the native row pass).
// ---------------------------------------------------------------------------
template <int L2>
__global__ void __launch_bounds__(kThreads, 3) k_blue_rows_r2c(R2CArgs a, BlueLine b) {
  constexpr int E = BlueCfg<L2>::E, T = BlueCfg<L2>::T, P = BlueCfg<L2>::P;
  extern __shared__ __align__(128) float2 smem[];
  const int team = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = smem + team * blue_stride<L2>(b);
  const int n = b.n;
  const int by = blockIdx.y, plane = a.plane0 + by;
  const int r0 = 2 * (blockIdx.x * P + team), r1 = r0 + 1;
  const bool a0 = r0 < a.M, a1 = r1 < a.M;
  const void* src = static_cast<const char*>(a.src) + (long long)by * a.src_plane_stride * stor_bytes(a.st);
  float f = 1.0f;
  int st = a.st;
  if (a.cplx) {  // FP32 real parts of a complex stack, c_i = sqrt(2) Re z_i (i >= 1)
    f = plane == 0 ? 1.0f : 1.41421356237309505f;
    st = FFST_STORE_F32;
  } else if (st != FFST_STORE_F32 && a.plane_scale) {
    f = 1.0f / __ldg(&a.plane_scale[plane]);
  }
  float2 v[E];
  // one loop per storage type, so that all 2E loads of a thread are in
  // flight together (a type switch per element serialises them)
  if (st == FFST_STORE_F32) load_row_pair<E, T, FFST_STORE_F32>(v, src, r0, r1, a0, a1, n, t, f);
  else if (st == FFST_STORE_F16) load_row_pair<E, T, FFST_STORE_F16>(v, src, r0, r1, a0, a1, n, t, f);
  else load_row_pair<E, T, FFST_STORE_BF16>(v, src, r0, r1, a0, a1, n, t, f);
  blue_dft<L2, false>(v, buf, t, b);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = t + T * m;
    if (k < n) buf[k] = v[m];
  }
  __syncthreads();
  int c0 = a.c0, W = a.W, ld = a.ld;
  float2* dst = a.dst;
  if (a.planes) {  // the plane's slot: pitch ldw, column c at c - c0al
    const PlaneDesc d = a.planes[plane];
    c0 = d.c0;
    W = d.W;
    ld = d.ldw;
    dst = a.dst + d.off + (d.c0 - d.c0al);
  }
  for (int idx = t; idx < W; idx += T) {
    const int k = c0 + idx;  // 0 .. n/2
    const float2 zk = buf[k];
    const float2 zn = buf[k == 0 ? 0 : n - k];
    if (a0) __stcg(&dst[(long long)r0 * ld + idx], make_float2(zk.x + zn.x, zk.y - zn.y));
    if (a1) __stcg(&dst[(long long)r1 * ld + idx], make_float2(zk.y + zn.y, zn.x - zk.x));
  }
}

// ---------------------------------------------------------------------------
// row C2R: the half spectra of rows r0, r0 + 1 are completed Hermitian
// (X[k] = conj X[n-k] for 2k > n; the imaginary parts of X[0] and, for even
// n, X[n/2] dropped, as the native C2R), packed as X_a + i X_b, and one
// inverse DFT gives x_a + i x_b.  Then the native epilogue: factor
// scale * s_i, per-plane statistics and shrinkage, storage.
// ---------------------------------------------------------------------------
template <int L2>
__global__ void __launch_bounds__(kThreads, 3) k_blue_rows_c2r(C2RArgs a, BlueLine b) {
  constexpr int E = BlueCfg<L2>::E, T = BlueCfg<L2>::T, P = BlueCfg<L2>::P;
  extern __shared__ __align__(128) float2 smem[];
  __shared__ float red[kThreads / 32];
  const int team = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = smem + team * blue_stride<L2>(b);
  const int n = b.n;
  const int by = blockIdx.y, plane = a.plane0 + by;
  const int r0 = 2 * (blockIdx.x * P + team), r1 = r0 + 1;
  const bool a0 = r0 < a.M, a1 = r1 < a.M;
  int c0 = a.c0, W = a.W, ld = a.ld;
  const float2* src = a.src;
  if (a.planes) {
    const PlaneDesc d = a.planes[plane];
    c0 = d.c0;
    W = d.W;
    ld = d.ldw;
    src = a.src + d.off + (d.c0 - d.c0al);
  }
  const float ps = c2r_plane_factor(a, by);
  const float s = a.scale * ps;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = t + T * m;
    float2 x0 = make_float2(0.f, 0.f), x1 = make_float2(0.f, 0.f);
    if (k < n) {
      const bool upper = 2 * k > n;
      const int q = (upper ? n - k : k) - c0;
      if ((unsigned)q < (unsigned)W) {
        if (a0) x0 = __ldcg(&src[(long long)r0 * ld + q]);
        if (a1) x1 = __ldcg(&src[(long long)r1 * ld + q]);
      }
      if (upper) {
        x0.y = -x0.y;
        x1.y = -x1.y;
      }
      if (k == 0 || 2 * k == n) {
        x0.y = 0.f;
        x1.y = 0.f;
      }
    }
    v[m] = make_float2(x0.x - x1.y, x0.y + x1.x);  // X_a + i X_b
  }
  blue_dft<L2, true>(v, buf, t, b);
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = make_float2(v[m].x * s, v[m].y * s);
  if (a.shrink || a.abs_partials) {  // uniform over the launch; v holds c * ps
    const float tau = a.shrink ? __ldg(&a.thresh[plane]) * ps : 0.0f;
    float acc = 0.0f;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      if (t + T * m >= n) continue;
      float x = v[m].x, y = v[m].y;
      acc += (a0 ? fabsf(x) : 0.0f) + (a1 ? fabsf(y) : 0.0f);
      if (a.shrink == 1) {
        x = copysignf(fmaxf(fabsf(x) - tau, 0.0f), x);
        y = copysignf(fmaxf(fabsf(y) - tau, 0.0f), y);
      } else if (a.shrink == 2) {
        x = fabsf(x) > tau ? x : 0.0f;
        y = fabsf(y) > tau ? y : 0.0f;
      }
      v[m] = make_float2(x, y);
    }
    if (a.abs_partials) {  // fixed reduction order: deterministic
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        float sum = 0.0f;
        for (int q = 0; q < kThreads / 32; ++q) sum += red[q];
        a.abs_partials[(long long)plane * a.rbx + blockIdx.x] = sum / ps;
      }
    }
  }
  void* dst = static_cast<char*>(a.dst) + (long long)by * a.dst_plane_stride * stor_bytes(a.st);
  if (a.st == FFST_STORE_F32) store_row_pair<E, T, FFST_STORE_F32>(v, dst, r0, r1, a0, a1, n, t);
  else if (a.st == FFST_STORE_F16) store_row_pair<E, T, FFST_STORE_F16>(v, dst, r0, r1, a0, a1, n, t);
  else store_row_pair<E, T, FFST_STORE_BF16>(v, dst, r0, r1, a0, a1, n, t);
}

template <int L2>
static cudaError_t rows_r2c_L2(const BlueLine& b, const R2CArgs& a, int nplanes, cudaStream_t s) {
  constexpr int P = BlueCfg<L2>::P;
  const dim3 grid((unsigned)(((a.M + 1) / 2 + P - 1) / P), (unsigned)nplanes);
  if (nplanes <= 0 || a.M <= 0) return cudaSuccess;
  cudaError_t e = set_smem(k_blue_rows_r2c<L2>, blue_smem<L2>(b));
  if (e != cudaSuccess) return e;
  k_blue_rows_r2c<L2><<<grid, kThreads, blue_smem<L2>(b), s>>>(a, b);
  return cudaGetLastError();
}

template <int L2>
static cudaError_t rows_c2r_L2(const BlueLine& b, const C2RArgs& a, int nplanes, cudaStream_t s) {
  constexpr int P = BlueCfg<L2>::P;
  const dim3 grid((unsigned)(((a.M + 1) / 2 + P - 1) / P), (unsigned)nplanes);
  if (nplanes <= 0 || a.M <= 0) return cudaSuccess;
  cudaError_t e = set_smem(k_blue_rows_c2r<L2>, blue_smem<L2>(b));
  if (e != cudaSuccess) return e;
  k_blue_rows_c2r<L2><<<grid, kThreads, blue_smem<L2>(b), s>>>(a, b);
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

cudaError_t launch_blue_rows_r2c(const BlueLine& b, const R2CArgs& a, int nplanes, cudaStream_t s) {
#define CALL_(LL) rows_r2c_L2<LL>(b, a, nplanes, s)
  FFST_DISPATCH_BLUE(b.L2, CALL_)
#undef CALL_
}

cudaError_t launch_blue_rows_c2r(const BlueLine& b, const C2RArgs& a, int nplanes, cudaStream_t s) {
#define CALL_(LL) rows_c2r_L2<LL>(b, a, nplanes, s)
  FFST_DISPATCH_BLUE(b.L2, CALL_)
#undef CALL_
}

}  // namespace ffst
