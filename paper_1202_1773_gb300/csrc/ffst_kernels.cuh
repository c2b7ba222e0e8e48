// Device bodies of the transform kernels.  Each body works on one logical
// block (given explicitly), so the same code runs in a standalone kernel or
// inside a fused launch that interleaves row-pass and column-pass blocks.
// All bodies assume kThreads (256) threads per block.
//
// Row passes (real rows of length N <-> half spectra, columns 0..N/2): a real
// row x is transformed as the complex line z[n] = x[2n] + i x[2n+1] of
// length L = N/2 (the real-input FFT of the signal-processing literature):
//  R2C: Z = FFT_L(z);  X[k] = E[k] + W_N^k O[k] with
//       E[k] = (Z[k] + conj Z[L-k]) / 2,  O[k] = (Z[k] - conj Z[L-k]) / (2i),
//       for the kept columns k in [c0, c0 + W) of [0, N/2] (W_N = e^{-2 pi i/N}).
//       The kernel writes 2 X[k] (kR2CGain): the halving is left to the
//       consumers, which fold it into a scale they apply anyway.
//  C2R: Z[k] = (X[k] + conj X[L-k]) + i W_N^{-k} (X[k] - conj X[L-k]),
//       k in [0, L); z = IFFT_L(Z) holds x[2n] + i x[2n+1] (times N for the
//       unnormalised inverse).  Columns outside [c0, c0 + W) are zero (the
//       plane's spectral support); the imaginary parts of X[0] and X[N/2]
//       are dropped (Hermitian part).
//
// Column passes (half-spectrum buffers [M][ld], complex, row-major): a block
// owns a panel of P adjacent columns.  In cols_fft_body and inv_cols_body
// thread (t, c) is threadIdx.x = t*P + c, so the P columns of one row are
// read or written by consecutive lanes, and the exchanges use block
// barriers; fwd_cols_body gives each column a contiguous team of T threads
// with its own barrier.  Within a plane's support column, psi_hat is nonzero
// only on one cyclic row interval (start, len) computed at plan time; the
// window is generated and F is read only there.
#pragma once

#include "ffst_fft.cuh"
#include "ffst_tma.cuh"
#include "ffst_window.cuh"

namespace ffst {

// ---------------------------------------------------------------------------
// storage of a coefficient stack (runtime code, uniform over a launch)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int stor_bytes(int st) { return st == FFST_STORE_F32 ? 4 : 2; }

// Stack and image rows are touched once per transform: loads and stores use
// the streaming (evict-first) cache policy so they do not push the plane
// group intermediates out of L2.
__device__ __forceinline__ float2 load_pair(const void* p, long long i, int st) {  // elements i, i+1 (i even)
  if (st == FFST_STORE_F32) return __ldcs(reinterpret_cast<const float2*>(static_cast<const float*>(p) + i));
  if (st == FFST_STORE_F16)
    return __half22float2(__ldcs(reinterpret_cast<const __half2*>(static_cast<const __half*>(p) + i)));
  return __bfloat1622float2(__ldcs(reinterpret_cast<const __nv_bfloat162*>(static_cast<const __nv_bfloat16*>(p) + i)));
}

__device__ __forceinline__ void store_pair(void* p, long long i, float a, float b, int st) {
  if (st == FFST_STORE_F32)
    __stcs(reinterpret_cast<float2*>(static_cast<float*>(p) + i), make_float2(a, b));
  else if (st == FFST_STORE_F16)
    __stcs(reinterpret_cast<__half2*>(static_cast<__half*>(p) + i), __floats2half2_rn(a, b));
  else
    __stcs(reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(p) + i), __floats2bfloat162_rn(a, b));
}

// Every half spectrum the row R2C writes is kR2CGain times the DFT.
constexpr float kR2CGain = 2.0f;

// Bounds checks of the debug build (-DFFST_CHECK): every global access of the
// transform bodies is tested against its buffer's extent (bytes from the
// buffer's base, carried in the argument structs).  An access outside is
// skipped (a load reads zero) and sets kErrBounds in the plan's error word,
// which ffst_plan_check reports as FFST_ERR_BOUNDS; nothing traps.  In
// normal builds the checks compile to nothing.
constexpr int kErrBounds = 8;
#ifdef FFST_CHECK
__device__ __forceinline__ bool ck(const void* p, int bytes, const void* base, long long extent, int* err) {
  const char* q = static_cast<const char*>(p);
  const char* b = static_cast<const char*>(base);
  const bool ok = q >= b && q + bytes <= b + extent;
  if (!ok && err) atomicOr(err, kErrBounds);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool ck(const void*, int, const void*, long long, int*) { return true; }
#endif

// load_pair / store_pair checked against [base, base + extent) bytes.
__device__ __forceinline__ float2 load_pair_ck(const void* p, long long i, int st, const void* base, long long ext,
                                               int* err) {
  const int es = stor_bytes(st);
  if (!ck(static_cast<const char*>(p) + i * es, 2 * es, base, ext, err)) return make_float2(0.f, 0.f);
  return load_pair(p, i, st);
}
__device__ __forceinline__ void store_pair_ck(void* p, long long i, float x, float y, int st, const void* base,
                                              long long ext, int* err) {
  const int es = stor_bytes(st);
  if (ck(static_cast<char*>(p) + i * es, 2 * es, base, ext, err)) store_pair(p, i, x, y, st);
}


// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
// Row-line geometry with EL elements per thread (default row_E(L)); the
// 32-element variant of the long lines (radix 32 x 32 at L = 1024, one warp
// per line) is a tuning choice of the standalone row kernels.
template <int L, int EL = row_E(L)>
struct RowCfg {
  static_assert(supported_line(L), "unsupported row line length");
  static constexpr int E = EL;
  static constexpr int T = L / E;
  static constexpr int TEAMS = (T >= kThreads) ? 1 : kThreads / T;  // rows per block
  static constexpr int SYNC = T <= 32 ? kSyncWarp : (T < kThreads ? kSyncNamed : kSyncBlock);
  static constexpr int BUF = team_stride(L, E, T < 16 ? T : 0);
  static constexpr size_t SMEM = sizeof(float2) * TEAMS * BUF;
  static_assert(TEAMS * T == kThreads, "row teams must fill the block");
};

template <int L>
struct ColCfg {
  static_assert(supported_line(L), "unsupported column length");
  static constexpr int E = col_E(L);
  static constexpr int T = L / E;
  static constexpr int P = kThreads / T;  // columns per block
  static constexpr int BUF = team_stride(L, E, P >= 16 ? 1 : 16 / P);
  static constexpr size_t SMEM = sizeof(float2) * P * BUF;
  static_assert(P * T == kThreads, "column teams must fill the block");
};

// v[m] for a runtime m (a chain of selects, no local memory).
template <int E>
__device__ __forceinline__ float2 pick(const float2 (&v)[E], int m) {
  float2 r = v[0];
#pragma unroll
  for (int k = 1; k < E; ++k)
    if (m == k) r = v[k];
  return r;
}

template <int M>
__device__ __forceinline__ bool in_range(int row, int2 rg) {
  return mod_l<M>(row - rg.x) < rg.y;
}

// ---------------------------------------------------------------------------
// row passes
// ---------------------------------------------------------------------------
struct R2CArgs {
  const void* src;           // plane 0 of the batch (row-major rows x 2L)
  long long src_plane_stride;
  int st;                    // storage code of src
  const float* plane_scale;  // per plane s_i (low-precision storage) or null
  int cplx;                  // input is Re z of one-sided coefficients: c_i = sqrt(2) Re z_i, i >= 1
  int plane0;                // plane index of by == 0 (for descriptors/scales)
  int M;                     // rows
  float2* dst;               // grouped: base of the group's intermediate
  const PlaneDesc* planes;   // non-null: grouped output (per-plane c0, W, off)
  int c0, W, ld;             // used when planes == null
  const float2* tw;          // pass table (L, E)
  const float2* rtw;         // W_N^k, k = 0..L
  long long src_bytes;       // extents from src and dst (bounds checks of FFST_CHECK builds)
  long long dst_bytes;
  int* err;                  // plan error word (FFST_CHECK builds)
};

template <int L, int EL = row_E(L), bool XSHFL = false>
__device__ __forceinline__ void rows_r2c_body(const R2CArgs& a, int bx, int by, float2* smem) {
  using C = RowCfg<L, EL>;
  static_assert(!XSHFL || (L == 1024 && EL == 32), "the shuffle exchange is built for 1024-point lines of one warp");
  constexpr int E = C::E, T = C::T, N = 2 * L;
  const int team = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = smem + team * C::BUF;
  const int plane = a.plane0 + by;
  const int row = bx * C::TEAMS + team;
  const bool act = row < a.M;
  const void* src = static_cast<const char*>(a.src) + (long long)by * a.src_plane_stride * stor_bytes(a.st);
  const float us = (a.st != FFST_STORE_F32 && a.plane_scale) ? 1.0f / __ldg(&a.plane_scale[plane]) : 1.0f;
  float2 v[E];
  const long long rbase = (long long)row * N + 2 * t;
  if (!act) {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = make_float2(0.f, 0.f);
  } else if (a.cplx) {  // FP32 real parts of a complex stack, c_i = sqrt(2) Re z_i (i >= 1)
    const float cs = plane == 0 ? 1.0f : 1.41421356237309505f;
#pragma unroll
    for (int m = 0; m < E; ++m)
      v[m] = cscale(load_pair_ck(src, rbase + 2 * T * m, FFST_STORE_F32, a.src, a.src_bytes, a.err), cs);
  } else if (a.st == FFST_STORE_F32) {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = load_pair_ck(src, rbase + 2 * T * m, FFST_STORE_F32, a.src, a.src_bytes, a.err);
  } else if (a.st == FFST_STORE_F16) {  // one loop per type: the loads of a thread fly together
#pragma unroll
    for (int m = 0; m < E; ++m)
      v[m] = cscale(load_pair_ck(src, rbase + 2 * T * m, FFST_STORE_F16, a.src, a.src_bytes, a.err), us);
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m)
      v[m] = cscale(load_pair_ck(src, rbase + 2 * T * m, FFST_STORE_BF16, a.src, a.src_bytes, a.err), us);
  }
  if constexpr (XSHFL) line_fft_shfl1024<false>(v, t, a.tw);
  else line_fft<L, E, false, C::SYNC>(v, buf, t, a.tw, 1 + team);
  team_store<E, T>(buf, t, v);
  team_sync<C::SYNC, T>(1 + team);
  if (!act) return;
  int c0 = a.c0, W = a.W, ld = a.ld;
  float2* dst = a.dst;
  if (a.planes) {  // the plane's slot: pitch ldw, column c at c - c0al
    const PlaneDesc d = a.planes[plane];
    c0 = d.c0;
    W = d.W;
    ld = d.ldw;
    dst = a.dst + d.off + (d.c0 - d.c0al);
  }
  float2* drow = dst + (long long)row * ld;
  for (int idx = t; idx < W; idx += T) {
    const int k = c0 + idx;  // 0 .. L
    const float2 zk = buf[spad<E>(mod_l<L>(k))];
    const float2 zn = buf[spad<E>(mod_l<L>(L - k))];
    const float2 e = make_float2(zk.x + zn.x, zk.y - zn.y);  // 2 E[k]
    const float2 o = make_float2(zk.y + zn.y, zn.x - zk.x);  // 2 O[k]
    const float2 w = __ldg(&a.rtw[k]);
    if (ck(&drow[idx], 8, a.dst, a.dst_bytes, a.err))
      __stcg(&drow[idx], make_float2(e.x + w.x * o.x - w.y * o.y, e.y + w.x * o.y + w.y * o.x));
  }
}

struct C2RArgs {
  const float2* src;        // grouped: base of the group's intermediate
  const PlaneDesc* planes;  // non-null: grouped input (per-plane c0, W, off)
  int c0, W, ld;            // used when planes == null
  int M;
  int plane0;
  void* dst;                // plane 0 of the batch
  long long dst_plane_stride;
  int st;                   // storage code of dst
  const float* plane_scale;  // low-precision storage: multiply by s_i before rounding
  float scale;               // output factor (1 when the producer already normalised)
  const float2* tw;
  const float2* rtw;
  // fused per-plane statistics and shrinkage of the coefficients c (plane rows only)
  int shrink;                // 0 none, 1 soft, 2 hard
  const float* thresh;       // per-plane threshold on |c| (shrink != 0)
  float* abs_partials;       // per (plane, row block): sum |c| before shrinkage, or null
  int rbx;                   // row blocks per plane (stride of abs_partials)
  int cplx;                  // complex planar output (Sec. 3.8.2): factor 1/sqrt(2) on planes i >= 1
  long long src_bytes;       // extents from src and dst (bounds checks of FFST_CHECK builds)
  long long dst_bytes;
  int* err;                  // plan error word (FFST_CHECK builds)
};

// Factor s_i of plane a.plane0 + by for low-precision storage (1 otherwise),
// read from the caller's per-plane scales.
__device__ __forceinline__ float c2r_plane_factor(const C2RArgs& a, int by) {
  if (a.cplx) return (a.plane0 + by) == 0 ? 1.0f : 0.70710678118654752f;  // z_i = (c_i + i d_i) / sqrt(2)
  return (a.st != FFST_STORE_F32 && a.plane_scale) ? __ldg(&a.plane_scale[a.plane0 + by]) : 1.0f;
}

// s_i = 2^floor(log2(target / B_i)), B_i = sum of the plane's forward column
// partials (item order: deterministic), clamped to 2^+-100; 1 for a zero
// plane.  The partials are read through L2, so a persistent kernel may call
// this for partials written by other blocks of the same launch.
__device__ __forceinline__ float plane_scale_of(const float* partials, int item0, int nitems, float target) {
  float sum = 0.0f;
  for (int q = 0; q < nitems; ++q) sum += __ldcg(&partials[item0 + q]);
  float s = 1.0f;
  if (sum > 0.0f && isfinite(sum)) {
    int e = (int)floorf(log2f(target / sum));
    e = e < -100 ? -100 : (e > 100 ? 100 : e);
    s = ldexpf(1.0f, e);
  }
  return s;
}

// `ps` is the plane factor s_i multiplied into the output (c2r_plane_factor).
// The statistics partials always cover RowCfg<L>::TEAMS rows (the default
// geometry), so a block of another geometry writes TEAMS / that of them.
template <int L, int EL = row_E(L), bool XSHFL = false>
__device__ __forceinline__ void rows_c2r_body(const C2RArgs& a, int bx, int by, float2* smem, float ps) {
  using C = RowCfg<L, EL>;
  static_assert(!XSHFL || (L == 1024 && EL == 32), "the shuffle exchange is built for 1024-point lines of one warp");
  constexpr int E = C::E, T = C::T, N = 2 * L;
  const int team = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = smem + team * C::BUF;
  const int plane = a.plane0 + by;
  const int row = bx * C::TEAMS + team;
  const bool act = row < a.M;
  int c0 = a.c0, W = a.W, ld = a.ld;
  const float2* src = a.src;
  if (a.planes) {  // the plane's slot: pitch ldw, column c at c - c0al
    const PlaneDesc d = a.planes[plane];
    c0 = d.c0;
    W = d.W;
    ld = d.ldw;
    src = a.src + d.off + (d.c0 - d.c0al);
  }
  const float2* srow = src + (long long)row * ld;
  const float s = a.scale * ps;
  float2 v[E];
  // W_N^k for k = t + T m is W_N^t W_{2E}^m: one table entry per thread and
  // a compile-time root per element (keeps the loads off the L1 pipe;
  // forward 1.25 -> 1.22 ms at 2048x2048 J=5)
  const float2 wt = __ldg(&a.rtw[t]);
  static_for<0, E>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    const int k = t + T * m;
    const int ia = k - c0, ib = L - k - c0;
    float2 xa = (act && (unsigned)ia < (unsigned)W && ck(&srow[ia], 8, a.src, a.src_bytes, a.err))
                    ? __ldcg(&srow[ia]) : make_float2(0.f, 0.f);
    float2 xb = (act && (unsigned)ib < (unsigned)W && ck(&srow[ib], 8, a.src, a.src_bytes, a.err))
                    ? __ldcg(&srow[ib]) : make_float2(0.f, 0.f);
    if (m == 0 && t == 0) {  // X[0] and X[N/2]: Hermitian part is real
      xa.y = 0.f;
      xb.y = 0.f;
    }
    const float2 e = make_float2(xa.x + xb.x, xa.y - xb.y);  // X[k] + conj X[L-k]
    // X[k] - conj X[L-k], times conj(W_N^k) = conj(W_N^t) conj(W_{2E}^m)
    const float2 d = twiddle_c<2 * E, m, true>(make_float2(xa.x - xb.x, xa.y + xb.y));
    const float2 wd = make_float2(wt.x * d.x + wt.y * d.y, wt.x * d.y - wt.y * d.x);
    v[m] = make_float2(e.x - wd.y, e.y + wd.x);
  });
  if (s != 1.0f) {  // the transform is linear: scale before it, where the values are in registers
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = make_float2(v[m].x * s, v[m].y * s);
  }
  if constexpr (XSHFL) line_fft_shfl1024<true>(v, t, a.tw);
  else line_fft<L, E, true, C::SYNC>(v, buf, t, a.tw, 1 + team);
  if (a.shrink || a.abs_partials) {  // uniform over the launch
    // v holds c * ps: threshold and statistics act on c (ps is a power of two)
    __shared__ float red[kThreads / 32];
    const float tau = a.shrink ? __ldg(&a.thresh[plane]) * ps : 0.0f;
    float acc = 0.0f;
    if (act) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        float x = v[m].x, y = v[m].y;
        acc += fabsf(x) + fabsf(y);
        if (a.shrink == 1) {
          x = copysignf(fmaxf(fabsf(x) - tau, 0.0f), x);
          y = copysignf(fmaxf(fabsf(y) - tau, 0.0f), y);
        } else if (a.shrink == 2) {
          x = fabsf(x) > tau ? x : 0.0f;
          y = fabsf(y) > tau ? y : 0.0f;
        }
        v[m] = make_float2(x, y);
      }
    }
    if (a.abs_partials) {  // fixed reduction order: deterministic
      constexpr int ratio = C::TEAMS / RowCfg<L>::TEAMS;  // partials per block
      constexpr int wpp = kThreads / 32 / ratio;          // warps per partial
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x < ratio) {
        float sum = 0.0f;
        for (int q = 0; q < wpp; ++q) sum += red[threadIdx.x * wpp + q];
        a.abs_partials[(long long)plane * a.rbx + bx * ratio + threadIdx.x] = sum / ps;
      }
    }
  }
  if (!act) return;
  void* dst = static_cast<char*>(a.dst) + (long long)by * a.dst_plane_stride * stor_bytes(a.st);
  const long long rbase = (long long)row * N + 2 * t;
  if (a.st == FFST_STORE_F32) {
#pragma unroll
    for (int m = 0; m < E; ++m)
      store_pair_ck(dst, rbase + 2 * T * m, v[m].x, v[m].y, FFST_STORE_F32, a.dst, a.dst_bytes, a.err);
  } else if (a.st == FFST_STORE_F16) {
#pragma unroll
    for (int m = 0; m < E; ++m)
      store_pair_ck(dst, rbase + 2 * T * m, v[m].x, v[m].y, FFST_STORE_F16, a.dst, a.dst_bytes, a.err);
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m)
      store_pair_ck(dst, rbase + 2 * T * m, v[m].x, v[m].y, FFST_STORE_BF16, a.dst, a.dst_bytes, a.err);
  }
}

// ---------------------------------------------------------------------------
// column passes
// ---------------------------------------------------------------------------

// In-place column FFTs of columns [0, width) of buf (row stride ld).  With
// nsum > 1 the input is the sum of nsum arrays of that layout, sstride
// elements apart (the inverse's partial accumulators), added in index order
// and written to the first.  When `scale_tab` is given (same layout), each
// element is multiplied by it next.
// buf_bytes: extent of buf and its partial sums (bounds checks of FFST_CHECK
// builds; scale_tab has the layout of one of them in floats).
template <int L, bool INV>
__device__ __forceinline__ void cols_fft_body(float2* __restrict__ buf, int width, int ld,
                                              const float* __restrict__ scale_tab, const float2* __restrict__ tw,
                                              int nsum, long long sstride, int bx, float2* smem, long long buf_bytes,
                                              int* err) {
  constexpr int E = ColCfg<L>::E, T = ColCfg<L>::T, P = ColCfg<L>::P;
  const int t = threadIdx.x / P, cl = threadIdx.x % P;
  const int c = bx * P + cl;
  const bool act = c < width;
  float2* col = buf + (long long)t * ld + c;  // element (t + T m, c) at col[m * T * ld]
  const long long step = (long long)T * ld;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m)
    v[m] = act && ck(&col[m * step], 8, buf, buf_bytes, err) ? col[m * step] : make_float2(0.f, 0.f);
  for (int k = 1; k < nsum && act; ++k) {
    const float2* part = col + k * sstride;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float2 y = ck(&part[m * step], 8, buf, buf_bytes, err) ? __ldcs(&part[m * step]) : make_float2(0.f, 0.f);
      v[m] = make_float2(v[m].x + y.x, v[m].y + y.y);
    }
  }
  if (scale_tab && act) {
    const float* sc = scale_tab + (long long)t * ld + c;
#pragma unroll
    for (int m = 0; m < E; ++m)
      v[m] = cscale(v[m], ck(&sc[m * step], 4, scale_tab, buf_bytes / 2, err) ? __ldg(&sc[m * step]) : 0.0f);
  }
  line_fft<L, E, INV, kSyncBlock>(v, smem + cl * ColCfg<L>::BUF, t, tw);
  if (act) {
#pragma unroll
    for (int m = 0; m < E; ++m)
      if (ck(&col[m * step], 8, buf, buf_bytes, err)) col[m * step] = v[m];
  }
}

struct FwdColsArgs {
  const float2* F;          // image half spectrum [M][Hc]
  int Hc;
  const PlaneDesc* planes;
  const ColItem* items;     // items of this group (index 0 = first item of the group)
  int nitems;               // items of this group (set by the launchers)
  const int2* rng;
  float2* H;                // base of the group's intermediate
  WinParams w;
  const float2* tw;
  float* partials;          // per item sum |G| (low-precision storage), or null
  float gain;               // G = gain * psi_hat * F (folds the 1/(M N) of the inverse DFT)
  const CUtensorMap* tmaps; // per plane: tensor map of its slot (TMA panel stores), or null
  int odd;                  // one-sided shearlets, imaginary part: G = -i sign(omega) G (Sec. 3.8.2)
  long long F_bytes;        // extents from F and H (bounds checks of FFST_CHECK builds)
  long long H_bytes;
  int* err;                 // plan error word (FFST_CHECK builds)
};

// Forward column items per block (one: a block's work is one panel).
constexpr int kFwdItems = 1;

// Forward column pass of plane panels (Sec. 3.1 eq. shearletTransform):
// G = psi_hat_i * F on the panel's columns, then the column IFFT; the result
// goes to the plane's slot of the group intermediate, [M][W_i] starting at
// column c0_i.  Column cl of the panel belongs to the contiguous team of
// threads [cl T, (cl + 1) T), which synchronises alone (named barriers), so
// the P column FFTs of a block do not wait for one another.  Each thread
// evaluates the window and reads F at its own FFT rows t + T m that lie in
// the column's support (one cyclic row interval computed at plan time):
// the spectrum goes straight into the register layout of the FFT, without a
// shared-memory staging step.  With `partials` the block also writes sum |G|
// per item, each column counted once for itself and once for its conjugate
// partner (columns 0 and N/2 are their own partners); a plane's partials add
// up to sum_omega |G(omega)| >= max_m |c_i(m)| (G carries the 1/(M N) of the
// inverse DFT through `gain`).
template <int L>
__device__ __forceinline__ void fwd_cols_body(const FwdColsArgs& a, int blk, float2* smem) {
  constexpr int E = ColCfg<L>::E, T = ColCfg<L>::T, P = ColCfg<L>::P;
  constexpr int SYNC = T <= 32 ? kSyncWarp : (T < kThreads ? kSyncNamed : kSyncBlock);
  __shared__ float red[kThreads / 32];
  const int cl = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = smem + cl * ColCfg<L>::BUF;
  const int item = blk;  // kFwdItems == 1
  if (item >= a.nitems) return;  // uniform over the block
  const ColItem it = a.items[item];
  const PlaneDesc d = a.planes[it.plane];
  const int c = it.col + cl;
  const bool act = c >= d.c0 && c < d.c0 + d.W;
  const int2 rg = act ? a.rng[d.rng_off + (c - d.c0)] : make_int2(0, 0);
  float2 v[E];
  unsigned mask = 0;  // this thread's FFT rows inside the support
#pragma unroll
  for (int m = 0; m < E; ++m) {
    v[m] = make_float2(0.f, 0.f);
    if (in_range<L>(t + T * m, rg)) mask |= 1u << m;
  }
  float mag = 0.0f;
  for (unsigned rest = mask; rest; rest &= rest - 1) {  // one copy of the window code
    const int m = __ffs(rest) - 1;
    const int row = t + T * m;
    float psi = win_at(a.w, d, row, c);
    if (a.odd) psi *= (float)half_sign(a.w, d.kappa, row, c);
    const float2* fp = a.F + (long long)row * a.Hc + c;
    float2 g = cscale(ck(fp, 8, a.F, a.F_bytes, a.err) ? *fp : make_float2(0.f, 0.f), psi * a.gain);
    if (a.odd) g = make_float2(g.y, -g.x);  // -i g (the sign is in psi)
    if (a.partials) mag += sqrtf(g.x * g.x + g.y * g.y);
#pragma unroll
    for (int q = 0; q < E; ++q)
      if (q == m) v[q] = g;
  }
  if (a.partials) {  // fixed reduction order: deterministic
    const bool self_partner = (c == 0) || (2 * c == a.w.N);
    mag *= self_partner ? 1.0f : 2.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mag += __shfl_xor_sync(0xffffffffu, mag, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mag;
  }
  line_fft<L, E, true, SYNC>(v, buf, t, a.tw, 1 + cl);
  if (a.tmaps) {
    // the panel [L][P] through shared memory (aliasing the FFT buffers, which
    // every team has finished with at the block barrier) and one TMA store;
    // columns outside the support store zeros
    __syncthreads();
    float2* tile = smem;
#pragma unroll
    for (int m = 0; m < E; ++m) tile[(t + T * m) * P + cl] = act ? v[m] : make_float2(0.f, 0.f);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      if (a.partials) {
        float sum = 0.0f;
        for (int q = 0; q < kThreads / 32; ++q) sum += red[q];
        a.partials[item] = sum;
      }
      tma_store_panel(&a.tmaps[it.plane], tile, 2 * (it.col - d.c0al));
    }
    __syncthreads();  // the copy has read the panel before the buffers are reused
  } else {
    if (a.partials) {
      __syncthreads();
      if (threadIdx.x == 0) {
        float sum = 0.0f;
        for (int q = 0; q < kThreads / 32; ++q) sum += red[q];
        a.partials[item] = sum;
      }
    }
    if (act) {
      float2* out = a.H + d.off + (c - d.c0al);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        float2* o = &out[(long long)(t + T * m) * d.ldw];
        if (ck(o, 8, a.H, a.H_bytes, a.err)) __stcg(o, v[m]);
      }
    }
  }
}

struct InvColsArgs {
  const float2* H;          // base of the group's intermediate
  int Hc;
  const PlaneDesc* planes;
  int p0, p1;               // planes of the group
  const int2* rng;
  float2* S;                // nsplit partial accumulators [M][Hc] (zeroed before the first group)
  long long sstride;        // elements between partial accumulators
  int npanels;              // column panels
  int eta, nsplit;          // plane chunk k: planes [eta k / nsplit, eta (k + 1) / nsplit)
  int k0, nchunks;          // the chunks that meet [p0, p1)
  WinParams w;
  const float2* tw;
  const CUtensorMap* tmaps; // per plane: tensor map of its slot (TMA panel loads), or null
  int* err;                 // sticky error word (a TMA wait that ran out sets bit 2; FFST_CHECK: kErrBounds)
  long long H_bytes;        // extents from H and S (bounds checks of FFST_CHECK builds)
  long long S_bytes;
};

// Block bx of an inverse column launch (npanels x nchunks blocks): panel
// bx % npanels over the group's planes in chunk k = k0 + bx / npanels,
// summed into partial accumulator k.
__device__ __forceinline__ int inv_chunk(const InvColsArgs& a, int bx, int* q0, int* q1, float2** S) {
  const int j = bx / a.npanels, k = a.k0 + j;
  *q0 = max(a.p0, (int)((long long)a.eta * k / a.nsplit));
  *q1 = min(a.p1, (int)((long long)a.eta * (k + 1) / a.nsplit));
  *S = a.S + k * a.sstride;
  return bx - j * a.npanels;
}

// Inverse column pass (Sec. 3.3 eq. inverseShearletTransform): for every plane
// of [p0, p1) whose support meets panel bx, column FFT of the plane's row
// spectra, then S += psi_hat_i * (that) on the column's support rows (one
// cyclic interval).  Each block owns its columns of S and visits planes in
// index order, so the sums are deterministic.  S is read through L2: in the
// persistent schedule successive plane batches of a panel may run on
// different SMs.
//
// Software pipeline: the next plane's panel (TMA) or column loads are issued
// as soon as the current spectrum has left the shared buffers, so they fly
// during the accumulation; a thread's first accumulator element and its
// window value are fetched before the FFT.
template <int L>
__device__ __forceinline__ void inv_cols_body(const InvColsArgs& a, int bx, int p0, int p1, float2* S,
                                              float2* smem) {
  constexpr int E = ColCfg<L>::E, T = ColCfg<L>::T, P = ColCfg<L>::P;
  __shared__ uint64_t mbar;  // TMA panel loads
  const int t = threadIdx.x / P, cl = threadIdx.x % P;
  float2* buf = smem + cl * ColCfg<L>::BUF;
  const int cbase = bx * P;
  const int c = cbase + cl;
  const bool tma = a.tmaps != nullptr;
  // next plane at or after p whose support meets the panel (uniform over the block)
  auto next_plane = [&](int p) {
    for (; p < p1; ++p) {
      const int c0 = a.planes[p].c0, W = a.planes[p].W;
      if (W != 0 && c0 < cbase + P && c0 + W > cbase) break;
    }
    return p;
  };
  auto load_cols = [&](int p, float2 (&v)[E]) {
    const int c0 = a.planes[p].c0, W = a.planes[p].W, ldw = a.planes[p].ldw;
    const bool act = c >= c0 && c < c0 + W;
    const float2* in = a.H + a.planes[p].off + (c - a.planes[p].c0al);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float2* q = &in[(long long)(t + T * m) * ldw];
      v[m] = act && ck(q, 8, a.H, a.H_bytes, a.err) ? __ldcg(q) : make_float2(0.f, 0.f);
    }
  };
  // TMA: the panel [L][P] of plane p into shared memory (aliasing the FFT
  // buffers); x may be negative (leading columns read as zeros)
  auto issue_panel = [&](int p) {
    if (threadIdx.x == 0)
      tma_load_panel(&a.tmaps[p], smem, &mbar, 2 * (cbase - a.planes[p].c0al), (unsigned)(L * P * sizeof(float2)));
  };
  if (tma) {
    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
  }
  unsigned phase = 0;
  int p = next_plane(p0);
  float2 v[E];
  if (p < p1) {
    if (tma) issue_panel(p);
    else load_cols(p, v);
  }
  while (p < p1) {
    const PlaneDesc d = a.planes[p];
    const bool act = c >= d.c0 && c < d.c0 + d.W;
    const int2 rg = act ? a.rng[d.rng_off + (c - d.c0)] : make_int2(0, 0);
    if (tma) {
      // Rows t + T m of the support interval stay with the thread that holds
      // them after the FFT: it accumulates them from its registers, so the
      // shared buffers are free as soon as the FFT ends and the next plane's
      // panel load overlaps the accumulation.  A row always belongs to the
      // same thread, so the sums stay in plane order without a barrier.
      unsigned mask = 0;
#pragma unroll
      for (int m = 0; m < E; ++m)
        if (in_range<L>(t + T * m, rg)) mask |= 1u << m;
      const int m0 = mask ? __ffs(mask) - 1 : 0;
      const int row0 = t + T * m0;
      float2 s0 = make_float2(0.f, 0.f);
      float psi0 = 0.0f;
      if (mask) {  // first row's accumulator and window, ahead of the FFT
        const float2* sp0 = &S[(long long)row0 * a.Hc + c];
        s0 = ck(sp0, 8, a.S, a.S_bytes, a.err) ? __ldcg(sp0) : make_float2(0.f, 0.f);
        psi0 = win_at(a.w, d, row0, c);
      }
      if (!__syncthreads_and(mbar_wait(&mbar, phase, a.err))) return;
      phase ^= 1;
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = act ? smem[(t + T * m) * P + cl] : make_float2(0.f, 0.f);
      __syncthreads();  // panel read before the FFT reuses the buffers
      line_fft<L, E, false, kSyncBlock>(v, buf, t, a.tw);  // ends with a barrier after its last buffer read
      const int pn = next_plane(p + 1);
      if (pn < p1) issue_panel(pn);
      if (mask) {
        const float2 x = pick(v, m0);
        float2* sp0 = &S[(long long)row0 * a.Hc + c];
        if (ck(sp0, 8, a.S, a.S_bytes, a.err)) *sp0 = make_float2(fmaf(psi0, x.x, s0.x), fmaf(psi0, x.y, s0.y));
        for (unsigned rest = mask & (mask - 1); rest; rest &= rest - 1) {
          const int m = __ffs(rest) - 1;
          const int row = t + T * m;
          const float psi = win_at(a.w, d, row, c);
          const float2 y = pick(v, m);
          float2* sp = S + (long long)row * a.Hc + c;
          if (!ck(sp, 8, a.S, a.S_bytes, a.err)) continue;
          const float2 old = __ldcg(sp);
          *sp = make_float2(fmaf(psi, y.x, old.x), fmaf(psi, y.y, old.y));
        }
      }
      p = pn;
      continue;
    }
    // plain loads: the support rows go through the shared buffers to
    // consecutive threads while the next plane's column loads fly
    const bool first = t < rg.y;
    const int row0 = mod_l<L>(rg.x + t);
    float2 s0 = make_float2(0.f, 0.f);
    float psi0 = 0.0f;
    if (first) {
      const float2* sp0 = &S[(long long)row0 * a.Hc + c];
      s0 = ck(sp0, 8, a.S, a.S_bytes, a.err) ? __ldcg(sp0) : make_float2(0.f, 0.f);
      psi0 = win_at(a.w, d, row0, c);
    }
    line_fft<L, E, false, kSyncBlock>(v, buf, t, a.tw);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int row = t + T * m;
      if (in_range<L>(row, rg)) buf[spad<E>(row)] = v[m];
    }
    const int pn = next_plane(p + 1);
    if (pn < p1) load_cols(pn, v);
    __syncthreads();
    if (first) {
      const float2 x = buf[spad<E>(row0)];
      float2* sp0 = &S[(long long)row0 * a.Hc + c];
      if (ck(sp0, 8, a.S, a.S_bytes, a.err)) *sp0 = make_float2(fmaf(psi0, x.x, s0.x), fmaf(psi0, x.y, s0.y));
    }
    for (int q = t + T; q < rg.y; q += T) {
      const int row = mod_l<L>(rg.x + q);
      const float psi = win_at(a.w, d, row, c);
      const float2 x = buf[spad<E>(row)];
      float2* sp = S + (long long)row * a.Hc + c;
      if (!ck(sp, 8, a.S, a.S_bytes, a.err)) continue;
      const float2 old = __ldcg(sp);
      *sp = make_float2(fmaf(psi, x.x, old.x), fmaf(psi, x.y, old.y));
    }
    __syncthreads();  // buf reads and S writes done before the next plane
    p = pn;
  }
}

// Block b of a launch whose nc column blocks come first (they run longest).
__device__ __forceinline__ bool split_cols_first(int b, int nc, int* ci, int* ri) {
  if (b < nc) {
    *ci = b;
    return true;
  }
  *ri = b - nc;
  return false;
}

// ---------------------------------------------------------------------------
// launchers (ffst_rows.cu, ffst_cols.cu, ffst_fused.cu)
// ---------------------------------------------------------------------------
// `variant`: the row kernel variant (ffst_rows.cu; 0 = RowCfg<L>); Args.tw must
// be the pass table of that variant's elements per thread.
cudaError_t launch_rows_r2c(int L, const R2CArgs& a, int nplanes, cudaStream_t s, int variant = 0);
cudaError_t launch_rows_c2r(int L, const C2RArgs& a, int nplanes, cudaStream_t s, int variant = 0);
cudaError_t launch_cols_fft(int L, float2* buf, int width, int ld, bool inverse, const float* scale_tab,
                            const float2* tw, cudaStream_t s, int nsum, long long sstride, long long buf_bytes,
                            int* err);
cudaError_t launch_fwd_cols(int L, const FwdColsArgs& a, int nitems, cudaStream_t s);
cudaError_t launch_inv_cols(int L, const InvColsArgs& a, cudaStream_t s);  // a.npanels x a.nchunks blocks
// Fused launches exist for square power-of-two images with 256 <= M <= 4096
// (fused_supported); other sizes run the standalone kernels.
bool fused_supported(int M, int N);
// Persistent schedule (ffst_sched.cu): one launch for all plane passes of a
// forward (column items + row C2R) or an inverse (row R2C + column panels).
// The argument structs are completed inside (ring, descriptors, items).
cudaError_t launch_fwd_sched(const ffst_plan_s* p, FwdColsArgs ca, C2RArgs ra, float target, float* scale_out,
                             cudaStream_t st);
cudaError_t launch_inv_sched(const ffst_plan_s* p, R2CArgs ra, InvColsArgs ca, cudaStream_t st);
cudaError_t launch_fwd_fused(int M, const FwdColsArgs& ca, int nitems, const C2RArgs& ra, int nplanes,
                             cudaStream_t s);
cudaError_t launch_inv_fused(int M, const R2CArgs& ra, int nplanes, const InvColsArgs& ca, cudaStream_t s);

}  // namespace ffst
