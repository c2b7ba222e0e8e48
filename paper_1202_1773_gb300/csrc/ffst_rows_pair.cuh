// Row C2R pass on two rows per team with packed FP32 pairs.
//
// Same result contract as rows_c2r_body (ffst_kernels.cuh): for every row of
// the block, the half-spectrum row X[0..N/2] (nonzero only on the plane's
// support columns) becomes the real row x = IDFT_N(X) (times the scale and
// plane factor), stored once.  A team of T = L/16 threads transforms rows A
// = 2p and B = 2p + 1 together: the Hermitian pre-processing, the length-L
// line IFFT and the scaling run as packed two-lane instructions
// (ffst_fft_pair.cuh), which halves the floating-point instruction count of
// the pass; loads, stores and the epilogue stay per row.  A block of
// kThreads threads holds TEAMS = kThreads/T teams, 2 TEAMS rows.
#pragma once

#include "ffst_fft_pair.cuh"
#include "ffst_kernels.cuh"

namespace ffst {

template <int L>
struct RowPairCfg {
  static_assert(is_pow2c(L) && L >= 256 && L <= 2048, "paired rows: power-of-two half lengths 256..2048");
  static constexpr int E = 16;
  static constexpr int T = L / E;
  static constexpr int TEAMS = kThreads / T;  // row pairs per block
  static constexpr int ROWS = 2 * TEAMS;
  static constexpr int SYNC = T <= 32 ? kSyncWarp : (T < kThreads ? kSyncNamed : kSyncBlock);
  static constexpr int BUF = team_stride(L, E, 0);  // 16-byte slots per team
  static constexpr size_t SMEM = sizeof(float4) * TEAMS * BUF;
  static_assert(TEAMS * T == kThreads, "row teams must fill the block");
  static_assert(TEAMS % 2 == 0, "the statistics halves need an even team count");
};

// Rows of a paired block: 2 RowPairCfg::TEAMS, i.e. twice those of the
// one-row block of the same length; the statistics partials keep the
// one-row block's granularity (two per paired block).
template <int L>
__device__ __forceinline__ void rows_c2r_pair_body(const C2RArgs& a, int bx, int by, float4* smem, float ps) {
  using C = RowPairCfg<L>;
  constexpr int E = C::E, T = C::T, N = 2 * L;
  const int team = threadIdx.x / T, t = threadIdx.x % T;
  float4* buf = smem + team * C::BUF;
  const int plane = a.plane0 + by;
  const int rowA = bx * C::ROWS + 2 * team;
  const bool act = rowA < a.M;
  const bool actB = rowA + 1 < a.M;  // odd M: the last pair has no row B (zeros in, nothing stored)
  int c0 = a.c0, W = a.W, ld = a.ld;
  const float2* src = a.src;
  if (a.planes) {  // the plane's slot: pitch ldw, column c at c - c0al
    const PlaneDesc d = a.planes[plane];
    c0 = d.c0;
    W = d.W;
    ld = d.ldw;
    src = a.src + d.off + (d.c0 - d.c0al);
  }
  const float2* sA = src + (long long)rowA * ld;
  const float2* sB = sA + ld;
  const float s = a.scale * ps;
  const float2 wt = __ldg(&a.rtw[t]);
  P2 v[E];
  static_for<0, E>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    const int k = t + T * m;
    const int ia = k - c0, ib = L - k - c0;
    const bool ina = (unsigned)ia < (unsigned)W, inb = (unsigned)ib < (unsigned)W;
    const float2 z = make_float2(0.f, 0.f);
    const void* b0 = a.src;
    float2 aA = act && ina && ck(&sA[ia], 8, b0, a.src_bytes, a.err) ? __ldcg(&sA[ia]) : z;
    float2 aB = actB && ina && ck(&sB[ia], 8, b0, a.src_bytes, a.err) ? __ldcg(&sB[ia]) : z;
    float2 bA = act && inb && ck(&sA[ib], 8, b0, a.src_bytes, a.err) ? __ldcg(&sA[ib]) : z;
    float2 bB = actB && inb && ck(&sB[ib], 8, b0, a.src_bytes, a.err) ? __ldcg(&sB[ib]) : z;
    if (m == 0 && t == 0) {  // X[0] and X[N/2]: Hermitian part is real
      aA.y = aB.y = bA.y = bB.y = 0.f;
    }
    const P2 xa{make_float2(aA.x, aB.x), make_float2(aA.y, aB.y)};
    const P2 xb{make_float2(bA.x, bB.x), make_float2(bA.y, bB.y)};
    // e = X[k] + conj X[L-k];  d = (X[k] - conj X[L-k]) conj(W_N^k), W_N^k = W_N^t W_{2E}^m
    const P2 e{padd(xa.re, xb.re), psub(xa.im, xb.im)};
    const P2 d0 = p2twiddle_c<2 * E, m, true>(P2{psub(xa.re, xb.re), padd(xa.im, xb.im)});
    const P2 wd = p2rot(d0, wt.x, -wt.y);
    // Z[k] = e + i wd
    v[m] = P2{psub(e.re, wd.im), padd(e.im, wd.re)};
  });
  if (s != 1.0f) {  // linear transform: scale before it
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = P2{pmul(v[m].re, bc2(s)), pmul(v[m].im, bc2(s))};
  }
  p2line_fft<L, E, true, C::SYNC>(v, buf, t, a.tw, 1 + team);
  if (a.shrink || a.abs_partials) {  // uniform over the launch
    // v holds c * ps: threshold and statistics act on c (ps is a power of two)
    __shared__ float red[kThreads / 32];
    const float tau = a.shrink ? __ldg(&a.thresh[plane]) * ps : 0.0f;
    float acc = 0.0f;
    if (act) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        float q[4] = {v[m].re.x, v[m].re.y, v[m].im.x, v[m].im.y};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc += fabsf(q[u]);
          if (a.shrink == 1) q[u] = copysignf(fmaxf(fabsf(q[u]) - tau, 0.0f), q[u]);
          else if (a.shrink == 2) q[u] = fabsf(q[u]) > tau ? q[u] : 0.0f;
        }
        v[m] = P2{make_float2(q[0], q[1]), make_float2(q[2], q[3])};
      }
    }
    if (a.abs_partials) {  // fixed reduction order: deterministic; one partial per half block
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x < 2) {
        constexpr int half = kThreads / 64;  // warps per half block
        float sum = 0.0f;
        for (int q = 0; q < half; ++q) sum += red[threadIdx.x * half + q];
        a.abs_partials[(long long)plane * a.rbx + 2 * bx + threadIdx.x] = sum / ps;
      }
    }
  }
  if (!act) return;
  void* dst = static_cast<char*>(a.dst) + (long long)by * a.dst_plane_stride * stor_bytes(a.st);
  const long long rA = (long long)rowA * N + 2 * t, rB = rA + N;
  if (a.st == FFST_STORE_F32) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      store_pair_ck(dst, rA + 2 * T * m, v[m].re.x, v[m].im.x, FFST_STORE_F32, a.dst, a.dst_bytes, a.err);
      if (actB)
        store_pair_ck(dst, rB + 2 * T * m, v[m].re.y, v[m].im.y, FFST_STORE_F32, a.dst, a.dst_bytes, a.err);
    }
  } else if (a.st == FFST_STORE_F16) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      store_pair_ck(dst, rA + 2 * T * m, v[m].re.x, v[m].im.x, FFST_STORE_F16, a.dst, a.dst_bytes, a.err);
      if (actB)
        store_pair_ck(dst, rB + 2 * T * m, v[m].re.y, v[m].im.y, FFST_STORE_F16, a.dst, a.dst_bytes, a.err);
    }
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      store_pair_ck(dst, rA + 2 * T * m, v[m].re.x, v[m].im.x, FFST_STORE_BF16, a.dst, a.dst_bytes, a.err);
      if (actB)
        store_pair_ck(dst, rB + 2 * T * m, v[m].re.y, v[m].im.y, FFST_STORE_BF16, a.dst, a.dst_bytes, a.err);
    }
  }
}

}  // namespace ffst
