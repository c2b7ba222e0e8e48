// Line FFTs on two lines at once with packed FP32 pairs.
//
// A thread transforms the same elements of two lines A and B in lockstep.
// Each complex pair is held split by part, P2{re = (Re a, Re b), im = (Im a,
// Im b)}, so every add, multiply and fused multiply-add of the butterflies
// is one packed two-lane FP32 instruction (add/mul/fma .f32x2) serving both
// lines: the arithmetic and the shared-memory exchanges take half the
// instructions of a one-line-per-thread FFT, with identical per-line
// results for the same operation order.
//
// Layout contract (as the one-line engine of ffst_fft.cuh): a line of length
// L is run by T = L/E threads; thread t holds v[m] = (x_A, x_B)[t + T m] on
// entry and X[t + T m] on exit.  Pass s (radix R = min(E, L/Ns)) takes the
// R-point DFT of x[j + r L/R] after the twiddles W_{Ns R}^{(j mod Ns) r}
// and scatters to y[(j/Ns) Ns R + (j mod Ns) + r Ns] (Stockham auto-sort);
// the exchange between passes goes through one 16-byte shared slot per
// element pair, (Re a, Re b, Im a, Im b).
#pragma once

#include "ffst_fft.cuh"

namespace ffst {

struct P2 {
  float2 re;  // (Re of line A, Re of line B)
  float2 im;  // (Im of line A, Im of line B)
};

__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }

// Packed FP32 arithmetic on (line A, line B) lanes.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, bc2(-1.0f), a); }  // exact a - b
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ P2 p2add(P2 a, P2 b) { return P2{padd(a.re, b.re), padd(a.im, b.im)}; }
__device__ __forceinline__ P2 p2sub(P2 a, P2 b) { return P2{psub(a.re, b.re), psub(a.im, b.im)}; }

// x * (c + i s) for the same root on both lines.
__device__ __forceinline__ P2 p2rot(P2 x, float c, float s) {
  return P2{pfma(x.re, bc2(c), pmul(x.im, bc2(-s))), pfma(x.re, bc2(s), pmul(x.im, bc2(c)))};
}

// x * W_R^m (W_R = exp(-2 pi i / R), conjugated for INV), a compile-time root;
// multiples of pi/4 special-cased.
template <int R, int m, bool INV>
__device__ __forceinline__ P2 p2twiddle_c(P2 x) {
  constexpr int mm = ((m % R) + R) % R;
  if constexpr (mm == 0) {
    return x;
  } else if constexpr ((8 * mm) % R == 0) {
    constexpr int o0 = (8 * mm) / R;
    constexpr int oct = INV ? (8 - o0) % 8 : o0;  // multiply by exp(-i oct pi/4)
    constexpr float s = 0.70710678118654752440f;
    if constexpr (oct == 1) return P2{pmul(padd(x.re, x.im), bc2(s)), pmul(psub(x.im, x.re), bc2(s))};
    else if constexpr (oct == 2) return P2{x.im, pmul(x.re, bc2(-1.0f))};
    else if constexpr (oct == 3) return P2{pmul(psub(x.im, x.re), bc2(s)), pmul(padd(x.re, x.im), bc2(-s))};
    else if constexpr (oct == 4) return P2{pmul(x.re, bc2(-1.0f)), pmul(x.im, bc2(-1.0f))};
    else if constexpr (oct == 5) return P2{pmul(padd(x.re, x.im), bc2(-s)), pmul(psub(x.re, x.im), bc2(s))};
    else if constexpr (oct == 6) return P2{pmul(x.im, bc2(-1.0f)), x.re};
    else return P2{pmul(psub(x.re, x.im), bc2(s)), pmul(padd(x.re, x.im), bc2(s))};
  } else {
    constexpr float c = root_cos(mm, R);
    constexpr float sn = INV ? root_sin(mm, R) : -root_sin(mm, R);
    return p2rot(x, c, sn);
  }
}

// In-place R-point DFT (natural order in and out), R in {1, 2, 4, 8, 16}.
// Same decomposition as dft<R> of ffst_fft.cuh: R = R1 R2, R1 interleaved
// DFTs of length R2, twiddles W_R^{n1 k2}, then R2 DFTs of length R1.  The
// factors -i / +i of the radix-4 butterflies are folded into the adds.
template <int R, bool INV>
__device__ __forceinline__ void p2dft(P2 (&x)[R]) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    const P2 a = x[0], b = x[1];
    x[0] = p2add(a, b);
    x[1] = p2sub(a, b);
  } else if constexpr (R == 4) {
    const P2 t0 = p2add(x[0], x[2]), t1 = p2sub(x[0], x[2]);
    const P2 t2 = p2add(x[1], x[3]), t3 = p2sub(x[1], x[3]);
    x[0] = p2add(t0, t2);
    x[2] = p2sub(t0, t2);
    // forward: t1 -/+ i t3 -> X1 = t1 - i t3, X3 = t1 + i t3; inverse swaps them
    const P2 a{padd(t1.re, t3.im), psub(t1.im, t3.re)};  // t1 - i t3
    const P2 b{psub(t1.re, t3.im), padd(t1.im, t3.re)};  // t1 + i t3
    x[1] = INV ? b : a;
    x[3] = INV ? a : b;
  } else {
    constexpr int R1 = (R == 8) ? 2 : 4;
    constexpr int R2 = R / R1;
    P2 y[R1][R2];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) y[n1][n2] = x[n1 + R1 * n2];
      p2dft<R2, INV>(y[n1]);
    }
    static_for<1, R1>([&](auto n1c) {
      static_for<1, R2>([&](auto k2c) {
        constexpr int n1 = decltype(n1c)::value, k2 = decltype(k2c)::value;
        y[n1][k2] = p2twiddle_c<R, n1 * k2, INV>(y[n1][k2]);
      });
    });
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      P2 z[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) z[n1] = y[n1][k2];
      p2dft<R1, INV>(z);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) x[k2 + R2 * k1] = z[k1];
    }
  }
}

// x[r] *= w^r (r = 1..R-1) for the butterfly twiddle w = W_{Ns R}^kk, read
// from the pass table at p[(r - 1) Ns] as in pass_twiddles (ffst_fft.cuh):
// w and w^4 are read, the other powers formed in FP32 (scalar, shared by both
// lines), each applied to both lines with packed products.
template <int R, bool INV>
__device__ __forceinline__ void p2pass_twiddles(P2 (&x)[R], const float2* __restrict__ p, int Ns) {
  float2 w1 = __ldg(p);
  if (INV) w1.y = -w1.y;
  const float2 w2 = cmul(w1, w1);
  const float2 w3 = cmul(w2, w1);
  float2 w4 = make_float2(1.f, 0.f);
  if constexpr (R > 4) {
    w4 = __ldg(p + 3 * Ns);
    if (INV) w4.y = -w4.y;
  }
  float2 wa = make_float2(1.f, 0.f);  // (w^4)^a
  static_for<1, R>([&](auto rc) {
    constexpr int r = decltype(rc)::value, a = r / 4, b = r % 4;
    if constexpr (b == 0) wa = (a == 1) ? w4 : cmul(wa, w4);
    const float2 wb = b == 1 ? w1 : (b == 2 ? w2 : w3);
    const float2 w = a == 0 ? wb : (b == 0 ? wa : cmul(wb, wa));
    x[r] = p2rot(x[r], w.x, w.y);
  });
}

__device__ __forceinline__ float4 p2pack(P2 v) { return make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }
__device__ __forceinline__ P2 p2unpack(float4 q) { return P2{make_float2(q.x, q.y), make_float2(q.z, q.w)}; }

// Register layout <-> team buffer of 16-byte slots (pad scheme of spad<E>).
template <int E, int T>
__device__ __forceinline__ void p2team_store(float4* buf, int t, const P2 (&v)[E]) {
  static_assert(T % E == 0, "paired lines need T a multiple of E");
  float4* p = buf + spad<E>(t);
#pragma unroll
  for (int m = 0; m < E; ++m) p[m * (T + T / E)] = p2pack(v[m]);
}

template <int E, int T>
__device__ __forceinline__ void p2team_load(const float4* buf, int t, P2 (&v)[E]) {
  static_assert(T % E == 0, "paired lines need T a multiple of E");
  const float4* p = buf + spad<E>(t);
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = p2unpack(p[m * (T + T / E)]);
}

// Stockham passes from sub-transform length Ns (powers of two).
template <int L, int E, bool INV, int Ns, int SYNC>
__device__ __forceinline__ void p2stockham(P2 (&v)[E], float4* buf, int t, const float2* __restrict__ tw, int bar) {
  constexpr int T = L / E;
  constexpr int REM = L / Ns;
  constexpr int R = REM >= E ? E : REM;
  constexpr int B = E / R;
  static_assert(E % R == 0, "radix must divide the elements per thread");
#pragma unroll
  for (int q = 0; q < B; ++q) {
    P2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[q + B * r];
    const int j = t + T * q;
    const int kk = j & (Ns - 1);
    if constexpr (Ns > 1) p2pass_twiddles<R, INV>(x, tw + (Ns - 1) + kk, Ns);
    p2dft<R, INV>(x);
    if constexpr (Ns * R == L) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q + B * r] = x[r];
    } else {
      static_assert(Ns == 1 ? R == E : Ns % E == 0, "pass start must be 1 (radix E) or a multiple of E");
      constexpr int kStep = Ns == 1 ? 1 : Ns + Ns / E;
      float4* dst = buf + spad<E>((j / Ns) * Ns * R + kk);
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * kStep] = p2pack(x[r]);
    }
  }
  if constexpr (Ns * R < L) {
    team_sync<SYNC, T>(bar);
    p2team_load<E, T>(buf, t, v);
    team_sync<SYNC, T>(bar);
    p2stockham<L, E, INV, Ns * R, SYNC>(v, buf, t, tw, bar);
  }
}

// Full paired line FFT (unnormalised), powers of two.  Team buffer: 16-byte
// slots, team_stride(L, E, skew) of them.
template <int L, int E, bool INV, int SYNC>
__device__ __forceinline__ void p2line_fft(P2 (&v)[E], float4* buf, int t, const float2* __restrict__ tw, int bar = 0) {
  static_assert(is_pow2c(L), "paired lines: powers of two");
  p2stockham<L, E, INV, 1, SYNC>(v, buf, t, tw, bar);
}

}  // namespace ffst
