// Self-written FFT engine: radix-R DFTs in registers and a register-resident
// Stockham line FFT whose passes exchange data through shared memory.
//
// Layout contract of a line FFT of length L run by a team of T = L/E
// threads: thread t holds v[m] = x[t + T*m], m = 0..E-1, on entry (natural
// order input) and v[m] = X[t + T*m] on exit (natural order output).
// Consecutive threads therefore touch consecutive elements, so the loads
// before and the stores after the transform are coalesced.
//
// Pass s (radix R = min(E, L/Ns), Ns = product of the earlier radices)
// computes, for every butterfly index j in [0, L/R), the R-point DFT of
// x[j + r*L/R] after the twiddles W_{Ns R}^{(j mod Ns) r}, and scatters the
// results to y[(j/Ns) Ns R + (j mod Ns) + r Ns] (the Stockham auto-sort of
// the FFT literature); the last pass lands exactly in the register layout.
//
// Twiddle table of a (L, E) line: pass s reads W_{Ns R}^{kk r} at index
// (Ns - 1) + (r - 1) Ns + kk, so consecutive butterflies (consecutive kk)
// read consecutive addresses; the passes together use L - 1 entries.
#pragma once

#include <type_traits>

#include "ffst_internal.cuh"

namespace ffst {

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// x * W_R^m with W_R = exp(-2 pi i / R) (forward) or its conjugate (inverse).
// Multiples of pi/4 are special-cased so no multiply by 0 or 1 is emitted.
template <int R, int m, bool INV>
__device__ __forceinline__ float2 twiddle_c(float2 x) {
  constexpr int mm = ((m % R) + R) % R;
  if constexpr (mm == 0) {
    return x;
  } else if constexpr ((8 * mm) % R == 0) {
    constexpr int o0 = (8 * mm) / R;
    constexpr int oct = INV ? (8 - o0) % 8 : o0;  // multiply by exp(-i oct pi/4)
    constexpr float s = 0.70710678118654752440f;
    if constexpr (oct == 1) return make_float2((x.x + x.y) * s, (x.y - x.x) * s);
    else if constexpr (oct == 2) return make_float2(x.y, -x.x);
    else if constexpr (oct == 3) return make_float2((x.y - x.x) * s, -(x.x + x.y) * s);
    else if constexpr (oct == 4) return make_float2(-x.x, -x.y);
    else if constexpr (oct == 5) return make_float2(-(x.x + x.y) * s, (x.x - x.y) * s);
    else if constexpr (oct == 6) return make_float2(-x.y, x.x);
    else return make_float2((x.x - x.y) * s, (x.x + x.y) * s);
  } else {
    constexpr float c = root_cos(mm, R);
    constexpr float sn = INV ? root_sin(mm, R) : -root_sin(mm, R);
    return make_float2(x.x * c - x.y * sn, x.x * sn + x.y * c);
  }
}

// In-place R-point DFT of x (natural order in and out), R in {1,2,4,8,16,32,64}
// and the odd radices 3, 5, 7.
// R = R1*R2: R1 interleaved DFTs of length R2, twiddles W_R^{n1 k2}, then R2
// DFTs of length R1 (X[k2 + R2 k1]).
template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&x)[R]) {
  if constexpr (R == 1) {
  } else if constexpr (R == 3 || R == 5 || R == 7) {
    // odd radices of mixed-radix lines: the DFT sum with constant roots
    float2 y[R];
    static_for<0, R>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      float2 acc = x[0];
      static_for<1, R>([&](auto nc) {
        constexpr int n = decltype(nc)::value;
        acc = cadd(acc, twiddle_c<R, n * k, INV>(x[n]));
      });
      y[k] = acc;
    });
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = y[k];
  } else if constexpr (R == 2) {
    const float2 a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const float2 t0 = cadd(x[0], x[2]), t1 = csub(x[0], x[2]);
    const float2 t2 = cadd(x[1], x[3]), t3 = csub(x[1], x[3]);
    x[0] = cadd(t0, t2);
    x[2] = csub(t0, t2);
    // t1 -/+ i t3 (forward / inverse), componentwise: the swapped pair never
    // has to be formed
    if constexpr (INV) {
      x[1] = make_float2(t1.x - t3.y, t1.y + t3.x);
      x[3] = make_float2(t1.x + t3.y, t1.y - t3.x);
    } else {
      x[1] = make_float2(t1.x + t3.y, t1.y - t3.x);
      x[3] = make_float2(t1.x - t3.y, t1.y + t3.x);
    }
  } else {
    constexpr int R1 = (R == 8) ? 2 : ((R == 16 || R == 32) ? 4 : 8);
    constexpr int R2 = R / R1;
    float2 y[R1][R2];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) y[n1][n2] = x[n1 + R1 * n2];
      dft<R2, INV>(y[n1]);
    }
    static_for<1, R1>([&](auto n1c) {
      static_for<1, R2>([&](auto k2c) {
        constexpr int n1 = decltype(n1c)::value, k2 = decltype(k2c)::value;
        y[n1][k2] = twiddle_c<R, n1 * k2, INV>(y[n1][k2]);
      });
    });
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      float2 z[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) z[n1] = y[n1][k2];
      dft<R1, INV>(z);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) x[k2 + R2 * k1] = z[k1];
    }
  }
}

// Shared-memory slot of element i of a team buffer: one pad slot per E
// elements keeps the pass-1 scatter (stride E) free of bank conflicts.
template <int E>
__device__ __forceinline__ int spad(int i) {
  return i + (i >> ilog2c(E));
}

// Register layout <-> team buffer: thread t's element m is x[t + T*m].  When
// T is a multiple of E the pad term splits, spad(t + T m) = spad(t) +
// m (T + T/E), so one address serves all E slots.
template <int E, int T>
__device__ __forceinline__ void team_store(float2* buf, int t, const float2 (&v)[E]) {
  if constexpr (T % E == 0) {
    float2* p = buf + spad<E>(t);
#pragma unroll
    for (int m = 0; m < E; ++m) p[m * (T + T / E)] = v[m];
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) buf[spad<E>(t + T * m)] = v[m];
  }
}

template <int E, int T>
__device__ __forceinline__ void team_load(const float2* buf, int t, float2 (&v)[E]) {
  if constexpr (T % E == 0) {
    const float2* p = buf + spad<E>(t);
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = p[m * (T + T / E)];
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = buf[spad<E>(t + T * m)];
  }
}

// float2 slots per team buffer for a line of length L with E per thread,
// rounded so that (stride mod 16) == skew; consecutive team buffers then
// start on different banks (skew chosen by the kernel's lane layout).
__host__ __device__ constexpr int team_stride(int L, int E, int skew) {
  const int base = is_pow2c(L) ? L + L / E : 2 * L;
  return base + ((skew - base % 16) % 16 + 16) % 16;
}

// Sync policy of a team's shared-memory exchange.
//  kSyncWarp:  the team is <= 32 consecutive threads inside one warp.
//  kSyncNamed: the team is a run of whole consecutive warps (NT threads);
//              it uses hardware barrier `bar` (1..15), other teams do not wait.
//  kSyncBlock: teams interleaved across warps (or filling the block): the
//              whole block synchronises and must run the same passes.
enum { kSyncWarp = 0, kSyncNamed = 1, kSyncBlock = 2 };

template <int SYNC, int NT>
__device__ __forceinline__ void team_sync(int bar) {
  if constexpr (SYNC == kSyncWarp) {
    __syncwarp();
  } else if constexpr (SYNC == kSyncNamed) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(NT) : "memory");
  } else {
    __syncthreads();
  }
}

// x[r] *= w^r, r = 1..R-1, for the butterfly twiddle w = W_{Ns R}^kk whose
// powers sit in the pass table at p[(r - 1) Ns].  Only w and w^4 are read;
// w^r = (w^4)^a w^b (r = 4a + b) is formed with at most R/4 + 1 products,
// which keeps the twiddles off the L1 pipe (the busiest unit of the row and
// column kernels) at a few ulps of extra error: 2048x2048 J=5 inverse
// 1.30 -> 1.25 ms against reading all R - 1 entries.
template <int R, bool INV>
__device__ __forceinline__ void pass_twiddles(float2 (&x)[R], const float2* __restrict__ p, int Ns) {
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
    if constexpr (a == 0) x[r] = cmul(x[r], wb);
    else if constexpr (b == 0) x[r] = cmul(x[r], wa);
    else x[r] = cmul(cmul(x[r], wb), wa);
  });
}

// Stockham passes starting at sub-transform length Ns.  `tw` is the (L, E)
// pass table (FP64-generated, rounded to FP32), conjugated for INV.
template <int L, int E, bool INV, int Ns, int SYNC>
__device__ __forceinline__ void stockham(float2 (&v)[E], float2* buf, int t, const float2* __restrict__ tw, int bar) {
  constexpr int T = L / E;
  constexpr int REM = L / Ns;
  constexpr int R = REM >= E ? E : REM;
  constexpr int B = E / R;  // butterflies per thread in this pass
  static_assert(E % R == 0, "radix must divide the elements per thread");
#pragma unroll
  for (int q = 0; q < B; ++q) {
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[q + B * r];
    const int j = t + T * q;
    const int kk = j & (Ns - 1);
    if constexpr (Ns > 1) {
      pass_twiddles<R, INV>(x, tw + (Ns - 1) + kk, Ns);
    }
    dft<R, INV>(x);
    if constexpr (Ns * R == L) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q + B * r] = x[r];
    } else {
      // Ns is 1 (then base is a multiple of R = E) or a multiple of E, so the
      // pad term of base + r Ns splits and the R slots sit at fixed offsets
      static_assert(Ns == 1 ? R == E : Ns % E == 0, "pass start must be 1 (radix E) or a multiple of E");
      constexpr int kStep = Ns == 1 ? 1 : Ns + Ns / E;
      float2* dst = buf + spad<E>((j / Ns) * Ns * R + kk);
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * kStep] = x[r];
    }
  }
  if constexpr (Ns * R < L) {
    team_sync<SYNC, T>(bar);
    team_load<E, T>(buf, t, v);
    team_sync<SYNC, T>(bar);
    stockham<L, E, INV, Ns * R, SYNC>(v, buf, t, tw, bar);
  }
}

// Register array of one lane rotated left by a lane-dependent amount s in
// [0, 32): u[i] <- u[(i + s) mod 32], as five conditional rotations by
// 1, 2, 4, 8, 16 (selects on the bits of s; no local memory).
__device__ __forceinline__ void rotate_regs32(float2 (&u)[32], int s) {
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    const bool on = (s >> b) & 1;
    constexpr int kHead = 16;
    const int d = 1 << b;
    float2 head[kHead];  // u[0, d) before it is overwritten
#pragma unroll
    for (int i = 0; i < kHead; ++i)
      if (i < d) head[i] = u[i];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const float2 src = (i + d < 32) ? u[i + d] : head[(i + d - 32) % kHead];
      u[i] = on ? src : u[i];
    }
  }
}

// Transpose of a warp's 32 x 32 register tile by warp shuffles: register r
// of lane l moves to register l of lane r.  Lane l first rotates its
// registers by l, so that shuffle k can take the same register k from every
// lane (source lane l - k delivers its element for lane l); the received
// elements arrive in the order of their source lanes reversed and rotated by
// l, which the second rotation undoes.  64 shuffles and about 640 selects
// per lane, against 32 stores and 32 loads through shared memory.
__device__ __forceinline__ void warp_transpose32(float2 (&v)[32], int lane) {
  rotate_regs32(v, lane);  // v[i] = a[lane][(i + lane) mod 32]
  float2 z[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int src = (lane - i) & 31;  // src's register i holds a[src][lane]
    z[(32 - i) & 31] = make_float2(__shfl_sync(0xffffffffu, v[i].x, src), __shfl_sync(0xffffffffu, v[i].y, src));
  }
  // z[j] = a[(lane + j) mod 32][lane]; wanted v[s] = a[s][lane] = z[(s - lane) mod 32]
  rotate_regs32(z, (32 - lane) & 31);
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = z[i];
}

// A 1024-point line run by one warp with 32 elements per lane (the layout
// contract above with T = E = 32) whose one exchange is warp_transpose32
// instead of shared memory: the same two radix-32 passes, twiddles and
// results as stockham<1024, 32>.
template <bool INV>
__device__ __forceinline__ void line_fft_shfl1024(float2 (&v)[32], int t, const float2* __restrict__ tw) {
  dft<32, INV>(v);                               // pass 1 (Ns = 1): y[32 t + r] = v[r]
  warp_transpose32(v, t);                        // v[r] = y[t + 32 r]
  pass_twiddles<32, INV>(v, tw + 31 + t, 32);    // pass 2 (Ns = 32, kk = t)
  dft<32, INV>(v);                               // v[r] = X[t + 32 r]
}

// Mixed-radix lines (L not a power of two): the same Stockham passes, with
// the data in shared memory between all passes (ping-pong between buf[0, L)
// and buf[L, 2L)); NT threads share each pass's butterflies.
template <int L, int E, bool INV, int Ns, int SYNC, int NT>
__device__ __forceinline__ void mixed_passes(float2* a, float2* b, int t, const float2* __restrict__ tw, int bar) {
  if constexpr (Ns < L) {
    constexpr int R = next_radix(L, E, Ns);
    constexpr int NB = L / R;
    for (int j = t; j < NB; j += NT) {
      float2 x[R];
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = a[j + r * NB];
      const int kk = j % Ns;
      if constexpr (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = __ldg(&tw[(Ns - 1) + (r - 1) * Ns + kk]);
          if (INV) w.y = -w.y;
          x[r] = cmul(x[r], w);
        }
      }
      dft<R, INV>(x);
      const int base = (j / Ns) * Ns * R + kk;
#pragma unroll
      for (int r = 0; r < R; ++r) b[base + r * Ns] = x[r];
    }
    team_sync<SYNC, NT>(bar);
    mixed_passes<L, E, INV, Ns * R, SYNC, NT>(b, a, t, tw, bar);
  }
}

// Full line FFT (unnormalised).  Forward: X[k] = sum x[n] e^{-2 pi i nk/L};
// inverse: the same with e^{+2 pi i nk/L}.  Mixed-radix lines need a team
// buffer of 2L slots.
template <int L, int E, bool INV, int SYNC>
__device__ __forceinline__ void line_fft(float2 (&v)[E], float2* buf, int t, const float2* __restrict__ tw,
                                         int bar = 0) {
  if constexpr (is_pow2c(L)) {
    stockham<L, E, INV, 1, SYNC>(v, buf, t, tw, bar);
  } else {
    constexpr int T = L / E;
#pragma unroll
    for (int m = 0; m < E; ++m) buf[t + T * m] = v[m];
    team_sync<SYNC, T>(bar);
    mixed_passes<L, E, INV, 1, SYNC, T>(buf, buf + L, t, tw, bar);
    const float2* res = (num_passes(L, E) % 2 == 0) ? buf : buf + L;
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = res[t + T * m];
    team_sync<SYNC, T>(bar);
  }
}

// i mod L for i in [-L, 2L)
template <int L>
__device__ __forceinline__ int mod_l(int i) {
  if constexpr (is_pow2c(L)) return i & (L - 1);
  else return i < 0 ? i + L : (i >= L ? i - L : i);
}

}  // namespace ffst
