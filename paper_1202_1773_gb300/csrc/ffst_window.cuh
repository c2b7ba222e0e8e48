// In-register generator of the shearlet spectra psi_hat_i (FP32).
//
// Definitions (arXiv:1202.1773):
//   v          Sec. 2.1 eq. (v)      polynomial piece p(x) = x^4 (35 - 84x + 70x^2 - 20x^3)
//   smooth     Sec. 3.4 eqs. (newPsi1), (smoothPsi) and Sec. 2.4 eq. (Phi): a
//              2-D radial factor for both cones, tensor low-pass
//   psi2_hat   Sec. 2.1 eq. (Psi2)   sqrt(v(1 - |u|)), zero for |u| >= 1
//   psi1_hat   Sec. 2.1 eq. (Psi1)   per-scale 1-D table, FP64-generated on the host
//   varphi     Sec. 2.4              1-D table, FP64-generated on the host
//   cones      Sec. 2.3              exact integer test on the frequency indices
//   spectra    Sec. 3.1 eq. (shearletTransform), glued seam shearlets for |k| = 2^j
//   grid       Sec. 3.5.1            xi = omega * X / g, X = 2^{2 j0 - 1}, one step
//                                    (g = floor(max(M, N)/2)) or per axis (g = floor(L/2))
//   fix        Sec. 3.8.1            Nyquist row/column mirrored, squares averaged
//
// Accuracy notes.  The shear argument u = 2^j xi2/xi1 + k (h cone) is formed
// as one fraction of exact integers, (2^j o2 gn + k o1 gm) / (o1 gm) with the
// grid denominators gm, gn, so the cancellation against k happens exactly and u has
// FP32 relative accuracy on the support |u| < 1.  v near 1 is evaluated as
// 1 - p(1 - x) (the symmetry v(x) + v(1-x) = 1 of Sec. 2.1), so
// psi2 keeps ~1 ulp absolute accuracy near its peak.
#pragma once

#include "ffst_internal.cuh"

namespace ffst {

__device__ __forceinline__ float vpoly(float x) {
  const float x2 = x * x;
  return x2 * x2 * fmaf(x, fmaf(x, fmaf(x, -20.0f, 70.0f), -84.0f), 35.0f);
}

// v(x) for x in [0, 1/2] in the plan's variant; v(1 - x) = 1 - v(x) covers
// the other half in every variant.
__device__ __forceinline__ float vhalf(const WinParams& w, float x) {
  if (w.vkind == FFST_V_MEYER) return vpoly(x);
  if (w.vkind == FFST_V_QUADRATIC) return 2.0f * x * x;
  if (w.vkind == FFST_V_POLY) {
    float acc = w.vc[w.vdeg];
    for (int n = w.vdeg - 1; n >= 0; --n) acc = fmaf(acc, x, w.vc[n]);
    return acc;
  }
  // FFST_V_CINF: s(x-1) / (s(x-1) + s(x)), s(y) = exp(-(1/(1+y)^2 + 1/(1-y)^2))
  if (x <= 0.0f) return 0.0f;
  const float s0 = expf(-(1.0f / (x * x) + 1.0f / ((2.0f - x) * (2.0f - x))));
  const float s1 = expf(-(1.0f / ((1.0f + x) * (1.0f + x)) + 1.0f / ((1.0f - x) * (1.0f - x))));
  return s0 / (s0 + s1);
}

__device__ __forceinline__ float psi2_hat(const WinParams& w, float u) {
  const float y = fabsf(u);
  if (y >= 1.0f) return 0.0f;
  const float vv = (y < 0.5f) ? 1.0f - vhalf(w, y) : vhalf(w, 1.0f - y);
  return sqrtf(vv);
}

// Radial factor of the smooth shearlets of scale j (Sec. 3.4 eq. newPsi1):
// Psi1(w) = sqrt(Phi(w/4)^2 - Phi(w)^2), Phi = varphi x varphi, at
// w = 4^-j xi.  Where both |w_i| <= 2, Phi(w/4) = 1 and the difference is
// 1 - (1 - s1)(1 - s2) = s1 + s2 - s1 s2 with s = 1 - varphi(w)^2 read from a
// table generated in FP64 (no cancellation near the inner edge); elsewhere
// varphi(w) = 0 on the axis beyond 2 and the difference is Phi(w/4)^2.
__device__ __forceinline__ float smooth_radial(const WinParams& w, int j, int a1, int a2) {
  const float ac = __ldg(&w.alp_col[j * (w.hn + 1) + a1]);
  const float ar = __ldg(&w.alp_row[j * (w.hm + 1) + a2]);
  float r2;
  if (ac == 1.0f && ar == 1.0f) {
    const float sc = __ldg(&w.sig_col[j * (w.hn + 1) + a1]);
    const float sr = __ldg(&w.sig_row[j * (w.hm + 1) + a2]);
    r2 = fmaf(-sc, sr, sc + sr);
  } else {
    r2 = ac * ar;
  }
  return sqrtf(r2);
}

// Unfixed spectrum of plane (kappa, j, k) at integer frequency (o2, o1).
// |o1| <= floor(N/2), |o2| <= floor(M/2), gm, gn <= 2048 and j <= 7 keep every
// product below 2^31.
__device__ __forceinline__ float win_raw(const WinParams& w, int kappa, int j, int k, int o2, int o1) {
  const int a2 = abs(o2), a1 = abs(o1);
  const int lhs = a2 * w.gn;  // |xi2| ~ lhs, |xi1| ~ rhs (common factor X/(gm gn))
  const int rhs = a1 * w.gm;
  if (kappa == kLowpass) {
    if (w.smooth) return __ldg(&w.phi_col[a1]) * __ldg(&w.phi_row[a2]);  // Sec. 2.4 eq. (Phi)
    return (lhs <= rhs) ? __ldg(&w.phi_col[a1]) : __ldg(&w.phi_row[a2]);
  }
  bool use_h;
  if (lhs < rhs) {
    use_h = true;
  } else if (lhs > rhs) {
    use_h = false;
  } else {
    // seam line |xi1| = |xi2| (or the origin): only the glued seam shearlet, h formula
    if (kappa != kSeam || (a1 | a2) == 0) return 0.0f;
    use_h = true;
  }
  if ((use_h && kappa == kV) || (!use_h && kappa == kH)) return 0.0f;
  float p1;
  int num, den;
  if (use_h) {
    p1 = w.smooth ? 0.0f : __ldg(&w.psi1_col[j * (w.hn + 1) + a1]);
    num = (1 << j) * o2 * w.gn + k * o1 * w.gm;
    den = o1 * w.gm;
  } else {
    p1 = w.smooth ? 0.0f : __ldg(&w.psi1_row[j * (w.hm + 1) + a2]);
    num = (1 << j) * o1 * w.gm + k * o2 * w.gn;
    den = o2 * w.gn;
  }
  if (w.smooth) p1 = smooth_radial(w, j, a1, a2);  // both cones (Sec. 3.4 eq. smoothPsi)
  if (p1 == 0.0f) return 0.0f;
  const float u = __int2float_rn(num) / __int2float_rn(den);
  return p1 * psi2_hat(w, u);
}

// Spectrum with the Sec. 3.8.1 fix at half-spectrum position (pr, pc):
// pr in [0, M) (omega_2 in FFT order), pc in [0, N/2] (omega_1 >= 0, and
// -N/2 at pc = N/2).  On the Nyquist row (or column) the value is
// sqrt((psi(w)^2 + psi(w')^2)/2) with w' the point mirrored across the axis;
// the corner (-M/2, -N/2) is its own conjugate partner and stays unchanged.
__device__ __forceinline__ float win_at(const WinParams& w, const PlaneDesc& d, int pr, int pc) {
  const int o2 = (2 * pr < w.M) ? pr : pr - w.M;
  const int o1 = (2 * pc < w.N) ? pc : pc - w.N;
  const bool nyq_r = (w.M % 2 == 0) && (2 * pr == w.M);
  const bool nyq_c = (w.N % 2 == 0) && (2 * pc == w.N);
  const float a = win_raw(w, d.kappa, d.j, d.k, o2, o1);
  if (nyq_r == nyq_c) return a;
  const float b = nyq_r ? win_raw(w, d.kappa, d.j, d.k, -o2, o1) : win_raw(w, d.kappa, d.j, d.k, o2, -o1);
  return sqrtf(0.5f * (a * a + b * b));
}

// Side of the one-sided (complex) shearlets of Sec. 3.8.2 at half-spectrum
// position (pr, pc): +1 kept, -1 dropped, 0 on the self-conjugate grid
// points and for the low-pass (two-sided).  On C^h and the seam lines the
// side omega_1 > 0, on C^v omega_2 > 0; on the Nyquist column the sign of
// omega_2 decides and on the Nyquist row the sign of omega_1, so that of
// every pair {omega, -omega} exactly one point is kept.
__device__ __forceinline__ int half_sign(const WinParams& w, int kappa, int pr, int pc) {
  if (kappa == kLowpass) return 0;
  const int o2 = (2 * pr < w.M) ? pr : pr - w.M;
  const int o1 = (2 * pc < w.N) ? pc : pc - w.N;
  const bool ny_r = (w.M % 2 == 0) && (2 * pr == w.M);
  const bool ny_c = (w.N % 2 == 0) && (2 * pc == w.N);
  auto sgn = [](int x) { return (x > 0) - (x < 0); };
  const bool use_h = abs(o2) * w.gn <= abs(o1) * w.gm;  // C^h, seam lines (and the origin)
  if (use_h) return ny_c ? (ny_r ? 0 : sgn(o2)) : sgn(o1);
  return ny_r ? (ny_c ? 0 : sgn(o1)) : sgn(o2);
}

}  // namespace ffst
