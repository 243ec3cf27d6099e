// dg_common.cuh -- device helpers shared by the libdg kernels: index maps,
// double-double arithmetic for the metric construction, and the point-wise
// physics of the compressible Navier-Stokes equations (Sec. 2.1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_types.h"

namespace dg {

// ---------------------------------------------------------------------------
// Index maps.  Node index inside an element: i + n (j + n k).
// Local faces f = 2 d + s (d: xi, eta, zeta; s = 0 minus, 1 plus face).
// Face frame (p, q): (j, k) for d = 0, (i, k) for d = 1, (i, j) for d = 2.
// ---------------------------------------------------------------------------
template <int n>
__host__ __device__ __forceinline__ int face_vol_node(int f, int p, int q) {
  const int d = f >> 1, end = (f & 1) ? n - 1 : 0;
  return d == 0 ? end + n * (p + n * q) : (d == 1 ? p + n * (end + n * q) : p + n * (q + n * end));
}

// Flip convention: the slave face node (ps, qs) (slave's own face frame)
// coincides with master node (pm, qm) = T(ps, qs), where T first swaps the
// two coordinates if bit 2 is set, then reverses p (bit 0) and q (bit 1).
template <int n>
__host__ __device__ __forceinline__ void flip_to_master(int flip, int ps, int qs, int& pm, int& qm) {
  int a = (flip & 4) ? qs : ps;
  int b = (flip & 4) ? ps : qs;
  pm = (flip & 1) ? n - 1 - a : a;
  qm = (flip & 2) ? n - 1 - b : b;
}
template <int n>
__host__ __device__ __forceinline__ void flip_to_slave(int flip, int pm, int qm, int& ps, int& qs) {
  int a = (flip & 1) ? n - 1 - pm : pm;
  int b = (flip & 2) ? n - 1 - qm : qm;
  ps = (flip & 4) ? b : a;
  qs = (flip & 4) ? a : b;
}

// elem_side packing: side index << 4 | is_slave << 3 | flip
__host__ __device__ __forceinline__ int es_side(int v) { return v >> 4; }
__host__ __device__ __forceinline__ int es_slave(int v) { return (v >> 3) & 1; }
__host__ __device__ __forceinline__ int es_flip(int v) { return v & 7; }

// ---------------------------------------------------------------------------
// Double-double arithmetic (Knuth's two-sum, an FMA-based exact product, and
// renormalisation), used only at initialisation for the curl-form metrics.
// ---------------------------------------------------------------------------
struct dd {
  double hi, lo;
};
__device__ __forceinline__ dd dd_from(double a) { return {a, 0.0}; }
__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dd quick_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  double e = __dadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, e);
  e = __dadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  double p = __dmul_rn(a.hi, b.hi);
  double e = __fma_rn(a.hi, b.hi, -p);
  e = __fma_rn(a.hi, b.lo, e);
  e = __fma_rn(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ double dd_to_double(dd a) { return __dadd_rn(a.hi, a.lo); }

// ---------------------------------------------------------------------------
// binary64 <-> binary32 conversions on the integer pipe.  The FP32-bulk
// kernels convert FP64 state values to FP32 and their FP32 results back; a
// GB300 runs FP64 at 1/64 of the FP32 rate and the hardware conversions
// share that unit, where they used half or more of its cycles in those
// kernels.  These do the same conversions with 32/64-bit integer operations,
// written from the IEEE 754 formats: binary64 -> binary32 rounds to nearest,
// ties to even (normal, subnormal, overflow to infinity, zero, NaN to the
// quiet NaN 0x7fffffff); binary32 -> binary64 is exact.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  // the common case, a binary32 normal (biased binary64 exponent 897..1150):
  // adding half an ulp minus one, plus the kept last bit, to the magnitude
  // rounds to nearest, ties to even, at the 29th bit; a carry runs into the
  // exponent field (up to infinity from the top binade), and the exponent
  // bias changes from 1023 to 127 by one subtraction (modulo 2^32, the
  // result fits 31 bits)
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  if (mag >= (897ull << 52) && mag < (1151ull << 52)) {
    const unsigned long long r = mag + 0x0FFFFFFFull + ((mag >> 29) & 1ull);
    return __uint_as_float(sign | ((unsigned)(r >> 29) - (896u << 23)));
  }
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;  // 52 fraction bits
  if (e == 0x7ff) return __uint_as_float(m ? 0x7fffffffu : (sign | 0x7f800000u));
  const int ef = e - 1023 + 127;  // biased binary32 exponent
  if (ef >= 0xff) return __uint_as_float(sign | 0x7f800000u);
  if (ef > 0) {
    // keep 23 fraction bits; the 29 dropped bits decide the rounding; a carry
    // out of the fraction increments the exponent (to infinity at the top)
    unsigned q = ((unsigned)ef << 23) | (unsigned)(m >> 29);
    const unsigned long long rem = m & 0x1FFFFFFFull, half = 0x10000000ull;
    if (rem > half || (rem == half && (q & 1u))) ++q;
    return __uint_as_float(sign | q);
  }
  if (ef < -24 || e == 0) return __uint_as_float(sign);  // below half the smallest subnormal (or a binary64 subnormal)
  // binary32 subnormal: 53-bit significand shifted right by 30 - ef
  const unsigned long long mm = m | (1ull << 52);
  const int shift = 30 - ef;
  unsigned long long q = mm >> shift;
  const unsigned long long rem = mm & ((1ull << shift) - 1), half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (q & 1ull))) ++q;
  return __uint_as_float(sign | (unsigned)q);
}

__device__ __forceinline__ double f64_of(float f) {
  const unsigned u = __float_as_uint(f);
  // the common case, a binary32 normal: the fraction moves up by 29 bits and
  // the biased exponent grows by 1023 - 127 = 896, in the high word
  const unsigned mag = u & 0x7fffffffu;
  if (mag >= 0x00800000u && mag < 0x7f800000u)
    return __hiloint2double((int)((u & 0x80000000u) | ((mag >> 3) + (896u << 20))), (int)(mag << 29));
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xff, m = u & 0x7fffffu;
  if (e == 0xff) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | ((unsigned long long)m << 29)));
  if (e == 0) {
    if (m == 0) return __longlong_as_double((long long)sign);
    // subnormal: normalise the fraction (leading one moved to bit 23)
    const int lz = __clz(m) - 8;  // zeros between bit 22 and the leading one, plus one
    const unsigned mn = (m << lz) & 0x7fffffu;
    const unsigned long long e64 = (unsigned long long)(1023 - 126 - lz);
    return __longlong_as_double((long long)(sign | (e64 << 52) | ((unsigned long long)mn << 29)));
  }
  const unsigned long long e64 = (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double((long long)(sign | (e64 << 52) | ((unsigned long long)m << 29)));
}

// an FP64 value in the arithmetic type T (FP32: rounded on the integer pipe)
template <typename T>
__device__ __forceinline__ T from_f64(double v) {
  if constexpr (sizeof(T) == sizeof(float)) return f32_rn(v);
  else return v;
}
// a value of the arithmetic type T in FP64 (exact; FP32 on the integer pipe)
template <typename T>
__device__ __forceinline__ double to_f64(T v) {
  if constexpr (sizeof(T) == sizeof(float)) return f64_of(v);
  else return v;
}

// ---------------------------------------------------------------------------
// Point-wise physics, templated on the arithmetic type T.
// ---------------------------------------------------------------------------
struct Gas {
  double gamma, R, Pr, mu;
  double gm1;     // gamma - 1
  double lambda;  // heat conductivity gamma R mu / ((gamma - 1) Pr)
};

template <typename T>
struct Prim {
  T rho, u, v, w, p, T_;  // density, velocity, pressure, temperature
};

// Eqs. eos_p / eos_T
template <typename T>
__device__ __forceinline__ Prim<T> cons_to_prim(const T U[5], T gm1, T Rinv) {
  Prim<T> q;
  T ri = T(1) / U[0];
  q.rho = U[0];
  q.u = U[1] * ri;
  q.v = U[2] * ri;
  q.w = U[3] * ri;
  q.p = gm1 * (U[4] - T(0.5) * (U[1] * q.u + U[2] * q.v + U[3] * q.w));
  q.T_ = q.p * ri * Rinv;
  return q;
}

// Euler flux contracted with nv (Eq. nse)
template <typename T>
__device__ __forceinline__ void euler_flux(const T U[5], const Prim<T>& q, const T nv[3], T f[5]) {
  T un = q.u * nv[0] + q.v * nv[1] + q.w * nv[2];
  f[0] = U[0] * un;
  f[1] = U[1] * un + q.p * nv[0];
  f[2] = U[2] * un + q.p * nv[1];
  f[3] = U[3] * un + q.p * nv[2];
  f[4] = (U[4] + q.p) * un;
}

// Roe's approximate Riemann solver, unit normal n, no entropy fix.
template <typename T>
__device__ __forceinline__ void roe_flux(const T UL[5], const Prim<T>& qL, const T UR[5], const Prim<T>& qR,
                                         const T n[3], T gm1, T f[5]) {
  T fL[5], fR[5];
  euler_flux(UL, qL, n, fL);
  euler_flux(UR, qR, n, fR);
  T sL = sqrt(qL.rho), sR = sqrt(qR.rho);
  T inv = T(1) / (sL + sR);
  T HL = (UL[4] + qL.p) / qL.rho, HR = (UR[4] + qR.p) / qR.rho;
  T ut0 = (sL * qL.u + sR * qR.u) * inv;
  T ut1 = (sL * qL.v + sR * qR.v) * inv;
  T ut2 = (sL * qL.w + sR * qR.w) * inv;
  T Ht = (sL * HL + sR * HR) * inv;
  T rt = sL * sR;
  T q2 = ut0 * ut0 + ut1 * ut1 + ut2 * ut2;
  T c2 = gm1 * (Ht - T(0.5) * q2);
  T c = sqrt(c2);
  T c2i = T(1) / c2;
  T un = ut0 * n[0] + ut1 * n[1] + ut2 * n[2];
  T drho = qR.rho - qL.rho, dp = qR.p - qL.p;
  T du0 = qR.u - qL.u, du1 = qR.v - qL.v, du2 = qR.w - qL.w;
  T dun = du0 * n[0] + du1 * n[1] + du2 * n[2];
  T a1 = T(0.5) * (dp - rt * c * dun) * c2i;
  T a2 = drho - dp * c2i;
  T a5 = T(0.5) * (dp + rt * c * dun) * c2i;
  T l1 = fabs(un - c) * a1, l2 = fabs(un), l5 = fabs(un + c) * a5;
  T l2a = l2 * a2, l2r = l2 * rt;
  T dt0 = du0 - dun * n[0], dt1 = du1 - dun * n[1], dt2 = du2 - dun * n[2];
  T D0 = l1 + l2a + l5;
  T D1 = l1 * (ut0 - c * n[0]) + l2a * ut0 + l5 * (ut0 + c * n[0]) + l2r * dt0;
  T D2 = l1 * (ut1 - c * n[1]) + l2a * ut1 + l5 * (ut1 + c * n[1]) + l2r * dt1;
  T D3 = l1 * (ut2 - c * n[2]) + l2a * ut2 + l5 * (ut2 + c * n[2]) + l2r * dt2;
  T D4 = l1 * (Ht - un * c) + l2a * T(0.5) * q2 + l5 * (Ht + un * c) +
         l2r * (ut0 * dt0 + ut1 * dt1 + ut2 * dt2);
  f[0] = T(0.5) * (fL[0] + fR[0] - D0);
  f[1] = T(0.5) * (fL[1] + fR[1] - D1);
  f[2] = T(0.5) * (fL[2] + fR[2] - D2);
  f[3] = T(0.5) * (fL[3] + fR[3] - D3);
  f[4] = T(0.5) * (fL[4] + fR[4] - D4);
}

// Local Lax-Friedrichs (Rusanov), unit normal n.
template <typename T>
__device__ __forceinline__ void lf_flux(const T UL[5], const Prim<T>& qL, const T UR[5], const Prim<T>& qR,
                                        const T n[3], T gamma, T f[5]) {
  T fL[5], fR[5];
  euler_flux(UL, qL, n, fL);
  euler_flux(UR, qR, n, fR);
  T cL = sqrt(gamma * qL.p / qL.rho), cR = sqrt(gamma * qR.p / qR.rho);
  T lL = fabs(qL.u * n[0] + qL.v * n[1] + qL.w * n[2]) + cL;
  T lR = fabs(qR.u * n[0] + qR.v * n[1] + qR.w * n[2]) + cR;
  T lm = lL > lR ? lL : lR;
#pragma unroll
  for (int k = 0; k < 5; ++k) f[k] = T(0.5) * (fL[k] + fR[k] - lm * (UR[k] - UL[k]));
}

// Viscous stress and the energy "work + conduction" vector from the lifted
// gradients g[qv*3 + x] = d(u, v, w, T)_qv / dx_x (Eq. nse, stress tensor,
// Fourier law).  tau = (xx, yy, zz, xy, xz, yz), W_x = tau_x . u + lambda T_x.
template <typename T>
__device__ __forceinline__ void viscous_parts(const T g[12], T u, T v, T w, T mu, T lam, T tau[6], T W[3]) {
  T div = g[0] + g[4] + g[8];
  T tw = T(2.0 / 3.0) * div;
  tau[0] = mu * (T(2) * g[0] - tw);
  tau[1] = mu * (T(2) * g[4] - tw);
  tau[2] = mu * (T(2) * g[8] - tw);
  tau[3] = mu * (g[1] + g[3]);
  tau[4] = mu * (g[2] + g[6]);
  tau[5] = mu * (g[5] + g[7]);
  W[0] = tau[0] * u + tau[3] * v + tau[4] * w + lam * g[9];
  W[1] = tau[3] * u + tau[1] * v + tau[5] * w + lam * g[10];
  W[2] = tau[4] * u + tau[5] * v + tau[2] * w + lam * g[11];
}

// The spectral radii of the CFL rule at one node (dg_time_step in dg.h):
// convective aa = sum_d (|u . Ja^d| + c |Ja^d|) / J and viscous
// bb = kv(T) |Ja|^2 / (rho J^2), from the node's conservative state Uv, its
// metrics M (Ja^d_c at 3 d + c, 1/J at 9) and kv = max(4/3, gamma / Pr) mu
// (times Sutherland's mu(T) / mu_ref).  FP64: the geometry factors G (|Ja^d|
// for d = 0, 1, 2, then sum_d |Ja^d|^2) are read, formed once from the FP64
// metrics.
__device__ __forceinline__ void cfl_radii(const double Uv[5], const double M[10], const double G[4], double gamma,
                                          double gm1, double Rinv, double kv, int sutherland, double inv_Tref,
                                          double& aa, double& bb) {
  const double ri = 1.0 / Uv[0];
  const double u = Uv[1] * ri, v = Uv[2] * ri, w = Uv[3] * ri;
  const double p = gm1 * (Uv[4] - 0.5 * (Uv[1] * u + Uv[2] * v + Uv[3] * w));
  const double c = sqrt(gamma * p * ri);
  double a = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) a += fabs(u * M[d * 3] + v * M[d * 3 + 1] + w * M[d * 3 + 2]) + c * G[d];
  aa = a * M[9];
  double kvn = kv;
  if (sutherland) {  // mu(T) / mu_ref by Sutherland's law (Eq. sutherland)
    const double th = p * ri * Rinv * inv_Tref;
    kvn = kvn * 1.4042 * th * sqrt(th) / (th + 0.4042);
  }
  bb = kvn * ri * G[3] * M[9] * M[9];
}
// FP32: the geometry factors are formed here from the FP32 metrics, so the
// radii need nothing beyond the state and the metrics; every product and sum
// is a separately rounded operation written out, so the CFL reduction kernel
// and the two-kernel stage's epilogue, which both call this, form bitwise
// the same radii whatever the compiler fuses around them.
__device__ __forceinline__ void cfl_radii(const float Uv[5], const float M[10], float gamma, float gm1, float Rinv,
                                          float kv, int sutherland, float inv_Tref, float& aa, float& bb) {
  const float ri = 1.0f / Uv[0];
  const float u = __fmul_rn(Uv[1], ri), v = __fmul_rn(Uv[2], ri), w = __fmul_rn(Uv[3], ri);
  const float m2 = __fmaf_rn(Uv[3], w, __fmaf_rn(Uv[2], v, __fmul_rn(Uv[1], u)));
  const float p = __fmul_rn(gm1, __fsub_rn(Uv[4], __fmul_rn(0.5f, m2)));
  const float c = sqrtf(__fmul_rn(__fmul_rn(gamma, p), ri));
  float a = 0.0f, g2 = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float j0 = M[d * 3], j1 = M[d * 3 + 1], j2 = M[d * 3 + 2];
    const float nj2 = __fmaf_rn(j2, j2, __fmaf_rn(j1, j1, __fmul_rn(j0, j0)));
    g2 = __fadd_rn(g2, nj2);
    const float un = __fmaf_rn(w, j2, __fmaf_rn(v, j1, __fmul_rn(u, j0)));
    a = __fadd_rn(a, __fmaf_rn(c, sqrtf(nj2), fabsf(un)));
  }
  aa = __fmul_rn(a, M[9]);
  float kvn = kv;
  if (sutherland) {  // mu(T) / mu_ref by Sutherland's law (Eq. sutherland)
    const float th = __fmul_rn(__fmul_rn(__fmul_rn(p, ri), Rinv), inv_Tref);
    kvn = __fmul_rn(__fmul_rn(__fmul_rn(kvn, 1.4042f), th), sqrtf(th)) / __fadd_rn(th, 0.4042f);
  }
  bb = __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(kvn, ri), g2), M[9]), M[9]);
}

// F_v . nv  (4 non-zero components: momentum x, y, z and energy)
template <typename T>
__device__ __forceinline__ void viscous_flux_n(const T tau[6], const T W[3], const T nv[3], T f[4]) {
  f[0] = tau[0] * nv[0] + tau[3] * nv[1] + tau[4] * nv[2];
  f[1] = tau[3] * nv[0] + tau[1] * nv[1] + tau[5] * nv[2];
  f[2] = tau[4] * nv[0] + tau[5] * nv[1] + tau[2] * nv[2];
  f[3] = W[0] * nv[0] + W[1] * nv[1] + W[2] * nv[2];
}

}  // namespace dg
