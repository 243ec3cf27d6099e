// dg_stage.cuh -- the kernels of one evaluation of the DG time derivative
// (Eq. dgsem with the split-form volume integral and BR1 lifting) and of the
// fused low-storage RK stage, templated on the arithmetic type T of the
// flux, volume and surface work (double: the FP64 path; float: the FP32-bulk
// path, in which the state, the RK register, the metrics and the final
// combination stay in FP64).
//
// Per stage:
//   k_surf_prims  ProlongToFace of the lifted primitives (u, v, w, T) and the
//                 BR1 surface flux q* (s n) on every side node   (Lift_FillFlux)
//   k_lift        lifted gradients, weak form: volume part with Dhat, surface
//                 part from the sides, 1/J                      (Lift_VolInt,
//                                                                Lift_SurfInt,
//                                                                Lift_ApplyJac)
//   k_surf_flux   Roe / LF flux plus BR1 viscous flux times s   (FillFlux)
//   k_volume      split-form KEP volume integral, viscous volume term,
//                 optional DG/FV blending, SurfInt, ApplyJac and either Ut or
//                 the RK update dU = A dU + dt Ut, U += B dU   (VolInt, SurfInt,
//                                                                ApplyJac, RK)
//
// Shifted primitives.  The fluxes work with p' = p - p_ref, H' = H - H_ref and
// T' = T - T_ref for constants (p_ref, H_ref, T_ref) held per context (all zero
// on the FP64 path).  This is exact algebra: the p_ref and T_ref parts of the
// volume and surface terms add up to p_ref (resp. T_ref) times the discrete
// metric identities, which vanish to round-off; the H_ref part of the energy
// equation is exactly H_ref times the mass equation and is added back in FP64
// from the density right-hand side.  At Ma = 0.1 (p ~ 71, fluctuations ~ 0.06)
// this keeps FP32 rounding relative to the fluctuations, not to p.
//
// Data layout: element-major SoA, U[e][v][node], node = i + n (j + n k).
#pragma once
#include <algorithm>
#include <cmath>

#include "dg_common.cuh"
#include "dg_launch.h"

namespace dg {

// Element blocks: EPB elements per thread block, one thread per node.
// EPB_ = 0 takes the default (about 256 threads); the autotuner may pick
// twice as many elements per block.
template <int N, int EPB_ = 0>
struct Shape {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  static constexpr int EPB_DEFAULT = n3 >= 256 ? 1 : 256 / n3;
  static constexpr int EPB = EPB_ > 0 ? EPB_ : EPB_DEFAULT;  // elements per block
  static constexpr int THREADS = EPB * n3;
  // FP32-bulk volume kernel: at least 1024 resident threads per SM (it is
  // latency-bound); the FP64 one is bound by the FP64 pipe at one block
  template <typename T>
  static constexpr int vol_min_blocks() {
    return sizeof(T) == sizeof(float) && THREADS <= 512 ? 1024 / THREADS : 1;
  }
};

// buffers of the arithmetic type T
template <typename T>
struct TBuf;
template <>
struct TBuf<double> {
  static __host__ __device__ double* g(const StageArgs& a) { return a.g; }
  static __host__ __device__ double* lflux(const StageArgs& a) { return a.lflux; }
  static __host__ __device__ double* fstar(const StageArgs& a) { return a.fstar; }
  static __host__ __device__ double* gfc(const StageArgs& a) { return a.gfc; }
};
template <>
struct TBuf<float> {
  static __host__ __device__ float* g(const StageArgs& a) { return a.g32; }
  static __host__ __device__ float* lflux(const StageArgs& a) { return a.lflux32; }
  static __host__ __device__ float* fstar(const StageArgs& a) { return a.fstar32; }
  static __host__ __device__ float* gfc(const StageArgs& a) { return a.gfc32; }
};

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async, 4, 8 or 16 bytes per thread and call)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 16 bytes, both addresses 16-byte aligned (bypasses L1)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// waits until at most K of this thread's committed groups are still in flight
template <int K>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

// ---------------------------------------------------------------------------
// Shifted primitive state and the fluxes written in it
// ---------------------------------------------------------------------------
template <typename T>
struct SPrim {
  T rho, u, v, w, p, H, Tt;  // p, H, Tt shifted by the context's references
};

// Parameters that may differ between the cases of a serving pool.  The
// reference state (zero on the FP64 path) is a state at rest: rr, pr, its
// total energy Er = pr / (gamma - 1), enthalpy Hr = (Er + pr) / rr and
// temperature Tr = pr / (rr R).
// The FP32 fields are the same constants rounded once, on the host or by the
// kernel that sets the references, so that no kernel converts them per thread.
struct CaseParams {
  double mu, lam, pr, Hr, Tr, rr, Er;
  int riemann;
  float fmu, flam, fpr, fHr, fTr, fgm1, fRinv, fgamma;
};
__device__ __forceinline__ CaseParams case_params(const StageArgs& a, int c) {
  if (a.cases) {
    const CaseData& d = a.cases[c < 0 ? 0 : c];
    return {d.mu,     d.lam,     d.ref_p,   d.ref_H,   d.ref_T, d.ref_rho, d.ref_E,  d.riemann,
            d.f_mu,   d.f_lam,   d.f_ref_p, d.f_ref_H, d.f_ref_T, a.f_gm1, a.f_Rinv, a.f_gamma};
  }
  const DevScalars* s = a.scal;
  return {a.mu,   a.lam,   s->ref_p,   s->ref_H,   s->ref_T, s->ref_rho, s->ref_E,  a.riemann,
          a.f_mu, a.f_lam, s->f_ref_p, s->f_ref_H, s->f_ref_T, a.f_gm1, a.f_Rinv, a.f_gamma};
}
// the constant in the arithmetic type: the FP64 value, or its FP32 copy
template <typename T>
__device__ __forceinline__ T pick(double d, float f) {
  if constexpr (sizeof(T) == sizeof(float)) return f;
  else return d;
}

// viscosity and heat conductivity at a node of (shifted) temperature Tt:
// constant, or Sutherland's law (Eq. sutherland) with lambda = kappa mu
template <typename T>
__device__ __forceinline__ void visc_coeffs(const StageArgs& a, const CaseParams& cp, T Tt, T& mu, T& lam) {
  const T mu0 = pick<T>(cp.mu, cp.fmu);
  if (!a.sutherland) {
    mu = mu0;
    lam = pick<T>(cp.lam, cp.flam);
    return;
  }
  const T th = (Tt + pick<T>(cp.Tr, cp.fTr)) * pick<T>(a.inv_Tref, a.f_inv_Tref);
  mu = mu0 * T(1.4042) * th * sqrt(th) / (th + T(0.4042));
  lam = mu * pick<T>(a.kappa, a.f_kappa);
}
// Manufactured-solution source of Sec. 5.1 (Eq. mms) at node coordinates x
// and time ts, FP64: with phi = 2 pi (x + y + z - a t), rho = rho u = rho v =
// rho w = 2 + A sin(phi) and rho e = rho^2 (velocity (1, 1, 1), no stress),
// Q = U_t + div F_c - div F_v of that state:
//   Q_rho = (3 - a) c,  Q_m = Q_rho + (gamma - 1)(2 rho - 3/2) c,
//   Q_E = -2 a rho c + 3 (2 rho + (gamma - 1)(2 rho - 3/2)) c
//         + 3 lambda (gamma - 1) / R (2 pi)^2 A sin(phi)   (viscous),
// c = 2 pi A cos(phi).
__device__ __forceinline__ void mms_source(const StageArgs& a, const double* x, double ts, double Q[5]) {
  const double w = 2.0 * 3.141592653589793;
  const double phi = w * (x[0] + x[1] + x[2] - a.src_a * ts);
  double sn, cs;
  sincos(phi, &sn, &cs);
  sn *= a.src_A;
  const double c = w * a.src_A * cs;
  const double rho = 2.0 + sn, g1 = a.gm1;
  Q[0] = (3.0 - a.src_a) * c;
  const double qm = Q[0] + g1 * (2.0 * rho - 1.5) * c;
  Q[1] = qm;
  Q[2] = qm;
  Q[3] = qm;
  Q[4] = -2.0 * a.src_a * rho * c + 3.0 * (2.0 * rho + g1 * (2.0 * rho - 1.5)) * c;
  if (a.viscous) Q[4] += 3.0 * a.lam * g1 * a.Rinv * w * w * sn;
}
// the time of the stage being evaluated: the state's time for a plain
// right-hand side (mode 0); within a step the device time is already t_n + dt
__device__ __forceinline__ double stage_time(const StageArgs& a, int mode) {
  return mode == 0 ? a.scal->t : a.scal->t - (1.0 - a.rkC) * a.scal->dt;
}

__device__ __forceinline__ double case_dt(const StageArgs& a, int c) {
  return a.cases ? a.cases[c < 0 ? 0 : c].dt : a.scal->dt;
}

// ConsToPrim (Eqs. eos_p, eos_T).  FP64 path: in FP64 with a zero reference.
// FP32-bulk: the shifted primitives from the two deviations that cancel,
// d_rho = rho - rr and d_E = rho e - Er, taken in FP64; the rest in FP32.
// With Er = pr / (gamma - 1) and Hr = (Er + pr) / rr, exactly
//   p' = (gamma - 1)(d_E - |m|^2 / (2 rho)),
//   H' = (d_E + p' - Hr d_rho) / rho,
//   T' = (p' / R - Tr d_rho) / rho.
// INTCVT: the FP32 conversions on the integer pipe (f32_rn / f64_of: the
// same values as the hardware conversions, off the FP64 unit).  That pays
// in the volume kernel, whose FP64 unit also carries the RK update; in the
// lifting and surface kernels the extra integer instructions cost more than
// the conversions they replace.
template <typename T, bool INTCVT = false>
__device__ __forceinline__ SPrim<T> shifted_prim(const double U[5], double gm1, double Rinv, const CaseParams& cp,
                                                double* p_full = nullptr) {
  if constexpr (sizeof(T) == sizeof(float)) {
    auto cvt = [](double x) -> float {
      if constexpr (INTCVT) return f32_rn(x);
      else return float(x);
    };
    const float drho = cvt(U[0] - cp.rr), dE = cvt(U[4] - cp.Er);
    const float rho = cvt(U[0]), m0 = cvt(U[1]), m1 = cvt(U[2]), m2 = cvt(U[3]);
    const float ri = 1.0f / rho;
    const float u = m0 * ri, v = m1 * ri, w = m2 * ri;
    const float pp = cp.fgm1 * (dE - 0.5f * (m0 * u + m1 * v + m2 * w));
    const float Hp = (dE + pp - cp.fHr * drho) * ri;
    const float Tp = (pp * cp.fRinv - cp.fTr * drho) * ri;
    if (p_full) *p_full = cp.pr + (INTCVT ? f64_of(pp) : double(pp));
    return {rho, u, v, w, pp, Hp, Tp};
  } else {
    const double ri = 1.0 / U[0];
    const double u = U[1] * ri, v = U[2] * ri, w = U[3] * ri;
    const double p = gm1 * (U[4] - 0.5 * (U[1] * u + U[2] * v + U[3] * w));
    const double H = (U[4] + p) * ri;
    const double Tm = p * ri * Rinv;
    if (p_full) *p_full = p;
    return {T(U[0]), T(u), T(v), T(w), T(p - cp.pr), T(H - cp.Hr), T(Tm - cp.Tr)};
  }
}

// metric component c (0..8: J a^d_x at 3d + x; 9: 1/J) of node t of element e
template <typename T>
__device__ __forceinline__ T metric_at(const StageArgs& a, size_t e, int c, int t, int n3) {
  return T(a.metric[(e * 10 + c) * n3 + t]);
}
template <>
__device__ __forceinline__ float metric_at<float>(const StageArgs& a, size_t e, int c, int t, int n3) {
  return a.metric32[(e * 10 + c) * n3 + t];
}

// Euler flux contracted with nv, energy component minus H_ref times mass flux
template <typename T>
__device__ __forceinline__ void euler_flux_s(const SPrim<T>& q, const T nv[3], T f[5]) {
  const T un = q.u * nv[0] + q.v * nv[1] + q.w * nv[2];
  const T m = q.rho * un;
  f[0] = m;
  f[1] = m * q.u + q.p * nv[0];
  f[2] = m * q.v + q.p * nv[1];
  f[3] = m * q.w + q.p * nv[2];
  f[4] = m * q.H;
}

// Roe's approximate Riemann solver, unit normal n, no entropy fix
template <typename T>
__device__ __forceinline__ void roe_flux_s(const SPrim<T>& L, const SPrim<T>& R, const T n[3], T gm1, T Href,
                                           T f[5]) {
  T fL[5], fR[5];
  euler_flux_s(L, n, fL);
  euler_flux_s(R, n, fR);
  const T sL = sqrt(L.rho), sR = sqrt(R.rho);
  const T inv = T(1) / (sL + sR);
  const T ut0 = (sL * L.u + sR * R.u) * inv;
  const T ut1 = (sL * L.v + sR * R.v) * inv;
  const T ut2 = (sL * L.w + sR * R.w) * inv;
  const T Ht = (sL * L.H + sR * R.H) * inv;  // shifted Roe-average enthalpy
  const T rt = sL * sR;
  const T q2 = ut0 * ut0 + ut1 * ut1 + ut2 * ut2;
  const T c2 = gm1 * ((Href + Ht) - T(0.5) * q2);
  const T c = sqrt(c2);
  const T c2i = T(1) / c2;
  const T un = ut0 * n[0] + ut1 * n[1] + ut2 * n[2];
  const T drho = R.rho - L.rho, dp = R.p - L.p;
  const T du0 = R.u - L.u, du1 = R.v - L.v, du2 = R.w - L.w;
  const T dun = du0 * n[0] + du1 * n[1] + du2 * n[2];
  const T a1 = T(0.5) * (dp - rt * c * dun) * c2i;
  const T a2 = drho - dp * c2i;
  const T a5 = T(0.5) * (dp + rt * c * dun) * c2i;
  const T l1 = fabs(un - c) * a1, l2 = fabs(un), l5 = fabs(un + c) * a5;
  const T l2a = l2 * a2, l2r = l2 * rt;
  const T dt0 = du0 - dun * n[0], dt1 = du1 - dun * n[1], dt2 = du2 - dun * n[2];
  const T D0 = l1 + l2a + l5;
  const T D1 = l1 * (ut0 - c * n[0]) + l2a * ut0 + l5 * (ut0 + c * n[0]) + l2r * dt0;
  const T D2 = l1 * (ut1 - c * n[1]) + l2a * ut1 + l5 * (ut1 + c * n[1]) + l2r * dt1;
  const T D3 = l1 * (ut2 - c * n[2]) + l2a * ut2 + l5 * (ut2 + c * n[2]) + l2r * dt2;
  const T D4 = l1 * (Ht - un * c) + l2a * (T(0.5) * q2 - Href) + l5 * (Ht + un * c) +
               l2r * (ut0 * dt0 + ut1 * dt1 + ut2 * dt2);
  f[0] = T(0.5) * (fL[0] + fR[0] - D0);
  f[1] = T(0.5) * (fL[1] + fR[1] - D1);
  f[2] = T(0.5) * (fL[2] + fR[2] - D2);
  f[3] = T(0.5) * (fL[3] + fR[3] - D3);
  f[4] = T(0.5) * (fL[4] + fR[4] - D4);
}

// Local Lax-Friedrichs (Rusanov), unit normal n
template <typename T>
__device__ __forceinline__ void lf_flux_s(const SPrim<T>& L, const SPrim<T>& R, const T n[3], T gamma, T pref,
                                          T f[5]) {
  T fL[5], fR[5];
  euler_flux_s(L, n, fL);
  euler_flux_s(R, n, fR);
  const T cL = sqrt(gamma * (L.p + pref) / L.rho), cR = sqrt(gamma * (R.p + pref) / R.rho);
  const T lL = fabs(L.u * n[0] + L.v * n[1] + L.w * n[2]) + cL;
  const T lR = fabs(R.u * n[0] + R.v * n[1] + R.w * n[2]) + cR;
  const T lm = lL > lR ? lL : lR;
  // jumps of the conservative variables; energy minus H_ref times density:
  // rho e - H_ref rho = rho H' - p' - p_ref, whose jump is that of rho H' - p'
  const T d[5] = {R.rho - L.rho, R.rho * R.u - L.rho * L.u, R.rho * R.v - L.rho * L.v, R.rho * R.w - L.rho * L.w,
                  (R.rho * R.H - R.p) - (L.rho * L.H - L.p)};
#pragma unroll
  for (int k = 0; k < 5; ++k) f[k] = T(0.5) * (fL[k] + fR[k] - lm * d[k]);
}

// ---------------------------------------------------------------------------
// Boundary conditions (rows of include/dg.h's dg_mesh_desc.bc): the BR1
// lifting value and the surface flux at a boundary side node, from the inner
// state q (shifted primitives), its gradients g, the outward unit normal nu,
// the surface element sA and sn = sA nu.  In the shifted variables the
// momentum flux carries p' (the p_ref part cancels by the discrete metric
// identities, as on inner sides); the energy flux is the full one, the mass
// flux being zero at walls.
// ---------------------------------------------------------------------------
// the outer state of a prescribed-state or outflow condition, in FP64
__device__ __forceinline__ void bc_outer_state(const StageArgs& a, const double* b, const double U[5], double Ue[5]) {
  if ((int)b[0] == DG_BC_STATE) {
#pragma unroll
    for (int k = 0; k < 5; ++k) Ue[k] = b[1 + k];
    return;
  }
  const double ri = 1.0 / U[0];
  const double u = U[1] * ri, v = U[2] * ri, w = U[3] * ri;
  Ue[0] = U[0], Ue[1] = U[1], Ue[2] = U[2], Ue[3] = U[3];
  Ue[4] = b[1] / a.gm1 + 0.5 * (U[1] * u + U[2] * v + U[3] * w);
}

template <typename T>
__device__ __forceinline__ void bc_lift_value(const StageArgs& a, const CaseParams& cp, int row, const double U[5],
                                              const SPrim<T>& q, const T nu[3], T qs[4]) {
  const double* b = a.bcdata + (size_t)row * 9;
  const int type = (int)b[0];
  if (type == DG_BC_WALL_ISOTHERMAL) {
    qs[0] = T(b[1]), qs[1] = T(b[2]), qs[2] = T(b[3]), qs[3] = T(b[4] - cp.Tr);
  } else if (type == DG_BC_WALL_ADIABATIC) {
    qs[0] = T(b[1]), qs[1] = T(b[2]), qs[2] = T(b[3]), qs[3] = q.Tt;
  } else if (type == DG_BC_SLIP) {
    const T un = q.u * nu[0] + q.v * nu[1] + q.w * nu[2];
    qs[0] = q.u - un * nu[0], qs[1] = q.v - un * nu[1], qs[2] = q.w - un * nu[2], qs[3] = q.Tt;
  } else {
    double Ue[5];
    bc_outer_state(a, b, U, Ue);
    const SPrim<T> qe = shifted_prim<T>(Ue, a.gm1, a.Rinv, cp);
    qs[0] = (q.u + qe.u) / T(2), qs[1] = (q.v + qe.v) / T(2), qs[2] = (q.w + qe.w) / T(2);
    qs[3] = (q.Tt + qe.Tt) / T(2);
  }
}

template <typename T>
__device__ __forceinline__ void bc_flux(const StageArgs& a, const CaseParams& cp, int row, const double U[5],
                                        const SPrim<T>& q, const T g[12], const T nu[3], T sA, const T sn[3],
                                        T f[5]) {
  const double* b = a.bcdata + (size_t)row * 9;
  const int type = (int)b[0];
  if (type == DG_BC_STATE || type == DG_BC_OUTFLOW) {
    double Ue[5];
    bc_outer_state(a, b, U, Ue);
    const SPrim<T> qe = shifted_prim<T>(Ue, a.gm1, a.Rinv, cp);
    if (cp.riemann == DG_RIEMANN_ROE) roe_flux_s(q, qe, nu, pick<T>(a.gm1, a.f_gm1), pick<T>(cp.Hr, cp.fHr), f);
    else lf_flux_s(q, qe, nu, pick<T>(a.gamma, a.f_gamma), pick<T>(cp.pr, cp.fpr), f);
#pragma unroll
    for (int k = 0; k < 5; ++k) f[k] *= sA;
    if (a.viscous) {
      T tau[6], W[3], f1[4], f2[4], vmu, vlam;
      visc_coeffs<T>(a, cp, q.Tt, vmu, vlam);
      viscous_parts(g, q.u, q.v, q.w, vmu, vlam, tau, W);
      viscous_flux_n(tau, W, sn, f1);
      visc_coeffs<T>(a, cp, qe.Tt, vmu, vlam);
      viscous_parts(g, qe.u, qe.v, qe.w, vmu, vlam, tau, W);
      viscous_flux_n(tau, W, sn, f2);
#pragma unroll
      for (int k = 0; k < 4; ++k) f[1 + k] -= (f1[k] + f2[k]) / T(2);
    }
    return;
  }
  T uw[3] = {T(0), T(0), T(0)};
  if (type != DG_BC_SLIP) uw[0] = T(b[1]), uw[1] = T(b[2]), uw[2] = T(b[3]);
  f[0] = T(0);
  f[1] = q.p * nu[0] * sA;
  f[2] = q.p * nu[1] * sA;
  f[3] = q.p * nu[2] * sA;
  f[4] = (q.p + pick<T>(cp.pr, cp.fpr)) * (uw[0] * nu[0] + uw[1] * nu[1] + uw[2] * nu[2]) * sA;
  if (a.viscous && type != DG_BC_SLIP) {
    T gw[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) gw[k] = g[k];
    if (type == DG_BC_WALL_ADIABATIC) gw[9] = gw[10] = gw[11] = T(0);
    const T Tw = type == DG_BC_WALL_ISOTHERMAL ? T(b[4] - cp.Tr) : q.Tt;
    T tau[6], W[3], fv[4], vmu, vlam;
    visc_coeffs<T>(a, cp, Tw, vmu, vlam);
    viscous_parts(gw, uw[0], uw[1], uw[2], vmu, vlam, tau, W);
    viscous_flux_n(tau, W, sn, fv);
#pragma unroll
    for (int k = 0; k < 4; ++k) f[1 + k] -= fv[k];
  }
}

// ---------------------------------------------------------------------------
// BR1 surface flux of the lifted primitives
// ---------------------------------------------------------------------------
// GL: the side's two face states come from the ProlongToFace array (master
// face frame) instead of the face nodes of the elements
template <int N, typename T, bool GL = false>
__global__ void __launch_bounds__(256) k_surf_prims(StageArgs a) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)a.S * n2) return;
  const int si = (int)(tid / n2), pq = (int)(tid % n2);
  const int s = a.side_list ? a.side_list[si] : si;
  const int p = pq % n, q = pq / n;
  const int cs = a.side_case ? a.side_case[s] : 0;
  if (cs < 0) return;  // free side slot of a serving pool
  if (a.cases && a.cases[cs].dt == 0.0) return;  // a case that finished or sits this step out
  const CaseParams cp = case_params(a, cs);
  const int2 ee = a.side_e[s];
  const int sf = a.side_f[s];
  const int fM = sf & 15, fS = (sf >> 4) & 15, flip = sf >> 8;
  T sn[3], nu[3];
  if constexpr (sizeof(T) == sizeof(float)) {
    const float* nr = a.nrm32 + (size_t)s * 7 * n2 + pq;
    sn[0] = nr[0], sn[1] = nr[n2], sn[2] = nr[2 * n2];
    nu[0] = nr[3 * n2], nu[1] = nr[4 * n2], nu[2] = nr[5 * n2];
  } else {
    const double* nr = a.nrm + (size_t)s * 4 * n2 + pq;
    sn[0] = nr[0], sn[1] = nr[n2], sn[2] = nr[2 * n2];
    const double invd = 1.0 / nr[3 * n2];
    nu[0] = sn[0] * invd, nu[1] = sn[1] * invd, nu[2] = sn[2] * invd;
  }
  const int vM = face_vol_node<n>(fM, p, q);
  double UM[5];
  const double* uM = GL ? a.Ufc + (size_t)s * 10 * n2 + pq : a.U + (size_t)ee.x * 5 * n3 + vM;
  constexpr int ust = GL ? n2 : n3;
#pragma unroll
  for (int k = 0; k < 5; ++k) UM[k] = uM[k * ust];
  const SPrim<T> qM = shifted_prim<T>(UM, a.gm1, a.Rinv, cp);
  T qa[4];
  const int brow = a.side_bc ? a.side_bc[s] : -1;
  if (brow >= 0) {
    bc_lift_value<T>(a, cp, brow, UM, qM, nu, qa);  // boundary side: the condition's value
  } else {
    int ps, qs;
    flip_to_slave<n>(flip, p, q, ps, qs);
    const int vS = face_vol_node<n>(fS, ps, qs);
    double US[5];
    const double* uS = GL ? a.Ufc + (size_t)s * 10 * n2 + 5 * n2 + pq : a.U + (size_t)ee.y * 5 * n3 + vS;
#pragma unroll
    for (int k = 0; k < 5; ++k) US[k] = uS[k * ust];
    const SPrim<T> qS = shifted_prim<T>(US, a.gm1, a.Rinv, cp);
    qa[0] = T(0.5) * (qM.u + qS.u), qa[1] = T(0.5) * (qM.v + qS.v), qa[2] = T(0.5) * (qM.w + qS.w);
    qa[3] = T(0.5) * (qM.Tt + qS.Tt);
  }
  T* out = TBuf<T>::lflux(a) + (size_t)s * 12 * n2 + pq;
#pragma unroll
  for (int qv = 0; qv < 4; ++qv)
#pragma unroll
    for (int x = 0; x < 3; ++x) out[(qv * 3 + x) * n2] = qa[qv] * sn[x];
}

// ---------------------------------------------------------------------------
// Lifted gradients (weak form, Eq. lifting)
// ---------------------------------------------------------------------------
// FP64 shared-memory layout of k_lift (line tasks): the tables (Dhat, then
// for even n its even and odd half matrices), then per element the q planes
// (4), the metric planes (9) and the sums (12), each a padded node plane of
// n^3 + n^2 doubles (one pad after every line of n nodes: the tasks' 64-bit
// loads along any direction then fall in distinct banks)
template <int N, int EPB_ = 0>
struct Lift64Smem {
  using S = Shape<N, EPB_>;
  static constexpr int h = S::n / 2, Pn = S::n3 + S::n2;
  static constexpr int ntab = (S::n2 + 2 * h * h + 1) & ~1;
  static constexpr size_t bytes = sizeof(double) * (ntab + (size_t)S::EPB * 25 * Pn);
};

// The FP64 lifting (Eq. lifting, volume part, then the surface part and
// 1/J) by line tasks: per direction d, one task per (line, variable) loads
// the line's q and Ja^d once, forms the three products and applies Dhat;
// for even n through its even and odd half matrices (Dhat is
// centro-antisymmetric on LGL nodes: with e_j = P_j + P_(n-1-j) and
// o_j = P_j - P_(n-1-j), y_i = (De e)_i / 2 + (Do o)_i / 2 and
// y_(n-1-i) = (Do o)_i / 2 - (De e)_i / 2, with De_ij = Dhat_ij +
// Dhat_i(n-1-j) and Do_ij = Dhat_ij - Dhat_i(n-1-j)): 6 n + 3 n / 2 FP64
// operations per line and product column instead of n^2, where the lifting
// is bound by the FP64 unit.  The sums collect in shared memory (written for
// the first direction, added for the others).
template <int N, int EPB_>
__device__ __forceinline__ void lift_lines64(const StageArgs& a) {
  using S = Shape<N, EPB_>;
  using L = Lift64Smem<N, EPB_>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB, Pn = L::Pn, h = L::h;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* sD = reinterpret_cast<double*>(smraw);  // [n][n] Dhat
  double* sDe = sD + n2;                          // [h][h] even half
  double* sDo = sDe + h * h;                      // [h][h] odd half, each halved
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  double* q = sD + L::ntab + (size_t)le * 25 * Pn;  // [4][Pn] u, v, w, T'
  double* J = q + 4 * Pn;                           // [9][Pn] Ja^d_c
  double* W = J + 9 * Pn;                           // [12][Pn] the sums
  const int ei = blockIdx.x * EPB + le < a.E ? blockIdx.x * EPB + le : a.E - 1;
  const int e = a.elem_list ? a.elem_list[ei] : ei;
  const int ce = a.elem_case ? a.elem_case[e] : 0;
  const bool valid = blockIdx.x * EPB + le < a.E && ce >= 0;
  const bool busy = valid && !(a.cases && a.cases[ce].dt == 0.0);
  if (a.elem_case && __syncthreads_and(!busy)) return;
  const CaseParams cp = case_params(a, ce);
  for (int k = threadIdx.x; k < n2; k += blockDim.x) sD[k] = a.ops->Dhat[k];
  for (int k = threadIdx.x; k < h * h; k += blockDim.x) {
    const int i = k / h, j = k % h;
    const double* D = a.ops->Dhat + i * n;
    sDe[k] = 0.5 * (D[j] + D[n - 1 - j]);
    sDo[k] = 0.5 * (D[j] - D[n - 1 - j]);
  }
  const int vp = t + t / n;  // padded index of node t
  {
    double U[5];
    const double* u = a.U + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k] = u[k * n3];
    const SPrim<double> pr = shifted_prim<double>(U, a.gm1, a.Rinv, cp);
    q[vp] = pr.u, q[Pn + vp] = pr.v, q[2 * Pn + vp] = pr.w, q[3 * Pn + vp] = pr.Tt;
#pragma unroll
    for (int c = 0; c < 9; ++c) J[c * Pn + vp] = metric_at<double>(a, e, c, t, n3);
  }
  const double Ji = metric_at<double>(a, e, 9, t, n3);
  __syncwarp();
  __syncthreads();
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    const int sd = d == 0 ? 1 : (d == 1 ? n : n2);
    for (int task = t; task < 4 * n2; task += n3) {
      const int qv = task / n2, l = task % n2, lp = l % n, lq = l / n;
      const int bl = d == 0 ? n * (lp + n * lq) : (d == 1 ? lp + n2 * lq : lp + n * lq);
      double P0[n], P1[n], P2[n];
#pragma unroll
      for (int al = 0; al < n; ++al) {
        const int v = bl + al * sd, pv = v + v / n;
        const double qq = q[qv * Pn + pv];
        P0[al] = J[(3 * d) * Pn + pv] * qq;
        P1[al] = J[(3 * d + 1) * Pn + pv] * qq;
        P2[al] = J[(3 * d + 2) * Pn + pv] * qq;
      }
      auto put = [&](int i, double y0, double y1, double y2) {
        const int v = bl + i * sd;
        double* w = W + (qv * 3) * Pn + v + v / n;
        if (d == 0) {
          w[0] = y0, w[Pn] = y1, w[2 * Pn] = y2;
        } else {
          w[0] += y0, w[Pn] += y1, w[2 * Pn] += y2;
        }
      };
      if constexpr (n % 2 == 0) {
        double E0[h], E1[h], E2[h], O0[h], O1[h], O2[h];
#pragma unroll
        for (int j = 0; j < h; ++j) {
          E0[j] = P0[j] + P0[n - 1 - j], O0[j] = P0[j] - P0[n - 1 - j];
          E1[j] = P1[j] + P1[n - 1 - j], O1[j] = P1[j] - P1[n - 1 - j];
          E2[j] = P2[j] + P2[n - 1 - j], O2[j] = P2[j] - P2[n - 1 - j];
        }
#pragma unroll
        for (int i = 0; i < h; ++i) {
          double e0 = 0.0, e1 = 0.0, e2 = 0.0, p0 = 0.0, p1 = 0.0, p2 = 0.0;
#pragma unroll
          for (int j = 0; j < h; ++j) {
            const double ce = sDe[i * h + j], co = sDo[i * h + j];
            e0 += ce * E0[j], e1 += ce * E1[j], e2 += ce * E2[j];
            p0 += co * O0[j], p1 += co * O1[j], p2 += co * O2[j];
          }
          put(i, p0 + e0, p1 + e1, p2 + e2);
          put(n - 1 - i, p0 - e0, p1 - e1, p2 - e2);
        }
      } else {
#pragma unroll
        for (int i = 0; i < n; ++i) {
          double y0 = 0.0, y1 = 0.0, y2 = 0.0;
#pragma unroll
          for (int al = 0; al < n; ++al) {
            const double c = sD[i * n + al];
            y0 += c * P0[al], y1 += c * P1[al], y2 += c * P2[al];
          }
          put(i, y0, y1, y2);
        }
      }
    }
    __syncwarp();
    __syncthreads();
  }
  if (!valid) return;
  double acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = W[k * Pn + vp];
  // surface part: on LGL nodes only face nodes receive it
  const int idx[3] = {t % n, (t / n) % n, t / n2};
  const double* Lf = a.lflux;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id = idx[d];
    if (id != 0 && id != n - 1) continue;
    const int f = 2 * d + (id == n - 1 ? 1 : 0);
    const int es = a.elem_side[(size_t)e * 6 + f];
    const int s = es_side(es);
    const int p = d == 0 ? idx[1] : idx[0];
    const int qq = d == 2 ? idx[1] : idx[2];
    int pm = p, qm = qq;
    if (es_slave(es)) flip_to_master<n>(es_flip(es), p, qq, pm, qm);
    const double sg = es_slave(es) ? -a.ops->winv[id] : a.ops->winv[id];
    const double* Lr = Lf + (size_t)s * 12 * n2 + pm + n * qm;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] += sg * Lr[k * n2];
  }
  double* g = a.g + (size_t)e * 12 * n3 + t;
#pragma unroll
  for (int k = 0; k < 12; ++k) g[k * n3] = acc[k] * Ji;
}

template <int N, typename T, int EPB_ = 0>
__global__ void __launch_bounds__(Shape<N, EPB_>::THREADS) k_lift(StageArgs a) {
  if constexpr (sizeof(T) == sizeof(double)) {
    lift_lines64<N, EPB_>(a);
    return;
  }
  using S = Shape<N, EPB_>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  constexpr int n2p = (n2 + 3) & ~3;  // keeps the arrays below 16-byte aligned
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sDh = reinterpret_cast<T*>(smraw);  // [n2p]
  T* sq = sDh + n2p;                     // [EPB][4][n3]
  T* sF = sq + EPB * 4 * n3;             // [EPB][12][n3]
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  // Slots past the last element redo the last element in their own shared
  // memory slot, so that every thread of a block runs the same path through
  // the barriers; only the final global stores are masked.
  const int ei = blockIdx.x * EPB + le < a.E ? blockIdx.x * EPB + le : a.E - 1;
  const int e = a.elem_list ? a.elem_list[ei] : ei;
  const int ce = a.elem_case ? a.elem_case[e] : 0;
  // free element slots of a serving pool compute on whatever they hold and
  // store nothing, like the slots past the last element
  const bool valid = blockIdx.x * EPB + le < a.E && ce >= 0;
  // a block of free pool slots, or of cases that have reached their end time
  // (time step 0), only leaves (every thread takes this barrier)
  const bool busy = valid && !(a.cases && a.cases[ce].dt == 0.0);
  if (a.elem_case && __syncthreads_and(!busy)) return;
  const CaseParams cp = case_params(a, ce);
  for (int k = threadIdx.x; k < n2; k += blockDim.x) sDh[k] = T(a.ops->Dhat[k]);
  T* q = sq + le * 4 * n3;
  T* F = sF + le * 12 * n3;
  // FP32: the node's ten metric values are loaded up front, so that their
  // latency overlaps the state loads instead of following each barrier
  constexpr bool pre = sizeof(T) == sizeof(float);
  T Mpre[pre ? 10 : 1];
  if constexpr (pre) {
#pragma unroll
    for (int c = 0; c < 10; ++c) Mpre[c] = metric_at<T>(a, e, c, t, n3);
  }
  auto Mv = [&](int c) -> T {
    if constexpr (pre) return Mpre[c];
    else return metric_at<T>(a, e, c, t, n3);
  };
  {
    double U[5];
    const double* u = a.U + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k] = u[k * n3];
    const SPrim<T> pr = shifted_prim<T>(U, a.gm1, a.Rinv, cp);
    q[t] = pr.u;
    q[n3 + t] = pr.v;
    q[2 * n3 + t] = pr.w;
    q[3 * n3 + t] = pr.Tt;
  }
  __syncwarp();
  __syncthreads();
  const int idx[3] = {t % n, (t / n) % n, t / n2};
  constexpr int str[3] = {1, n, n2};
  T acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = T(0);
  // FP32 (bound by shared-memory load instructions): the products are stored
  // as six float2 planes, halving the loads of the line sums
  constexpr bool pairs2 = sizeof(T) == sizeof(float);
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    {
      const T J0 = Mv(d * 3 + 0), J1 = Mv(d * 3 + 1), J2 = Mv(d * 3 + 2);
      T pr[12];
#pragma unroll
      for (int qv = 0; qv < 4; ++qv) {
        const T qq = q[qv * n3 + t];
        pr[qv * 3 + 0] = J0 * qq;
        pr[qv * 3 + 1] = J1 * qq;
        pr[qv * 3 + 2] = J2 * qq;
      }
      if constexpr (pairs2) {
        float2* F2 = reinterpret_cast<float2*>(F);
#pragma unroll
        for (int k = 0; k < 6; ++k) F2[k * n3 + t] = make_float2(pr[2 * k], pr[2 * k + 1]);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) F[k * n3 + t] = pr[k];
      }
    }
    __syncwarp();
    __syncthreads();
    {
      const int id = idx[d], base = t - id * str[d];
#pragma unroll
      for (int al = 0; al < n; ++al) {
        const T c = sDh[id * n + al];
        const int nb = base + al * str[d];
        if constexpr (pairs2) {
          const float2* F2 = reinterpret_cast<const float2*>(F);
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            const float2 v = F2[k * n3 + nb];
            acc[2 * k] += c * v.x;
            acc[2 * k + 1] += c * v.y;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 12; ++k) acc[k] += c * F[k * n3 + nb];
        }
      }
    }
    __syncwarp();
    __syncthreads();
  }
  if (!valid) return;
  // surface part: on LGL nodes only face nodes receive it
  const T* Lf = TBuf<T>::lflux(a);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id = idx[d];
    if (id != 0 && id != n - 1) continue;
    const int f = 2 * d + (id == n - 1 ? 1 : 0);
    const int es = a.elem_side[(size_t)e * 6 + f];
    const int s = es_side(es);
    const int p = d == 0 ? idx[1] : idx[0];
    const int qq = d == 2 ? idx[1] : idx[2];
    int pm = p, qm = qq;
    if (es_slave(es)) flip_to_master<n>(es_flip(es), p, qq, pm, qm);
    const T sg = T(es_slave(es) ? -a.ops->winv[id] : a.ops->winv[id]);
    const T* L = Lf + (size_t)s * 12 * n2 + pm + n * qm;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] += sg * L[k * n2];
  }
  const T Ji = Mv(9);
  T* g = TBuf<T>::g(a) + (size_t)e * 12 * n3 + t;
#pragma unroll
  for (int k = 0; k < 12; ++k) g[k * n3] = acc[k] * Ji;
}

// ---------------------------------------------------------------------------
// FillFlux: Riemann flux + BR1 viscous flux, times the surface element
// ---------------------------------------------------------------------------
// GL: states and lifted gradients from the ProlongToFace arrays
template <int N, typename T, bool GL = false>
__global__ void __launch_bounds__(256) k_surf_flux(StageArgs a) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)a.S * n2) return;
  const int si = (int)(tid / n2), pq = (int)(tid % n2);
  const int s = a.side_list ? a.side_list[si] : si;
  const int p = pq % n, q = pq / n;
  const int cs = a.side_case ? a.side_case[s] : 0;
  if (cs < 0) return;  // free side slot of a serving pool
  if (a.cases && a.cases[cs].dt == 0.0) return;  // a case that finished or sits this step out
  const CaseParams cp = case_params(a, cs);
  const int2 ee = a.side_e[s];
  const int sf = a.side_f[s];
  const int fM = sf & 15, fS = (sf >> 4) & 15, flip = sf >> 8;
  T sn[3], nu[3], sA;
  if constexpr (sizeof(T) == sizeof(float)) {
    const float* nr = a.nrm32 + (size_t)s * 7 * n2 + pq;
    sn[0] = nr[0], sn[1] = nr[n2], sn[2] = nr[2 * n2];
    nu[0] = nr[3 * n2], nu[1] = nr[4 * n2], nu[2] = nr[5 * n2];
    sA = nr[6 * n2];
  } else {
    const double* nr = a.nrm + (size_t)s * 4 * n2 + pq;
    sn[0] = nr[0], sn[1] = nr[n2], sn[2] = nr[2 * n2];
    const double sAd = nr[3 * n2];
    const double invd = 1.0 / sAd;
    sA = sAd;
    nu[0] = nr[0] * invd, nu[1] = nr[n2] * invd, nu[2] = nr[2 * n2] * invd;
  }
  const int vM = face_vol_node<n>(fM, p, q);
  double UM[5];
  const double* uM = GL ? a.Ufc + (size_t)s * 10 * n2 + pq : a.U + (size_t)ee.x * 5 * n3 + vM;
  constexpr int ust = GL ? n2 : n3;
#pragma unroll
  for (int k = 0; k < 5; ++k) UM[k] = uM[k * ust];
  const SPrim<T> qM = shifted_prim<T>(UM, a.gm1, a.Rinv, cp);
  const T* G = TBuf<T>::g(a);
  const T* Gf = TBuf<T>::gfc(a);
  T f[5];
  const int brow = a.side_bc ? a.side_bc[s] : -1;
  if (brow >= 0) {  // boundary side
    T gM[12];
    if (a.viscous) {
      const T* pgM = GL ? Gf + (size_t)s * 24 * n2 + pq : G + (size_t)ee.x * 12 * n3 + vM;
#pragma unroll
      for (int k = 0; k < 12; ++k) gM[k] = pgM[k * ust];
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) gM[k] = T(0);
    }
    bc_flux<T>(a, cp, brow, UM, qM, gM, nu, sA, sn, f);
  } else {
    int ps, qs;
    flip_to_slave<n>(flip, p, q, ps, qs);
    const int vS = face_vol_node<n>(fS, ps, qs);
    double US[5];
    const double* uS = GL ? a.Ufc + (size_t)s * 10 * n2 + 5 * n2 + pq : a.U + (size_t)ee.y * 5 * n3 + vS;
#pragma unroll
    for (int k = 0; k < 5; ++k) US[k] = uS[k * ust];
    const SPrim<T> qS = shifted_prim<T>(US, a.gm1, a.Rinv, cp);
    if (cp.riemann == DG_RIEMANN_ROE) roe_flux_s(qM, qS, nu, pick<T>(a.gm1, a.f_gm1), pick<T>(cp.Hr, cp.fHr), f);
    else lf_flux_s(qM, qS, nu, pick<T>(a.gamma, a.f_gamma), pick<T>(cp.pr, cp.fpr), f);
#pragma unroll
    for (int k = 0; k < 5; ++k) f[k] *= sA;
    if (a.viscous) {
      T gM[12], gS[12];
      const T* pgM = GL ? Gf + (size_t)s * 24 * n2 + pq : G + (size_t)ee.x * 12 * n3 + vM;
      const T* pgS = GL ? Gf + (size_t)s * 24 * n2 + 12 * n2 + pq : G + (size_t)ee.y * 12 * n3 + vS;
#pragma unroll
      for (int k = 0; k < 12; ++k) { gM[k] = pgM[k * ust]; gS[k] = pgS[k * ust]; }
      T tau[6], W[3], fvM[4], fvS[4], vmu, vlam;
      visc_coeffs<T>(a, cp, qM.Tt, vmu, vlam);
      viscous_parts(gM, qM.u, qM.v, qM.w, vmu, vlam, tau, W);
      viscous_flux_n(tau, W, sn, fvM);
      visc_coeffs<T>(a, cp, qS.Tt, vmu, vlam);
      viscous_parts(gS, qS.u, qS.v, qS.w, vmu, vlam, tau, W);
      viscous_flux_n(tau, W, sn, fvS);
#pragma unroll
      for (int k = 0; k < 4; ++k) f[1 + k] -= T(0.5) * (fvM[k] + fvS[k]);
    }
  }
  T* out = TBuf<T>::fstar(a) + (size_t)s * 5 * n2 + pq;
#pragma unroll
  for (int k = 0; k < 5; ++k) out[k * n2] = f[k];
}

// ---------------------------------------------------------------------------
// Hennemann indicator on rho p (modal energy of the top modes), Sec. 2.3, in
// FP64 on both paths.  Every thread of the element runs the same
// instructions (no single-thread branch in front of a barrier): row sums are
// formed by all threads (rows are formed twice or more, with identical
// values), then every thread adds the row sums itself.
// sT1 / sT2: n3 doubles each, sRow: 4 n2 doubles.
// ---------------------------------------------------------------------------
template <int n>
__device__ double element_alpha(double rp, double* sT1, double* sT2, double* sRow, const double* sVinv, int t,
                                double amin, double amax) {
  constexpr int n2 = n * n, N = n - 1;
  const int i = t % n, j = (t / n) % n, k = t / n2;
  sT1[t] = rp;
  __syncwarp();
  __syncthreads();
  double s = 0.0;
  for (int x = 0; x < n; ++x) s += sVinv[i * n + x] * sT1[x + n * (j + n * k)];
  sT2[t] = s;
  __syncwarp();
  __syncthreads();
  s = 0.0;
  for (int x = 0; x < n; ++x) s += sVinv[j * n + x] * sT2[i + n * (x + n * k)];
  sT1[t] = s;
  __syncwarp();
  __syncthreads();
  s = 0.0;
  for (int x = 0; x < n; ++x) s += sVinv[k * n + x] * sT1[i + n * (j + n * x)];
  sT2[t] = s * s;  // energy of mode (i, j, k)
  __syncwarp();
  __syncthreads();
  {
    // row r = (j, k): sums over i by the maximum degree max(i, j, k)
    const int r = t % n2, rj = r % n, rk = r / n;
    double mN = 0, mN1 = 0, tot = 0, tot1 = 0;
    for (int x = 0; x < n; ++x) {
      const int dv = max(x, max(rj, rk));
      const double m2 = sT2[x + n * r];
      tot += m2;
      tot1 += dv <= N - 1 ? m2 : 0.0;
      mN += dv == N ? m2 : 0.0;
      mN1 += dv == N - 1 ? m2 : 0.0;
    }
    sRow[r] = mN;
    sRow[n2 + r] = mN1;
    sRow[2 * n2 + r] = tot;
    sRow[3 * n2 + r] = tot1;
  }
  __syncwarp();
  __syncthreads();
  double mN = 0, mN1 = 0, tot = 0, tot1 = 0;
  for (int r = 0; r < n2; ++r) {
    mN += sRow[r];
    mN1 += sRow[n2 + r];
    tot += sRow[2 * n2 + r];
    tot1 += sRow[3 * n2 + r];
  }
  const double e1 = tot > 0 ? mN / tot : 0.0;
  const double e2 = tot1 > 0 ? mN1 / tot1 : 0.0;
  const double E = e1 > e2 ? e1 : e2;
  const double T = 0.5 * pow(10.0, -1.8 * pow((double)(N + 1), 0.25));
  const double sh = log((1.0 - 1e-4) / 1e-4);
  double al = 1.0 / (1.0 + exp(-sh * (E - T) / T));
  if (al < amin) al = 0.0;
  if (al > amax) al = amax;
  __syncwarp();
  __syncthreads();  // sT1 / sT2 / sRow may be reused after this
  return al;
}

// shared-memory layout of k_volume: FP64 part first, then the T arrays
template <int N, typename T, int EPB_ = 0, bool PAIRS = sizeof(T) == sizeof(double)>
struct VolumeSmem {
  using S = Shape<N, EPB_>;
  // FP32: node-major primitives (float4 + float2) and metrics (one float4 per
  // direction), so a partner is read with three loads
  static constexpr bool aos = sizeof(T) == sizeof(float);
  static_assert(!(aos && PAIRS), "the line-pair two-point sums are an FP64 mapping");
  static constexpr int n2p = (S::n2 + 3) & ~3;
  static constexpr int nJ = aos ? 12 : 9;
  // Vinv, indicator scratch, FP32: the node's state and RK register copied in
  // asynchronously (even count: the T arrays start 16-byte aligned)
  static constexpr int nUd = aos ? 10 * S::n3 : 0;
  static constexpr size_t n_dbl = (S::n2 + S::EPB * (2 * S::n3 + 4 * S::n2 + nUd) + 1) & ~size_t(1);
  // per-element stride of the primitives: a multiple of 4 floats in FP32, so
  // that every element's float4 view starts 16-byte aligned
  static constexpr int pstride = aos ? 6 * ((S::n3 + 3) & ~3) : 6 * S::n3;
  // viscous / FV fluxes: FP32 keeps the four viscous components of a node in
  // one float4 (element stride padded like the primitives)
  static constexpr int gstride = aos ? 5 * ((S::n3 + 3) & ~3) : 5 * S::n3;
  // per-direction two-point sums: only the line-pair tasks need them (the
  // per-node sums stay in registers)
  static constexpr int nA = PAIRS ? 15 : 0;
  static constexpr size_t n_t = 2 * n2p + S::EPB * (pstride + nJ * S::n3 + gstride + nA * S::n3);
  static constexpr size_t bytes = sizeof(double) * n_dbl + sizeof(T) * n_t;
};

// ---------------------------------------------------------------------------
// Volume integral + SurfInt + ApplyJac (+ RK update)
// ---------------------------------------------------------------------------
// PAIRS: each unordered pair of a line forms its two-point flux once (one
// task per line, FP64); otherwise each node sums over all its partners.
template <int N, int MODE, typename T, int EPB_ = 0, bool PAIRS = sizeof(T) == sizeof(double)>
__global__ void __launch_bounds__(Shape<N, EPB_>::THREADS, Shape<N, EPB_>::template vol_min_blocks<T>())
    k_volume(StageArgs a) {
  using S = Shape<N, EPB_>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ __align__(16) unsigned char smraw[];
  using L = VolumeSmem<N, T, EPB_, PAIRS>;
  constexpr bool aos = L::aos;
  double* sVi = reinterpret_cast<double*>(smraw);  // [n2] Vinv (FP64)
  double* sX = sVi + n2;                           // [EPB][2 n3 + 4 n2] indicator scratch (FP64)
  T* sDs = reinterpret_cast<T*>(reinterpret_cast<double*>(smraw) + L::n_dbl);  // [n2] Dsplit
  T* sDh = sDs + L::n2p;                                                       // [n2] Dhat
  T* sP = sDh + L::n2p;                  // [EPB][6][n3] rho u v w p' H', halved (FP32: [n3] float4 + [n3] float2)
  T* sJ = sP + EPB * L::pstride;         // [EPB][9][n3] metrics, halved (FP32: [3][n3] float4)
  T* sG = sJ + EPB * L::nJ * n3;         // [EPB][5][n3] viscous / FV fluxes (FP32 viscous: [n3] float4)
  T* sA = sG + EPB * L::gstride;         // [EPB][3][5][n3] two-point sums (FP64 only)
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  double* sUd = sX + EPB * (2 * n3 + 4 * n2) + le * L::nUd;  // FP32: [2][5][n3] U and dU of the element
  // slots past the last element redo the last element, free slots of a
  // serving pool compute on what they hold; neither stores (see k_lift)
  const int ei = blockIdx.x * EPB + le < a.E ? blockIdx.x * EPB + le : a.E - 1;
  const int e = a.elem_list ? a.elem_list[ei] : ei;
  const int ce = a.elem_case ? a.elem_case[e] : 0;
  const bool valid = blockIdx.x * EPB + le < a.E && ce >= 0;
  // a block of free pool slots, or of cases that have reached their end time
  // (time step 0), only leaves (every thread takes this barrier)
  const bool busy = valid && !(a.cases && a.cases[ce].dt == 0.0);
  if (a.elem_case && __syncthreads_and(!busy)) return;
  const CaseParams cp = case_params(a, ce);
  for (int k = threadIdx.x; k < n2; k += blockDim.x) {
    sDs[k] = T(a.ops->Dsplit[k]);
    sDh[k] = T(a.ops->Dhat[k]);
    sVi[k] = a.ops->Vinv[k];
  }
  T* P = sP + le * L::pstride;
  T* Jm = sJ + le * L::nJ * n3;
  T* G = sG + le * L::gstride;
  float4* G4 = reinterpret_cast<float4*>(G);
  // FP32 views of the same memory
  float4* P4 = reinterpret_cast<float4*>(P);
  float2* P2 = reinterpret_cast<float2*>(P + 4 * n3);
  float4* J4 = reinterpret_cast<float4*>(Jm);
  // halved metric component c of direction d at a node
  auto Jc = [&](int d, int c, int node) -> T {
    if constexpr (aos) return reinterpret_cast<const float*>(J4 + d * n3 + node)[c];
    else return Jm[(d * 3 + c) * n3 + node];
  };
  T* A = sA + le * L::nA * n3;
  const double H_ref = cp.Hr;
  double U[5];
  double p_full;
  SPrim<T> me;
  T g[12];
  {
    const double* u = a.U + (size_t)e * 5 * n3 + t;
    if constexpr (aos) {
      // the state now, the RK register (read only at the end) in a second group
#pragma unroll
      for (int k = 0; k < 5; ++k) cp_async8(sUd + k * n3 + t, u + k * n3);
      cp_async_commit();
      if (MODE == 1 && !a.first_stage) {
        const double* du = a.dU + (size_t)e * 5 * n3 + t;
#pragma unroll
        for (int k = 0; k < 5; ++k) cp_async8(sUd + (5 + k) * n3 + t, du + k * n3);
      }
      cp_async_commit();
      cp_async_wait<1>();
#pragma unroll
      for (int k = 0; k < 5; ++k) U[k] = sUd[k * n3 + t];
    } else {
#pragma unroll
      for (int k = 0; k < 5; ++k) U[k] = u[k * n3];
    }
    me = shifted_prim<T, true>(U, a.gm1, a.Rinv, cp, &p_full);
    // halved values: every arithmetic mean of the two-point flux is then one
    // addition, bit-identical to (a + b) / 2
    if constexpr (aos) {
      P4[t] = make_float4(0.5f * me.rho, 0.5f * me.u, 0.5f * me.v, 0.5f * me.w);
      P2[t] = make_float2(0.5f * me.p, 0.5f * me.H);
#pragma unroll
      for (int d = 0; d < 3; ++d)
        J4[d * n3 + t] = make_float4(0.5f * metric_at<T>(a, e, 3 * d, t, n3), 0.5f * metric_at<T>(a, e, 3 * d + 1, t, n3),
                                     0.5f * metric_at<T>(a, e, 3 * d + 2, t, n3), 0.0f);
    } else {
      P[t] = T(0.5) * me.rho;
      P[n3 + t] = T(0.5) * me.u;
      P[2 * n3 + t] = T(0.5) * me.v;
      P[3 * n3 + t] = T(0.5) * me.w;
      P[4 * n3 + t] = T(0.5) * me.p;
      P[5 * n3 + t] = T(0.5) * me.H;
#pragma unroll
      for (int c = 0; c < 9; ++c) Jm[c * n3 + t] = T(0.5) * metric_at<T>(a, e, c, t, n3);
    }
    if (a.viscous) {
      const T* pg = TBuf<T>::g(a) + (size_t)e * 12 * n3 + t;
#pragma unroll
      for (int k = 0; k < 12; ++k) g[k] = pg[k * n3];
    }
  }
  __syncwarp();
  __syncthreads();
  const int idx[3] = {t % n, (t / n) % n, t / n2};
  constexpr int str[3] = {1, n, n2};
  T accC[5] = {0, 0, 0, 0, 0};  // convective DG volume term
  T acc[5] = {0, 0, 0, 0, 0};   // viscous volume + surface terms
  T tau[6] = {0, 0, 0, 0, 0, 0}, W[3] = {0, 0, 0};
  if (a.viscous) {
    T vmu, vlam;
    visc_coeffs<T>(a, cp, me.Tt, vmu, vlam);
    viscous_parts(g, me.u, me.v, me.w, vmu, vlam, tau, W);
  }
  // ---- split-form KEP volume integral ----
  // FP64 (bound by the FP64 pipe): one line per task; every unordered pair
  // (i, alpha) of the line forms the symmetric two-point flux once and adds
  // Dsplit_{i alpha} f to node i and Dsplit_{alpha i} f to node alpha, which
  // halves the flux evaluations.  FP32 (bound by latency, not arithmetic):
  // one node per thread over all its partners, which keeps every thread busy.
  // Each direction has its own sum array.
  constexpr bool kPairs = PAIRS;
  if constexpr (!kPairs) {
    const int idl[3] = {t % n, (t / n) % n, t / n2};
    // halved primitives and direction-d metrics of a node, either layout
    auto node = [&](int d, int v, T& r, T& u0, T& u1, T& u2, T& pp, T& H, T& j0, T& j1, T& j2) {
      if constexpr (aos) {
        const float4 a4 = P4[v];
        const float2 a2 = P2[v];
        const float4 jj = J4[d * n3 + v];
        r = a4.x, u0 = a4.y, u1 = a4.z, u2 = a4.w, pp = a2.x, H = a2.y, j0 = jj.x, j1 = jj.y, j2 = jj.z;
      } else {
        r = P[v], u0 = P[n3 + v], u1 = P[2 * n3 + v], u2 = P[3 * n3 + v], pp = P[4 * n3 + v], H = P[5 * n3 + v];
        j0 = Jm[(d * 3) * n3 + v], j1 = Jm[(d * 3 + 1) * n3 + v], j2 = Jm[(d * 3 + 2) * n3 + v];
      }
    };
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      const int id = idl[d], base = t - id * str[d];
      T ri, ui, vvi, wi, pi, Hi, j0, j1, j2;
      node(d, t, ri, ui, vvi, wi, pi, Hi, j0, j1, j2);
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0), s4 = T(0);
#pragma unroll
      for (int al = 0; al < n; ++al) {
        if (al == id) continue;
        const int va = base + al * str[d];
        T ra, ua, va_, wa, pa, Ha, ja0, ja1, ja2;
        node(d, va, ra, ua, va_, wa, pa, Ha, ja0, ja1, ja2);
        const T m0 = j0 + ja0, m1 = j1 + ja1, m2 = j2 + ja2;
        const T rho = ri + ra;
        const T u0 = ui + ua, u1 = vvi + va_, u2 = wi + wa;
        const T pp = pi + pa;
        const T H = Hi + Ha;
        const T fr = rho * (u0 * m0 + u1 * m1 + u2 * m2);
        const T dv = sDs[id * n + al];
        s0 += dv * fr;
        s1 += dv * (fr * u0 + pp * m0);
        s2 += dv * (fr * u1 + pp * m1);
        s3 += dv * (fr * u2 + pp * m2);
        s4 += dv * (fr * H);
      }
      // same association as the line-pair path's (A_0 + A_1) + A_2
      if (d == 0) {
        accC[0] = s0, accC[1] = s1, accC[2] = s2, accC[3] = s3, accC[4] = s4;
      } else {
        accC[0] += s0, accC[1] += s1, accC[2] += s2, accC[3] += s3, accC[4] += s4;
      }
    }
  }
  if constexpr (kPairs)
  for (int lt = t; lt < 3 * n2; lt += n3) {
    const int d = lt / n2, line = lt % n2;
    const int lp = line % n, lq = line / n;
    const int base = d == 0 ? n * (lp + n * lq) : (d == 1 ? lp + n2 * lq : lp + n * lq);
    const int st = d == 0 ? 1 : (d == 1 ? n : n2);
    const T* J0 = Jm + (d * 3 + 0) * n3;
    const T* J1 = Jm + (d * 3 + 1) * n3;
    const T* J2 = Jm + (d * 3 + 2) * n3;
    // this task is the only writer of the line's nodes in direction d's array:
    // node i keeps its sums in registers, partner contributions go straight
    // to shared memory
    T* Ad = A + d * 5 * n3;
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
      for (int k = 0; k < 5; ++k) Ad[k * n3 + base + i * st] = T(0);
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const int vi = base + i * st;
      const T ri = P[vi], ui = P[n3 + vi], vvi = P[2 * n3 + vi], wi = P[3 * n3 + vi];
      const T pi = P[4 * n3 + vi], Hi = P[5 * n3 + vi];
      const T j0 = J0[vi], j1 = J1[vi], j2 = J2[vi];
      T ai0 = T(0), ai1 = T(0), ai2 = T(0), ai3 = T(0), ai4 = T(0);
#pragma unroll
      for (int al = i + 1; al < n; ++al) {
        const int va = base + al * st;
        const T m0 = j0 + J0[va], m1 = j1 + J1[va], m2 = j2 + J2[va];
        const T rho = ri + P[va];
        const T u0 = ui + P[n3 + va], u1 = vvi + P[2 * n3 + va], u2 = wi + P[3 * n3 + va];
        const T pp = pi + P[4 * n3 + va];
        const T H = Hi + P[5 * n3 + va];
        const T fr = rho * (u0 * m0 + u1 * m1 + u2 * m2);
        const T f1 = fr * u0 + pp * m0, f2 = fr * u1 + pp * m1, f3 = fr * u2 + pp * m2, f4 = fr * H;
        const T dia = sDs[i * n + al], dai = sDs[al * n + i];
        ai0 += dia * fr;
        ai1 += dia * f1;
        ai2 += dia * f2;
        ai3 += dia * f3;
        ai4 += dia * f4;
        Ad[va] += dai * fr;
        Ad[n3 + va] += dai * f1;
        Ad[2 * n3 + va] += dai * f2;
        Ad[3 * n3 + va] += dai * f3;
        Ad[4 * n3 + va] += dai * f4;
      }
      Ad[vi] += ai0;
      Ad[n3 + vi] += ai1;
      Ad[2 * n3 + vi] += ai2;
      Ad[3 * n3 + vi] += ai3;
      Ad[4 * n3 + vi] += ai4;
    }
  }

  // ---- viscous volume term: collocated weak form, per direction ----
  if (a.viscous) {
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      {
        const T nv[3] = {T(2) * Jc(d, 0, t), T(2) * Jc(d, 1, t), T(2) * Jc(d, 2, t)};
        T fv[4];
        viscous_flux_n(tau, W, nv, fv);
        if constexpr (aos) {
          G4[t] = make_float4(fv[0], fv[1], fv[2], fv[3]);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) G[k * n3 + t] = fv[k];
        }
      }
      __syncwarp();
      __syncthreads();
      {
        const int id = idx[d], base = t - id * str[d];
#pragma unroll
        for (int al = 0; al < n; ++al) {
          const T c = sDh[id * n + al];
          const int nb = base + al * str[d];
          if constexpr (aos) {
            const float4 gv = G4[nb];
            acc[1] -= c * gv.x;
            acc[2] -= c * gv.y;
            acc[3] -= c * gv.z;
            acc[4] -= c * gv.w;
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[1 + k] -= c * G[k * n3 + nb];
          }
        }
      }
      __syncwarp();
      __syncthreads();
    }
  }
  __syncwarp();
  __syncthreads();
  if constexpr (kPairs) {
#pragma unroll
    for (int k = 0; k < 5; ++k) accC[k] = (A[k * n3 + t] + A[(5 + k) * n3 + t]) + A[(10 + k) * n3 + t];
  }

  // ---- shock capturing: indicator and FV sub-cell blending (Sec. 2.3) ----
  if (a.shock) {
    double al;
    if (a.alpha_force >= 0) {
      al = a.alpha_force;
    } else {
      double* X1 = sX + le * (2 * n3 + 4 * n2);
      // all threads of the block take part in the barriers inside
      al = element_alpha<n>(U[0] * p_full, X1, X1 + n3, X1 + 2 * n3, sVi, t, a.alpha_min, a.alpha_max);
    }
    if (valid && t == 0) a.alpha[e] = al;
    // block-uniform condition: the FV pass has barriers, and the elements of
    // one block may have different blending factors
    if (__syncthreads_or(al > 0)) {
      T vfv[5] = {0, 0, 0, 0, 0};
      const double* FVm = a.fvmetric + (size_t)e * 3 * (n - 1) * 3 * n2;
#pragma unroll 1
      for (int d = 0; d < 3; ++d) {
        const int id = idx[d];
        // the flux through interface id + 1/2 is formed by the node on its
        // left; the last node of a line forms a dummy one (same instructions
        // for every thread) that is not stored
        const bool right = id < n - 1;
        const int line = d == 0 ? idx[1] + n * idx[2] : (d == 1 ? idx[0] + n * idx[2] : idx[0] + n * idx[1]);
        const double* fm = FVm + (size_t)(d * (n - 1) + (right ? id : n - 2)) * 3 * n2 + line;
        const double mv[3] = {fm[0], fm[n2], fm[2 * n2]};
        const double sAd = sqrt(mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2]);
        const T nu[3] = {T(mv[0] / sAd), T(mv[1] / sAd), T(mv[2] / sAd)};
        const int nb = right ? t + str[d] : t;
        double UR[5];
        const double* ur = a.U + (size_t)e * 5 * n3 + nb;
#pragma unroll
        for (int k = 0; k < 5; ++k) UR[k] = ur[k * n3];
        const SPrim<T> qR = shifted_prim<T>(UR, a.gm1, a.Rinv, cp);
        T fb[5];
        lf_flux_s(me, qR, nu, pick<T>(a.gamma, a.f_gamma), pick<T>(cp.pr, cp.fpr), fb);
        if (right) {
#pragma unroll
          for (int k = 0; k < 5; ++k) G[k * n3 + t] = fb[k] * T(sAd);
        }
        __syncwarp();
        __syncthreads();
        if (right) {
#pragma unroll
          for (int k = 0; k < 5; ++k) vfv[k] += G[k * n3 + t] / T(a.ops->w[id]);
        }
        if (id > 0) {
          const int nl = t - str[d];
#pragma unroll
          for (int k = 0; k < 5; ++k) vfv[k] -= G[k * n3 + nl] / T(a.ops->w[id]);
        }
        __syncwarp();
        __syncthreads();
      }
      if (al > 0) {
        const T alt = T(al);
#pragma unroll
        for (int k = 0; k < 5; ++k) accC[k] = (1 - alt) * accC[k] + alt * vfv[k];
      }
    }
  }
  if constexpr (aos) cp_async_wait<0>();
  if (!valid) return;
  // a serving case that finished or sits this step out keeps its state (its
  // surface fluxes were not formed this step)
  if (MODE == 1 && a.cases && a.cases[ce].dt == 0.0) return;

  // ---- SurfInt: face nodes receive +-f* lhat ----
  const T* Fst = TBuf<T>::fstar(a);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id = idx[d];
    if (id != 0 && id != n - 1) continue;
    const int f = 2 * d + (id == n - 1 ? 1 : 0);
    const int es = a.elem_side[(size_t)e * 6 + f];
    const int s = es_side(es);
    const int p = d == 0 ? idx[1] : idx[0];
    const int qq = d == 2 ? idx[1] : idx[2];
    int pm = p, qm = qq;
    if (es_slave(es)) flip_to_master<n>(es_flip(es), p, qq, pm, qm);
    const T sg = T(es_slave(es) ? -a.ops->winv[id] : a.ops->winv[id]);
    const T* Fs = Fst + (size_t)s * 5 * n2 + pm + n * qm;
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += sg * Fs[k * n2];
  }
  // ---- ApplyJac; the energy equation gets H_ref times the mass equation back ----
  // in the arithmetic type (FP32-bulk: 1/J rounded to FP32 scales all five
  // components alike); the H_ref part of the energy equation in FP64
  const T Ji = metric_at<T>(a, e, 9, t, n3);
  double Ut[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) Ut[k] = to_f64<T>(-(accC[k] + acc[k]) * Ji);
  Ut[4] += H_ref * Ut[0];
  if (a.sponge_sigma) {  // sponge source -sigma (U - U_base), FP64
    const double sg = a.sponge_sigma[(size_t)e * n3 + t];
    const double* ub = a.sponge_base + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) Ut[k] -= sg * ((aos ? sUd[k * n3 + t] : U[k]) - ub[k * n3]);
  }
  if (a.source) {  // manufactured-solution source, FP64
    double Q[5];
    mms_source(a, a.xyzs + ((size_t)e * n3 + t) * 3, stage_time(a, MODE), Q);
#pragma unroll
    for (int k = 0; k < 5; ++k) Ut[k] += Q[k];
  }
  if (MODE == 0) {
    double* o = a.Ut + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) o[k * n3] = Ut[k];
  } else {
    const double dt = case_dt(a, ce);
    double* du = a.dU + (size_t)e * 5 * n3 + t;
    double* uo = a.Urk + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      // FP32-bulk: the state and the RK register from the shared-memory copies
      const double duk = aos ? sUd[(5 + k) * n3 + t] : du[k * n3];
      const double uk = aos ? sUd[k * n3 + t] : U[k];
      const double r = a.first_stage ? dt * Ut[k] : a.rkA * duk + dt * Ut[k];
      du[k * n3] = r;
      uo[k * n3] = uk + a.rkB * r;
    }
  }
}

}  // namespace dg

#include "dg_stage_gl.cuh"
#include "dg_fused32.cuh"

namespace dg {

// ---------------------------------------------------------------------------
// host side: launch arguments, shared-memory sizes, one RHS evaluation
// ---------------------------------------------------------------------------
inline StageArgs make_stage_args(dg_ctx* c, const double* U) {
  StageArgs a{};
  a.E = (int)c->E;
  a.S = (int)c->S;
  a.U = U;
  a.metric = c->metric;
  a.metric32 = c->metric32;
  a.nrm = c->nrm;
  a.nrm32 = c->nrm32;
  a.elem_side = c->elem_side;
  a.side_e = c->side_e;
  a.side_f = c->side_f;
  a.g = c->g;
  a.lflux = c->lflux;
  a.fstar = c->fstar;
  a.g32 = c->g32;
  a.lflux32 = c->lflux32;
  a.fstar32 = c->fstar32;
  a.alpha = c->alpha;
  a.fvmetric = c->fvmetric;
  a.ops = c->ops;
  a.gamma = c->prm.gamma;
  a.gm1 = c->prm.gamma - 1.0;
  a.Rinv = 1.0 / c->prm.R;
  a.mu = c->prm.mu;
  a.lam = c->prm.gamma * c->prm.R * c->prm.mu / ((c->prm.gamma - 1.0) * c->prm.Pr);
  a.f_gamma = (float)a.gamma;
  a.f_gm1 = (float)a.gm1;
  a.f_Rinv = (float)a.Rinv;
  a.f_mu = (float)a.mu;
  a.f_lam = (float)a.lam;
  a.sutherland = c->prm.sutherland;
  a.inv_Tref = 1.0 / c->prm.T_ref;
  a.kappa = c->prm.gamma * c->prm.R / ((c->prm.gamma - 1.0) * c->prm.Pr);
  a.f_inv_Tref = (float)a.inv_Tref;
  a.f_kappa = (float)a.kappa;
  a.riemann = c->prm.riemann;
  a.viscous = c->prm.viscous;
  a.shock = c->prm.shock_capturing;
  a.alpha_min = c->prm.alpha_min;
  a.alpha_max = c->prm.alpha_max;
  a.alpha_force = c->prm.alpha_force;
  a.scal = c->scal;
  a.elem_case = c->elem_case;
  a.side_case = c->side_case;
  a.cases = c->cases;
  a.elem_list = c->elem_list;
  a.side_list = c->side_list;
  a.side_bc = c->side_bc;
  a.bcdata = c->bcdata;
  a.sponge_sigma = c->sponge_sigma;
  a.sponge_base = c->sponge_base;
  a.Ufc = c->Ufc;
  a.gfc = c->gfc;
  a.gfc32 = c->gfc32;
  a.source = c->xyzs ? c->prm.source : 0;
  a.src_A = c->prm.source_A;
  a.src_a = c->prm.source_a;
  a.xyzs = c->xyzs;
  a.rkC = c->stage_c;
  a.tr32 = c->tr32;
  a.pfv32 = c->pfv32;
  a.qs32 = c->qs32;
  a.wv32 = c->wv32;
  a.cfl_out = c->stage_cfl;
  a.scal_cfl = c->scal;
  a.f_cflkv = (float)(std::max(4.0 / 3.0, c->prm.gamma / c->prm.Pr) * c->prm.mu);
  a.epilogue = 0;
  a.prefetch = 0;
  a.elem_off = 0;
  a.E_all = (int)c->E;
  if (c->elem_list) {
    a.E = (int)c->n_elem_list;
    a.S = (int)c->n_side_list;
  }
  return a;
}

template <int N, typename T, int E = 0>
inline size_t lift_smem_bytes() {
  using S = Shape<N, E>;
  if constexpr (sizeof(T) == sizeof(double)) return Lift64Smem<N, E>::bytes;
  return sizeof(T) * (((S::n2 + 3) & ~3) + S::EPB * 16 * S::n3);
}

// Launch variants the autotuner chooses among: the default elements per
// block D and 2D (lifting up to 1024 threads, volume up to 512), and for FP64
// the volume kernel's two thread mappings.
template <int N, typename T>
struct Variants {
  static constexpr int D = Shape<N>::EPB_DEFAULT;
  static constexpr int n3 = Shape<N>::n3;
  static constexpr bool lift2 = 2 * D * n3 <= 1024;
  static constexpr bool vol2 = 2 * D * n3 <= 512;
  static constexpr bool fp64 = sizeof(T) == sizeof(double);
};

template <int N, typename T, int E>
inline void launch_lift(const StageArgs& a, cudaStream_t st) {
  using S = Shape<N, E>;
  k_lift<N, T, E><<<(unsigned)((a.E + S::EPB - 1) / S::EPB), S::THREADS, lift_smem_bytes<N, T, E>(), st>>>(a);
}
template <int N, int MODE, typename T, int E, bool PR>
inline void launch_vol(const StageArgs& a, cudaStream_t st) {
  using S = Shape<N, E>;
  k_volume<N, MODE, T, E, PR>
      <<<(unsigned)((a.E + S::EPB - 1) / S::EPB), S::THREADS, VolumeSmem<N, T, E, PR>::bytes, st>>>(a);
}
template <int N, typename T, bool GL = false>
inline void launch_side(const StageArgs& a, int block, cudaStream_t st, bool prims) {
  const int64_t side_nodes = (int64_t)a.S * Shape<N>::n2;
  const int b = block == 128 ? 128 : 256;
  const unsigned g = (unsigned)((side_nodes + b - 1) / b);
  if (prims) k_surf_prims<N, T, GL><<<g, b, 0, st>>>(a);
  else k_surf_flux<N, T, GL><<<g, b, 0, st>>>(a);
}

template <int N, typename T>
inline void lift_variant(const StageArgs& a, int epb, cudaStream_t st) {
  using V = Variants<N, T>;
  if constexpr (V::lift2) {
    if (epb == 2 * V::D) return launch_lift<N, T, 2 * V::D>(a, st);
  }
  launch_lift<N, T, 0>(a, st);
}
template <int N, int MODE, typename T>
inline void vol_variant(const StageArgs& a, int epb, int pairs, cudaStream_t st) {
  using V = Variants<N, T>;
  if constexpr (MODE == 0) {
    // dg_rhs and the diagnostics: the default variant
    launch_vol<N, 0, T, 0, V::fp64>(a, st);
  } else {
    const bool pr = V::fp64 && (pairs < 0 ? true : pairs != 0);
    if constexpr (V::vol2) {
      if (epb == 2 * V::D) {
        if constexpr (V::fp64) {
          if (!pr) return launch_vol<N, 1, T, 2 * V::D, false>(a, st);
        }
        return launch_vol<N, 1, T, 2 * V::D, V::fp64>(a, st);
      }
    }
    if constexpr (V::fp64) {
      if (!pr) return launch_vol<N, 1, T, 0, false>(a, st);
    }
    launch_vol<N, 1, T, 0, V::fp64>(a, st);
  }
}

template <int N, int E>
inline int felem_wave();
template <int N>
inline int persist_grid();

template <int N, typename T>
cudaError_t stage_set_attrs() {
  using V = Variants<N, T>;
  const int maxsm = 227 * 1024;
  auto lift = [&](auto kern, size_t bytes) {
    if (bytes <= (size_t)maxsm) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  lift(k_lift<N, T, 0>, lift_smem_bytes<N, T, 0>());
  if constexpr (V::lift2) lift(k_lift<N, T, 2 * V::D>, lift_smem_bytes<N, T, 2 * V::D>());
  lift(k_prolong_gl<N>, gl_prolong_smem<N>());
  lift(k_lift_gl<N, T>, gl_lift_smem<N, T>());
  lift(k_volume_gl<N, 0, T>, gl_volume_smem<N, T>());
  lift(k_volume_gl<N, 1, T>, gl_volume_smem<N, T>());
  lift(k_volume<N, 0, T, 0, V::fp64>, VolumeSmem<N, T, 0, V::fp64>::bytes);
  lift(k_volume<N, 1, T, 0, V::fp64>, VolumeSmem<N, T, 0, V::fp64>::bytes);
  if constexpr (V::fp64) lift(k_volume<N, 1, T, 0, false>, VolumeSmem<N, T, 0, false>::bytes);
  if constexpr (V::vol2) {
    lift(k_volume<N, 1, T, 2 * V::D, V::fp64>, VolumeSmem<N, T, 2 * V::D, V::fp64>::bytes);
    if constexpr (V::fp64) lift(k_volume<N, 1, T, 2 * V::D, false>, VolumeSmem<N, T, 2 * V::D, false>::bytes);
  }
  if constexpr (!V::fp64) {
    lift(k_fprep<N>, FusedSmem<N>::bytes);
    lift(k_felem<N, 0, 0>, FusedSmem<N, 0>::bytes);
    lift(k_felem<N, 1, 0>, FusedSmem<N, 0>::bytes);
    if constexpr (V::vol2) lift(k_felem<N, 1, 2 * V::D>, FusedSmem<N, 2 * V::D>::bytes);
    // the prefetch distances, queried here (context set-up) and not during
    // the capture of a step graph
    felem_wave<N, 0>();
    if constexpr (V::vol2) felem_wave<N, 2 * V::D>();
    lift(k_fpersist<N>, FusedSmem<N>::bytes);
    persist_grid<N>();
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The two-kernel FP32-bulk stage (dg_fused32.cuh)
// ---------------------------------------------------------------------------
// blocks of k_felem<N, 1, E> resident per SM times the SM count: the L2
// prefetch distance (one wave ahead)
template <int N, int E>
inline int felem_wave() {
  static int wave = 0;
  if (wave == 0) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_felem<N, 1, E>, Shape<N, E>::THREADS,
                                                      FusedSmem<N, E>::bytes) == cudaSuccess &&
        sms > 0 && per > 0)
      wave = sms * per;
    else
      wave = -1;  // unknown: no prefetch
  }
  return wave;
}
// blocks of the persistent kernel the GPU holds at once (its grid)
template <int N>
inline int persist_grid() {
  static int grid = 0;
  if (grid == 0) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fpersist<N>, Shape<N>::THREADS,
                                                      FusedSmem<N>::bytes) == cudaSuccess &&
        sms > 0 && per > 0)
      grid = sms * per;
    else
      grid = -1;
  }
  return grid;
}

// One persistent launch for all stages of a step (two-kernel FP32-bulk
// stage); extra / spin: the barrier test hook and the wait limit in polls.
template <int N>
cudaError_t persist_launch(dg_ctx* c, int ns, const double* A, const double* B, const double* C, unsigned extra,
                           unsigned spin) {
  using S = Shape<N>;
  StageArgs a = make_stage_args(c, c->U);
  if (a.E == 0) return cudaSuccess;
  a.Ut = c->Ut;
  a.Urk = c->U;
  a.dU = c->dU;
  a.epilogue = 1;
  const int nblk = (a.E + S::EPB - 1) / S::EPB;
  const int cap = persist_grid<N>();
  if (cap <= 0) return cudaErrorInvalidConfiguration;
  const int grid = std::min(nblk, cap);
  a.prefetch = c->cfg.prefetch ? grid : 0;  // the element this block takes next
  PersistArgs p{};
  p.ns = ns;
  for (int s = 0; s < ns; ++s) p.A[s] = A[s], p.B[s] = B[s], p.C[s] = C[s];
  p.bar = c->scal->bar;
  p.timeout = &c->scal->timeout;
  p.expect_extra = extra;
  p.spin_limit = spin;
  p.nblk = nblk;
  cudaError_t e = cudaMemsetAsync(p.bar, 0, sizeof(unsigned) * 2, c->stream);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(S::THREADS);
  cfg.dynamicSmemBytes = FusedSmem<N>::bytes;
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;  // every block resident at once
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  prof_begin(c, PK_VOLUME);
  e = cudaLaunchKernelEx(&cfg, k_fpersist<N>, a, p);
  prof_end(c);
  count_launch();
  return e;
}

template <int N, int MODE, int E>
inline void launch_felem(StageArgs a, int prefetch, cudaStream_t st) {
  using S = Shape<N, E>;
  a.prefetch = prefetch ? std::max(0, felem_wave<N, E>()) : 0;
  k_felem<N, MODE, E><<<(unsigned)((a.E + S::EPB - 1) / S::EPB), S::THREADS, FusedSmem<N, E>::bytes, st>>>(a);
}
template <int N>
inline void launch_fflux(const StageArgs& a, int block, cudaStream_t st) {
  const int64_t side_nodes = (int64_t)a.S * Shape<N>::n2;
  const int b = block == 128 ? 128 : 256;
  k_fflux<N><<<(unsigned)((side_nodes + b - 1) / b), b, 0, st>>>(a);
}
// face data of state U: every element of the context (a serving pool: its
// occupied elements), or, with E_range >= 0, the elements e0 .. e0 + E_range - 1
template <int N>
inline cudaError_t fprep_launch(dg_ctx* c, const double* U, int64_t e0 = 0, int64_t E_range = -1,
                                cudaStream_t st = nullptr) {
  using S = Shape<N>;
  StageArgs a = make_stage_args(c, U);
  if (E_range >= 0) {
    a.elem_list = nullptr;
    a.elem_off = (int)e0;
    a.E = (int)E_range;
  }
  if (a.E == 0) return cudaSuccess;
  k_fprep<N><<<(unsigned)((a.E + S::EPB - 1) / S::EPB), S::THREADS, FusedSmem<N>::bytes, st ? st : c->stream>>>(a);
  count_launch();
  return cudaGetLastError();
}
template <int N>
inline void felem_variant(const StageArgs& a, int mode, int epb, int prefetch, cudaStream_t st) {
  using V = Variants<N, float>;
  if (mode == 0) return launch_felem<N, 0, 0>(a, 0, st);
  if constexpr (V::vol2) {
    if (epb == 2 * V::D) return launch_felem<N, 1, 2 * V::D>(a, prefetch, st);
  }
  launch_felem<N, 1, 0>(a, prefetch, st);
}

// One stage in the two-kernel form.  Mode 0 (dg_rhs) first forms the face
// data of U; mode 1 expects them from the previous stage (or k_fprep, run by
// the stepping loop before the first step) and leaves those of the updated
// state behind.
template <int N>
cudaError_t stage_launch_fused(dg_ctx* c, const double* U, int mode, double rkA, double rkB, int first) {
  StageArgs a = make_stage_args(c, U);
  a.Ut = c->Ut;
  a.Urk = c->U;
  a.dU = c->dU;
  a.rkA = rkA;
  a.rkB = rkB;
  a.f_rkA = (float)rkA;
  a.first_stage = first;
  a.epilogue = mode == 1;
  if (a.E == 0) return cudaSuccess;
  const StageConfig& g = c->cfg;
  if (mode == 0) {
    prof_begin(c, PK_SURF_PRIMS);
    cudaError_t e = fprep_launch<N>(c, U);
    prof_end(c);
    if (e != cudaSuccess) return e;
    c->traces_valid = false;  // they now describe U, not necessarily the context's state
  }
  prof_begin(c, PK_SURF_FLUX);
  launch_fflux<N>(a, g.side_block, c->stream);
  prof_end(c);
  prof_begin(c, PK_VOLUME);
  felem_variant<N>(a, mode, g.vol_epb, g.prefetch, c->stream);
  prof_end(c);
  count_launch(2);
  return cudaGetLastError();
}

// One stage of the standard DGSEM on Gauss-Legendre nodes: ProlongToFace,
// (lifting,) surface flux, volume integral with SurfInt and ApplyJac
template <int N, typename T>
cudaError_t stage_launch_gl(dg_ctx* c, const double* U, int mode, double rkA, double rkB, int first) {
  using S = Shape<N>;
  StageArgs a = make_stage_args(c, U);
  a.Ut = c->Ut;
  a.Urk = c->U;
  a.dU = c->dU;
  a.rkA = rkA;
  a.rkB = rkB;
  a.first_stage = first;
  if (a.E == 0) return cudaSuccess;
  const unsigned nb = (unsigned)((a.E + S::EPB - 1) / S::EPB);
  const int sb = c->cfg.side_block;
  prof_begin(c, PK_SURF_PRIMS);
  k_prolong_gl<N><<<nb, S::THREADS, gl_prolong_smem<N>(), c->stream>>>(a);
  if (c->prm.viscous) launch_side<N, T, true>(a, sb, c->stream, true);
  prof_end(c);
  if (c->prm.viscous) {
    prof_begin(c, PK_LIFT);
    k_lift_gl<N, T><<<nb, S::THREADS, gl_lift_smem<N, T>(), c->stream>>>(a);
    prof_end(c);
    count_launch(2);
  }
  prof_begin(c, PK_SURF_FLUX);
  launch_side<N, T, true>(a, sb, c->stream, false);
  prof_end(c);
  prof_begin(c, PK_VOLUME);
  if (mode == 0) k_volume_gl<N, 0, T><<<nb, S::THREADS, gl_volume_smem<N, T>(), c->stream>>>(a);
  else k_volume_gl<N, 1, T><<<nb, S::THREADS, gl_volume_smem<N, T>(), c->stream>>>(a);
  prof_end(c);
  count_launch(3);
  return cudaGetLastError();
}

template <int N, typename T>
cudaError_t stage_launch(dg_ctx* c, const double* U, int mode, double rkA, double rkB, int first) {
  if (c->gauss) return stage_launch_gl<N, T>(c, U, mode, rkA, rkB, first);
  if constexpr (sizeof(T) == sizeof(float)) {
    if (fused_active(c)) return stage_launch_fused<N>(c, U, mode, rkA, rkB, first);
  }
  StageArgs a = make_stage_args(c, U);
  a.Ut = c->Ut;
  a.Urk = c->U;
  a.dU = c->dU;
  a.rkA = rkA;
  a.rkB = rkB;
  a.first_stage = first;
  if (a.E == 0) return cudaSuccess;
  const StageConfig& g = c->cfg;
  if (c->prm.viscous) {
    prof_begin(c, PK_SURF_PRIMS);
    launch_side<N, T>(a, g.side_block, c->stream, true);
    prof_end(c);
    prof_begin(c, PK_LIFT);
    lift_variant<N, T>(a, g.lift_epb, c->stream);
    prof_end(c);
    count_launch(2);
  }
  prof_begin(c, PK_SURF_FLUX);
  launch_side<N, T>(a, g.side_block, c->stream, false);
  prof_end(c);
  prof_begin(c, PK_VOLUME);
  if (mode == 0) vol_variant<N, 0, T>(a, g.vol_epb, g.vol_pairs, c->stream);
  else vol_variant<N, 1, T>(a, g.vol_epb, g.vol_pairs, c->stream);
  prof_end(c);
  count_launch(2);
  return cudaGetLastError();
}

// Autotuner: times every launch variant of the stage kernels on the context's
// own data and keeps the fastest of each kernel.  The runs write only scratch
// arrays: the lifted gradients and surface fluxes (recomputed by every
// stage), and an RK update redirected into the Ut and public-layout buffers;
// the state is untouched.  ms[]: per variant, mean ms over the timed
// repetitions, in the order lift D, lift 2D, volume (D, default mapping),
// volume (D, other mapping), volume (2D, default), volume (2D, other), side
// 256, side 128 (-1 where a variant does not exist).
// Autotuner of the two-kernel FP32-bulk stage: the element kernel at D and
// 2D elements per block (ms[2], ms[4]) and the side kernel at 256 and 128
// threads (ms[6], ms[7]); the runs read the face data of the state (formed
// first) and write the RK update and the epilogue's face data to scratch.
template <int N>
cudaError_t stage_autotune_fused(dg_ctx* c, double* ms) {
  using V = Variants<N, float>;
  StageArgs a = make_stage_args(c, c->U);
  a.Ut = c->Ut;
  a.Urk = c->Ut;
  a.dU = c->Upub;
  a.rkA = 0.5;
  a.rkB = 0.5;
  a.f_rkA = 0.5f;
  a.first_stage = 0;
  a.epilogue = 1;
  for (int i = 0; i < 8; ++i) ms[i] = -1.0;
  if (a.E == 0) return cudaSuccess;
  cudaStream_t st = c->stream;
  cudaError_t e = cudaMemsetAsync(c->Upub, 0, sizeof(double) * c->E * 5 * c->n3, st);
  if (e == cudaSuccess) e = fprep_launch<N>(c, c->U);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int reps = 3;
  auto timed = [&](auto&& launch) -> double {
    launch();  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    count_launch(reps + 1);
    return t / reps;
  };
  StageConfig best = c->cfg;
  if (e == cudaSuccess) {
    const int pf = c->cfg.prefetch;
    ms[6] = timed([&] { launch_fflux<N>(a, 256, st); });
    ms[7] = timed([&] { launch_fflux<N>(a, 128, st); });
    best.side_block = ms[7] < ms[6] ? 128 : 256;
    ms[2] = timed([&] { launch_felem<N, 1, 0>(a, pf, st); });
    best.vol_epb = V::D;
    if constexpr (V::vol2) {
      ms[4] = timed([&] { launch_felem<N, 1, 2 * V::D>(a, pf, st); });
      if (ms[4] < ms[2]) best.vol_epb = 2 * V::D;
    }
    e = cudaGetLastError();
    // the runs' epilogues wrote the face data of a scratch state: form the
    // state's own again (a serving pool steps on without re-forming them)
    if (e == cudaSuccess) e = fprep_launch<N>(c, c->U);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) {
    c->cfg = best;
    c->tuned = true;
  }
  return e;
}

template <int N, typename T>
cudaError_t stage_autotune(dg_ctx* c, double* ms) {
  using V = Variants<N, T>;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (fused_active(c)) return stage_autotune_fused<N>(c, ms);
  }
  StageArgs a = make_stage_args(c, c->U);
  a.Ut = c->Ut;
  a.Urk = c->Ut;
  a.dU = c->Upub;
  a.rkA = 0.5;
  a.rkB = 0.5;
  a.first_stage = 0;
  for (int i = 0; i < 8; ++i) ms[i] = -1.0;
  if (a.E == 0) return cudaSuccess;
  cudaStream_t st = c->stream;
  cudaError_t e = cudaMemsetAsync(c->Upub, 0, sizeof(double) * c->E * 5 * c->n3, st);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int reps = 3;
  auto timed = [&](auto&& launch) -> double {
    launch();  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    count_launch(reps + 1);
    return t / reps;
  };
  StageConfig best = c->cfg;
  if (e == cudaSuccess) {
    // inputs of the volume kernel: gradients and surface fluxes
    if (c->prm.viscous) {
      launch_side<N, T>(a, 256, st, true);
      launch_lift<N, T, 0>(a, st);
    }
    launch_side<N, T>(a, 256, st, false);
    count_launch(3);
    if (c->prm.viscous) {
      ms[0] = timed([&] { launch_lift<N, T, 0>(a, st); });
      best.lift_epb = V::D;
      if constexpr (V::lift2) {
        ms[1] = timed([&] { launch_lift<N, T, 2 * V::D>(a, st); });
        if (ms[1] < ms[0]) best.lift_epb = 2 * V::D;
      }
    }
    double vbest = 1e30;
    auto vol = [&](int slot, double t, int epb, int pairs) {
      ms[slot] = t;
      if (t < vbest) {
        vbest = t;
        best.vol_epb = epb;
        best.vol_pairs = pairs;
      }
    };
    const bool other = !c->tune_keep_mapping;  // also try the other thread mapping
    vol(2, timed([&] { launch_vol<N, 1, T, 0, V::fp64>(a, st); }), V::D, V::fp64 ? 1 : 0);
    if constexpr (V::fp64) {
      if (other) vol(3, timed([&] { launch_vol<N, 1, T, 0, false>(a, st); }), V::D, 0);
    }
    if constexpr (V::vol2) {
      vol(4, timed([&] { launch_vol<N, 1, T, 2 * V::D, V::fp64>(a, st); }), 2 * V::D, V::fp64 ? 1 : 0);
      if constexpr (V::fp64) {
        if (other) vol(5, timed([&] { launch_vol<N, 1, T, 2 * V::D, false>(a, st); }), 2 * V::D, 0);
      }
    }
    ms[6] = timed([&] {
      if (c->prm.viscous) launch_side<N, T>(a, 256, st, true);
      launch_side<N, T>(a, 256, st, false);
    });
    ms[7] = timed([&] {
      if (c->prm.viscous) launch_side<N, T>(a, 128, st, true);
      launch_side<N, T>(a, 128, st, false);
    });
    best.side_block = ms[7] < ms[6] ? 128 : 256;
    e = cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) {
    c->cfg = best;
    c->tuned = true;
  }
  return e;
}

// Entry points of one degree (each degree is its own translation unit)
#define DG_STAGE_ENTRY_POINTS(K)                                                                  \
  cudaError_t stage_attrs_n##K() {                                                                \
    cudaError_t e = stage_set_attrs<K, double>();                                                 \
    if (e == cudaSuccess) e = stage_set_attrs<K, float>();                                        \
    return e;                                                                                     \
  }                                                                                               \
  cudaError_t stage_launch_n##K(dg_ctx* c, const double* U, int mode, double A, double B, int f) { \
    return c->prm.precision == DG_FP32_BULK ? stage_launch<K, float>(c, U, mode, A, B, f)         \
                                            : stage_launch<K, double>(c, U, mode, A, B, f);       \
  }                                                                                               \
  cudaError_t stage_autotune_n##K(dg_ctx* c, double* ms) {                                        \
    return c->prm.precision == DG_FP32_BULK ? stage_autotune<K, float>(c, ms)                     \
                                            : stage_autotune<K, double>(c, ms);                   \
  }                                                                                               \
  cudaError_t fprep_n##K(dg_ctx* c, const double* U, int64_t e0, int64_t E, cudaStream_t st) {    \
    return fprep_launch<K>(c, U, e0, E, st);                                                      \
  }                                                                                               \
  cudaError_t persist_n##K(dg_ctx* c, int ns, const double* A, const double* B, const double* C,    \
                           unsigned extra, unsigned spin) {                                       \
    return persist_launch<K>(c, ns, A, B, C, extra, spin);                                        \
  }

#define DG_DISPATCH(N_, CALL)                      \
  switch (N_) {                                    \
    case 1: { constexpr int NN = 1; CALL; } break; \
    case 2: { constexpr int NN = 2; CALL; } break; \
    case 3: { constexpr int NN = 3; CALL; } break; \
    case 4: { constexpr int NN = 4; CALL; } break; \
    case 5: { constexpr int NN = 5; CALL; } break; \
    case 6: { constexpr int NN = 6; CALL; } break; \
    case 7: { constexpr int NN = 7; CALL; } break; \
    default: return cudaErrorInvalidValue;         \
  }

}  // namespace dg
