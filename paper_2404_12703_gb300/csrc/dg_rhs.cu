// dg_rhs.cu -- the kernels of one evaluation of the DG time derivative
// (Eq. dgsem with the split-form volume integral and BR1 lifting) and of the
// fused low-storage RK stage, FP64.
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
// Data layout: element-major SoA, U[e][v][node], node = i + n (j + n k).
#include <algorithm>
#include <cmath>

#include "dg_common.cuh"
#include "dg_launch.h"

namespace dg {

template <int N>
struct Shape {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  static constexpr int EPB = n3 >= 256 ? 1 : 256 / n3;  // elements per block
  static constexpr int THREADS = EPB * n3;
};

// ---------------------------------------------------------------------------
// BR1 surface flux of the lifted primitives
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) k_surf_prims(StageArgs a) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)a.S * n2) return;
  const int s = (int)(tid / n2), pq = (int)(tid % n2);
  const int p = pq % n, q = pq / n;
  const int2 ee = a.side_e[s];
  const int sf = a.side_f[s];
  const int fM = sf & 15, fS = (sf >> 4) & 15, flip = sf >> 8;
  int ps, qs;
  flip_to_slave<n>(flip, p, q, ps, qs);
  const int vM = face_vol_node<n>(fM, p, q), vS = face_vol_node<n>(fS, ps, qs);
  double UM[5], US[5];
  const double* uM = a.U + (size_t)ee.x * 5 * n3 + vM;
  const double* uS = a.U + (size_t)ee.y * 5 * n3 + vS;
#pragma unroll
  for (int k = 0; k < 5; ++k) { UM[k] = uM[k * n3]; US[k] = uS[k * n3]; }
  const Prim<double> qM = cons_to_prim(UM, a.gm1, a.Rinv);
  const Prim<double> qS = cons_to_prim(US, a.gm1, a.Rinv);
  const double qa[4] = {0.5 * (qM.u + qS.u), 0.5 * (qM.v + qS.v), 0.5 * (qM.w + qS.w), 0.5 * (qM.T_ + qS.T_)};
  const double* nr = a.nrm + (size_t)s * 4 * n2 + pq;
  const double sn[3] = {nr[0], nr[n2], nr[2 * n2]};
  double* out = a.lflux + (size_t)s * 12 * n2 + pq;
#pragma unroll
  for (int qv = 0; qv < 4; ++qv)
#pragma unroll
    for (int x = 0; x < 3; ++x) out[(qv * 3 + x) * n2] = qa[qv] * sn[x];
}

// ---------------------------------------------------------------------------
// Lifted gradients (weak form, Eq. lifting)
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Shape<N>::THREADS) k_lift(StageArgs a) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ __align__(16) double sm[];
  double* sDh = sm;                 // [n2]
  double* sq = sDh + n2;            // [EPB][4][n3]
  double* sF = sq + EPB * 4 * n3;   // [EPB][12][n3]
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  // Slots past the last element redo the last element in their own shared
  // memory slot, so that every thread of a block runs the same path through
  // the barriers; only the final global stores are masked.
  const bool valid = blockIdx.x * EPB + le < a.E;
  const int e = valid ? blockIdx.x * EPB + le : a.E - 1;
  for (int k = threadIdx.x; k < n2; k += blockDim.x) sDh[k] = a.ops->Dhat[k];
  double* q = sq + le * 4 * n3;
  double* F = sF + le * 12 * n3;
  const double* Me = a.metric + (size_t)e * 10 * n3;
  {
    double U[5];
    const double* u = a.U + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k] = u[k * n3];
    const Prim<double> pr = cons_to_prim(U, a.gm1, a.Rinv);
    q[t] = pr.u;
    q[n3 + t] = pr.v;
    q[2 * n3 + t] = pr.w;
    q[3 * n3 + t] = pr.T_;
  }
  __syncwarp();
  __syncthreads();
  const int idx[3] = {t % n, (t / n) % n, t / n2};
  constexpr int str[3] = {1, n, n2};
  double acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = 0.0;
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    {
      const double J0 = Me[(d * 3 + 0) * n3 + t], J1 = Me[(d * 3 + 1) * n3 + t], J2 = Me[(d * 3 + 2) * n3 + t];
#pragma unroll
      for (int qv = 0; qv < 4; ++qv) {
        const double qq = q[qv * n3 + t];
        F[(qv * 3 + 0) * n3 + t] = J0 * qq;
        F[(qv * 3 + 1) * n3 + t] = J1 * qq;
        F[(qv * 3 + 2) * n3 + t] = J2 * qq;
      }
    }
    __syncwarp();
    __syncthreads();
    {
      const int id = idx[d], base = t - id * str[d];
#pragma unroll
      for (int al = 0; al < n; ++al) {
        const double c = sDh[id * n + al];
        const int nb = base + al * str[d];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] += c * F[k * n3 + nb];
      }
    }
    __syncwarp();
    __syncthreads();
  }
  if (!valid) return;
  // surface part: on LGL nodes only face nodes receive it
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
    const double* L = a.lflux + (size_t)s * 12 * n2 + pm + n * qm;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] += sg * L[k * n2];
  }
  const double Ji = Me[9 * n3 + t];
  double* g = a.g + (size_t)e * 12 * n3 + t;
#pragma unroll
  for (int k = 0; k < 12; ++k) g[k * n3] = acc[k] * Ji;
}

// ---------------------------------------------------------------------------
// FillFlux: Riemann flux + BR1 viscous flux, times the surface element
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) k_surf_flux(StageArgs a) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)a.S * n2) return;
  const int s = (int)(tid / n2), pq = (int)(tid % n2);
  const int p = pq % n, q = pq / n;
  const int2 ee = a.side_e[s];
  const int sf = a.side_f[s];
  const int fM = sf & 15, fS = (sf >> 4) & 15, flip = sf >> 8;
  int ps, qs;
  flip_to_slave<n>(flip, p, q, ps, qs);
  const int vM = face_vol_node<n>(fM, p, q), vS = face_vol_node<n>(fS, ps, qs);
  double UM[5], US[5];
  const double* uM = a.U + (size_t)ee.x * 5 * n3 + vM;
  const double* uS = a.U + (size_t)ee.y * 5 * n3 + vS;
#pragma unroll
  for (int k = 0; k < 5; ++k) { UM[k] = uM[k * n3]; US[k] = uS[k * n3]; }
  const Prim<double> qM = cons_to_prim(UM, a.gm1, a.Rinv);
  const Prim<double> qS = cons_to_prim(US, a.gm1, a.Rinv);
  const double* nr = a.nrm + (size_t)s * 4 * n2 + pq;
  const double sn[3] = {nr[0], nr[n2], nr[2 * n2]};
  const double sA = nr[3 * n2];
  const double inv = 1.0 / sA;
  const double nu[3] = {sn[0] * inv, sn[1] * inv, sn[2] * inv};
  double f[5];
  if (a.riemann == DG_RIEMANN_ROE) roe_flux(UM, qM, US, qS, nu, a.gm1, f);
  else lf_flux(UM, qM, US, qS, nu, a.gamma, f);
#pragma unroll
  for (int k = 0; k < 5; ++k) f[k] *= sA;
  if (a.viscous) {
    double gM[12], gS[12];
    const double* pgM = a.g + (size_t)ee.x * 12 * n3 + vM;
    const double* pgS = a.g + (size_t)ee.y * 12 * n3 + vS;
#pragma unroll
    for (int k = 0; k < 12; ++k) { gM[k] = pgM[k * n3]; gS[k] = pgS[k * n3]; }
    double tau[6], W[3], fvM[4], fvS[4];
    viscous_parts(gM, qM.u, qM.v, qM.w, a.mu, a.lam, tau, W);
    viscous_flux_n(tau, W, sn, fvM);
    viscous_parts(gS, qS.u, qS.v, qS.w, a.mu, a.lam, tau, W);
    viscous_flux_n(tau, W, sn, fvS);
#pragma unroll
    for (int k = 0; k < 4; ++k) f[1 + k] -= 0.5 * (fvM[k] + fvS[k]);
  }
  double* out = a.fstar + (size_t)s * 5 * n2 + pq;
#pragma unroll
  for (int k = 0; k < 5; ++k) out[k * n2] = f[k];
}

// ---------------------------------------------------------------------------
// Hennemann indicator on rho p (modal energy of the top modes), Sec. 2.3
// ---------------------------------------------------------------------------
// Every thread of the element runs the same instructions (no single-thread
// branch in front of a barrier): row sums are formed by all threads (rows
// are formed twice or more, with identical values), then every thread adds
// the row sums itself.  sT1 / sT2: n3 doubles each, sRow: 4 n2 doubles.
template <int n>
__device__ double element_alpha(const double* sP /* rho at 0, p at 4*n3 */, double* sT1, double* sT2,
                                double* sRow, const double* sVinv, int t, double amin, double amax) {
  constexpr int n2 = n * n, n3 = n2 * n, N = n - 1;
  const int i = t % n, j = (t / n) % n, k = t / n2;
  sT1[t] = sP[t] * sP[4 * n3 + t];
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

// ---------------------------------------------------------------------------
// Volume integral + SurfInt + ApplyJac (+ RK update)
// ---------------------------------------------------------------------------
template <int N, int MODE>
__global__ void __launch_bounds__(Shape<N>::THREADS) k_volume(StageArgs a) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ __align__(16) double sm[];
  double* sDs = sm;                  // [n2] Dsplit
  double* sDh = sDs + n2;            // [n2] Dhat
  double* sVi = sDh + n2;            // [n2] Vinv
  double* sP = sVi + n2;             // [EPB][6][n3] rho u v w p H
  double* sJ = sP + EPB * 6 * n3;    // [EPB][9][n3]
  double* sG = sJ + EPB * 9 * n3;    // [EPB][5][n3] viscous contravariant flux / FV flux
  double* sX = sG + EPB * 5 * n3;    // [EPB][2 n3 + 4 n2] indicator scratch
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  // slots past the last element redo the last element (see k_lift)
  const bool valid = blockIdx.x * EPB + le < a.E;
  const int e = valid ? blockIdx.x * EPB + le : a.E - 1;
  for (int k = threadIdx.x; k < n2; k += blockDim.x) {
    sDs[k] = a.ops->Dsplit[k];
    sDh[k] = a.ops->Dhat[k];
    sVi[k] = a.ops->Vinv[k];
  }
  double* P = sP + le * 6 * n3;
  double* Jm = sJ + le * 9 * n3;
  double* G = sG + le * 5 * n3;
  const double* Me = a.metric + (size_t)e * 10 * n3;
  double U[5];
  double g[12];
  {
    const double* u = a.U + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k] = u[k * n3];
    const Prim<double> pr = cons_to_prim(U, a.gm1, a.Rinv);
    P[t] = pr.rho;
    P[n3 + t] = pr.u;
    P[2 * n3 + t] = pr.v;
    P[3 * n3 + t] = pr.w;
    P[4 * n3 + t] = pr.p;
    P[5 * n3 + t] = (U[4] + pr.p) / pr.rho;
#pragma unroll
    for (int c = 0; c < 9; ++c) Jm[c * n3 + t] = Me[c * n3 + t];
    if (a.viscous) {
      const double* pg = a.g + (size_t)e * 12 * n3 + t;
#pragma unroll
      for (int k = 0; k < 12; ++k) g[k] = pg[k * n3];
    }
  }
  __syncwarp();
  __syncthreads();
  const int idx[3] = {t % n, (t / n) % n, t / n2};
  constexpr int str[3] = {1, n, n2};
  double accC[5] = {0, 0, 0, 0, 0};  // convective DG volume term
  double acc[5] = {0, 0, 0, 0, 0};   // viscous volume + surface terms
  double tau[6] = {0, 0, 0, 0, 0, 0}, W[3] = {0, 0, 0};
  if (a.viscous) viscous_parts(g, P[n3 + t], P[2 * n3 + t], P[3 * n3 + t], a.mu, a.lam, tau, W);
  const double ri = P[t], ui = P[n3 + t], vi = P[2 * n3 + t];
  const double wi = P[3 * n3 + t], pi = P[4 * n3 + t], Hi = P[5 * n3 + t];
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    const double Ji0 = Jm[(d * 3 + 0) * n3 + t], Ji1 = Jm[(d * 3 + 1) * n3 + t], Ji2 = Jm[(d * 3 + 2) * n3 + t];
    if (a.viscous) {
      {
        const double nv[3] = {Ji0, Ji1, Ji2};
        double fv[4];
        viscous_flux_n(tau, W, nv, fv);
#pragma unroll
        for (int k = 0; k < 4; ++k) G[k * n3 + t] = fv[k];
      }
      __syncwarp();
      __syncthreads();
    }
    {
      const int id = idx[d], base = t - id * str[d];
#pragma unroll
      for (int al = 0; al < n; ++al) {
        if (al == id) continue;
        const int nb = base + al * str[d];
        const double Dv = sDs[id * n + al];
        const double m0 = (Ji0 + Jm[(d * 3 + 0) * n3 + nb]) / 2;
        const double m1 = (Ji1 + Jm[(d * 3 + 1) * n3 + nb]) / 2;
        const double m2 = (Ji2 + Jm[(d * 3 + 2) * n3 + nb]) / 2;
        const double rho = (ri + P[nb]) / 2;
        const double u0 = (ui + P[n3 + nb]) / 2, u1 = (vi + P[2 * n3 + nb]) / 2, u2 = (wi + P[3 * n3 + nb]) / 2;
        const double pp = (pi + P[4 * n3 + nb]) / 2;
        const double H = (Hi + P[5 * n3 + nb]) / 2;
        const double fr = rho * (u0 * m0 + u1 * m1 + u2 * m2);
        accC[0] += Dv * fr;
        accC[1] += Dv * (fr * u0 + pp * m0);
        accC[2] += Dv * (fr * u1 + pp * m1);
        accC[3] += Dv * (fr * u2 + pp * m2);
        accC[4] += Dv * (fr * H);
      }
      if (a.viscous) {
#pragma unroll
        for (int al = 0; al < n; ++al) {
          const double c = sDh[id * n + al];
          const int nb = base + al * str[d];
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[1 + k] -= c * G[k * n3 + nb];
        }
      }
    }
    if (a.viscous) {
      __syncwarp();
      __syncthreads();
    }
  }

  // ---- shock capturing: indicator and FV sub-cell blending (Sec. 2.3) ----
  if (a.shock) {
    double al;
    if (a.alpha_force >= 0) {
      al = a.alpha_force;
    } else {
      double* X1 = sX + le * (2 * n3 + 4 * n2);
      // all threads of the block take part in the barriers inside
      al = element_alpha<n>(P, X1, X1 + n3, X1 + 2 * n3, sVi, t, a.alpha_min, a.alpha_max);
    }
    if (valid && t == 0) a.alpha[e] = al;
    // block-uniform condition: the FV pass has barriers, and the elements of
    // one block may have different blending factors
    if (__syncthreads_or(al > 0)) {
      double vfv[5] = {0, 0, 0, 0, 0};
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
        const double sA = sqrt(mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2]);
        const double nu[3] = {mv[0] / sA, mv[1] / sA, mv[2] / sA};
        const int nb = right ? t + str[d] : t;
        double UR[5];
        const double* ur = a.U + (size_t)e * 5 * n3 + nb;
#pragma unroll
        for (int k = 0; k < 5; ++k) UR[k] = ur[k * n3];
        const Prim<double> qL = cons_to_prim(U, a.gm1, a.Rinv);
        const Prim<double> qR = cons_to_prim(UR, a.gm1, a.Rinv);
        double fb[5];
        lf_flux(U, qL, UR, qR, nu, a.gamma, fb);
        if (right) {
#pragma unroll
          for (int k = 0; k < 5; ++k) G[k * n3 + t] = fb[k] * sA;
        }
        __syncwarp();
        __syncthreads();
        if (right) {
#pragma unroll
          for (int k = 0; k < 5; ++k) vfv[k] += G[k * n3 + t] / a.ops->w[id];
        }
        if (id > 0) {
          const int nl = t - str[d];
#pragma unroll
          for (int k = 0; k < 5; ++k) vfv[k] -= G[k * n3 + nl] / a.ops->w[id];
        }
        __syncwarp();
        __syncthreads();
      }
      if (al > 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) accC[k] = (1 - al) * accC[k] + al * vfv[k];
      }
    }
  }
  if (!valid) return;

  // ---- SurfInt: face nodes receive +-f* lhat ----
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
    const double* Fs = a.fstar + (size_t)s * 5 * n2 + pm + n * qm;
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += sg * Fs[k * n2];
  }
  // ---- ApplyJac ----
  const double Ji = Me[9 * n3 + t];
  double Ut[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) Ut[k] = -(accC[k] + acc[k]) * Ji;
  if (MODE == 0) {
    double* o = a.Ut + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) o[k * n3] = Ut[k];
  } else {
    const double dt = a.scal->dt;
    double* du = a.dU + (size_t)e * 5 * n3 + t;
    double* uo = a.Urk + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const double r = a.first_stage ? dt * Ut[k] : a.rkA * du[k * n3] + dt * Ut[k];
      du[k * n3] = r;
      uo[k * n3] = U[k] + a.rkB * r;
    }
  }
}

// ---------------------------------------------------------------------------
// CFL reduction (the paper gives no rule; see dg_time_step in dg.h)
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256) k_cfl(int E, const double* __restrict__ U, const double* __restrict__ metric,
                                            double gamma, double gm1, double Rinv, double kv, int viscous,
                                            DevScalars* scal) {
  constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
  double lc = 0.0, lv = 0.0;
  int bad = 0;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < (int64_t)E * n3;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = x / n3;
    const int t = (int)(x % n3);
    double Uv[5];
    const double* u = U + e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) Uv[k] = u[k * n3];
    const Prim<double> q = cons_to_prim(Uv, gm1, Rinv);
    const double c = sqrt(gamma * q.p / q.rho);
    const double* Me = metric + e * 10 * n3 + t;
    const double Ji = Me[9 * n3];
    double aa = 0.0, bb = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double j0 = Me[(d * 3) * n3], j1 = Me[(d * 3 + 1) * n3], j2 = Me[(d * 3 + 2) * n3];
      const double nj2 = j0 * j0 + j1 * j1 + j2 * j2;
      aa += fabs(q.u * j0 + q.v * j1 + q.w * j2) + c * sqrt(nj2);
      bb += nj2;
    }
    aa *= Ji;
    bb = kv / q.rho * bb * Ji * Ji;
    if (!isfinite(aa) || !isfinite(bb)) bad = 1;
    lc = fmax(lc, aa);
    lv = fmax(lv, bb);
  }
  // block reduction
  __shared__ double rc[32], rv[32];
  __shared__ int rb;
  if (threadIdx.x == 0) rb = 0;
  for (int o = 16; o > 0; o >>= 1) {
    lc = fmax(lc, __shfl_xor_sync(0xffffffffu, lc, o));
    lv = fmax(lv, __shfl_xor_sync(0xffffffffu, lv, o));
  }
  __syncwarp();
  __syncthreads();
  if (bad) atomicOr(&rb, 1);
  if ((threadIdx.x & 31) == 0) { rc[threadIdx.x >> 5] = lc; rv[threadIdx.x >> 5] = lv; }
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { lc = fmax(lc, rc[w]); lv = fmax(lv, rv[w]); }
    atomicMax(&scal->lam_c, (unsigned long long)__double_as_longlong(lc));
    if (viscous) atomicMax(&scal->lam_v, (unsigned long long)__double_as_longlong(lv));
    if (rb) atomicOr(&scal->nonfinite, 1);
  }
}

__global__ void k_dt(DevScalars* scal, double cfl, double dfl, int N, int viscous) {
  const double np1 = (double)(N + 1);
  double dt;
  if (scal->dt_fixed > 0) {
    dt = scal->dt_fixed;
  } else {
    const double lc = __longlong_as_double((long long)scal->lam_c);
    const double lv = __longlong_as_double((long long)scal->lam_v);
    dt = cfl * 2.0 / (np1 * np1 * lc);
    if (viscous && lv > 0) {
      const double dv = dfl * 4.0 / (np1 * np1 * np1 * np1 * lv);
      if (dv < dt) dt = dv;
    }
  }
  scal->dt = dt;
  scal->t += dt;
  scal->lam_c = 0ull;
  scal->lam_v = 0ull;
}

// ---------------------------------------------------------------------------
// layout conversion and reductions
// ---------------------------------------------------------------------------
__global__ void k_to_internal(int64_t E, int n3, const double* __restrict__ pub, double* __restrict__ in) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= E * n3 * 5) return;
  const int64_t e = x / (5 * n3);
  const int r = (int)(x % (5 * n3));
  const int v = r / n3, t = r % n3;
  in[x] = pub[(e * n3 + t) * 5 + v];
}
__global__ void k_to_public(int64_t E, int n3, const double* __restrict__ in, double* __restrict__ pub) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= E * n3 * 5) return;
  const int64_t e = x / (5 * n3);
  const int r = (int)(x % (5 * n3));
  const int t = r / 5, v = r % 5;
  pub[x] = in[e * 5 * n3 + (int64_t)v * n3 + t];
}

template <int N>
__global__ void __launch_bounds__(256) k_kinetic(int E, const double* __restrict__ U, const double* __restrict__ Ut,
                                                 const double* __restrict__ metric, const Ops* __restrict__ ops,
                                                 DevScalars* scal) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  double vol = 0, ek = 0, rate = 0;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < (int64_t)E * n3;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = x / n3;
    const int t = (int)(x % n3);
    const double wq = ops->w[t % n] * ops->w[(t / n) % n] * ops->w[t / n2] / metric[e * 10 * n3 + 9 * n3 + t];
    const double* u = U + e * 5 * n3 + t;
    const double r = u[0], vx = u[n3] / r, vy = u[2 * n3] / r, vz = u[3 * n3] / r;
    const double v2 = vx * vx + vy * vy + vz * vz;
    vol += wq;
    ek += wq * r * v2 / 2;
    if (Ut) {
      const double* ut = Ut + e * 5 * n3 + t;
      rate += wq * (vx * ut[n3] + vy * ut[2 * n3] + vz * ut[3 * n3] - v2 * ut[0] / 2);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    vol += __shfl_xor_sync(0xffffffffu, vol, o);
    ek += __shfl_xor_sync(0xffffffffu, ek, o);
    rate += __shfl_xor_sync(0xffffffffu, rate, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&scal->kin[0], ek);
    atomicAdd(&scal->kin[1], rate);
    atomicAdd(&scal->kin[2], vol);
  }
}

// ---------------------------------------------------------------------------
// verification copies
// ---------------------------------------------------------------------------
template <int N>
__global__ void k_debug_metrics(int E, const double* __restrict__ metric, double* Ja, double* J) {
  constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= (int64_t)E * n3) return;
  const int64_t e = x / n3;
  const int t = (int)(x % n3);
  const double* Me = metric + e * 10 * n3 + t;
  for (int c = 0; c < 9; ++c) Ja[x * 9 + c] = Me[c * n3];
  J[x] = 1.0 / Me[9 * n3];
}

template <int N>
__global__ void k_debug_maps(int E, const int* __restrict__ elem_side, const int2* __restrict__ side_e,
                             const int* __restrict__ side_f, int* nbr, int* nodes) {
  constexpr int n = N + 1, n2 = n * n;
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= (int64_t)E * 6) return;
  const int e = (int)(x / 6);
  const int es = elem_side[x];
  const int s = es_side(es), slave = es_slave(es), flip = es_flip(es);
  const int2 ee = side_e[s];
  const int sf = side_f[s];
  const int fM = sf & 15, fS = (sf >> 4) & 15;
  nbr[x * 3 + 0] = slave ? ee.x : ee.y;
  nbr[x * 3 + 1] = slave ? fM : fS;
  nbr[x * 3 + 2] = slave ? 0 : 1;
  (void)e;
  for (int pq = 0; pq < n2; ++pq) {
    const int p = pq % n, q = pq / n;
    int a, b;
    if (slave) flip_to_master<n>(flip, p, q, a, b);
    else flip_to_slave<n>(flip, p, q, a, b);
    nodes[x * n2 + pq] = a + n * b;
  }
}

template <int N>
__global__ void k_debug_grad(int E, const double* __restrict__ g, double* out) {
  constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= (int64_t)E * n3) return;
  const int64_t e = x / n3;
  const int t = (int)(x % n3);
  for (int c = 0; c < 12; ++c) out[x * 12 + c] = g[e * 12 * n3 + (int64_t)c * n3 + t];
}

template <int N>
__global__ void k_debug_fstar(int E, const int* __restrict__ elem_side, const double* __restrict__ fstar,
                              double* out) {
  constexpr int n2 = (N + 1) * (N + 1);
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= (int64_t)E * 6 * n2) return;
  const int64_t ef = x / n2;
  const int pq = (int)(x % n2);
  const int es = elem_side[ef];
  for (int k = 0; k < 5; ++k)
    out[x * 5 + k] = es_slave(es) ? 0.0 : fstar[(int64_t)es_side(es) * 5 * n2 + k * n2 + pq];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static StageArgs make_args(dg_ctx* c, const double* U) {
  StageArgs a{};
  a.E = (int)c->E;
  a.S = (int)c->S;
  a.U = U;
  a.metric = c->metric;
  a.nrm = c->nrm;
  a.elem_side = c->elem_side;
  a.side_e = c->side_e;
  a.side_f = c->side_f;
  a.g = c->g;
  a.lflux = c->lflux;
  a.fstar = c->fstar;
  a.alpha = c->alpha;
  a.fvmetric = c->fvmetric;
  a.ops = c->ops;
  a.gamma = c->prm.gamma;
  a.gm1 = c->prm.gamma - 1.0;
  a.Rinv = 1.0 / c->prm.R;
  a.mu = c->prm.mu;
  a.lam = c->prm.gamma * c->prm.R * c->prm.mu / ((c->prm.gamma - 1.0) * c->prm.Pr);
  a.riemann = c->prm.riemann;
  a.viscous = c->prm.viscous;
  a.shock = c->prm.shock_capturing;
  a.alpha_min = c->prm.alpha_min;
  a.alpha_max = c->prm.alpha_max;
  a.alpha_force = c->prm.alpha_force;
  a.scal = c->scal;
  return a;
}

template <int N>
static size_t volume_smem() {
  using S = Shape<N>;
  return sizeof(double) * (3 * S::n2 + S::EPB * ((6 + 9 + 5 + 2) * S::n3 + 4 * S::n2));
}
template <int N>
static size_t lift_smem() {
  using S = Shape<N>;
  return sizeof(double) * (S::n2 + S::EPB * 16 * S::n3);
}

template <int N>
static cudaError_t set_attrs() {
  cudaFuncSetAttribute(k_lift<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lift_smem<N>());
  cudaFuncSetAttribute(k_volume<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)volume_smem<N>());
  cudaFuncSetAttribute(k_volume<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)volume_smem<N>());
  return cudaGetLastError();
}

template <int N>
static cudaError_t rhs_impl(dg_ctx* c, const double* U, int mode, double rkA, double rkB, int first) {
  using S = Shape<N>;
  StageArgs a = make_args(c, U);
  a.Ut = c->Ut;
  a.Urk = c->U;
  a.dU = c->dU;
  a.rkA = rkA;
  a.rkB = rkB;
  a.first_stage = first;
  const int64_t side_nodes = c->S * S::n2;
  const unsigned sb = (unsigned)((side_nodes + 255) / 256);
  const unsigned eb = (unsigned)((c->E + S::EPB - 1) / S::EPB);
  if (c->prm.viscous) {
    prof_begin(c, PK_SURF_PRIMS);
    k_surf_prims<N><<<sb, 256, 0, c->stream>>>(a);
    prof_end(c);
    prof_begin(c, PK_LIFT);
    k_lift<N><<<eb, S::THREADS, lift_smem<N>(), c->stream>>>(a);
    prof_end(c);
    count_launch(2);
  }
  prof_begin(c, PK_SURF_FLUX);
  k_surf_flux<N><<<sb, 256, 0, c->stream>>>(a);
  prof_end(c);
  prof_begin(c, PK_VOLUME);
  if (mode == 0) k_volume<N, 0><<<eb, S::THREADS, volume_smem<N>(), c->stream>>>(a);
  else k_volume<N, 1><<<eb, S::THREADS, volume_smem<N>(), c->stream>>>(a);
  prof_end(c);
  count_launch(2);
  return cudaGetLastError();
}

#define DG_DISPATCH(N_, CALL)          \
  switch (N_) {                        \
    case 1: { constexpr int NN = 1; CALL; } break; \
    case 2: { constexpr int NN = 2; CALL; } break; \
    case 3: { constexpr int NN = 3; CALL; } break; \
    case 4: { constexpr int NN = 4; CALL; } break; \
    case 5: { constexpr int NN = 5; CALL; } break; \
    case 6: { constexpr int NN = 6; CALL; } break; \
    case 7: { constexpr int NN = 7; CALL; } break; \
    default: return cudaErrorInvalidValue;         \
  }

cudaError_t init_kernel_attributes(int N) {
  DG_DISPATCH(N, return set_attrs<NN>());
  return cudaSuccess;
}

cudaError_t launch_rhs(dg_ctx* c, const double* U, int mode, double rkA, double rkB, int first) {
  DG_DISPATCH(c->N, return rhs_impl<NN>(c, U, mode, rkA, rkB, first));
  return cudaSuccess;
}

static int cfl_blocks(dg_ctx* c) {
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t need = (c->E * c->n3 + 255) / 256;
  return (int)std::min<int64_t>(need, (int64_t)sms * 8);
}

cudaError_t launch_cfl(dg_ctx* c) {
  const double kv = std::max(4.0 / 3.0, c->prm.gamma / c->prm.Pr) * c->prm.mu;
  const int nb = cfl_blocks(c);
  prof_begin(c, PK_CFL);
  DG_DISPATCH(c->N, (k_cfl<NN><<<nb, 256, 0, c->stream>>>((int)c->E, c->U, c->metric, c->prm.gamma,
                                                          c->prm.gamma - 1.0, 1.0 / c->prm.R, kv, c->prm.viscous,
                                                          c->scal)));
  k_dt<<<1, 1, 0, c->stream>>>(c->scal, c->prm.cfl, c->prm.dfl, c->N, c->prm.viscous);
  prof_end(c);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_to_internal(dg_ctx* c, const double* pub, double* internal) {
  const int64_t tot = c->E * c->n3 * 5;
  k_to_internal<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(c->E, c->n3, pub, internal);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_to_public(dg_ctx* c, const double* internal, double* pub) {
  const int64_t tot = c->E * c->n3 * 5;
  k_to_public<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(c->E, c->n3, internal, pub);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_kinetic(dg_ctx* c, const double* U, const double* Ut) {
  const int nb = cfl_blocks(c);
  DG_DISPATCH(c->N, (k_kinetic<NN><<<nb, 256, 0, c->stream>>>((int)c->E, U, Ut, c->metric, c->ops, c->scal)));
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_debug_metrics(dg_ctx* c, double* Ja, double* J) {
  const int64_t tot = c->E * c->n3;
  DG_DISPATCH(c->N, (k_debug_metrics<NN><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>((int)c->E,
                                                                                               c->metric, Ja, J)));
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_debug_maps(dg_ctx* c, int* nbr, int* nodes) {
  const int64_t tot = c->E * 6;
  DG_DISPATCH(c->N, (k_debug_maps<NN><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
                        (int)c->E, c->elem_side, c->side_e, c->side_f, nbr, nodes)));
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_debug_grad(dg_ctx* c, double* out) {
  const int64_t tot = c->E * c->n3;
  DG_DISPATCH(c->N, (k_debug_grad<NN><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>((int)c->E, c->g, out)));
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_debug_fstar(dg_ctx* c, double* out) {
  const int64_t tot = c->E * 6 * c->n2;
  DG_DISPATCH(c->N, (k_debug_fstar<NN><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
                        (int)c->E, c->elem_side, c->fstar, out)));
  count_launch();
  return cudaGetLastError();
}

}  // namespace dg
