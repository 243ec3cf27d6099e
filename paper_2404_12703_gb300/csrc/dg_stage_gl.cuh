// dg_stage_gl.cuh -- the element kernels of the standard DGSEM on
// Gauss-Legendre nodes (Eq. dgsem with lhat+-_i = l_i(+-1) / w_i; Sec. 5.1
// runs this scheme's convergence test), templated on the arithmetic type T
// like the LGL kernels (the side kernels are shared, reading the face states
// from the arrays written here).
//
// Per stage:
//   k_prolong_gl   ProlongToFace: the state interpolated to the six faces
//                  with l(+-1), stored per side in the master's face frame
//   k_surf_prims   BR1 surface flux of the lifted primitives  (GL variant)
//   k_lift_gl      lifted gradients: volume part with Dhat, surface part
//                  spread over every node of a line with l(+-1)/w, 1/J;
//                  then the ProlongToFace of the gradients
//   k_surf_flux    Riemann + BR1 viscous flux times s          (GL variant)
//   k_volume_gl    collocated flux divergence sum_a Dhat_ia (J a . (F_c -
//                  F_v))_a, SurfInt over every node, ApplyJac and Ut or the
//                  RK update
// Unlike on LGL nodes, no face value is a nodal value, and every node of an
// element receives surface contributions from both faces of each of its
// three lines.
#pragma once

namespace dg {

// face-frame index (p + n q) of node idx on the faces normal to direction d
template <int n>
__device__ __forceinline__ int line_face_pq(int d, const int idx[3]) {
  const int p = d == 0 ? idx[1] : idx[0];
  const int q = d == 2 ? idx[1] : idx[2];
  return p + n * q;
}

// the side of local face f of element e, whether e is its slave, and face
// point (p, q) of e's face frame in the master's face frame
struct FaceRef {
  int s, pqm;
  bool slave;
};
template <int n>
__device__ __forceinline__ FaceRef face_ref(const StageArgs& a, int e, int f, int p, int q) {
  const int es = a.elem_side[(size_t)e * 6 + f];
  int pm = p, qm = q;
  if (es_slave(es)) flip_to_master<n>(es_flip(es), p, q, pm, qm);
  return {es_side(es), pm + n * qm, es_slave(es) != 0};
}

// node 0 of the line of direction f / 2 through face point (p, q), and the stride
template <int n>
__device__ __forceinline__ void face_line(int f, int p, int q, int& v0, int& st) {
  constexpr int n2 = n * n;
  const int d = f >> 1;
  st = d == 0 ? 1 : (d == 1 ? n : n2);
  v0 = face_vol_node<n>(f, p, q) - ((f & 1) ? n - 1 : 0) * st;
}

// shared-memory sizes (bytes)
template <int N>
constexpr size_t gl_prolong_smem() {
  using S = Shape<N>;
  return sizeof(double) * S::EPB * 5 * S::n3;
}
template <int N>
constexpr int gl_lift_nf() {  // products, staged face fluxes and gradients share one array
  using S = Shape<N>;
  return 12 * S::n3 > 72 * S::n2 ? 12 * S::n3 : 72 * S::n2;
}
template <int N, typename T>
constexpr size_t gl_lift_smem() {
  using S = Shape<N>;
  return sizeof(T) * (((S::n2 + 3) & ~3) + 16 + S::EPB * (4 * S::n3 + gl_lift_nf<N>()));
}
template <int N, typename T>
constexpr size_t gl_volume_smem() {
  using S = Shape<N>;
  return sizeof(T) * (((S::n2 + 3) & ~3) + 16 + S::EPB * (5 * S::n3 + 30 * S::n2));
}

// ---------------------------------------------------------------------------
// ProlongToFace of the state (FP64 in both precisions: the FP32-bulk
// primitives are formed from FP64 deviations)
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Shape<N>::THREADS) k_prolong_gl(StageArgs a) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* sU = reinterpret_cast<double*>(smraw);  // [EPB][5][n3]
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  // slots past the last element redo the last one and store nothing
  const bool valid = blockIdx.x * EPB + le < a.E;
  const int e = valid ? blockIdx.x * EPB + le : a.E - 1;
  double* U = sU + le * 5 * n3;
  const double* u = a.U + (size_t)e * 5 * n3 + t;
#pragma unroll
  for (int k = 0; k < 5; ++k) U[k * n3 + t] = u[k * n3];
  __syncwarp();
  __syncthreads();
  if (!valid) return;
  for (int task = t; task < 6 * n2; task += n3) {
    const int f = task / n2, pq = task % n2, p = pq % n, q = pq / n;
    int v0, st;
    face_line<n>(f, p, q, v0, st);
    const double* L = (f & 1) ? a.ops->Lp : a.ops->Lm;
    double val[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int al = 0; al < n; ++al) {
      const double c = L[al];
#pragma unroll
      for (int k = 0; k < 5; ++k) val[k] += c * U[k * n3 + v0 + al * st];
    }
    const FaceRef r = face_ref<n>(a, e, f, p, q);
    double* o = a.Ufc + ((size_t)r.s * 2 + (r.slave ? 1 : 0)) * 5 * n2 + r.pqm;
#pragma unroll
    for (int k = 0; k < 5; ++k) o[k * n2] = val[k];
  }
}

// ---------------------------------------------------------------------------
// Lifted gradients (weak form, Eq. lifting) and their ProlongToFace
// ---------------------------------------------------------------------------
template <int N, typename T>
__global__ void __launch_bounds__(Shape<N>::THREADS) k_lift_gl(StageArgs a) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  constexpr int n2p = (n2 + 3) & ~3;
  constexpr int nF = gl_lift_nf<N>();
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sDh = reinterpret_cast<T*>(smraw);  // [n2p] Dhat
  T* sLw = sDh + n2p;                    // [16]: l_i(-1) / w_i at i, l_i(+1) / w_i at 8 + i
  T* sq = sLw + 16;                      // [EPB][4][n3] lifted primitives
  T* sF = sq + EPB * 4 * n3;             // [EPB][nF] products / face fluxes / gradients
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  const bool valid = blockIdx.x * EPB + le < a.E;
  const int e = valid ? blockIdx.x * EPB + le : a.E - 1;
  const CaseParams cp = case_params(a, 0);
  for (int k = threadIdx.x; k < n2; k += blockDim.x) sDh[k] = T(a.ops->Dhat[k]);
  if (threadIdx.x < n) {
    sLw[threadIdx.x] = T(a.ops->Lm[threadIdx.x] * a.ops->winv[threadIdx.x]);
    sLw[8 + threadIdx.x] = T(a.ops->Lp[threadIdx.x] * a.ops->winv[threadIdx.x]);
  }
  T* q = sq + le * 4 * n3;
  T* F = sF + le * nF;
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
  // volume part: sum_d sum_a Dhat_ia (J a^d q)_a along each line
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    {
      const T J0 = metric_at<T>(a, e, d * 3, t, n3), J1 = metric_at<T>(a, e, d * 3 + 1, t, n3),
              J2 = metric_at<T>(a, e, d * 3 + 2, t, n3);
#pragma unroll
      for (int qv = 0; qv < 4; ++qv) {
        const T qq = q[qv * n3 + t];
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
        const T c = sDh[id * n + al];
        const int nb = base + al * str[d];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] += c * F[k * n3 + nb];
      }
    }
    __syncwarp();
    __syncthreads();
  }
  // surface part: the six faces' lifting fluxes q* (s n), signed for this
  // element (the slave's outward normal is minus the master's), in this
  // element's face frame, then spread over the lines with l(+-1) / w
  const T* Lf = TBuf<T>::lflux(a);
  for (int task = t; task < 6 * n2; task += n3) {
    const int f = task / n2, pq = task % n2;
    const FaceRef r = face_ref<n>(a, e, f, pq % n, pq / n);
    const T sg = r.slave ? T(-1) : T(1);
    const T* L = Lf + (size_t)r.s * 12 * n2 + r.pqm;
#pragma unroll
    for (int k = 0; k < 12; ++k) F[(f * 12 + k) * n2 + pq] = sg * L[k * n2];
  }
  __syncwarp();
  __syncthreads();
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id = idx[d], pq = line_face_pq<n>(d, idx);
    const T cm = sLw[id], cpl = sLw[8 + id];
#pragma unroll
    for (int k = 0; k < 12; ++k)
      acc[k] += cm * F[(2 * d * 12 + k) * n2 + pq] + cpl * F[((2 * d + 1) * 12 + k) * n2 + pq];
  }
  const T Ji = metric_at<T>(a, e, 9, t, n3);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] *= Ji;
  if (valid) {
    T* g = TBuf<T>::g(a) + (size_t)e * 12 * n3 + t;
#pragma unroll
    for (int k = 0; k < 12; ++k) g[k * n3] = acc[k];
  }
  __syncwarp();
  __syncthreads();  // the staged face fluxes are read by all threads
#pragma unroll
  for (int k = 0; k < 12; ++k) F[k * n3 + t] = acc[k];
  __syncwarp();
  __syncthreads();
  if (!valid) return;
  // ProlongToFace of the gradients
  T* Gf = TBuf<T>::gfc(a);
  for (int task = t; task < 6 * n2; task += n3) {
    const int f = task / n2, pq = task % n2, p = pq % n, qq = pq / n;
    int v0, st;
    face_line<n>(f, p, qq, v0, st);
    const double* L = (f & 1) ? a.ops->Lp : a.ops->Lm;
    T val[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) val[k] = T(0);
#pragma unroll
    for (int al = 0; al < n; ++al) {
      const T c = T(L[al]);
#pragma unroll
      for (int k = 0; k < 12; ++k) val[k] += c * F[k * n3 + v0 + al * st];
    }
    const FaceRef r = face_ref<n>(a, e, f, p, qq);
    T* o = Gf + ((size_t)r.s * 2 + (r.slave ? 1 : 0)) * 12 * n2 + r.pqm;
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k * n2] = val[k];
  }
}

// ---------------------------------------------------------------------------
// Volume integral (collocated flux divergence) + SurfInt + ApplyJac (+ RK)
// ---------------------------------------------------------------------------
template <int N, int MODE, typename T>
__global__ void __launch_bounds__(Shape<N>::THREADS) k_volume_gl(StageArgs a) {
  using S = Shape<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  constexpr int n2p = (n2 + 3) & ~3;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sDh = reinterpret_cast<T*>(smraw);  // [n2p] Dhat
  T* sLw = sDh + n2p;                    // [16]: l(-1) / w, l(+1) / w
  T* sG = sLw + 16;                      // [EPB][5][n3] contravariant fluxes
  T* sFs = sG + EPB * 5 * n3;            // [EPB][6][5][n2] signed surface fluxes
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  const bool valid = blockIdx.x * EPB + le < a.E;
  const int e = valid ? blockIdx.x * EPB + le : a.E - 1;
  const CaseParams cp = case_params(a, 0);
  for (int k = threadIdx.x; k < n2; k += blockDim.x) sDh[k] = T(a.ops->Dhat[k]);
  if (threadIdx.x < n) {
    sLw[threadIdx.x] = T(a.ops->Lm[threadIdx.x] * a.ops->winv[threadIdx.x]);
    sLw[8 + threadIdx.x] = T(a.ops->Lp[threadIdx.x] * a.ops->winv[threadIdx.x]);
  }
  T* G = sG + le * 5 * n3;
  T* Fs = sFs + le * 30 * n2;
  double U[5];
  {
    const double* u = a.U + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k] = u[k * n3];
  }
  const SPrim<T> me = shifted_prim<T, true>(U, a.gm1, a.Rinv, cp);
  T tau[6] = {0, 0, 0, 0, 0, 0}, W[3] = {0, 0, 0};
  if (a.viscous) {
    T g[12];
    const T* pg = TBuf<T>::g(a) + (size_t)e * 12 * n3 + t;
#pragma unroll
    for (int k = 0; k < 12; ++k) g[k] = pg[k * n3];
    T vmu, vlam;
    visc_coeffs<T>(a, cp, me.Tt, vmu, vlam);
    viscous_parts(g, me.u, me.v, me.w, vmu, vlam, tau, W);
  }
  const int idx[3] = {t % n, (t / n) % n, t / n2};
  constexpr int str[3] = {1, n, n2};
  T acc[5] = {0, 0, 0, 0, 0};
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    {
      const T nv[3] = {metric_at<T>(a, e, 3 * d, t, n3), metric_at<T>(a, e, 3 * d + 1, t, n3),
                       metric_at<T>(a, e, 3 * d + 2, t, n3)};
      T fc[5];
      euler_flux_s(me, nv, fc);
      if (a.viscous) {
        T fv[4];
        viscous_flux_n(tau, W, nv, fv);
#pragma unroll
        for (int k = 0; k < 4; ++k) fc[1 + k] -= fv[k];
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) G[k * n3 + t] = fc[k];
    }
    __syncwarp();
    __syncthreads();
    {
      const int id = idx[d], base = t - id * str[d];
#pragma unroll
      for (int al = 0; al < n; ++al) {
        const T c = sDh[id * n + al];
        const int nb = base + al * str[d];
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += c * G[k * n3 + nb];
      }
    }
    __syncwarp();
    __syncthreads();
  }
  // SurfInt: the six faces' fluxes f* s, signed for this element, spread
  // over the lines with l(+-1) / w
  const T* Fst = TBuf<T>::fstar(a);
  for (int task = t; task < 6 * n2; task += n3) {
    const int f = task / n2, pq = task % n2;
    const FaceRef r = face_ref<n>(a, e, f, pq % n, pq / n);
    const T sg = r.slave ? T(-1) : T(1);
    const T* src = Fst + (size_t)r.s * 5 * n2 + r.pqm;
#pragma unroll
    for (int k = 0; k < 5; ++k) Fs[(f * 5 + k) * n2 + pq] = sg * src[k * n2];
  }
  __syncwarp();
  __syncthreads();
  if (!valid) return;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id = idx[d], pq = line_face_pq<n>(d, idx);
    const T cm = sLw[id], cpl = sLw[8 + id];
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += cm * Fs[(2 * d * 5 + k) * n2 + pq] + cpl * Fs[((2 * d + 1) * 5 + k) * n2 + pq];
  }
  // ApplyJac; the energy equation gets H_ref times the mass equation back
  const T Ji = metric_at<T>(a, e, 9, t, n3);
  double Ut[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) Ut[k] = to_f64<T>(-acc[k] * Ji);
  Ut[4] += cp.Hr * Ut[0];
  if (a.sponge_sigma) {  // sponge source -sigma (U - U_base), FP64
    const double sg = a.sponge_sigma[(size_t)e * n3 + t];
    const double* ub = a.sponge_base + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) Ut[k] -= sg * (U[k] - ub[k * n3]);
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

}  // namespace dg
