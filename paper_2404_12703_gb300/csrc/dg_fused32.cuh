// dg_fused32.cuh -- the FP32-bulk stage in two kernels (included by
// dg_stage.cuh).
//
// The four-kernel stage (k_surf_prims, k_lift, k_surf_flux, k_volume) sends
// the lifted gradients [E][12][n3] and the BR1 lifting fluxes through HBM
// and gathers face values out of element-major arrays.  In FP32-bulk, where
// a stage is bound by memory traffic and latency rather than arithmetic, this
// form moves only the state, the RK register, the metrics and per-side face
// data:
//
//   k_fflux  (one thread per side node)  FillFlux and Lift_FillFlux: the Roe
//            or LF flux from the two elements' face traces, the BR1 mean q*
//            of the lifted primitives, and the BR1 viscous flux
//            -1/2 (F_v(L) + F_v(R)) . s n, with each side's face gradient
//            completed here from its element's partial viscous flux
//   k_felem  (one block per element)     ConsToPrim, the lifting (volume part
//            and the six faces' q*), the split-form KEP volume integral, the
//            viscous volume term, the optional FV blending, SurfInt, ApplyJac
//            and the RK update, then an epilogue that prepares the next
//            stage's face data from the updated state
//   k_fprep  (one block per element)     the epilogue alone, for a state that
//            no stage produced (a new state, dg_rhs)
//
// Face data, per side and element of the side (half 0: master, 1: slave),
// at every face node in the master's face frame:
//   tr32  [S][2][n2][8] floats: (u, v, w, T') and (rho, p', H', 1/J) of the
//         element's face node (shifted primitives, as ConsToPrim forms them)
//   pfv32 [S][2][n2][4] floats: F_v(q, g_part) . (s n), with g_part the
//         element's lifted gradient at the node without its neighbours'
//         halves of q*:  g_part = (1/J) [ sum_d Dhat (Ja^d q) +
//         sum_{faces f through the node} +-lhat (q_own / 2) (s n)_f ]
//   qs32  [S][n2] float4: q* = (q_master + q_slave) / 2 of (u, v, w, T')
//
// Why the split is exact: BR1's face gradient is
//   g = g_part + (1/J) sum_{f through the node} +-lhat (q_nbr(f) / 2) (s n)_f
// and F_v(q, g) is linear in g for fixed (u, v, w, mu, lambda) (Eq. nse,
// stress tensor and Fourier law; Sutherland's mu depends on T only), so
// F_v(q, g) . n = F_v(q, g_part) . n + F_v(q, g - g_part) . n.  The second
// part needs the neighbours' traces across every face through the node: one
// face for a face-interior node, two or three at element edges and corners
// (the diagonal neighbours, reached through the element's side map).
//
// Data flow of stage s: k_fflux reads the face data of U_s (written by the
// previous stage's epilogue, or by k_fprep) and writes f* and q*; k_felem
// reads U_s, the RK register, the metrics, q* and f*, and writes U_{s+1}, the
// register and the face data of U_{s+1}.  Inside k_felem no element reads
// face data that another element's epilogue writes (q* and f* come from
// k_fflux), so the update in place is race-free.
#pragma once
#ifdef DG_CHECK
#include <cstdio>
#endif

namespace dg {

// Debug builds (-DDG_CHECK): every index into global memory and into the
// element's shared-memory arrays is checked before use; a bad one is
// printed with the source line and the access is skipped.
#ifdef DG_CHECK
static __device__ __noinline__ bool dg_chk(bool ok, int line, long long v) {
  if (!ok) printf("DG_CHECK line %d block %d thread %d value %lld\n", line, (int)blockIdx.x, (int)threadIdx.x, v);
  return ok;
}
#define DG_CHK(cond, v) dg_chk((cond), __LINE__, (long long)(v))
#else
#define DG_CHK(cond, v) true
#endif

// ---------------------------------------------------------------------------
// Shared-memory layout of the element kernels (FP32 arrays after the FP64 ones)
// ---------------------------------------------------------------------------
template <int N, int EPB_ = 0>
struct FusedSmem {
  using S = Shape<N, EPB_>;
  static constexpr int n2d = (S::n2 + 1) & ~1;  // Vinv (FP64), even count: 16-byte aligned after it
  static constexpr int n2p = (S::n2 + 3) & ~3;  // Dsplit / Dhat (FP32)
  static constexpr int n4 = (S::n + 3) & ~3;    // a row of Dhat padded to whole float4s
  // a node plane with one pad word after every line of n nodes (pad_idx):
  // lines along any direction then fall in distinct banks
  static constexpr int Pn = S::n3 + S::n2;
  // per element: P (2 float4 per node: (rho, u, v, w) / 2 and (p', H') / 2, T'),
  // J (3 float4 planes, (Ja^d) / 2), q (4 planes: u, v, w, T'), W (12 planes:
  // lifting sums; also viscous / FV fluxes and the FP64 indicator scratch),
  // face normals (6 faces x n2 float4: s n and the SurfInt sign)
  static constexpr int offJ = 8 * S::n3, offQ = offJ + 12 * Pn, offW = offQ + 4 * Pn, offN = offW + 12 * Pn;
  static constexpr int per_elem_f = offN + 24 * S::n2;
  static constexpr size_t bytes =
      sizeof(double) * n2d + sizeof(float) * (2 * n2p + S::n * n4 + S::EPB * per_elem_f);
  static_assert(2 * S::n3 + 4 * S::n2 <= 6 * Pn, "the indicator scratch fits the W workspace");
  static_assert((2 * n2p + S::n * n4) % 4 == 0 && per_elem_f % 4 == 0 && offQ % 4 == 0 && offW % 4 == 0 &&
                    offN % 4 == 0,
                "16-byte alignment of the float4 planes");
};

// padded plane index of node t: one pad word after each line of n nodes
template <int n>
__device__ __forceinline__ int pad_idx(int t) {
  return t + t / n;
}

// the side record of element e's face f at its face-frame node (p, q):
// side s, half (0: e is the master, 1: the slave), node index in the master frame
template <int n>
__device__ __forceinline__ void face_record(const int* __restrict__ elem_side, int e, int f, int p, int q, int& s,
                                            int& half, int& pq) {
  const int es = DG_CHK(f >= 0 && f < 6 && p >= 0 && p < n && q >= 0 && q < n, f * 100 + p * 10 + q)
                     ? elem_side[(size_t)e * 6 + f]
                     : 0;
  s = es_side(es);
  half = es_slave(es);
  int pm = p, qm = q;
  if (half) flip_to_master<n>(es_flip(es), p, q, pm, qm);
  pq = pm + n * qm;
}

// face-frame coordinates (p, q) of node idx on a face of direction d:
// (j, k) for d = 0, (i, k) for d = 1, (i, j) for d = 2
__device__ __forceinline__ void face_pq(int d, const int idx[3], int& p, int& q) {
  p = d == 0 ? idx[1] : idx[0];
  q = d == 2 ? idx[1] : idx[2];
}

// node t's index along direction d and the node stride of direction d, as
// register selects: the loops over d below index no local-memory arrays
template <int n>
__device__ __forceinline__ int dir_index(int t, int d) {
  return d == 0 ? t % n : (d == 1 ? (t / n) % n : t / (n * n));
}
template <int n>
__device__ __forceinline__ int dir_stride(int d) {
  return d == 0 ? 1 : (d == 1 ? n : n * n);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// L2 prefetch of a byte range [p, p + bytes) kept inside [lo, hi) (both ends
// rounded inwards to 16 bytes, as the bulk prefetch requires)
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes, const void* lo, const void* hi) {
  uintptr_t a = (uintptr_t)p, b = a + bytes;
  const uintptr_t l = (uintptr_t)lo, h = (uintptr_t)hi;
  if (a < l) a = l;
  if (b > h) b = h;
  a = (a + 15) & ~(uintptr_t)15;
  b &= ~(uintptr_t)15;
  if (b <= a) return;
  if (!DG_CHK(a >= l && b <= h && ((a | b) & 15) == 0, (long long)(b - a))) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a), "r"((unsigned)(b - a)) : "memory");
}

// ---------------------------------------------------------------------------
// The weak-form volume part of the lifting (Eq. lifting) at node t:
//   acc[qv * 3 + x] = sum_d sum_al Dhat[id_d][al] (Ja^d_x q_qv)_al
// Register-blocked: per direction, one task per (line, variable) loads the
// line's q_qv and Ja^d once, forms the three products in registers and applies
// the n x n matrix Dhat (rows read as broadcast float4s) to them; the three
// sums of each node go to the W planes (written for the first direction,
// added for the others).  Qs: the element's q planes (u, v, w, T'); J4: its
// halved metrics; W: its 12 workspace planes; sDr: Dhat with rows padded to
// n4 floats.  Every thread of the block calls it (it holds barriers); W may
// be reused after the caller's next barrier.
// ---------------------------------------------------------------------------
// FACES: only the sums at the element's face nodes are needed (the
// epilogue): a line inside the element in both other directions computes its
// two end nodes only; every face node lies on a line that computes it for
// each direction.
template <int n, int n4, bool FACES = false>
__device__ __forceinline__ void lift_volume(const float* Qs, const float4* J4, float* W, const float* sDr, int t,
                                            float acc[12]) {
  constexpr int n2 = n * n, n3 = n2 * n, Pn = n3 + n2;
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    const int sd = dir_stride<n>(d);
    for (int task = t; task < 4 * n2; task += n3) {
      const int qv = task / n2, l = task % n2, lp = l % n, lq = l / n;
      const int base = d == 0 ? n * (lp + n * lq) : (d == 1 ? lp + n2 * lq : lp + n * lq);
      float P0[n], P1[n], P2[n];
#pragma unroll
      for (int al = 0; al < n; ++al) {
        const int v = pad_idx<n>(base + al * sd);
        const float q = Qs[qv * Pn + v];
        const float4 j = J4[d * Pn + v];
        P0[al] = (2.0f * j.x) * q;  // exact: the halving undone
        P1[al] = (2.0f * j.y) * q;
        P2[al] = (2.0f * j.z) * q;
      }
      const bool inner = FACES && lp > 0 && lp < n - 1 && lq > 0 && lq < n - 1;
#pragma unroll
      for (int i = 0; i < n; ++i) {
        if (inner && i > 0 && i < n - 1) continue;
        float r[n4];
#pragma unroll
        for (int c = 0; c < n4; c += 4) {
          const float4 v4 = *reinterpret_cast<const float4*>(sDr + i * n4 + c);
          r[c] = v4.x, r[c + 1] = v4.y, r[c + 2] = v4.z, r[c + 3] = v4.w;
        }
        float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f;
#pragma unroll
        for (int al = 0; al < n; ++al) {
          o0 += r[al] * P0[al];
          o1 += r[al] * P1[al];
          o2 += r[al] * P2[al];
        }
        float* w = W + (qv * 3) * Pn + pad_idx<n>(base + i * sd);
        if (d == 0) {
          w[0] = o0, w[Pn] = o1, w[2 * Pn] = o2;
        } else {
          w[0] += o0, w[Pn] += o1, w[2 * Pn] += o2;
        }
      }
    }
    __syncwarp();
    __syncthreads();
  }
  const int v = pad_idx<n>(t);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = W[k * Pn + v];
}

// Loads the element's face normals into shared memory: sSn[f][pq] = (s n of
// the side, in the master's direction; SurfInt / lifting sign +-1/w_0), for
// each face f and face-frame node pq of the element.
template <int n>
__device__ __forceinline__ void load_face_normals(const StageArgs& a, int e, int t, float4* sSn) {
  constexpr int n2 = n * n;
  const float w0 = (float)a.ops->winv[0];  // = 1 / w_N on LGL nodes
  for (int k = t; k < 6 * n2; k += n2 * n) {
    const int f = k / n2, pq = k % n2;
    int s, half, pm;
    face_record<n>(a.elem_side, e, f, pq % n, pq / n, s, half, pm);
    if (!DG_CHK(s >= 0 && s < a.S && pm >= 0 && pm < n2 && e >= 0 && e < a.E, s)) continue;
    const float* nr = a.nrm32 + (size_t)s * 7 * n2 + pm;
    sSn[k] = make_float4(nr[0], nr[n2], nr[2 * n2], half ? -w0 : w0);
  }
}

// ---------------------------------------------------------------------------
// Epilogue: the face data of a state for the next k_fflux.  me: the node's
// shifted primitives; Jinv its 1/J; sSn the element's face normals.  All
// threads of the block call it (the lifting holds barriers); `valid` masks
// the stores.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void face_epilogue(const StageArgs& a, const CaseParams& cp, int e, int t, bool valid,
                                              const SPrim<float>& me, float Jinv, const float4* J4, float* Qs,
                                              float* Wk, const float* sDr, const float4* sSn) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  constexpr int Pn = n3 + n2, n4 = (n + 3) & ~3;
  const int idx[3] = {t % n, (t / n) % n, t / n2};
  const float q[4] = {me.u, me.v, me.w, me.Tt};
  float acc[12];
  if (a.viscous) {  // block-uniform condition
    const int v = pad_idx<n>(t);
#pragma unroll
    for (int k = 0; k < 4; ++k) Qs[k * Pn + v] = q[k];
    __syncwarp();
    __syncthreads();
    lift_volume<n, n4, true>(Qs, J4, Wk, sDr, t, acc);
  }
  if (!valid) return;
  bool on[3];
  int sd[3], hd[3], pqd[3];
  float4 nd[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    on[d] = idx[d] == 0 || idx[d] == n - 1;
    if (!on[d]) continue;
    const int f = 2 * d + (idx[d] == n - 1 ? 1 : 0);
    int p, qq;
    face_pq(d, idx, p, qq);
    face_record<n>(a.elem_side, e, f, p, qq, sd[d], hd[d], pqd[d]);
    nd[d] = DG_CHK(f * n2 + p + n * qq < 6 * n2, f * n2 + p + n * qq) ? sSn[f * n2 + p + n * qq] : make_float4(0, 0, 0, 0);
  }
  if (!(on[0] || on[1] || on[2])) return;
  // own halves of q* on every face through the node
  float tau[6], W[3];
  if (a.viscous) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (!on[d]) continue;
      const float4 sn = nd[d];
#pragma unroll
      for (int qv = 0; qv < 4; ++qv) {
        const float h = sn.w * (0.5f * q[qv]);
        acc[qv * 3 + 0] += h * sn.x;
        acc[qv * 3 + 1] += h * sn.y;
        acc[qv * 3 + 2] += h * sn.z;
      }
    }
    float g[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) g[k] = acc[k] * Jinv;
    float vmu, vlam;
    visc_coeffs<float>(a, cp, me.Tt, vmu, vlam);
    viscous_parts(g, me.u, me.v, me.w, vmu, vlam, tau, W);
  }
  const float4 r0 = make_float4(me.u, me.v, me.w, me.Tt), r1 = make_float4(me.rho, me.p, me.H, Jinv);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!on[d]) continue;
    const size_t rec = ((size_t)sd[d] * 2 + hd[d]) * n2 + pqd[d];
    if (!DG_CHK(sd[d] >= 0 && sd[d] < a.S && pqd[d] >= 0 && pqd[d] < n2 && (hd[d] == 0 || hd[d] == 1), rec)) continue;
    st4(a.tr32 + rec * 8, r0);
    st4(a.tr32 + rec * 8 + 4, r1);
    if (a.viscous) {
      const float snv[3] = {nd[d].x, nd[d].y, nd[d].z};
      float fv[4];
      viscous_flux_n(tau, W, snv, fv);
      st4(a.pfv32 + rec * 4, make_float4(fv[0], fv[1], fv[2], fv[3]));
    }
  }
}

// ---------------------------------------------------------------------------
// k_fprep: face data of the state a.U
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Shape<N>::THREADS) k_fprep(StageArgs a) {
  using S = Shape<N>;
  using L = FusedSmem<N>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* sDs = reinterpret_cast<float*>(reinterpret_cast<double*>(smraw) + L::n2d);
  float* sDh = sDs + L::n2p;
  float* sDr = sDh + L::n2p;  // [n][n4] Dhat, rows padded
  float* base = sDr + n * L::n4;
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  float* mine = base + (size_t)le * L::per_elem_f;
  float4* J4 = reinterpret_cast<float4*>(mine + L::offJ);
  float* Qs = mine + L::offQ;
  float* Wk = mine + L::offW;
  float4* sSn = reinterpret_cast<float4*>(mine + L::offN);
  // the element: a.elem_off + the block's slot, or an entry of the element
  // list (a serving pool's occupied elements); slots past the end redo the
  // last element and store nothing
  const int ei = blockIdx.x * EPB + le < a.E ? blockIdx.x * EPB + le : a.E - 1;
  const int el = a.elem_list ? a.elem_list[ei] : a.elem_off + ei;
  const int ce = a.elem_case ? a.elem_case[el] : 0;
  const bool valid = blockIdx.x * EPB + le < a.E && ce >= 0;
  const int e = DG_CHK(el >= 0 && t < n3 && le < EPB, el) ? el : 0;
  const CaseParams cp = case_params(a, ce);
  for (int k = threadIdx.x; k < n * L::n4; k += blockDim.x) {
    const int i = k / L::n4, al = k % L::n4;
    sDr[k] = al < n ? (float)a.ops->Dhat[i * n + al] : 0.0f;
  }
  load_face_normals<n>(a, e, t, sSn);
  double U[5];
  const double* u = a.U + (size_t)e * 5 * n3 + t;
#pragma unroll
  for (int k = 0; k < 5; ++k) U[k] = u[k * n3];
  const SPrim<float> me = shifted_prim<float, true>(U, a.gm1, a.Rinv, cp);
  const int vp = pad_idx<n>(t);
#pragma unroll
  for (int d = 0; d < 3; ++d)
    J4[d * L::Pn + vp] = make_float4(0.5f * metric_at<float>(a, e, 3 * d, t, n3),
                                     0.5f * metric_at<float>(a, e, 3 * d + 1, t, n3),
                                     0.5f * metric_at<float>(a, e, 3 * d + 2, t, n3), 0.0f);
  const float Jinv = metric_at<float>(a, e, 9, t, n3);
  __syncwarp();
  __syncthreads();
  face_epilogue<N>(a, cp, e, t, valid, me, Jinv, J4, Qs, Wk, sDr, sSn);
}

// ---------------------------------------------------------------------------
// k_fflux: FillFlux (Roe / LF + BR1 viscous) and the lifting's q*, per side node
// ---------------------------------------------------------------------------
// the neighbours' halves of q* on the faces through an element's face node,
// times 1/J:  gc = (1/J) sum_f +-lhat (q_nbr(f) / 2) (s n)_f, for the
// element of half h of side s at master-frame node (p, q)
template <int n>
__device__ __forceinline__ void nbr_lift_part(const StageArgs& a, int s, int h, int eh, int fh, int p, int q,
                                              const float4& qn_side, const float sn_side[3], float w0, float Jinv,
                                              float gc[12]) {
  constexpr int n2 = n * n;
  // this side's own face: the neighbour is the other half
  {
    const float sg = h ? -w0 : w0;
    const float qn[4] = {qn_side.x, qn_side.y, qn_side.z, qn_side.w};
#pragma unroll
    for (int qv = 0; qv < 4; ++qv) {
      const float hq = sg * (0.5f * qn[qv]);
      gc[qv * 3 + 0] = hq * sn_side[0];
      gc[qv * 3 + 1] = hq * sn_side[1];
      gc[qv * 3 + 2] = hq * sn_side[2];
    }
  }
  // the element's own face-frame node and its volume index
  int ph = p, qh = q;
  if (h) {
    const int flip = a.side_f[s] >> 8;
    flip_to_slave<n>(flip, p, q, ph, qh);
  }
  const int t = face_vol_node<n>(fh, ph, qh);
  if (!DG_CHK(t >= 0 && t < n * n2 && fh >= 0 && fh < 6 && eh >= 0 && eh < a.E, t)) return;
  const int idx[3] = {t % n, (t / n) % n, t / n2};
  const int dh = fh >> 1;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d == dh || !(idx[d] == 0 || idx[d] == n - 1)) continue;
    const int f = 2 * d + (idx[d] == n - 1 ? 1 : 0);
    int fp, fq, s2, h2, pq2;
    face_pq(d, idx, fp, fq);
    face_record<n>(a.elem_side, eh, f, fp, fq, s2, h2, pq2);
    if (!DG_CHK(s2 >= 0 && s2 < a.S && pq2 >= 0 && pq2 < n2 && (h2 == 0 || h2 == 1), s2)) continue;
    const float4 qn4 = ld4(a.tr32 + (((size_t)s2 * 2 + (1 - h2)) * n2 + pq2) * 8);
    const float* nr = a.nrm32 + (size_t)s2 * 7 * n2 + pq2;
    const float sn[3] = {nr[0], nr[n2], nr[2 * n2]};
    const float sg = h2 ? -w0 : w0;
    const float qn[4] = {qn4.x, qn4.y, qn4.z, qn4.w};
#pragma unroll
    for (int qv = 0; qv < 4; ++qv) {
      const float hq = sg * (0.5f * qn[qv]);
      gc[qv * 3 + 0] += hq * sn[0];
      gc[qv * 3 + 1] += hq * sn[1];
      gc[qv * 3 + 2] += hq * sn[2];
    }
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) gc[k] *= Jinv;
}

// the work of side node tid (side list entry tid / n2, node tid % n2)
template <int N>
__device__ __forceinline__ void fflux_body(const StageArgs& a, int64_t tid) {
  constexpr int n = N + 1, n2 = n * n;
  if (tid >= (int64_t)a.S * n2) return;
  const int si = (int)(tid / n2), pq = (int)(tid % n2);
  const int s = a.side_list ? a.side_list[si] : si;
  const int cs = a.side_case ? a.side_case[s] : 0;
  if (cs < 0) return;                              // free side slot of a serving pool
  if (a.cases && a.cases[cs].dt == 0.0) return;  // a case that finished or sits this step out
  const CaseParams cp = case_params(a, cs);
  const float* nr = a.nrm32 + (size_t)s * 7 * n2 + pq;
  const float sn[3] = {nr[0], nr[n2], nr[2 * n2]};
  const float nu[3] = {nr[3 * n2], nr[4 * n2], nr[5 * n2]};
  const float sA = nr[6 * n2];
  const float* trM = a.tr32 + ((size_t)s * 2 * n2 + pq) * 8;
  const float* trS = trM + (size_t)n2 * 8;
  const float4 aM = ld4(trM), bM = ld4(trM + 4), aS = ld4(trS), bS = ld4(trS + 4);
  const SPrim<float> qM{bM.x, aM.x, aM.y, aM.z, bM.y, bM.z, aM.w};
  const SPrim<float> qS{bS.x, aS.x, aS.y, aS.z, bS.y, bS.z, aS.w};
  float f[5];
  if (cp.riemann == DG_RIEMANN_ROE) roe_flux_s(qM, qS, nu, a.f_gm1, cp.fHr, f);
  else lf_flux_s(qM, qS, nu, a.f_gamma, cp.fpr, f);
#pragma unroll
  for (int k = 0; k < 5; ++k) f[k] *= sA;
  if (a.viscous) {
    const float w0 = (float)a.ops->winv[0];
    const int2 ee = a.side_e[s];
    const int sf = a.side_f[s];
    const int fM = sf & 15, fS = (sf >> 4) & 15;
    const int p = pq % n, q = pq / n;
    if (!DG_CHK(ee.x >= 0 && ee.x < a.E && ee.y >= 0 && ee.y < a.E && fM < 6 && fS < 6, ee.y)) return;
    float fsum[4];
    {
      const float4 pf = ld4(a.pfv32 + ((size_t)s * 2 * n2 + pq) * 4);
      float gc[12];
      nbr_lift_part<n>(a, s, 0, ee.x, fM, p, q, aS, sn, w0, bM.w, gc);
      float tau[6], W[3], fv[4], vmu, vlam;
      visc_coeffs<float>(a, cp, qM.Tt, vmu, vlam);
      viscous_parts(gc, qM.u, qM.v, qM.w, vmu, vlam, tau, W);
      viscous_flux_n(tau, W, sn, fv);
      fsum[0] = pf.x + fv[0], fsum[1] = pf.y + fv[1], fsum[2] = pf.z + fv[2], fsum[3] = pf.w + fv[3];
    }
    {
      const float4 pf = ld4(a.pfv32 + ((size_t)s * 2 * n2 + n2 + pq) * 4);
      float gc[12];
      nbr_lift_part<n>(a, s, 1, ee.y, fS, p, q, aM, sn, w0, bS.w, gc);
      float tau[6], W[3], fv[4], vmu, vlam;
      visc_coeffs<float>(a, cp, qS.Tt, vmu, vlam);
      viscous_parts(gc, qS.u, qS.v, qS.w, vmu, vlam, tau, W);
      viscous_flux_n(tau, W, sn, fv);
      fsum[0] += pf.x + fv[0], fsum[1] += pf.y + fv[1], fsum[2] += pf.z + fv[2], fsum[3] += pf.w + fv[3];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) f[1 + k] -= 0.5f * fsum[k];
    st4(reinterpret_cast<float*>(a.qs32) + ((size_t)s * n2 + pq) * 4,
        make_float4(0.5f * (qM.u + qS.u), 0.5f * (qM.v + qS.v), 0.5f * (qM.w + qS.w), 0.5f * (qM.Tt + qS.Tt)));
  }
  float* out = a.fstar32 + (size_t)s * 5 * n2 + pq;
#pragma unroll
  for (int k = 0; k < 5; ++k) out[k * n2] = f[k];
}

template <int N>
__global__ void __launch_bounds__(256) k_fflux(StageArgs a) {
  fflux_body<N>(a, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// k_felem: one stage of one element (FP32-bulk arithmetic, FP64 state)
// ---------------------------------------------------------------------------
// MODE 0: writes Ut; MODE 1: the RK update, then (a.epilogue) the face data
// of the updated state.  a.prefetch > 0: each block first asks L2 for the
// state, RK register and metrics of the element a.prefetch blocks further on
// (the next wave on the GPU), so that wave's loads find them in L2.
// the coefficients of one low-storage RK stage
struct StageCoef {
  double A, B, C;  // dU = A dU + dt Ut, U += B dU; stage time t + C dt
  float fA;        // A in FP32 (the FP32 register update)
  int first;       // the first stage (A is not used)
};

// the work of element block blk (elements blk * EPB ... of the element list)
template <int N, int MODE, int EPB_>
__device__ __forceinline__ void felem_body(const StageArgs& a, const StageCoef& sc, unsigned blk,
                                           unsigned char* smraw) {
  using S = Shape<N, EPB_>;
  using L = FusedSmem<N, EPB_>;
  constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
  double* sVi = reinterpret_cast<double*>(smraw);  // [n2] Vinv (FP64)
  float* sDs = reinterpret_cast<float*>(sVi + L::n2d);
  float* sDh = sDs + L::n2p;
  float* sDr = sDh + L::n2p;  // [n][n4] Dhat, rows padded
  float* base = sDr + n * L::n4;
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  float* mine = base + (size_t)le * L::per_elem_f;
  float4* P4 = reinterpret_cast<float4*>(mine);                   // [n3] (rho, u, v, w) / 2
  float4* Q4 = P4 + n3;                                           // [n3] (p' / 2, H' / 2, T', 0)
  float4* J4 = reinterpret_cast<float4*>(mine + L::offJ);         // [3][Pn] (Ja^d) / 2, padded index
  float* Qs = mine + L::offQ;                                     // [4][Pn] u, v, w, T', padded index
  float* Wk = mine + L::offW;                                     // [12][Pn] workspace
  float4* G4 = reinterpret_cast<float4*>(Wk);
  float4* sSn = reinterpret_cast<float4*>(mine + L::offN);        // [6][n2] face normals and signs
  constexpr int Pn = L::Pn;
  // slots past the last element redo the last element, free slots of a
  // serving pool compute on what they hold; neither stores
  const int ei = (int)blk * EPB + le < a.E ? (int)blk * EPB + le : a.E - 1;
  const int el = a.elem_list ? a.elem_list[ei] : ei;
  const int ce = a.elem_case ? a.elem_case[el] : 0;
  // elements of cases that finished or sit this step out (time step 0) keep
  // their state and face data; a block made only of such slots leaves at once
  const bool valid = (int)blk * EPB + le < a.E && ce >= 0 && !(a.cases && a.cases[ce].dt == 0.0);
  if (a.elem_case && __syncthreads_and(!valid)) return;
  const int e = DG_CHK(el >= 0 && t < n3 && le < EPB, el) ? el : 0;
  const CaseParams cp = case_params(a, ce);
  if (a.prefetch > 0 && threadIdx.x == 0 && !a.elem_list) {
    const int64_t e2 = (int64_t)(blk + a.prefetch) * EPB;
    if (e2 < a.E) {
      const int64_t ne = min((int64_t)EPB, (int64_t)a.E - e2);
      const size_t ub = sizeof(double) * 5 * n3;
      prefetch_l2(a.U + e2 * 5 * n3, ub * ne, a.U, a.U + (size_t)a.E * 5 * n3);
      if (MODE == 1 && !sc.first) {
        const float* d32 = reinterpret_cast<const float*>(a.dU);
        prefetch_l2(d32 + e2 * 5 * n3, sizeof(float) * 5 * n3 * ne, d32, d32 + (size_t)a.E * 5 * n3);
      }
      prefetch_l2(a.metric32 + e2 * 10 * n3, sizeof(float) * 10 * n3 * ne, a.metric32,
                  a.metric32 + (size_t)a.E * 10 * n3);
    }
  }
  // this element's later gathers, asked of L2 now: its six sides' q* and f*
  // records (read after the lifting and in SurfInt) and its RK register (read
  // by the update), so that those reads do not each wait on HBM
  if (t < 6) {
    const int sf = es_side(a.elem_side[(size_t)e * 6 + t]);
    if (a.viscous)
      prefetch_l2(a.qs32 + (size_t)sf * n2 * 4, sizeof(float) * 4 * n2, a.qs32, a.qs32 + (size_t)a.S * n2 * 4);
    prefetch_l2(a.fstar32 + (size_t)sf * 5 * n2, sizeof(float) * 5 * n2, a.fstar32, a.fstar32 + (size_t)a.S * 5 * n2);
  } else if (t == 6 && MODE == 1 && !sc.first) {
    const float* d32 = reinterpret_cast<const float*>(a.dU);
    prefetch_l2(d32 + (size_t)e * 5 * n3, sizeof(float) * 5 * n3, d32, d32 + (size_t)a.E * 5 * n3);
  }
  for (int k = threadIdx.x; k < n2; k += blockDim.x) {
    sDs[k] = (float)a.ops->Dsplit[k];
    sDh[k] = (float)a.ops->Dhat[k];
    sVi[k] = a.ops->Vinv[k];
  }
  for (int k = threadIdx.x; k < n * L::n4; k += blockDim.x) {
    const int i = k / L::n4, al = k % L::n4;
    sDr[k] = al < n ? (float)a.ops->Dhat[i * n + al] : 0.0f;
  }
  load_face_normals<n>(a, e, t, sSn);
  double U[5];
  double p_full;
  {
    const double* u = a.U + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k] = u[k * n3];
  }
  // the FP64 pressure only for the indicator (one FP64 addition less otherwise)
  const SPrim<float> me = shifted_prim<float, true>(U, a.gm1, a.Rinv, cp, a.shock ? &p_full : nullptr);
  // halved values: every arithmetic mean of the two-point flux is one addition
  P4[t] = make_float4(0.5f * me.rho, 0.5f * me.u, 0.5f * me.v, 0.5f * me.w);
  Q4[t] = make_float4(0.5f * me.p, 0.5f * me.H, me.Tt, 0.0f);
  const int vp = pad_idx<n>(t);
  Qs[vp] = me.u, Qs[Pn + vp] = me.v, Qs[2 * Pn + vp] = me.w, Qs[3 * Pn + vp] = me.Tt;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    J4[d * Pn + vp] = make_float4(0.5f * metric_at<float>(a, e, 3 * d, t, n3),
                                  0.5f * metric_at<float>(a, e, 3 * d + 1, t, n3),
                                  0.5f * metric_at<float>(a, e, 3 * d + 2, t, n3), 0.0f);
  const float Jinv = metric_at<float>(a, e, 9, t, n3);
  __syncwarp();
  __syncthreads();
  const int idx[3] = {t % n, (t / n) % n, t / n2};  // indexed by unrolled (constant) d only
  float tau[6] = {0, 0, 0, 0, 0, 0}, W[3] = {0, 0, 0};
  // ---- BR1 lifting of the stage's state: volume part, then q* of the six faces ----
  if (a.viscous) {
    float g[12];
    lift_volume<n, L::n4>(Qs, J4, Wk, sDr, t, g);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int id = idx[d];
      if (id != 0 && id != n - 1) continue;
      const int f = 2 * d + (id == n - 1 ? 1 : 0);
      int p, qq;
      face_pq(d, idx, p, qq);
      const int es = a.elem_side[(size_t)e * 6 + f];
      int pm = p, qm = qq;
      if (es_slave(es)) flip_to_master<n>(es_flip(es), p, qq, pm, qm);
      if (!DG_CHK(es_side(es) >= 0 && es_side(es) < a.S && pm >= 0 && pm < n && qm >= 0 && qm < n, es_side(es)))
        continue;
      const float4 qs = ld4(a.qs32 + ((size_t)es_side(es) * n2 + pm + n * qm) * 4);
      const float4 sn = sSn[f * n2 + p + n * qq];
      const float qa[4] = {qs.x, qs.y, qs.z, qs.w};
#pragma unroll
      for (int qv = 0; qv < 4; ++qv) {
        g[qv * 3 + 0] += sn.w * (qa[qv] * sn.x);
        g[qv * 3 + 1] += sn.w * (qa[qv] * sn.y);
        g[qv * 3 + 2] += sn.w * (qa[qv] * sn.z);
      }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) g[k] *= Jinv;
    float vmu, vlam;
    visc_coeffs<float>(a, cp, me.Tt, vmu, vlam);
    viscous_parts(g, me.u, me.v, me.w, vmu, vlam, tau, W);
  }
  // ---- split-form KEP volume integral, one node per thread over its partners ----
  float accC[5] = {0, 0, 0, 0, 0};  // convective DG volume term
  float acc[5] = {0, 0, 0, 0, 0};   // viscous volume + surface terms
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    const int id = dir_index<n>(t, d), sd = dir_stride<n>(d), bse = t - id * sd;
    const float4 ai = P4[t];
    const float4 bi = Q4[t];
    const float4 ji = J4[d * Pn + vp];
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
#pragma unroll
    for (int al = 0; al < n; ++al) {
      if (al == id) continue;
      const int va = bse + al * sd;
      if (!DG_CHK(va >= 0 && va < n3, va)) continue;
      const float4 aa = P4[va];
      const float4 ba = Q4[va];
      const float4 ja = J4[d * Pn + pad_idx<n>(va)];
      const float m0 = ji.x + ja.x, m1 = ji.y + ja.y, m2 = ji.z + ja.z;
      const float rho = ai.x + aa.x;
      const float u0 = ai.y + aa.y, u1 = ai.z + aa.z, u2 = ai.w + aa.w;
      const float pp = bi.x + ba.x;
      const float H = bi.y + ba.y;
      const float fr = rho * (u0 * m0 + u1 * m1 + u2 * m2);
      const float dv = sDs[id * n + al];
      s0 += dv * fr;
      s1 += dv * (fr * u0 + pp * m0);
      s2 += dv * (fr * u1 + pp * m1);
      s3 += dv * (fr * u2 + pp * m2);
      s4 += dv * (fr * H);
    }
    if (d == 0) {
      accC[0] = s0, accC[1] = s1, accC[2] = s2, accC[3] = s3, accC[4] = s4;
    } else {
      accC[0] += s0, accC[1] += s1, accC[2] += s2, accC[3] += s3, accC[4] += s4;
    }
  }
  // ---- viscous volume term: collocated weak form, per direction ----
  if (a.viscous) {
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      {
        const float4 jj = J4[d * Pn + vp];
        const float nv[3] = {2.0f * jj.x, 2.0f * jj.y, 2.0f * jj.z};
        float fv[4];
        viscous_flux_n(tau, W, nv, fv);
        G4[t] = make_float4(fv[0], fv[1], fv[2], fv[3]);
      }
      __syncwarp();
      __syncthreads();
      {
        const int id = dir_index<n>(t, d), sd = dir_stride<n>(d), bse = t - id * sd;
#pragma unroll
        for (int al = 0; al < n; ++al) {
          const float c = sDh[id * n + al];
          const float4 gv = G4[bse + al * sd];
          acc[1] -= c * gv.x;
          acc[2] -= c * gv.y;
          acc[3] -= c * gv.z;
          acc[4] -= c * gv.w;
        }
      }
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
      double* X1 = reinterpret_cast<double*>(Wk);  // the workspace is free here
      al = element_alpha<n>(U[0] * p_full, X1, X1 + n3, X1 + 2 * n3, sVi, t, a.alpha_min, a.alpha_max);
    }
    if (valid && t == 0) a.alpha[e] = al;
    if (__syncthreads_or(al > 0)) {
      float vfv[5] = {0, 0, 0, 0, 0};
      float* G = Wk;
      const double* FVm = a.fvmetric + (size_t)e * 3 * (n - 1) * 3 * n2;
#pragma unroll 1
      for (int d = 0; d < 3; ++d) {
        const int id = dir_index<n>(t, d), sd = dir_stride<n>(d);
        const bool right = id < n - 1;
        const int line = d == 0 ? idx[1] + n * idx[2] : (d == 1 ? idx[0] + n * idx[2] : idx[0] + n * idx[1]);
        const double* fm = FVm + (size_t)(d * (n - 1) + (right ? id : n - 2)) * 3 * n2 + line;
        const double mv[3] = {fm[0], fm[n2], fm[2 * n2]};
        const double sAd = sqrt(mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2]);
        const float nu[3] = {float(mv[0] / sAd), float(mv[1] / sAd), float(mv[2] / sAd)};
        const int nb = right ? t + sd : t;
        double UR[5];
        const double* ur = a.U + (size_t)e * 5 * n3 + nb;
#pragma unroll
        for (int k = 0; k < 5; ++k) UR[k] = ur[k * n3];
        const SPrim<float> qR = shifted_prim<float>(UR, a.gm1, a.Rinv, cp);
        float fb[5];
        lf_flux_s(me, qR, nu, a.f_gamma, cp.fpr, fb);
        if (right) {
#pragma unroll
          for (int k = 0; k < 5; ++k) G[k * n3 + t] = fb[k] * float(sAd);
        }
        __syncwarp();
        __syncthreads();
        if (right) {
#pragma unroll
          for (int k = 0; k < 5; ++k) vfv[k] += G[k * n3 + t] / float(a.ops->w[id]);
        }
        if (id > 0) {
          const int nl = t - sd;
#pragma unroll
          for (int k = 0; k < 5; ++k) vfv[k] -= G[k * n3 + nl] / float(a.ops->w[id]);
        }
        __syncwarp();
        __syncthreads();
      }
      if (al > 0) {
        const float alt = float(al);
#pragma unroll
        for (int k = 0; k < 5; ++k) accC[k] = (1 - alt) * accC[k] + alt * vfv[k];
      }
    }
  }
  // ---- SurfInt: face nodes receive +-f* lhat ----
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id = idx[d];
    if (id != 0 && id != n - 1) continue;
    const int f = 2 * d + (id == n - 1 ? 1 : 0);
    int p, qq;
    face_pq(d, idx, p, qq);
    const int es = a.elem_side[(size_t)e * 6 + f];
    int pm = p, qm = qq;
    if (es_slave(es)) flip_to_master<n>(es_flip(es), p, qq, pm, qm);
    if (!DG_CHK(es_side(es) >= 0 && es_side(es) < a.S && pm >= 0 && pm < n && qm >= 0 && qm < n, es_side(es)))
      continue;
    const float sg = sSn[f * n2 + p + n * qq].w;
    const float* Fs = a.fstar32 + (size_t)es_side(es) * 5 * n2 + pm + n * qm;
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += sg * Fs[k * n2];
  }
  // ---- ApplyJac; the energy equation gets H_ref times the mass equation back ----
  float ut32[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) ut32[k] = -(accC[k] + acc[k]) * Jinv;
  // the FP64 tendency: for dg_rhs, and in a stage with sources
  const bool sources = a.sponge_sigma || a.source;
  double Ut[5];
  if (MODE == 0 || sources) {
#pragma unroll
    for (int k = 0; k < 5; ++k) Ut[k] = f64_of(ut32[k]);
    Ut[4] += cp.Hr * Ut[0];
    if (a.sponge_sigma) {  // sponge source -sigma (U - U_base), FP64
      const double sg = a.sponge_sigma[(size_t)e * n3 + t];
      const double* ub = a.sponge_base + (size_t)e * 5 * n3 + t;
#pragma unroll
      for (int k = 0; k < 5; ++k) Ut[k] -= sg * (U[k] - ub[k * n3]);
    }
    if (a.source) {  // manufactured-solution source, FP64
      double Q[5];
      const double ts = MODE == 0 ? a.scal->t : a.scal->t - (1.0 - sc.C) * a.scal->dt;
      mms_source(a, a.xyzs + ((size_t)e * n3 + t) * 3, ts, Q);
#pragma unroll
      for (int k = 0; k < 5; ++k) Ut[k] += Q[k];
    }
  }
  if constexpr (MODE == 0) {
    if (valid) {
      double* o = a.Ut + (size_t)e * 5 * n3 + t;
#pragma unroll
      for (int k = 0; k < 5; ++k) o[k * n3] = Ut[k];
    }
  } else {
    // RK update.  This stage form keeps the RK register in FP32 (the state
    // stays FP64): dU = A dU + dt Ut in FP32, U += B dU in FP64.  The
    // register is O(dt |Ut|) and rounds at the level of the FP32 fluxes
    // already in Ut; the energy tendency's H_ref part is added in FP32, its
    // rounding far below the FP32 error that Ut_rho already carries times H_ref.
    float utf[5];
    if (sources) {
#pragma unroll
      for (int k = 0; k < 5; ++k) utf[k] = f32_rn(Ut[k]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) utf[k] = ut32[k];
      utf[4] = ut32[4] + cp.fHr * ut32[0];
    }
    const float dtf = f32_rn(case_dt(a, ce));
    float* du = reinterpret_cast<float*>(a.dU) + (size_t)e * 5 * n3 + t;
    double* uo = a.Urk + (size_t)e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float r = sc.first ? dtf * utf[k] : fmaf(sc.fA, du[k * n3], dtf * utf[k]);
      U[k] += sc.B * f64_of(r);  // the updated state
      if (valid) {
        du[k * n3] = r;
        uo[k * n3] = U[k];
      }
    }
    if (a.epilogue) {
      // ---- the face data of the updated state for the next stage ----
      const SPrim<float> mn = shifted_prim<float, true>(U, a.gm1, a.Rinv, cp);
      __syncwarp();
      __syncthreads();  // the workspace is read by no thread any more
      face_epilogue<N>(a, cp, e, t, valid, mn, Jinv, J4, Qs, Wk, sDr, sSn);
    }
  }
}

template <int N, int MODE, int EPB_ = 0>
__global__ void __launch_bounds__(Shape<N, EPB_>::THREADS, Shape<N, EPB_>::template vol_min_blocks<float>())
    k_felem(StageArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const StageCoef sc{a.rkA, a.rkB, a.rkC, a.f_rkA, a.first_stage};
  felem_body<N, MODE, EPB_>(a, sc, blockIdx.x, smraw);
}

// ---------------------------------------------------------------------------
// Persistent form: one launch runs every stage of a step.  Each stage is a
// side phase (FillFlux over all side nodes, grid-stride) and an element phase
// (the element blocks, grid-stride), separated by grid-wide barriers.  The
// grid is at most the number of blocks the GPU holds at once (a cooperative
// launch), and every barrier wait gives up after a bounded spin: it then sets
// the context's timeout flag and every block leaves, so a missing
// participant ends the launch with an error the host reads
// (DG_ERR_TIMEOUT) instead of a hang.
// ---------------------------------------------------------------------------
struct PersistArgs {
  int ns;                           // stages
  double A[32], B[32], C[32];       // the low-storage scheme
  unsigned* bar;                    // [2]: arrivals, generation (zero at launch)
  int* timeout;                     // sticky flag
  unsigned expect_extra;            // arrivals beyond the grid the barriers wait for (0; a test raises it)
  unsigned spin_limit;              // polls of 200 ns before a barrier wait gives up
  int nblk;                         // element blocks of the element phase
};

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned expected, int* flag, unsigned limit) {
  __shared__ int ok;
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    volatile int* vflag = flag;
    const unsigned g = *gen;
    __threadfence();
    int good = 1;
    if (atomicAdd(bar, 1u) + 1u == expected) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned it = 0;
      while (*gen == g) {
        if (*vflag || ++it > limit) {
          atomicExch(flag, 1);
          good = 0;
          break;
        }
        __nanosleep(200);
      }
    }
    __threadfence();
    ok = good && !*vflag;
  }
  __syncwarp();
  __syncthreads();
  return ok != 0;
}

template <int N>
__global__ void __launch_bounds__(Shape<N>::THREADS, Shape<N>::template vol_min_blocks<float>())
    k_fpersist(StageArgs a, PersistArgs p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const unsigned expected = gridDim.x + p.expect_extra;
  const int64_t side_work = (int64_t)a.S * Shape<N>::n2;
  for (int st = 0; st < p.ns; ++st) {
    for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < side_work;
         tid += (int64_t)gridDim.x * blockDim.x)
      fflux_body<N>(a, tid);
    if (!grid_barrier(p.bar, expected, p.timeout, p.spin_limit)) return;
    const StageCoef sc{p.A[st], p.B[st], p.C[st], (float)p.A[st], st == 0};
    for (unsigned blk = blockIdx.x; blk < (unsigned)p.nblk; blk += gridDim.x) {
      felem_body<N, 1, 0>(a, sc, blk, smraw);
      __syncwarp();
      __syncthreads();  // the next element reuses the shared memory
    }
    if (st + 1 < p.ns && !grid_barrier(p.bar, expected, p.timeout, p.spin_limit)) return;
  }
}

}  // namespace dg
