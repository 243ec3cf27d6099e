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
// and per element, at every node:
//   wv32  [E][12][n3] floats: the volume part of the lifting,
//         sum_d Dhat (Ja^d q), before 1/J.  The epilogue forms it for the
//         updated state anyway (for g_part); the next stage's element kernel
//         reads it instead of forming the same sums again.
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
  // per element: P (2 float4 planes, padded index: (rho, u, v, w) / 2 and
  // (p', H') / 2, T'; padded like every plane the line sums read, so that the
  // four lines of eight nodes a warp holds along the first direction fall in
  // distinct banks), J (3 float4 planes, (Ja^d) / 2), q (4 planes: u, v, w, T'), W (12 planes:
  // lifting sums; also viscous / FV fluxes and the FP64 indicator scratch),
  // face normals (6 faces x n2 float4: s n and the SurfInt sign), and the
  // element's gathered face and RK data: q* of its six sides (6 x n2 float4),
  // their f* (5 planes of 6 n2) and its FP32 RK register (5 planes of n3)
  static constexpr int offJ = 8 * Pn, offQ = offJ + 12 * Pn, offW = offQ + 4 * Pn, offN = offW + 12 * Pn;
  static constexpr int offQS = offN + 24 * S::n2, offFS = offQS + 24 * S::n2;
  static constexpr int offDU = (offFS + 30 * S::n2 + 3) & ~3;  // (rounded to whole float4s)
  static constexpr int per_elem_f = (offDU + 5 * S::n3 + 3) & ~3;
  static constexpr size_t bytes =
      sizeof(double) * n2d + sizeof(float) * (2 * n2p + S::n * n4 + S::EPB * per_elem_f);
  static_assert(2 * S::n3 + 4 * S::n2 <= 6 * Pn, "the indicator scratch fits the W workspace");
  static_assert(Pn <= 2 * S::n3, "a padded float4 node plane fits the P planes (the epilogue's R4)");
  static_assert((2 * n2p + S::n * n4) % 4 == 0 && per_elem_f % 4 == 0 && offQ % 4 == 0 && offW % 4 == 0 &&
                    offN % 4 == 0 && offQS % 4 == 0 && offFS % 4 == 0 && offDU % 4 == 0,
                "16-byte alignment of the float4 planes");
  static_assert(EPB_ != 0 || bytes <= 113 * 1024, "two blocks per SM at the default elements per block");
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
// halved metrics; W: its 12 workspace planes; sDr2: 2 Dhat with rows padded
// to n4 floats (the factor 2 undoes the halving of the metrics, exactly:
// (2 Dhat) (J/2 q) rounds as Dhat (J q)).  READ: node t's twelve sums are
// read back into acc (else they stay in W only).  Every thread of the block
// calls it (it holds barriers); W may be reused after the caller's next
// barrier.
// ---------------------------------------------------------------------------
template <int n, int n4, bool READ = true>
__device__ __forceinline__ void lift_volume(const float* Qs, const float4* J4, float* W, const float* sDr2, int t,
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
        P0[al] = j.x * q;
        P1[al] = j.y * q;
        P2[al] = j.z * q;
      }
#pragma unroll
      for (int i = 0; i < n; ++i) {
        float r[n4];
#pragma unroll
        for (int c = 0; c < n4; c += 4) {
          const float4 v4 = *reinterpret_cast<const float4*>(sDr2 + i * n4 + c);
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
  if constexpr (READ) {
    const int v = pad_idx<n>(t);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = W[k * Pn + v];
  }
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

// The element's face data for a stage: the side normals as load_face_normals
// stores them, and, by asynchronous copies (cp.async, one group with the
// caller's), for each face f and face-frame node pq: the side's q* record
// (sQs[f n2 + pq], when `lift`) and its f* (sFs[k][f n2 + pq]).  The copies
// are issued as soon as the side record is known, so that their latency
// overlaps the loads of the element's state and metrics; the caller commits
// the group and waits before its block-wide barrier.
template <int n>
__device__ __forceinline__ void load_face_data(const StageArgs& a, int e, int t, float4* sSn, float4* sQs,
                                               float* sFs, bool lift) {
  constexpr int n2 = n * n;
  const float w0 = (float)a.ops->winv[0];
  for (int k = t; k < 6 * n2; k += n2 * n) {
    const int f = k / n2, pq = k % n2;
    int s, half, pm;
    face_record<n>(a.elem_side, e, f, pq % n, pq / n, s, half, pm);
    if (!DG_CHK(s >= 0 && s < a.S && pm >= 0 && pm < n2, s)) continue;
    if (lift) cp_async16(sQs + k, a.qs32 + ((size_t)s * n2 + pm) * 4);
    const float* fs = a.fstar32 + (size_t)s * 5 * n2 + pm;
#pragma unroll
    for (int c = 0; c < 5; ++c) cp_async4(sFs + c * 6 * n2 + k, fs + c * n2);
    const float* nr = a.nrm32 + (size_t)s * 7 * n2 + pm;
    sSn[k] = make_float4(nr[0], nr[n2], nr[2 * n2], half ? -w0 : w0);
  }
}

// ---------------------------------------------------------------------------
// Epilogue: the face data of a state for the next k_fflux.  me: the node's
// shifted primitives; Jinv its 1/J; sSn the element's face normals; R4 a
// free float4 plane of the element (n3 + n2 entries, padded node index).  All threads of the block
// call it (the lifting holds barriers); `valid` masks the stores.
// The node values go to shared memory (q in the Qs planes, (rho, p', H', 1/J)
// in R4), the lifting leaves its volume sums in the W planes, and
// then one thread per (face, face node) slot forms that record: the node's
// own halves of q* on every face through it, g_part, the viscous parts and
// the partial viscous flux through the slot's face (edge and corner nodes
// form g_part once per face they lie on, in the same order of operations).
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void face_epilogue(const StageArgs& a, const CaseParams& cp, int e, int t, bool valid,
                                              const SPrim<float>& me, float Jinv, const float4* J4, float* Qs,
                                              float4* R4, float* Wk, const float* sDr, const float4* sSn) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  constexpr int Pn = n3 + n2, n4 = (n + 3) & ~3;
  {
    const int v = pad_idx<n>(t);
    Qs[v] = me.u, Qs[Pn + v] = me.v, Qs[2 * Pn + v] = me.w, Qs[3 * Pn + v] = me.Tt;
    R4[v] = make_float4(me.rho, me.p, me.H, Jinv);  // padded: face slots read it with a node stride of n
  }
  __syncwarp();
  __syncthreads();
  if (a.viscous) {  // block-uniform condition
    // the volume sums at every node, left in the W planes: computing only the
    // face nodes' sums saves no time (a warp's lines mix both kinds, and
    // warp-uniform task orders for them meet shared-memory bank conflicts)
    float unused[12];
    lift_volume<n, n4, false>(Qs, J4, Wk, sDr, t, unused);
    // the node's twelve sums for the next stage's lifting, which would form
    // them again from the same state and metrics
    if (valid) {
      const int v = pad_idx<n>(t);
      float* ws = a.wv32 + (size_t)e * 12 * n3 + t;
#pragma unroll
      for (int k = 0; k < 12; ++k) ws[k * n3] = Wk[k * Pn + v];
    }
  }
  if (!valid) return;
  for (int slot = t; slot < 6 * n2; slot += n3) {
    const int f = slot / n2, pq = slot % n2, p = pq % n, qq = pq / n, df = f >> 1;
    const int side = (f & 1) ? n - 1 : 0;
    // the node of the slot: face-frame (p, q) is (j, k) on x-faces, (i, k) on
    // y-faces, (i, j) on z-faces
    const int i0 = df == 0 ? side : p, i1 = df == 0 ? p : (df == 1 ? side : qq), i2 = df == 2 ? side : qq;
    const int idx[3] = {i0, i1, i2};  // indexed by unrolled (constant) d only
    const int node = i0 + n * (i1 + n * i2), vn = pad_idx<n>(node);
    if (!DG_CHK(node >= 0 && node < n3, node)) continue;
    const float q[4] = {Qs[vn], Qs[Pn + vn], Qs[2 * Pn + vn], Qs[3 * Pn + vn]};
    float tau[6], W[3];
    if (a.viscous) {
      float acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = Wk[k * Pn + vn];
      // own halves of q* on every face through the node
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (idx[d] != 0 && idx[d] != n - 1) continue;
        const int fd = 2 * d + (idx[d] == n - 1 ? 1 : 0);
        int pd, qd;
        face_pq(d, idx, pd, qd);
        const float4 sn = sSn[fd * n2 + pd + n * qd];
#pragma unroll
        for (int qv = 0; qv < 4; ++qv) {
          const float h = sn.w * (0.5f * q[qv]);
          acc[qv * 3 + 0] += h * sn.x;
          acc[qv * 3 + 1] += h * sn.y;
          acc[qv * 3 + 2] += h * sn.z;
        }
      }
      const float Jn = R4[vn].w;
      float g[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) g[k] = acc[k] * Jn;
      float vmu, vlam;
      visc_coeffs<float>(a, cp, q[3], vmu, vlam);
      viscous_parts(g, q[0], q[1], q[2], vmu, vlam, tau, W);
    }
    int sd, hd, pqd;
    face_record<n>(a.elem_side, e, f, p, qq, sd, hd, pqd);
    const size_t rec = ((size_t)sd * 2 + hd) * n2 + pqd;
    if (!DG_CHK(sd >= 0 && sd < a.S && pqd >= 0 && pqd < n2 && (hd == 0 || hd == 1), rec)) continue;
    st4(a.tr32 + rec * 8, make_float4(q[0], q[1], q[2], q[3]));
    st4(a.tr32 + rec * 8 + 4, R4[vn]);
    if (a.viscous) {
      const float4 sn = sSn[slot];
      const float snv[3] = {sn.x, sn.y, sn.z};
      float fv[4];
      viscous_flux_n(tau, W, snv, fv);
      st4(a.pfv32 + rec * 4, make_float4(fv[0], fv[1], fv[2], fv[3]));
    }
  }
}

// The CFL spectral radii of the state an element block prepares, for the
// next step's time step (two-kernel FP32-bulk steps; the CFL reduction
// kernel then does not read the state again).  Each thread forms its node's
// radii with cfl_radii from the same FP32 values k_cfl<N, float> uses (the
// state rounded to FP32 and the FP32 metrics, which J4 holds halved), so the
// radii are bitwise k_cfl's and need no load beyond the element's own; the
// lanes of a warp take their maxima, and lane 0 leaves them in red[2 w]
// (convective), red[2 w + 1] (viscous) and red[64 + w] (1: a non-finite
// radius) for warp w.  Every thread of the block calls it; after the
// block's next barrier thread 0 calls cfl_block_finish.
template <int n>
__device__ __forceinline__ void cfl_block_radii(const StageArgs& a, bool valid, const double U[5], const float4* J4,
                                                int vp, float Jinv, float* red) {
  constexpr int n3 = n * n * n, Pn = n3 + n * n;
  float Uv[5], M[10];
#pragma unroll
  for (int k = 0; k < 5; ++k) Uv[k] = f32_rn(U[k]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float4 j = J4[d * Pn + vp];
    M[3 * d] = 2.0f * j.x, M[3 * d + 1] = 2.0f * j.y, M[3 * d + 2] = 2.0f * j.z;
  }
  M[9] = Jinv;
  float aa, bb;
  cfl_radii(Uv, M, a.f_gamma, a.f_gm1, a.f_Rinv, a.f_cflkv, a.sutherland, a.f_inv_Tref, aa, bb);
  const bool bad = valid && !(isfinite(aa) && isfinite(bb));
  if (!valid) aa = bb = 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    aa = fmaxf(aa, __shfl_xor_sync(0xffffffffu, aa, o));
    bb = fmaxf(bb, __shfl_xor_sync(0xffffffffu, bb, o));
  }
  const bool wbad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    const int w = threadIdx.x >> 5;
    red[2 * w] = aa;
    red[2 * w + 1] = bb;
    red[64 + w] = wbad ? 1.0f : 0.0f;
  }
}
// thread 0: the block's maxima into the step scalars (as k_cfl adds its blocks')
__device__ __forceinline__ void cfl_block_finish(const StageArgs& a, const float* red, int nwarps) {
  float lc = 0.0f, lv = 0.0f;
  bool bad = false;
  for (int w = 0; w < nwarps; ++w) {
    lc = fmaxf(lc, red[2 * w]);
    lv = fmaxf(lv, red[2 * w + 1]);
    bad = bad || red[64 + w] != 0.0f;
  }
  atomicMax(&a.scal_cfl->lam_c_next, (unsigned long long)__double_as_longlong(f64_of(lc)));
  if (a.viscous) atomicMax(&a.scal_cfl->lam_v_next, (unsigned long long)__double_as_longlong(f64_of(lv)));
  if (bad) atomicOr(&a.scal_cfl->nonfinite, 1);
}

// ---------------------------------------------------------------------------
// k_fprep: face data of the state a.U
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Shape<N>::THREADS) k_fprep(StageArgs a) {
  using S = Shape<N>;
  using L = FusedSmem<N>;
  constexpr int n = S::n, n3 = S::n3, EPB = S::EPB;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* sDs = reinterpret_cast<float*>(reinterpret_cast<double*>(smraw) + L::n2d);
  float* sDh = sDs + L::n2p;
  float* sDr = sDh + L::n2p;  // [n][n4] 2 Dhat, rows padded (lift_volume)
  float* base = sDr + n * L::n4;
  const int le = threadIdx.x / n3, t = threadIdx.x % n3;
  float* mine = base + (size_t)le * L::per_elem_f;
  float4* R4 = reinterpret_cast<float4*>(mine);  // the P planes, free here
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
    sDr[k] = al < n ? 2.0f * (float)a.ops->Dhat[i * n + al] : 0.0f;
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
  float* red = base + L::offQS;  // element 0's q* records (unused here)
  if (a.cfl_out) cfl_block_radii<n>(a, valid, U, J4, vp, Jinv, red);
  __syncwarp();
  __syncthreads();
  face_epilogue<N>(a, cp, e, t, valid, me, Jinv, J4, Qs, R4, Wk, sDr, sSn);
  if (a.cfl_out && threadIdx.x == 0) cfl_block_finish(a, red, (int)(blockDim.x >> 5));
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
// k_felem: one stage of one element block (the work is in dg_felem_body.cuh)
// ---------------------------------------------------------------------------
// the coefficients of one low-storage RK stage, read where they are used
// (dU = A dU + dt Ut, U += B dU; stage time t + C dt; fA: A in FP32; first:
// the first stage, whose A is not used): from the launch arguments of a
// per-stage launch, or from the scheme of a persistent launch
struct CoefOfStage {
  const StageArgs& a;
  __device__ __forceinline__ double A() const { return a.rkA; }
  __device__ __forceinline__ double B() const { return a.rkB; }
  __device__ __forceinline__ double C() const { return a.rkC; }
  __device__ __forceinline__ float fA() const { return a.f_rkA; }
  __device__ __forceinline__ bool first() const { return a.first_stage != 0; }
};

template <int N, int MODE, int EPB_ = 0>
__global__ void __launch_bounds__(Shape<N, EPB_>::THREADS, Shape<N, EPB_>::template vol_min_blocks<float>())
    k_felem(StageArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const unsigned blk = blockIdx.x;
  const CoefOfStage sc{a};
#include "dg_felem_body.cuh"
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
struct PersistArgs;
// the coefficients of stage st of a persistent launch's scheme
struct CoefOfScheme {
  const PersistArgs& p;
  int st;
  __device__ __forceinline__ double A() const;
  __device__ __forceinline__ double B() const;
  __device__ __forceinline__ double C() const;
  __device__ __forceinline__ float fA() const { return (float)A(); }
  __device__ __forceinline__ bool first() const { return st == 0; }
};

struct PersistArgs {
  int ns;                           // stages
  double A[32], B[32], C[32];       // the low-storage scheme
  unsigned* bar;                    // [2]: arrivals, generation (zero at launch)
  int* timeout;                     // sticky flag
  unsigned expect_extra;            // arrivals beyond the grid the barriers wait for (0; a test raises it)
  unsigned spin_limit;              // polls of 200 ns before a barrier wait gives up
  int nblk;                         // element blocks of the element phase
};

__device__ __forceinline__ double CoefOfScheme::A() const { return p.A[st]; }
__device__ __forceinline__ double CoefOfScheme::B() const { return p.B[st]; }
__device__ __forceinline__ double CoefOfScheme::C() const { return p.C[st]; }

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
    for (unsigned blk = blockIdx.x; blk < (unsigned)p.nblk; blk += gridDim.x) {
      constexpr int MODE = 1, EPB_ = 0;
      const CoefOfScheme sc{p, st};
#include "dg_felem_body.cuh"
      __syncwarp();
      __syncthreads();  // the next element reuses the shared memory
    }
    if (st + 1 < p.ns && !grid_barrier(p.bar, expected, p.timeout, p.spin_limit)) return;
  }
}

}  // namespace dg
