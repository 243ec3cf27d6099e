// The work of one element block of the two-kernel FP32-bulk stage: one stage
// of elements blk * EPB ... of the element list (FP32-bulk arithmetic, FP64
// state).  MODE 0 writes Ut (and, viscous, the lifted gradients); MODE 1 does
// the RK update, then (a.epilogue) forms the face data of the updated state.
// a.prefetch > 0: each block first asks L2 for the state, RK register and
// metrics of the element a.prefetch blocks further on (the next wave on the
// GPU), so that wave's loads find them in L2.
//
// This file is included inside the body of each kernel that runs this work
// (k_felem, k_fpersist), with in scope: the template parameters N, MODE and
// EPB_, the kernel's StageArgs parameter `a`, the element block `blk`, the
// stage coefficients `sc` (A(), B(), C(), fA(), first()) and the dynamic
// shared memory `smraw`.  It is text, not a function: behind a function that
// takes the StageArgs by reference, the compiler holds the parameter fields
// it needs in registers instead of reading them from the parameter bank where
// they are used, and k_felem<7, 1> spilled 112 bytes where it spills 64.  A
// block all of whose slots are idle leaves through the `break` of the
// enclosing do-while.
do {
    using S = Shape<N, EPB_>;
    using L = FusedSmem<N, EPB_>;
    constexpr int n = S::n, n2 = S::n2, n3 = S::n3, EPB = S::EPB;
    double* sVi = reinterpret_cast<double*>(smraw);  // [n2] Vinv (FP64)
    float* sDs = reinterpret_cast<float*>(sVi + L::n2d);
    float* sDh = sDs + L::n2p;
    float* sDr = sDh + L::n2p;  // [n][n4] 2 Dhat, rows padded (lift_volume)
    float* base = sDr + n * L::n4;
    const int le = threadIdx.x / n3, t = threadIdx.x % n3;
    float* mine = base + (size_t)le * L::per_elem_f;
    float4* P4 = reinterpret_cast<float4*>(mine);                   // [Pn] (rho, u, v, w) / 2, padded index
    float4* Q4 = P4 + L::Pn;                                        // [Pn] (p' / 2, H' / 2, T', 0), padded index
    float4* J4 = reinterpret_cast<float4*>(mine + L::offJ);         // [3][Pn] (Ja^d) / 2, padded index
    float* Qs = mine + L::offQ;                                     // [4][Pn] u, v, w, T', padded index
    float* Wk = mine + L::offW;                                     // [12][Pn] workspace
    float4* G4 = reinterpret_cast<float4*>(Wk);                     // [Pn] viscous fluxes, padded index
    float4* sSn = reinterpret_cast<float4*>(mine + L::offN);        // [6][n2] face normals and signs
    float4* sQst = reinterpret_cast<float4*>(mine + L::offQS);      // [6][n2] q* of the six sides
    float* sFst = mine + L::offFS;                                  // [5][6 n2] f* of the six sides
    float* sDU = mine + L::offDU;                                   // [5][n3] the RK register
    constexpr int Pn = L::Pn;
    // slots past the last element redo the last element, free slots of a
    // serving pool compute on what they hold; neither stores
    const int ei = (int)blk * EPB + le < a.E ? (int)blk * EPB + le : a.E - 1;
    const int el = a.elem_list ? a.elem_list[ei] : ei;
    const int ce = a.elem_case ? a.elem_case[el] : 0;
    // elements of cases that finished or sit this step out (time step 0) keep
    // their state and face data; a block made only of such slots leaves at once
    const bool valid = (int)blk * EPB + le < a.E && ce >= 0 && !(a.cases && a.cases[ce].dt == 0.0);
    if (a.elem_case && __syncthreads_and(!valid)) break;
    const int e = DG_CHK(el >= 0 && t < n3 && le < EPB, el) ? el : 0;
    const CaseParams cp = case_params(a, ce);
    if (a.prefetch > 0 && threadIdx.x == 0) {
      // the elements of the block a.prefetch blocks further on, when they are
      // one contiguous range (always without an element list; in a serving
      // pool, unless the block spans two cases' ranges)
      const int64_t i2 = (int64_t)(blk + a.prefetch) * EPB;
      if (i2 < a.E) {
        const int64_t ne = min((int64_t)EPB, (int64_t)a.E - i2);
        const int64_t e2 = a.elem_list ? a.elem_list[i2] : i2;
        if (!a.elem_list || a.elem_list[i2 + ne - 1] == e2 + ne - 1) {
          const size_t ub = sizeof(double) * 5 * n3, Ea = (size_t)a.E_all;
          prefetch_l2(a.U + e2 * 5 * n3, ub * ne, a.U, a.U + Ea * 5 * n3);
          if (MODE == 1 && !sc.first()) {
            const float* d32 = reinterpret_cast<const float*>(a.dU);
            prefetch_l2(d32 + e2 * 5 * n3, sizeof(float) * 5 * n3 * ne, d32, d32 + Ea * 5 * n3);
          }
          prefetch_l2(a.metric32 + e2 * 10 * n3, sizeof(float) * 10 * n3 * ne, a.metric32, a.metric32 + Ea * 10 * n3);
          if (a.viscous)
            prefetch_l2(a.wv32 + e2 * 12 * n3, sizeof(float) * 12 * n3 * ne, a.wv32, a.wv32 + Ea * 12 * n3);
        }
      }
    }
    for (int k = threadIdx.x; k < n2; k += blockDim.x) {
      sDs[k] = (float)a.ops->Dsplit[k];
      sDh[k] = (float)a.ops->Dhat[k];
      sVi[k] = a.ops->Vinv[k];
    }
    for (int k = threadIdx.x; k < n * L::n4; k += blockDim.x) {
      const int i = k / L::n4, al = k % L::n4;
      sDr[k] = al < n ? 2.0f * (float)a.ops->Dhat[i * n + al] : 0.0f;
    }
    // the element's state and metrics first, then its face data (normals;
    // q*, f* and the RK register by asynchronous copies), so that the side
    // map's round trip overlaps those loads and nothing later in the element
    // waits on global memory
    double U[5];
    double p_full;
    {
      const double* u = a.U + (size_t)e * 5 * n3 + t;
  #pragma unroll
      for (int k = 0; k < 5; ++k) U[k] = u[k * n3];
    }
    float mt[10];
  #pragma unroll
    for (int c = 0; c < 10; ++c) mt[c] = metric_at<float>(a, e, c, t, n3);
    load_face_data<n>(a, e, t, sSn, sQst, sFst, a.viscous != 0);
    if (a.viscous) {  // the lifting's volume sums of this state, formed by the face-data pass
      const float* ws = a.wv32 + (size_t)e * 12 * n3 + t;
  #pragma unroll
      for (int k = 0; k < 12; ++k) cp_async4(Wk + k * Pn + pad_idx<n>(t), ws + k * n3);
    }
    if (MODE == 1 && !sc.first()) {
      const float* d32 = reinterpret_cast<const float*>(a.dU) + (size_t)e * 5 * n3 + t;
  #pragma unroll
      for (int k = 0; k < 5; ++k) cp_async4(sDU + k * n3 + t, d32 + k * n3);
    }
    cp_async_commit();
    // the FP64 pressure only for the indicator (one FP64 addition less otherwise)
    const SPrim<float> me = shifted_prim<float, true>(U, a.gm1, a.Rinv, cp, a.shock ? &p_full : nullptr);
    // halved values: every arithmetic mean of the two-point flux is one addition
    const int vp = pad_idx<n>(t);
    P4[vp] = make_float4(0.5f * me.rho, 0.5f * me.u, 0.5f * me.v, 0.5f * me.w);
    Q4[vp] = make_float4(0.5f * me.p, 0.5f * me.H, me.Tt, 0.0f);
  #pragma unroll
    for (int d = 0; d < 3; ++d)
      J4[d * Pn + vp] = make_float4(0.5f * mt[3 * d], 0.5f * mt[3 * d + 1], 0.5f * mt[3 * d + 2], 0.0f);
    const float Jinv = mt[9];
    cp_async_wait<0>();  // this thread's copies; the barrier makes every thread's visible
    __syncwarp();
    __syncthreads();
    const int idx[3] = {t % n, (t / n) % n, t / n2};  // indexed by unrolled (constant) d only
    float tau[6] = {0, 0, 0, 0, 0, 0}, W[3] = {0, 0, 0};
    // ---- BR1 lifting of the stage's state: volume part (read), then q* of the six faces ----
    if (a.viscous) {
      float g[12];
  #pragma unroll
      for (int k = 0; k < 12; ++k) g[k] = Wk[k * Pn + vp];  // this thread's own copies (waited for above)
  #pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int id = idx[d];
        if (id != 0 && id != n - 1) continue;
        const int f = 2 * d + (id == n - 1 ? 1 : 0);
        int p, qq;
        face_pq(d, idx, p, qq);
        const float4 qs = sQst[f * n2 + p + n * qq];
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
      if (MODE == 0 && valid) {
        // dg_rhs: the lifted gradients for the verification copy (DG_DEBUG_GRAD)
        float* go = a.g32 + (size_t)e * 12 * n3 + t;
  #pragma unroll
        for (int k = 0; k < 12; ++k) go[k * n3] = g[k];
      }
      float vmu, vlam;
      visc_coeffs<float>(a, cp, me.Tt, vmu, vlam);
      viscous_parts(g, me.u, me.v, me.w, vmu, vlam, tau, W);
    }
    // ---- split-form KEP volume integral, one node per thread over its partners ----
    float accC[5] = {0, 0, 0, 0, 0};  // convective DG volume term
    float acc[5] = {0, 0, 0, 0, 0};   // viscous volume + surface terms
    // unrolled over the directions: each partner's shared-memory offsets,
    // padding included, are then compile-time constants
  #pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int id = dir_index<n>(t, d), sd = dir_stride<n>(d), bse = t - id * sd;
      const float4 ai = P4[vp];
      const float4 bi = Q4[vp];
      const float4 ji = J4[d * Pn + vp];
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
  #pragma unroll
      for (int al = 0; al < n; ++al) {
        if (al == id) continue;
        const int va = bse + al * sd;
        if (!DG_CHK(va >= 0 && va < n3, va)) continue;
        const int pva = pad_idx<n>(va);
        const float4 aa = P4[pva];
        const float4 ba = Q4[pva];
        const float4 ja = J4[d * Pn + pva];
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
      // its flux planes overlay the W planes whose sums every thread has read
      __syncwarp();
      __syncthreads();
  #pragma unroll 1
      for (int d = 0; d < 3; ++d) {
        {
          const float4 jj = J4[d * Pn + vp];
          const float nv[3] = {2.0f * jj.x, 2.0f * jj.y, 2.0f * jj.z};
          float fv[4];
          viscous_flux_n(tau, W, nv, fv);
          G4[vp] = make_float4(fv[0], fv[1], fv[2], fv[3]);
        }
        __syncwarp();
        __syncthreads();
        {
          const int id = dir_index<n>(t, d), sd = dir_stride<n>(d), bse = t - id * sd;
  #pragma unroll
          for (int al = 0; al < n; ++al) {
            const float c = sDh[id * n + al];
            const float4 gv = G4[pad_idx<n>(bse + al * sd)];
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
      const int slot = f * n2 + p + n * qq;
      const float sg = sSn[slot].w;
  #pragma unroll
      for (int k = 0; k < 5; ++k) acc[k] += sg * sFst[k * 6 * n2 + slot];
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
        const double ts = MODE == 0 ? a.scal->t : a.scal->t - (1.0 - sc.C()) * a.scal->dt;
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
        const float r = sc.first() ? dtf * utf[k] : fmaf(sc.fA(), sDU[k * n3 + t], dtf * utf[k]);
        U[k] += sc.B() * f64_of(r);  // the updated state
        if (valid) {
          du[k * n3] = r;
          uo[k * n3] = U[k];
        }
      }
      if (a.epilogue) {
        // ---- the face data of the updated state for the next stage ----
        const SPrim<float> mn = shifted_prim<float, true>(U, a.gm1, a.Rinv, cp);
        // the last stage of a step: the CFL radii of the updated state, for
        // the next step's time step (element 0's q* records hold the warps'
        // maxima: every thread read its q* in the lifting)
        float* red = base + L::offQS;
        if (a.cfl_out) cfl_block_radii<n>(a, valid, U, J4, vp, Jinv, red);
        __syncwarp();
        __syncthreads();  // the workspace is read by no thread any more
        face_epilogue<N>(a, cp, e, t, valid, mn, Jinv, J4, Qs, P4, Wk, sDr, sSn);  // P4, Q4 are free after the KEP sums
        if (a.cfl_out && threadIdx.x == 0) cfl_block_finish(a, red, (int)(blockDim.x >> 5));
      }
    }
} while (0);
