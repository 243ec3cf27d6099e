// dg_rhs.cu -- FP64 instantiation of the stage kernels (dg_stage.cuh), the CFL
// reduction, layout conversion, kinetic-energy reductions and verification
// copies, and the host launchers.
#include <algorithm>
#include <cmath>

#include "dg_stage.cuh"

namespace dg {

// ---------------------------------------------------------------------------
// CFL reduction (the paper gives no rule; see dg_time_step in dg.h)
// ---------------------------------------------------------------------------
// T = float (FP32-bulk): the spectral radii in FP32, from the FP32 metrics alone
template <int N, typename T>
__global__ void __launch_bounds__(256) k_cfl(int E, const double* __restrict__ U, const double* __restrict__ metric,
                                            const float* __restrict__ metric32, const double* __restrict__ geo,
                                            double gamma, double gm1, double Rinv, double kv, int viscous,
                                            int sutherland, double inv_Tref, DevScalars* scal) {
  constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
  constexpr bool f32 = sizeof(T) == sizeof(float);
  T lcT = T(0), lvT = T(0);  // per-thread maxima in the arithmetic type
  int bad = 0;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < (int64_t)E * n3;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = x / n3;
    const int t = (int)(x % n3);
    T Uv[5], M[10];
    const double* up = U + e * 5 * n3 + t;
#pragma unroll
    for (int k = 0; k < 5; ++k) Uv[k] = T(up[k * n3]);
#pragma unroll
    for (int k = 0; k < 10; ++k) M[k] = f32 ? T(metric32[(e * 10 + k) * n3 + t]) : T(metric[(e * 10 + k) * n3 + t]);
    T aa, bb;
    if constexpr (f32) {
      cfl_radii(Uv, M, T(gamma), T(gm1), T(Rinv), T(kv), sutherland, T(inv_Tref), aa, bb);
    } else {
      T G[4];
      const double* Gm = geo + e * 4 * n3 + t;
#pragma unroll
      for (int k = 0; k < 4; ++k) G[k] = Gm[k * n3];
      cfl_radii(Uv, M, G, gamma, gm1, Rinv, kv, sutherland, inv_Tref, aa, bb);
    }
    if (!isfinite(aa) || !isfinite(bb)) bad = 1;
    lcT = fmax(lcT, aa);
    lvT = fmax(lvT, bb);
  }
  double lc = to_f64<T>(lcT), lv = to_f64<T>(lvT);
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

// the integer-pipe conversions, for dg_selftest_convert
__global__ void k_convert_check(const double* __restrict__ in, float* __restrict__ out, double* __restrict__ back,
                                int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float f = f32_rn(in[i]);
  out[i] = f;
  back[i] = f64_of(f);
}

cudaError_t launch_convert_check(const double* in, float* out, double* back, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_convert_check<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, back, n);
  count_launch();
  return cudaGetLastError();
}

// the CFL rule from the reduced spectral radii
__device__ __forceinline__ double cfl_dt(const DevScalars* scal, double cfl, double dfl, int N, int viscous) {
  const double np1 = (double)(N + 1);
  const double lc = __longlong_as_double((long long)scal->lam_c);
  const double lv = __longlong_as_double((long long)scal->lam_v);
  double dt = cfl * 2.0 / (np1 * np1 * lc);
  if (viscous && lv > 0) {
    const double dv = dfl * 4.0 / (np1 * np1 * np1 * np1 * lv);
    if (dv < dt) dt = dv;
  }
  return dt;
}

// reports the CFL time step of the current state without stepping
__global__ void k_dt_report(DevScalars* scal, double cfl, double dfl, int N, int viscous) {
  scal->dt_cfl = cfl_dt(scal, cfl, dfl, N, viscous);
  scal->lam_c = 0ull;
  scal->lam_v = 0ull;
}

// next: the radii come from the previous step's last stage (lam_*_next)
__global__ void k_dt(DevScalars* scal, double cfl, double dfl, int N, int viscous, int next = 0) {
  if (next) {
    scal->lam_c = scal->lam_c_next;
    scal->lam_v = scal->lam_v_next;
    scal->lam_c_next = 0ull;
    scal->lam_v_next = 0ull;
  }
  double dt = scal->dt_fixed > 0 ? scal->dt_fixed : cfl_dt(scal, cfl, dfl, N, viscous);
  double tn = scal->t + dt;
  if (scal->t_end > 0) {
    const double rest = scal->t_end - scal->t;
    if (!(rest > 0)) {
      dt = 0.0;
      tn = scal->t;
    } else if (dt >= rest) {
      dt = rest;
      tn = scal->t_end;
    }
  }
  scal->dt = dt;
  scal->t = tn;
  if (dt > 0) scal->steps += 1;
  scal->lam_c = 0ull;
  scal->lam_v = 0ull;
}

// ---------------------------------------------------------------------------
// layout conversion and reductions
// ---------------------------------------------------------------------------
// layout conversion, one element per block through shared memory, so that
// both the reads and the writes are contiguous (the source may be pinned
// host memory read over the host link)
__global__ void __launch_bounds__(256) k_to_internal(int n3, const double* __restrict__ pub, double* __restrict__ in) {
  extern __shared__ double sbuf[];  // [n3][5]
  const int64_t e = blockIdx.x;
  const double* src = pub + e * 5 * n3;
  double* dst = in + e * 5 * n3;
  for (int i = threadIdx.x; i < 5 * n3; i += blockDim.x) sbuf[i] = src[i];
  __syncthreads();
  for (int i = threadIdx.x; i < 5 * n3; i += blockDim.x) {
    const int v = i / n3, t = i % n3;
    dst[i] = sbuf[t * 5 + v];
  }
}
__global__ void __launch_bounds__(256) k_to_public(int n3, const double* __restrict__ in, double* __restrict__ pub) {
  extern __shared__ double sbuf[];  // [5][n3]
  const int64_t e = blockIdx.x;
  const double* src = in + e * 5 * n3;
  double* dst = pub + e * 5 * n3;
  for (int i = threadIdx.x; i < 5 * n3; i += blockDim.x) sbuf[i] = src[i];
  __syncthreads();
  for (int i = threadIdx.x; i < 5 * n3; i += blockDim.x) {
    const int t = i / 5, v = i % 5;
    dst[i] = sbuf[v * n3 + t];
  }
}

// E_k, its rate and the volume (Sec. 5.2), in a fixed order of summation, so
// that dg_kinetic gives bitwise the same values on every call: a fixed grid
// walks the nodes, each block adds its threads' sums in a fixed tree and
// writes them to part[block][3]; k_kinetic_sum adds the blocks in order
template <int N>
__global__ void __launch_bounds__(256) k_kinetic(int E, const double* __restrict__ U, const double* __restrict__ Ut,
                                                 const double* __restrict__ metric, const Ops* __restrict__ ops,
                                                 double* __restrict__ part) {
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
  // butterfly over the warp: every lane ends with the same sums
  for (int o = 16; o > 0; o >>= 1) {
    vol += __shfl_xor_sync(0xffffffffu, vol, o);
    ek += __shfl_xor_sync(0xffffffffu, ek, o);
    rate += __shfl_xor_sync(0xffffffffu, rate, o);
  }
  __shared__ double red[3][8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = ek;
    red[1][w] = rate;
    red[2][w] = vol;
  }
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double a = red[k][0];
      for (int j = 1; j < nw; ++j) a += red[k][j];
      part[(size_t)blockIdx.x * 3 + k] = a;
    }
  }
}

__global__ void __launch_bounds__(256) k_kinetic_sum(int nb, const double* __restrict__ part, DevScalars* scal) {
  __shared__ double s[3][256];
  double a = 0, b = 0, c = 0;
  for (int i = threadIdx.x; i < nb; i += 256) {
    a += part[(size_t)i * 3 + 0];
    b += part[(size_t)i * 3 + 1];
    c += part[(size_t)i * 3 + 2];
  }
  s[0][threadIdx.x] = a;
  s[1][threadIdx.x] = b;
  s[2][threadIdx.x] = c;
  __syncwarp();
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s[0][threadIdx.x] += s[0][threadIdx.x + h];
      s[1][threadIdx.x] += s[1][threadIdx.x + h];
      s[2][threadIdx.x] += s[2][threadIdx.x + h];
    }
    __syncwarp();
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scal->kin[0] = s[0][0];
    scal->kin[1] = s[1][0];
    scal->kin[2] = s[2][0];
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
  if (!slave && ee.y < 0) {  // boundary face: no partner
    nbr[x * 3 + 1] = -1;
    for (int pq = 0; pq < n2; ++pq) nodes[x * n2 + pq] = -1;
    return;
  }
  for (int pq = 0; pq < n2; ++pq) {
    const int p = pq % n, q = pq / n;
    int a, b;
    if (slave) flip_to_master<n>(flip, p, q, a, b);
    else flip_to_slave<n>(flip, p, q, a, b);
    nodes[x * n2 + pq] = a + n * b;
  }
}

template <int N, typename S>
__global__ void k_debug_grad(int E, const S* __restrict__ g, double* out) {
  constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= (int64_t)E * n3) return;
  const int64_t e = x / n3;
  const int t = (int)(x % n3);
  for (int c = 0; c < 12; ++c) out[x * 12 + c] = g[e * 12 * n3 + (int64_t)c * n3 + t];
}

template <int N, typename S>
__global__ void k_debug_fstar(int E, const int* __restrict__ elem_side, const S* __restrict__ fstar,
                              double* out) {
  constexpr int n2 = (N + 1) * (N + 1);
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= (int64_t)E * 6 * n2) return;
  const int64_t ef = x / n2;
  const int pq = (int)(x % n2);
  const int es = elem_side[ef];
  for (int k = 0; k < 5; ++k)
    out[x * 5 + k] = es_slave(es) ? 0.0 : (double)fstar[(int64_t)es_side(es) * 5 * n2 + k * n2 + pq];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t init_kernel_attributes(int N) {
  switch (N) {
    case 1: return stage_attrs_n1();
    case 2: return stage_attrs_n2();
    case 3: return stage_attrs_n3();
    case 4: return stage_attrs_n4();
    case 5: return stage_attrs_n5();
    case 6: return stage_attrs_n6();
    case 7: return stage_attrs_n7();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rhs(dg_ctx* c, const double* U, int mode, double rkA, double rkB, int first) {
  switch (c->N) {
    case 1: return stage_launch_n1(c, U, mode, rkA, rkB, first);
    case 2: return stage_launch_n2(c, U, mode, rkA, rkB, first);
    case 3: return stage_launch_n3(c, U, mode, rkA, rkB, first);
    case 4: return stage_launch_n4(c, U, mode, rkA, rkB, first);
    case 5: return stage_launch_n5(c, U, mode, rkA, rkB, first);
    case 6: return stage_launch_n6(c, U, mode, rkA, rkB, first);
    case 7: return stage_launch_n7(c, U, mode, rkA, rkB, first);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fprep(dg_ctx* c, const double* U, int64_t e0, int64_t E, cudaStream_t st) {
  switch (c->N) {
    case 1: return fprep_n1(c, U, e0, E, st);
    case 2: return fprep_n2(c, U, e0, E, st);
    case 3: return fprep_n3(c, U, e0, E, st);
    case 4: return fprep_n4(c, U, e0, E, st);
    case 5: return fprep_n5(c, U, e0, E, st);
    case 6: return fprep_n6(c, U, e0, E, st);
    case 7: return fprep_n7(c, U, e0, E, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_persist(dg_ctx* c, int ns, const double* A, const double* B, const double* C, unsigned extra,
                           unsigned spin) {
  switch (c->N) {
    case 1: return persist_n1(c, ns, A, B, C, extra, spin);
    case 2: return persist_n2(c, ns, A, B, C, extra, spin);
    case 3: return persist_n3(c, ns, A, B, C, extra, spin);
    case 4: return persist_n4(c, ns, A, B, C, extra, spin);
    case 5: return persist_n5(c, ns, A, B, C, extra, spin);
    case 6: return persist_n6(c, ns, A, B, C, extra, spin);
    case 7: return persist_n7(c, ns, A, B, C, extra, spin);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_autotune(dg_ctx* c, double* ms) {
  switch (c->N) {
    case 1: return stage_autotune_n1(c, ms);
    case 2: return stage_autotune_n2(c, ms);
    case 3: return stage_autotune_n3(c, ms);
    case 4: return stage_autotune_n4(c, ms);
    case 5: return stage_autotune_n5(c, ms);
    case 6: return stage_autotune_n6(c, ms);
    case 7: return stage_autotune_n7(c, ms);
    default: return cudaErrorInvalidValue;
  }
}

// reference state of the shifted primitives: zero on the FP64 path; on the
// FP32-bulk path the density and pressure at the first node of element 0,
// at rest
__global__ void k_refs(const double* __restrict__ U, int n3, double gm1, double R, int use, DevScalars* s) {
  if (!use) {
    s->ref_p = s->ref_H = s->ref_T = s->ref_rho = s->ref_E = 0.0;
    s->f_ref_p = s->f_ref_H = s->f_ref_T = 0.0f;
    return;
  }
  const double r = U[0];
  const double mu = U[n3], mv = U[2 * n3], mw = U[3 * n3], E = U[4 * n3];
  const double p = gm1 * (E - 0.5 * (mu * mu + mv * mv + mw * mw) / r);
  s->ref_rho = r;
  s->ref_p = p;
  s->ref_E = p / gm1;
  s->ref_H = (s->ref_E + p) / r;
  s->ref_T = p / (r * R);
  s->f_ref_p = (float)s->ref_p;
  s->f_ref_H = (float)s->ref_H;
  s->f_ref_T = (float)s->ref_T;
}

cudaError_t launch_refs(dg_ctx* c) {
  k_refs<<<1, 1, 0, c->stream>>>(c->U, c->n3, c->prm.gamma - 1.0, c->prm.R,
                                 c->prm.precision == DG_FP32_BULK ? 1 : 0, c->scal);
  count_launch();
  return cudaGetLastError();
}

static int cfl_blocks(dg_ctx* c) {
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t need = (c->E * c->n3 + 255) / 256;
  return (int)std::min<int64_t>(need, (int64_t)sms * 8);
}

cudaError_t launch_cfl(dg_ctx* c, bool report_only) {
  const double kv = std::max(4.0 / 3.0, c->prm.gamma / c->prm.Pr) * c->prm.mu;
  const int nb = cfl_blocks(c);
  prof_begin(c, PK_CFL);
  if (c->prm.precision == DG_FP32_BULK) {
    DG_DISPATCH(c->N, (k_cfl<NN, float><<<nb, 256, 0, c->stream>>>((int)c->E, c->U, c->metric, c->metric32, c->cflgeo,
                                                                 c->prm.gamma, c->prm.gamma - 1.0, 1.0 / c->prm.R, kv,
                                                                 c->prm.viscous, c->prm.sutherland,
                                                                 1.0 / c->prm.T_ref, c->scal)));
  } else {
    DG_DISPATCH(c->N, (k_cfl<NN, double><<<nb, 256, 0, c->stream>>>((int)c->E, c->U, c->metric, c->metric32,
                                                                  c->cflgeo, c->prm.gamma, c->prm.gamma - 1.0,
                                                                  1.0 / c->prm.R, kv, c->prm.viscous,
                                                                  c->prm.sutherland, 1.0 / c->prm.T_ref, c->scal)));
  }
  if (report_only)
    k_dt_report<<<1, 1, 0, c->stream>>>(c->scal, c->prm.cfl, c->prm.dfl, c->N, c->prm.viscous);
  else
    k_dt<<<1, 1, 0, c->stream>>>(c->scal, c->prm.cfl, c->prm.dfl, c->N, c->prm.viscous);
  prof_end(c);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_dt_next(dg_ctx* c) {
  prof_begin(c, PK_CFL);
  k_dt<<<1, 1, 0, c->stream>>>(c->scal, c->prm.cfl, c->prm.dfl, c->N, c->prm.viscous, 1);
  prof_end(c);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_clear_next(DevScalars* scal) {
  scal->lam_c_next = 0ull;
  scal->lam_v_next = 0ull;
}
cudaError_t launch_clear_next(dg_ctx* c) {
  k_clear_next<<<1, 1, 0, c->stream>>>(c->scal);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_to_internal(dg_ctx* c, const double* pub, double* internal) {
  if (c->E == 0) return cudaSuccess;
  k_to_internal<<<(unsigned)c->E, 256, sizeof(double) * 5 * c->n3, c->stream>>>(c->n3, pub, internal);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_to_public(dg_ctx* c, const double* internal, double* pub) {
  if (c->E == 0) return cudaSuccess;
  k_to_public<<<(unsigned)c->E, 256, sizeof(double) * 5 * c->n3, c->stream>>>(c->n3, internal, pub);
  count_launch();
  return cudaGetLastError();
}

int kinetic_blocks(dg_ctx* c) { return cfl_blocks(c); }

cudaError_t launch_kinetic(dg_ctx* c, const double* U, const double* Ut) {
  const int nb = cfl_blocks(c);
  if (!c->kin_part || c->kin_part_blocks < nb) return cudaErrorInvalidValue;
  DG_DISPATCH(c->N, (k_kinetic<NN><<<nb, 256, 0, c->stream>>>((int)c->E, U, Ut, c->metric, c->ops, c->kin_part)));
  k_kinetic_sum<<<1, 256, 0, c->stream>>>(nb, c->kin_part, c->scal);
  count_launch(2);
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
  if (c->prm.precision == DG_FP32_BULK) {
    DG_DISPATCH(c->N, (k_debug_grad<NN, float><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
                          (int)c->E, c->g32, out)));
  } else {
    DG_DISPATCH(c->N, (k_debug_grad<NN, double><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
                          (int)c->E, c->g, out)));
  }
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_debug_fstar(dg_ctx* c, double* out) {
  const int64_t tot = c->E * 6 * c->n2;
  if (c->prm.precision == DG_FP32_BULK) {
    DG_DISPATCH(c->N, (k_debug_fstar<NN, float><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
                          (int)c->E, c->elem_side, c->fstar32, out)));
  } else {
    DG_DISPATCH(c->N, (k_debug_fstar<NN, double><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
                          (int)c->E, c->elem_side, c->fstar, out)));
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace dg
