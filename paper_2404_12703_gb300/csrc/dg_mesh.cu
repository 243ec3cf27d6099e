// dg_mesh.cu -- mesh set-up on the device: element<->side maps with face
// orientation found from corner vertex ids (the unstructured-mesh mappings of
// Sec. 2.2 / App. A ProlongToFace and SurfInt), curl-form metrics
// (Sec. 2.2, Mapping the Equations) in double-double, surface normals and the
// sub-cell interface metrics used by the FV blending (Sec. 2.3).
#include <cstdio>
#include <string>
#include <vector>

#include "dg_common.cuh"
#include "dg_launch.h"

namespace dg {

// ---------------------------------------------------------------------------
// Face keys and matching
// ---------------------------------------------------------------------------
__device__ __forceinline__ int corner_of_face(int f, int a, int b) {
  const int d = f >> 1, s = f & 1;
  int bi, bj, bk;
  if (d == 0) { bi = s; bj = a; bk = b; }
  else if (d == 1) { bi = a; bj = s; bk = b; }
  else { bi = a; bj = b; bk = s; }
  return bi + 2 * bj + 4 * bk;
}

struct Key4 {
  long long v[4];
};

__device__ __forceinline__ Key4 face_key(const long long* cvid, int F) {
  const int e = F / 6, f = F % 6;
  Key4 k;
  for (int c = 0; c < 4; ++c) k.v[c] = cvid[(size_t)e * 8 + corner_of_face(f, c & 1, c >> 1)];
  // sort 4 values (small network)
#define DG_SWAP(a, b) if (k.v[a] > k.v[b]) { long long t_ = k.v[a]; k.v[a] = k.v[b]; k.v[b] = t_; }
  DG_SWAP(0, 1) DG_SWAP(2, 3) DG_SWAP(0, 2) DG_SWAP(1, 3) DG_SWAP(1, 2)
#undef DG_SWAP
  return k;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return x;
}

__global__ void k_face_insert(int64_t F_total, const long long* cvid, int* table, unsigned long long mask,
                              int* partner, int* err) {
  int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= F_total) return;
  Key4 k = face_key(cvid, (int)F);
  if (k.v[0] == k.v[1] || k.v[1] == k.v[2] || k.v[2] == k.v[3]) {
    atomicOr(err, 1);  // repeated corner id on one face
    return;
  }
  unsigned long long h = mix64((unsigned long long)k.v[0] * 0x9E3779B97F4A7C15ULL ^
                               mix64((unsigned long long)k.v[1] + 0x632BE59BD9B4E019ULL) ^
                               mix64((unsigned long long)k.v[2] * 3 + 1) ^ mix64((unsigned long long)k.v[3] * 7 + 5));
  unsigned long long slot = h & mask;
  for (unsigned long long probe = 0; probe <= mask; ++probe) {
    int cur = table[slot];
    if (cur == -1) {
      int old = atomicCAS(&table[slot], -1, (int)F);
      if (old == -1) return;  // first of the pair: its partner will find it
      cur = old;
    }
    Key4 o = face_key(cvid, cur);
    if (o.v[0] == k.v[0] && o.v[1] == k.v[1] && o.v[2] == k.v[2] && o.v[3] == k.v[3]) {
      if (atomicCAS(&partner[cur], -1, (int)F) == -1) {
        partner[F] = cur;
      } else {
        atomicOr(err, 2);  // three or more faces with the same corners
      }
      return;
    }
    slot = (slot + 1) & mask;
  }
  atomicOr(err, 4);  // table full (cannot happen with load factor <= 1/2)
}

// face_bc (may be null): > 0 marks a boundary face (it has no partner and
// forms a side of its own)
__global__ void k_face_check(int64_t F_total, const int* partner, const int* face_bc, int* master_flag, int* err) {
  int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= F_total) return;
  const int P = partner[F];
  const int bc = face_bc ? face_bc[F] : 0;
  if (P == -1 && bc > 0) {
    master_flag[F] = 1;  // boundary face
    return;
  }
  if (P < 0 || P >= F_total || partner[P] != (int)F || P == (int)F || bc != 0) {
    atomicOr(err, 8);  // open face without a condition, a condition on an inner face, or bad pairing
    master_flag[F] = 0;
    return;
  }
  master_flag[F] = (int)F < P ? 1 : 0;
}

// exclusive scan of 0/1 flags by one block of 1024 threads, chunk by chunk
__global__ void __launch_bounds__(1024) k_scan_flags(int64_t n, const int* flag, int* out, int* total) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += 1024) {
    int64_t i = base + threadIdx.x;
    int v = i < n ? flag[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncwarp();
    __syncthreads();
    if (wid == 0) {
      int s = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;
    }
    __syncwarp();
    __syncthreads();
    int incl = x + (wid > 0 ? warp_sums[wid - 1] : 0);
    if (i < n) out[i] = carry + incl - v;
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 1023) carry += incl;
    __syncwarp();
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_fill_sides(int64_t F_total, const long long* cvid, const int* partner, const int* master_flag,
                             const int* side_of, const int* face_bc, int* elem_side, int2* side_e, int* side_f,
                             int* side_bc, int* err) {
  int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (F >= F_total || !master_flag[F]) return;
  const int P = partner[F];
  const int s = side_of[F];
  if (P < 0) {  // boundary side: master only, condition row face_bc - 1
    side_e[s] = make_int2((int)(F / 6), -1);
    side_f[s] = (int)(F % 6) | (15 << 4);
    elem_side[F] = s << 4;
    side_bc[s] = face_bc[F] - 1;
    return;
  }
  side_bc[s] = -1;
  const int eM = (int)(F / 6), fM = (int)(F % 6), eS = P / 6, fS = P % 6;
  long long vm[4], vs[4];
  for (int c = 0; c < 4; ++c) {
    vm[c] = cvid[(size_t)eM * 8 + corner_of_face(fM, c & 1, c >> 1)];
    vs[c] = cvid[(size_t)eS * 8 + corner_of_face(fS, c & 1, c >> 1)];
  }
  int found = -1, count = 0;
  for (int fl = 0; fl < 8; ++fl) {
    bool ok = true;
    for (int c = 0; c < 4; ++c) {
      int pm, qm;
      flip_to_master<2>(fl, c & 1, c >> 1, pm, qm);
      if (vs[c] != vm[pm + 2 * qm]) ok = false;
    }
    if (ok) { found = fl; ++count; }
  }
  if (count != 1) {
    atomicOr(err, 16);  // the two faces' corners are not related by a square symmetry
    found = 0;
  }
  side_e[s] = make_int2(eM, eS);
  side_f[s] = fM | (fS << 4) | (found << 8);
  elem_side[F] = (s << 4) | found;
  elem_side[P] = (s << 4) | 8 | found;
}

// ---------------------------------------------------------------------------
// Metrics in double-double (curl form) on the LGL nodes of the geometry; on
// Gauss-Legendre nodes the same polynomials (J a^d and dx/dxi) evaluated at
// the GL nodes by exact interpolation, J = det(dx/dxi) there.  1/J; the
// solution nodes' coordinates.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__((N + 1) * (N + 1) * (N + 1)) k_metrics(int E, const double* __restrict__ xyz,
                                                                        const Ops* __restrict__ ops, int gauss,
                                                                        double* __restrict__ metric,
                                                                        double* __restrict__ xyzs) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* sD = reinterpret_cast<dd*>(smem_raw);      // [n2] LGL D
  dd* sI = sD + n2;                              // [n2] LGL -> solution nodes
  dd* sX = sI + n2;                              // [3][n3]
  dd* sV = sX + 3 * n3;                          // [3][n3]
  const int e = blockIdx.x;
  const int t = threadIdx.x;
  if (e >= E) return;
  for (int k = t; k < n2; k += n3) {
    sD[k] = {ops->Dg[k], ops->Dg_lo[k]};
    sI[k] = {ops->Ig[k], ops->Ig_lo[k]};
  }
  const double* X = xyz + (size_t)e * n3 * 3;
  for (int c = 0; c < 3; ++c) sX[c * n3 + t] = two_sum(X[t * 3 + c], -X[c]);
  __syncwarp();
  __syncthreads();
  const int idx[3] = {t % n, (t / n) % n, t / n2};
  const int str[3] = {1, n, n2};
  dd dx[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dd s = dd_from(0.0);
      const int base = t - idx[d] * str[d];
#pragma unroll
      for (int a = 0; a < n; ++a) s = dd_add(s, dd_mul(sD[idx[d] * n + a], sX[c * n3 + base + a * str[d]]));
      dx[c][d] = s;
    }
  dd Ja[3][3];  // Ja[d][c] = (J a^d)_c
  for (int nc = 0; nc < 3; ++nc) {
    const int m = (nc + 1) % 3, l = (nc + 2) % 3;
#pragma unroll
    for (int d = 0; d < 3; ++d) sV[d * n3 + t] = dd_mul(sX[l * n3 + t], dx[m][d]);
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < 3; ++ii) {
      const int i1 = (ii + 1) % 3, i2 = (ii + 2) % 3;
      dd a1 = dd_from(0.0), a2 = dd_from(0.0);
      const int b1 = t - idx[i1] * str[i1], b2 = t - idx[i2] * str[i2];
#pragma unroll
      for (int a = 0; a < n; ++a) {
        a1 = dd_add(a1, dd_mul(sD[idx[i1] * n + a], sV[i2 * n3 + b1 + a * str[i1]]));
        a2 = dd_add(a2, dd_mul(sD[idx[i2] * n + a], sV[i1 * n3 + b2 + a * str[i2]]));
      }
      Ja[ii][nc] = dd_neg(dd_sub(a1, a2));
    }
    __syncthreads();
  }
  dd Xs[3];  // relative coordinates of the solution node
#pragma unroll
  for (int c = 0; c < 3; ++c) Xs[c] = sX[c * n3 + t];
  if (gauss) {
    // tensor-product interpolation to the GL nodes, one direction at a time
    // (sV is free now); every thread takes every barrier
    dd* B0 = sV;
    dd* B1 = sV + n3;
    auto interp = [&](dd v) -> dd {
      B0[t] = v;
      __syncthreads();
#pragma unroll 1
      for (int d = 0; d < 3; ++d) {
        const dd* src = d == 1 ? B1 : B0;
        dd* dst = d == 1 ? B0 : B1;
        const int base = t - idx[d] * str[d];
        dd s = dd_from(0.0);
        for (int a = 0; a < n; ++a) s = dd_add(s, dd_mul(sI[idx[d] * n + a], src[base + a * str[d]]));
        dst[t] = s;
        __syncthreads();
      }
      const dd r = B1[t];
      __syncthreads();
      return r;
    };
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) {
        dx[c][d] = interp(dx[c][d]);
        Ja[c][d] = interp(Ja[c][d]);
      }
    for (int c = 0; c < 3; ++c) Xs[c] = interp(Xs[c]);
  }
  // J = det(dx / dxi)
  dd J = dd_sub(dd_mul(dx[1][1], dx[2][2]), dd_mul(dx[1][2], dx[2][1]));
  J = dd_mul(dx[0][0], J);
  J = dd_sub(J, dd_mul(dx[0][1], dd_sub(dd_mul(dx[1][0], dx[2][2]), dd_mul(dx[1][2], dx[2][0]))));
  J = dd_add(J, dd_mul(dx[0][2], dd_sub(dd_mul(dx[1][0], dx[2][1]), dd_mul(dx[1][1], dx[2][0]))));
  double* Me = metric + (size_t)e * 10 * n3;
  Me[9 * n3 + t] = 1.0 / dd_to_double(J);
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int c = 0; c < 3; ++c) Me[(d * 3 + c) * n3 + t] = dd_to_double(Ja[d][c]);
#pragma unroll
  for (int c = 0; c < 3; ++c) xyzs[((size_t)e * n3 + t) * 3 + c] = dd_to_double(dd_add(Xs[c], dd_from(X[c])));
}

// sub-cell interface metrics of the FV blending (LGL), by telescoping the
// discrete derivative of J a^d along each line: one thread per line and
// direction, formed when shock capturing is first enabled
template <int N>
__global__ void k_fv_metrics(int E, const double* __restrict__ metric, const Ops* __restrict__ ops,
                             double* __restrict__ fvm) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)E * 3 * n2) return;
  const int64_t e = tid / (3 * n2);
  const int tt = (int)(tid % (3 * n2));
  const int d = tt / n2, line = tt % n2;
  const int p = line % n, q = line / n;
  int base, st;
  if (d == 0) { base = n * (p + n * q); st = 1; }
  else if (d == 1) { base = p + n2 * q; st = n; }
  else { base = p + n * q; st = n2; }
  const double* Me = metric + (size_t)e * 10 * n3;
  double* F = fvm + (size_t)e * 3 * (n - 1) * 3 * n2;
  for (int c = 0; c < 3; ++c) {
    const double* Jd_c = Me + (d * 3 + c) * n3;
    double Jh = Jd_c[base];
    for (int i = 0; i < n - 1; ++i) {
      double dj = 0.0;
      for (int a = 0; a < n; ++a) dj += ops->D[i * n + a] * Jd_c[base + a * st];
      Jh = Jh + ops->w[i] * dj;
      F[((d * (n - 1) + i) * 3 + c) * n2 + line] = Jh;
    }
  }
}

// surface normal s n (outward for the master) and surface element s of every
// side node: J a^d of the master's face direction at the face node (LGL) or
// interpolated to the face with l(+-1) (GL)
template <int N>
__global__ void k_side_geom(int S, const int2* __restrict__ side_e, const int* __restrict__ side_f,
                            const double* __restrict__ metric, const Ops* __restrict__ ops, int gauss,
                            double* __restrict__ nrm) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)S * n2) return;
  const int s = (int)(tid / n2), pq = (int)(tid % n2);
  const int eM = side_e[s].x, fM = side_f[s] & 15;
  const int v = face_vol_node<n>(fM, pq % n, pq / n);
  const double sg = (fM & 1) ? 1.0 : -1.0;
  const double* Me = metric + (size_t)eM * 10 * n3 + (fM >> 1) * 3 * n3;
  double sn[3];
  if (gauss) {
    const int d = fM >> 1, st = d == 0 ? 1 : (d == 1 ? n : n2);
    const int v0 = v - ((fM & 1) ? n - 1 : 0) * st;  // node 0 of the line
    const double* L = (fM & 1) ? ops->Lp : ops->Lm;
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int a = 0; a < n; ++a) acc += L[a] * Me[c * n3 + v0 + a * st];
      sn[c] = sg * acc;
    }
  } else {
    for (int c = 0; c < 3; ++c) sn[c] = sg * Me[c * n3 + v];
  }
  double* out = nrm + (size_t)s * 4 * n2;
  out[pq] = sn[0];
  out[n2 + pq] = sn[1];
  out[2 * n2 + pq] = sn[2];
  out[3 * n2 + pq] = sqrt(sn[0] * sn[0] + sn[1] * sn[1] + sn[2] * sn[2]);
}

// per-node geometric factors of the time-step rule: |J a^d| and sum_d |J a^d|^2
template <int N>
__global__ void k_cfl_geo(int E, const double* __restrict__ metric, double* __restrict__ geo) {
  constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= (int64_t)E * n3) return;
  const int64_t e = x / n3;
  const int t = (int)(x % n3);
  const double* Me = metric + e * 10 * n3 + t;
  double* G = geo + e * 4 * n3 + t;
  double b = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double j0 = Me[(d * 3) * n3], j1 = Me[(d * 3 + 1) * n3], j2 = Me[(d * 3 + 2) * n3];
    const double nj2 = j0 * j0 + j1 * j1 + j2 * j2;
    G[d * n3] = sqrt(nj2);
    b += nj2;
  }
  G[3 * n3] = b;
}

// FP32 side geometry: s n, the unit normal and s, each rounded once
__global__ void k_nrm32(int64_t nodes, int n2, const double* __restrict__ nrm, float* __restrict__ nrm32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nodes) return;
  const int64_t s = i / n2;
  const int pq = (int)(i % n2);
  const double* in = nrm + s * 4 * n2 + pq;
  float* out = nrm32 + s * 7 * n2 + pq;
  const double sA = in[3 * n2];
  for (int k = 0; k < 3; ++k) {
    out[k * n2] = (float)in[k * n2];
    out[(3 + k) * n2] = (float)(in[k * n2] / sA);
  }
  out[6 * n2] = (float)sA;
}

// FP32 copy of an FP64 array (round to nearest)
__global__ void k_round_f32(int64_t n, const double* __restrict__ src, float* __restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

template <int N>
static cudaError_t launch_metrics(dg_ctx* c, const double* d_xyz) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const size_t sm = sizeof(dd) * (2 * n2 + 6 * n3);
  cudaFuncSetAttribute(k_metrics<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_metrics<N><<<(unsigned)c->E, n3, sm, c->stream>>>((int)c->E, d_xyz, c->ops, c->gauss, c->metric, c->xyzs);
  count_launch();
  const int64_t tot = c->S * n2;
  k_side_geom<N><<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>((int)c->S, c->side_e, c->side_f, c->metric,
                                                                       c->ops, c->gauss, c->nrm);
  const int64_t nodes = c->E * n3;
  k_cfl_geo<N><<<(unsigned)((nodes + 255) / 256), 256, 0, c->stream>>>((int)c->E, c->metric, c->cflgeo);
  count_launch(2);
  return cudaGetLastError();
}

// FP32 copies of the metrics and side geometry (FP32-bulk), from the FP64 ones
cudaError_t launch_fp32_geometry(dg_ctx* c, cudaStream_t st) {
  const int64_t tot = c->S * c->n2;
  if (tot > 0) k_nrm32<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, c->n2, c->nrm, c->nrm32);
  const int64_t mwords = c->E * 10 * c->n3;
  if (mwords > 0) k_round_f32<<<(unsigned)((mwords + 255) / 256), 256, 0, st>>>(mwords, c->metric, c->metric32);
  count_launch(2);
  return cudaGetLastError();
}

// sub-cell interface metrics (shock capturing), from the FP64 metrics
cudaError_t launch_fv_metrics(dg_ctx* c, cudaStream_t st) {
  const int64_t tot = c->E * 3 * c->n2;
  if (tot == 0) return cudaSuccess;
  const unsigned nb = (unsigned)((tot + 127) / 128);
  switch (c->N) {
    case 1: k_fv_metrics<1><<<nb, 128, 0, st>>>((int)c->E, c->metric, c->ops, c->fvmetric); break;
    case 2: k_fv_metrics<2><<<nb, 128, 0, st>>>((int)c->E, c->metric, c->ops, c->fvmetric); break;
    case 3: k_fv_metrics<3><<<nb, 128, 0, st>>>((int)c->E, c->metric, c->ops, c->fvmetric); break;
    case 4: k_fv_metrics<4><<<nb, 128, 0, st>>>((int)c->E, c->metric, c->ops, c->fvmetric); break;
    case 5: k_fv_metrics<5><<<nb, 128, 0, st>>>((int)c->E, c->metric, c->ops, c->fvmetric); break;
    case 6: k_fv_metrics<6><<<nb, 128, 0, st>>>((int)c->E, c->metric, c->ops, c->fvmetric); break;
    case 7: k_fv_metrics<7><<<nb, 128, 0, st>>>((int)c->E, c->metric, c->ops, c->fvmetric); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

// Builds maps and geometry.  Returns a DG_* status and an error message.
int build_mesh(dg_ctx* c, const int64_t* h_cvid, const double* h_xyz, const int* h_face_bc, std::string& msg) {
  const int64_t E = c->E, F = 6 * E;
  int* d_fbc = nullptr;
  const int n3 = c->n3;
  long long* d_cvid = nullptr;
  double* d_xyz = nullptr;
  int *d_table = nullptr, *d_partner = nullptr, *d_flag = nullptr, *d_sideof = nullptr, *d_misc = nullptr;
  unsigned long long tsize = 1;
  while (tsize < (unsigned long long)(2 * F)) tsize <<= 1;
  int status = DG_OK;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && status == DG_OK) {
      msg = std::string(what) + ": " + cudaGetErrorString(e);
      status = e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
    }
  };
  // temporaries: from the library pool for pool-stream contexts
  auto tmp_alloc = [&](auto** p, size_t bytes, const char* what) {
    cudaError_t e = c->pool_stream ? pool_alloc((void**)p, bytes, c->pool_stream) : cudaMalloc((void**)p, bytes);
    ck(e, what);
  };
  auto tmp_free = [&](void* p) {
    if (!p) return;
    if (c->pool_stream) cudaFreeAsync(p, c->pool_stream);
    else cudaFree(p);
  };
  tmp_alloc(&d_cvid, sizeof(long long) * E * 8, "allocating cvid");
  tmp_alloc(&d_xyz, sizeof(double) * E * n3 * 3, "allocating xyz");
  tmp_alloc(&d_table, sizeof(int) * tsize, "allocating table");
  tmp_alloc(&d_partner, sizeof(int) * F, "allocating partner");
  tmp_alloc(&d_flag, sizeof(int) * F, "allocating flag");
  tmp_alloc(&d_sideof, sizeof(int) * F, "allocating sideof");
  tmp_alloc(&d_misc, sizeof(int) * 4, "allocating misc");
  if (h_face_bc) tmp_alloc(&d_fbc, sizeof(int) * F, "allocating face_bc");
  if (status == DG_OK) {
    ck(cudaMemcpyAsync(d_cvid, h_cvid, sizeof(long long) * E * 8, cudaMemcpyHostToDevice, c->stream), "copy cvid");
    ck(cudaMemcpyAsync(d_xyz, h_xyz, sizeof(double) * E * n3 * 3, cudaMemcpyHostToDevice, c->stream), "copy xyz");
    ck(cudaMemsetAsync(d_table, 0xff, sizeof(int) * tsize, c->stream), "memset table");
    ck(cudaMemsetAsync(d_partner, 0xff, sizeof(int) * F, c->stream), "memset partner");
    ck(cudaMemsetAsync(d_misc, 0, sizeof(int) * 4, c->stream), "memset misc");
    if (h_face_bc)
      ck(cudaMemcpyAsync(d_fbc, h_face_bc, sizeof(int) * F, cudaMemcpyHostToDevice, c->stream), "copy face_bc");
  }
  const unsigned nb = (unsigned)((F + 255) / 256);
  int h_misc[4] = {0, 0, 0, 0};
  if (status == DG_OK) {
    k_face_insert<<<nb, 256, 0, c->stream>>>(F, d_cvid, d_table, tsize - 1, d_partner, d_misc);
    k_face_check<<<nb, 256, 0, c->stream>>>(F, d_partner, d_fbc, d_flag, d_misc);
    k_scan_flags<<<1, 1024, 0, c->stream>>>(F, d_flag, d_sideof, d_misc + 1);
    count_launch(3);
    ck(cudaGetLastError(), "map kernels");
    ck(cudaMemcpyAsync(h_misc, d_misc, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream), "copy misc");
    ck(cudaStreamSynchronize(c->stream), "sync maps");
  }
  if (status == DG_OK && h_misc[0] != 0) {
    msg = "mesh faces do not pair up (code " + std::to_string(h_misc[0]) +
          "): every face needs exactly one partner with the same four distinct corner ids, "
          "or a boundary condition if it has none (a periodic direction needs at least three elements)";
    status = DG_ERR_MESH;
  }
  if (status == DG_OK && ((!h_face_bc && h_misc[1] != 3 * E) || h_misc[1] < 3 * E)) {
    msg = "unexpected number of sides";
    status = DG_ERR_MESH;
  }
  if (status == DG_OK) {
    c->S = h_misc[1];
    status = alloc_side_arrays(c, msg);
  }
  if (status == DG_OK) {
    ck(cudaMemsetAsync(d_misc, 0, sizeof(int) * 4, c->stream), "memset misc");
    k_fill_sides<<<nb, 256, 0, c->stream>>>(F, d_cvid, d_partner, d_flag, d_sideof, d_fbc, c->elem_side,
                                            c->side_e, c->side_f, c->side_bc, d_misc);
    count_launch();
    ck(cudaGetLastError(), "fill sides");
    cudaError_t le = cudaSuccess;
    switch (c->N) {
      case 1: le = launch_metrics<1>(c, d_xyz); break;
      case 2: le = launch_metrics<2>(c, d_xyz); break;
      case 3: le = launch_metrics<3>(c, d_xyz); break;
      case 4: le = launch_metrics<4>(c, d_xyz); break;
      case 5: le = launch_metrics<5>(c, d_xyz); break;
      case 6: le = launch_metrics<6>(c, d_xyz); break;
      case 7: le = launch_metrics<7>(c, d_xyz); break;
      default: break;
    }
    ck(le, "metric kernels");
    ck(cudaMemcpyAsync(h_misc, d_misc, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream), "copy misc");
    ck(cudaStreamSynchronize(c->stream), "sync metrics");
    if (status == DG_OK && h_misc[0] != 0) {
      msg = "a face pair's corners are not related by a rotation or reflection of the square";
      status = DG_ERR_MESH;
    }
  }
  tmp_free(d_cvid);
  tmp_free(d_xyz);
  tmp_free(d_table);
  tmp_free(d_partner);
  tmp_free(d_flag);
  tmp_free(d_sideof);
  tmp_free(d_misc);
  tmp_free(d_fbc);
  return status;
}

}  // namespace dg
