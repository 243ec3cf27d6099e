// dg_api.cu -- the C ABI of libdg (include/dg.h): context life cycle, the 1D
// operators, state transfer, RHS evaluation and graph-launched LSERK steps.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dg_common.cuh"
#include "dg_launch.h"

namespace dg {

static std::atomic<int64_t> g_launches{0};
void count_launch(int k) { g_launches += k; }

void prof_begin(dg_ctx* c, int kind) {
  Profiler* p = c->prof;
  if (!p || p->used >= Profiler::MAX_EV) return;
  p->slot[p->used] = kind;
  cudaEventRecord(p->ev[p->used][0], c->stream);
}
void prof_end(dg_ctx* c) {
  Profiler* p = c->prof;
  if (!p || p->used >= Profiler::MAX_EV) return;
  cudaEventRecord(p->ev[p->used][1], c->stream);
  ++p->used;
}

static thread_local std::string g_last_error;
static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
static int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// 1D operators (Sec. 2.2): LGL nodes as -1, +1 and the zeros of the Jacobi
// polynomial P^(1,1)_{N-1} (proportional to P_N'), weights 2/(N(N+1)P_N^2),
// the derivative matrix from barycentric weights, all in long double.
// ---------------------------------------------------------------------------
typedef long double ld;

static void jacobi11(int m, ld x, ld& Pm, ld& Pm1) {
  // P^(1,1)_0 = 1, P^(1,1)_1 = 2x,
  // k (k+2) P_k = (2k+1)(k+1) x P_{k-1} - k (k+1) P_{k-2}
  ld a = 1, b = 2 * x;
  if (m == 0) { Pm = 1; Pm1 = 0; return; }
  for (int k = 2; k <= m; ++k) {
    ld c = ((2 * k + 1) * (ld)(k + 1) * x * b - (ld)k * (k + 1) * a) / ((ld)k * (k + 2));
    a = b;
    b = c;
  }
  Pm = b;
  Pm1 = a;
}

static ld legendreP(int N, ld x) {
  ld a = 1, b = x;
  if (N == 0) return 1;
  for (int k = 2; k <= N; ++k) {
    ld c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    a = b;
    b = c;
  }
  return b;
}

// LGL nodes and weights of degree N
static void lgl_nodes(int N, ld* x, ld* w) {
  x[0] = -1;
  x[N] = 1;
  const int m = N - 1;
  for (int j = 1; j < N; ++j) {
    ld t = -std::cos((ld)M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      ld P, Pp;
      jacobi11(m, t, P, Pp);
      // (1 - x^2) P_m' = -m x P_m + (m + 1) P_{m-1}
      ld dP = (-(ld)m * t * P + (ld)(m + 1) * Pp) / (1 - t * t);
      ld step = P / dP;
      t -= step;
      if (std::fabs(step) < 1e-30L) break;
    }
    x[j] = t;
  }
  for (int j = 0; j <= N; ++j) {
    ld P = legendreP(N, x[j]);
    w[j] = 2 / ((ld)N * (N + 1) * P * P);
  }
}

// Gauss-Legendre nodes (the zeros of P_{N+1}) and weights
// 2 / ((1 - x^2) P_{N+1}'(x)^2), with P_m' = m (P_{m-1} - x P_m) / (1 - x^2)
static void gauss_nodes(int N, ld* x, ld* w) {
  const int m = N + 1;
  for (int j = 0; j < m; ++j) {
    ld t = -std::cos((ld)M_PI * (j + 0.75L) / (m + 0.5L));
    ld dP = 1;
    for (int it = 0; it < 100; ++it) {
      const ld P = legendreP(m, t), P1 = legendreP(m - 1, t);
      dP = (ld)m * (P1 - t * P) / (1 - t * t);
      const ld step = P / dP;
      t -= step;
      if (std::fabs(step) < 1e-30L) break;
    }
    const ld P1 = legendreP(m - 1, t), P = legendreP(m, t);
    dP = (ld)m * (P1 - t * P) / (1 - t * t);
    x[j] = t;
    w[j] = 2 / ((1 - t * t) * dP * dP);
  }
}

// D[i][j] = l_j'(x_i) from barycentric weights
static void derivative_matrix(int n, const ld* x, ld* D) {
  ld lam[NPMAX];
  for (int j = 0; j < n; ++j) {
    ld p = 1;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= (x[j] - x[k]);
    lam[j] = 1 / p;
  }
  for (int i = 0; i < n; ++i) {
    ld s = 0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[i * n + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
      s += D[i * n + j];
    }
    D[i * n + i] = -s;
  }
}

// Lagrange basis l_j(y) of the nodes x
static ld lagrange(int n, const ld* x, int j, ld y) {
  ld v = 1;
  for (int k = 0; k < n; ++k)
    if (k != j) v *= (y - x[k]) / (x[j] - x[k]);
  return v;
}

static void build_ops(int N, int gauss, Ops& o) {
  const int n = N + 1;
  ld xl[NPMAX], wl[NPMAX], Dl[NPMAX * NPMAX];
  ld x[NPMAX], w[NPMAX], D[NPMAX * NPMAX];
  lgl_nodes(N, xl, wl);
  derivative_matrix(n, xl, Dl);
  if (gauss) {
    gauss_nodes(N, x, w);
    derivative_matrix(n, x, D);
  } else {
    for (int i = 0; i < n; ++i) x[i] = xl[i], w[i] = wl[i];
    for (int i = 0; i < n * n; ++i) D[i] = Dl[i];
  }
  memset(&o, 0, sizeof(o));
  for (int i = 0; i < n; ++i) {
    o.x[i] = (double)x[i];
    o.w[i] = (double)w[i];
    o.winv[i] = (double)(1 / w[i]);
    o.Lp[i] = gauss ? (double)lagrange(n, x, i, 1) : (i == N ? 1.0 : 0.0);
    o.Lm[i] = gauss ? (double)lagrange(n, x, i, -1) : (i == 0 ? 1.0 : 0.0);
  }
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < n; ++a) {
      const ld d = D[i * n + a];
      o.D[i * n + a] = (double)d;
      o.Dlo[i * n + a] = (double)(d - (ld)o.D[i * n + a]);
      // weak operator: Dhat_ia = -(w_a / w_i) D_ai
      o.Dhat[i * n + a] = (double)(-(w[a] / w[i]) * D[a * n + i]);
      // split operator (LGL): 2 D plus the two surface corrections
      ld ds = 2 * d;
      if (i == N && a == N) ds -= 1 / w[N];
      if (i == 0 && a == 0) ds += 1 / w[0];
      o.Dsplit[i * n + a] = gauss ? 0.0 : (double)ds;
      const ld dg = Dl[i * n + a];
      o.Dg[i * n + a] = (double)dg;
      o.Dg_lo[i * n + a] = (double)(dg - (ld)o.Dg[i * n + a]);
      const ld ig = gauss ? lagrange(n, xl, a, x[i]) : (ld)(i == a ? 1 : 0);
      o.Ig[i * n + a] = (double)ig;
      o.Ig_lo[i * n + a] = (double)(ig - (ld)o.Ig[i * n + a]);
    }
  // inverse Vandermonde of the orthonormal Legendre basis by discrete
  // orthogonality of the quadrature (exact to degree 2N - 1 on LGL, 2N + 1 on
  // GL): c_m = sum_i w_i L_m(x_i) u_i / gamma_m
  ld L[NPMAX * NPMAX];
  for (int mm = 0; mm < n; ++mm)
    for (int i = 0; i < n; ++i) L[mm * n + i] = std::sqrt((ld)(2 * mm + 1) / 2) * legendreP(mm, x[i]);
  for (int mm = 0; mm < n; ++mm) {
    ld gam = 0;
    for (int i = 0; i < n; ++i) gam += w[i] * L[mm * n + i] * L[mm * n + i];
    for (int i = 0; i < n; ++i) o.Vinv[mm * n + i] = (double)(w[i] * L[mm * n + i] / gam);
  }
}

int set_error(int code, const std::string& msg) { return fail(code, msg); }

void quadrature_weights(int N, int gauss, double* w) {
  Ops o;
  build_ops(N, gauss, o);
  for (int i = 0; i <= N; ++i) w[i] = o.w[i];
}

// Stream-ordered allocations from a pool owned by the library (one per
// device), which keeps freed memory for reuse: contexts created for the
// server's cases allocate and free without the device-wide waits of
// cudaMalloc / cudaFree.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  static std::mutex m;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(m);
    if (!pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pools[dev], &props);
      if (e != cudaSuccess) {
        pools[dev] = nullptr;
        return e;
      }
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pool = pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

template <typename T>
static cudaError_t dalloc(dg_ctx* c, T** p, size_t count) {
  cudaError_t e = c->pool_stream ? pool_alloc((void**)p, sizeof(T) * count, c->pool_stream)
                                 : cudaMalloc((void**)p, sizeof(T) * count);
  if (e == cudaSuccess) c->bytes += (int64_t)(sizeof(T) * count);
  return e;
}

static void dfree(dg_ctx* c, void* p) {
  if (!p) return;
  if (c->pool_stream) cudaFreeAsync(p, c->pool_stream);
  else cudaFree(p);
}

// side arrays common to both precisions (the working arrays of one
// precision come from ensure_arrays)
int alloc_side_arrays(dg_ctx* c, std::string& msg) {
  cudaError_t e = cudaSuccess;
  const int64_t S = c->S, n2 = c->n2;
  if (e == cudaSuccess) e = dalloc(c, &c->nrm, S * 4 * n2);
  if (e == cudaSuccess) e = dalloc(c, &c->side_e, S);
  if (e == cudaSuccess) e = dalloc(c, &c->side_f, S);
  if (e == cudaSuccess) e = dalloc(c, &c->side_bc, S);
  if (c->gauss && e == cudaSuccess) e = dalloc(c, &c->Ufc, S * 2 * 5 * n2);
  if (e != cudaSuccess) {
    msg = std::string("side arrays: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
  }
  return DG_OK;
}

// The working arrays of the parameters' precision (FP64: lifted gradients,
// lifting and surface fluxes; FP32-bulk: their FP32 twins and the FP32
// metrics and side geometry, rounded from the FP64 ones) and, with shock
// capturing, the sub-cell interface metrics.  Each set is allocated and
// formed the first time a parameter set needs it, so a context holds only
// what it uses.  E and S are the context's capacities (a serving pool's).
int ensure_arrays(dg_ctx* c, const dg_params* p, std::string& msg) {
  const int64_t E = c->cap_E, S = c->cap_S;
  const int64_t n3 = c->n3, n2 = c->n2;
  cudaStream_t st = c->pool_stream ? c->pool_stream : c->stream;
  // one set of arrays, all or nothing: on any failure the set's arrays are
  // freed again and its pointers stay null, so a later call starts afresh
  struct Want {
    void** slot;
    size_t bytes;
  };
  auto take = [&](const std::vector<Want>& set) -> cudaError_t {
    std::vector<void*> got;
    cudaError_t e = cudaSuccess;
    for (const Want& w : set) {
      void* q = nullptr;
      e = c->pool_stream ? pool_alloc(&q, w.bytes, c->pool_stream) : cudaMalloc(&q, w.bytes);
      if (e != cudaSuccess) break;
      got.push_back(q);
    }
    if (e != cudaSuccess) {
      for (void* q : got) dfree(c, q);
      return e;
    }
    size_t i = 0;
    for (const Want& w : set) {
      *w.slot = got[i++];
      c->bytes += (int64_t)w.bytes;
    }
    return cudaSuccess;
  };
  cudaError_t e = cudaSuccess;
  if (p->precision == DG_FP64 && !c->g) {
    std::vector<Want> set = {{(void**)&c->g, sizeof(double) * E * 12 * n3},
                             {(void**)&c->lflux, sizeof(double) * S * 12 * n2},
                             {(void**)&c->fstar, sizeof(double) * S * 5 * n2}};
    if (c->gauss) set.push_back({(void**)&c->gfc, sizeof(double) * S * 2 * 12 * n2});
    e = take(set);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->g, 0, sizeof(double) * E * 12 * n3, st);
  }
  if (e == cudaSuccess && p->precision == DG_FP32_BULK && !c->g32) {
    std::vector<Want> set = {{(void**)&c->g32, sizeof(float) * E * 12 * n3},
                             {(void**)&c->metric32, sizeof(float) * E * 10 * n3},
                             {(void**)&c->lflux32, sizeof(float) * S * 12 * n2},
                             {(void**)&c->fstar32, sizeof(float) * S * 5 * n2},
                             {(void**)&c->nrm32, sizeof(float) * S * 7 * n2}};
    if (c->gauss) set.push_back({(void**)&c->gfc32, sizeof(float) * S * 2 * 12 * n2});
    // face data of the two-kernel stage: periodic LGL meshes of a single context
    if (fused_eligible(c)) {
      set.push_back({(void**)&c->tr32, sizeof(float) * S * 2 * n2 * 8});
      set.push_back({(void**)&c->pfv32, sizeof(float) * S * 2 * n2 * 4});
      set.push_back({(void**)&c->qs32, sizeof(float) * S * n2 * 4});
      set.push_back({(void**)&c->wv32, sizeof(float) * E * 12 * n3});
    }
    e = take(set);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->g32, 0, sizeof(float) * E * 12 * n3, st);
    if (e == cudaSuccess) e = launch_fp32_geometry(c, st);
  }
  if (e == cudaSuccess && p->shock_capturing && !c->fvmetric) {
    e = take({{(void**)&c->fvmetric, sizeof(double) * E * 3 * (c->n - 1) * 3 * n2}});  // one array
    if (e == cudaSuccess) e = launch_fv_metrics(c, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    msg = std::string("working arrays: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
  }
  return DG_OK;
}

// Carpenter-Kennedy RK4(3)5 2N-storage coefficients (Sec. 2.2 cites them)
static const double RKA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                              -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double RKB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                              1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                              2277821191437.0 / 14882151754819.0};
// stage times t_n + c_s dt
static const double RKC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363218457.0,
                              2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

__global__ void k_set_scalars(DevScalars* s, double dt_fixed, int set_t, double t, int reset_flags,
                              double t_end = 0.0) {
  s->dt_fixed = dt_fixed;
  s->t_end = t_end;
  if (set_t) s->t = t;
  if (reset_flags) s->nonfinite = 0, s->timeout = 0;
}
// saves (restore = 0) or restores (restore = 1) the reference state of the
// shifted primitives around a dg_rhs of another state
__global__ void k_keep_refs(DevScalars* s, int restore) {
  double* r[5] = {&s->ref_p, &s->ref_H, &s->ref_T, &s->ref_rho, &s->ref_E};
  float* f[3] = {&s->f_ref_p, &s->f_ref_H, &s->f_ref_T};
  for (int k = 0; k < 5; ++k) {
    if (restore) *r[k] = s->keep_ref[k];
    else s->keep_ref[k] = *r[k];
  }
  for (int k = 0; k < 3; ++k) {
    if (restore) *f[k] = s->keep_f_ref[k];
    else s->keep_f_ref[k] = *f[k];
  }
}
__global__ void k_clear_timeout(DevScalars* s) { s->timeout = 0; }
__global__ void k_zero_kin(DevScalars* s) {
  s->kin[0] = s->kin[1] = s->kin[2] = s->kin[3] = 0.0;
  s->lam_c = 0ull;
  s->lam_v = 0ull;
}
static void destroy_graph(dg_ctx* c) {
  if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
  c->step_graph = nullptr;
  c->step_graph_kind = -1;
}

static int check_params(const dg_params* p) {
  if (!p) return fail(DG_ERR_ARG, "params is NULL");
  if (!(p->gamma > 1.0) || !(p->R > 0) || !(p->Pr > 0) || !(p->mu >= 0) || !(p->cfl > 0) || !(p->dfl > 0))
    return fail(DG_ERR_ARG, "invalid physical parameters");
  if (p->riemann != DG_RIEMANN_ROE && p->riemann != DG_RIEMANN_LF) return fail(DG_ERR_ARG, "unknown Riemann solver");
  if (p->precision != DG_FP64 && p->precision != DG_FP32_BULK) return fail(DG_ERR_ARG, "unknown precision");
  if (p->sutherland && !(p->T_ref > 0)) return fail(DG_ERR_ARG, "Sutherland's law needs T_ref > 0");
  if (p->source != DG_SOURCE_NONE && p->source != DG_SOURCE_MMS) return fail(DG_ERR_ARG, "unknown source");
  if (p->source && p->sutherland)
    return fail(DG_ERR_ARG, "the manufactured-solution source is written for a constant viscosity");
  if (p->source && !std::isfinite(p->source_A + p->source_a)) return fail(DG_ERR_ARG, "source parameters");
  return DG_OK;
}

}  // namespace dg

using namespace dg;

extern "C" {

void dg_default_params(dg_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->gamma = 1.4;
  p->R = 1.0;
  p->Pr = 0.72;
  p->mu = 1.0 / 1600.0;
  p->riemann = DG_RIEMANN_ROE;
  p->viscous = 1;
  p->shock_capturing = 0;
  p->alpha_min = 1e-3;
  p->alpha_max = 0.5;
  p->cfl = 0.9;
  p->dfl = 0.9;
  p->precision = DG_FP64;
  p->alpha_force = -1.0;
  p->sutherland = 0;
  p->T_ref = 1.0;
  p->source = DG_SOURCE_NONE;
  p->source_A = 0.1;
  p->source_a = 1.0;
}

const char* dg_error_string(int code) {
  switch (code) {
    case DG_OK: return "ok";
    case DG_ERR_ARG: return "invalid argument";
    case DG_ERR_MESH: return "invalid mesh";
    case DG_ERR_OOM: return "out of device memory";
    case DG_ERR_CUDA: return "CUDA error";
    case DG_ERR_NONFINITE: return "non-finite value in the solution";
    case DG_ERR_TIMEOUT: return "device-side wait timed out";
    case DG_ERR_STATE: return "invalid call for the context's state";
    case DG_PENDING: return "pending";
    default: return "unknown error";
  }
}

const char* dg_last_error(void) { return g_last_error.c_str(); }

int64_t dg_launch_count(void) { return g_launches.load(); }

void dg_destroy(dg_ctx* c) {
  if (!c) return;
  destroy_graph(c);
  dfree(c, c->U);
  dfree(c, c->dU);
  dfree(c, c->Ut);
  dfree(c, c->Upub);
  dfree(c, c->metric);
  dfree(c, c->metric32);
  dfree(c, c->g);
  dfree(c, c->nrm);
  dfree(c, c->nrm32);
  dfree(c, c->lflux);
  dfree(c, c->fstar);
  dfree(c, c->g32);
  dfree(c, c->lflux32);
  dfree(c, c->fstar32);
  dfree(c, c->alpha);
  dfree(c, c->fvmetric);
  dfree(c, c->cflgeo);
  dfree(c, c->elem_side);
  dfree(c, c->elem_case);
  dfree(c, c->side_case);
  dfree(c, c->elem_list);
  dfree(c, c->side_list);
  dfree(c, c->side_e);
  dfree(c, c->side_f);
  dfree(c, c->side_bc);
  dfree(c, c->bcdata);
  dfree(c, c->sponge_sigma);
  dfree(c, c->sponge_base);
  dfree(c, c->xyzs);
  dfree(c, c->Ufc);
  dfree(c, c->gfc);
  dfree(c, c->gfc32);
  dfree(c, c->tr32);
  dfree(c, c->pfv32);
  dfree(c, c->qs32);
  dfree(c, c->wv32);
  dfree(c, c->ops);
  dfree(c, c->scal);
  dfree(c, c->kin_part);
  if (c->scal_host) cudaFreeHost(c->scal_host);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

}  // extern "C"

namespace dg {

// A serving pool: the arrays of a context sized for capE elements and 3 capE
// sides, every slot free (case maps -1, other arrays zero), no mesh yet.
int create_pool_ctx(dg_ctx** out, int N, int64_t capE, const dg_params* params, cudaStream_t stream,
                    std::string& msg) {
  *out = nullptr;
  dg_ctx* c = new dg_ctx();
  cudaGetDevice(&c->device);
  c->stream = stream;
  c->prm = *params;
  c->N = N;
  c->n = N + 1;
  c->n2 = c->n * c->n;
  c->n3 = c->n2 * c->n;
  c->E = 0;
  c->S = 0;
  const int64_t E = capE, S = 3 * capE, n3 = c->n3, n2 = c->n2;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(dalloc(c, &c->U, E * 5 * n3));
  A(dalloc(c, &c->dU, E * 5 * n3));
  A(dalloc(c, &c->Ut, E * 5 * n3));
  A(dalloc(c, &c->Upub, E * 5 * n3));
  A(dalloc(c, &c->metric, E * 10 * n3));
  A(dalloc(c, &c->alpha, E));
  A(dalloc(c, &c->cflgeo, E * 4 * n3));
  A(dalloc(c, &c->elem_side, E * 6));
  A(dalloc(c, &c->elem_case, E));
  A(dalloc(c, &c->nrm, S * 4 * n2));
  A(dalloc(c, &c->side_e, S));
  A(dalloc(c, &c->side_f, S));
  A(dalloc(c, &c->side_case, S));
  A(dalloc(c, &c->side_bc, S));
  A(dalloc(c, &c->ops, 1));
  A(dalloc(c, &c->scal, 1));
  if (e == cudaSuccess) e = cudaMallocHost(&c->scal_host, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = init_kernel_attributes(N);
  if (e == cudaSuccess) {
    Ops ops;
    build_ops(N, 0, ops);
    A(cudaMemcpyAsync(c->ops, &ops, sizeof(Ops), cudaMemcpyHostToDevice, stream));
    A(cudaMemsetAsync(c->scal, 0, sizeof(DevScalars), stream));
    A(cudaMemsetAsync(c->U, 0, sizeof(double) * E * 5 * n3, stream));
    A(cudaMemsetAsync(c->dU, 0, sizeof(double) * E * 5 * n3, stream));
    A(cudaMemsetAsync(c->metric, 0, sizeof(double) * E * 10 * n3, stream));
    A(cudaMemsetAsync(c->cflgeo, 0, sizeof(double) * E * 4 * n3, stream));
    A(cudaMemsetAsync(c->elem_side, 0, sizeof(int) * E * 6, stream));
    A(cudaMemsetAsync(c->side_e, 0, sizeof(int2) * S, stream));
    A(cudaMemsetAsync(c->side_f, 0, sizeof(int) * S, stream));
    A(cudaMemsetAsync(c->nrm, 0, sizeof(double) * S * 4 * n2, stream));
    A(cudaMemsetAsync(c->elem_case, 0xff, sizeof(int) * E, stream));
    A(cudaMemsetAsync(c->side_case, 0xff, sizeof(int) * S, stream));
    A(cudaMemsetAsync(c->side_bc, 0xff, sizeof(int) * S, stream));
    A(cudaStreamSynchronize(stream));
  }
  c->cap_E = E;
  c->cap_S = S;
  if (e == cudaSuccess) {
    // the working arrays of the pool's precision (the geometry is all zero here)
    std::string m2;
    const int st = ensure_arrays(c, params, m2);
    if (st != DG_OK) {
      msg = "pool allocation: " + m2;
      dg_destroy(c);
      return st;
    }
  }
  if (e != cudaSuccess) {
    msg = std::string("pool allocation: ") + cudaGetErrorString(e);
    const int code = e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
    dg_destroy(c);
    return code;
  }
  c->state_set = true;
  *out = c;
  return DG_OK;
}

// pool_stream non-null: a context for the server's cases, whose device
// arrays come from the library pool in that stream's order and which has no
// pinned mirror or capture stream (it is only built, loaded and copied from)
int init_mesh_impl(dg_ctx** out, const dg_mesh_desc* mesh, const dg_params* params, cudaStream_t stream,
                   cudaStream_t pool_stream) {
  if (!out) return fail(DG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!mesh || !mesh->corner_vid || !mesh->xyz) return fail(DG_ERR_ARG, "mesh description incomplete");
  if (mesh->N < 1 || mesh->N > NMAX) return fail(DG_ERR_ARG, "N must be in [1, 7]");
  if (mesh->n_elems < 1 || mesh->n_elems > (int64_t)1 << 26) return fail(DG_ERR_ARG, "bad element count");
  if (mesh->face_bc) {
    if (mesh->n_bc < 1 || mesh->n_bc > 64 || !mesh->bc) return fail(DG_ERR_ARG, "face_bc needs 1..64 condition rows");
    for (int k = 0; k < mesh->n_bc; ++k) {
      const int type = (int)mesh->bc[k * 9];
      if (type < DG_BC_WALL_ISOTHERMAL || type > DG_BC_OUTFLOW || (double)type != mesh->bc[k * 9])
        return fail(DG_ERR_ARG, "unknown boundary-condition type");
      if (type == DG_BC_WALL_ISOTHERMAL && !(mesh->bc[k * 9 + 4] > 0)) return fail(DG_ERR_ARG, "wall temperature must be > 0");
      if (type == DG_BC_STATE && !(mesh->bc[k * 9 + 1] > 0)) return fail(DG_ERR_ARG, "prescribed density must be > 0");
      if (type == DG_BC_OUTFLOW && !(mesh->bc[k * 9 + 1] > 0)) return fail(DG_ERR_ARG, "outflow pressure must be > 0");
    }
    for (int64_t a = 0; a < 6 * mesh->n_elems; ++a)
      if (mesh->face_bc[a] < 0 || mesh->face_bc[a] > mesh->n_bc) return fail(DG_ERR_ARG, "face_bc out of range");
  }
  if (mesh->nodes != DG_NODES_LGL && mesh->nodes != DG_NODES_GAUSS) return fail(DG_ERR_ARG, "unknown node set");
  int st = check_params(params);
  if (st != DG_OK) return st;
  if (mesh->nodes == DG_NODES_GAUSS && params->shock_capturing)
    return fail(DG_ERR_ARG, "shock capturing needs LGL nodes (the sub-cell FV scheme lives on the LGL sub-cells)");
  dg_ctx* c = new dg_ctx();
  cudaGetDevice(&c->device);
  c->stream = stream;
  c->pool_stream = pool_stream;
  c->gauss = mesh->nodes == DG_NODES_GAUSS;
  c->prm = *params;
  c->N = mesh->N;
  c->n = c->N + 1;
  c->n2 = c->n * c->n;
  c->n3 = c->n2 * c->n;
  c->E = mesh->n_elems;
  const int64_t E = c->E, n3 = c->n3;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(dalloc(c, &c->U, E * 5 * n3));
  A(dalloc(c, &c->dU, E * 5 * n3));
  A(dalloc(c, &c->Ut, E * 5 * n3));
  A(dalloc(c, &c->Upub, E * 5 * n3));
  A(dalloc(c, &c->metric, E * 10 * n3));
  A(dalloc(c, &c->alpha, E));
  A(dalloc(c, &c->cflgeo, E * 4 * n3));
  A(dalloc(c, &c->elem_side, E * 6));
  A(dalloc(c, &c->xyzs, E * n3 * 3));
  A(dalloc(c, &c->ops, 1));
  A(dalloc(c, &c->scal, 1));
  if (e == cudaSuccess && !pool_stream) e = cudaMallocHost(&c->scal_host, sizeof(DevScalars));
  if (e == cudaSuccess && !pool_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    int r = cuda_fail(e, "allocation");
    dg_destroy(c);
    return r;
  }
  if (e == cudaSuccess) e = init_kernel_attributes(c->N);
  Ops ops;
  build_ops(c->N, c->gauss, ops);
  A(cudaMemcpyAsync(c->ops, &ops, sizeof(Ops), cudaMemcpyHostToDevice, c->stream));
  A(cudaMemsetAsync(c->scal, 0, sizeof(DevScalars), c->stream));
  A(cudaMemsetAsync(c->alpha, 0, sizeof(double) * E, c->stream));
  A(cudaStreamSynchronize(c->stream));
  if (e != cudaSuccess) {
    int r = cuda_fail(e, "initialisation");
    dg_destroy(c);
    return r;
  }
  std::string msg;
  if (mesh->face_bc) {
    c->n_bc = mesh->n_bc;
    e = dalloc(c, &c->bcdata, (size_t)9 * mesh->n_bc);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->bcdata, mesh->bc, sizeof(double) * 9 * mesh->n_bc, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      int r = cuda_fail(e, "boundary conditions");
      dg_destroy(c);
      return r;
    }
  }
  st = build_mesh(c, mesh->corner_vid, mesh->xyz, mesh->face_bc, msg);
  if (st == DG_OK) {
    c->cap_E = c->E;
    c->cap_S = c->S;
    st = ensure_arrays(c, &c->prm, msg);
  }
  if (st != DG_OK) {
    dg_destroy(c);
    return fail(st, msg);
  }
  *out = c;
  return DG_OK;
}

}  // namespace dg

extern "C" {

int dg_init_mesh(dg_ctx** out, const dg_mesh_desc* mesh, const dg_params* params, void* stream) {
  return dg::init_mesh_impl(out, mesh, params, (cudaStream_t)stream, nullptr);
}

int dg_selftest_convert(const double* in, float* out, double* back, int64_t n, void* stream) {
  if (!in || !out || !back || n < 0 || n > ((int64_t)1 << 40)) return fail(DG_ERR_ARG, "bad buffers or size");
  cudaError_t e = launch_convert_check(in, out, back, n, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "dg_selftest_convert");
  return DG_OK;
}

int dg_quadrature_weights(const dg_ctx* c, double* w) {
  if (!c || !w) return fail(DG_ERR_ARG, "ctx or w is NULL");
  Ops o;
  build_ops(c->N, c->gauss, o);
  for (int i = 0; i <= c->N; ++i) w[i] = o.w[i];
  return DG_OK;
}

int dg_node_coords(dg_ctx* c, double* xyz, int on_device) {
  if (!c || !xyz) return fail(DG_ERR_ARG, "ctx or xyz is NULL");
  if (!c->xyzs) return fail(DG_ERR_STATE, "the context has no mesh of its own");
  cudaError_t e = cudaMemcpyAsync(xyz, c->xyzs, sizeof(double) * c->E * c->n3 * 3,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dg_node_coords");
  return DG_OK;
}

int dg_set_stream(dg_ctx* c, void* stream) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  c->stream = (cudaStream_t)stream;
  return DG_OK;
}

int dg_set_params(dg_ctx* c, const dg_params* p) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  int st = check_params(p);
  if (st != DG_OK) return st;
  if (c->gauss && p->shock_capturing)
    return fail(DG_ERR_ARG, "shock capturing needs LGL nodes (the sub-cell FV scheme lives on the LGL sub-cells)");
  {
    std::string msg;
    const int sa = ensure_arrays(c, p, msg);  // a new precision's working arrays, or the FV metrics
    if (sa != DG_OK) return fail(sa, msg);
  }
  c->prm = *p;
  destroy_graph(c);
  c->traces_valid = false;
  if (c->state_set) {
    cudaError_t e = launch_refs(c);
    if (e != cudaSuccess) return cuda_fail(e, "dg_set_params");
  }
  return DG_OK;
}

int dg_sizes(const dg_ctx* c, int* N, int64_t* E, int64_t* S, int64_t* bytes) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (N) *N = c->N;
  if (E) *E = c->E;
  if (S) *S = c->S;
  if (bytes) *bytes = c->bytes;
  return DG_OK;
}

// the device address of pinned (page-locked) host memory, or null for
// other memory: pinned host arrays are read and written by the layout
// conversion kernels directly over the host link, without a staging copy
static void* pinned_device_address(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int dg_set_state(dg_ctx* c, const double* U, int on_device, double t) {
  if (!c || !U) return fail(DG_ERR_ARG, "ctx or U is NULL");
  const size_t bytes = sizeof(double) * c->E * 5 * c->n3;
  cudaError_t e = cudaSuccess;
  const double* src = U;
  if (!on_device) {
    const double* mapped = static_cast<const double*>(pinned_device_address(U));
    if (mapped) {
      src = mapped;
    } else {
      e = cudaMemcpyAsync(c->Upub, U, bytes, cudaMemcpyHostToDevice, c->stream);
      src = c->Upub;
    }
  }
  if (e == cudaSuccess) e = launch_to_internal(c, src, c->U);
  if (e == cudaSuccess) e = launch_refs(c);
  if (e == cudaSuccess) {
    k_set_scalars<<<1, 1, 0, c->stream>>>(c->scal, 0.0, 1, t, 1);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->stream);
  c->traces_valid = false;
  if (e != cudaSuccess) return cuda_fail(e, "dg_set_state");
  c->t_host = t;
  c->state_set = true;
  return DG_OK;
}

int dg_get_state(dg_ctx* c, double* U, int on_device, double* t) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (!c->scal_host) return fail(DG_ERR_STATE, "internal case context: no host mirror");
  const size_t bytes = sizeof(double) * c->E * 5 * c->n3;
  cudaError_t e = cudaSuccess;
  if (U) {
    double* mapped = on_device ? nullptr : static_cast<double*>(pinned_device_address(U));
    if (on_device || mapped) {
      e = launch_to_public(c, c->U, on_device ? U : mapped);
    } else {
      e = launch_to_public(c, c->U, c->Upub);
      if (e == cudaSuccess) e = cudaMemcpyAsync(U, c->Upub, bytes, cudaMemcpyDeviceToHost, c->stream);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->scal_host, c->scal, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dg_get_state");
  c->t_host = c->scal_host->t;
  if (t) *t = c->t_host;
  if (c->scal_host->timeout) return fail(DG_ERR_TIMEOUT, "a persistent step's grid-wide wait ran out");
  if (c->scal_host->nonfinite) return fail(DG_ERR_NONFINITE, "a time step met a non-finite value");
  return DG_OK;
}

int dg_rhs(dg_ctx* c, const double* U_dev, double* Ut_dev) {
  if (!c || !Ut_dev) return fail(DG_ERR_ARG, "ctx or Ut is NULL");
  if (!U_dev && !c->state_set) return fail(DG_ERR_STATE, "no state set");
  cudaError_t e = cudaSuccess;
  const double* Uin = c->U;
  if (U_dev) {
    // the RK register is free between steps: use it for the internal copy
    e = launch_to_internal(c, U_dev, c->dU);
    Uin = c->dU;
  }
  // reference state of the shifted primitives taken from the evaluated state
  // (any constant is exact; this one keeps the FP32-bulk rounding small); the
  // context's own is kept and put back, so later steps are unchanged
  if (e == cudaSuccess && U_dev && c->state_set) {
    k_keep_refs<<<1, 1, 0, c->stream>>>(c->scal, 0);
    count_launch();
    e = cudaGetLastError();
  }
  if (U_dev) {  // the context's own state keeps the reference it was set with
    double* Ukeep = c->U;
    c->U = const_cast<double*>(Uin);
    if (e == cudaSuccess) e = launch_refs(c);
    c->U = Ukeep;
  }
  if (e == cudaSuccess) e = launch_rhs(c, Uin, 0, 0.0, 0.0, 0);
  if (e == cudaSuccess) e = launch_to_public(c, c->Ut, Ut_dev);
  if (e == cudaSuccess && U_dev && c->state_set) {
    k_keep_refs<<<1, 1, 0, c->stream>>>(c->scal, 1);
    count_launch();
    e = cudaGetLastError();
  }
  c->traces_valid = false;
  if (e != cudaSuccess) return cuda_fail(e, "dg_rhs");
  return DG_OK;
}

static cudaError_t enqueue_step(dg_ctx* c) {
  // two-kernel FP32-bulk steps take the radii of their state from the
  // previous step's last stage, whose epilogue reduces those of the state
  // it writes; otherwise the CFL reduction reads the state
  const bool fcfl = cfl_fused(c);
  cudaError_t e = fcfl ? launch_dt_next(c) : launch_cfl(c, false);
  const bool own = c->rk_ns > 0;
  const int ns = own ? c->rk_ns : 5;
  if (e == cudaSuccess && persist_active(c)) {
    // every stage in one persistent launch
    return launch_persist(c, ns, own ? c->rk_a : RKA, own ? c->rk_b : RKB, own ? c->rk_c : RKC);
  }
  for (int s = 0; s < ns && e == cudaSuccess; ++s) {
    c->stage_c = own ? c->rk_c[s] : RKC[s];
    c->stage_cfl = fcfl && s == ns - 1;
    e = launch_rhs(c, c->U, 1, own ? c->rk_a[s] : RKA[s], own ? c->rk_b[s] : RKB[s], s == 0);
  }
  c->stage_c = 0.0;
  c->stage_cfl = 0;
  return e;
}

// captures the whole time step once (CFL reduction + 5 stages)
static cudaError_t ensure_step_graph(dg_ctx* c) {
  cudaError_t e = cudaSuccess;
  if (!c->step_graph) {
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = enqueue_step(c);
      e = cudaStreamEndCapture(c->cap_stream, &graph);
      if (e == cudaSuccess) e = le;
    }
    c->stream = user;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->step_graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) c->step_graph = nullptr;
  }
  return e;
}

// the two-kernel FP32-bulk stage reads the face data of the step's state:
// formed here when no step left them behind
// (and, when the steps take their time step from the previous step's last
// stage, the CFL radii of the state: the face-data pass reduces them too)
static cudaError_t ensure_face_data(dg_ctx* c) {
  if (!fused_active(c)) return cudaSuccess;
  const bool fcfl = cfl_fused(c);
  if (c->traces_valid && (!fcfl || c->lam_next_valid)) return cudaSuccess;
  cudaError_t e = fcfl ? launch_clear_next(c) : cudaSuccess;
  c->stage_cfl = fcfl;
  if (e == cudaSuccess) e = launch_fprep(c, c->U);
  c->stage_cfl = 0;
  if (e == cudaSuccess) {
    c->traces_valid = true;
    c->lam_next_valid = fcfl;
  }
  return e;
}

static cudaError_t launch_steps(dg_ctx* c, int64_t n_steps) {
  cudaError_t e = ensure_step_graph(c);
  if (e == cudaSuccess) e = ensure_face_data(c);
  if (e != cudaSuccess) return e;
  for (int64_t i = 0; i < n_steps && e == cudaSuccess; ++i) {
    e = cudaGraphLaunch(c->step_graph, c->stream);
    const int per_stage = fused_active(c) ? 2 : (c->prm.viscous ? 4 : 2);
    count_launch(persist_active(c) ? 3 : (cfl_fused(c) ? 1 : 2) + (c->rk_ns > 0 ? c->rk_ns : 5) * per_stage);
  }
  // a persistent step leaves the face data of its state but not its radii
  if (!cfl_fused(c)) c->lam_next_valid = false;
  return e;
}

int dg_step(dg_ctx* c, int n_steps, double dt, double* t_out) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (!c->state_set) return fail(DG_ERR_STATE, "no state set");
  if (!c->cap_stream) return fail(DG_ERR_STATE, "internal case context: no capture stream");
  if (n_steps < 0) return fail(DG_ERR_ARG, "n_steps < 0");
  cudaError_t e = cudaSuccess;
  if (n_steps > 0) {
    k_set_scalars<<<1, 1, 0, c->stream>>>(c->scal, dt > 0 ? dt : 0.0, 0, 0.0, 0);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_steps(c, n_steps);
  }
  if (e == cudaSuccess && t_out) {
    // the time reached, read back through the pinned mirror
    e = cudaMemcpyAsync(c->scal_host, c->scal, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "dg_step");
  if (t_out) {
    c->t_host = c->scal_host->t;
    *t_out = c->t_host;
    if (c->scal_host->timeout) return fail(DG_ERR_TIMEOUT, "a persistent step's grid-wide wait ran out");
    if (c->scal_host->nonfinite) return fail(DG_ERR_NONFINITE, "a time step met a non-finite value");
  }
  return DG_OK;
}

int dg_advance(dg_ctx* c, double t_end, int64_t max_steps, double* t_out, int64_t* steps_out) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (!c->state_set) return fail(DG_ERR_STATE, "no state set");
  if (!(t_end > 0) || !std::isfinite(t_end)) return fail(DG_ERR_ARG, "t_end must be finite and > 0");
  if (max_steps < 0) return fail(DG_ERR_ARG, "max_steps < 0");
  DevScalars* h = c->scal_host;
  if (!h) return fail(DG_ERR_STATE, "internal case context: no host mirror");
  auto read_back = [&]() {
    cudaError_t r = cudaMemcpyAsync(h, c->scal, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream);
    if (r == cudaSuccess) r = cudaStreamSynchronize(c->stream);
    return r;
  };
  k_set_scalars<<<1, 1, 0, c->stream>>>(c->scal, 0.0, 0, 0.0, 0, t_end);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = read_back();
  const long long steps0 = h->steps;
  int64_t launched = 0;
  double dt_last = 0.0;
  while (e == cudaSuccess && h->t < t_end && launched < max_steps && !h->nonfinite && !h->timeout) {
    // a batch that ends just short of t_end at the last step's size; the
    // last few steps go one at a time
    int64_t K = 1;
    if (dt_last > 0) K = std::max<int64_t>(1, (int64_t)(0.95 * (t_end - h->t) / dt_last));
    K = std::min<int64_t>(K, max_steps - launched);
    e = launch_steps(c, K);
    launched += K;
    if (e == cudaSuccess) e = read_back();
    dt_last = h->dt;
  }
  // later dg_step calls take no end time
  if (e == cudaSuccess) {
    k_set_scalars<<<1, 1, 0, c->stream>>>(c->scal, 0.0, 0, 0.0, 0, 0.0);
    count_launch();
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(e, "dg_advance");
  c->t_host = h->t;
  if (t_out) *t_out = h->t;
  if (steps_out) *steps_out = (int64_t)(h->steps - steps0);
  if (h->timeout) return fail(DG_ERR_TIMEOUT, "a persistent step's grid-wide wait ran out");
  if (h->nonfinite) return fail(DG_ERR_NONFINITE, "a time step met a non-finite value");
  return DG_OK;
}

int dg_profile_step(dg_ctx* c, int n_steps, double dt, double* ms, int64_t* launches) {
  if (!c || !ms || !launches) return fail(DG_ERR_ARG, "NULL argument");
  if (!c->state_set) return fail(DG_ERR_STATE, "no state set");
  if (!c->cap_stream) return fail(DG_ERR_STATE, "internal case context: no capture stream");
  Profiler* p = new Profiler();
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < Profiler::MAX_EV && e == cudaSuccess; ++i) {
    e = cudaEventCreate(&p->ev[i][0]);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev[i][1]);
  }
  if (e == cudaSuccess) {
    k_set_scalars<<<1, 1, 0, c->stream>>>(c->scal, dt > 0 ? dt : 0.0, 0, 0.0, 0);
    count_launch();
    e = ensure_face_data(c);
    c->prof = p;
    for (int s = 0; s < n_steps && e == cudaSuccess; ++s) {
      p->used = 0;
      e = enqueue_step(c);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      for (int k = 0; k < p->used && e == cudaSuccess; ++k) {
        float t = 0;
        e = cudaEventElapsedTime(&t, p->ev[k][0], p->ev[k][1]);
        p->ms[p->slot[k]] += t;
        p->launches[p->slot[k]] += 1;
      }
    }
    c->prof = nullptr;
  }
  for (int k = 0; k < 5; ++k) {
    ms[k] = p->ms[k];
    launches[k] = p->launches[k];
  }
  for (int i = 0; i < Profiler::MAX_EV; ++i) {
    if (p->ev[i][0]) cudaEventDestroy(p->ev[i][0]);
    if (p->ev[i][1]) cudaEventDestroy(p->ev[i][1]);
  }
  delete p;
  if (e != cudaSuccess) return cuda_fail(e, "dg_profile_step");
  return DG_OK;
}

int dg_set_rk(dg_ctx* c, int n_stages, const double* A, const double* B, const double* cc) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (!A) {
    c->rk_ns = 0;
    destroy_graph(c);
    return DG_OK;
  }
  if (!B || !cc || n_stages < 1 || n_stages > 32) return fail(DG_ERR_ARG, "1..32 stages with A, B and c");
  if (A[0] != 0.0) return fail(DG_ERR_ARG, "A[0] must be 0");
  for (int s = 0; s < n_stages; ++s)
    if (!std::isfinite(A[s]) || !std::isfinite(B[s]) || !std::isfinite(cc[s]))
      return fail(DG_ERR_ARG, "non-finite coefficient");
  for (int s = 0; s < n_stages; ++s) {
    c->rk_a[s] = A[s];
    c->rk_b[s] = B[s];
    c->rk_c[s] = cc[s];
  }
  c->rk_ns = n_stages;
  destroy_graph(c);  // the step graph holds the stages
  return DG_OK;
}

// Niegemann, Diehl and Busch's fourteen-stage fourth-order 2N-storage scheme
// (Sec. 2.2 cites it; Sec. 6 runs the application with it), as published
static const double NDB14_A[14] = {0.0, -0.7188012108672410, -0.7785331173421570, -0.0053282796654044,
                                   -0.8552979934029281, -3.9564138245774565, -1.5780575380587385,
                                   -2.0837094552574054, -0.7483334182761610, -0.7032861106563359,
                                   0.0013917096117681, -0.0932075369637460, -0.9514200470875948,
                                   -7.1151571693922548};
static const double NDB14_B[14] = {0.0367762454319673, 0.3136296607553959, 0.1531848691869027,
                                   0.0030097086818182, 0.3326293790646110, 0.2440251405350864,
                                   0.3718879239592277, 0.6204126221582444, 0.1524043173028741,
                                   0.0760894927419266, 0.0077604214040978, 0.0024647284755382,
                                   0.0780348340049386, 5.5059777270269628};
static const double NDB14_C[14] = {0.0, 0.0367762454319673, 0.1249685262725025, 0.2446177702277698,
                                   0.2476149531070420, 0.2969311120382472, 0.3978149645802642,
                                   0.5270854589440328, 0.6981269994175695, 0.8190890835352128,
                                   0.8527059887098624, 0.8604711817462826, 0.8627060376969976,
                                   0.8734213127600976};

int dg_set_rk_scheme(dg_ctx* c, int scheme) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (scheme == DG_RK_CK5) return dg_set_rk(c, 0, nullptr, nullptr, nullptr);
  if (scheme == DG_RK_NDB14) return dg_set_rk(c, 14, NDB14_A, NDB14_B, NDB14_C);
  return fail(DG_ERR_ARG, "unknown scheme (DG_RK_CK5 or DG_RK_NDB14)");
}

int dg_set_sponge(dg_ctx* c, const double* sigma, const double* U_base) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (!c->cap_stream) return fail(DG_ERR_STATE, "internal case context");
  destroy_graph(c);  // the step graph captures the sponge arrays
  if (!sigma) {
    cudaStreamSynchronize(c->stream);
    dfree(c, c->sponge_sigma);
    dfree(c, c->sponge_base);
    c->sponge_sigma = c->sponge_base = nullptr;
    return DG_OK;
  }
  if (!U_base) return fail(DG_ERR_ARG, "U_base is NULL");
  const int64_t nn = c->E * c->n3;
  for (int64_t i = 0; i < nn; ++i)
    if (!(sigma[i] >= 0) || !std::isfinite(sigma[i])) return fail(DG_ERR_ARG, "sigma must be finite and >= 0");
  cudaError_t e = cudaSuccess;
  if (!c->sponge_sigma) e = dalloc(c, &c->sponge_sigma, nn);
  if (e == cudaSuccess && !c->sponge_base) e = dalloc(c, &c->sponge_base, nn * 5);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->sponge_sigma, sigma, sizeof(double) * nn, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->Upub, U_base, sizeof(double) * nn * 5, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = launch_to_internal(c, c->Upub, c->sponge_base);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    // no half-set sponge: the kernels read the base state whenever sigma is set
    cudaStreamSynchronize(c->stream);
    dfree(c, c->sponge_sigma);
    dfree(c, c->sponge_base);
    c->sponge_sigma = c->sponge_base = nullptr;
    return cuda_fail(e, "dg_set_sponge");
  }
  return DG_OK;
}

static void variants_of(int N, int& D, bool& lift2, bool& vol2) {
  const int n3 = (N + 1) * (N + 1) * (N + 1);
  D = n3 >= 256 ? 1 : 256 / n3;
  lift2 = 2 * D * n3 <= 1024;
  vol2 = 2 * D * n3 <= 512;
}

int dg_autotune(dg_ctx* c, int* config, double* ms) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (!c->state_set) return fail(DG_ERR_STATE, "no state set");
  if (c->gauss) return fail(DG_ERR_STATE, "the Gauss-Legendre kernels have one launch configuration");
  double t[8];
  cudaError_t e = launch_autotune(c, t);
  c->traces_valid = false;  // the tuner's runs write the face arrays
  if (e != cudaSuccess) return cuda_fail(e, "dg_autotune");
  destroy_graph(c);  // the next step captures the chosen variants
  if (config) dg_get_config(c, config);
  if (ms) memcpy(ms, t, sizeof(t));
  return DG_OK;
}

int dg_set_config(dg_ctx* c, const int* config) {
  if (!c || !config) return fail(DG_ERR_ARG, "ctx or config is NULL");
  int D;
  bool lift2, vol2;
  variants_of(c->N, D, lift2, vol2);
  const int le = config[0], ve = config[1], pr = config[2], sb = config[3], sf = config[4], pf = config[5];
  const int ps = config[6];
  if (!(le == 0 || le == D || (lift2 && le == 2 * D))) return fail(DG_ERR_ARG, "lift elements per block");
  if (!(ve == 0 || ve == D || (vol2 && ve == 2 * D))) return fail(DG_ERR_ARG, "volume elements per block");
  if (!(pr == -1 || pr == 0 || pr == 1)) return fail(DG_ERR_ARG, "volume mapping");
  if (pr == 1 && c->prm.precision == DG_FP32_BULK) return fail(DG_ERR_ARG, "line pairs are an FP64 mapping");
  if (!(sb == 0 || sb == 128 || sb == 256)) return fail(DG_ERR_ARG, "side block size");
  if (!(sf == 0 || sf == 1)) return fail(DG_ERR_ARG, "stage form (0: default, 1: four kernels)");
  if (!(pf == 0 || pf == 1)) return fail(DG_ERR_ARG, "prefetch (0 or 1)");
  if (!(ps == 0 || ps == 1)) return fail(DG_ERR_ARG, "launch form (0: per kernel, 1: persistent)");
  c->cfg.lift_epb = le;
  c->cfg.vol_epb = ve;
  c->cfg.vol_pairs = pr;
  c->cfg.side_block = sb == 0 ? 256 : sb;
  c->cfg.stage_form = sf;
  c->cfg.prefetch = pf;
  c->cfg.persistent = ps;
  destroy_graph(c);
  c->traces_valid = false;  // the other stage form does not keep the face data
  return DG_OK;
}

int dg_get_config(const dg_ctx* c, int* config) {
  if (!c || !config) return fail(DG_ERR_ARG, "ctx or config is NULL");
  int D;
  bool lift2, vol2;
  variants_of(c->N, D, lift2, vol2);
  config[0] = c->cfg.lift_epb > 0 ? c->cfg.lift_epb : D;
  config[1] = c->cfg.vol_epb > 0 ? c->cfg.vol_epb : D;
  config[2] = c->cfg.vol_pairs >= 0 ? c->cfg.vol_pairs : (c->prm.precision == DG_FP32_BULK ? 0 : 1);
  config[3] = c->cfg.side_block;
  config[4] = c->cfg.stage_form;
  config[5] = c->cfg.prefetch;
  config[6] = c->cfg.persistent;
  return DG_OK;
}

int dg_selftest_wait_timeout(dg_ctx* c, unsigned spin_polls) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  if (!fused_active(c)) return fail(DG_ERR_STATE, "the context does not use the two-kernel stage");
  if (!c->scal_host) return fail(DG_ERR_STATE, "internal case context: no host mirror");
  // one persistent step launch whose barriers wait for a participant that
  // does not exist; the element phase never runs, so the state is unchanged
  cudaError_t e = launch_persist(c, 5, RKA, RKB, RKC, 1u, spin_polls);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->scal_host, c->scal, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dg_selftest_wait_timeout");
  const int ran_out = c->scal_host->timeout;
  k_clear_timeout<<<1, 1, 0, c->stream>>>(c->scal);
  count_launch();
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dg_selftest_wait_timeout");
  if (ran_out) return fail(DG_ERR_TIMEOUT, "the barrier waits ran out (expected)");
  return DG_OK;
}

int dg_stage_form(const dg_ctx* c) {
  if (!c) return fail(DG_ERR_ARG, "ctx is NULL");
  return fused_active(c) ? 2 : 4;
}

int dg_time_step(dg_ctx* c, double* dt) {
  if (!c || !dt) return fail(DG_ERR_ARG, "ctx or dt is NULL");
  if (!c->state_set) return fail(DG_ERR_STATE, "no state set");
  if (!c->scal_host) return fail(DG_ERR_STATE, "internal case context: no host mirror");
  // the CFL reduction of a step, reported instead of taken
  cudaError_t e = launch_cfl(c, true);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->scal_host, c->scal, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dg_time_step");
  *dt = c->scal_host->dt_cfl;
  if (c->scal_host->nonfinite) return fail(DG_ERR_NONFINITE, "non-finite value in the state");
  return DG_OK;
}

int dg_kinetic(dg_ctx* c, double* out) {
  if (!c || !out) return fail(DG_ERR_ARG, "ctx or out is NULL");
  if (!c->state_set) return fail(DG_ERR_STATE, "no state set");
  if (!c->scal_host) return fail(DG_ERR_STATE, "internal case context: no host mirror");
  const int nb = kinetic_blocks(c);
  if (c->kin_part_blocks < nb) {
    dfree(c, c->kin_part);
    c->kin_part = nullptr;
    c->kin_part_blocks = 0;
    cudaError_t ea = dalloc(c, &c->kin_part, (int64_t)nb * 3);
    if (ea != cudaSuccess) return cuda_fail(ea, "dg_kinetic");
    c->kin_part_blocks = nb;
  }
  cudaError_t e = launch_rhs(c, c->U, 0, 0.0, 0.0, 0);
  c->traces_valid = false;
  if (e == cudaSuccess) {
    k_zero_kin<<<1, 1, 0, c->stream>>>(c->scal);
    count_launch();
    e = launch_kinetic(c, c->U, c->Ut);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->scal_host, c->scal, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dg_kinetic");
  out[0] = c->scal_host->kin[0] / c->scal_host->kin[2];
  out[1] = c->scal_host->kin[1] / c->scal_host->kin[2];
  out[2] = c->scal_host->kin[2];
  return DG_OK;
}

int dg_debug(dg_ctx* c, int what, void* out0, void* out1) {
  if (!c || !out0) return fail(DG_ERR_ARG, "ctx or out0 is NULL");
  cudaError_t e = cudaSuccess;
  switch (what) {
    case DG_DEBUG_METRICS:
      if (!out1) return fail(DG_ERR_ARG, "out1 is NULL");
      e = launch_debug_metrics(c, (double*)out0, (double*)out1);
      break;
    case DG_DEBUG_MAPS:
      if (!out1) return fail(DG_ERR_ARG, "out1 is NULL");
      e = launch_debug_maps(c, (int*)out0, (int*)out1);
      break;
    case DG_DEBUG_GRAD: e = launch_debug_grad(c, (double*)out0); break;
    case DG_DEBUG_FSTAR: e = launch_debug_fstar(c, (double*)out0); break;
    case DG_DEBUG_ALPHA:
      e = cudaMemcpyAsync(out0, c->alpha, sizeof(double) * c->E, cudaMemcpyDeviceToDevice, c->stream);
      break;
    default: return fail(DG_ERR_ARG, "unknown debug item");
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dg_debug");
  return DG_OK;
}

}  // extern "C"
