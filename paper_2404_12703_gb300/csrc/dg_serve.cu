// dg_serve.cu -- continuous-batching request loop over many flow cases
// (include/dg.h, "Serving").
//
// Cases of one degree N share a pool (a context whose arrays hold many cases
// at element and side offsets, with per-element and per-side case maps and a
// shared case table).  A worker thread repeats:
//   admit   -- waiting cases that fit a free element range, side range and
//              case slot: maps and metrics are built by dg_init_mesh on a set-up
//              stream while resident cases keep stepping, then copied into the
//              pool (side and element indices shifted) on the step stream;
//   step    -- one CUDA graph = per pool a per-case CFL reduction, then the
//              per-case time steps, then 5 LSERK stages of every pool, each
//              kernel launched once over the pool's occupied range;
//   retire  -- cases whose time reached their end time: state copied out,
//              slots and ranges freed, time to solution recorded.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dg_common.cuh"
#include "dg_launch.h"

namespace dg {

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// per-case CFL reduction: one block per element, one atomic per element.
// T = float (FP32-bulk pools): the spectral radii in FP32 from the FP32
// metrics, as for a standalone FP32-bulk context.
template <int N, typename T>
__global__ void __launch_bounds__(128) k_cfl_cases(int64_t nlist, const int* __restrict__ elist,
                                                   const double* __restrict__ U, const double* __restrict__ metric,
                                                   const float* __restrict__ metric32,
                                                   const double* __restrict__ geo, const int* __restrict__ ecase,
                                                   double gamma, double gm1, double kvf, CaseData* cases) {
  constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
  constexpr bool f32 = sizeof(T) == sizeof(float);
  if (blockIdx.x >= nlist) return;
  const int64_t e = elist[blockIdx.x];
  const int c = ecase[e];
  // free slot, a case at its end time or one sitting out the step: the
  // whole block leaves together
  if (c < 0 || !(cases[c].t < cases[c].t_end) || cases[c].paused) return;
  const T kv = T(kvf * cases[c].mu);
  T lcT = T(0), lvT = T(0);
  int bad = 0;
  for (int t = threadIdx.x; t < n3; t += 128) {
    const double* up = U + e * 5 * n3 + t;
    const T r = T(up[0]), ri = T(1) / r;
    const T m0 = T(up[n3]), m1 = T(up[2 * n3]), m2 = T(up[3 * n3]);
    const T u = m0 * ri, v = m1 * ri, w = m2 * ri;
    const T p = T(gm1) * (T(up[4 * n3]) - T(0.5) * (m0 * u + m1 * v + m2 * w));
    const T cs = sqrt(T(gamma) * p * ri);
    auto M = [&](int k) { return f32 ? T(metric32[(e * 10 + k) * n3 + t]) : T(metric[(e * 10 + k) * n3 + t]); };
    const double* Gm = geo + e * 4 * n3 + t;
    const T Ji = M(9);
    T aa = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d)
      aa += fabs(u * M(d * 3) + v * M(d * 3 + 1) + w * M(d * 3 + 2)) + cs * T(Gm[d * n3]);
    aa *= Ji;
    const T bb = kv * ri * T(Gm[3 * n3]) * Ji * Ji;
    if (!isfinite(aa) || !isfinite(bb)) bad = 1;
    lcT = fmax(lcT, aa);
    lvT = fmax(lvT, bb);
  }
  double lc = to_f64<T>(lcT), lv = to_f64<T>(lvT);
  __shared__ double rc[4], rv[4];
  __shared__ int rb;
  if (threadIdx.x == 0) rb = 0;
  for (int o = 16; o > 0; o >>= 1) {
    lc = fmax(lc, __shfl_xor_sync(0xffffffffu, lc, o));
    lv = fmax(lv, __shfl_xor_sync(0xffffffffu, lv, o));
  }
  __syncwarp();
  __syncthreads();
  if (bad) atomicOr(&rb, 1);
  if ((threadIdx.x & 31) == 0) {
    rc[threadIdx.x >> 5] = lc;
    rv[threadIdx.x >> 5] = lv;
  }
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 4; ++w) {
      lc = fmax(lc, rc[w]);
      lv = fmax(lv, rv[w]);
    }
    atomicMax(&cases[c].lam_c, (unsigned long long)__double_as_longlong(lc));
    atomicMax(&cases[c].lam_v, (unsigned long long)__double_as_longlong(lv));
    if (rb) atomicOr(&cases[c].nonfinite, 1);
  }
}

// per-case time step: CFL rule, clipped at the end time; 0 once finished or
// non-finite (the stages then leave the state unchanged)
__global__ void k_dt_cases(int nslots, CaseData* cases) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nslots) return;
  CaseData& d = cases[c];
  if (!d.active) return;
  if (d.paused) {  // sits out this step: time step 0, state unchanged
    d.dt = 0.0;
    d.lam_c = 0ull;
    d.lam_v = 0ull;
    return;
  }
  const double np1 = d.N + 1.0;
  const double lc = __longlong_as_double((long long)d.lam_c);
  const double lv = __longlong_as_double((long long)d.lam_v);
  double dt = d.cfl * 2.0 / (np1 * np1 * lc);
  if (lv > 0) dt = fmin(dt, d.dfl * 4.0 / (np1 * np1 * np1 * np1 * lv));
  const double rest = d.t_end - d.t;
  if (dt >= rest) dt = rest;
  if (!(rest > 0) || d.nonfinite || !(dt > 0)) dt = 0.0;
  d.dt = dt;
  d.t = dt > 0 ? (dt == rest ? d.t_end : d.t + dt) : d.t;
  if (dt > 0) d.steps += 1;
  d.lam_c = 0ull;
  d.lam_v = 0ull;
}

// sit-out flags of the case slots (priority policy), one bit per slot
struct PauseMask {
  unsigned long long w[64];
};
__global__ void k_set_pause(CaseData* cases, int nslots, PauseMask m) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nslots) cases[c].paused = (int)((m.w[c >> 6] >> (c & 63)) & 1ull);
}

__global__ void k_fill_int(int* p, int64_t n, int v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
// copy with an index shift: element -> side ids (elem_side packs side << 4)
__global__ void k_shift_elem_side(const int* __restrict__ src, int* __restrict__ dst, int64_t n, int s0) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] + (s0 << 4);
}
__global__ void k_shift_side_e(const int2* __restrict__ src, int2* __restrict__ dst, int64_t n, int e0) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = make_int2(src[i].x + e0, src[i].y + e0);
}

template <int N>
static void launch_cfl_cases(dg_ctx* p, double kvf, cudaStream_t st) {
  const int64_t nl = p->n_elem_list;
  if (nl <= 0) return;
  if (p->prm.precision == DG_FP32_BULK)
    k_cfl_cases<N, float><<<(unsigned)nl, 128, 0, st>>>(nl, p->elem_list, p->U, p->metric, p->metric32, p->cflgeo,
                                                          p->elem_case, p->prm.gamma, p->prm.gamma - 1.0, kvf,
                                                          p->cases);
  else
    k_cfl_cases<N, double><<<(unsigned)nl, 128, 0, st>>>(nl, p->elem_list, p->U, p->metric, p->metric32, p->cflgeo,
                                                           p->elem_case, p->prm.gamma, p->prm.gamma - 1.0, kvf,
                                                           p->cases);
}

// marks a case slot free (stream-ordered; no host buffer involved)
__global__ void k_deactivate(CaseData* d) { d->active = 0; }

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using Clock = std::chrono::steady_clock;

static double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

// first-fit allocator of [0, cap) ranges
struct RangeAlloc {
  int64_t cap = 0;
  std::map<int64_t, int64_t> free_;  // offset -> length
  void init(int64_t c) {
    cap = c;
    free_.clear();
    if (c > 0) free_[0] = c;
  }
  int64_t take(int64_t len) {
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= len) {
        const int64_t off = it->first, rest = it->second - len;
        free_.erase(it);
        if (rest > 0) free_[off + len] = rest;
        return off;
      }
    return -1;
  }
  void give(int64_t off, int64_t len) {
    auto it = free_.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  // one past the highest occupied index
  int64_t high() const {
    if (free_.empty()) return cap;
    auto last = std::prev(free_.end());
    return last->first + last->second == cap ? last->first : cap;
  }
};

struct Pool {
  int N = 0;
  dg_ctx* ctx = nullptr;
  RangeAlloc elems, sides;
  cudaStream_t branch = nullptr;  // capture-only stream: the pool's branch of the step graph
  cudaEvent_t fork = nullptr, join = nullptr;
  int* h_elist[2] = {nullptr, nullptr};  // pinned staging of the occupied-element / side lists,
  int* h_slist[2] = {nullptr, nullptr};  // alternating between rebuilds
  int list_buf = 0;
  int* h_timeout = nullptr;  // pinned [2]: the pool's persistent-launch timeout flag after step k
};

struct Request {
  int64_t ticket = 0;
  int N = 0;
  int64_t E = 0;
  std::vector<int64_t> cvid;
  std::vector<double> xyz, U0;
  double t_end = 0, mu = 0, cfl = 0.9;
  int riemann = 0;
  double t_submit = 0;
  dg_ctx* prepared = nullptr;  // maps, metrics and state built by the set-up thread
  double* out_buf = nullptr;   // pinned buffer the final state is copied to
  size_t out_cap = 0;          // its size in doubles
};

struct Slot {
  bool used = false;
  int64_t ticket = -1;
  int N = 0;
  int64_t e0 = 0, E = 0, s0 = 0, S = 0;
  double t_submit = 0, t_admit = 0, t_end = 0;
  int64_t first_step = 0;       // index of the first batched step the case takes part in
  CaseData* staging = nullptr;  // pinned, per slot
  double* out_buf = nullptr;    // pinned output buffer of the resident case
  size_t out_cap = 0;
};

// a retired case whose final state is still being copied out
struct Retiring {
  int64_t ticket = 0;
  double* buf = nullptr;
  size_t cap = 0, count = 0;
  cudaEvent_t ev = nullptr;
  double t_submit = 0, t_admit = 0;
  double stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

struct Result {
  std::vector<double> U;
  double stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

struct PendingFree {
  dg_ctx* ctx;
  cudaEvent_t ev;
};

}  // namespace dg

struct dg_server {
  dg_server_config cfg{};
  dg_params prm{};
  int device = 0;
  cudaStream_t stream = nullptr, setup_stream = nullptr, cap_stream = nullptr;
  std::map<int, dg::Pool> pools;
  dg::CaseData* d_cases = nullptr;
  dg::CaseData* h_cases = nullptr;    // two buffers: case records after step k and k+1
  cudaEvent_t step_ev[2] = {nullptr, nullptr};   // after step k's records are copied (timing)
  cudaEvent_t step_t0[2] = {nullptr, nullptr};   // before step k's graph launch (timing)
  int64_t launched = 0;               // batched steps launched so far
  std::vector<dg::Slot> slots;
  std::thread worker;
  std::thread preparer;               // builds cases' maps and metrics off the step loop
  std::deque<dg::Request> ready;      // prepared, waiting for pool room
  std::mutex m;
  std::condition_variable cv;
  bool stop = false;
  std::deque<dg::Request> pending;
  std::map<int64_t, dg::Result> results;
  std::map<int64_t, int> running;  // ticket -> slot
  std::map<int64_t, int> admitting;  // tickets taken off the queue, being admitted
  int64_t next_ticket = 1;
  cudaGraphExec_t graph = nullptr;
  std::vector<std::pair<cudaGraphExec_t, cudaEvent_t>> old_graphs;  // replaced, maybe still in flight
  bool dirty = true;
  std::vector<dg::PendingFree> frees;
  int64_t resident_dof = 0;                     // step thread only
  std::vector<dg::Retiring> retiring;           // step thread only
  std::multimap<size_t, double*> pinned_free;   // reusable output buffers (size in doubles)
  std::vector<cudaEvent_t> events_free;         // step thread only
  double stat_steps = 0, stat_finished = 0, stat_captures = 0, stat_dofstages = 0, stat_device_s = 0;
  double stat_capture_s = 0, stat_prepare_s = 0, stat_insert_s = 0;  // host time
  std::string worker_error;
  dg::PauseMask pause{};  // sit-out flags last sent to the device (step thread only)
};

namespace dg {

static thread_local std::string g_serve_err;

// Rebuilds each pool's lists of occupied elements and sides from the case
// slots (in element order) and copies them to the device on the step stream:
// work already queued still reads the old lists, later steps the new ones.
// A pinned staging buffer is reused two rebuilds later, after the step loop
// has waited for a step queued behind its copy.
static cudaError_t rebuild_lists(dg_server* s) {
  cudaError_t e = cudaSuccess;
  for (auto& kv : s->pools) {
    Pool& P = kv.second;
    std::vector<std::pair<int64_t, int>> occ;  // (e0, slot)
    for (int i = 0; i < (int)s->slots.size(); ++i)
      if (s->slots[i].used && s->slots[i].N == P.N) occ.emplace_back(s->slots[i].e0, i);
    std::sort(occ.begin(), occ.end());
    int* he = P.h_elist[P.list_buf];
    int* hs = P.h_slist[P.list_buf];
    int64_t ne = 0, ns = 0;
    for (auto& o : occ) {
      const Slot& sl = s->slots[o.second];
      for (int64_t k = 0; k < sl.E; ++k) he[ne++] = (int)(sl.e0 + k);
      for (int64_t k = 0; k < sl.S; ++k) hs[ns++] = (int)(sl.s0 + k);
    }
    if (ne > 0 && e == cudaSuccess)
      e = cudaMemcpyAsync(P.ctx->elem_list, he, sizeof(int) * ne, cudaMemcpyHostToDevice, s->stream);
    if (ns > 0 && e == cudaSuccess)
      e = cudaMemcpyAsync(P.ctx->side_list, hs, sizeof(int) * ns, cudaMemcpyHostToDevice, s->stream);
    P.ctx->n_elem_list = ne;
    P.ctx->n_side_list = ns;
    P.list_buf ^= 1;
  }
  return e;
}

// the whole batched step for the pools' current ranges, captured once
static cudaError_t capture_step(dg_server* s) {
  static const double RKA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                                -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
  static const double RKB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                                1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                                2277821191437.0 / 14882151754819.0};
  static const double RKC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363218457.0,
                                2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};
  const double kvf = std::max(4.0 / 3.0, s->prm.gamma / s->prm.Pr);
  // The graph forks into one branch per pool, so that the kernels of
  // different pools (degrees) can run side by side:
  //   fork -> [CFL of each pool] -> join -> per-case dt -> fork -> [5 stages of
  //   each pool] -> join
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (le == cudaSuccess) le = r; };
  auto fork = [&]() {
    for (auto& kv : s->pools) {
      chk(cudaEventRecord(kv.second.fork, s->cap_stream));
      chk(cudaStreamWaitEvent(kv.second.branch, kv.second.fork, 0));
    }
  };
  auto join = [&]() {
    for (auto& kv : s->pools) {
      chk(cudaEventRecord(kv.second.join, kv.second.branch));
      chk(cudaStreamWaitEvent(s->cap_stream, kv.second.join, 0));
    }
  };
  fork();
  for (auto& kv : s->pools) {
    Pool& P = kv.second;
    switch (P.N) {
      case 1: launch_cfl_cases<1>(P.ctx, kvf, P.branch); break;
      case 2: launch_cfl_cases<2>(P.ctx, kvf, P.branch); break;
      case 3: launch_cfl_cases<3>(P.ctx, kvf, P.branch); break;
      case 4: launch_cfl_cases<4>(P.ctx, kvf, P.branch); break;
      case 5: launch_cfl_cases<5>(P.ctx, kvf, P.branch); break;
      case 6: launch_cfl_cases<6>(P.ctx, kvf, P.branch); break;
      default: launch_cfl_cases<7>(P.ctx, kvf, P.branch); break;
    }
    count_launch();
  }
  join();
  k_dt_cases<<<(s->cfg.max_cases + 127) / 128, 128, 0, s->cap_stream>>>(s->cfg.max_cases, s->d_cases);
  count_launch();
  fork();
  for (auto& kv : s->pools) {
    Pool& P = kv.second;
    if (P.ctx->n_elem_list == 0) continue;
    cudaStream_t keep = P.ctx->stream;
    P.ctx->stream = P.branch;
    if (persist_active(P.ctx)) {
      // every stage in one persistent launch; the pools' persistent launches
      // follow one another on the main capture stream (each grid fills the
      // GPU, and its blocks must all be resident at once)
      P.ctx->stream = s->cap_stream;
      le = launch_persist(P.ctx, 5, RKA, RKB, RKC);
    } else {
      for (int st = 0; st < 5 && le == cudaSuccess; ++st) le = launch_rhs(P.ctx, P.ctx->U, 1, RKA[st], RKB[st], st == 0);
    }
    P.ctx->stream = keep;
  }
  join();
  e = cudaStreamEndCapture(s->cap_stream, &g);
  if (e == cudaSuccess) e = le;
  // Same topology (only grid sizes changed): update the executable graph in
  // place, which affects later launches only.  Otherwise instantiate a new
  // one; the old one is destroyed once its last launch has completed.
  bool updated = false;
  if (e == cudaSuccess && s->graph) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(s->graph, g, &info) == cudaSuccess) {
      updated = true;
    } else {
      cudaGetLastError();
      cudaEvent_t ev = nullptr;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
          cudaEventRecord(ev, s->stream) == cudaSuccess) {
        s->old_graphs.push_back({s->graph, ev});
      } else {
        cudaStreamSynchronize(s->stream);
        cudaGraphExecDestroy(s->graph);
        if (ev) cudaEventDestroy(ev);
      }
      s->graph = nullptr;
    }
  }
  if (e == cudaSuccess && !updated) e = cudaGraphInstantiate(&s->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  // executable graphs whose last launch has completed
  for (size_t i = 0; i < s->old_graphs.size();) {
    if (cudaEventQuery(s->old_graphs[i].second) == cudaSuccess) {
      cudaGraphExecDestroy(s->old_graphs[i].first);
      cudaEventDestroy(s->old_graphs[i].second);
      s->old_graphs.erase(s->old_graphs.begin() + i);
    } else {
      ++i;
    }
  }
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stat_captures += 1;
  }
  return e;
}

}  // namespace dg

namespace dg {

static bool slot_fits(dg_server* s, const Request& r) {
  auto it = s->pools.find(r.N);
  if (it == s->pools.end()) return false;
  return it->second.elems.cap >= r.E && it->second.sides.cap >= 3 * r.E;
}

// Builds the case's maps, metrics and state in a temporary context on the
// set-up stream (set-up thread).
static bool prepare(dg_server* s, Request& r, std::string& err) {
  dg_params prm = s->prm;
  prm.mu = r.mu;
  prm.viscous = 1;
  prm.riemann = r.riemann;
  dg_mesh_desc desc{r.N, r.E, r.cvid.data(), r.xyz.data()};
  dg_ctx* tmp = nullptr;
  int st = init_mesh_impl(&tmp, &desc, &prm, s->setup_stream, s->setup_stream);
  if (st == DG_OK) st = dg_set_state(tmp, r.U0.data(), 0, 0.0);
  if (st == DG_OK && cudaStreamSynchronize(s->setup_stream) != cudaSuccess) st = DG_ERR_CUDA;
  if (st != DG_OK) {
    err = std::string("case set-up failed: ") + dg_last_error();
    if (tmp) dg_destroy(tmp);
    return false;
  }
  r.prepared = tmp;
  // pinned output buffer, reused from retired cases when one is large enough
  const size_t need = (size_t)r.E * (r.N + 1) * (r.N + 1) * (r.N + 1) * 5;
  {
    std::lock_guard<std::mutex> lk(s->m);
    auto it = s->pinned_free.lower_bound(need);
    if (it != s->pinned_free.end()) {
      r.out_buf = it->second;
      r.out_cap = it->first;
      s->pinned_free.erase(it);
    }
  }
  if (!r.out_buf) {
    if (cudaMallocHost(&r.out_buf, sizeof(double) * need) != cudaSuccess) {
      r.out_buf = nullptr;
      err = "case set-up failed: no pinned host memory for the result";
      dg_destroy(tmp);
      r.prepared = nullptr;
      return false;
    }
    r.out_cap = need;
  }
  return true;
}

static void give_pinned(dg_server* s, double* buf, size_t cap) {
  if (!buf) return;
  std::lock_guard<std::mutex> lk(s->m);
  s->pinned_free.emplace(cap, buf);
}

// Copies a prepared case into its pool on the step stream (step thread).
// Returns false (nothing changed) when the pool has no room or no slot is free.
static bool admit(dg_server* s, Request& r, std::string& err) {
  Pool& P = s->pools[r.N];
  int slot = -1;
  for (int i = 0; i < (int)s->slots.size(); ++i)
    if (!s->slots[i].used) { slot = i; break; }
  if (slot < 0) return false;
  const int64_t e0 = P.elems.take(r.E);
  if (e0 < 0) return false;
  const int64_t s0 = P.sides.take(3 * r.E);
  if (s0 < 0) {
    P.elems.give(e0, r.E);
    return false;
  }
  dg_ctx* tmp = r.prepared;
  r.prepared = nullptr;
  dg_ctx* p = P.ctx;
  const int n2 = p->n2, n3 = p->n3;
  const int64_t E = r.E, S = 3 * r.E;
  cudaStream_t q = s->stream;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, q);
  };
  cp(p->U + e0 * 5 * n3, tmp->U, sizeof(double) * E * 5 * n3);
  cp(p->metric + e0 * 10 * n3, tmp->metric, sizeof(double) * E * 10 * n3);
  if (p->metric32 && tmp->metric32) cp(p->metric32 + e0 * 10 * n3, tmp->metric32, sizeof(float) * E * 10 * n3);
  cp(p->cflgeo + e0 * 4 * n3, tmp->cflgeo, sizeof(double) * E * 4 * n3);
  if (p->fvmetric && tmp->fvmetric)
    cp(p->fvmetric + e0 * 3 * (p->n - 1) * 3 * n2, tmp->fvmetric, sizeof(double) * E * 3 * (p->n - 1) * 3 * n2);
  cp(p->nrm + s0 * 4 * n2, tmp->nrm, sizeof(double) * S * 4 * n2);
  if (p->nrm32 && tmp->nrm32) cp(p->nrm32 + s0 * 7 * n2, tmp->nrm32, sizeof(float) * S * 7 * n2);
  cp(p->side_f + s0, tmp->side_f, sizeof(int) * S);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->dU + e0 * 5 * n3, 0, sizeof(double) * E * 5 * n3, q);
  if (e == cudaSuccess) {
    k_shift_elem_side<<<(unsigned)((E * 6 + 255) / 256), 256, 0, q>>>(tmp->elem_side, p->elem_side + e0 * 6, E * 6,
                                                                       (int)s0);
    k_shift_side_e<<<(unsigned)((S + 255) / 256), 256, 0, q>>>(tmp->side_e, p->side_e + s0, S, (int)e0);
    k_fill_int<<<(unsigned)((E + 255) / 256), 256, 0, q>>>(p->elem_case + e0, E, slot);
    k_fill_int<<<(unsigned)((S + 255) / 256), 256, 0, q>>>(p->side_case + s0, S, slot);
    count_launch(4);
    e = cudaGetLastError();
  }
  // case record: reference state from the case's first node (FP32-bulk), or 0
  Slot& sl = s->slots[slot];
  CaseData& d = *sl.staging;
  memset(&d, 0, sizeof(d));
  d.t_end = r.t_end;
  d.mu = r.mu;
  d.lam = s->prm.gamma * s->prm.R * r.mu / ((s->prm.gamma - 1.0) * s->prm.Pr);
  d.f_mu = (float)d.mu;
  d.f_lam = (float)d.lam;
  d.cfl = r.cfl;
  d.dfl = s->prm.dfl;
  d.riemann = r.riemann;
  d.active = 1;
  d.N = r.N;
  if (s->prm.precision == DG_FP32_BULK) {
    // the density and pressure of the case's first node, at rest (as for a
    // standalone FP32-bulk context)
    const double* u0 = r.U0.data();
    const double gm1 = s->prm.gamma - 1.0, rho = u0[0];
    const double pp = gm1 * (u0[4] - 0.5 * (u0[1] * u0[1] + u0[2] * u0[2] + u0[3] * u0[3]) / rho);
    d.ref_rho = rho;
    d.ref_p = pp;
    d.ref_E = pp / gm1;
    d.ref_H = (d.ref_E + pp) / rho;
    d.ref_T = pp / (rho * s->prm.R);
    d.f_ref_p = (float)d.ref_p;
    d.f_ref_H = (float)d.ref_H;
    d.f_ref_T = (float)d.ref_T;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_cases + slot, &d, sizeof(CaseData), cudaMemcpyHostToDevice, q);
  // the two-kernel FP32-bulk stage: the face data of the case's initial state
  if (e == cudaSuccess && fused_active(p)) e = launch_fprep(p, p->U, e0, E, q);
  cudaEvent_t ev = nullptr;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, q);
  if (e != cudaSuccess) {
    err = std::string("case insertion: ") + cudaGetErrorString(e);
    if (ev) cudaEventDestroy(ev);
    cudaStreamSynchronize(q);
    dg_destroy(tmp);
    return false;
  }
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->frees.push_back({tmp, ev});  // the temporary context is freed once the copies are done
  }
  sl.used = true;
  sl.ticket = r.ticket;
  sl.N = r.N;
  sl.e0 = e0;
  sl.E = E;
  sl.s0 = s0;
  sl.S = S;
  sl.t_submit = r.t_submit;
  sl.t_admit = now_s();
  sl.t_end = r.t_end;
  sl.first_step = s->launched;
  sl.out_buf = r.out_buf;
  sl.out_cap = r.out_cap;
  r.out_buf = nullptr;
  p->E = P.elems.high();
  p->S = P.sides.high();
  s->dirty = true;  // the occupied lists change
  return true;
}

// Frees the temporary contexts whose insertion copies have completed (all of
// them with wait).  Runs on the set-up thread: cudaFree may wait for the
// device, which the step loop must not.
static void reap_frees(dg_server* s, bool wait) {
  std::vector<PendingFree> done;
  {
    std::lock_guard<std::mutex> lk(s->m);
    for (size_t i = 0; i < s->frees.size();) {
      if (wait || cudaEventQuery(s->frees[i].ev) == cudaSuccess) {
        done.push_back(s->frees[i]);
        s->frees.erase(s->frees.begin() + i);
      } else {
        ++i;
      }
    }
  }
  for (auto& f : done) {
    cudaEventSynchronize(f.ev);
    cudaEventDestroy(f.ev);
    dg_destroy(f.ctx);
  }
}

// Starts copying the case's state out (public layout, into its pinned output
// buffer) and frees its slot and ranges at once: later work on them is
// ordered after the copy on the step stream.  The result is published by
// finish_retired once the copy has completed.
static void retire(dg_server* s, int slot, const CaseData& rec) {
  Slot& sl = s->slots[slot];
  Pool& P = s->pools[sl.N];
  dg_ctx* p = P.ctx;
  const int n3 = p->n3;
  cudaStream_t q = s->stream;
  dg_ctx view = {};
  view.E = sl.E;
  view.n3 = n3;
  view.stream = q;
  launch_to_public(&view, p->U + sl.e0 * 5 * n3, p->Upub + sl.e0 * 5 * n3);
  Retiring r;
  r.ticket = sl.ticket;
  r.buf = sl.out_buf;
  r.cap = sl.out_cap;
  r.count = (size_t)sl.E * n3 * 5;
  cudaMemcpyAsync(r.buf, p->Upub + sl.e0 * 5 * n3, sizeof(double) * r.count, cudaMemcpyDeviceToHost, q);
  k_fill_int<<<(unsigned)((sl.E + 255) / 256), 256, 0, q>>>(p->elem_case + sl.e0, sl.E, -1);
  k_fill_int<<<(unsigned)((sl.S + 255) / 256), 256, 0, q>>>(p->side_case + sl.s0, sl.S, -1);
  k_deactivate<<<1, 1, 0, q>>>(s->d_cases + slot);
  count_launch(4);
  if (s->events_free.empty()) {
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    s->events_free.push_back(ev);
  }
  r.ev = s->events_free.back();
  s->events_free.pop_back();
  cudaEventRecord(r.ev, q);
  r.t_submit = sl.t_submit;
  r.t_admit = sl.t_admit;
  r.stats[3] = rec.t;
  r.stats[4] = rec.steps;
  r.stats[5] = (double)sl.E;
  r.stats[6] = sl.N;
  r.stats[7] = rec.nonfinite ? 1.0 : 0.0;
  s->retiring.push_back(r);
  P.elems.give(sl.e0, sl.E);
  P.sides.give(sl.s0, sl.S);
  p->E = P.elems.high();
  p->S = P.sides.high();
  s->dirty = true;  // the occupied lists change
  s->resident_dof -= sl.E * (int64_t)(sl.N + 1) * (sl.N + 1) * (sl.N + 1);
  sl.used = false;
  sl.ticket = -1;
  sl.out_buf = nullptr;
}

// Publishes the results whose copies have completed (all of them with wait).
static void finish_retired(dg_server* s, bool wait) {
  for (size_t i = 0; i < s->retiring.size();) {
    Retiring& r = s->retiring[i];
    if (!wait && cudaEventQuery(r.ev) != cudaSuccess) {
      ++i;
      continue;
    }
    cudaEventSynchronize(r.ev);
    const double t_done = now_s();
    Result res;
    res.U.assign(r.buf, r.buf + r.count);
    memcpy(res.stats, r.stats, sizeof(res.stats));
    res.stats[0] = t_done - r.t_submit;
    res.stats[1] = r.t_admit - r.t_submit;
    res.stats[2] = t_done - r.t_admit;
    s->events_free.push_back(r.ev);
    give_pinned(s, r.buf, r.cap);
    {
      std::lock_guard<std::mutex> lk(s->m);
      s->results[r.ticket] = std::move(res);
      s->running.erase(r.ticket);
      s->stat_finished += 1;
    }
    s->retiring.erase(s->retiring.begin() + i);
  }
}

// Step loop.  Keeps one batched step queued behind the one it inspects: after
// launching step k+1 it waits for the case records of step k and retires the
// cases that had reached their end time there.  Such a case takes part in
// step k+1 with time step 0, which leaves its state unchanged and whose blocks
// exit at once.
static void worker_loop(dg_server* s) {
  cudaSetDevice(s->device);
  bool inflight = false;  // a step whose records have not been inspected
  for (;;) {
    // 1. insertion of prepared cases that fit (first fit, arrival order)
    std::vector<Request> take;
    {
      std::unique_lock<std::mutex> lk(s->m);
      if (s->stop) break;
      bool resident = false;
      for (auto& sl : s->slots) resident = resident || sl.used;
      if (!resident && s->ready.empty() && !inflight) {
        if (!s->retiring.empty()) {
          lk.unlock();
          finish_retired(s, true);
          continue;
        }
        s->cv.wait_for(lk, std::chrono::milliseconds(5));
        if (s->stop) break;
      }
      while (!s->ready.empty()) {
        take.push_back(std::move(s->ready.front()));
        s->ready.pop_front();
      }
    }
    std::vector<Request> back;
    const double ti0 = now_s();
    bool blocked = false;  // strict order: a case that waits holds back the later ones
    for (auto& r : take) {
      std::string err;
      const int64_t dof = r.E * (r.N + 1) * (r.N + 1) * (r.N + 1);
      const int64_t cap = s->cfg.max_resident_dof;
      if (cap > 0 && (blocked || (s->resident_dof > 0 && s->resident_dof + dof > cap))) {
        blocked = true;
        back.push_back(std::move(r));
        continue;
      }
      if (admit(s, r, err)) {
        s->resident_dof += dof;
        std::lock_guard<std::mutex> lk(s->m);
        s->running[r.ticket] = -1;
        for (int i = 0; i < (int)s->slots.size(); ++i)
          if (s->slots[i].used && s->slots[i].ticket == r.ticket) s->running[r.ticket] = i;
        s->admitting.erase(r.ticket);
      } else if (!err.empty()) {
        give_pinned(s, r.out_buf, r.out_cap);
        r.out_buf = nullptr;
        Result res;
        res.stats[7] = 2.0;
        std::lock_guard<std::mutex> lk(s->m);
        s->results[r.ticket] = std::move(res);
        s->worker_error = err;
        s->admitting.erase(r.ticket);
      } else {
        if (cap > 0) blocked = true;
        back.push_back(std::move(r));  // no room yet: stays prepared
      }
    }
    {
      std::lock_guard<std::mutex> lk(s->m);
      for (auto it = back.rbegin(); it != back.rend(); ++it) s->ready.push_front(std::move(*it));
      if (!take.empty()) s->stat_insert_s += now_s() - ti0;
    }
    s->cv.notify_all();
    bool have = false;
    for (auto& sl : s->slots) have = have || sl.used;
    // 2. launch step k+1 of every resident case
    if (have) {
      const bool membership_changed = s->dirty;
      if (s->dirty) {
        // an executable graph still in flight is released when it completes
        const double tc0 = now_s();
        cudaError_t e = rebuild_lists(s);
        // a pool's launch configuration is tuned once, when its cases first
        // fill the GPU several times over (about four waves of default
        // blocks: tuning on a few small cases would pick for tiny grids)
        int nsm = 152;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
        for (auto& kv : s->pools) {
          dg_ctx* pc = kv.second.ctx;
          const int n3 = pc->n3, D = n3 >= 256 ? 1 : 256 / n3;
          if (e != cudaSuccess || pc->tuned || pc->n_elem_list < (int64_t)4 * 2 * nsm * D) continue;
          cudaStream_t keep = pc->stream;
          pc->stream = s->stream;
          // the thread mapping stays the default one: a case's result must not
          // depend on which cases the pool was tuned on
          pc->tune_keep_mapping = true;
          double ms[8];
          e = launch_autotune(pc, ms);
          pc->stream = keep;
        }
        if (e == cudaSuccess) e = capture_step(s);
        {
          std::lock_guard<std::mutex> lk(s->m);
          s->stat_capture_s += now_s() - tc0;
        }
        if (e != cudaSuccess) {
          std::lock_guard<std::mutex> lk(s->m);
          s->worker_error = std::string("graph capture: ") + cudaGetErrorString(e);
          s->stop = true;
          break;
        }
        s->dirty = false;
      }
      if (s->cfg.priority_dof > 0) {
        // priority policy: resident cases in submission order, first fit
        // within the DOF bound, the oldest always; the rest sit this step out
        std::vector<int> order;
        for (int i = 0; i < (int)s->slots.size(); ++i)
          if (s->slots[i].used) order.push_back(i);
        std::sort(order.begin(), order.end(),
                  [&](int x, int y) { return s->slots[x].ticket < s->slots[y].ticket; });
        PauseMask m{};
        int64_t run = 0;
        bool first = true;
        for (int i : order) {
          const Slot& sl = s->slots[i];
          const int64_t dof = sl.E * (sl.N + 1) * (sl.N + 1) * (sl.N + 1);
          if (first || run + dof <= s->cfg.priority_dof) {
            run += dof;
            first = false;
          } else {
            m.w[i >> 6] |= 1ull << (i & 63);
          }
        }
        if (membership_changed || memcmp(&m, &s->pause, sizeof(m)) != 0) {
          const int ns = (int)s->slots.size();
          k_set_pause<<<(ns + 127) / 128, 128, 0, s->stream>>>(s->d_cases, ns, m);
          count_launch(1);
          s->pause = m;
        }
      }
      const int b = (int)(s->launched & 1);
      cudaEventRecord(s->step_t0[b], s->stream);
      cudaGraphLaunch(s->graph, s->stream);
      count_launch(1);
      cudaMemcpyAsync(s->h_cases + b * s->cfg.max_cases, s->d_cases, sizeof(CaseData) * s->cfg.max_cases,
                      cudaMemcpyDeviceToHost, s->stream);
      for (auto& kv : s->pools)
        if (kv.second.h_timeout)
          cudaMemcpyAsync(kv.second.h_timeout + b, &kv.second.ctx->scal->timeout, sizeof(int), cudaMemcpyDeviceToHost,
                          s->stream);
      cudaEventRecord(s->step_ev[b], s->stream);
      s->launched += 1;
    }
    if (!inflight) {
      inflight = have;
      continue;
    }
    // 3. records of step k (the one before the step just launched, or the
    //    last one when nothing is resident any more)
    const int64_t k = have ? s->launched - 2 : s->launched - 1;
    const int b = (int)(k & 1);
    cudaError_t e = cudaEventSynchronize(s->step_ev[b]);
    if (e != cudaSuccess) {
      std::lock_guard<std::mutex> lk(s->m);
      s->worker_error = std::string("batched step: ") + cudaGetErrorString(e);
      s->stop = true;
      break;
    }
    inflight = have;
    bool timed_out = false;
    for (auto& kv : s->pools) timed_out = timed_out || (kv.second.h_timeout && kv.second.h_timeout[b]);
    if (timed_out) {
      std::lock_guard<std::mutex> lk(s->m);
      s->worker_error = "batched step: a persistent launch's grid-wide wait ran out";
      s->stop = true;
      break;
    }
    const CaseData* rec = s->h_cases + b * s->cfg.max_cases;
    float step_ms = 0.0f;
    cudaEventElapsedTime(&step_ms, s->step_t0[b], s->step_ev[b]);
    {
      std::lock_guard<std::mutex> lk(s->m);
      s->stat_steps += 1;
      s->stat_device_s += 1e-3 * step_ms;
    }
    for (int i = 0; i < (int)s->slots.size(); ++i) {
      Slot& sl = s->slots[i];
      if (!sl.used || sl.first_step > k) continue;  // admitted after step k
      const CaseData d = rec[i];
      if (d.dt > 0) {
        std::lock_guard<std::mutex> lk(s->m);
        s->stat_dofstages += 5.0 * (double)sl.E * (sl.N + 1) * (sl.N + 1) * (sl.N + 1);
      }
      if (d.t >= sl.t_end || d.nonfinite) retire(s, i, d);
    }
    finish_retired(s, false);
  }
  cudaStreamSynchronize(s->stream);
  finish_retired(s, true);
}

// Set-up thread: takes queued cases in arrival order and prepares up to
// kReady of them ahead of pool admission.
static void prepare_loop(dg_server* s) {
  constexpr size_t kReady = 4;
  cudaSetDevice(s->device);
  for (;;) {
    Request r;
    {
      std::unique_lock<std::mutex> lk(s->m);
      s->cv.wait_for(lk, std::chrono::milliseconds(5),
                     [&] { return s->stop || (!s->pending.empty() && s->ready.size() < kReady); });
      if (s->stop) break;
      if (s->pending.empty() || s->ready.size() >= kReady) {
        lk.unlock();
        reap_frees(s, false);
        continue;
      }
      r = std::move(s->pending.front());
      s->pending.pop_front();
      s->admitting[r.ticket] = 1;
    }
    std::string err;
    reap_frees(s, false);
    const double tp0 = now_s();
    const bool ok = prepare(s, r, err);
    {
      std::lock_guard<std::mutex> lk(s->m);
      s->stat_prepare_s += now_s() - tp0;
    }
    std::lock_guard<std::mutex> lk(s->m);
    if (ok) {
      s->ready.push_back(std::move(r));
      s->cv.notify_all();
    } else {
      Result res;
      res.stats[7] = 2.0;  // failed set-up
      s->results[r.ticket] = std::move(res);
      s->worker_error = err;
      s->admitting.erase(r.ticket);
    }
  }
}

}  // namespace dg

using namespace dg;

extern "C" {

void dg_server_default_config(dg_server_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->gamma = 1.4;
  c->R = 1.0;
  c->Pr = 0.72;
  c->dfl = 0.9;
  c->precision = DG_FP64;
  c->max_cases = 64;
  c->pool_elems[3] = 262144;
  c->pool_elems[5] = 262144;
  c->pool_elems[7] = 65536;
}

void dg_server_destroy(dg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->preparer.joinable()) s->preparer.join();
  for (auto& r : s->ready) {
    if (r.prepared) dg_destroy(r.prepared);
    if (r.out_buf) cudaFreeHost(r.out_buf);
  }
  s->ready.clear();
  for (auto& sl : s->slots)
    if (sl.out_buf) cudaFreeHost(sl.out_buf);
  for (auto& kv : s->pinned_free) cudaFreeHost(kv.second);
  s->pinned_free.clear();
  for (auto ev : s->events_free) cudaEventDestroy(ev);
  s->events_free.clear();
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  reap_frees(s, true);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  for (auto& og : s->old_graphs) {
    cudaGraphExecDestroy(og.first);
    cudaEventDestroy(og.second);
  }
  for (auto& kv : s->pools) {
    kv.second.ctx->cases = nullptr;  // owned by the server
    dg_destroy(kv.second.ctx);
    if (kv.second.branch) cudaStreamDestroy(kv.second.branch);
    for (int b = 0; b < 2; ++b) {
      if (kv.second.h_elist[b]) cudaFreeHost(kv.second.h_elist[b]);
      if (kv.second.h_slist[b]) cudaFreeHost(kv.second.h_slist[b]);
    }
    if (kv.second.h_timeout) cudaFreeHost(kv.second.h_timeout);
    if (kv.second.fork) cudaEventDestroy(kv.second.fork);
    if (kv.second.join) cudaEventDestroy(kv.second.join);
  }
  for (auto& sl : s->slots)
    if (sl.staging) cudaFreeHost(sl.staging);
  if (s->h_cases) cudaFreeHost(s->h_cases);
  for (int b = 0; b < 2; ++b) {
    if (s->step_ev[b]) cudaEventDestroy(s->step_ev[b]);
    if (s->step_t0[b]) cudaEventDestroy(s->step_t0[b]);
  }
  if (s->d_cases) cudaFree(s->d_cases);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->setup_stream) cudaStreamDestroy(s->setup_stream);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  delete s;
}

int dg_server_create(dg_server** out, const dg_server_config* cfg) {
  if (!out || !cfg) return set_error(DG_ERR_ARG, "dg_server_create: NULL argument");
  *out = nullptr;
  if (cfg->max_cases < 1 || cfg->max_cases > 4096) return set_error(DG_ERR_ARG, "max_cases must be in [1, 4096]");
  if (cfg->max_resident_dof < 0) return set_error(DG_ERR_ARG, "max_resident_dof must be >= 0");
  if (cfg->priority_dof < 0) return set_error(DG_ERR_ARG, "priority_dof must be >= 0");
  if (cfg->precision != DG_FP64 && cfg->precision != DG_FP32_BULK) return set_error(DG_ERR_ARG, "bad precision");
  dg_server* s = new dg_server();
  s->cfg = *cfg;
  dg_default_params(&s->prm);
  s->prm.gamma = cfg->gamma;
  s->prm.R = cfg->R;
  s->prm.Pr = cfg->Pr;
  s->prm.dfl = cfg->dfl;
  s->prm.precision = cfg->precision;
  s->prm.viscous = 1;
  s->prm.shock_capturing = 0;
  cudaGetDevice(&s->device);
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  // case set-up kernels are short: they get the higher priority, so that they
  // start between the blocks of the step kernels instead of after them
  int prio_low = 0, prio_high = 0;
  cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->setup_stream, cudaStreamNonBlocking, prio_high);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_cases, sizeof(CaseData) * cfg->max_cases);
  if (e == cudaSuccess) e = cudaMemset(s->d_cases, 0, sizeof(CaseData) * cfg->max_cases);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_cases, 2 * sizeof(CaseData) * cfg->max_cases);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaEventCreate(&s->step_ev[b]);
    if (e == cudaSuccess) e = cudaEventCreate(&s->step_t0[b]);
  }
  s->slots.resize(cfg->max_cases);
  for (auto& sl : s->slots)
    if (e == cudaSuccess) e = cudaMallocHost(&sl.staging, sizeof(CaseData));
  if (e != cudaSuccess) {
    dg_server_destroy(s);
    return set_error(e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,
                     std::string("dg_server_create: ") + cudaGetErrorString(e));
  }
  for (int N = 1; N <= NMAX; ++N) {
    if (cfg->pool_elems[N] <= 0) continue;
    Pool P;
    P.N = N;
    std::string msg;
    const int st = create_pool_ctx(&P.ctx, N, cfg->pool_elems[N], &s->prm, s->stream, msg);
    if (st != DG_OK) {
      dg_server_destroy(s);
      return set_error(st, "dg_server_create: " + msg);
    }
    P.ctx->cases = s->d_cases;
    P.ctx->n_case_slots = cfg->max_cases;
    P.ctx->cfg.persistent = cfg->persistent ? 1 : 0;
    cudaError_t pe = cudaStreamCreateWithFlags(&P.branch, cudaStreamNonBlocking);
    if (pe == cudaSuccess) pe = cudaMalloc(&P.ctx->elem_list, sizeof(int) * cfg->pool_elems[N]);
    if (pe == cudaSuccess) pe = cudaMalloc(&P.ctx->side_list, sizeof(int) * 3 * cfg->pool_elems[N]);
    for (int b = 0; b < 2 && pe == cudaSuccess; ++b) {
      pe = cudaMallocHost(&P.h_elist[b], sizeof(int) * cfg->pool_elems[N]);
      if (pe == cudaSuccess) pe = cudaMallocHost(&P.h_slist[b], sizeof(int) * 3 * cfg->pool_elems[N]);
    }
    if (pe == cudaSuccess && cfg->persistent) {
      pe = cudaMallocHost(&P.h_timeout, 2 * sizeof(int));
      if (pe == cudaSuccess) P.h_timeout[0] = P.h_timeout[1] = 0;
    }
    if (pe == cudaSuccess) pe = cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming);
    if (pe == cudaSuccess) pe = cudaEventCreateWithFlags(&P.join, cudaEventDisableTiming);
    if (pe != cudaSuccess) {
      s->pools[N] = P;
      dg_server_destroy(s);
      return set_error(DG_ERR_CUDA, std::string("dg_server_create: ") + cudaGetErrorString(pe));
    }
    P.elems.init(cfg->pool_elems[N]);
    P.sides.init(3 * cfg->pool_elems[N]);
    s->pools[N] = P;
  }
  if (s->pools.empty()) {
    dg_server_destroy(s);
    return set_error(DG_ERR_ARG, "dg_server_create: no pool (all pool_elems are 0)");
  }
  s->worker = std::thread(worker_loop, s);
  s->preparer = std::thread(prepare_loop, s);
  *out = s;
  return DG_OK;
}

int dg_submit(dg_server* s, const dg_case_desc* d, int64_t* ticket) {
  if (!s || !d || !ticket) return set_error(DG_ERR_ARG, "dg_submit: NULL argument");
  const dg_mesh_desc& m = d->mesh;
  if (!m.corner_vid || !m.xyz || !d->U0 || m.n_elems < 1 || m.N < 1 || m.N > NMAX)
    return set_error(DG_ERR_ARG, "dg_submit: incomplete case description");
  if (!(d->t_end > 0) || !(d->mu >= 0) || !(d->cfl > 0) ||
      (d->riemann != DG_RIEMANN_ROE && d->riemann != DG_RIEMANN_LF))
    return set_error(DG_ERR_ARG, "dg_submit: bad t_end, mu, cfl or riemann");
  if (m.face_bc) return set_error(DG_ERR_ARG, "dg_submit: serving takes periodic meshes only");
  if (m.nodes != DG_NODES_LGL) return set_error(DG_ERR_ARG, "dg_submit: serving takes LGL-node cases only");
  Request r;
  r.N = m.N;
  r.E = m.n_elems;
  if (!slot_fits(s, r)) return set_error(DG_ERR_ARG, "dg_submit: no pool of this degree can hold the case");
  const int64_t n3 = (int64_t)(m.N + 1) * (m.N + 1) * (m.N + 1);
  r.cvid.assign(m.corner_vid, m.corner_vid + r.E * 8);
  r.xyz.assign(m.xyz, m.xyz + r.E * n3 * 3);
  r.U0.assign(d->U0, d->U0 + r.E * n3 * 5);
  r.t_end = d->t_end;
  r.mu = d->mu;
  r.cfl = d->cfl;
  r.riemann = d->riemann;
  r.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->m);
    if (s->stop) return set_error(DG_ERR_STATE, "dg_submit: server stopped: " + s->worker_error);
    r.ticket = s->next_ticket++;
    *ticket = r.ticket;
    s->pending.push_back(std::move(r));
  }
  s->cv.notify_all();
  return DG_OK;
}

int dg_poll(dg_server* s, int64_t ticket, double* U_out, double* stats) {
  if (!s) return set_error(DG_ERR_ARG, "dg_poll: NULL server");
  std::lock_guard<std::mutex> lk(s->m);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) {
    if (s->running.count(ticket) || s->admitting.count(ticket)) return DG_PENDING;
    for (const auto& r : s->pending)
      if (r.ticket == ticket) return DG_PENDING;
    if (s->stop && !s->worker_error.empty()) return set_error(DG_ERR_CUDA, "dg_poll: " + s->worker_error);
    return set_error(DG_ERR_ARG, "dg_poll: unknown ticket");
  }
  const Result& res = it->second;
  if (res.stats[7] == 2.0) return set_error(DG_ERR_MESH, "dg_poll: " + s->worker_error);
  if (U_out && !res.U.empty()) memcpy(U_out, res.U.data(), sizeof(double) * res.U.size());
  if (stats) memcpy(stats, res.stats, sizeof(res.stats));
  return DG_OK;
}

int dg_server_stats(dg_server* s, double* out) {
  if (!s || !out) return set_error(DG_ERR_ARG, "dg_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(s->m);
  out[0] = s->stat_steps;
  out[1] = s->stat_finished;
  out[2] = (double)s->running.size();
  out[3] = (double)(s->pending.size() + s->ready.size());
  out[4] = s->stat_captures;
  out[5] = s->stat_dofstages;
  out[6] = s->stat_device_s;
  out[7] = s->stat_capture_s;
  out[8] = s->stat_prepare_s;
  out[9] = s->stat_insert_s;
  return DG_OK;
}

}  // extern "C"
