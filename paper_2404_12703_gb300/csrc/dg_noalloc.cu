// dg_noalloc.cu -- kinetic-energy diagnostics of a caller-owned state without
// any device allocation.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// handed out up front by their own arena or pool allocator, and loops that
// must not take the implicit device synchronisation a cudaMalloc / cudaFree
// can cause while other work is in flight.  dg_kinetic_noalloc() serves them:
// its scratch (one partial sum per element) lives in a file-scope device
// array that every GPU loading this library holds until the process exits,
// and the caller passes every input and output buffer.
#include <mutex>

#include "dg_common.cuh"
#include "dg_launch.h"

namespace dg {

// Largest element count the scratch array can hold: 64^3 elements.
constexpr int64_t KIN_NOALLOC_MAX_ELEMS = 262144;

// Three partial sums per element (E_k, dE_k/dt, volume): 6 MiB.  Shared by
// every call; a call overwrites the entries it reads before reading them.
static __device__ __align__(256) double g_kin_scratch[3 * KIN_NOALLOC_MAX_ELEMS];

struct QuadWeights {
  double w[NPMAX];
};

constexpr int KIN_THREADS = 128;

// Pass 1: one block per element, fixed-order tree reduction, one write of the
// element's three sums.
template <int N>
__global__ void __launch_bounds__(KIN_THREADS) k_kin_noalloc_elem(const double* __restrict__ U,
                                                                  const double* __restrict__ J,
                                                                  const double* __restrict__ Ut, QuadWeights qw,
                                                                  double* __restrict__ part) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  __shared__ double s[3][KIN_THREADS];
  const int64_t e = blockIdx.x;
  double ek = 0, rate = 0, vol = 0;
  for (int t = threadIdx.x; t < n3; t += KIN_THREADS) {
    const double wq = qw.w[t % n] * qw.w[(t / n) % n] * qw.w[t / n2] * J[e * n3 + t];
    const double* u = U + (e * n3 + t) * 5;
    const double r = u[0], vx = u[1] / r, vy = u[2] / r, vz = u[3] / r;
    const double v2 = vx * vx + vy * vy + vz * vz;
    vol += wq;
    ek += wq * r * v2 / 2;
    if (Ut) {
      const double* ut = Ut + (e * n3 + t) * 5;
      rate += wq * (vx * ut[1] + vy * ut[2] + vz * ut[3] - v2 * ut[0] / 2);
    }
  }
  s[0][threadIdx.x] = ek;
  s[1][threadIdx.x] = rate;
  s[2][threadIdx.x] = vol;
  __syncwarp();
  __syncthreads();
  for (int h = KIN_THREADS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s[0][threadIdx.x] += s[0][threadIdx.x + h];
      s[1][threadIdx.x] += s[1][threadIdx.x + h];
      s[2][threadIdx.x] += s[2][threadIdx.x + h];
    }
    __syncwarp();
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[e * 3 + 0] = s[0][0];
    part[e * 3 + 1] = s[1][0];
    part[e * 3 + 2] = s[2][0];
  }
}

// Pass 2: one block adds the element sums in a fixed order and normalises.
__global__ void __launch_bounds__(256) k_kin_noalloc_final(int64_t E, const double* __restrict__ part,
                                                           double* __restrict__ out) {
  __shared__ double s[3][256];
  double a = 0, b = 0, c = 0;
  for (int64_t e = threadIdx.x; e < E; e += 256) {
    a += part[e * 3 + 0];
    b += part[e * 3 + 1];
    c += part[e * 3 + 2];
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
    out[0] = s[0][0] / s[2][0];
    out[1] = s[1][0] / s[2][0];
    out[2] = s[2][0];
  }
}

// Device address of the scratch array, looked up once per device.
static std::mutex g_addr_mutex;
static double* g_addr[64] = {nullptr};

static cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_kin_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace dg

using namespace dg;

extern "C" int dg_kinetic_noalloc(int N, int nodes, int64_t n_elems, const double* U, const double* J,
                                  const double* Ut, double* out, void* stream) {
  if (N < 1 || N > NMAX) return set_error(DG_ERR_ARG, "dg_kinetic_noalloc: N must be in [1, 7]");
  if (nodes != DG_NODES_LGL && nodes != DG_NODES_GAUSS)
    return set_error(DG_ERR_ARG, "dg_kinetic_noalloc: nodes must be DG_NODES_LGL or DG_NODES_GAUSS");
  if (n_elems < 1) return set_error(DG_ERR_ARG, "dg_kinetic_noalloc: n_elems must be positive");
  if (n_elems > KIN_NOALLOC_MAX_ELEMS)
    return set_error(DG_ERR_ARG, "dg_kinetic_noalloc: n_elems exceeds the maximum of 262144 elements "
                                 "that its built-in scratch holds; use dg_kinetic instead");
  if (!U || !J || !out) return set_error(DG_ERR_ARG, "dg_kinetic_noalloc: U, J and out must not be NULL");
  double* part = nullptr;
  cudaError_t e = scratch_address(&part);
  if (e != cudaSuccess)
    return set_error(DG_ERR_CUDA, std::string("dg_kinetic_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  QuadWeights qw;
  for (int i = 0; i < NPMAX; ++i) qw.w[i] = 0.0;
  quadrature_weights(N, nodes == DG_NODES_GAUSS ? 1 : 0, qw.w);  // the weights of the state's node set
  cudaStream_t st = (cudaStream_t)stream;
  switch (N) {
    case 1: k_kin_noalloc_elem<1><<<(unsigned)n_elems, KIN_THREADS, 0, st>>>(U, J, Ut, qw, part); break;
    case 2: k_kin_noalloc_elem<2><<<(unsigned)n_elems, KIN_THREADS, 0, st>>>(U, J, Ut, qw, part); break;
    case 3: k_kin_noalloc_elem<3><<<(unsigned)n_elems, KIN_THREADS, 0, st>>>(U, J, Ut, qw, part); break;
    case 4: k_kin_noalloc_elem<4><<<(unsigned)n_elems, KIN_THREADS, 0, st>>>(U, J, Ut, qw, part); break;
    case 5: k_kin_noalloc_elem<5><<<(unsigned)n_elems, KIN_THREADS, 0, st>>>(U, J, Ut, qw, part); break;
    case 6: k_kin_noalloc_elem<6><<<(unsigned)n_elems, KIN_THREADS, 0, st>>>(U, J, Ut, qw, part); break;
    default: k_kin_noalloc_elem<7><<<(unsigned)n_elems, KIN_THREADS, 0, st>>>(U, J, Ut, qw, part); break;
  }
  k_kin_noalloc_final<<<1, 256, 0, st>>>(n_elems, part, out);
  count_launch(2);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_error(DG_ERR_CUDA, std::string("dg_kinetic_noalloc: launch: ") + cudaGetErrorString(e));
  return DG_OK;
}
