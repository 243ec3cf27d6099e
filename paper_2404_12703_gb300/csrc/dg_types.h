// dg_types.h -- internal data structures of libdg shared by the host code and
// the kernels (no CUDA-specific types beyond the runtime API).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dg.h"

namespace dg {

constexpr int NMAX = 7;
constexpr int NPMAX = NMAX + 1;

// 1D operators of one degree N on the solution nodes (LGL or Gauss-Legendre),
// rounded to double from extended-precision values (Sec. 2.2, Eq. dgsem and
// the operator definitions after it), and the LGL operators of the geometry.
struct Ops {
  double x[NPMAX], w[NPMAX], winv[NPMAX];
  double D[NPMAX * NPMAX];       // D[i][a] = l_a'(x_i)
  double Dhat[NPMAX * NPMAX];    // -(w_a / w_i) D[a][i]
  double Dsplit[NPMAX * NPMAX];  // 2 D + corner corrections (diagonal zero), LGL
  double Dlo[NPMAX * NPMAX];     // D - (double)D (double-double tail)
  double Vinv[NPMAX * NPMAX];    // nodal -> orthonormal Legendre modes
  double Lp[NPMAX], Lm[NPMAX];   // l_i(+1), l_i(-1) (unit vectors on LGL)
  // geometry: the LGL derivative matrix (double-double) and the
  // interpolation from the LGL nodes to the solution nodes (double-double;
  // the identity on LGL)
  double Dg[NPMAX * NPMAX], Dg_lo[NPMAX * NPMAX];
  double Ig[NPMAX * NPMAX], Ig_lo[NPMAX * NPMAX];
};

// Scalars kept on the device (one block, one per context).
struct DevScalars {
  double dt;                 // time step of the current step
  double t;                  // time of the state
  double dt_fixed;           // > 0: fixed step
  unsigned long long lam_c;  // max convective spectral radius (bits of a positive double)
  unsigned long long lam_v;  // max viscous spectral radius
  int nonfinite;             // sticky: a non-finite value met in the CFL reduction
  int mesh_error;            // set by the map construction kernels
  int pad[2];
  double kin[4];             // kinetic-energy reductions
  double ref_p, ref_H, ref_T;  // reference state of the shifted primitives (0 in FP64)
  double t_end;              // > 0: CFL steps are clipped to end on t_end
  long long steps;           // steps taken with dt > 0
  double dt_cfl;             // CFL time step of the current state (dg_time_step)
  double ref_rho, ref_E;     // reference density and total energy (state at rest)
  float f_ref_p, f_ref_H, f_ref_T, f_pad;  // FP32 copies for the FP32-bulk kernels
  // the context's reference state, kept while dg_rhs evaluates another state
  double keep_ref[5];
  float keep_f_ref[4];
  // grid-wide barrier of the persistent stage kernel (arrivals, generation;
  // zeroed before each launch) and its sticky timeout flag
  unsigned bar[2];
  int timeout;
  int pad2;
  // two-kernel FP32-bulk steps: the spectral radii of the state a step ends
  // with, reduced by its last stage (or by the face-data pass of a new
  // state) for the next step's time step (bits of positive doubles)
  unsigned long long lam_c_next, lam_v_next;
};

// Per-case data of a serving pool (device, one entry per case slot).
struct CaseData {
  double dt, t, t_end;
  double mu, lam;              // viscosity and heat conductivity (0: Euler)
  double ref_p, ref_H, ref_T;  // reference state of the shifted primitives
  double ref_rho, ref_E;
  double cfl, dfl;
  unsigned long long lam_c, lam_v;  // CFL reductions (bits of positive doubles)
  int riemann;
  int active;     // 1 while the case is resident
  int nonfinite;  // sticky
  int steps;      // completed steps
  int N;          // polynomial degree of the case's pool
  int paused;     // 1: the case sits out the next step (priority policy)
  float f_mu, f_lam, f_ref_p, f_ref_H, f_ref_T, f_pad;  // FP32 copies (FP32-bulk kernels)
};

// Launch configuration of the stage kernels (the autotuner's choice).
struct StageConfig {
  int lift_epb = 0;     // elements per block of the lifting kernel (0: default)
  int vol_epb = 0;      // elements per block of the volume kernel (0: default)
  int vol_pairs = -1;   // 1: line-pair two-point sums, 0: per node, -1: default
  int side_block = 256; // threads per block of the side kernels (128 or 256)
  // FP32-bulk stage: 0 the two-kernel stage where it applies (periodic LGL
  // meshes of a single context), else the four-kernel one; 1 always the
  // four-kernel stage
  int stage_form = 0;
  int prefetch = 1;     // two-kernel stage: L2 prefetch of the next wave's element data (0: off)
  int persistent = 0;   // two-kernel stage: one persistent launch per step for all stages (1)
};

// Per-stage launch parameters of the RHS kernels.
struct StageArgs {
  int E, S;
  const double* U;       // [E][5][n3] internal state
  const double* metric;  // [E][10][n3]: J a^d_c at d*3+c, then 1/J
  const float* metric32;  // the same, rounded to FP32 (FP32-bulk)
  const double* nrm;     // [S][4][n2]: s n (3), s
  const float* nrm32;    // [S][7][n2]: s n (3), unit n (3), s, in FP32 (FP32-bulk)
  const int* elem_side;  // [E][6]
  const int2* side_e;    // [S] (eM, eS)
  const int* side_f;     // [S] fM | fS << 4 | flip << 8
  double* g;             // [E][12][n3] lifted gradients
  double* lflux;         // [S][12][n2]
  double* fstar;         // [S][5][n2]
  float* g32;            // FP32-bulk copies of the three arrays above
  float* lflux32;
  float* fstar32;
  double* alpha;         // [E]
  const double* fvmetric;  // [E][3][n2][(n-1)*3] sub-cell interface metrics
  const Ops* ops;
  double gamma, gm1, Rinv, mu, lam;
  float f_gamma, f_gm1, f_Rinv, f_mu, f_lam;  // FP32 copies (FP32-bulk kernels)
  // Sutherland's law: mu(T) at every node, lambda = kappa mu(T)
  int sutherland;
  double inv_Tref, kappa;
  float f_inv_Tref, f_kappa;
  int riemann, viscous, shock;
  double alpha_min, alpha_max, alpha_force;
  // output: either Ut (mode 0) or the RK update (mode 1)
  double* Ut;       // [E][5][n3] internal layout
  double* Urk;      // state updated in place
  double* dU;       // RK register
  const DevScalars* scal;
  double rkA, rkB;
  float f_rkA;  // rkA in FP32 (the two-kernel FP32-bulk stage's register update)
  int first_stage;
  // serving pools: case of every element / side (-1: free slot) and the
  // per-case data; null for a single-mesh context
  const int* elem_case;
  const int* side_case;
  const CaseData* cases;
  // serving pools: the occupied elements and sides; the launch grids cover
  // these (E and S are then their counts), so freed ranges cost nothing
  const int* elem_list;
  const int* side_list;
  // boundary conditions: row of every side (-1: inner side), rows [n][9]
  const int* side_bc;
  const double* bcdata;
  // sponge zone (null: none): sigma [E][n3], base state [E][5][n3]
  const double* sponge_sigma;
  const double* sponge_base;
  // Gauss-Legendre nodes: face values of the state [S][2][5][n2] and of the
  // lifted gradients [S][2][12][n2] (master, slave; master face frame)
  double* Ufc;
  double* gfc;
  float* gfc32;
  // manufactured-solution source (Sec. 5.1): on/off, amplitude, speed, the
  // solution nodes' coordinates [E][n3][3] and the stage's RK c coefficient
  int source;
  double src_A, src_a;
  const double* xyzs;
  double rkC;
  // two-kernel FP32-bulk stage (dg_fused32.cuh): face traces [S][2][n2][8],
  // partial viscous fluxes [S][2][n2][4], BR1 means q* [S][n2][4]; the
  // element kernel's epilogue on / off; L2 prefetch distance in blocks (0: off)
  float* tr32;
  float* pfv32;
  float* qs32;
  float* wv32;  // the lifting's volume sums of the state [E][12][n3] (Eq. lifting, before 1/J)
  int epilogue;
  // the element kernel's epilogue (and k_fprep) also reduces the CFL radii
  // of the state it prepares into scal->lam_*_next (f_cflkv: max(4/3,
  // gamma / Pr) mu in FP32)
  int cfl_out;
  float f_cflkv;
  DevScalars* scal_cfl;  // the step scalars the reduction writes (scal, writable)
  int prefetch;
  int elem_off;  // k_fprep without an element list: elements elem_off .. elem_off + E - 1
  int E_all;     // elements of the context's arrays (E, or a serving pool's capacity)
};

}  // namespace dg

struct dg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;      // user stream: all work is ordered on it
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  cudaStream_t pool_stream = nullptr;  // non-null: arrays from the library pool, in this stream's order
  int N = 0, n = 0, n2 = 0, n3 = 0;
  int64_t E = 0, S = 0;
  dg_params prm{};
  // device memory
  double* U = nullptr;       // [E][5][n3]
  double* dU = nullptr;      // [E][5][n3]
  double* Ut = nullptr;      // [E][5][n3] scratch for dg_rhs
  double* Upub = nullptr;    // [E][n3][5] scratch for layout conversion
  double* metric = nullptr;  // [E][10][n3]
  float* metric32 = nullptr;  // [E][10][n3] rounded to FP32 (FP32-bulk)
  double* g = nullptr;       // [E][12][n3]
  double* nrm = nullptr;     // [S][4][n2]
  float* nrm32 = nullptr;    // [S][7][n2]: s n, unit n, s in FP32 (FP32-bulk)
  double* lflux = nullptr;   // [S][12][n2]
  double* fstar = nullptr;   // [S][5][n2]
  float* g32 = nullptr;      // FP32-bulk: [E][12][n3]
  float* lflux32 = nullptr;  // FP32-bulk: [S][12][n2]
  float* fstar32 = nullptr;  // FP32-bulk: [S][5][n2]
  double* alpha = nullptr;   // [E]
  double* fvmetric = nullptr;  // [E][3][n2][(n-1)*3]
  double* cflgeo = nullptr;    // [E][4][n3]: |J a^d| (d = 0..2), sum_d |J a^d|^2
  int* elem_side = nullptr;  // [E][6]
  int2* side_e = nullptr;    // [S]
  int* side_f = nullptr;     // [S]
  int* side_bc = nullptr;    // [S] boundary-condition row (-1: inner side)
  double* bcdata = nullptr;  // [n_bc][9] boundary-condition rows (type, 8 parameters)
  int n_bc = 0;
  double* sponge_sigma = nullptr;  // [E][n3]
  double* sponge_base = nullptr;   // [E][5][n3] internal layout
  dg::Ops* ops = nullptr;    // device copy of the operators of degree N
  dg::DevScalars* scal = nullptr;
  double* kin_part = nullptr;  // [blocks][3] per-block kinetic-energy sums (dg_kinetic)
  int kin_part_blocks = 0;
  dg::DevScalars* scal_host = nullptr;  // pinned mirror
  int64_t cap_E = 0, cap_S = 0;  // allocated element and side capacity (a pool's, or E and S)
  int gauss = 0;              // solution on Gauss-Legendre nodes (standard DGSEM)
  double stage_c = 0.0;       // RK c coefficient of the stage being enqueued (stage time)
  int stage_cfl = 0;          // the stage (or face-data pass) being enqueued reduces the next CFL radii
  bool lam_next_valid = false;  // scal->lam_*_next hold the radii of the current state
  int rk_ns = 0;              // low-storage RK scheme of dg_step (0: the default five-stage one)
  double rk_a[32] = {}, rk_b[32] = {}, rk_c[32] = {};
  double* xyzs = nullptr;     // [E][n3][3] coordinates of the solution nodes
  double* Ufc = nullptr;      // GL: [S][2][5][n2] face values of the state
  double* gfc = nullptr;      // GL: [S][2][12][n2] face values of the lifted gradients
  float* gfc32 = nullptr;     // GL, FP32-bulk: the same in FP32
  // two-kernel FP32-bulk stage: face data (see StageArgs); traces_valid: the
  // face data hold the current state's (set by a step's last stage, cleared by
  // anything else that writes the state or the face arrays)
  float* tr32 = nullptr;
  float* pfv32 = nullptr;
  float* qs32 = nullptr;
  float* wv32 = nullptr;  // the lifting's volume sums of the face data's state
  bool traces_valid = false;
  int64_t bytes = 0;
  double t_host = 0.0;
  bool state_set = false;
  // CUDA graphs of one time step (CFL or fixed dt)
  cudaGraphExec_t step_graph = nullptr;
  int step_graph_kind = -1;
  // per-kernel event timing (dg_profile_step); null when not profiling
  struct Profiler* prof = nullptr;
  // serving pool (null for a single-mesh context): case maps and case table
  int* elem_case = nullptr;
  int* side_case = nullptr;
  dg::CaseData* cases = nullptr;
  int n_case_slots = 0;
  dg::StageConfig cfg;       // launch configuration of the stage kernels
  bool tuned = false;        // cfg chosen by the autotuner
  bool tune_keep_mapping = false;  // autotune elements per block and side blocks only
                                   // (results then do not depend on the tuning)
  int* elem_list = nullptr;  // occupied elements / sides of a serving pool (device)
  int* side_list = nullptr;
  int64_t n_elem_list = 0, n_side_list = 0;
};

// Event pairs around each kernel launch, grouped by kernel kind.
struct Profiler {
  static constexpr int MAX_EV = 256;
  cudaEvent_t ev[MAX_EV][2];
  int slot[MAX_EV];
  int used = 0;
  double ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};
