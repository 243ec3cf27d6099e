// dg_launch.h -- host-side interfaces between the translation units of libdg.
#pragma once
#include <string>

#include "dg_types.h"

namespace dg {

// launch accounting (dg_launch_count)
void count_launch(int k = 1);

// kernel kinds timed by dg_profile_step
enum { PK_CFL = 0, PK_SURF_PRIMS = 1, PK_LIFT = 2, PK_SURF_FLUX = 3, PK_VOLUME = 4 };
// record an event before / after a kernel launch when c->prof is set
void prof_begin(dg_ctx* c, int kind);
void prof_end(dg_ctx* c);

// records the thread's last error message and returns code
int set_error(int code, const std::string& msg);

// quadrature weights of degree N (n = N + 1 entries) on the LGL nodes
// (gauss = 0) or the Gauss-Legendre nodes (gauss = 1)
void quadrature_weights(int N, int gauss, double* w);

// allocation of the side arrays once the number of sides is known
int alloc_side_arrays(dg_ctx* c, std::string& msg);

// stream-ordered allocation from the library's device memory pool (dg_api.cu)
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);

// dg_init_mesh; with pool_stream non-null the context's arrays come from the
// library pool in that stream's order and it has no pinned mirror or capture
// stream (the server's per-case contexts)
int init_mesh_impl(dg_ctx** out, const dg_mesh_desc* mesh, const dg_params* params, cudaStream_t stream,
                   cudaStream_t pool_stream);

// serving pool of capE elements with every slot free (dg_api.cu)
int create_pool_ctx(dg_ctx** out, int N, int64_t capE, const dg_params* params, cudaStream_t stream,
                    std::string& msg);

// FP32 copies of the metrics and side geometry, and the sub-cell interface
// metrics of the FV blending, from the FP64 geometry (dg_mesh.cu)
cudaError_t launch_fp32_geometry(dg_ctx* c, cudaStream_t st);
cudaError_t launch_fv_metrics(dg_ctx* c, cudaStream_t st);

// the two-kernel FP32-bulk stage serves periodic LGL meshes (no boundary
// sides): single contexts and serving pools, not the server's temporary
// per-case contexts; its face arrays exist only there
inline bool fused_eligible(const dg_ctx* c) {
  return !c->gauss && !c->pool_stream && c->n_bc == 0;
}
// the stage launches of c use the two-kernel FP32-bulk form
inline bool fused_active(const dg_ctx* c) {
  return c->prm.precision == DG_FP32_BULK && c->tr32 && fused_eligible(c) && c->cfg.stage_form != 1;
}
// face data of the context's state for the two-kernel stage (dg_rhs.cu):
// every element (a pool's occupied ones), or with E >= 0 the elements
// e0 .. e0 + E - 1, on stream st (null: the context's stream)
cudaError_t launch_fprep(dg_ctx* c, const double* U, int64_t e0 = 0, int64_t E = -1, cudaStream_t st = nullptr);

// the steps of a two-kernel FP32-bulk context run as one persistent launch
inline bool persist_active(const dg_ctx* c) { return fused_active(c) && c->cfg.persistent == 1; }
// the CFL reduction of a step is part of the previous step's last stage: the
// two-kernel FP32-bulk steps of a single context launched per kernel (not
// serving pools, whose cases each take their own time step, and not the
// persistent launch)
inline bool cfl_fused(const dg_ctx* c) { return fused_active(c) && !persist_active(c) && !c->elem_case; }
// one persistent launch of every stage of a step (dg_rhs.cu); spin: polls of
// a barrier wait before it gives up; extra: the barrier test hook (0)
constexpr unsigned PERSIST_SPIN = 5000000u;  // about a second of 200 ns polls
cudaError_t launch_persist(dg_ctx* c, int ns, const double* A, const double* B, const double* C, unsigned extra = 0,
                           unsigned spin = PERSIST_SPIN);

// the arrays a parameter set needs (FP64 or FP32 working arrays, FV
// interface metrics), allocated and formed on first use (dg_api.cu)
int ensure_arrays(dg_ctx* c, const dg_params* p, std::string& msg);

// device mesh set-up (dg_mesh.cu)
// h_face_bc (may be null): [E][6] boundary-condition row + 1 of every face (0: inner)
int build_mesh(dg_ctx* c, const int64_t* h_cvid, const double* h_xyz, const int* h_face_bc, std::string& msg);

// one evaluation of the right-hand side (dg_rhs.cu).
//   mode 0: write Ut (internal layout) into c->Ut for state U
//   mode 1: RK stage update of c->U / c->dU with coefficients (A, B)
cudaError_t launch_rhs(dg_ctx* c, const double* U, int mode, double rkA, double rkB, int first_stage);

// CFL reduction: writes dt (and advances nothing); fixed dt if dt_fixed > 0
// report_only: writes the CFL time step to dt_cfl instead of taking the step
cudaError_t launch_cfl(dg_ctx* c, bool report_only);
// two-kernel FP32-bulk steps: the time step from the radii that the previous
// step's last stage (or the face-data pass of a new state) reduced into
// lam_*_next, which it clears for the step's own last stage
cudaError_t launch_dt_next(dg_ctx* c);
// clears lam_*_next before a face-data pass reduces a new state's radii
cudaError_t launch_clear_next(dg_ctx* c);

// raises the dynamic shared-memory limits of the kernels of degree N
cudaError_t init_kernel_attributes(int N);

// stage kernels of one degree, both precisions (dg_stage_n<K>.cu)
#define DG_DECLARE_STAGE_N(K)                                                                    \
  cudaError_t stage_attrs_n##K();                                                                \
  cudaError_t stage_launch_n##K(dg_ctx* c, const double* U, int mode, double A, double B, int f); \
  cudaError_t stage_autotune_n##K(dg_ctx* c, double* ms);                                        \
  cudaError_t fprep_n##K(dg_ctx* c, const double* U, int64_t e0, int64_t E, cudaStream_t st);           \
  cudaError_t persist_n##K(dg_ctx* c, int ns, const double* A, const double* B, const double* C, unsigned extra, \
                           unsigned spin);
DG_DECLARE_STAGE_N(1)
DG_DECLARE_STAGE_N(2)
DG_DECLARE_STAGE_N(3)
DG_DECLARE_STAGE_N(4)
DG_DECLARE_STAGE_N(5)
DG_DECLARE_STAGE_N(6)
DG_DECLARE_STAGE_N(7)
#undef DG_DECLARE_STAGE_N

// autotuner of the stage kernels' launch variants (ms: 8 timings, see
// stage_autotune in dg_stage.cuh)
cudaError_t launch_autotune(dg_ctx* c, double* ms);

// reference state of the shifted primitives from the context's state
cudaError_t launch_refs(dg_ctx* c);

// layout conversion public [E][n3][5] <-> internal [E][5][n3]
cudaError_t launch_to_internal(dg_ctx* c, const double* pub, double* internal);
cudaError_t launch_to_public(dg_ctx* c, const double* internal, double* pub);

// kinetic energy reductions into c->scal->kin (U internal, Ut internal or null)
// the grid of the kinetic-energy reduction (its per-block sums need that many [3] entries)
int kinetic_blocks(dg_ctx* c);
cudaError_t launch_kinetic(dg_ctx* c, const double* U, const double* Ut);

// the integer-pipe binary64 <-> binary32 conversions over n values (dg_rhs.cu)
cudaError_t launch_convert_check(const double* in, float* out, double* back, int64_t n, cudaStream_t st);

// verification copies
cudaError_t launch_debug_metrics(dg_ctx* c, double* Ja, double* J);
cudaError_t launch_debug_maps(dg_ctx* c, int* nbr, int* nodes);
cudaError_t launch_debug_grad(dg_ctx* c, double* out);
cudaError_t launch_debug_fstar(dg_ctx* c, double* out);

}  // namespace dg
