/*
 * dg.h -- C ABI of libdg: the DGSEM time derivative Ut = R(U) of the
 * compressible Navier-Stokes equations on unstructured, curved hexahedral
 * meshes and its low-storage Runge-Kutta time stepping, on one NVIDIA GB300
 * (sm_103a).  The method is that of GALAEXI (arXiv 2404.12703):
 *
 *   Sec. 2.1  Eq. nse, stress tensor, Fourier law, Eqs. eos_p / eos_T
 *   Sec. 2.2  curl-form metrics, Eq. transformed_goveq, Eq. weak_form,
 *             Eq. ansatz (LGL nodes), Eq. dgsem (VolInt, FillFlux, SurfInt,
 *             ApplyJac), split-form KEP volume integral, BR1 lifting
 *             (Eq. lifting), five-stage low-storage RK (Time integration)
 *   Sec. 2.3  a-priori indicator and convex DG / FV sub-cell blending
 *   Sec. 3.3  / App. A  ProlongToFace, FillFlux, SurfInt, ApplyJac
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns a status (DG_OK = 0, negative on error).  Nothing
 *    throws across the ABI.  After an error the context keeps its last
 *    consistent state; dg_last_error() gives a human-readable message.
 *  - Node index inside an element: node = i + n*(j + n*k), n = N + 1,
 *    i along the element's local xi direction.  Public state layout:
 *    U[e][node][v], v = (rho, rho u, rho v, rho w, rho e), float64.
 *  - Input pointers are borrowed for the duration of the call only.  Output
 *    buffers belong to the caller.  The library owns (and frees in
 *    dg_destroy) all device memory it allocates.
 *  - "Device pointer" means memory on the device the context was created on.
 *    Work is enqueued on the context's stream (see dg_init_mesh); calls that
 *    return data to the host synchronise that stream.
 *  - Every face either has exactly one partner face with the same four
 *    distinct corner ids or carries a boundary condition (dg_mesh_desc
 *    face_bc).  A periodic direction needs at least three elements: with two,
 *    the faces across the other directions of both layers share all corner ids.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DG_OK = 0,
  DG_ERR_ARG = -1,        /* invalid argument (null pointer, N out of range, ...) */
  DG_ERR_MESH = -2,       /* faces do not pair up (nor carry a condition)       */
  DG_ERR_OOM = -3,        /* device allocation failed                           */
  DG_ERR_CUDA = -4,       /* a CUDA runtime call failed                         */
  DG_ERR_NONFINITE = -5,  /* the time-step reduction met a NaN / Inf            */
  DG_ERR_TIMEOUT = -6,    /* a bounded device-side wait gave up                 */
  DG_ERR_STATE = -7,      /* call not valid in the context's current state      */
  DG_PENDING = 1          /* serving: request not finished yet                  */
};

enum { DG_RIEMANN_ROE = 0, DG_RIEMANN_LF = 1 };
enum { DG_FP64 = 0, DG_FP32_BULK = 1 };

/* Physical and numerical parameters (Sec. 2.1 - 2.3). */
typedef struct {
  double gamma;          /* ratio of specific heats                               */
  double R;              /* specific gas constant                                 */
  double Pr;             /* Prandtl number                                        */
  double mu;             /* dynamic viscosity (with sutherland: its value at T_ref) */
  int riemann;           /* DG_RIEMANN_ROE (no entropy fix) or DG_RIEMANN_LF      */
  int viscous;           /* 0: Euler; 1: Navier-Stokes with BR1 lifting            */
  int shock_capturing;   /* 1: Hennemann indicator + FV sub-cell blending         */
  double alpha_min;      /* blending factors below this are set to 0              */
  double alpha_max;      /* upper bound of the blending factor                    */
  double cfl, dfl;       /* convective / viscous time-step factors                */
  int precision;         /* DG_FP64 or DG_FP32_BULK                               */
  double alpha_force;    /* < 0: use the indicator; >= 0: every element uses this
                            blending factor (verification)                       */
  int sutherland;        /* 1: mu(T) = mu 1.4042 (T/T_ref)^(3/2) / (T/T_ref + 0.4042)
                            at every node (Eq. sutherland), lambda following mu at
                            constant Pr; 0: constant mu.  Standalone contexts only:
                            the server's cases use a constant mu                 */
  double T_ref;          /* Sutherland reference temperature (> 0)                */
  int source;            /* DG_SOURCE_NONE, or DG_SOURCE_MMS: the source of the
                            manufactured solution of Sec. 5.1 (Eq. mms), added to
                            Ut at every node in FP64 at the stage time: with
                            phi = 2 pi (x + y + z - a t), density and momentum
                            components 2 + A sin(phi), total energy their square;
                            constant viscosity only (DG_ERR_ARG with sutherland) */
  double source_A;       /* its amplitude A (Sec. 5.1: 0.1)                      */
  double source_a;       /* its advection speed a (Sec. 5.1: 1)                  */
} dg_params;

enum { DG_SOURCE_NONE = 0, DG_SOURCE_MMS = 1 };

/* Fills p with the defaults: gamma 1.4, R 1, Pr 0.72, mu 1/1600, Roe, viscous,
   no shock capturing, alpha in [1e-3, 0.5], CFL = DFL = 0.9, FP64. */
void dg_default_params(dg_params* p);

/* Mesh description (host memory).
   corner_vid[e][c]: vertex id of corner c = bi + 2 bj + 4 bk of element e,
     where bi = 0 for i = 0 and 1 for i = N (likewise j, k).  Faces are
     matched by their sets of corner ids; periodic images must share ids.
   xyz[e][node][3]: physical coordinates of the LGL nodes (Eq. ansatz): the
     geometry, a polynomial of degree N per element, for both node sets. */
typedef struct {
  int N;                       /* polynomial degree, 1 <= N <= 7 */
  int64_t n_elems;             /* number of elements E >= 1      */
  const int64_t* corner_vid;   /* [E][8] host                    */
  const double* xyz;           /* [E][(N+1)^3][3] host            */
  /* Boundary conditions (all optional: NULL / 0 for a mesh in which every
     face has a partner).  face_bc: [E][6] host, 0 for a face with a partner,
     k = 1..n_bc for a boundary face with condition row k - 1 of bc; bc:
     [n_bc][9] host rows (type, 8 parameters):
       DG_BC_WALL_ISOTHERMAL (u_w, v_w, w_w, T_w): no-slip wall moving with
         the (tangential) velocity u_w at temperature T_w; lifting value
         (u_w, T_w), convective flux (0, p n, p u_w.n), viscous flux at the
         wall state with the inner gradients;
       DG_BC_WALL_ADIABATIC (u_w, v_w, w_w): as above with the inner
         temperature and no heat flux;
       DG_BC_SLIP: lifting value with the normal velocity removed,
         convective flux (0, p n, 0), no viscous flux;
       DG_BC_STATE (rho, rho u, rho v, rho w, rho e): the Riemann flux and
         BR1 means between the inner and the prescribed state (farfield);
       DG_BC_OUTFLOW (p_out): as DG_BC_STATE with the outer state the inner
         density and velocity at the pressure p_out (subsonic outflow).
     The paper names wall and farfield conditions for its application
     without stating them (Sec. 6); these are the library's.  Serving
     (dg_submit) takes periodic meshes only. */
  const int* face_bc;
  int n_bc;
  const double* bc;
  /* Node set of the solution (Sec. 2.2: GL or LGL interpolation points;
     Sec. 5.1 runs the split form on LGL and the standard form on GL nodes):
       DG_NODES_LGL (0): split-form DGSEM on Legendre-Gauss-Lobatto nodes;
       DG_NODES_GAUSS (1): standard DGSEM on Legendre-Gauss nodes.  Its face
         values are interpolations with l(+-1) (ProlongToFace), its volume
         term the collocated flux divergence sum_a Dhat_ia (J a . F)_a, and
         SurfInt reaches every node of a line with lhat+-_i = l_i(+-1)/w_i.
         The metrics are the LGL curl-form polynomials evaluated at the GL
         nodes (so both elements of a face agree on its normal and free
         streams are preserved), J = det(dx/dxi) there.  No shock capturing
         and no serving (dg_submit) on GL nodes; dg_node_coords gives the
         solution nodes' coordinates. */
  int nodes;
} dg_mesh_desc;

enum { DG_NODES_LGL = 0, DG_NODES_GAUSS = 1 };

enum { DG_BC_WALL_ISOTHERMAL = 1, DG_BC_WALL_ADIABATIC = 2, DG_BC_SLIP = 3, DG_BC_STATE = 4, DG_BC_OUTFLOW = 5 };

typedef struct dg_ctx dg_ctx;

/* Builds a context for one mesh on the current CUDA device.
   On the device: element<->side maps with face orientation (flip) found from
   corner ids (Sec. 2.2 "unstructured mesh topology", App. A ProlongToFace),
   curl-form metrics J a^i and J (Sec. 2.2, Mapping the Equations) formed in
   double-double and rounded, surface normals and surface elements.
   stream: a cudaStream_t (NULL = legacy default stream) on which all later
   work of this context is enqueued.  The call synchronises before returning.
   Errors: DG_ERR_ARG for bad sizes, DG_ERR_MESH if faces do not pair up or a
   face's orientation cannot be determined, DG_ERR_OOM / DG_ERR_CUDA.
   On error *out is set to NULL. */
int dg_init_mesh(dg_ctx** out, const dg_mesh_desc* mesh, const dg_params* params, void* stream);

/* Coordinates of the solution nodes, [E][node][3] float64, on the host
   (on_device = 0) or the device (1): the LGL nodes as given, or the
   geometry polynomial evaluated at the Gauss-Legendre nodes.  Synchronises
   the context's stream. */
int dg_node_coords(dg_ctx* ctx, double* xyz, int on_device);

/* The 1D quadrature weights of the solution nodes (N + 1 values: LGL or
   Gauss-Legendre), for integrals of nodal data: sum_ijk w_i w_j w_k J_ijk f_ijk. */
int dg_quadrature_weights(const dg_ctx* ctx, double* w);

/* Changes the stream later work is enqueued on. */
int dg_set_stream(dg_ctx* ctx, void* stream);

/* Replaces the parameters (same mesh).  The precision may be changed too.
   DG_ERR_ARG for shock capturing on Gauss-Legendre nodes. */
int dg_set_params(dg_ctx* ctx, const dg_params* params);

/* Copies a state into the context and sets the time t.
   U: [E][node][5] float64, on the host (on_device = 0) or the device (1).
   Stream-ordered; a host source is copied before the call returns. */
int dg_set_state(dg_ctx* ctx, const double* U, int on_device, double t);

/* Copies the context's state out and reports its time (either may be NULL).
   Synchronises the context's stream.  Returns DG_ERR_NONFINITE if a time step
   since the last dg_set_state met a non-finite value. */
int dg_get_state(dg_ctx* ctx, double* U, int on_device, double* t);

/* Ut = R(U), Eq. dgsem with the split-form volume integral (LGL nodes) or
   the standard one (GL nodes), BR1 lifting and (if enabled, LGL only)
   sub-cell blending, for the state U_dev (device, public layout)
   or the context's own state when U_dev is NULL.  Ut_dev: caller-owned device
   buffer [E][node][5].  Stream-ordered (asynchronous). */
int dg_rhs(dg_ctx* ctx, const double* U_dev, double* Ut_dev);

/* Advances the context's state by n_steps steps of the five-stage
   low-storage RK4 (Sec. 2.2, Time integration).  dt > 0: fixed step;
   dt <= 0: each step uses the CFL rule evaluated on the device from the
   step's initial state (in the two-kernel FP32-bulk stage form the spectral
   radii of that state are reduced by the previous step's last stage, or by
   the face-data pass of a state no step wrote; the time step is bitwise the
   one dg_time_step gives for the same state).  t_out NULL: stream-ordered (asynchronous,
   graph-launched); the time stays on the device (dg_get_state reads it).
   t_out non-NULL: the call then synchronises the context's stream and
   stores the time reached in *t_out, returning DG_ERR_NONFINITE if a step
   since the last dg_set_state met a non-finite value. */
int dg_step(dg_ctx* ctx, int n_steps, double dt, double* t_out);

/* Advances the context's state with CFL time steps (as dg_step with dt <= 0)
   to exactly t_end: the device clips a step that would pass t_end to end on
   it, and steps taken after t_end is reached have dt = 0 and leave the state
   unchanged.  The host launches the steps in batches sized from the last
   time step, reading the time back between batches.  Stops early after
   max_steps steps.  *t_out (may be NULL): the time reached; *steps_out (may
   be NULL): the number of steps with dt > 0.  Synchronises the context's
   stream.  Returns DG_ERR_NONFINITE if a step met a non-finite value.
   (Sec. 2.2 advances the LSERK scheme to a prescribed end time; the exact
   stop is this library's.) */
int dg_advance(dg_ctx* ctx, double t_end, int64_t max_steps, double* t_out, int64_t* steps_out);

/* The low-storage Runge-Kutta scheme of dg_step and dg_advance (Sec. 2.2:
   GALAEXI offers several explicit low-storage schemes; its validation uses
   the five-stage fourth-order scheme of Carpenter and Kennedy, the default
   here, and its application a 14-stage one).  n_stages (1..32) stages of
   the 2N-storage form dU <- A_s dU + dt R(U, t + c_s dt), U <- U + B_s dU;
   A[0] must be 0 (the first stage starts the register), c gives the stage
   times (used by the manufactured-solution source).  A = NULL restores the
   default.  The CFL rule is unchanged: scale cfl and dfl to the scheme's
   stability region.  DG_ERR_ARG for a bad size or non-finite coefficients.
   Serving keeps the default scheme. */
int dg_set_rk(dg_ctx* ctx, int n_stages, const double* A, const double* B, const double* c);

/* The library's built-in schemes, as dg_set_rk would set them:
   DG_RK_CK5: the five-stage fourth-order scheme of Carpenter and Kennedy
   (the default);  DG_RK_NDB14: the fourteen-stage fourth-order scheme of
   Niegemann, Diehl and Busch (Sec. 2.2 cites it, Sec. 6 runs the
   application with it).  Its stability region reaches about 18.5 along the
   negative real axis and 6.1 along the imaginary axis (the five-stage
   scheme: 4.7 and 3.3), so it takes a larger cfl and dfl.  DG_ERR_ARG for
   another value. */
enum { DG_RK_CK5 = 0, DG_RK_NDB14 = 1 };
int dg_set_rk_scheme(dg_ctx* ctx, int scheme);

/* Same work as dg_step, launched kernel by kernel (no graph) with CUDA events
   recorded on the context's stream around every launch.  Accumulates, per
   kernel kind k, the summed device time ms[k] and the launch count
   launches[k]: k = 0 CFL reduction, 1 BR1 surface prolongation (on GL
   nodes also the ProlongToFace of the state), 2 lifting, 3 surface flux,
   4 volume integral + SurfInt + ApplyJac + RK update.  Both
   arrays have 5 entries.  Synchronises after every step. */
int dg_profile_step(dg_ctx* ctx, int n_steps, double dt, double* ms, int64_t* launches);

/* Sponge zone (the paper's application damps outgoing waves in sponge
   zones, Sec. 6): adds the source -sigma (U - U_base) to Ut at every node,
   in FP64 in both precisions.  sigma: [E][node] host, >= 0; U_base:
   [E][node][5] host (public layout); sigma NULL removes the sponge.  The
   time-step rule does not see the source: keep sigma dt of order one or
   below.  Copies the arrays (synchronises). */
int dg_set_sponge(dg_ctx* ctx, const double* sigma, const double* U_base);

/* Autotuner of the stage kernels' launch configuration (the paper plans
   launch-configuration tuning, Sec. 3.3; this is the library's own).  Times
   every launch variant on the context's current state and keeps the fastest:
   elements per thread block of the lifting and volume kernels (the default,
   about 256 threads, or twice as many elements), the volume kernel's thread
   mapping for the split-form sums (FP64: one task per line pair, or one per
   node) and the side kernels' block size (128 or 256 threads).  In the
   two-kernel FP32-bulk stage (see dg_stage_form) the volume entries apply to
   its element kernel and the side entry to its side kernel.  Only scratch
   arrays are written; the state is unchanged.  config (may be NULL, 6 ints,
   as in dg_set_config).  ms (may be NULL, 8 doubles): mean time per launch
   of each variant (-1 where a variant does not exist), in the order lift D,
   lift 2D, volume D default mapping, volume D other mapping, volume 2D
   default, volume 2D other, side kernels at 256, at 128.  Synchronises.
   Elements per block change no arithmetic; the volume mapping changes the
   summation order of the split-form sums (both within the FP64 parity).
   DG_ERR_STATE on Gauss-Legendre nodes (their kernels have one launch
   configuration). */
int dg_autotune(dg_ctx* ctx, int* config, double* ms);

/* Sets or reads back the launch configuration, 7 ints: lift elements per
   block, volume elements per block, line pairs (1) or per node (0), side
   block size (0 / -1 entries select the defaults), the FP32-bulk stage form
   (0: the two-kernel stage where it applies, else four kernels; 1: always
   the four-kernel stage), the two-kernel stage's L2 prefetch of the next
   wave's element data (1 on, the default; 0 off) and its launch form (0:
   one launch per kernel and stage, the default; 1: one persistent launch
   per step running every stage, its phases separated by grid-wide barriers
   whose waits give up after about a second: a step that loses a
   participant ends with DG_ERR_TIMEOUT from dg_get_state instead of a
   hang).  DG_ERR_ARG for a value that is not one of the variants. */
int dg_set_config(dg_ctx* ctx, const int* config);
int dg_get_config(const dg_ctx* ctx, int* config);

/* The stage form the context's steps use: 2 for the two-kernel FP32-bulk
   stage (FillFlux per side node, then everything else per element; periodic
   LGL meshes of a single context in FP32-bulk), 4 for the four-kernel stage
   (surface prolongation, lifting, surface flux, volume), the form of FP64,
   Gauss-Legendre nodes, boundary conditions and serving pools. */
int dg_stage_form(const dg_ctx* ctx);

/* Time step the CFL rule gives for the context's state (synchronises). */
int dg_time_step(dg_ctx* ctx, double* dt);

/* Kinetic energy E_k = 1/(2|Omega|) int rho |u|^2 and its exact rate from the
   right-hand side, dE_k/dt = 1/|Omega| int (u.(rho u)_t - |u|^2 rho_t / 2)
   (Sec. 5.2), of the context's state; out[0] = E_k, out[1] = dE_k/dt,
   out[2] = |Omega|.  FP64 reductions on the device in a fixed order of
   summation, so repeated calls on the same state return bitwise the same
   values; the first call allocates a small per-context array of partial
   sums (a few tens of KB); synchronises. */
int dg_kinetic(dg_ctx* ctx, double* out);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over many flow cases.
 * (An addition around the paper's method: the per-case arithmetic is exactly
 * that of dg_step.)
 *
 * Cases of one polynomial degree N share a device pool: their elements and
 * sides sit side by side in one set of arrays, and one launch of each stage
 * kernel (captured with the rest of the time step in a CUDA graph) advances
 * every resident case of that N by one LSERK4 step, each with its own CFL
 * time step, time and end time.  A worker thread admits waiting cases as
 * soon as their pool has room (a free element range, a free side range and a
 * free case slot: admission by device memory), builds their maps and metrics
 * on a second stream while the resident cases keep stepping, retires cases
 * that reached their end time, and records each case's time to solution.
 * Per-element arithmetic does not depend on the other cases of a launch, so a
 * case's result is the same alone and in any mix.  Each pool's launch
 * configuration is autotuned on its first cases (elements per block and side
 * block sizes only: the volume kernel keeps its default thread mapping, so
 * that the results do not depend on the tuning either).
 * ------------------------------------------------------------------------ */
typedef struct dg_server dg_server;

typedef struct {
  double gamma, R, Pr;     /* common to every case                           */
  double dfl;              /* viscous time-step factor                       */
  int precision;           /* DG_FP64 or DG_FP32_BULK                        */
  int max_cases;           /* case slots (resident cases), >= 1               */
  int64_t pool_elems[8];   /* pool capacity in elements for N = 1..7 (index N);
                              0 = that N is not served                      */
  int64_t max_resident_dof;/* admission policy: 0 = admit every case that fits
                              its pool (in arrival order, later cases may pass
                              one that does not fit); > 0 = admit in strict
                              arrival order while the resident DOF stay within
                              this bound (a case is always admitted onto an
                              idle server)                                  */
  int64_t priority_dof;    /* step policy: 0 = every resident case advances in
                              every batched step; > 0 = each step advances
                              the resident cases in submission order (first
                              fit) while their DOF stay within this bound,
                              the oldest always; the others sit out that
                              step with their state unchanged (their blocks
                              leave at once), so the oldest cases run at
                              close to their own speed and small cases fill
                              the rest of the GPU                           */
  int persistent;          /* FP32-bulk pools: 1 = each pool runs a step's
                              stages in one persistent launch (grid-wide
                              barriers with bounded waits) instead of one
                              launch per kernel and stage; 0 (default) = the
                              per-kernel launches                           */
} dg_server_config;

typedef struct {
  dg_mesh_desc mesh;       /* as for dg_init_mesh (host memory, copied)      */
  const double* U0;        /* initial state [E][node][5], host, copied       */
  double t_end;            /* end time (the state starts at t = 0)           */
  double mu;               /* viscosity; 0 gives the Euler equations         */
  int riemann;             /* DG_RIEMANN_ROE or DG_RIEMANN_LF                */
  double cfl;              /* CFL factor of the case                         */
} dg_case_desc;

/* Fills cfg with defaults: gamma 1.4, R 1, Pr 0.72, DFL 0.9, FP64, 64 case
   slots, pools of 262,144 elements for N = 3 and N = 5 and 65,536 elements
   for N = 7 (about 48 GB in FP64; set the capacities to fit the device). */
void dg_server_default_config(dg_server_config* cfg);

/* Creates the server, its pools (device memory of all capacities is
   allocated here) and its worker thread, on the current device.
   Errors: DG_ERR_ARG, DG_ERR_OOM, DG_ERR_CUDA. */
int dg_server_create(dg_server** out, const dg_server_config* cfg);

/* Queues one case (non-blocking; mesh and state are copied).  *ticket
   identifies it in dg_poll.  DG_ERR_ARG if its N has no pool or it can never
   fit its pool. */
int dg_submit(dg_server* srv, const dg_case_desc* desc, int64_t* ticket);

/* DG_PENDING while the case is waiting or running; DG_OK once finished, then
   U_out (host, [E][node][5], may be NULL) receives the final state and
   stats (may be NULL) 8 doubles: time to solution (s, submit to done), queue
   wait (submit to admission), service time (admission to done), final time,
   steps, elements, N, 1 if the case met a non-finite value (else 0).
   A finished case can be polled any number of times; DG_ERR_ARG for an
   unknown ticket. */
int dg_poll(dg_server* srv, int64_t ticket, double* U_out, double* stats);

/* Server counters (out: 10 doubles): out[0] batched steps completed,
   out[1] cases finished, out[2] cases resident, out[3] cases waiting,
   out[4] graph captures, out[5] DOF-stage updates done (sum over cases of
   DOF x 5 per step), out[6] device time of the batched steps in seconds
   (CUDA events around each step's graph launch); host seconds spent in
   out[7] graph captures, out[8] case set-up (set-up thread), out[9] case
   insertion (step loop). */
int dg_server_stats(dg_server* srv, double* out);

/* Stops the worker after the current step and frees everything. */
void dg_server_destroy(dg_server* srv);

/* Kinetic energy of a caller-owned state, allocating no device memory.
   The paper has no counterpart: this is an interface addition for callers that
   cannot call cudaMalloc -- applications whose device memory is handed out in
   advance by their own arena or pool, and loops that must not take the
   implicit device synchronisation a cudaMalloc / cudaFree can cause.
   Inputs (device, caller-owned): U [E][node][5] (public layout), J [E][node]
   (Jacobians, e.g. from dg_debug DG_DEBUG_METRICS), Ut [E][node][5] or NULL.
   nodes: the node set the state lives on, DG_NODES_LGL or DG_NODES_GAUSS
   (the quadrature weights of E_k and |Omega| are those of that set, as in
   dg_kinetic for a context of that set); anything else gives DG_ERR_ARG.
   Output (device, caller-owned, 3 doubles): out[0] = E_k, out[1] = dE_k/dt
   (0 when Ut is NULL), out[2] = |Omega|, with the definitions of dg_kinetic.
   N in [1, 7]; n_elems at most 262144 (its built-in scratch holds one partial
   sum triple per element), else DG_ERR_ARG.  Stream-ordered on `stream`; no
   synchronisation.  U, J, Ut, out and the stream must belong to the current
   device: the scratch used is the current device's.  The scratch is a single
   file-scope device array (6 MiB, held by every GPU that loads the library
   until the process exits), shared by all calls on a device: calls whose
   work overlaps on the GPU (for example on two streams) race on it.  Each
   call overwrites every scratch entry it reads, so nothing needs clearing.
   The first call on a device looks up the array's device address
   (cudaGetSymbolAddress) and caches it for the life of the process: make
   that first call before any stream capture.  The cached address belongs to
   the device's primary context; after cudaDeviceReset (or anything else that
   destroys and recreates that context) it is stale, so do not call this
   entry point again in that process. */
int dg_kinetic_noalloc(int N, int nodes, int64_t n_elems, const double* U, const double* J, const double* Ut,
                       double* out, void* stream);

/* Arithmetic peak probe for the roofline denominators of the benchmark (a
   measurement aid; the paper reports no peaks).  kind 0: FP64 FMA rate (the
   bound of the FP64 path, Sec. 4 measures against its own hardware); 1: FP64
   tensor rate (mma.sync m8n8k4 DMMA); 2: both issued from the same warps, in
   equal numbers per iteration (a rate near the sum of kinds 0 and 1 shows
   separate pipes, one near either alone a shared one); 3: FP32 FMA rate.
   One launch of iters iterations over eight 256-thread blocks per SM on the
   current device, timed with CUDA events after a warm-up launch; an FMA
   counts 2 flops, one m8n8k4 MMA 512 per warp.  *flops_per_s: the rate;
   *ms (may be NULL): the timed launch.  Allocates and frees a small output
   buffer; synchronises `stream`.  DG_ERR_ARG for a bad kind or iters < 1. */
int dg_peak_probe(int kind, int iters, double* flops_per_s, double* ms, void* stream);

/* Verification access to intermediate arrays (device buffers, caller-owned).
   what = DG_DEBUG_METRICS: out0 = Ja [E][node][3][3] ((J a^d)_c at [d][c]),
                            out1 = J [E][node]
   what = DG_DEBUG_MAPS:    out0 = int32 [E][6][3] (neighbour element,
                            neighbour face, 1 if this side is the master),
                            out1 = int32 [E][6][n^2] partner face node
   what = DG_DEBUG_GRAD:    out0 = lifted gradients [E][node][4][3] of the
                            last dg_rhs / stage (d(u,v,w,T)/dx_c); in the
                            two-kernel FP32-bulk stage (dg_stage_form 2),
                            of the last dg_rhs only
   what = DG_DEBUG_FSTAR:   out0 = surface flux times s-hat [E][6][n^2][5]
                            on master faces (zero on slave faces), face node
                            p + n q in the master's face frame, last dg_rhs
   what = DG_DEBUG_ALPHA:   out0 = blending factor [E] of the last dg_rhs
   Synchronises. */
/* Verification of the library's own binary64 -> binary32 (round to nearest,
   ties to even) and binary32 -> binary64 conversions, which the FP32-bulk
   kernels run on the integer pipe instead of the FP64 unit: out[i] =
   binary32(in[i]), back[i] = binary64(out[i]); device buffers of n values,
   stream-ordered on `stream`.  DG_ERR_ARG for NULL buffers or n < 0. */
int dg_selftest_convert(const double* in, float* out, double* back, int64_t n, void* stream);

/* Verification of the persistent launch's bounded waits: runs one persistent
   step launch of the context (two-kernel FP32-bulk stage) whose grid-wide
   barriers wait for one participant more than the grid holds, with waits of
   about spin_polls x 200 ns.  The first barrier cannot complete: every block
   gives up and leaves, the launch ends, the timeout flag is read back and
   cleared.  Returns DG_ERR_TIMEOUT when the waits ran out as they must
   (DG_OK would mean a barrier passed without its missing participant);
   the context's state is unchanged (the element phase never ran).
   DG_ERR_STATE if the context does not use the two-kernel stage.
   Synchronises. */
int dg_selftest_wait_timeout(dg_ctx* ctx, unsigned spin_polls);

enum { DG_DEBUG_METRICS = 0, DG_DEBUG_MAPS = 1, DG_DEBUG_GRAD = 2, DG_DEBUG_FSTAR = 3,
       DG_DEBUG_ALPHA = 4 };
int dg_debug(dg_ctx* ctx, int what, void* out0, void* out1);

/* Basic sizes of a context. */
int dg_sizes(const dg_ctx* ctx, int* N, int64_t* n_elems, int64_t* n_sides, int64_t* bytes);

/* Releases every device allocation of the context.  NULL is ignored. */
void dg_destroy(dg_ctx* ctx);

/* Static description of an error code, and the last error message of this
   thread (never NULL). */
const char* dg_error_string(int code);
const char* dg_last_error(void);

/* Number of kernel launches the library has enqueued since load (all
   contexts), for launch accounting in benchmarks. */
int64_t dg_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
