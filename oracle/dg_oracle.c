/*
 * dg_oracle.c -- plain, slow, FP64 CPU restatement of the DGSEM operator of
 * GALAEXI (arXiv 2404.12703), used as TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may load
 * this library.  It shares no code with the CUDA path: it builds its own
 * 1D operators, its own connectivity (by matching node coordinates, not
 * vertex ids), its own metrics, and evaluates every sum as a plain loop in the
 * order the paper writes it.  Compiled twice: with REAL = double (the oracle)
 * and with REAL = long double (-DORC_QUAD, to measure the FP64 rounding floor).
 *
 * What it computes (paper sections / equations):
 *   - LGL nodes, weights, D_ij = l_j'(x_i), the weak operator
 *     Dhat_ij = -(w_j/w_i) D_ji (Eq. dgsem and the definitions after it; the
 *     printed weight ratio is read with i and j exchanged, the reading that makes
 *     the weak form of Eq. weak_form come out), and the split operator
 *     Dsplit = 2D with the two corner corrections (Sec. 2.2, Nonlinear Stability).
 *   - curl-form metrics J a^i_n = -xhat_i . curl_xi (x_l grad_xi x_m) (Sec. 2.2,
 *     Mapping the Equations), J = det(dx/dxi).
 *   - BR1 lifting of (u, v, w, T) in weak form (Eq. lifting, Sec. 2.2).
 *   - KEP split-form volume integral (Pirozzoli two-point flux with averaged
 *     metrics) plus the collocated viscous volume term (Eq. dgsem).
 *   - Roe (no entropy fix) or Lax-Friedrichs surface flux, BR1 viscous surface
 *     flux, times the surface element (FillFlux); SurfInt by a loop over faces
 *     in the manner of Algorithm 3; ApplyJac.
 *   - Hennemann a-priori indicator and convex DG/FV sub-cell blending
 *     (Sec. 2.3, Eq. of the blended operator).
 *   - Carpenter-Kennedy five-stage 2N-storage RK4 (Sec. 2.2, Time integration)
 *     and a CFL time step (the paper gives no rule; see the reading in dg_dt).
 *   - kinetic energy E_k and its exact rate, and the solenoidal and
 *     dilatational dissipation rates eps_S, eps_D from the lifted velocity
 *     gradients (Sec. 5.2).
 *   - the manufactured-solution source of Sec. 5.1 (Eq. mms) and any
 *     2N-storage low-storage RK scheme given by its coefficients.
 *   - boundary conditions (walls, prescribed state, pressure outflow), a sponge
 *     source, and Sutherland's law for mu(T) (Sec. 6 application, Sec. 2.1).
 *   - the standard (non-split) DGSEM on Gauss-Legendre nodes (Sec. 2.2,
 *     Eq. dgsem with lhat+-_i = l_i(+-1)/w_i; Sec. 5.1): nodes the roots of
 *     P_{N+1}, ProlongToFace by interpolation with l(+-1), the collocated
 *     flux divergence as volume term, SurfInt over every node of a line.
 *
 * Node index inside an element: node = i + n*(j + n*k), i along xi.
 * Public state layout: U[e][node][v], v = (rho, rho u, rho v, rho w, rho e).
 * Local faces: f = 2*d + s, d in {xi, eta, zeta}, s = 0 for the minus face
 * (index 0) and 1 for the plus face (index N).  Face frame (p, q): (j, k) for
 * d = 0, (i, k) for d = 1, (i, j) for d = 2.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORC_QUAD
typedef long double real;
#define RSQRT(x) sqrtl(x)
#define RABS(x) fabsl(x)
#define REXP(x) expl(x)
#define RLOG(x) logl(x)
#define RPOW(x, y) powl(x, y)
#define RFLOOR(x) floorl(x)
#define RSIN(x) sinl(x)
#define RCOS(x) cosl(x)
#define REPS LDBL_EPSILON
#define ORC(name) orcq_##name
#else
typedef double real;
#define RSQRT(x) sqrt(x)
#define RABS(x) fabs(x)
#define REXP(x) exp(x)
#define RLOG(x) log(x)
#define RPOW(x, y) pow(x, y)
#define RFLOOR(x) floor(x)
#define RSIN(x) sin(x)
#define RCOS(x) cos(x)
#define REPS DBL_EPSILON
#define ORC(name) orc_##name
#endif

#define NMAX 16

/* ------------------------------------------------------------------ */
/* Parameters, passed as a flat double array from Python.              */
/* ------------------------------------------------------------------ */
enum {
  P_GAMMA = 0, P_R, P_PR, P_MU, P_RIEMANN, P_VISCOUS, P_SHOCK,
  P_ALPHA_MIN, P_ALPHA_MAX, P_CFL, P_DFL, P_ALPHA_FORCE, P_SUTHERLAND, P_TREF,
  P_SOURCE, P_SRC_A, P_SRC_SPEED, P_COUNT
};

typedef struct {
  real gamma, R, Pr, mu;
  int riemann;  /* 0 = Roe, 1 = Lax-Friedrichs */
  int viscous;
  int shock;
  real alpha_min, alpha_max, cfl, dfl;
  real alpha_force;  /* >= 0: every element blends with this alpha (tests) */
  int sutherland;    /* 1: mu = mu(T) by Sutherland's law, mu being its value at T_ref */
  real T_ref;
  int source;        /* 1: the manufactured-solution source of Sec. 5.1 */
  real src_A, src_a; /* its amplitude A and advection speed a */
} params_t;

static params_t read_params(const double* p) {
  params_t P;
  P.gamma = p[P_GAMMA];
  P.R = p[P_R];
  P.Pr = p[P_PR];
  P.mu = p[P_MU];
  P.riemann = (int)p[P_RIEMANN];
  P.viscous = (int)p[P_VISCOUS];
  P.shock = (int)p[P_SHOCK];
  P.alpha_min = p[P_ALPHA_MIN];
  P.alpha_max = p[P_ALPHA_MAX];
  P.cfl = p[P_CFL];
  P.dfl = p[P_DFL];
  P.alpha_force = p[P_ALPHA_FORCE];
  P.sutherland = (int)p[P_SUTHERLAND];
  P.T_ref = p[P_TREF];
  P.source = (int)p[P_SOURCE];
  P.src_A = p[P_SRC_A];
  P.src_a = p[P_SRC_SPEED];
  return P;
}

/* ------------------------------------------------------------------ */
/* 1D operators                                                        */
/* ------------------------------------------------------------------ */

/* The 1D operators are formed in long double and rounded to REAL, so that
   they are (nearly) correctly rounded: at low Mach numbers the row sums of D
   multiply a large background pressure, and a few ulp of difference in D
   would otherwise dominate the comparison with another implementation. */
typedef long double oreal;

/* Legendre polynomial P_N and derivative by the three-term recurrence. */
static void legendre(int N, oreal x, oreal* P, oreal* dP) {
  oreal p0 = 1, p1 = x, d1 = 1;
  if (N == 0) { *P = 1; *dP = 0; return; }
  for (int k = 2; k <= N; ++k) {
    oreal p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    oreal d2 = k * p1 + x * d1;   /* P_k' = k P_{k-1} + x P_{k-1}' */
    p0 = p1; p1 = p2; d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

/* LGL nodes: -1, +1 and the roots of P_N'; weights 2 / (N (N+1) P_N(x)^2). */
static void lgl(int N, oreal* x, oreal* w) {
  x[0] = -1;
  x[N] = 1;
  for (int j = 1; j < N; ++j) {
    oreal t = -cosl(M_PI * (long double)j / (long double)N);
    for (int it = 0; it < 200; ++it) {
      oreal P, dP;
      legendre(N, t, &P, &dP);
      /* Legendre ODE: (1 - x^2) P'' = 2 x P' - N (N+1) P */
      oreal d2P = (2 * t * dP - (oreal)N * (N + 1) * P) / (1 - t * t);
      oreal dt = dP / d2P;
      t -= dt;
      if (fabsl(dt) <= 4 * LDBL_EPSILON) break;
    }
    x[j] = t;
  }
  for (int j = 0; j <= N; ++j) {
    oreal P, dP;
    legendre(N, x[j], &P, &dP);
    w[j] = 2 / ((oreal)N * (N + 1) * P * P);
  }
}

/* Gauss-Legendre nodes: the N + 1 roots of P_{N+1}; weights
   2 / ((1 - x^2) P_{N+1}'(x)^2). */
static void gauss_legendre(int N, oreal* x, oreal* w) {
  const int n = N + 1;
  for (int j = 0; j < n; ++j) {
    oreal t = -cosl(M_PI * ((long double)j + 0.75L) / ((long double)n + 0.5L));
    for (int it = 0; it < 200; ++it) {
      oreal P, dP;
      legendre(n, t, &P, &dP);
      oreal dt = P / dP;
      t -= dt;
      if (fabsl(dt) <= 4 * LDBL_EPSILON) break;
    }
    oreal P, dP;
    legendre(n, t, &P, &dP);
    x[j] = t;
    w[j] = 2 / ((1 - t * t) * dP * dP);
  }
}

/* l_j(y) for the nodes x (Lagrange basis) */
static oreal lagrange(int n, const oreal* x, int j, oreal y) {
  oreal v = 1;
  for (int m = 0; m < n; ++m)
    if (m != j) v *= (y - x[m]) / (x[j] - x[m]);
  return v;
}

/* D[i][j] = l_j'(x_i) with l_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m). */
static void lagrange_derivative(int n, const oreal* x, oreal* D) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      oreal s = 0;
      for (int m = 0; m < n; ++m) {
        if (m == j) continue;
        oreal prod = 1 / (x[j] - x[m]);
        for (int k = 0; k < n; ++k) {
          if (k == j || k == m) continue;
          prod *= (x[i] - x[k]) / (x[j] - x[k]);
        }
        s += prod;
      }
      D[i * n + j] = s;
    }
}

/* Gauss-Jordan inverse with partial pivoting of an n x n matrix. */
static int invert(int n, const oreal* A, oreal* Ainv) {
  oreal a[NMAX * 2 * NMAX];
  int m = 2 * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j)
      a[i * m + j] = j < n ? A[i * n + j] : (j - n == i ? 1 : 0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(a[r * m + c]) > fabsl(a[piv * m + c])) piv = r;
    if (a[piv * m + c] == 0) return -1;
    if (piv != c)
      for (int j = 0; j < m; ++j) {
        oreal t = a[c * m + j]; a[c * m + j] = a[piv * m + j]; a[piv * m + j] = t;
      }
    oreal d = a[c * m + c];
    for (int j = 0; j < m; ++j) a[c * m + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      oreal f = a[r * m + c];
      for (int j = 0; j < m; ++j) a[r * m + j] -= f * a[c * m + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = a[i * m + n + j];
  return 0;
}

typedef struct {
  int N, n;
  real x[NMAX], w[NMAX];
  real D[NMAX * NMAX];      /* D[i][a] = l_a'(x_i)                         */
  real Dhat[NMAX * NMAX];   /* Dhat[i][a] = -(w_a / w_i) D[a][i]           */
  real Dsplit[NMAX * NMAX]; /* 2 D[i][a] - d_iN d_aN / w_N + d_i0 d_a0 / w_0 */
  real Vinv[NMAX * NMAX];   /* inverse of V[i][m] = Ltilde_m(x_i)          */
  oreal Dl[NMAX * NMAX];    /* D in long double, for the metrics          */
  int gauss;                /* 0: LGL nodes, 1: Gauss-Legendre nodes       */
  real Lp[NMAX], Lm[NMAX];  /* l_i(+1), l_i(-1): interpolation to the faces */
  oreal xl[NMAX];           /* the nodes in long double                   */
} ops_t;

static int build_ops(int N, int gauss, ops_t* o) {
  if (N < 1 || N + 1 > NMAX) return -1;
  int n = N + 1;
  o->N = N;
  o->n = n;
  o->gauss = gauss;
  oreal x[NMAX], w[NMAX], V[NMAX * NMAX], Vi[NMAX * NMAX];
  if (gauss) gauss_legendre(N, x, w);
  else lgl(N, x, w);
  for (int i = 0; i < n; ++i) {
    o->xl[i] = x[i];
    o->Lp[i] = (real)lagrange(n, x, i, 1);
    o->Lm[i] = (real)lagrange(n, x, i, -1);
  }
  lagrange_derivative(n, x, o->Dl);
  for (int i = 0; i < n; ++i) { o->x[i] = (real)x[i]; o->w[i] = (real)w[i]; }
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < n; ++a) {
      o->D[i * n + a] = (real)o->Dl[i * n + a];
      o->Dhat[i * n + a] = (real)(-(w[a] / w[i]) * o->Dl[a * n + i]);
      oreal ds = 2 * o->Dl[i * n + a];
      if (i == N && a == N) ds -= 1 / w[N];
      if (i == 0 && a == 0) ds += 1 / w[0];
      o->Dsplit[i * n + a] = (real)ds;
    }
  /* orthonormal Legendre modes Ltilde_m = sqrt((2m+1)/2) P_m */
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < n; ++m) {
      oreal P, dP;
      legendre(m, x[i], &P, &dP);
      V[i * n + m] = sqrtl((oreal)(2 * m + 1) / 2) * P;
    }
  if (invert(n, V, Vi)) return -1;
  for (int i = 0; i < n * n; ++i) o->Vinv[i] = (real)Vi[i];
  return 0;
}

/* ------------------------------------------------------------------ */
/* Mesh                                                                */
/* ------------------------------------------------------------------ */
typedef struct {
  ops_t o;
  int N, n, n2, n3;
  long E;
  real period[3];
  real* xyz;     /* [E][n3][3] at the LGL nodes (geometry input)  */
  real* xyzs;    /* [E][n3][3] at the solution nodes (= xyz on LGL) */
  real* Ja;      /* [E][n3][3][3]  Ja[.][d][c] = (J a^d)_c       */
  real* J;       /* [E][n3]                                      */
  int* nbr_e;    /* [E*6]                                        */
  int* nbr_f;    /* [E*6]                                        */
  int* master;   /* [E*6] 1 if this element side owns the normal */
  int* nbr_node; /* [E*6][n2] partner face node, in partner frame */
  int status;
  /* boundary conditions: face_bc[E*6] = 0 for a face with a partner, else
     k in 1..nbc, the row of bcv (type, then 8 parameters) */
  int* face_bc;
  int nbc;
  real bcv[17][9];
  /* sponge zone (may be NULL): source -sigma (U - U_base) at every node */
  real* sponge_sigma;  /* [E][n3] */
  real* sponge_base;   /* [E][n3][5] */
} mesh_t;

static inline long node_of(int n, int i, int j, int k) { return i + (long)n * (j + (long)n * k); }

/* volume node of face f at face coordinates (p, q) */
static long face_node(int n, int f, int p, int q) {
  int d = f / 2, end = (f % 2) ? n - 1 : 0;
  if (d == 0) return node_of(n, end, p, q);
  if (d == 1) return node_of(n, p, end, q);
  return node_of(n, p, q, end);
}

/* index of node along direction d and the node with that index replaced by a */
static inline int line_index(int n, long node, int d) {
  long s = d == 0 ? 1 : (d == 1 ? n : (long)n * n);
  return (int)((node / s) % n);
}
static inline long line_node(int n, long node, int d, int a) {
  long s = d == 0 ? 1 : (d == 1 ? n : (long)n * n);
  int cur = (int)((node / s) % n);
  return node + (long)(a - cur) * s;
}

static real wrap(real v, real L, real tol) {
  if (L <= 0) return v;
  v = v - L * RFLOOR(v / L);
  if (v > L - tol) v -= L;
  return v;
}
static real pdist(real a, real b, real L) {
  real d = RABS(a - b);
  if (L > 0) {
    real d2 = RABS(d - L);
    if (d2 < d) d = d2;
  }
  return d;
}

typedef struct { real c[3]; long id; } fkey_t;
static int cmp_fkey(const void* A, const void* B) {
  const fkey_t* a = (const fkey_t*)A;
  const fkey_t* b = (const fkey_t*)B;
  if (a->c[0] < b->c[0]) return -1;
  if (a->c[0] > b->c[0]) return 1;
  return a->id < b->id ? -1 : (a->id > b->id ? 1 : 0);
}

static int build_connectivity(mesh_t* M) {
  int n = M->n, n2 = M->n2;
  long E = M->E, F = E * 6;
  /* tolerance: a small fraction of the first element's extent */
  real ext = 0;
  for (int c = 0; c < 3; ++c) {
    real lo = M->xyz[c], hi = M->xyz[c];
    for (long v = 0; v < M->n3; ++v) {
      real t = M->xyz[v * 3 + c];
      if (t < lo) lo = t;
      if (t > hi) hi = t;
    }
    if (hi - lo > ext) ext = hi - lo;
  }
  real tol = 1e-7 * ext;
  fkey_t* keys = (fkey_t*)malloc(sizeof(fkey_t) * F);
  if (!keys) return -1;
  for (long e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      real c[3] = {0, 0, 0};
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          long v = face_node(n, f, p, q);
          for (int d = 0; d < 3; ++d) c[d] += M->xyz[(e * M->n3 + v) * 3 + d];
        }
      fkey_t* k = &keys[e * 6 + f];
      for (int d = 0; d < 3; ++d) k->c[d] = wrap(c[d] / n2, M->period[d], tol);
      k->id = e * 6 + f;
    }
  qsort(keys, F, sizeof(fkey_t), cmp_fkey);
  for (long a = 0; a < F; ++a) M->nbr_e[a] = -1;
  int err = 0;
  for (long a = 0; a < F && !err; ++a) {
    long ia = keys[a].id;
    for (long b = a + 1; b < F; ++b) {
      if (keys[b].c[0] - keys[a].c[0] > tol) break;
      if (pdist(keys[a].c[1], keys[b].c[1], M->period[1]) > tol) continue;
      if (pdist(keys[a].c[2], keys[b].c[2], M->period[2]) > tol) continue;
      long ib = keys[b].id;
      if (M->nbr_e[ia] >= 0 || M->nbr_e[ib] >= 0) { err = 1; break; }
      M->nbr_e[ia] = (int)(ib / 6); M->nbr_f[ia] = (int)(ib % 6);
      M->nbr_e[ib] = (int)(ia / 6); M->nbr_f[ib] = (int)(ia % 6);
      M->master[ia] = ia < ib;
      M->master[ib] = ib < ia;
    }
  }
  /* x-wrap: faces whose wrapped centroid sits within tol of 0 from below were
     moved to ~0 by wrap(); nothing else straddles.  Every face needs a partner. */
  for (long a = 0; a < F && !err; ++a) {
    const int bc = M->face_bc ? M->face_bc[a] : 0;
    if (M->nbr_e[a] < 0 && bc <= 0) err = 2;       /* an open face without a boundary condition */
    if (M->nbr_e[a] >= 0 && bc > 0) err = 2;       /* a boundary condition on an inner face */
    if (M->nbr_e[a] < 0) M->master[a] = 1;         /* boundary faces own their normal */
    if (M->nbr_e[a] < 0) {
      M->nbr_f[a] = -1;
      for (int pq = 0; pq < n2; ++pq) M->nbr_node[a * n2 + pq] = -1;
    }
  }
  free(keys);
  if (err) return -2;
  /* node correspondence by coordinates */
  for (long e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      long ef = e * 6 + f;
      long e2 = M->nbr_e[ef];
      int f2 = M->nbr_f[ef];
      if (e2 < 0) continue;  /* boundary face */
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          const real* xa = &M->xyz[(e * M->n3 + face_node(n, f, p, q)) * 3];
          int found = -1;
          for (int q2 = 0; q2 < n; ++q2)
            for (int p2 = 0; p2 < n; ++p2) {
              const real* xb = &M->xyz[(e2 * M->n3 + face_node(n, f2, p2, q2)) * 3];
              int ok = 1;
              for (int d = 0; d < 3; ++d)
                if (pdist(xa[d], xb[d], M->period[d]) > tol) ok = 0;
              if (ok) {
                if (found >= 0) return -3;
                found = p2 + n * q2;
              }
            }
          if (found < 0) return -4;
          M->nbr_node[ef * n2 + p + n * q] = found;
        }
    }
  return 0;
}

/* Metrics are formed in long double and rounded to REAL at the end.  The curl
   form applies D twice to products of coordinates, which multiplies rounding
   by about (sum_a |D_ia|)^2 ~ 2500 at N = 7; in plain double that leaves the
   discrete metric identities and the two sides of a face inconsistent at the
   1e-12 level, which a background pressure of p0 ~ 71 (Ma = 0.1) turns into
   free-stream errors far above round-off.  In extended precision the rounded
   metrics are within a few ulp of exact. */
typedef long double mreal;

static mreal mline(int n, const mreal* Dm, const mreal* fld, int stride, long v, int d) {
  int i = line_index(n, v, d);
  mreal s = 0;
  for (int a = 0; a < n; ++a) s += Dm[i * n + a] * fld[line_node(n, v, d, a) * stride];
  return s;
}

/* one-dimensional interpolation along direction d of a field with ncomp
   components per node: out[i] = sum_a I[i][a] in[a] on every line */
static void interp_dir(int n, const mreal* I, const mreal* in, mreal* out, int ncomp, int d) {
  long n3 = (long)n * n * n;
  for (long v = 0; v < n3; ++v) {
    int i = line_index(n, v, d);
    for (int c = 0; c < ncomp; ++c) {
      mreal s = 0;
      for (int a = 0; a < n; ++a) s += I[i * n + a] * in[line_node(n, v, d, a) * ncomp + c];
      out[v * ncomp + c] = s;
    }
  }
}

/* tensor-product interpolation I x I x I, applied one direction at a time */
static void interp3(int n, const mreal* I, mreal* f, mreal* tmp, int ncomp) {
  interp_dir(n, I, f, tmp, ncomp, 0);
  interp_dir(n, I, tmp, f, ncomp, 1);
  interp_dir(n, I, f, tmp, ncomp, 2);
  memcpy(f, tmp, sizeof(mreal) * n * n * n * ncomp);
}

static mreal det3(const mreal* a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
         a[2] * (a[3] * a[7] - a[4] * a[6]);
}

/* need: NULL for every element, else a 0/1 mask of the elements whose metrics
   are formed (the others are left as NaN).
   The geometry is the degree-N polynomial through the given LGL node
   coordinates.  The curl-form metrics are formed on the LGL nodes, where the
   normal metric component on a face depends on that face's coordinates only
   (so both elements of a face agree on it).  On Gauss-Legendre nodes the same
   polynomials (J a^d and the Jacobian matrix dx/dxi) are evaluated at the GL
   nodes by exact interpolation, and J = det(dx/dxi) there; the face normals
   of the GL scheme are these metrics interpolated to the face (Sec. 2.2
   reading), which then equal the LGL face values. */
static void build_metrics(mesh_t* M, const unsigned char* need) {
  int n = M->n, n3 = M->n3;
  ops_t lglops;
  const ops_t* og = &M->o;
  if (M->o.gauss) {
    build_ops(M->N, 0, &lglops);
    og = &lglops;
  }
  const mreal* Dm = og->Dl;
  mreal Ig[NMAX * NMAX];   /* Ig[g][l] = l^LGL_l(x^GL_g) */
  if (M->o.gauss)
    for (int g = 0; g < n; ++g)
      for (int l = 0; l < n; ++l) Ig[g * n + l] = lagrange(n, og->xl, l, M->o.xl[g]);
  mreal* dx = (mreal*)malloc(sizeof(mreal) * 9 * n3);   /* dx[v][c][d] = d x_c / d xi_d */
  mreal* V = (mreal*)malloc(sizeof(mreal) * 3 * n3);    /* V[v][d]                    */
  mreal* X = (mreal*)malloc(sizeof(mreal) * 3 * n3);
  mreal* Ja = (mreal*)malloc(sizeof(mreal) * 9 * n3);   /* Ja[v][d][c]                */
  mreal* tmp = (mreal*)malloc(sizeof(mreal) * 9 * n3);
  for (long e = 0; e < M->E; ++e) {
    const real* Xa = &M->xyz[e * n3 * 3];
    if (M->o.gauss) {
      for (long v = 0; v < n3 * 3; ++v) X[v] = (mreal)Xa[v];
      interp3(n, Ig, X, tmp, 3);
      for (long v = 0; v < n3 * 3; ++v) M->xyzs[e * n3 * 3 + v] = (real)X[v];
    }
    if (need && !need[e]) {
      for (long v = 0; v < n3; ++v) {
        M->J[e * n3 + v] = NAN;
        for (int k = 0; k < 9; ++k) M->Ja[(e * n3 + v) * 9 + k] = NAN;
      }
      continue;
    }
    /* the curl form is invariant under a translation of the coordinates; use
       coordinates relative to the element's first node so that the products
       x_l grad x_m carry rounding relative to the element size, not to the
       distance from the origin */
    for (long v = 0; v < n3; ++v)
      for (int c = 0; c < 3; ++c) X[v * 3 + c] = (mreal)Xa[v * 3 + c] - (mreal)Xa[c];
    for (long v = 0; v < n3; ++v)
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) dx[v * 9 + c * 3 + d] = mline(n, Dm, X + c, 3, v, d);
    for (int nc = 0; nc < 3; ++nc) {
      int m = (nc + 1) % 3, l = (nc + 2) % 3;
      for (long v = 0; v < n3; ++v)
        for (int d = 0; d < 3; ++d) V[v * 3 + d] = X[v * 3 + l] * dx[v * 9 + m * 3 + d];
      for (long v = 0; v < n3; ++v)
        for (int i = 0; i < 3; ++i) {
          int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
          mreal curl = mline(n, Dm, V + i2, 3, v, i1) - mline(n, Dm, V + i1, 3, v, i2);
          Ja[(v * 3 + i) * 3 + nc] = -curl;
        }
    }
    if (M->o.gauss) {
      interp3(n, Ig, Ja, tmp, 9);
      interp3(n, Ig, dx, tmp, 9);
    }
    for (long v = 0; v < n3; ++v) {
      M->J[e * n3 + v] = (real)det3(&dx[v * 9]);
      for (int k = 0; k < 9; ++k) M->Ja[(e * n3 + v) * 9 + k] = (real)Ja[v * 9 + k];
    }
  }
  free(dx);
  free(V);
  free(X);
  free(Ja);
  free(tmp);
}

/* ------------------------------------------------------------------ */
/* Point-wise physics                                                  */
/* ------------------------------------------------------------------ */

/* primitive variables q = (rho, u, v, w, p, T) by Eqs. eos_p, eos_T */
static void cons_to_prim(const params_t* P, const real* U, real* q) {
  q[0] = U[0];
  q[1] = U[1] / U[0];
  q[2] = U[2] / U[0];
  q[3] = U[3] / U[0];
  q[4] = (P->gamma - 1) * (U[4] - (real)0.5 * (U[1] * q[1] + U[2] * q[2] + U[3] * q[3]));
  q[5] = q[4] / (U[0] * P->R);
}

/* Euler flux contracted with a (not necessarily unit) vector nv (Eq. nse) */
static void euler_flux(const real* U, const real* q, const real* nv, real* f) {
  real un = q[1] * nv[0] + q[2] * nv[1] + q[3] * nv[2];
  f[0] = U[0] * un;
  f[1] = U[1] * un + q[4] * nv[0];
  f[2] = U[2] * un + q[4] * nv[1];
  f[3] = U[3] * un + q[4] * nv[2];
  f[4] = (U[4] + q[4]) * un;
}

/* Pirozzoli kinetic-energy-preserving two-point flux with metric m */
static void kep_flux(const real* UL, const real* qL, const real* UR, const real* qR,
                     const real* m, real* f) {
  real rho = (qL[0] + qR[0]) / 2;
  real u[3] = {(qL[1] + qR[1]) / 2, (qL[2] + qR[2]) / 2, (qL[3] + qR[3]) / 2};
  real p = (qL[4] + qR[4]) / 2;
  real H = ((UL[4] + qL[4]) / qL[0] + (UR[4] + qR[4]) / qR[0]) / 2;
  real un = u[0] * m[0] + u[1] * m[1] + u[2] * m[2];
  f[0] = rho * un;
  for (int c = 0; c < 3; ++c) f[1 + c] = rho * un * u[c] + p * m[c];
  f[4] = rho * un * H;
}

/* Roe flux with unit normal n, no entropy fix */
static void roe_flux(const params_t* P, const real* UL, const real* qL, const real* UR,
                     const real* qR, const real* n, real* f) {
  real fL[5], fR[5];
  euler_flux(UL, qL, n, fL);
  euler_flux(UR, qR, n, fR);
  real sL = RSQRT(qL[0]), sR = RSQRT(qR[0]);
  real HL = (UL[4] + qL[4]) / qL[0], HR = (UR[4] + qR[4]) / qR[0];
  real ut[3];
  for (int c = 0; c < 3; ++c) ut[c] = (sL * qL[1 + c] + sR * qR[1 + c]) / (sL + sR);
  real Ht = (sL * HL + sR * HR) / (sL + sR);
  real rt = sL * sR;
  real q2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
  real c2 = (P->gamma - 1) * (Ht - q2 / 2);
  real c = RSQRT(c2);
  real un = ut[0] * n[0] + ut[1] * n[1] + ut[2] * n[2];
  real drho = qR[0] - qL[0], dp = qR[4] - qL[4];
  real du[3] = {qR[1] - qL[1], qR[2] - qL[2], qR[3] - qL[3]};
  real dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2];
  real a1 = (dp - rt * c * dun) / (2 * c2);
  real a2 = drho - dp / c2;
  real a5 = (dp + rt * c * dun) / (2 * c2);
  real l1 = RABS(un - c), l2 = RABS(un), l5 = RABS(un + c);
  real dut[3] = {du[0] - dun * n[0], du[1] - dun * n[1], du[2] - dun * n[2]};
  real udut = ut[0] * dut[0] + ut[1] * dut[1] + ut[2] * dut[2];
  real D[5];
  D[0] = l1 * a1 + l2 * a2 + l5 * a5;
  for (int k = 0; k < 3; ++k)
    D[1 + k] = l1 * a1 * (ut[k] - c * n[k]) + l2 * a2 * ut[k] + l5 * a5 * (ut[k] + c * n[k]) +
               l2 * rt * dut[k];
  D[4] = l1 * a1 * (Ht - un * c) + l2 * a2 * q2 / 2 + l5 * a5 * (Ht + un * c) + l2 * rt * udut;
  for (int v = 0; v < 5; ++v) f[v] = (fL[v] + fR[v]) / 2 - D[v] / 2;
}

/* Local Lax-Friedrichs (Rusanov) flux with unit normal n */
static void lf_flux(const params_t* P, const real* UL, const real* qL, const real* UR,
                    const real* qR, const real* n, real* f) {
  real fL[5], fR[5];
  euler_flux(UL, qL, n, fL);
  euler_flux(UR, qR, n, fR);
  real cL = RSQRT(P->gamma * qL[4] / qL[0]), cR = RSQRT(P->gamma * qR[4] / qR[0]);
  real uL = qL[1] * n[0] + qL[2] * n[1] + qL[3] * n[2];
  real uR = qR[1] * n[0] + qR[2] * n[1] + qR[3] * n[2];
  real lL = RABS(uL) + cL, lR = RABS(uR) + cR;
  real lm = lL > lR ? lL : lR;
  for (int v = 0; v < 5; ++v) f[v] = (fL[v] + fR[v]) / 2 - lm * (UR[v] - UL[v]) / 2;
}

static void riemann(const params_t* P, int kind, const real* UL, const real* qL, const real* UR,
                    const real* qR, const real* n, real* f) {
  if (kind == 0) roe_flux(P, UL, qL, UR, qR, n, f);
  else lf_flux(P, UL, qL, UR, qR, n, f);
}

/* dynamic viscosity at temperature T: constant, or Sutherland's law
   (Eq. sutherland) mu(T) = mu_ref 1.4042 (T/T_ref)^(3/2) / (T/T_ref + 0.4042) */
static real viscosity(const params_t* P, real T) {
  if (!P->sutherland) return P->mu;
  real th = T / P->T_ref;
  return P->mu * (real)1.4042 * th * RSQRT(th) / (th + (real)0.4042);
}

/* Manufactured solution of Sec. 5.1 (Eq. mms): with phi = 2 pi (x + y + z - a t),
   rho = rho u = rho v = rho w = 2 + A sin(phi) and rho e = (2 + A sin(phi))^2
   (the bold u of Eq. mms read as the momentum: with a velocity of that size
   the pressure would be negative).  The velocity is (1, 1, 1), so tau = 0;
   p = (gamma - 1)(rho^2 - 3 rho / 2), T = p / (rho R).  The source is
   Q = U_t + div F_c - div F_v of that state, written out:
     Q_rho = (3 - a) c,
     Q_m   = (3 - a) c + (gamma - 1)(2 rho - 3/2) c           (each component),
     Q_E   = -2 a rho c + 3 (2 rho + (gamma - 1)(2 rho - 3/2)) c
             + 3 lambda (gamma - 1) / R (2 pi)^2 A sin(phi)      (viscous only),
   with c = 2 pi A cos(phi); constant viscosity. */
static void mms_source(const params_t* P, const real* x, real t, real* Q) {
  const real w = 2 * (real)3.14159265358979323846264338327950288L;
  const real phi = w * (x[0] + x[1] + x[2] - P->src_a * t);
  const real sn = P->src_A * RSIN(phi), c = w * P->src_A * RCOS(phi);
  const real rho = 2 + sn, g1 = P->gamma - 1;
  Q[0] = (3 - P->src_a) * c;
  for (int k = 1; k <= 3; ++k) Q[k] = (3 - P->src_a) * c + g1 * (2 * rho - (real)1.5) * c;
  Q[4] = -2 * P->src_a * rho * c + 3 * (2 * rho + g1 * (2 * rho - (real)1.5)) * c;
  if (P->viscous) {
    const real lam = P->gamma * P->R * P->mu / (g1 * P->Pr);
    Q[4] += 3 * lam * g1 / P->R * w * w * sn;
  }
}

/* viscous flux F_v = (0, tau, tau.u - q) contracted with nv (Eq. nse, stress and
   Fourier law, heat conductivity lambda = gamma R mu / ((gamma - 1) Pr));
   g[qv][x] = d(u, v, w, T)_qv / dx_x */
static void visc_flux(const params_t* P, const real* q, const real* g, const real* nv, real* f) {
  real ux = g[0], uy = g[1], uz = g[2];
  real vx = g[3], vy = g[4], vz = g[5];
  real wx = g[6], wy = g[7], wz = g[8];
  real Tx = g[9], Ty = g[10], Tz = g[11];
  real mu = viscosity(P, q[5]);
  real lam = P->gamma * P->R * mu / ((P->gamma - 1) * P->Pr);
  real div = ux + vy + wz;
  real txx = mu * (2 * ux - (real)2 / 3 * div);
  real tyy = mu * (2 * vy - (real)2 / 3 * div);
  real tzz = mu * (2 * wz - (real)2 / 3 * div);
  real txy = mu * (uy + vx), txz = mu * (uz + wx), tyz = mu * (vz + wy);
  real u = q[1], v = q[2], w = q[3];
  real Fx[5] = {0, txx, txy, txz, txx * u + txy * v + txz * w + lam * Tx};
  real Fy[5] = {0, txy, tyy, tyz, txy * u + tyy * v + tyz * w + lam * Ty};
  real Fz[5] = {0, txz, tyz, tzz, txz * u + tyz * v + tzz * w + lam * Tz};
  for (int k = 0; k < 5; ++k) f[k] = Fx[k] * nv[0] + Fy[k] * nv[1] + Fz[k] * nv[2];
}

/* ------------------------------------------------------------------ */
/* Shock indicator (Hennemann a-priori indicator on rho*p)             */
/* ------------------------------------------------------------------ */
static real indicator(const mesh_t* M, const params_t* P, const real* qe /* [n3][6] */, real* Eout) {
  int n = M->n, N = M->N, n3 = M->n3;
  real s[NMAX * NMAX * NMAX], t1[NMAX * NMAX * NMAX], t2[NMAX * NMAX * NMAX];
  for (long v = 0; v < n3; ++v) s[v] = qe[v * 6 + 0] * qe[v * 6 + 4];
  /* modal coefficients: apply Vinv along i, then j, then k */
  const real* Vi = M->o.Vinv;
  for (long v = 0; v < n3; ++v) {
    int m = line_index(n, v, 0);
    real a = 0;
    for (int x = 0; x < n; ++x) a += Vi[m * n + x] * s[line_node(n, v, 0, x)];
    t1[v] = a;
  }
  for (long v = 0; v < n3; ++v) {
    int m = line_index(n, v, 1);
    real a = 0;
    for (int x = 0; x < n; ++x) a += Vi[m * n + x] * t1[line_node(n, v, 1, x)];
    t2[v] = a;
  }
  real mj[NMAX];
  for (int j = 0; j < n; ++j) mj[j] = 0;
  for (long v = 0; v < n3; ++v) {
    int m = line_index(n, v, 2);
    real a = 0;
    for (int x = 0; x < n; ++x) a += Vi[m * n + x] * t2[line_node(n, v, 2, x)];
    int mi = line_index(n, v, 0), mjj = line_index(n, v, 1), mk = m;
    int deg = mi > mjj ? mi : mjj;
    if (mk > deg) deg = mk;
    mj[deg] += a * a;
  }
  real totN = 0, totN1 = 0;
  for (int j = 0; j <= N; ++j) totN += mj[j];
  for (int j = 0; j <= N - 1; ++j) totN1 += mj[j];
  real e1 = totN > 0 ? mj[N] / totN : 0;
  real e2 = totN1 > 0 ? mj[N - 1] / totN1 : 0;
  real Ei = e1 > e2 ? e1 : e2;
  if (Eout) *Eout = Ei;
  real T = (real)0.5 * RPOW((real)10, (real)-1.8 * RPOW((real)(N + 1), (real)0.25));
  real sh = RLOG((1 - (real)1e-4) / (real)1e-4);
  real alpha = 1 / (1 + REXP(-sh * (Ei - T) / T));
  if (alpha < P->alpha_min) alpha = 0;
  if (alpha > P->alpha_max) alpha = P->alpha_max;
  return alpha;
}

/* ------------------------------------------------------------------ */
/* The DG operator                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
  real* q;    /* [E][n3][6]                          */
  real* g;    /* [E][n3][12] lifted gradients          */
  real* Bc;   /* [E][n3][5]  convective DG volume term */
  real* B;    /* [E][n3][5]  everything else           */
  real* alpha;/* [E]                                   */
} work_t;

static void work_free(work_t* w) {
  free(w->q); free(w->g); free(w->Bc); free(w->B); free(w->alpha);
}
static int work_alloc(const mesh_t* M, work_t* w) {
  long E = M->E, n3 = M->n3;
  w->q = (real*)calloc(E * n3 * 6, sizeof(real));
  w->g = (real*)calloc(E * n3 * 12, sizeof(real));
  w->Bc = (real*)calloc(E * n3 * 5, sizeof(real));
  w->B = (real*)calloc(E * n3 * 5, sizeof(real));
  w->alpha = (real*)calloc(E, sizeof(real));
  if (!w->q || !w->g || !w->Bc || !w->B || !w->alpha) { work_free(w); return -1; }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Boundary conditions (the paper names wall, farfield and outflow      */
/* conditions for its application case without formulas; these are the */
/* readings): per boundary face node, the BR1 lifting value q* and the  */
/* surface flux f*, from the inner state, its gradients and the outward */
/* unit normal nu (s: surface element, nv = s nu).                      */
/*   1 isothermal no-slip wall (u_w, T_w): q* = (u_w, T_w); convective  */
/*     flux (0, p nu, p u_w.nu); viscous flux F_v at (u_w, T_w) with the */
/*     inner gradients;                                                 */
/*   2 adiabatic no-slip wall (u_w): q* = (u_w, T); convective as 1;    */
/*     viscous F_v at (u_w, T) with no temperature gradient (q.n = 0);  */
/*   3 slip wall: q* = (u - (u.nu) nu, T); convective (0, p nu, 0); no  */
/*     viscous flux;                                                    */
/*   4 prescribed state U_ext: q* = (q + q_ext) / 2; the Riemann flux   */
/*     between U and U_ext; viscous (F_v(q, g) + F_v(q_ext, g)) / 2;    */
/*   5 pressure outflow (p_out): as 4 with U_ext the inner density and  */
/*     velocity at the pressure p_out.                                  */
/* ------------------------------------------------------------------ */
enum { BC_WALL_ISOTHERMAL = 1, BC_WALL_ADIABATIC = 2, BC_SLIP = 3, BC_STATE = 4, BC_OUTFLOW = 5 };

/* the outer state of a prescribed-state or outflow condition */
static void bc_outer_state(const params_t* P, const real* b, const real* U, const real* q, real* Ue) {
  if ((int)b[0] == BC_STATE) {
    for (int k = 0; k < 5; ++k) Ue[k] = b[1 + k];
    return;
  }
  Ue[0] = U[0];
  Ue[1] = U[1];
  Ue[2] = U[2];
  Ue[3] = U[3];
  Ue[4] = b[1] / (P->gamma - 1) + (real)0.5 * (U[1] * q[1] + U[2] * q[2] + U[3] * q[3]);
}

static void bc_lift_value(const mesh_t* M, const params_t* P, int bc, const real* U, const real* q, const real* nu,
                          real* qs) {
  const real* b = M->bcv[bc];
  switch ((int)b[0]) {
    case BC_WALL_ISOTHERMAL:
      qs[0] = b[1]; qs[1] = b[2]; qs[2] = b[3]; qs[3] = b[4];
      break;
    case BC_WALL_ADIABATIC:
      qs[0] = b[1]; qs[1] = b[2]; qs[2] = b[3]; qs[3] = q[5];
      break;
    case BC_SLIP: {
      real un = q[1] * nu[0] + q[2] * nu[1] + q[3] * nu[2];
      for (int c = 0; c < 3; ++c) qs[c] = q[1 + c] - un * nu[c];
      qs[3] = q[5];
      break;
    }
    default: {
      real Ue[5], qe[6];
      bc_outer_state(P, b, U, q, Ue);
      cons_to_prim(P, Ue, qe);
      qs[0] = (q[1] + qe[1]) / 2; qs[1] = (q[2] + qe[2]) / 2;
      qs[2] = (q[3] + qe[3]) / 2; qs[3] = (q[5] + qe[5]) / 2;
    }
  }
}

static void bc_flux(const mesh_t* M, const params_t* P, int bc, const real* U, const real* q, const real* g,
                    const real* nu, real s, const real* nv, real* fs) {
  const real* b = M->bcv[bc];
  const int type = (int)b[0];
  if (type == BC_STATE || type == BC_OUTFLOW) {
    real Ue[5], qe[6], fc[5];
    bc_outer_state(P, b, U, q, Ue);
    cons_to_prim(P, Ue, qe);
    riemann(P, P->riemann, U, q, Ue, qe, nu, fc);
    for (int k = 0; k < 5; ++k) fs[k] = fc[k] * s;
    if (P->viscous) {
      real f1[5], f2[5];
      visc_flux(P, q, g, nv, f1);
      visc_flux(P, qe, g, nv, f2);
      for (int k = 0; k < 5; ++k) fs[k] -= (f1[k] + f2[k]) / 2;
    }
    return;
  }
  const real p = q[4];
  real uw[3] = {0, 0, 0};
  if (type != BC_SLIP) { uw[0] = b[1]; uw[1] = b[2]; uw[2] = b[3]; }
  fs[0] = 0;
  for (int c = 0; c < 3; ++c) fs[1 + c] = p * nu[c] * s;
  fs[4] = p * (uw[0] * nu[0] + uw[1] * nu[1] + uw[2] * nu[2]) * s;
  if (P->viscous && type != BC_SLIP) {
    real qw[6] = {q[0], uw[0], uw[1], uw[2], q[4], type == BC_WALL_ISOTHERMAL ? b[4] : q[5]};
    real gw[12];
    for (int k = 0; k < 12; ++k) gw[k] = g[k];
    if (type == BC_WALL_ADIABATIC) gw[9] = gw[10] = gw[11] = 0;
    real fv[5];
    visc_flux(P, qw, gw, nv, fv);
    for (int k = 0; k < 5; ++k) fs[k] -= fv[k];
  }
}

/* J Ut = -[ V_conv + V_visc + S ], Eq. dgsem with the split-form volume term.
   want: NULL for every element, else a 0/1 mask of the elements whose Ut is
   wanted (their neighbours' gradients are formed as needed). */
static int rhs_impl(const mesh_t* M, const params_t* P, const real* U, real t, real* Ut,
                    const unsigned char* want, real* alpha_out, real* g_out, real* fstar_out,
                    work_t* w) {
  int n = M->n, n2 = M->n2, n3 = M->n3;
  long E = M->E;
  const ops_t* o = &M->o;
  unsigned char* needg = (unsigned char*)calloc(E, 1);
  for (long e = 0; e < E; ++e) {
    if (want && !want[e]) continue;
    needg[e] = 1;
    for (int f = 0; f < 6; ++f)
      if (M->nbr_e[e * 6 + f] >= 0) needg[M->nbr_e[e * 6 + f]] = 1;
  }
  /* ConsToPrim everywhere */
  for (long v = 0; v < E * n3; ++v) cons_to_prim(P, &U[v * 5], &w->q[v * 6]);
  memset(w->B, 0, sizeof(real) * E * n3 * 5);
  memset(w->Bc, 0, sizeof(real) * E * n3 * 5);

  /* ---- BR1 lifting of (u, v, w, T), weak form (Eq. lifting) ---- */
  static const int lifted[4] = {1, 2, 3, 5};
  if (P->viscous) {
    memset(w->g, 0, sizeof(real) * E * n3 * 12);
    for (long e = 0; e < E; ++e) {
      if (!needg[e]) continue;
      for (long v = 0; v < n3; ++v)
        for (int d = 0; d < 3; ++d) {
          int i = line_index(n, v, d);
          for (int a = 0; a < n; ++a) {
            long va = line_node(n, v, d, a);
            const real* Jaa = &M->Ja[((e * n3 + va) * 3 + d) * 3];
            for (int qv = 0; qv < 4; ++qv)
              for (int x = 0; x < 3; ++x)
                w->g[(e * n3 + v) * 12 + qv * 3 + x] +=
                    o->Dhat[i * n + a] * Jaa[x] * w->q[(e * n3 + va) * 6 + lifted[qv]];
          }
        }
    }
    /* surface: q* = (q_master + q_slave)/2 times the master's outward s n, with
       lhat = 1/w at the face node; the slave gets the opposite sign */
    for (long e = 0; e < E; ++e)
      for (int f = 0; f < 6; ++f) {
        long ef = e * 6 + f;
        if (!M->master[ef]) continue;
        long e2 = M->nbr_e[ef];
        int f2 = M->nbr_f[ef];
        real sgn = (f % 2) ? 1 : -1;
        if (e2 < 0) {  /* boundary face: the condition's lifting value */
          if (!needg[e]) continue;
          for (int qq = 0; qq < n; ++qq)
            for (int p = 0; p < n; ++p) {
              long vM = face_node(n, f, p, qq);
              const real* Jam = &M->Ja[((e * n3 + vM) * 3 + f / 2) * 3];
              real nv[3] = {sgn * Jam[0], sgn * Jam[1], sgn * Jam[2]};
              real s = RSQRT(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
              real nu[3] = {nv[0] / s, nv[1] / s, nv[2] / s};
              real qs[4];
              bc_lift_value(M, P, M->face_bc[ef], &U[(e * n3 + vM) * 5], &w->q[(e * n3 + vM) * 6], nu, qs);
              for (int qv = 0; qv < 4; ++qv)
                for (int x = 0; x < 3; ++x)
                  w->g[(e * n3 + vM) * 12 + qv * 3 + x] += qs[qv] * sgn * Jam[x] / o->w[(f % 2) ? n - 1 : 0];
            }
          continue;
        }
        if (!needg[e] && !needg[e2]) continue;
        for (int qq = 0; qq < n; ++qq)
          for (int p = 0; p < n; ++p) {
            long vM = face_node(n, f, p, qq);
            int a2 = M->nbr_node[ef * n2 + p + n * qq];
            long vS = face_node(n, f2, a2 % n, a2 / n);
            const real* Jam = &M->Ja[((e * n3 + vM) * 3 + f / 2) * 3];
            for (int qv = 0; qv < 4; ++qv) {
              real qs = (w->q[(e * n3 + vM) * 6 + lifted[qv]] + w->q[(e2 * n3 + vS) * 6 + lifted[qv]]) / 2;
              for (int x = 0; x < 3; ++x) {
                real fl = qs * sgn * Jam[x];
                w->g[(e * n3 + vM) * 12 + qv * 3 + x] += fl / o->w[(f % 2) ? n - 1 : 0];
                w->g[(e2 * n3 + vS) * 12 + qv * 3 + x] -= fl / o->w[(f2 % 2) ? n - 1 : 0];
              }
            }
          }
      }
    for (long e = 0; e < E; ++e) {
      if (!needg[e]) continue;
      for (long v = 0; v < n3; ++v)
        for (int k = 0; k < 12; ++k) w->g[(e * n3 + v) * 12 + k] /= M->J[e * n3 + v];
    }
  }

  /* ---- indicator ---- */
  for (long e = 0; e < E; ++e) w->alpha[e] = 0;
  if (P->shock)
    for (long e = 0; e < E; ++e) {
      if (want && !want[e]) continue;
      w->alpha[e] = P->alpha_force >= 0 ? P->alpha_force : indicator(M, P, &w->q[e * n3 * 6], NULL);
    }

  /* ---- volume integral ---- */
  for (long e = 0; e < E; ++e) {
    if (want && !want[e]) continue;
    for (long v = 0; v < n3; ++v)
      for (int d = 0; d < 3; ++d) {
        int i = line_index(n, v, d);
        const real* Jai = &M->Ja[((e * n3 + v) * 3 + d) * 3];
        for (int a = 0; a < n; ++a) {
          long va = line_node(n, v, d, a);
          const real* Jaa = &M->Ja[((e * n3 + va) * 3 + d) * 3];
          real m[3] = {(Jai[0] + Jaa[0]) / 2, (Jai[1] + Jaa[1]) / 2, (Jai[2] + Jaa[2]) / 2};
          real fs[5];
          kep_flux(&U[(e * n3 + v) * 5], &w->q[(e * n3 + v) * 6], &U[(e * n3 + va) * 5],
                   &w->q[(e * n3 + va) * 6], m, fs);
          for (int k = 0; k < 5; ++k) w->Bc[(e * n3 + v) * 5 + k] += o->Dsplit[i * n + a] * fs[k];
          if (P->viscous) {
            real fv[5];
            visc_flux(P, &w->q[(e * n3 + va) * 6], &w->g[(e * n3 + va) * 12], Jaa, fv);
            for (int k = 0; k < 5; ++k) w->B[(e * n3 + v) * 5 + k] -= o->Dhat[i * n + a] * fv[k];
          }
        }
      }
  }

  /* ---- FV sub-cell operator and convex blend (Sec. 2.3) ---- */
  if (P->shock) {
    real* vfv = (real*)malloc(sizeof(real) * n3 * 5);
    for (long e = 0; e < E; ++e) {
      if (want && !want[e]) continue;
      real al = w->alpha[e];
      if (al == 0) continue;
      memset(vfv, 0, sizeof(real) * n3 * 5);
      for (int d = 0; d < 3; ++d)
        for (long v0 = 0; v0 < n3; ++v0) {
          if (line_index(n, v0, d) != 0) continue;   /* one pass per line */
          /* interface metrics by telescoping the discrete derivative:
             Ja_{-1/2} = Ja_0, Ja_{i+1/2} = Ja_{i-1/2} + w_i (D Ja)_i */
          real Jh[NMAX + 1][3];
          for (int c = 0; c < 3; ++c) Jh[0][c] = M->Ja[((e * n3 + v0) * 3 + d) * 3 + c];
          for (int i = 0; i < n; ++i) {
            for (int c = 0; c < 3; ++c) {
              real dj = 0;
              for (int a = 0; a < n; ++a)
                dj += o->D[i * n + a] * M->Ja[((e * n3 + line_node(n, v0, d, a)) * 3 + d) * 3 + c];
              Jh[i + 1][c] = Jh[i][c] + o->w[i] * dj;
            }
          }
          for (int i = 0; i < n - 1; ++i) {
            long vl = line_node(n, v0, d, i), vr = line_node(n, v0, d, i + 1);
            const real* m = Jh[i + 1];
            real s = RSQRT(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            real nn[3] = {m[0] / s, m[1] / s, m[2] / s};
            real fb[5];
            lf_flux(P, &U[(e * n3 + vl) * 5], &w->q[(e * n3 + vl) * 6], &U[(e * n3 + vr) * 5],
                    &w->q[(e * n3 + vr) * 6], nn, fb);
            for (int k = 0; k < 5; ++k) {
              vfv[vl * 5 + k] += fb[k] * s / o->w[i];
              vfv[vr * 5 + k] -= fb[k] * s / o->w[i + 1];
            }
          }
        }
      for (long v = 0; v < n3; ++v)
        for (int k = 0; k < 5; ++k)
          w->Bc[(e * n3 + v) * 5 + k] = (1 - al) * w->Bc[(e * n3 + v) * 5 + k] + al * vfv[v * 5 + k];
    }
    free(vfv);
  }

  /* ---- FillFlux + SurfInt, looping over faces (Algorithm 3) ---- */
  for (long e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      long ef = e * 6 + f;
      if (!M->master[ef]) continue;
      long e2 = M->nbr_e[ef];
      int f2 = M->nbr_f[ef];
      real sgn = (f % 2) ? 1 : -1;
      if (e2 < 0) {  /* boundary face */
        if (want && !want[e]) continue;
        for (int qq = 0; qq < n; ++qq)
          for (int p = 0; p < n; ++p) {
            long vM = face_node(n, f, p, qq);
            const real* Jam = &M->Ja[((e * n3 + vM) * 3 + f / 2) * 3];
            real nv[3] = {sgn * Jam[0], sgn * Jam[1], sgn * Jam[2]};
            real s = RSQRT(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
            real nu[3] = {nv[0] / s, nv[1] / s, nv[2] / s};
            real fs[5];
            bc_flux(M, P, M->face_bc[ef], &U[(e * n3 + vM) * 5], &w->q[(e * n3 + vM) * 6],
                    &w->g[(e * n3 + vM) * 12], nu, s, nv, fs);
            if (fstar_out)
              for (int k = 0; k < 5; ++k) fstar_out[(ef * n2 + p + n * qq) * 5 + k] = fs[k];
            for (int k = 0; k < 5; ++k) w->B[(e * n3 + vM) * 5 + k] += fs[k] / o->w[(f % 2) ? n - 1 : 0];
          }
        continue;
      }
      if (want && !want[e] && !want[e2]) continue;
      for (int qq = 0; qq < n; ++qq)
        for (int p = 0; p < n; ++p) {
          long vM = face_node(n, f, p, qq);
          int a2 = M->nbr_node[ef * n2 + p + n * qq];
          long vS = face_node(n, f2, a2 % n, a2 / n);
          const real* Jam = &M->Ja[((e * n3 + vM) * 3 + f / 2) * 3];
          real nv[3] = {sgn * Jam[0], sgn * Jam[1], sgn * Jam[2]};
          real s = RSQRT(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
          real nu[3] = {nv[0] / s, nv[1] / s, nv[2] / s};
          const real* UM = &U[(e * n3 + vM) * 5];
          const real* US = &U[(e2 * n3 + vS) * 5];
          const real* qM = &w->q[(e * n3 + vM) * 6];
          const real* qS = &w->q[(e2 * n3 + vS) * 6];
          real fc[5], fs[5];
          riemann(P, P->riemann, UM, qM, US, qS, nu, fc);
          for (int k = 0; k < 5; ++k) fs[k] = fc[k] * s;
          if (P->viscous) {
            real fvM[5], fvS[5];
            visc_flux(P, qM, &w->g[(e * n3 + vM) * 12], nv, fvM);
            visc_flux(P, qS, &w->g[(e2 * n3 + vS) * 12], nv, fvS);
            for (int k = 0; k < 5; ++k) fs[k] -= (fvM[k] + fvS[k]) / 2;
          }
          if (fstar_out)
            for (int k = 0; k < 5; ++k) fstar_out[(ef * n2 + p + n * qq) * 5 + k] = fs[k];
          for (int k = 0; k < 5; ++k) {
            w->B[(e * n3 + vM) * 5 + k] += fs[k] / o->w[(f % 2) ? n - 1 : 0];
            w->B[(e2 * n3 + vS) * 5 + k] -= fs[k] / o->w[(f2 % 2) ? n - 1 : 0];
          }
        }
    }

  /* ---- ApplyJac; sponge source; manufactured-solution source ---- */
  for (long e = 0; e < E; ++e) {
    if (want && !want[e]) continue;
    for (long v = 0; v < n3; ++v)
      for (int k = 0; k < 5; ++k) {
        long x = (e * n3 + v) * 5 + k;
        Ut[x] = -(w->Bc[x] + w->B[x]) / M->J[e * n3 + v];
        if (M->sponge_sigma) Ut[x] -= M->sponge_sigma[e * n3 + v] * (U[x] - M->sponge_base[x]);
      }
    if (P->source)
      for (long v = 0; v < n3; ++v) {
        real Q[5];
        mms_source(P, &M->xyzs[(e * n3 + v) * 3], t, Q);
        for (int k = 0; k < 5; ++k) Ut[(e * n3 + v) * 5 + k] += Q[k];
      }
  }
  if (alpha_out)
    for (long e = 0; e < E; ++e) alpha_out[e] = w->alpha[e];
  if (g_out && P->viscous)
    for (long x = 0; x < E * n3 * 12; ++x) g_out[x] = w->g[x];
  free(needg);
  return 0;
}

/* ---- standard DGSEM on Gauss-Legendre nodes (Eq. dgsem, Sec. 5.1) ----
   The face values are interpolations along the lines normal to the face
   (ProlongToFace with l(+-1)); ConsToPrim then runs on the face values; the
   surface terms are spread over every node of the line with
   lhat+-_i = l_i(+-1) / w_i (SurfInt); the convective volume term is the
   collocated flux divergence sum_a Dhat[i][a] (J a^d . F(U))_a.  The lifting
   and viscous terms are those of the LGL scheme with the same face
   interpolation; the lifted gradients are interpolated to the faces for the
   viscous surface flux. */

/* value at face point (p, q) of face f: sum_a l_a(+-1) fld[line node a] */
static void face_value(const mesh_t* M, const real* fld, int ncomp, long e, int f, int p, int q, real* out) {
  int n = M->n;
  long n3 = M->n3;
  const real* L = (f % 2) ? M->o.Lp : M->o.Lm;
  long v0 = face_node(n, f, p, q);
  for (int c = 0; c < ncomp; ++c) out[c] = 0;
  for (int a = 0; a < n; ++a) {
    long va = line_node(n, v0, f / 2, a);
    for (int c = 0; c < ncomp; ++c) out[c] += L[a] * fld[(e * n3 + va) * ncomp + c];
  }
}

/* J a^d of the face's direction interpolated to face point (p, q), times the
   outward sign of face f */
static void face_normal(const mesh_t* M, long e, int f, int p, int q, real* nv) {
  int n = M->n, d = f / 2;
  long n3 = M->n3;
  const real* L = (f % 2) ? M->o.Lp : M->o.Lm;
  long v0 = face_node(n, f, p, q);
  real sgn = (f % 2) ? 1 : -1;
  for (int c = 0; c < 3; ++c) nv[c] = 0;
  for (int a = 0; a < n; ++a) {
    long va = line_node(n, v0, d, a);
    for (int c = 0; c < 3; ++c) nv[c] += L[a] * M->Ja[((e * n3 + va) * 3 + d) * 3 + c];
  }
  for (int c = 0; c < 3; ++c) nv[c] *= sgn;
}

/* acc[line node a] += sgn_add * val * l_a(+-1) / w_a along the line of face point (p, q) */
static void surf_spread(const mesh_t* M, real* acc, int ncomp, long e, int f, int p, int q, const real* val,
                        real sgn_add) {
  int n = M->n;
  long n3 = M->n3;
  const real* L = (f % 2) ? M->o.Lp : M->o.Lm;
  long v0 = face_node(n, f, p, q);
  for (int a = 0; a < n; ++a) {
    long va = line_node(n, v0, f / 2, a);
    for (int c = 0; c < ncomp; ++c) acc[(e * n3 + va) * ncomp + c] += sgn_add * val[c] * L[a] / M->o.w[a];
  }
}

static int rhs_gauss(const mesh_t* M, const params_t* P, const real* U, real t, real* Ut,
                     const unsigned char* want, real* g_out, real* fstar_out, work_t* w) {
  int n = M->n, n2 = M->n2, n3 = M->n3;
  long E = M->E, F = E * 6;
  const ops_t* o = &M->o;
  if (P->shock) return -7;  /* shock capturing is an LGL (split-form) feature */
  unsigned char* needg = (unsigned char*)calloc(E, 1);
  for (long e = 0; e < E; ++e) {
    if (want && !want[e]) continue;
    needg[e] = 1;
    for (int f = 0; f < 6; ++f)
      if (M->nbr_e[e * 6 + f] >= 0) needg[M->nbr_e[e * 6 + f]] = 1;
  }
  /* ProlongToFace of U, then ConsToPrim on the faces */
  real* Uf = (real*)malloc(sizeof(real) * F * n2 * 5);
  real* qf = (real*)malloc(sizeof(real) * F * n2 * 6);
  real* gf = (real*)calloc(F * n2 * 12, sizeof(real));
  for (long e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f)
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          long x = (e * 6 + f) * n2 + p + n * q;
          face_value(M, U, 5, e, f, p, q, &Uf[x * 5]);
          cons_to_prim(P, &Uf[x * 5], &qf[x * 6]);
        }
  for (long v = 0; v < E * n3; ++v) cons_to_prim(P, &U[v * 5], &w->q[v * 6]);
  memset(w->B, 0, sizeof(real) * E * n3 * 5);
  memset(w->Bc, 0, sizeof(real) * E * n3 * 5);

  /* ---- BR1 lifting ---- */
  static const int lifted[4] = {1, 2, 3, 5};
  if (P->viscous) {
    memset(w->g, 0, sizeof(real) * E * n3 * 12);
    for (long e = 0; e < E; ++e) {
      if (!needg[e]) continue;
      for (long v = 0; v < n3; ++v)
        for (int d = 0; d < 3; ++d) {
          int i = line_index(n, v, d);
          for (int a = 0; a < n; ++a) {
            long va = line_node(n, v, d, a);
            const real* Jaa = &M->Ja[((e * n3 + va) * 3 + d) * 3];
            for (int qv = 0; qv < 4; ++qv)
              for (int x = 0; x < 3; ++x)
                w->g[(e * n3 + v) * 12 + qv * 3 + x] +=
                    o->Dhat[i * n + a] * Jaa[x] * w->q[(e * n3 + va) * 6 + lifted[qv]];
          }
        }
    }
    for (long e = 0; e < E; ++e)
      for (int f = 0; f < 6; ++f) {
        long ef = e * 6 + f;
        if (!M->master[ef]) continue;
        long e2 = M->nbr_e[ef];
        int f2 = M->nbr_f[ef];
        if (e2 < 0 ? !needg[e] : (!needg[e] && !needg[e2])) continue;
        for (int qq = 0; qq < n; ++qq)
          for (int p = 0; p < n; ++p) {
            long xM = ef * n2 + p + n * qq;
            real nv[3];
            face_normal(M, e, f, p, qq, nv);
            real qs[4];
            if (e2 < 0) {
              real s = RSQRT(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
              real nu[3] = {nv[0] / s, nv[1] / s, nv[2] / s};
              bc_lift_value(M, P, M->face_bc[ef], &Uf[xM * 5], &qf[xM * 6], nu, qs);
            } else {
              long xS = ((long)e2 * 6 + f2) * n2 + M->nbr_node[xM];
              for (int qv = 0; qv < 4; ++qv) qs[qv] = (qf[xM * 6 + lifted[qv]] + qf[xS * 6 + lifted[qv]]) / 2;
            }
            real fl[12];
            for (int qv = 0; qv < 4; ++qv)
              for (int x = 0; x < 3; ++x) fl[qv * 3 + x] = qs[qv] * nv[x];
            surf_spread(M, w->g, 12, e, f, p, qq, fl, 1);
            if (e2 >= 0) {
              int a2 = M->nbr_node[xM];
              surf_spread(M, w->g, 12, e2, f2, a2 % n, a2 / n, fl, -1);
            }
          }
      }
    for (long e = 0; e < E; ++e) {
      if (!needg[e]) continue;
      for (long v = 0; v < n3; ++v)
        for (int k = 0; k < 12; ++k) w->g[(e * n3 + v) * 12 + k] /= M->J[e * n3 + v];
    }
    /* ProlongToFace of the lifted gradients */
    for (long e = 0; e < E; ++e) {
      if (!needg[e]) continue;
      for (int f = 0; f < 6; ++f)
        for (int q = 0; q < n; ++q)
          for (int p = 0; p < n; ++p)
            face_value(M, w->g, 12, e, f, p, q, &gf[((e * 6 + f) * n2 + p + n * q) * 12]);
    }
  }

  /* ---- volume integral: collocated flux divergence (standard weak form) ---- */
  for (long e = 0; e < E; ++e) {
    if (want && !want[e]) continue;
    for (long v = 0; v < n3; ++v)
      for (int d = 0; d < 3; ++d) {
        int i = line_index(n, v, d);
        for (int a = 0; a < n; ++a) {
          long va = line_node(n, v, d, a);
          const real* Jaa = &M->Ja[((e * n3 + va) * 3 + d) * 3];
          real fc[5];
          euler_flux(&U[(e * n3 + va) * 5], &w->q[(e * n3 + va) * 6], Jaa, fc);
          for (int k = 0; k < 5; ++k) w->Bc[(e * n3 + v) * 5 + k] += o->Dhat[i * n + a] * fc[k];
          if (P->viscous) {
            real fv[5];
            visc_flux(P, &w->q[(e * n3 + va) * 6], &w->g[(e * n3 + va) * 12], Jaa, fv);
            for (int k = 0; k < 5; ++k) w->B[(e * n3 + v) * 5 + k] -= o->Dhat[i * n + a] * fv[k];
          }
        }
      }
  }

  /* ---- FillFlux + SurfInt over the faces ---- */
  for (long e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      long ef = e * 6 + f;
      if (!M->master[ef]) continue;
      long e2 = M->nbr_e[ef];
      int f2 = M->nbr_f[ef];
      if (e2 < 0 ? (want && !want[e]) : (want && !want[e] && !want[e2])) continue;
      for (int qq = 0; qq < n; ++qq)
        for (int p = 0; p < n; ++p) {
          long xM = ef * n2 + p + n * qq;
          real nv[3];
          face_normal(M, e, f, p, qq, nv);
          real s = RSQRT(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
          real nu[3] = {nv[0] / s, nv[1] / s, nv[2] / s};
          real fs[5];
          if (e2 < 0) {
            bc_flux(M, P, M->face_bc[ef], &Uf[xM * 5], &qf[xM * 6], &gf[xM * 12], nu, s, nv, fs);
          } else {
            long xS = ((long)e2 * 6 + f2) * n2 + M->nbr_node[xM];
            real fc[5];
            riemann(P, P->riemann, &Uf[xM * 5], &qf[xM * 6], &Uf[xS * 5], &qf[xS * 6], nu, fc);
            for (int k = 0; k < 5; ++k) fs[k] = fc[k] * s;
            if (P->viscous) {
              real fvM[5], fvS[5];
              visc_flux(P, &qf[xM * 6], &gf[xM * 12], nv, fvM);
              visc_flux(P, &qf[xS * 6], &gf[xS * 12], nv, fvS);
              for (int k = 0; k < 5; ++k) fs[k] -= (fvM[k] + fvS[k]) / 2;
            }
          }
          if (fstar_out)
            for (int k = 0; k < 5; ++k) fstar_out[xM * 5 + k] = fs[k];
          surf_spread(M, w->B, 5, e, f, p, qq, fs, 1);
          if (e2 >= 0) {
            int a2 = M->nbr_node[xM];
            surf_spread(M, w->B, 5, e2, f2, a2 % n, a2 / n, fs, -1);
          }
        }
    }

  /* ---- ApplyJac; sponge source; manufactured-solution source ---- */
  for (long e = 0; e < E; ++e) {
    if (want && !want[e]) continue;
    for (long v = 0; v < n3; ++v)
      for (int k = 0; k < 5; ++k) {
        long x = (e * n3 + v) * 5 + k;
        Ut[x] = -(w->Bc[x] + w->B[x]) / M->J[e * n3 + v];
        if (M->sponge_sigma) Ut[x] -= M->sponge_sigma[e * n3 + v] * (U[x] - M->sponge_base[x]);
      }
    if (P->source)
      for (long v = 0; v < n3; ++v) {
        real Q[5];
        mms_source(P, &M->xyzs[(e * n3 + v) * 3], t, Q);
        for (int k = 0; k < 5; ++k) Ut[(e * n3 + v) * 5 + k] += Q[k];
      }
  }
  if (g_out && P->viscous)
    for (long x = 0; x < E * n3 * 12; ++x) g_out[x] = w->g[x];
  free(Uf);
  free(qf);
  free(gf);
  free(needg);
  return 0;
}

/* the DG operator of the mesh's node set */
static int rhs_any(const mesh_t* M, const params_t* P, const real* U, real t, real* Ut, const unsigned char* want,
                   real* alpha_out, real* g_out, real* fstar_out, work_t* w) {
  if (P->source && P->sutherland) return -8;  /* the source is written for a constant viscosity */
  if (M->o.gauss) {
    if (alpha_out)
      for (long e = 0; e < M->E; ++e) alpha_out[e] = 0;
    return rhs_gauss(M, P, U, t, Ut, want, g_out, fstar_out, w);
  }
  return rhs_impl(M, P, U, t, Ut, want, alpha_out, g_out, fstar_out, w);
}

/* ------------------------------------------------------------------ */
/* Time step and LSERK                                                 */
/* ------------------------------------------------------------------ */

/* Carpenter-Kennedy RK4(3)5 2N-storage coefficients (Sec. 2.2 cites them) */
static const double RK_A[5] = {0.0, -567301805773.0 / 1357537059087.0,
                               -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0,
                               -1275806237668.0 / 842570457699.0};
static const double RK_B[5] = {1432997174477.0 / 9575080441755.0,
                               5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0,
                               3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};
static const double RK_C[5] = {0.0, 1432997174477.0 / 9575080441755.0,
                               2526269341429.0 / 6820363218457.0,
                               2006345519317.0 / 3224310063776.0,
                               2802321613138.0 / 2924317926251.0};

/* Niegemann, Diehl and Busch's fourteen-stage fourth-order 2N-storage
   scheme (J. Comput. Phys. 231, 2012; Sec. 2.2 cites it, Sec. 6 runs the
   application with it): A, B and the abscissae c as published, 16 digits */
static const double RK14_A[14] = {0.0, -0.7188012108672410, -0.7785331173421570, -0.0053282796654044,
                                  -0.8552979934029281, -3.9564138245774565, -1.5780575380587385,
                                  -2.0837094552574054, -0.7483334182761610, -0.7032861106563359,
                                  0.0013917096117681, -0.0932075369637460, -0.9514200470875948,
                                  -7.1151571693922548};
static const double RK14_B[14] = {0.0367762454319673, 0.3136296607553959, 0.1531848691869027,
                                  0.0030097086818182, 0.3326293790646110, 0.2440251405350864,
                                  0.3718879239592277, 0.6204126221582444, 0.1524043173028741,
                                  0.0760894927419266, 0.0077604214040978, 0.0024647284755382,
                                  0.0780348340049386, 5.5059777270269628};
static const double RK14_C[14] = {0.0, 0.0367762454319673, 0.1249685262725025, 0.2446177702277698,
                                  0.2476149531070420, 0.2969311120382472, 0.3978149645802642,
                                  0.5270854589440328, 0.6981269994175695, 0.8190890835352128,
                                  0.8527059887098624, 0.8604711817462826, 0.8627060376969976,
                                  0.8734213127600976};

typedef void (*rhs_fn)(void* ctx, const real* U, real t, real* Ut);

/* one 2N-storage step: dU = A_s dU + dt R(U); U = U + B_s dU */
/* a 2N-storage low-storage RK scheme (Sec. 2.2 names several): ns stages,
   dU <- A_s dU + dt R(U, t + c_s dt), U <- U + B_s dU (A_1 is not used) */
typedef struct {
  int ns;
  real A[32], B[32], C[32];
} rk_t;

static rk_t rk_default(void) {
  rk_t r;
  r.ns = 5;
  for (int s = 0; s < 5; ++s) { r.A[s] = RK_A[s]; r.B[s] = RK_B[s]; r.C[s] = RK_C[s]; }
  return r;
}

static void lserk_step_rk(const rk_t* rk, real* U, real* dU, real* Ut, long len, real t, real dt, rhs_fn f,
                          void* ctx) {
  for (int s = 0; s < rk->ns; ++s) {
    f(ctx, U, t + rk->C[s] * dt, Ut);
    for (long x = 0; x < len; ++x) {
      dU[x] = (s == 0 ? 0 : rk->A[s] * dU[x]) + dt * Ut[x];
      U[x] = U[x] + rk->B[s] * dU[x];
    }
  }
}

static void lserk_step(real* U, real* dU, real* Ut, long len, real t, real dt, rhs_fn f, void* ctx) {
  const rk_t rk = rk_default();
  lserk_step_rk(&rk, U, dU, Ut, len, t, dt, f, ctx);
}

/* a scheme from its coefficient arrays (NULL: the default five-stage one) */
static rk_t rk_from(int ns, const double* A, const double* B, const double* C) {
  if (!A || ns < 1 || ns > 32) return rk_default();
  rk_t r;
  r.ns = ns;
  for (int s = 0; s < ns; ++s) { r.A[s] = A[s]; r.B[s] = B[s]; r.C[s] = C[s]; }
  return r;
}

/* Time step (the paper gives no rule; reading):
     lambda_c = sum_d (|u . Ja^d| + c |Ja^d|) / J,
     lambda_v = max(4/3, gamma/Pr) (mu(T)/rho) sum_d |Ja^d|^2 / J^2,
     dt = min(CFL 2 / ((N+1)^2 max lambda_c), DFL 4 / ((N+1)^4 max lambda_v)). */
static real time_step(const mesh_t* M, const params_t* P, const real* U, int* nonfinite) {
  long E = M->E, n3 = M->n3;
  real lc = 0, lv = 0;
  int bad = 0;
  for (long x = 0; x < E * n3; ++x) {
    real q[6];
    cons_to_prim(P, &U[x * 5], q);
    real c = RSQRT(P->gamma * q[4] / q[0]);
    real Jv = M->J[x];
    real a = 0, b = 0;
    for (int d = 0; d < 3; ++d) {
      const real* j = &M->Ja[(x * 3 + d) * 3];
      real nj2 = j[0] * j[0] + j[1] * j[1] + j[2] * j[2];
      a += RABS(q[1] * j[0] + q[2] * j[1] + q[3] * j[2]) + c * RSQRT(nj2);
      b += nj2;
    }
    a /= Jv;
    real kv = (real)4 / 3 > P->gamma / P->Pr ? (real)4 / 3 : P->gamma / P->Pr;
    b = kv * viscosity(P, q[5]) / q[0] * b / (Jv * Jv);
    if (!(a == a) || !(b == b) || !(c == c)) bad = 1;
    if (a > lc) lc = a;
    if (b > lv) lv = b;
  }
  if (nonfinite) *nonfinite = bad;
  real np1 = (real)(M->N + 1);
  real dt = P->cfl * 2 / (np1 * np1 * lc);
  if (P->viscous && lv > 0) {
    real dv = P->dfl * 4 / (np1 * np1 * np1 * np1 * lv);
    if (dv < dt) dt = dv;
  }
  return dt;
}

/* ------------------------------------------------------------------ */
/* Exported API (double at the boundary)                               */
/* ------------------------------------------------------------------ */
typedef struct {
  mesh_t M;
  work_t w;
  params_t P;
} handle_t;

static void to_real(const double* a, real* b, long n) { for (long i = 0; i < n; ++i) b[i] = a[i]; }
static void to_double(const real* a, double* b, long n) { for (long i = 0; i < n; ++i) b[i] = (double)a[i]; }

int ORC(ops)(int N, int gauss, double* x, double* w, double* D, double* Dhat, double* Dsplit, double* Vinv,
             double* Lp, double* Lm) {
  ops_t o;
  if (build_ops(N, gauss, &o)) return -1;
  to_double(o.Lp, Lp, N + 1);
  to_double(o.Lm, Lm, N + 1);
  int n = N + 1;
  to_double(o.x, x, n);
  to_double(o.w, w, n);
  to_double(o.D, D, n * n);
  to_double(o.Dhat, Dhat, n * n);
  to_double(o.Dsplit, Dsplit, n * n);
  to_double(o.Vinv, Vinv, n * n);
  return 0;
}

/* metric_mask: NULL, or a 0/1 mask over elements; metrics are then formed only
   for the masked elements and the two rings of face neighbours around them
   (enough for rhs() with the same mask as `want`). */
/* face_bc (may be NULL: every face has a partner): [E*6] boundary-condition
   row per face (0: inner face); bc: nbc rows of 9 doubles (type, 8 params) */
/* gauss: 0 for the split-form scheme on LGL nodes, 1 for the standard scheme
   on Gauss-Legendre nodes (xyz is still given at the LGL nodes: the geometry) */
void* ORC(mesh_new)(int N, int gauss, long E, const double* xyz, const double* period,
                    const unsigned char* metric_mask, const int* face_bc, int nbc, const double* bc, int* status) {
  handle_t* h = (handle_t*)calloc(1, sizeof(handle_t));
  mesh_t* M = &h->M;
  *status = 0;
  if (build_ops(N, gauss, &M->o)) { *status = -1; free(h); return NULL; }
  M->N = N; M->n = N + 1; M->n2 = M->n * M->n; M->n3 = M->n2 * M->n; M->E = E;
  for (int d = 0; d < 3; ++d) M->period[d] = period[d];
  long n3 = M->n3;
  M->xyz = (real*)malloc(sizeof(real) * E * n3 * 3);
  M->Ja = (real*)malloc(sizeof(real) * E * n3 * 9);
  M->J = (real*)malloc(sizeof(real) * E * n3);
  M->nbr_e = (int*)malloc(sizeof(int) * E * 6);
  M->nbr_f = (int*)malloc(sizeof(int) * E * 6);
  M->master = (int*)malloc(sizeof(int) * E * 6);
  M->nbr_node = (int*)malloc(sizeof(int) * E * 6 * M->n2);
  to_real(xyz, M->xyz, E * n3 * 3);
  M->xyzs = M->xyz;
  if (gauss) M->xyzs = (real*)malloc(sizeof(real) * E * n3 * 3);
  if (nbc > 16) { *status = -6; nbc = 16; }
  M->nbc = nbc;
  for (int k = 0; k < nbc; ++k)
    for (int c = 0; c < 9; ++c) M->bcv[k + 1][c] = bc[k * 9 + c];
  if (face_bc) {
    M->face_bc = (int*)malloc(sizeof(int) * E * 6);
    for (long a = 0; a < E * 6; ++a) {
      M->face_bc[a] = face_bc[a];
      if (face_bc[a] < 0 || face_bc[a] > nbc) *status = -6;
    }
  }
  int st = *status ? *status : build_connectivity(M);
  if (st) { *status = st; }
  unsigned char* need = NULL;
  if (metric_mask && !st) {
    /* the mask, its neighbours (their lifted gradients are needed) and their
       neighbours (master-side normals of the neighbours' faces) */
    need = (unsigned char*)calloc(E, 1);
    unsigned char* ring = (unsigned char*)calloc(E, 1);
    for (long e = 0; e < E; ++e) {
      if (!metric_mask[e]) continue;
      ring[e] = 1;
      for (int f = 0; f < 6; ++f)
        if (M->nbr_e[e * 6 + f] >= 0) ring[M->nbr_e[e * 6 + f]] = 1;
    }
    for (long e = 0; e < E; ++e) {
      if (!ring[e]) continue;
      need[e] = 1;
      for (int f = 0; f < 6; ++f)
        if (M->nbr_e[e * 6 + f] >= 0) need[M->nbr_e[e * 6 + f]] = 1;
    }
    free(ring);
  }
  build_metrics(M, need);
  free(need);
  if (work_alloc(M, &h->w)) *status = -5;
  return h;
}

/* sponge zone: sigma [E][n3] (NULL removes it), base state [E][n3][5] */
void ORC(set_sponge)(void* hv, const double* sigma, const double* base) {
  handle_t* h = (handle_t*)hv;
  mesh_t* M = &h->M;
  free(M->sponge_sigma);
  free(M->sponge_base);
  M->sponge_sigma = M->sponge_base = NULL;
  if (!sigma) return;
  long nn = M->E * M->n3;
  M->sponge_sigma = (real*)malloc(sizeof(real) * nn);
  M->sponge_base = (real*)malloc(sizeof(real) * nn * 5);
  to_real(sigma, M->sponge_sigma, nn);
  to_real(base, M->sponge_base, nn * 5);
}

void ORC(mesh_free)(void* hv) {
  handle_t* h = (handle_t*)hv;
  if (!h) return;
  mesh_t* M = &h->M;
  if (M->xyzs != M->xyz) free(M->xyzs);
  free(M->xyz); free(M->Ja); free(M->J); free(M->nbr_e); free(M->nbr_f); free(M->master);
  free(M->nbr_node);
  free(M->face_bc);
  free(M->sponge_sigma);
  free(M->sponge_base);
  work_free(&h->w);
  free(h);
}

void ORC(connectivity)(void* hv, int* nbr_e, int* nbr_f, int* master, int* nbr_node) {
  mesh_t* M = &((handle_t*)hv)->M;
  long F = M->E * 6;
  memcpy(nbr_e, M->nbr_e, sizeof(int) * F);
  memcpy(nbr_f, M->nbr_f, sizeof(int) * F);
  memcpy(master, M->master, sizeof(int) * F);
  memcpy(nbr_node, M->nbr_node, sizeof(int) * F * M->n2);
}

/* coordinates of the solution nodes [E][n3][3] */
void ORC(node_xyz)(void* hv, double* xyz) {
  mesh_t* M = &((handle_t*)hv)->M;
  to_double(M->xyzs, xyz, M->E * M->n3 * 3);
}

void ORC(metrics)(void* hv, double* Ja, double* J) {
  mesh_t* M = &((handle_t*)hv)->M;
  to_double(M->Ja, Ja, M->E * M->n3 * 9);
  to_double(M->J, J, M->E * M->n3);
}

static real* conv_state(const mesh_t* M, const double* U) {
  long len = M->E * M->n3 * 5;
  real* r = (real*)malloc(sizeof(real) * len);
  to_real(U, r, len);
  return r;
}

int ORC(rhs)(void* hv, const double* prm, const double* U, double t, double* Ut, const unsigned char* want,
             double* alpha, double* grad, double* fstar) {
  handle_t* h = (handle_t*)hv;
  mesh_t* M = &h->M;
  params_t P = read_params(prm);
  long len = M->E * M->n3 * 5;
  real* Ur = conv_state(M, U);
  real* Utr = (real*)calloc(len, sizeof(real));
  real* al = alpha ? (real*)calloc(M->E, sizeof(real)) : NULL;
  real* gr = grad ? (real*)calloc(M->E * M->n3 * 12, sizeof(real)) : NULL;
  real* fr = fstar ? (real*)calloc(M->E * 6 * M->n2 * 5, sizeof(real)) : NULL;
  int st = rhs_any(M, &P, Ur, (real)t, Utr, want, al, gr, fr, &h->w);
  if (fr) { to_double(fr, fstar, M->E * 6 * M->n2 * 5); free(fr); }
  for (long x = 0; x < len; ++x) Ut[x] = (double)Utr[x];
  if (al) { to_double(al, alpha, M->E); free(al); }
  if (gr) { to_double(gr, grad, M->E * M->n3 * 12); free(gr); }
  free(Ur);
  free(Utr);
  return st;
}

typedef struct { handle_t* h; params_t P; int status; } dgctx_t;
static void dg_rhs_cb(void* c, const real* U, real t, real* Ut) {
  dgctx_t* x = (dgctx_t*)c;
  x->status = rhs_any(&x->h->M, &x->P, U, t, Ut, NULL, NULL, NULL, NULL, &x->h->w);
}

double ORC(dt)(void* hv, const double* prm, const double* U, int* nonfinite) {
  handle_t* h = (handle_t*)hv;
  params_t P = read_params(prm);
  real* Ur = conv_state(&h->M, U);
  real dt = time_step(&h->M, &P, Ur, nonfinite);
  free(Ur);
  return (double)dt;
}

/* n_steps LSERK steps; dt_fixed > 0 uses that step, else the CFL rule each step */
int ORC(step)(void* hv, const double* prm, double* U, int n_steps, double dt_fixed, double* t_io,
              double* dt_last, int rk_ns, const double* rk_A, const double* rk_B, const double* rk_C) {
  const rk_t rk = rk_from(rk_ns, rk_A, rk_B, rk_C);
  handle_t* h = (handle_t*)hv;
  mesh_t* M = &h->M;
  dgctx_t c = {h, read_params(prm), 0};
  long len = M->E * M->n3 * 5;
  real* Ur = conv_state(M, U);
  real* dU = (real*)calloc(len, sizeof(real));
  real* Ut = (real*)calloc(len, sizeof(real));
  real t = *t_io, dt = 0;
  int st = 0;
  for (int s = 0; s < n_steps; ++s) {
    int bad = 0;
    dt = dt_fixed > 0 ? (real)dt_fixed : time_step(M, &c.P, Ur, &bad);
    if (bad) { st = -5; break; }
    lserk_step_rk(&rk, Ur, dU, Ut, len, t, dt, dg_rhs_cb, &c);
    if (c.status) { st = c.status; break; }
    t += dt;
  }
  to_double(Ur, U, len);
  *t_io = (double)t;
  if (dt_last) *dt_last = (double)dt;
  free(Ur); free(dU); free(Ut);
  return st;
}

/* E_k = 1/(2|Omega|) int rho |u|^2 and dE_k/dt = 1/|Omega| int (u.(rho u)_t - |u|^2 rho_t / 2)
   by the quadrature of the node set (Sec. 5.2, with rho0 = U0 = 1) */
void ORC(kinetic)(void* hv, const double* U, const double* Ut, double* out) {
  mesh_t* M = &((handle_t*)hv)->M;
  int n = M->n;
  real vol = 0, ek = 0, rate = 0;
  for (long e = 0; e < M->E; ++e)
    for (long v = 0; v < M->n3; ++v) {
      int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / ((long)n * n));
      real wq = M->o.w[i] * M->o.w[j] * M->o.w[k] * M->J[e * M->n3 + v];
      const double* u = &U[(e * M->n3 + v) * 5];
      real r = u[0], vx = u[1] / r, vy = u[2] / r, vz = u[3] / r;
      real v2 = vx * vx + vy * vy + vz * vz;
      vol += wq;
      ek += wq * r * v2 / 2;
      if (Ut) {
        const double* ut = &Ut[(e * M->n3 + v) * 5];
        rate += wq * (vx * ut[1] + vy * ut[2] + vz * ut[3] - v2 * ut[0] / 2);
      }
    }
  out[0] = (double)(ek / vol);
  out[1] = (double)(rate / vol);
  out[2] = (double)vol;
}

/* Solenoidal and dilatational dissipation rates of Sec. 5.2,
     eps_S = 1 / (Re |Omega|) int (mu(T) / mu_0) omega . omega,
     eps_D = 4 / (3 Re |Omega|) int (mu(T) / mu_0) (div u)^2,
   with rho_0 = U_0 = L = 1, so Re = 1 / mu_0 (mu_0 the parameter mu); omega
   and div u from the BR1 lifted velocity gradients of the state, integrated
   by the quadrature of the node set.  out[0] = eps_S, out[1] = eps_D. */
int ORC(dissipation)(void* hv, const double* prm, const double* U, double* out) {
  handle_t* h = (handle_t*)hv;
  mesh_t* M = &h->M;
  params_t P = read_params(prm);
  if (!P.viscous) return -1;
  long len = M->E * M->n3 * 5;
  real* Ur = conv_state(M, U);
  real* Utr = (real*)calloc(len, sizeof(real));
  real* g = (real*)calloc(M->E * M->n3 * 12, sizeof(real));
  int st = rhs_any(M, &P, Ur, 0, Utr, NULL, NULL, g, NULL, &h->w);
  int n = M->n;
  real vol = 0, es = 0, ed = 0;
  for (long e = 0; e < M->E && !st; ++e)
    for (long v = 0; v < M->n3; ++v) {
      int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / ((long)n * n));
      real wq = M->o.w[i] * M->o.w[j] * M->o.w[k] * M->J[e * M->n3 + v];
      const real* d = &g[(e * M->n3 + v) * 12];   /* d[3 a + b] = d u_a / d x_b */
      real q[6];
      cons_to_prim(&P, &Ur[(e * M->n3 + v) * 5], q);
      real r = viscosity(&P, q[5]) / P.mu;
      real wx = d[7] - d[5], wy = d[2] - d[6], wz = d[3] - d[1];
      real dv = d[0] + d[4] + d[8];
      vol += wq;
      es += wq * r * (wx * wx + wy * wy + wz * wz);
      ed += wq * r * dv * dv;
    }
  out[0] = (double)(P.mu * es / vol);
  out[1] = (double)(4 * P.mu * ed / (3 * vol));
  free(Ur); free(Utr); free(g);
  return st;
}

/* ---- point-wise hooks for the pin tests ---- */
void ORC(point_flux)(const double* prm, int kind, const double* UL, const double* UR,
                     const double* nv, double* f) {
  params_t P = read_params(prm);
  real uL[5], uR[5], qL[6], qR[6], n[3], fr[5];
  to_real(UL, uL, 5);
  to_real(UR, uR, 5);
  to_real(nv, n, 3);
  cons_to_prim(&P, uL, qL);
  cons_to_prim(&P, uR, qR);
  if (kind == 0) roe_flux(&P, uL, qL, uR, qR, n, fr);
  else if (kind == 1) lf_flux(&P, uL, qL, uR, qR, n, fr);
  else if (kind == 2) kep_flux(uL, qL, uR, qR, n, fr);
  else euler_flux(uL, qL, n, fr);
  to_double(fr, f, 5);
}

/* the manufactured-solution source at points x [n][3], time t */
void ORC(mms_source)(const double* prm, long npts, const double* x, double t, double* Q) {
  params_t P = read_params(prm);
  for (long i = 0; i < npts; ++i) {
    real xr[3] = {x[i * 3], x[i * 3 + 1], x[i * 3 + 2]}, q[5];
    mms_source(&P, xr, (real)t, q);
    for (int k = 0; k < 5; ++k) Q[i * 5 + k] = (double)q[k];
  }
}

void ORC(point_visc)(const double* prm, const double* U, const double* g, const double* nv, double* f) {
  params_t P = read_params(prm);
  real u[5], q[6], gg[12], n[3], fr[5];
  to_real(U, u, 5);
  to_real(g, gg, 12);
  to_real(nv, n, 3);
  cons_to_prim(&P, u, q);
  visc_flux(&P, q, gg, n, fr);
  to_double(fr, f, 5);
}

/* indicator of one element's state U[n3][5] at degree N */
double ORC(indicator)(int N, const double* prm, const double* U, double* E_out) {
  static mesh_t M;
  if (build_ops(N, 0, &M.o)) return -1;
  M.N = N; M.n = N + 1; M.n2 = M.n * M.n; M.n3 = M.n2 * M.n;
  params_t P = read_params(prm);
  real q[NMAX * NMAX * NMAX * 6], u[5];
  for (long v = 0; v < M.n3; ++v) {
    to_real(&U[v * 5], u, 5);
    cons_to_prim(&P, u, &q[v * 6]);
  }
  real Ei = 0;
  real a = indicator(&M, &P, q, &Ei);
  if (E_out) *E_out = (double)Ei;
  return (double)a;
}

/* LSERK on scalar ODEs, for the order and stability-polynomial pins.
   kind 0: y' = lam y;  kind 1: y' = -y^2 + cos(t) */
typedef struct { int kind; real lam; } odectx_t;
static void ode_cb(void* c, const real* y, real t, real* yt) {
  odectx_t* o = (odectx_t*)c;
  if (o->kind == 0) yt[0] = o->lam * y[0];
  else yt[0] = -y[0] * y[0] + (real)cos((double)t);
}
double ORC(lserk_ode)(int kind, double lam, double y0, double dt, int n_steps, int rk_ns, const double* rk_A,
                      const double* rk_B, const double* rk_C) {
  const rk_t rk = rk_from(rk_ns, rk_A, rk_B, rk_C);
  odectx_t c = {kind, (real)lam};
  real y = y0, dy = 0, yt = 0, t = 0;
  for (int s = 0; s < n_steps; ++s) {
    lserk_step_rk(&rk, &y, &dy, &yt, 1, t, (real)dt, ode_cb, &c);
    t += dt;
  }
  return (double)y;
}

void ORC(rk_coeffs)(double* A, double* B, double* C) {
  for (int s = 0; s < 5; ++s) { A[s] = RK_A[s]; B[s] = RK_B[s]; C[s] = RK_C[s]; }
}

/* the fourteen-stage table (14 entries each) */
void ORC(rk14_coeffs)(double* A, double* B, double* C) {
  for (int s = 0; s < 14; ++s) { A[s] = RK14_A[s]; B[s] = RK14_B[s]; C[s] = RK14_C[s]; }
}
