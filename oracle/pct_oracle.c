/*
 * pct_oracle.c -- plain, slow FP64 CPU oracle for the proton-CT hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg load this file. The product path
 * (the CUDA library) shares no code, header, table or constant generator with
 * it, and neither includes nor links the other.
 *
 * What it computes (arXiv 1707.05014):
 *   Sec. 2   : each proton's most-likely path (MLP) from its entry/exit
 *              position and direction; the path lengths in the voxels it
 *              touches form its row of A in A x = b (b = WEPL).
 *   Sec. 2.1 : DROP -- block-sequential diagonally relaxed orthogonal
 *              projections over a user-chosen number of blocks, a fixed
 *              number of iterations (Fig. 1).
 *   Sec. 2.2 : CARP -- strings swept from a common image, then component
 *              averaging (Fig. 2).
 *   Sec. 4.2 : total-variation superiorization inside DROP and CARP.
 *   Object hull: the cited MLP estimator runs inside the object and takes
 *              the path straight outside it; hull entry/exit nodes and a
 *              hull carved from the data.
 * Every function is pinned by tests against what the paper and the
 * mathematics fix (closed forms, limits, brute force, independent physics).
 * The paper cites the MLP formalism (Schulte et al. 2008) without printing it;
 * this file follows that published form directly:
 *     y1 = (S1^-1 + R1^T S2^-1 R1)^-1 (S1^-1 R0 y0 + R1^T S2^-1 y2),
 * with y = (lateral position, slope), S1/S2 the scattering matrices before and
 * after the node, integrated here by 64-point Gauss-Legendre quadrature.
 *
 * Readings where the paper is silent:
 *   - 1/(beta^2 p^2)(w) is Schulte's 5th-order water polynomial for 200 MeV,
 *     w = depth from the entry plane in cm; Highland factor
 *     E0^2 (1 + 0.038 ln(L/X0))^2 / X0 with L the sub-path length.
 *   - measurement planes at u = -R and +R, R the inscribed radius of the grid;
 *     nodes every du = 2R/K, K = ceil(2R / step), step = min(h)/2 by default;
 *     straight extensions before u0 / after u2 along the measured slopes.
 *   - nodes are quantised to Q20 fixed point in grid units (round half even,
 *     clamped to +-1000 voxels) and walked by an exact integer DDA: voxels
 *     are half-open, tied face crossings step together, zero-length runs are
 *     never emitted, a run is a maximal stretch in one voxel. In the FP32
 *     mode the grid coordinate is formed 16 voxels above its value
 *     (fma(p, 1/h, n/2 + 16)) and the 16 voxels are taken off after the
 *     rounding: every coordinate within 8 voxels of the grid is then at
 *     least 8, where an FP32 value is already a whole multiple of 2^-20, so
 *     the quantisation only rounds coordinates far outside the grid.
 *   - DROP: x <- x + lambda S_b^-1 sum_{i in b} a_i (b_i - a_i.x)/|a_i|^2 with
 *     S_b = diag(number of runs in voxel j over block b); block b holds
 *     protons [b N / B, (b+1) N / B).
 *
 * Two node modes: OR_MODE_FP64 evaluates the nodes in double; OR_MODE_FP32
 * evaluates them with a fixed single-precision operation order (fmaf, no
 * contraction -- compile with -ffp-contract=off) so that the quantised nodes,
 * and so the voxel index lists, are defined bit for bit. Chord lengths and the
 * solver always run in double.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_QBITS 20
#define OR_QONE ((int64_t)1 << OR_QBITS)
#define OR_QCLAMP 1000.0

#define OR_F_CONST_SCATTER 1 /* test only: 1/(beta^2 p^2) held at its entry value */
#define OR_F_NO_LOG 2        /* test only: drop the logarithmic Highland term   */

#define OR_MODE_FP64 0
#define OR_MODE_FP32 1

typedef struct {
  int nx, ny, nz;
  double hx, hy, hz;
  double node_step;     /* <= 0: min(h)/2 */
  const uint8_t *hull;  /* object hull, one byte per voxel (nonzero = inside); NULL: none */
} or_grid;

typedef struct {
  const float *t0, *v0, *st0, *sv0, *t2, *v2, *st2, *sv2, *wepl, *cphi, *sphi;
} or_rec;

typedef struct {
  double R, du, u0;
  int K; /* interior nodes k = 0..K, u_k = u0 + k du */
  int E; /* straight extension nodes per side */
} or_geom;

/* ------------------------------------------------------------------ */
/* Geometry                                                            */
/* ------------------------------------------------------------------ */

static void or_geometry(const or_grid *g, or_geom *o) {
  double X = g->nx * g->hx, Y = g->ny * g->hy;
  double hmin = fmin(g->hx, fmin(g->hy, g->hz));
  double step = g->node_step > 0 ? g->node_step : 0.5 * hmin;
  o->R = 0.5 * fmin(X, Y);
  o->K = (int)ceil(2.0 * o->R / step - 1e-9);
  o->du = 2.0 * o->R / o->K;
  o->u0 = -o->R;
  /* every point with |u| beyond the half diagonal of the xy box is outside */
  o->E = (int)ceil((0.5 * sqrt(X * X + Y * Y) - o->R) / o->du) + 2;
}

/* Planes at u = -R and +R, node spacing du, K node intervals between the
 * planes and E extension nodes on each side (Sec. 2 fixes none of these; the
 * readings are listed in the header comment). */
int or_geom_info(const or_grid *g, double *R, double *du, int *K, int *E) {
  or_geom o;
  or_geometry(g, &o);
  *R = o.R;
  *du = o.du;
  *K = o.K;
  *E = o.E;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Scattering model (Schulte et al. 2008, cited in Sec. 2)             */
/* ------------------------------------------------------------------ */

static const double OR_A[6] = {7.457e-6, 4.548e-7, -5.777e-8, 1.301e-8, -9.228e-10, 2.687e-11};
static const double OR_E0 = 13.6;  /* MeV  */
static const double OR_X0 = 36.08; /* cm, radiation length of water */

/* 1/(beta^2 p^2) at water depth w (cm), MeV^-2: the 200 MeV water polynomial
 * of the MLP formalism that Sec. 2 cites */
double or_inv_beta2p2(double w, int flags) {
  if (flags & OR_F_CONST_SCATTER) return OR_A[0];
  double s = 0.0, wp = 1.0;
  for (int i = 0; i < 6; ++i) {
    s += OR_A[i] * wp;
    wp *= w;
  }
  return s;
}

/* E0^2 (1 + 0.038 ln(L/X0))^2 / X0 */
static double or_highland(double L, int flags) {
  double f = 1.0;
  if (!(flags & OR_F_NO_LOG)) f = 1.0 + 0.038 * log(L / OR_X0);
  return OR_E0 * OR_E0 * f * f / OR_X0;
}

/* n-point Gauss-Legendre nodes/weights on [-1, 1] by Newton on P_n */
void or_gauss_legendre(int n, double *x, double *w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z; /* P_0, P_1 */
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      /* p1 = P_n(z), p0 = P_{n-1}(z) */
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

#define OR_NGL 64
static double or_glx[OR_NGL], or_glw[OR_NGL];
static int or_gl_ready = 0;

/* integral over w in [a, b] of (c - w)^m / (beta^2 p^2)(w) dw: the moments
 * that make up the MLP's scattering matrices (Sec. 2, cited formalism) */
double or_moment(double a, double b, double c, int m, int flags) {
  if (!or_gl_ready) {
    or_gauss_legendre(OR_NGL, or_glx, or_glw);
    or_gl_ready = 1;
  }
  double half = 0.5 * (b - a), mid = 0.5 * (a + b), s = 0.0;
  for (int i = 0; i < OR_NGL; ++i) {
    double w = mid + half * or_glx[i];
    s += or_glw[i] * pow(c - w, m) * or_inv_beta2p2(w, flags);
  }
  return s * half;
}

/* Scattering covariance of the (position, slope) state over the water slab
 * from depth a to depth b (cm): E0^2 (1 + 0.038 ln((b-a)/X0))^2 / X0 times
 * [int (b-w)^2 f, int (b-w) f, int f] over [a, b], f = 1/(beta^2 p^2)
 * (the cited MLP formalism; the log term takes the slab's own thickness).
 * out: position-position, position-slope, slope-slope (rad^2 for the last;
 * lengths in cm). */
void or_scatter_cov(double a, double b, int flags, double *out) {
  const double k = or_highland(b - a, flags);
  out[0] = k * or_moment(a, b, b, 2, flags);
  out[1] = k * or_moment(a, b, b, 1, flags);
  out[2] = k * or_moment(a, b, b, 0, flags);
}

static void inv2(const double a[2][2], double o[2][2]) {
  double det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
  o[0][0] = a[1][1] / det;
  o[0][1] = -a[0][1] / det;
  o[1][0] = -a[1][0] / det;
  o[1][1] = a[0][0] / det;
}

static void mul2(const double a[2][2], const double b[2][2], double o[2][2]) {
  double t[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) t[i][j] = a[i][0] * b[0][j] + a[i][1] * b[1][j];
  memcpy(o, t, sizeof t);
}

/*
 * MLP coefficients of the nodes m = 0..n, spaced du (mm), of a water layer of
 * thickness W (cm) that the proton enters at m = 0 and leaves at m = n: the
 * first rows of H^-1 S1^-1 R0 -> (c1, c2) and of H^-1 R1^T S2^-1 -> (c3, c4),
 * so that t_m = c1 t_in + c2 s_in + c3 t_out + c4 s_out (positions in mm,
 * c2/c4 in mm). The end nodes take the measured values exactly. out: (n+1)*4.
 */
static void or_table_fill(double W, double du, int n, int flags, double *out) {
  for (int k = 0; k <= n; ++k) {
    double *c = out + 4 * k;
    if (k == 0 || k == n) {
      c[0] = (k == 0);
      c[1] = 0.0;
      c[2] = (k == n);
      c[3] = 0.0;
      continue;
    }
    double w1 = k * du / 10.0; /* node depth, cm */
    double c1[3], c2[3];
    or_scatter_cov(0.0, w1, flags, c1); /* entry plane -> node */
    or_scatter_cov(w1, W, flags, c2);   /* node -> exit plane */
    double S1[2][2] = {{c1[0], c1[1]}, {c1[1], c1[2]}};
    double S2[2][2] = {{c2[0], c2[1]}, {c2[1], c2[2]}};
    double R0[2][2] = {{1.0, w1}, {0.0, 1.0}};
    double R1[2][2] = {{1.0, W - w1}, {0.0, 1.0}};
    double R1T[2][2] = {{1.0, 0.0}, {W - w1, 1.0}};
    double S1i[2][2], S2i[2][2], H[2][2], Hi[2][2], T[2][2], Ma[2][2], Mb[2][2];
    inv2(S1, S1i);
    inv2(S2, S2i);
    mul2(R1T, S2i, T); /* R1^T S2^-1 */
    mul2(T, R1, H);    /* R1^T S2^-1 R1 */
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) H[i][j] += S1i[i][j];
    inv2(H, Hi);
    mul2(Hi, S1i, Ma);
    mul2(Ma, R0, Ma); /* H^-1 S1^-1 R0 */
    mul2(Hi, T, Mb);  /* H^-1 R1^T S2^-1 */
    c[0] = Ma[0][0];
    c[1] = 10.0 * Ma[0][1];
    c[2] = Mb[0][0];
    c[3] = 10.0 * Mb[0][1];
  }
}

/* MLP table between the measurement planes (Sec. 2; the whole slab, W = 2R):
 * nodes k = 0..K at depth u_k. out: (K+1)*4. */
int or_mlp_table(const or_grid *g, int flags, double *out) {
  or_geom o;
  or_geometry(g, &o);
  or_table_fill(2.0 * o.R / 10.0, o.du, o.K, flags, out);
  return o.K;
}

/* Table of a hull of n node intervals (thickness n du; n = K is the slab):
 * the cited MLP estimator run inside the object only (Sec. 2). */
static double or_layer_cm(const or_geom *o, int n) { return n == o->K ? 2.0 * o->R / 10.0 : n * o->du / 10.0; }

int or_mlp_table_n(const or_grid *g, int flags, int n, double *out) {
  or_geom o;
  or_geometry(g, &o);
  if (n < 1 || n > o.K) return -1;
  or_table_fill(or_layer_cm(&o, n), o.du, n, flags, out);
  return n;
}

/* Tables per hull thickness, computed on first use for the current geometry. */
static double **or_fam = NULL;
static int or_fam_K = -1;
static double or_fam_du = 0.0, or_fam_R = 0.0;

static const double *or_family_locked(const or_geom *o, int n);

static const double *or_family(const or_geom *o, int n) {
  const double *t;
#ifdef _OPENMP
#pragma omp critical(or_family_cache)
#endif
  t = or_family_locked(o, n);
  return t;
}

static const double *or_family_locked(const or_geom *o, int n) {
  if (or_fam_K != o->K || or_fam_du != o->du || or_fam_R != o->R) {
    if (or_fam) {
      for (int i = 0; i <= or_fam_K; ++i) free(or_fam[i]);
      free(or_fam);
    }
    or_fam = (double **)calloc((size_t)o->K + 1, sizeof(double *));
    or_fam_K = o->K;
    or_fam_du = o->du;
    or_fam_R = o->R;
  }
  if (!or_fam[n]) {
    or_fam[n] = (double *)malloc(((size_t)n + 1) * 4 * sizeof(double));
    or_table_fill(or_layer_cm(o, n), o->du, n, 0, or_fam[n]);
  }
  return or_fam[n];
}

/* ------------------------------------------------------------------ */
/* Nodes                                                               */
/* ------------------------------------------------------------------ */

static int32_t or_quant_d(double q) {
  if (q < -OR_QCLAMP) q = -OR_QCLAMP;
  if (q > OR_QCLAMP) q = OR_QCLAMP;
  return (int32_t)lrint(q * (double)OR_QONE); /* default mode: half to even */
}

/* FP32 mode: grid coordinates are formed OR_QOFF voxels above their value and
 * the offset is removed after rounding (see the readings above). */
#define OR_QOFF 16

static int32_t or_quant_f(float q) {
  if (q < (float)-OR_QCLAMP) q = (float)-OR_QCLAMP;
  if (q > (float)OR_QCLAMP) q = (float)OR_QCLAMP;
  return (int32_t)lrintf(q * 1048576.0f) - (int32_t)(OR_QOFF * OR_QONE);
}

/*
 * Path of one proton: straight along the measured entry direction up to node
 * iin, the MLP of the layer between nodes iin and iout (table tab, entries
 * m = k - iin), straight along the measured exit direction from node iout.
 * Without a hull iin = 0, iout = K (the measurement planes, the slab table).
 * With one, iin is the first node k in [0, K] whose entry-ray point lies in a
 * hull voxel and iout the last node whose exit-ray point does (a proton with
 * no such pair keeps the slab).
 */
typedef struct {
  int iin, iout;
  const double *tab;
} or_path;

/* grid coordinates of the point (u, t, v) -> Q20 */
static void or_quantise_d(const or_grid *g, const or_rec *r, int64_t i, double u, double t, double v, int32_t Q[3]) {
  double cp = r->cphi[i], sp = r->sphi[i];
  double x = u * cp - t * sp, y = u * sp + t * cp, z = v;
  Q[0] = or_quant_d(x / g->hx + 0.5 * g->nx);
  Q[1] = or_quant_d(y / g->hy + 0.5 * g->ny);
  Q[2] = or_quant_d(z / g->hz + 0.5 * g->nz);
}

static void or_quantise_f(const or_grid *g, const or_rec *r, int64_t i, float u, float t, float v, int32_t Q[3]) {
  float cp = r->cphi[i], sp = r->sphi[i];
  float ts = t * sp, tc = t * cp;
  float x = fmaf(u, cp, -ts);
  float y = fmaf(u, sp, tc);
  float ihx = (float)(1.0 / g->hx), ihy = (float)(1.0 / g->hy), ihz = (float)(1.0 / g->hz);
  Q[0] = or_quant_f(fmaf(x, ihx, 0.5f * (float)g->nx + (float)OR_QOFF));
  Q[1] = or_quant_f(fmaf(y, ihy, 0.5f * (float)g->ny + (float)OR_QOFF));
  Q[2] = or_quant_f(fmaf(v, ihz, 0.5f * (float)g->nz + (float)OR_QOFF));
}

/* Lateral/vertical position at node k of the entry ray (exit = 0) or the
 * exit ray (exit = 1), both modes. */
static void or_ray_d(const or_geom *o, const or_rec *r, int64_t i, int exit, int k, double *t, double *v) {
  if (!exit) {
    *t = (double)r->t0[i] + (double)r->st0[i] * (k * o->du);
    *v = (double)r->v0[i] + (double)r->sv0[i] * (k * o->du);
  } else {
    *t = (double)r->t2[i] + (double)r->st2[i] * ((k - o->K) * o->du);
    *v = (double)r->v2[i] + (double)r->sv2[i] * ((k - o->K) * o->du);
  }
}

static void or_ray_f(const or_geom *o, const or_rec *r, int64_t i, int exit, int k, float *t, float *v) {
  float du = (float)o->du;
  if (!exit) {
    float dk = (float)k * du;
    *t = fmaf(r->st0[i], dk, r->t0[i]);
    *v = fmaf(r->sv0[i], dk, r->v0[i]);
  } else {
    float dk = (float)(k - o->K) * du;
    *t = fmaf(r->st2[i], dk, r->t2[i]);
    *v = fmaf(r->sv2[i], dk, r->v2[i]);
  }
}

/* Q20 point of node k on the entry or exit ray */
static void or_ray_node(const or_grid *g, const or_geom *o, const or_rec *r, int64_t i, int mode, int exit, int k,
                        int32_t Q[3]) {
  if (mode == OR_MODE_FP64) {
    double t, v;
    or_ray_d(o, r, i, exit, k, &t, &v);
    or_quantise_d(g, r, i, o->u0 + k * o->du, t, v, Q);
  } else {
    float t, v;
    or_ray_f(o, r, i, exit, k, &t, &v);
    or_quantise_f(g, r, i, fmaf((float)k, (float)o->du, (float)o->u0), t, v, Q);
  }
}

static int64_t or_floor_div(int64_t a);

/* the voxel holding Q is inside the grid and the hull */
static int or_in_hull(const or_grid *g, const int32_t Q[3]) {
  int64_t ix = or_floor_div(Q[0]), iy = or_floor_div(Q[1]), iz = or_floor_div(Q[2]);
  if (ix < 0 || ix >= g->nx || iy < 0 || iy >= g->ny || iz < 0 || iz >= g->nz) return 0;
  return g->hull[ix + (int64_t)g->nx * (iy + (int64_t)g->ny * iz)] != 0;
}

static void or_path_of(const or_grid *g, const or_geom *o, const double *tab, const or_rec *r, int64_t i, int mode,
                       or_path *p) {
  p->iin = 0;
  p->iout = o->K;
  p->tab = tab;
  if (!g->hull) return;
  int32_t Q[3];
  int iin = -1, iout = -1;
  for (int k = 0; k <= o->K && iin < 0; ++k) {
    or_ray_node(g, o, r, i, mode, 0, k, Q);
    if (or_in_hull(g, Q)) iin = k;
  }
  for (int k = o->K; k >= 0 && iout < 0; --k) {
    or_ray_node(g, o, r, i, mode, 1, k, Q);
    if (or_in_hull(g, Q)) iout = k;
  }
  if (iin < 0 || iout < 0 || iout <= iin) return; /* misses the hull */
  p->iin = iin;
  p->iout = iout;
  p->tab = iout - iin == o->K ? tab : or_family(o, iout - iin);
}

/* Quantised node k of proton i in grid units (Q20) on path p. */
static void or_node(const or_grid *g, const or_geom *o, const or_path *p, const or_rec *r, int64_t i, int mode, int k,
                    int32_t Q[3]) {
  if (k <= p->iin || k >= p->iout) {
    or_ray_node(g, o, r, i, mode, k >= p->iout, k, Q);
    return;
  }
  const double *c = p->tab + 4 * (k - p->iin);
  if (mode == OR_MODE_FP64) {
    double tin, vin, tout, vout;
    or_ray_d(o, r, i, 0, p->iin, &tin, &vin);
    or_ray_d(o, r, i, 1, p->iout, &tout, &vout);
    double t = c[0] * tin + c[1] * r->st0[i] + c[2] * tout + c[3] * r->st2[i];
    double v = c[0] * vin + c[1] * r->sv0[i] + c[2] * vout + c[3] * r->sv2[i];
    or_quantise_d(g, r, i, o->u0 + k * o->du, t, v, Q);
  } else {
    /* fixed single-precision order (the bit-exact contract) */
    float tin, vin, tout, vout;
    or_ray_f(o, r, i, 0, p->iin, &tin, &vin);
    or_ray_f(o, r, i, 1, p->iout, &tout, &vout);
    float c1 = (float)c[0], c2 = (float)c[1], c3 = (float)c[2], c4 = (float)c[3];
    float a = c1 * tin;
    float t = fmaf(c4, r->st2[i], fmaf(c3, tout, fmaf(c2, r->st0[i], a)));
    float b = c1 * vin;
    float v = fmaf(c4, r->sv2[i], fmaf(c3, vout, fmaf(c2, r->sv0[i], b)));
    or_quantise_f(g, r, i, fmaf((float)k, (float)o->du, (float)o->u0), t, v, Q);
  }
}

/* Hull entry/exit nodes of protons [first, first+count): out (count, 2)
 * (where the MLP of Sec. 2 starts and ends with an object hull). */
int or_hull_ranges(const or_grid *g, const double *tab, const or_rec *r, int64_t first, int64_t count, int mode,
                   int32_t *out) {
  or_geom o;
  or_geometry(g, &o);
  for (int64_t p = 0; p < count; ++p) {
    or_path pa;
    or_path_of(g, &o, tab, r, first + p, mode, &pa);
    out[2 * p] = pa.iin;
    out[2 * p + 1] = pa.iout;
  }
  return 0;
}

/* MLP nodes k = 0..K of protons [first, first+count) (Sec. 2), quantised:
 * out (count, K+1, 3) */
int or_nodes(const or_grid *g, const double *tab, const or_rec *r, int64_t first, int64_t count, int mode,
             int32_t *out) {
  or_geom o;
  or_geometry(g, &o);
  for (int64_t p = 0; p < count; ++p) {
    or_path pa;
    or_path_of(g, &o, tab, r, first + p, mode, &pa);
    for (int k = 0; k <= o.K; ++k) or_node(g, &o, &pa, r, first + p, mode, k, out + 3 * ((int64_t)p * (o.K + 1) + k));
  }
  return 0;
}

/* All polyline nodes k = -E..K+E of proton i (the MLP of Sec. 2 with its
 * straight extensions): out (K + 2E + 1, 3) */
int or_polyline(const or_grid *g, const double *tab, const or_rec *r, int64_t i, int mode, int32_t *out) {
  or_geom o;
  or_geometry(g, &o);
  or_path pa;
  or_path_of(g, &o, tab, r, i, mode, &pa);
  for (int k = -o.E; k <= o.K + o.E; ++k) or_node(g, &o, &pa, r, i, mode, k, out + 3 * (int64_t)(k + o.E));
  return o.K + 2 * o.E + 1;
}

/* ------------------------------------------------------------------ */
/* Voxel walk (row of A)                                               */
/* ------------------------------------------------------------------ */

typedef struct {
  int32_t *j;
  double *l;
  int64_t n, cap;
} or_row;

static void or_row_push(or_row *w, int32_t j, double l) {
  if (w->n == w->cap) {
    w->cap = w->cap ? 2 * w->cap : 256;
    w->j = (int32_t *)realloc(w->j, w->cap * sizeof(int32_t));
    w->l = (double *)realloc(w->l, w->cap * sizeof(double));
  }
  w->j[w->n] = j;
  w->l[w->n] = l;
  w->n++;
}

static int64_t or_floor_div(int64_t a) { /* floor(a / 2^20) */
  return a >= 0 ? a / OR_QONE : -((-a + OR_QONE - 1) / OR_QONE);
}

typedef struct {
  int64_t cur[3];   /* current voxel */
  double len;       /* run length so far, mm */
  int pos;          /* run has strictly positive extent */
  int started;
} or_walk;

static void or_emit(const or_grid *g, or_walk *s, or_row *row) {
  if (s->pos && s->cur[0] >= 0 && s->cur[0] < g->nx && s->cur[1] >= 0 && s->cur[1] < g->ny && s->cur[2] >= 0 &&
      s->cur[2] < g->nz)
    or_row_push(row, (int32_t)(s->cur[0] + (int64_t)g->nx * (s->cur[1] + (int64_t)g->ny * s->cur[2])), s->len);
  s->len = 0.0;
  s->pos = 0;
}

/* Walk the straight segment P -> E (Q20 grid units), appending finished runs. */
static void or_segment(const or_grid *g, const int32_t P[3], const int32_t E[3], or_walk *s, or_row *row) {
  const double h[3] = {g->hx, g->hy, g->hz};
  int64_t D[3], dist[3], step[3];
  int a;
  if (P[0] == E[0] && P[1] == E[1] && P[2] == E[2]) return;
  for (a = 0; a < 3; ++a) {
    int64_t c = or_floor_div(P[a]);
    if (!s->started) s->cur[a] = c;
    D[a] = (int64_t)E[a] - P[a];
    step[a] = D[a] > 0 ? 1 : (D[a] < 0 ? -1 : 0);
    /* distance from P to the next face in the direction of travel */
    dist[a] = D[a] > 0 ? (c + 1) * OR_QONE - P[a] : (D[a] < 0 ? P[a] - c * OR_QONE : 0);
  }
  s->started = 1;
  double L = 0.0;
  for (a = 0; a < 3; ++a) {
    double d = (double)D[a] * h[a] / (double)OR_QONE;
    L += d * d;
  }
  L = sqrt(L);
  /* previous crossing parameter as an exact fraction pn/pd (starts at 0) */
  int64_t pn = 0, pd = 1;
  double tprev = 0.0;
  for (;;) {
    /* axes whose next face lies within the segment: tau = dist/|D| <= 1 when
       moving up (a point on a face belongs to the higher voxel), < 1 down */
    int cand[3], any = 0;
    for (a = 0; a < 3; ++a) {
      int64_t ad = D[a] < 0 ? -D[a] : D[a];
      cand[a] = D[a] > 0 ? dist[a] <= ad : (D[a] < 0 ? dist[a] < ad : 0);
      any |= cand[a];
    }
    if (!any) break;
    /* smallest tau among candidates, compared exactly */
    int best = -1;
    for (a = 0; a < 3; ++a) {
      if (!cand[a]) continue;
      if (best < 0) {
        best = a;
        continue;
      }
      __int128 lhs = (__int128)dist[a] * (D[best] < 0 ? -D[best] : D[best]);
      __int128 rhs = (__int128)dist[best] * (D[a] < 0 ? -D[a] : D[a]);
      if (lhs < rhs) best = a;
    }
    int64_t bn = dist[best], bd = D[best] < 0 ? -D[best] : D[best];
    double tc = (double)bn / (double)bd;
    s->len += (tc - tprev) * L;
    if ((__int128)bn * pd > (__int128)pn * bd) s->pos = 1;
    or_emit(g, s, row);
    /* every axis tied with the minimum steps now */
    for (a = 0; a < 3; ++a) {
      if (!cand[a]) continue;
      int64_t ad = D[a] < 0 ? -D[a] : D[a];
      if ((__int128)dist[a] * bd == (__int128)bn * ad) {
        s->cur[a] += step[a];
        dist[a] += OR_QONE;
      }
    }
    pn = bn;
    pd = bd;
    tprev = tc;
  }
  s->len += (1.0 - tprev) * L;
  if (pn < pd) s->pos = 1;
}

/* Row of proton i: runs (voxel, chord mm) in path order. */
static void or_walk_row(const or_grid *g, const or_geom *o, const double *tab, const or_rec *r, int64_t i, int mode,
                        or_row *row) {
  or_walk s;
  memset(&s, 0, sizeof s);
  row->n = 0;
  int32_t P[3], E[3];
  or_path pa;
  or_path_of(g, o, tab, r, i, mode, &pa);
  or_node(g, o, &pa, r, i, mode, -o->E, P);
  for (int k = -o->E + 1; k <= o->K + o->E; ++k) {
    or_node(g, o, &pa, r, i, mode, k, E);
    or_segment(g, P, E, &s, row);
    P[0] = E[0];
    P[1] = E[1];
    P[2] = E[2];
  }
  or_emit(g, &s, row);
}

/*
 * Rows of A (Sec. 2: the path length of each proton in every voxel it
 * touches) for protons [first, first+count) in CSR form. row_ptr has count+1
 * entries. Writes at most cap runs; returns the number needed (>= 0).
 */
int64_t or_rows(const or_grid *g, const double *tab, const or_rec *r, int64_t first, int64_t count, int mode,
                int64_t *row_ptr, int32_t *vox, double *len, int64_t cap) {
  or_geom o;
  or_geometry(g, &o);
  or_row row = {0};
  int64_t tot = 0;
  row_ptr[0] = 0;
  for (int64_t p = 0; p < count; ++p) {
    or_walk_row(g, &o, tab, r, first + p, mode, &row);
    for (int64_t q = 0; q < row.n; ++q, ++tot)
      if (tot < cap) {
        vox[tot] = row.j[q];
        len[tot] = row.l[q];
      }
    row_ptr[p + 1] = tot;
  }
  free(row.j);
  free(row.l);
  return tot;
}

/*
 * Space-carved object hull: every voxel on the row of a proton whose WEPL is
 * at most wepl_max (it crossed air only) is outside the object; the hull is
 * the rest of the grid, grown by `dilate` steps of the 6-neighbourhood.
 * Rows are walked without a hull (g->hull is ignored). out: M bytes.
 */
int or_carve_hull(const or_grid *g, const double *tab, const or_rec *r, int64_t n, double wepl_max, int dilate,
                  int mode, uint8_t *out) {
  or_grid gp = *g;
  gp.hull = NULL;
  or_geom o;
  or_geometry(&gp, &o);
  const int64_t M = (int64_t)g->nx * g->ny * g->nz;
  for (int64_t j = 0; j < M; ++j) out[j] = 1;
  or_row row = {0};
  for (int64_t i = 0; i < n; ++i) {
    if (!(r->wepl[i] <= wepl_max)) continue;
    or_walk_row(&gp, &o, tab, r, i, mode, &row);
    for (int64_t q = 0; q < row.n; ++q) out[row.j[q]] = 0;
  }
  free(row.j);
  free(row.l);
  uint8_t *tmp = (uint8_t *)malloc((size_t)M);
  for (int it = 0; it < dilate; ++it) {
    memcpy(tmp, out, (size_t)M);
    for (int64_t z = 0; z < g->nz; ++z)
      for (int64_t y = 0; y < g->ny; ++y)
        for (int64_t x = 0; x < g->nx; ++x) {
          int64_t j = x + g->nx * (y + g->ny * z);
          if (tmp[j]) continue;
          int hit = (x > 0 && tmp[j - 1]) || (x + 1 < g->nx && tmp[j + 1]) || (y > 0 && tmp[j - g->nx]) ||
                    (y + 1 < g->ny && tmp[j + g->nx]) || (z > 0 && tmp[j - (int64_t)g->nx * g->ny]) ||
                    (z + 1 < g->nz && tmp[j + (int64_t)g->nx * g->ny]);
          if (hit) out[j] = 1;
        }
  }
  free(tmp);
  return 0;
}

/* y_i = a_i . x for protons [first, first+count): the WEPL the image x
 * predicts for each proton (Sec. 2, A x = b). */
int or_project(const or_grid *g, const double *tab, const or_rec *r, int64_t first, int64_t count, int mode,
               const double *x, double *y) {
  or_geom o;
  or_geometry(g, &o);
  or_row row = {0};
  for (int64_t p = 0; p < count; ++p) {
    or_walk_row(g, &o, tab, r, first + p, mode, &row);
    double s = 0.0;
    for (int64_t q = 0; q < row.n; ++q) s += row.l[q] * x[row.j[q]];
    y[p] = s;
  }
  free(row.j);
  free(row.l);
  return 0;
}

/* Run counts s_j of block b (rows of protons [b N/B, (b+1) N/B)): the
 * diagonal weights of the DROP block update (Sec. 2.1). out: M */
int or_block_counts(const or_grid *g, const double *tab, const or_rec *r, int64_t n, int n_blocks, int b, int mode,
                    double *out) {
  or_geom o;
  or_geometry(g, &o);
  int64_t M = (int64_t)g->nx * g->ny * g->nz;
  memset(out, 0, M * sizeof(double));
  or_row row = {0};
  int64_t lo = (int64_t)b * n / n_blocks, hi = (int64_t)(b + 1) * n / n_blocks;
  for (int64_t i = lo; i < hi; ++i) {
    or_walk_row(g, &o, tab, r, i, mode, &row);
    for (int64_t q = 0; q < row.n; ++q) out[row.j[q]] += 1.0;
  }
  free(row.j);
  free(row.l);
  return 0;
}

/* ------------------------------------------------------------------ */
/* DROP (Sec. 2.1, Fig. 1)                                             */
/* ------------------------------------------------------------------ */

/*
 * x (M, in/out: the initial guess on entry, the result on exit).
 * For sweep = 1..n_sweeps, for block b = 0..B-1:
 *   delta = 0, s = 0
 *   for i in block b: a_i = row i; r_i = lambda (b_i - a_i.x)/|a_i|^2
 *                     delta_j += a_ij r_i, s_j += 1 per run
 *   x_j += delta_j / s_j (s_j > 0); optionally x_j = max(x_j, clamp_min)
 * The next block starts from the updated x (Fig. 1). resid (n_sweeps, may be
 * NULL) receives sum_i (b_i - a_i.x)^2 accumulated while sweeping.
 */
int or_drop(const or_grid *g, const double *tab, const or_rec *r, int64_t n, int n_blocks, double lambda,
            int n_sweeps, int mode, int use_clamp, double clamp_min, double *x, double *resid) {
  or_geom o;
  or_geometry(g, &o);
  int64_t M = (int64_t)g->nx * g->ny * g->nz;
  double *delta = (double *)calloc(M, sizeof(double));
  double *cnt = (double *)calloc(M, sizeof(double));
  or_row row = {0};
  if (!delta || !cnt) return -1;
  for (int sw = 0; sw < n_sweeps; ++sw) {
    double rr = 0.0;
    for (int b = 0; b < n_blocks; ++b) {
      int64_t lo = (int64_t)b * n / n_blocks, hi = (int64_t)(b + 1) * n / n_blocks;
      memset(delta, 0, M * sizeof(double));
      memset(cnt, 0, M * sizeof(double));
      for (int64_t i = lo; i < hi; ++i) {
        or_walk_row(g, &o, tab, r, i, mode, &row);
        double ax = 0.0, nn = 0.0;
        for (int64_t q = 0; q < row.n; ++q) {
          ax += row.l[q] * x[row.j[q]];
          nn += row.l[q] * row.l[q];
        }
        if (nn <= 0.0) continue;
        double res = (double)r->wepl[i] - ax;
        rr += res * res;
        double ri = lambda * res / nn;
        for (int64_t q = 0; q < row.n; ++q) {
          delta[row.j[q]] += row.l[q] * ri;
          cnt[row.j[q]] += 1.0;
        }
      }
      for (int64_t j = 0; j < M; ++j) {
        if (cnt[j] > 0.0) x[j] += delta[j] / cnt[j];
        if (use_clamp && x[j] < clamp_min) x[j] = clamp_min;
      }
    }
    if (resid) resid[sw] = rr;
  }
  free(delta);
  free(cnt);
  free(row.j);
  free(row.l);
  return 0;
}

/*
 * The same DROP sweeps with the histories of each block split over `threads`
 * OpenMP threads (0: all available). Each thread accumulates its own update
 * and run counts; they are summed in thread order before the block update,
 * so the result differs from or_drop only in the order of the sums. Used to
 * time the oracle on all host cores.
 */
int or_drop_threads(const or_grid *g, const double *tab, const or_rec *r, int64_t n, int n_blocks, double lambda,
                    int n_sweeps, int mode, int threads, double *x, double *resid) {
#ifndef _OPENMP
  (void)threads;
  return or_drop(g, tab, r, n, n_blocks, lambda, n_sweeps, mode, 0, 0.0, x, resid);
#else
  or_geom o;
  or_geometry(g, &o);
  const int T = threads > 0 ? threads : omp_get_max_threads();
  const int64_t M = (int64_t)g->nx * g->ny * g->nz;
  double *delta = (double *)calloc((size_t)T * M, sizeof(double));
  int32_t *cnt = (int32_t *)calloc((size_t)T * M, sizeof(int32_t));
  if (!delta || !cnt) {
    free(delta);
    free(cnt);
    return -1;
  }
  for (int sw = 0; sw < n_sweeps; ++sw) {
    double rr = 0.0;
    for (int b = 0; b < n_blocks; ++b) {
      const int64_t lo = (int64_t)b * n / n_blocks, hi = (int64_t)(b + 1) * n / n_blocks;
#pragma omp parallel num_threads(T) reduction(+ : rr)
      {
        const int t = omp_get_thread_num();
        double *dt = delta + (size_t)t * M;
        int32_t *ct = cnt + (size_t)t * M;
        memset(dt, 0, M * sizeof(double));
        memset(ct, 0, M * sizeof(int32_t));
        or_row row = {0};
#pragma omp for schedule(static)
        for (int64_t i = lo; i < hi; ++i) {
          or_walk_row(g, &o, tab, r, i, mode, &row);
          double ax = 0.0, nn = 0.0;
          for (int64_t q = 0; q < row.n; ++q) {
            ax += row.l[q] * x[row.j[q]];
            nn += row.l[q] * row.l[q];
          }
          if (nn <= 0.0) continue;
          const double res = (double)r->wepl[i] - ax;
          rr += res * res;
          const double ri = lambda * res / nn;
          for (int64_t q = 0; q < row.n; ++q) {
            dt[row.j[q]] += row.l[q] * ri;
            ct[row.j[q]] += 1;
          }
        }
        free(row.j);
        free(row.l);
      }
#pragma omp parallel for num_threads(T) schedule(static)
      for (int64_t j = 0; j < M; ++j) {
        double d = 0.0;
        int64_t c = 0;
        for (int t = 0; t < T; ++t) {
          d += delta[(size_t)t * M + j];
          c += cnt[(size_t)t * M + j];
        }
        if (c > 0) x[j] += d / (double)c;
      }
    }
    if (resid) resid[sw] = rr;
  }
  free(delta);
  free(cnt);
  return 0;
#endif
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* CARP (Sec. 2.2, Fig. 2)                                             */
/* ------------------------------------------------------------------ */

/*
 * CARP with the strings formed by consecutive DROP blocks: string s holds
 * blocks [s B/S, (s+1) B/S) (block b: histories [b N/B, (b+1) N/B)). Every
 * string starts from the same x0 and sweeps its own rows sequentially, block
 * by block, with the DROP block update (the blocked form of the Kaczmarz
 * sweep of Gordon 2005): x_s = DROP(x0, blocks of s). The new x is the
 * component average over the strings whose rows touch voxel j,
 * x_j = (1/|T_j|) sum_{s in T_j} x_s,j (x_j unchanged if T_j is empty).
 * Repeated n_sweeps times. With one block per string each x_s is a single
 * simultaneous projection from x0.
 */
int or_carp(const or_grid *g, const double *tab, const or_rec *r, int64_t n, int n_blocks, int n_strings,
            double lambda, int n_sweeps, int mode, double *x, double *resid) {
  or_geom o;
  or_geometry(g, &o);
  int64_t M = (int64_t)g->nx * g->ny * g->nz;
  double *xs = (double *)calloc(M, sizeof(double));
  double *delta = (double *)calloc(M, sizeof(double));
  double *cnt = (double *)calloc(M, sizeof(double));
  double *sum = (double *)calloc(M, sizeof(double));
  double *touch = (double *)calloc(M, sizeof(double));
  char *hit = (char *)calloc(M, 1);
  or_row row = {0};
  if (!xs || !delta || !cnt || !sum || !touch || !hit) return -1;
  for (int sw = 0; sw < n_sweeps; ++sw) {
    double rr = 0.0;
    memset(sum, 0, M * sizeof(double));
    memset(touch, 0, M * sizeof(double));
    for (int st = 0; st < n_strings; ++st) {
      memcpy(xs, x, M * sizeof(double));
      memset(hit, 0, M);
      int b0 = (int)((int64_t)st * n_blocks / n_strings), b1 = (int)((int64_t)(st + 1) * n_blocks / n_strings);
      for (int b = b0; b < b1; ++b) {
        int64_t lo = (int64_t)b * n / n_blocks, hi = (int64_t)(b + 1) * n / n_blocks;
        memset(delta, 0, M * sizeof(double));
        memset(cnt, 0, M * sizeof(double));
        for (int64_t i = lo; i < hi; ++i) {
          or_walk_row(g, &o, tab, r, i, mode, &row);
          double ax = 0.0, nn = 0.0;
          for (int64_t q = 0; q < row.n; ++q) {
            ax += row.l[q] * xs[row.j[q]];
            nn += row.l[q] * row.l[q];
          }
          if (nn <= 0.0) continue;
          double res = (double)r->wepl[i] - ax;
          rr += res * res;
          double ri = lambda * res / nn;
          for (int64_t q = 0; q < row.n; ++q) {
            delta[row.j[q]] += row.l[q] * ri;
            cnt[row.j[q]] += 1.0;
          }
        }
        for (int64_t j = 0; j < M; ++j)
          if (cnt[j] > 0.0) {
            xs[j] += delta[j] / cnt[j];
            hit[j] = 1;
          }
      }
      for (int64_t j = 0; j < M; ++j)
        if (hit[j]) {
          sum[j] += xs[j];
          touch[j] += 1.0;
        }
    }
    for (int64_t j = 0; j < M; ++j)
      if (touch[j] > 0.0) x[j] = sum[j] / touch[j];
    if (resid) resid[sw] = rr;
  }
  free(xs);
  free(delta);
  free(cnt);
  free(sum);
  free(touch);
  free(hit);
  free(row.j);
  free(row.l);
  return 0;
}

/* ------------------------------------------------------------------ */
/* TVS: total-variation superiorization (Sec. 4.2)                     */
/* ------------------------------------------------------------------ */

/*
 * Reading (the paper names TVS and where it acts, not its form; this follows
 * Penfold et al. 2010): TV_eps(x) = sum over voxels of
 * sqrt(dx^2 + dy^2 + dz^2 + eps^2), forward differences, a difference across
 * the far boundary taken as 0. One perturbation per application: g = grad
 * TV, v = -g / rms(g) (rms over voxels, so beta is in RSP units), then for up
 * to `tries` trials x' = x + beta_l v with beta_l = beta0 alpha^l and l
 * counting every trial of the run; the first x' with TV(x') <= TV(x) is taken.
 */
typedef struct {
  double beta0, alpha, eps;
  int tries;
  long long ell; /* trials so far (state) */
} or_tvs;

static double or_tv_term(const or_grid *g, const double *x, int64_t i, int64_t j, int64_t k, double eps) {
  int64_t nx = g->nx, ny = g->ny, nz = g->nz;
  int64_t v = i + nx * (j + ny * k);
  double dx = i + 1 < nx ? x[v + 1] - x[v] : 0.0;
  double dy = j + 1 < ny ? x[v + nx] - x[v] : 0.0;
  double dz = k + 1 < nz ? x[v + nx * ny] - x[v] : 0.0;
  return sqrt(dx * dx + dy * dy + dz * dz + eps * eps);
}

double or_tv_value(const or_grid *g, const double *x, double eps) {
  double s = 0.0;
  for (int64_t k = 0; k < g->nz; ++k)
    for (int64_t j = 0; j < g->ny; ++j)
      for (int64_t i = 0; i < g->nx; ++i) s += or_tv_term(g, x, i, j, k, eps);
  return s;
}

/* gradient of TV_eps, written as the sum of the derivatives of every term */
int or_tv_grad(const or_grid *g, const double *x, double eps, double *grad) {
  int64_t nx = g->nx, ny = g->ny, nz = g->nz, M = nx * ny * nz;
  memset(grad, 0, M * sizeof(double));
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t v = i + nx * (j + ny * k);
        double t = or_tv_term(g, x, i, j, k, eps);
        if (i + 1 < nx) {
          double d = x[v + 1] - x[v];
          grad[v + 1] += d / t;
          grad[v] -= d / t;
        }
        if (j + 1 < ny) {
          double d = x[v + nx] - x[v];
          grad[v + nx] += d / t;
          grad[v] -= d / t;
        }
        if (k + 1 < nz) {
          double d = x[v + nx * ny] - x[v];
          grad[v + nx * ny] += d / t;
          grad[v] -= d / t;
        }
      }
  return 0;
}

/* One superiorization perturbation of x in place. Returns 1 if accepted. */
int or_tvs_apply(const or_grid *g, or_tvs *p, double *x) {
  int64_t M = (int64_t)g->nx * g->ny * g->nz;
  double *gr = (double *)malloc(M * sizeof(double));
  double *xp = (double *)malloc(M * sizeof(double));
  int accepted = 0;
  if (!gr || !xp) {
    free(gr);
    free(xp);
    return -1;
  }
  or_tv_grad(g, x, p->eps, gr);
  double n2 = 0.0;
  for (int64_t v = 0; v < M; ++v) n2 += gr[v] * gr[v];
  double rms = sqrt(n2 / M);
  double tv0 = or_tv_value(g, x, p->eps);
  for (int t = 0; t < p->tries && rms > 0.0; ++t) {
    double beta = p->beta0 * pow(p->alpha, (double)p->ell);
    p->ell++;
    for (int64_t v = 0; v < M; ++v) xp[v] = x[v] - beta * gr[v] / rms;
    if (or_tv_value(g, xp, p->eps) <= tv0) {
      memcpy(x, xp, M * sizeof(double));
      accepted = 1;
      break;
    }
  }
  free(gr);
  free(xp);
  return accepted;
}

/*
 * DROP (or_drop) with a TVS perturbation of the image entering every block
 * (Sec. 4.2 applies TVS to the image each DROP block starts from), or
 * CARP with `carp` strings (carp > 0) with one perturbation at the start of
 * every iteration.
 */
int or_solve_tvs(const or_grid *g, const double *tab, const or_rec *r, int64_t n, int n_blocks, double lambda,
                 int n_sweeps, int mode, int carp, double beta0, double alpha, double eps, int tries, double *x) {
  or_tvs p = {beta0, alpha, eps, tries, 0};
  for (int sw = 0; sw < n_sweeps; ++sw) {
    if (carp > 0) {
      if (or_tvs_apply(g, &p, x) < 0) return -1;
      if (or_carp(g, tab, r, n, n_blocks, carp, lambda, 1, mode, x, NULL) != 0) return -1;
    } else {
      for (int b = 0; b < n_blocks; ++b) {
        int64_t lo = (int64_t)b * n / n_blocks, hi = (int64_t)(b + 1) * n / n_blocks;
        or_rec rb = {r->t0 + lo, r->v0 + lo, r->st0 + lo, r->sv0 + lo, r->t2 + lo, r->v2 + lo,
                     r->st2 + lo, r->sv2 + lo, r->wepl + lo, r->cphi + lo, r->sphi + lo};
        if (or_tvs_apply(g, &p, x) < 0) return -1;
        if (or_drop(g, tab, &rb, hi - lo, 1, lambda, 1, mode, 0, 0.0, x, NULL) != 0) return -1;
      }
    }
  }
  return 0;
}
