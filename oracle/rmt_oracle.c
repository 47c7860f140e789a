/*
 * rmt_oracle.c -- plain FP64 CPU oracle of the 3D reference map technique's per-step
 * grid update (arXiv 2104.00095).  TEST INFRASTRUCTURE ONLY: used by tests/, by the
 * smoke check and by the benchmark's CPU-baseline leg; never by the product path.
 *
 * Written for a reader who checks it against the paper by eye: one loop per
 * formula, values fetched through small accessors that apply the boundary rules,
 * no blocking, fusion or reordering.  Linear systems are solved with plain
 * conjugate gradients to a tight tolerance (the discrete solution itself is the
 * reference; how it is reached does not matter).
 *
 * Compile with -ffp-contract=off so that the level-set values that decide the
 * integer masks are rounded exactly as written.
 */
#include "rmt_oracle.h"
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

enum { OK = 0, EINVAL_ = 1, ENOMEM_ = 2, ESTATE_ = 4, ENOCONV_ = 5, EDEGEN_ = 8 };

typedef struct {
  orc_solid_desc d;
  double *xi[3], *phi;  signed char *lay;    /* state at step n            */
  double *xn[3], *phin; signed char *layn;   /* predictor / step n+1       */
  double *xh[3], *phih;                      /* corrector n+1/2 (avail = layn >= 0) */
  double *xf[3][3];  signed char *xfok[3];   /* xi^{n+1/2} at d-faces       */
  double *xb[3][3];  signed char *xbok[3];   /* transverse "bar" xi states at e-faces */
} solid;

struct orc_grid {
  orc_grid_desc d;
  int n[3], per[3], nn[3];
  long N, NN, NF[3];
  double h, dt, t, eps, utol;
  long step;
  int inited;
  double *u[3], *p, *rho;
  /* intermediates kept for inspection */
  double *divtau_n[3], *divtau_h[3], *uf[3][3], *umac[3], *q, *adv[3], *ustar[3], *psi, *rho_h;
  double *ub[3][3], *vadv[3];               /* transverse bar velocity states at e-faces */
  double *rep[3];                           /* wall-repulsion acceleration used in u* */
  int nsol;
  solid* sol;
  int iters[2];
  double true_rel[2], last_true_rel;
  int degenerate;
  char err[256];
};

/* ------------------------------------------------------------------------------- */
/* indexing and boundary rules                                                       */
/* ------------------------------------------------------------------------------- */

static long cidx(const orc_grid* g, int i, int j, int k) { return i + (long)g->n[0] * (j + (long)g->n[1] * k); }
static long nidx(const orc_grid* g, int i, int j, int k) { return i + (long)g->nn[0] * (j + (long)g->nn[1] * k); }
/* face of direction d: the d-th index is the face index f in [0, n_d] (between cells f-1 and f) */
static long fidx(const orc_grid* g, int d, int i, int j, int k) {
  int e0 = g->n[0] + (d == 0), e1 = g->n[1] + (d == 1);
  return i + (long)e0 * (j + (long)e1 * k);
}

/* wrap a cell index on periodic axes; 0 if outside a wall */
static int wrap1(const orc_grid* g, int d, int i, int* o) {
  int n = g->n[d];
  if (g->per[d]) { i %= n; if (i < 0) i += n; *o = i; return 1; }
  if (i < 0 || i >= n) return 0;
  *o = i; return 1;
}
static int cellw(const orc_grid* g, int i, int j, int k, long* c) {
  int a, b, e;
  if (!wrap1(g, 0, i, &a) || !wrap1(g, 1, j, &b) || !wrap1(g, 2, k, &e)) return 0;
  *c = cidx(g, a, b, e);
  return 1;
}
static int nodew(const orc_grid* g, int i, int j, int k, long* c) {
  int ii[3] = {i, j, k};
  for (int d = 0; d < 3; d++) {
    if (g->per[d]) { ii[d] %= g->n[d]; if (ii[d] < 0) ii[d] += g->n[d]; }
    else if (ii[d] < 0 || ii[d] > g->n[d]) return 0;
  }
  *c = nidx(g, ii[0], ii[1], ii[2]);
  return 1;
}

/* Velocity with ghost values.  Reading: a no-slip wall is imposed through mirrored
 * ghosts u_ghost = 2 u_wall - u_mirror (Table pars caption: Dirichlet per face). */
static double uval(const orc_grid* g, int a, int i, int j, int k) {
  int ii[3] = {i, j, k};
  for (int d = 0; d < 3; d++) {
    if (g->per[d]) continue;
    int n = g->n[d];
    if (ii[d] < 0 || ii[d] >= n) {
      int m[3] = {ii[0], ii[1], ii[2]};
      int face = ii[d] < 0 ? 2 * d : 2 * d + 1;
      m[d] = ii[d] < 0 ? -1 - ii[d] : 2 * n - 1 - ii[d];
      return 2.0 * g->d.wall_u[face][a] - uval(g, a, m[0], m[1], m[2]);
    }
  }
  long c;
  cellw(g, i, j, k, &c);
  return g->u[a][c];
}

/* xi component of a solid from array set X with availability array L (>=0 present) */
static int xval(const orc_grid* g, double* const X[3], const signed char* L, int a, int i, int j, int k,
                double* v) {
  long c;
  if (!cellw(g, i, j, k, &c)) return 0;
  if (L[c] < 0) return 0;
  *v = X[a][c];
  return 1;
}

static void cell_center(const orc_grid* g, int i, int j, int k, double x[3]) {
  x[0] = g->d.lo[0] + (i + 0.5) * g->h;
  x[1] = g->d.lo[1] + (j + 0.5) * g->h;
  x[2] = g->d.lo[2] + (k + 0.5) * g->h;
}

/* ------------------------------------------------------------------------------- */
/* pointwise formulas                                                               */
/* ------------------------------------------------------------------------------- */

/* eq. sm_heavi */
double orc_heaviside(double phi, double eps) {
  if (phi <= -eps) return 0.0;
  if (phi >= eps) return 1.0;
  return 0.5 * (1.0 + phi / eps + sin(M_PI * phi / eps) / M_PI);
}
/* derivative of eq. sm_heavi (used by the artificial viscosity, SI "Governing equations") */
double orc_dheaviside(double phi, double eps) {
  if (phi <= -eps || phi >= eps) return 0.0;
  return 0.5 / eps * (1.0 + cos(M_PI * phi / eps));
}

/* Level set of the reference shape, phi_0(X) (main text "Blurred interface method").
 * Sphere: exact signed distance.  Reading for the ellipsoid (no closed-form distance):
 * g(X) = |D^-1 R^T (X-c)|, phi_0 = (g-1)/|grad g|, exact on the surface to first order. */
double orc_phi0(const orc_solid_desc* s, const double X[3]) {
  double r0 = X[0] - s->center[0], r1 = X[1] - s->center[1], r2 = X[2] - s->center[2];
  if (s->shape == ORC_SHAPE_SPHERE) return sqrt(r0 * r0 + r1 * r1 + r2 * r2) - s->semi_axes[0];
  const double* R = s->rot;
  double z0 = R[0] * r0 + R[3] * r1 + R[6] * r2;
  double z1 = R[1] * r0 + R[4] * r1 + R[7] * r2;
  double z2 = R[2] * r0 + R[5] * r1 + R[8] * r2;
  double y0 = z0 / s->semi_axes[0], y1 = z1 / s->semi_axes[1], y2 = z2 / s->semi_axes[2];
  double gg = sqrt(y0 * y0 + y1 * y1 + y2 * y2);
  if (gg < 1e-12) {
    double m = s->semi_axes[0];
    if (s->semi_axes[1] < m) m = s->semi_axes[1];
    if (s->semi_axes[2] < m) m = s->semi_axes[2];
    return -m;
  }
  double w0 = y0 / s->semi_axes[0], w1 = y1 / s->semi_axes[1], w2 = y2 / s->semi_axes[2];
  double wn = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
  return (gg - 1.0) * gg / wn;
}

/* direction of grad_X phi_0 (only the direction is used, by the WLS weights) */
static void phi0_graddir(const orc_solid_desc* s, const double X[3], double gdir[3]) {
  double r[3] = {X[0] - s->center[0], X[1] - s->center[1], X[2] - s->center[2]};
  if (s->shape == ORC_SHAPE_SPHERE) { gdir[0] = r[0]; gdir[1] = r[1]; gdir[2] = r[2]; return; }
  const double* R = s->rot;
  double w[3];
  for (int a = 0; a < 3; a++) {
    double z = R[0 + a] * r[0] + R[3 + a] * r[1] + R[6 + a] * r[2];
    w[a] = z / (s->semi_axes[a] * s->semi_axes[a]);
  }
  for (int a = 0; a < 3; a++) gdir[a] = R[3 * a + 0] * w[0] + R[3 * a + 1] * w[1] + R[3 * a + 2] * w[2];
}

/* Fourth-order monotonicity-limited slope (SI "Normal derivatives", after Colella 1990 /
 * Bell-Colella-Glaz 1989).  q[0..4] = q_{i-2..i+2}; ok[] marks present values.
 * Reading: with q_{i+-2} missing the second-order limited slope is used, with q_{i+-1}
 * missing the slope is zero (only happens for xi at the edge of the band). */
static double mc_lim(double qm, double q0, double qp) {
  double a = qp - q0, b = q0 - qm;
  if (a * b > 0.0) return 2.0 * fmin(fabs(a), fabs(b));
  return 0.0;
}
static double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }
static double dfl(double qm, double q0, double qp) {
  double dc = 0.5 * (qp - qm);
  return sgn(dc) * fmin(fabs(dc), mc_lim(qm, q0, qp));
}
double orc_limited_slope(const double q[5], const int ok[5], double h) {
  if (!ok[1] || !ok[2] || !ok[3]) return 0.0;
  double dc = 0.5 * (q[3] - q[1]);
  double dl = mc_lim(q[1], q[2], q[3]);
  if (!ok[0] || !ok[4]) return sgn(dc) * fmin(fabs(dc), dl) / h;
  double dfp = dfl(q[2], q[3], q[4]);
  double dfm = dfl(q[0], q[1], q[2]);
  double d4 = (4.0 / 3.0) * dc - (dfp + dfm) / 6.0;
  return sgn(dc) * fmin(fabs(d4), dl) / h;
}

/* SI "Godunov-type upwinding scheme": normal-velocity choice and upwinding of the rest.
 * Reading: the sign tests use a tolerance tol (the "= 0" cases hold for |v| <= tol), so that a
 * velocity that vanishes in exact arithmetic (a symmetry plane) does not pick its side from
 * rounding noise; the step uses tol = 1e-12 h/dt, the pins tol = 0. */
double orc_godunov_normal(double L, double R, double tol) {
  if (L > tol && L + R > tol) return L;
  if (R < -tol && L + R < -tol) return R;
  return 0.0;
}
double orc_upwind(double L, double R, double un, double tol) {
  if (un > tol) return L;
  if (un < -tol) return R;
  return 0.5 * (L + R);
}

/* Neo-Hookean deviatoric stress, SI "Stress calculations": F = (grad xi)^-1,
 * B = F F^T, tau = G (B - tr(B)/3 I).  Returns 0 if grad xi is singular. */
int orc_neohookean(const double A[9], double G, double tau[9]) {
  double F[9];
  double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (det == 0.0 || !isfinite(det)) return 0;
  F[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  F[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  F[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  F[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  F[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  F[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  F[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  F[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  F[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  double B[9];
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) B[3 * r + c] = F[3 * r] * F[3 * c] + F[3 * r + 1] * F[3 * c + 1] + F[3 * r + 2] * F[3 * c + 2];
  double tr3 = (B[0] + B[4] + B[8]) / 3.0;
  for (int r = 0; r < 9; r++) tau[r] = G * B[r];
  tau[0] -= G * tr3; tau[4] -= G * tr3; tau[8] -= G * tr3;
  return 1;
}

/* Multi-body mixing (SI eq. mod_heaviside and the tau_s combination rule above it).
 * Hm[m] = H_eps(phi_m).  w_out[m] = (1-H_m), divided by their sum when the sum exceeds 1.
 * Returns the blended fluid fraction H = max(1 - sum(1-H_m), 0). */
double orc_mix_weights(int S, const double* Hm, double* w_out) {
  double sum = 0.0;
  for (int m = 0; m < S; m++) { w_out[m] = 1.0 - Hm[m]; sum += w_out[m]; }
  if (sum > 1.0)
    for (int m = 0; m < S; m++) w_out[m] = w_out[m] / sum;
  double H = 1.0 - sum;
  return H > 0.0 ? H : 0.0;
}

/* ------------------------------------------------------------------------------- */
/* allocation                                                                        */
/* ------------------------------------------------------------------------------- */

static double* dalloc(long n) { return (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }
static signed char* calloc8(long n) { return (signed char*)calloc((size_t)(n > 0 ? n : 1), 1); }

int orc_create(const orc_grid_desc* d, orc_grid** out) {
  if (!d || !out) return EINVAL_;
  orc_grid* g = (orc_grid*)calloc(1, sizeof(orc_grid));
  if (!g) return ENOMEM_;
  g->d = *d;
  for (int a = 0; a < 3; a++) {
    if (d->n[a] < 4) { free(g); return EINVAL_; }
    g->n[a] = d->n[a];
    int p0 = d->bc[2 * a] == ORC_BC_PERIODIC, p1 = d->bc[2 * a + 1] == ORC_BC_PERIODIC;
    if (p0 != p1) { free(g); return EINVAL_; }
    g->per[a] = p0;
    g->nn[a] = g->per[a] ? g->n[a] : g->n[a] + 1;
  }
  g->h = (d->hi[0] - d->lo[0]) / d->n[0];
  for (int a = 1; a < 3; a++) {
    double ha = (d->hi[a] - d->lo[a]) / d->n[a];
    if (fabs(ha - g->h) > 1e-12 * g->h) { free(g); return EINVAL_; }
  }
  g->eps = d->eps_h * g->h;
  g->N = (long)g->n[0] * g->n[1] * g->n[2];
  g->NN = (long)g->nn[0] * g->nn[1] * g->nn[2];
  for (int a = 0; a < 3; a++) g->NF[a] = g->N / g->n[a] * (g->n[a] + 1);
  for (int a = 0; a < 3; a++) {
    g->u[a] = dalloc(g->N); g->divtau_n[a] = dalloc(g->N); g->divtau_h[a] = dalloc(g->N);
    g->adv[a] = dalloc(g->N); g->ustar[a] = dalloc(g->N); g->rep[a] = dalloc(g->N);
    g->umac[a] = dalloc(g->NF[a]); g->vadv[a] = dalloc(g->NF[a]);
    for (int b = 0; b < 3; b++) { g->uf[a][b] = dalloc(g->NF[a]); g->ub[a][b] = dalloc(g->NF[a]); }
  }
  g->p = dalloc(g->NN); g->psi = dalloc(g->NN);
  g->rho = dalloc(g->N); g->rho_h = dalloc(g->N); g->q = dalloc(g->N);
  for (long c = 0; c < g->N; c++) { g->rho[c] = d->rho_f; g->rho_h[c] = d->rho_f; }
  *out = g;
  return OK;
}

int orc_add_solid(orc_grid* g, const orc_solid_desc* s, int* id) {
  if (!g || !s || g->inited) return ESTATE_;
  solid* ns = (solid*)realloc(g->sol, sizeof(solid) * (g->nsol + 1));
  if (!ns) return ENOMEM_;
  g->sol = ns;
  solid* S = &g->sol[g->nsol];
  memset(S, 0, sizeof(*S));
  S->d = *s;
  for (int a = 0; a < 3; a++) {
    S->xi[a] = dalloc(g->N); S->xn[a] = dalloc(g->N); S->xh[a] = dalloc(g->N);
    for (int b = 0; b < 3; b++) { S->xf[a][b] = dalloc(g->NF[a]); S->xb[a][b] = dalloc(g->NF[a]); }
    S->xfok[a] = calloc8(g->NF[a]); S->xbok[a] = calloc8(g->NF[a]);
  }
  S->phi = dalloc(g->N); S->phin = dalloc(g->N); S->phih = dalloc(g->N);
  S->lay = calloc8(g->N); S->layn = calloc8(g->N);
  memset(S->lay, -1, (size_t)g->N); memset(S->layn, -1, (size_t)g->N);
  if (id) *id = g->nsol;
  g->nsol++;
  return OK;
}

void orc_destroy(orc_grid* g) {
  if (!g) return;
  for (int m = 0; m < g->nsol; m++) {
    solid* S = &g->sol[m];
    for (int a = 0; a < 3; a++) {
      free(S->xi[a]); free(S->xn[a]); free(S->xh[a]); free(S->xfok[a]); free(S->xbok[a]);
      for (int b = 0; b < 3; b++) { free(S->xf[a][b]); free(S->xb[a][b]); }
    }
    free(S->phi); free(S->phin); free(S->phih); free(S->lay); free(S->layn);
  }
  free(g->sol);
  for (int a = 0; a < 3; a++) {
    free(g->u[a]); free(g->divtau_n[a]); free(g->divtau_h[a]); free(g->adv[a]); free(g->ustar[a]); free(g->rep[a]);
    free(g->umac[a]); free(g->vadv[a]);
    for (int b = 0; b < 3; b++) { free(g->uf[a][b]); free(g->ub[a][b]); }
  }
  free(g->p); free(g->psi); free(g->rho); free(g->rho_h); free(g->q);
  free(g);
}

const char* orc_error(orc_grid* g) { return g ? g->err : "null grid"; }
double orc_dt(orc_grid* g) { return g->dt; }
int orc_last_iters(orc_grid* g, int which) { return g->iters[which ? 1 : 0]; }
double orc_last_true_residual(orc_grid* g, int which) { return g->true_rel[which ? 1 : 0]; }

/* ------------------------------------------------------------------------------- */
/* extrapolation of xi: layers + weighted least squares (main text "Extrapolation of  */
/* xi(x,t)", SI "Weighting scheme for weighted least squares-based extrapolation")   */
/* ------------------------------------------------------------------------------- */

/* LDL^T solve of the 4x4 normal equations with three right-hand sides.
 * Reading (the paper gives no criterion): degenerate when fewer than 4 data points carry
 * weight, or when a pivot falls to 1e-12 * trace(A)/4 or below. */
static int solve4(double A[4][4], double B[4][3], double X[4][3]) {
  double L[4][4] = {{0}}, D[4];
  double tr = A[0][0] + A[1][1] + A[2][2] + A[3][3];
  double tol = 1e-12 * tr / 4.0;
  for (int k = 0; k < 4; k++) {
    double s = A[k][k];
    for (int j = 0; j < k; j++) s -= L[k][j] * L[k][j] * D[j];
    D[k] = s;
    if (!(s > tol)) return 0;
    L[k][k] = 1.0;
    for (int i = k + 1; i < 4; i++) {
      double t = A[i][k];
      for (int j = 0; j < k; j++) t -= L[i][j] * L[k][j] * D[j];
      L[i][k] = t / D[k];
    }
  }
  for (int c = 0; c < 3; c++) {
    double y[4];
    for (int i = 0; i < 4; i++) {
      double t = B[i][c];
      for (int j = 0; j < i; j++) t -= L[i][j] * y[j];
      y[i] = t;
    }
    for (int i = 0; i < 4; i++) y[i] /= D[i];
    for (int i = 3; i >= 0; i--) {
      double t = y[i];
      for (int j = i + 1; j < 4; j++) t -= L[j][i] * X[j][c];
      X[i][c] = t;
    }
  }
  return 1;
}

/* One WLS fit at cell (i,j,k) of layer le with search radius rs.  mode 0: exponential
 * kernel only; mode 1: kernel times max(0, cos) against the normal nrm (eq. weight).
 * Reading: the model is affine, centred at x_e (xi = c + G (x - x_e)), so xi_e = c. */
static int wls_fit(const orc_grid* g, double* const X[3], const signed char* L, int i, int j, int k, int le,
                   int rs, int mode, const double nrm[3], double sol[4][3]) {
  double A[4][4] = {{0}}, B[4][3] = {{0}};
  int npos = 0;
  for (int dk = -rs; dk <= rs; dk++)
    for (int dj = -rs; dj <= rs; dj++)
      for (int di = -rs; di <= rs; di++) {
        long c;
        if (!cellw(g, i + di, j + dj, k + dk, &c)) continue;
        int ld = L[c];
        if (ld < 0 || ld >= le) continue;
        int s = abs(di) + abs(dj) + abs(dk);
        double w = ldexp(1.0, -s);
        if (mode == 1) {
          /* x' = x_e - x_d = -(di,dj,dk) h */
          double len = sqrt((double)(di * di + dj * dj + dk * dk));
          double cs = -((double)di * nrm[0] + (double)dj * nrm[1] + (double)dk * nrm[2]) / len;
          w = cs * w;
          if (!(w > 0.0)) continue;
        }
        double v[4] = {1.0, (double)di, (double)dj, (double)dk};
        for (int r = 0; r < 4; r++) {
          for (int q = 0; q < 4; q++) A[r][q] += w * v[r] * v[q];
          for (int a = 0; a < 3; a++) B[r][a] += w * v[r] * X[a][c];
        }
        npos++;
      }
  if (npos < 4) return 0;
  return solve4(A, B, sol);
}

/* Extrapolates one cell; returns 1 on success with xi_e in out[3]. */
static int wls_cell(const orc_grid* g, const solid* S, double* const X[3], const signed char* L, int i, int j,
                    int k, int le, double out[3]) {
  for (int rs = 2; rs <= 4; rs++) {
    double s1[4][3];
    if (!wls_fit(g, X, L, i, j, k, le, rs, 0, NULL, s1)) continue;
    if (le <= 2) {
      /* Reading: n_e = normalised grad_x phi_0(xi) from the kernel-only fit:
       * grad_x phi = (grad_x xi)^T grad_X phi_0(xi_e). */
      double c0[3] = {s1[0][0], s1[0][1], s1[0][2]}, gX[3], v[3];
      phi0_graddir(&S->d, c0, gX);
      for (int b = 0; b < 3; b++) v[b] = s1[1 + b][0] * gX[0] + s1[1 + b][1] * gX[1] + s1[1 + b][2] * gX[2];
      double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      if (!(nv > 0.0)) continue;
      double nrm[3] = {v[0] / nv, v[1] / nv, v[2] / nv};
      double s2[4][3];
      if (!wls_fit(g, X, L, i, j, k, le, rs, 1, nrm, s2)) continue;
      out[0] = s2[0][0]; out[1] = s2[0][1]; out[2] = s2[0][2];
      return 1;
    }
    out[0] = s1[0][0]; out[1] = s1[0][1]; out[2] = s1[0][2];
    return 1;
  }
  return 0;
}

/* Classify, mark layers and extrapolate one solid.  cand[c] != 0 marks cells whose xi
 * in X is a candidate primary value; layer 0 = candidates with phi_0(xi) < 0. */
static void extrapolate(orc_grid* g, solid* S, double* X[3], double* PH, signed char* L, const signed char* cand) {
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
#pragma omp parallel for schedule(static)
  for (long c = 0; c < g->N; c++) {
    L[c] = -1;
    if (cand[c]) {
      double xv[3] = {X[0][c], X[1][c], X[2][c]};
      if (orc_phi0(&S->d, xv) < 0.0) L[c] = 0;
    }
  }
  /* layers: unmarked face neighbours of layer l-1; walls stop the march, periodic axes wrap
   * (in place and race-free: a pass writes only l over -1 and tests only l-1) */
  for (int l = 1; l <= g->d.band_layers; l++)
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          long c = cidx(g, i, j, k);
          if (L[c] != -1) continue;
          static const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
          for (int f = 0; f < 6; f++) {
            long nb;
            if (!cellw(g, i + off[f][0], j + off[f][1], k + off[f][2], &nb)) continue;
            if (L[nb] == l - 1) { L[c] = (signed char)l; break; }
          }
        }
  /* WLS, layer by layer in ascending order (the fits of one layer read only lower layers) */
  for (int l = 1; l <= g->d.band_layers; l++) {
    int bad = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(+ : bad)
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          long c = cidx(g, i, j, k);
          if (L[c] != l) continue;
          double out[3];
          if (wls_cell(g, S, X, L, i, j, k, l, out)) {
            X[0][c] = out[0]; X[1][c] = out[1]; X[2][c] = out[2];
          } else {
            L[c] = -1;
            bad++;
          }
        }
    g->degenerate += bad;
  }
#pragma omp parallel for schedule(static)
  for (long c = 0; c < g->N; c++) {
    if (L[c] >= 0) {
      double xv[3] = {X[0][c], X[1][c], X[2][c]};
      PH[c] = orc_phi0(&S->d, xv);
    } else {
      X[0][c] = X[1][c] = X[2][c] = NAN;
      PH[c] = NAN;
    }
  }
}

/* ------------------------------------------------------------------------------- */
/* density and stress                                                               */
/* ------------------------------------------------------------------------------- */

/* rho by mixing (SI Initialization item 6, Timestepping 9 and 13; eq. mod_heaviside).
 * Reading: rho = H rho_f + sum_m w_m rho_m with the normalised weights of the stress rule. */
static void mix_density(orc_grid* g, int which, double* out) {
  int S = g->nsol;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < g->N; c++) {
    double Hm[64], w[64];
    int ids[64];
    int cnt = 0;
    for (int m = 0; m < S; m++) {
      const solid* s = &g->sol[m];
      const signed char* L = which == 0 ? s->lay : s->layn;
      const double* PH = which == 0 ? s->phi : (which == 1 ? s->phih : s->phin);
      if (L[c] < 0) continue;
      Hm[cnt] = orc_heaviside(PH[c], g->eps);
      ids[cnt++] = m;
    }
    double H = orc_mix_weights(cnt, Hm, w);
    double r = H * g->d.rho_f;
    for (int q = 0; q < cnt; q++) r += w[q] * g->sol[ids[q]].d.rho_s;
    out[c] = r;
  }
}

/* Face-normal row of the blended deviatoric stress at the d-face between cells a=(i,j,k)-e_d
 * and b=(i,j,k) (SI "Stress calculations", eq. mixed_stresses, multi-body rule).
 * which = 0: xi^n, which = 1: xi^{n+1/2}.  tau_f and tau_a use mu grad u^n only
 * (the grad u^T term is dropped, SI "Governing equations").  Reading: grad xi at the face
 * by centred differences (normal: two cells; transverse: four-cell average); phi at the
 * face = phi_0 of the face-averaged xi; an object lacking xi anywhere in the 10-cell
 * stencil counts as fluid at that face. */
static void face_traction(orc_grid* g, int d, int i, int j, int k, int which, double tt, double row[3]) {
  const double h = g->h;
  int ia[3] = {i, j, k};
  ia[d] -= 1; /* cell a */
  int ib[3] = {i, j, k};
  double du[3];
  for (int a = 0; a < 3; a++) du[a] = (uval(g, a, ib[0], ib[1], ib[2]) - uval(g, a, ia[0], ia[1], ia[2])) / h;
  double Hm[64], wgt[64], rows[64][3];
  int cnt = 0;
  for (int m = 0; m < g->nsol; m++) {
    solid* S = &g->sol[m];
    double* const* X = which == 0 ? S->xi : S->xh;
    const signed char* L = which == 0 ? S->lay : S->layn;
    double xa[3], xb[3], A[9];
    int ok = 1;
    for (int a = 0; a < 3 && ok; a++) {
      ok &= xval(g, X, L, a, ia[0], ia[1], ia[2], &xa[a]);
      ok &= xval(g, X, L, a, ib[0], ib[1], ib[2], &xb[a]);
    }
    if (!ok) continue;
    for (int a = 0; a < 3; a++) A[3 * a + d] = (xb[a] - xa[a]) / h;
    for (int e = 0; e < 3 && ok; e++) {
      if (e == d) continue;
      int ap[3] = {ia[0], ia[1], ia[2]}, am[3] = {ia[0], ia[1], ia[2]};
      int bp[3] = {ib[0], ib[1], ib[2]}, bm[3] = {ib[0], ib[1], ib[2]};
      ap[e]++; am[e]--; bp[e]++; bm[e]--;
      for (int a = 0; a < 3 && ok; a++) {
        double v1 = 0, v2 = 0, v3 = 0, v4 = 0;
        ok &= xval(g, X, L, a, ap[0], ap[1], ap[2], &v1);
        ok &= xval(g, X, L, a, bp[0], bp[1], bp[2], &v2);
        ok &= xval(g, X, L, a, am[0], am[1], am[2], &v3);
        ok &= xval(g, X, L, a, bm[0], bm[1], bm[2], &v4);
        if (ok) A[3 * a + e] = (v1 + v2 - v3 - v4) / (4.0 * h);
      }
    }
    if (!ok) continue;
    double xfc[3] = {0.5 * (xa[0] + xb[0]), 0.5 * (xa[1] + xb[1]), 0.5 * (xa[2] + xb[2])};
    double ph = orc_phi0(&S->d, xfc);
    double Hv = orc_heaviside(ph, g->eps);
    double tau[9];
    if (!orc_neohookean(A, S->d.G, tau)) continue;
    if (S->d.active_A != 0.0) {
      /* Active stress (main text "Swimming"): sigma_a = (3 Z sigma_0 / 2)(e e^T - I/3),
       * e = F E_X / |F E_X|.  Reading: sigma_0 = A sin(2 pi X / l - omega t), X, Z the
       * body-frame coordinates of xi; added to the solid stress before blending. */
      const double* R = S->d.rot;
      double r[3] = {xfc[0] - S->d.center[0], xfc[1] - S->d.center[1], xfc[2] - S->d.center[2]};
      double Xb = R[0] * r[0] + R[3] * r[1] + R[6] * r[2];
      double Zb = R[2] * r[0] + R[5] * r[1] + R[8] * r[2];
      double s0 = S->d.active_A * sin(2.0 * M_PI * Xb / S->d.active_len - S->d.active_omega * tt);
      /* F = A^-1 applied to E_X: solve A f = E_X via the adjugate */
      double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                   A[2] * (A[3] * A[7] - A[4] * A[6]);
      double F[9];
      F[0] = (A[4] * A[8] - A[5] * A[7]) / det;
      F[1] = (A[2] * A[7] - A[1] * A[8]) / det;
      F[2] = (A[1] * A[5] - A[2] * A[4]) / det;
      F[3] = (A[5] * A[6] - A[3] * A[8]) / det;
      F[4] = (A[0] * A[8] - A[2] * A[6]) / det;
      F[5] = (A[2] * A[3] - A[0] * A[5]) / det;
      F[6] = (A[3] * A[7] - A[4] * A[6]) / det;
      F[7] = (A[1] * A[6] - A[0] * A[7]) / det;
      F[8] = (A[0] * A[4] - A[1] * A[3]) / det;
      double EX[3] = {R[0], R[3], R[6]};
      double f[3];
      for (int a = 0; a < 3; a++) f[a] = F[3 * a] * EX[0] + F[3 * a + 1] * EX[1] + F[3 * a + 2] * EX[2];
      double fn = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
      double e[3] = {f[0] / fn, f[1] / fn, f[2] / fn};
      double amp = 1.5 * Zb * s0;
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) tau[3 * a + b] += amp * (e[a] * e[b] - (a == b ? 1.0 / 3.0 : 0.0));
    }
    double visc = S->d.mu_a * (1.0 + S->d.gamma_t * g->eps * orc_dheaviside(ph, g->eps));
    for (int a = 0; a < 3; a++) rows[cnt][a] = tau[3 * a + d] + visc * du[a];
    Hm[cnt] = Hv;
    cnt++;
  }
  double H = orc_mix_weights(cnt, Hm, wgt);
  for (int a = 0; a < 3; a++) {
    double v = H * g->d.mu * du[a];
    for (int q = 0; q < cnt; q++) v += wgt[q] * rows[q][a];
    row[a] = v;
  }
}

/* grad . tau at every cell: sum over directions of (row(+face) - row(-face)) / h */
static void stress_divergence(orc_grid* g, int which, double tt, double* out[3]) {
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        double acc[3] = {0, 0, 0};
        for (int d = 0; d < 3; d++) {
          int ip[3] = {i, j, k};
          ip[d] += 1;
          double rp[3], rm[3];
          face_traction(g, d, ip[0], ip[1], ip[2], which, tt, rp);
          face_traction(g, d, i, j, k, which, tt, rm);
          for (int a = 0; a < 3; a++) acc[a] += (rp[a] - rm[a]) / g->h;
        }
        long c = cidx(g, i, j, k);
        for (int a = 0; a < 3; a++) out[a][c] = acc[a];
      }
}

/* cell-centre gradient of the trilinear interpolant of a nodal field (used for grad p and
 * for the projection correction, SI "Approximate pressure-Poisson projection") */
static void grad_at_cell(const orc_grid* g, const double* P, int i, int j, int k, double gr[3]) {
  gr[0] = gr[1] = gr[2] = 0.0;
  for (int c = 0; c < 2; c++)
    for (int b = 0; b < 2; b++)
      for (int a = 0; a < 2; a++) {
        long nd;
        nodew(g, i + a, j + b, k + c, &nd);
        double v = P[nd];
        gr[0] += (a ? v : -v);
        gr[1] += (b ? v : -v);
        gr[2] += (c ? v : -v);
      }
  for (int d = 0; d < 3; d++) gr[d] /= 4.0 * g->h;
}

void orc_cell_grad(orc_grid* g, const double* nodal, double* out) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->n[2]; k++)
    for (int j = 0; j < g->n[1]; j++)
      for (int i = 0; i < g->n[0]; i++) {
        double gr[3];
        grad_at_cell(g, nodal, i, j, k, gr);
        long c = cidx(g, i, j, k);
        for (int d = 0; d < 3; d++) out[d * g->N + c] = gr[d];
      }
}

/* ------------------------------------------------------------------------------- */
/* Godunov predictor (SI "Evaluating the advective term")                           */
/* ------------------------------------------------------------------------------- */

static int is_wall_face(const orc_grid* g, int d, int f) { return !g->per[d] && (f == 0 || f == g->n[d]); }

static double slope_u(const orc_grid* g, int a, int d, int i, int j, int k) {
  double q[5];
  int ok[5] = {1, 1, 1, 1, 1};
  for (int s = -2; s <= 2; s++) {
    int ii[3] = {i, j, k};
    ii[d] += s;
    q[s + 2] = uval(g, a, ii[0], ii[1], ii[2]);
  }
  return orc_limited_slope(q, ok, g->h);
}
static double slope_x(const orc_grid* g, double* const X[3], const signed char* L, int a, int d, int i, int j,
                      int k) {
  double q[5];
  int ok[5];
  for (int s = -2; s <= 2; s++) {
    int ii[3] = {i, j, k};
    ii[d] += s;
    ok[s + 2] = xval(g, X, L, a, ii[0], ii[1], ii[2], &q[s + 2]);
    if (!ok[s + 2]) q[s + 2] = 0.0;
  }
  return orc_limited_slope(q, ok, g->h);
}

/* transverse ("bar") states at every e-face: velocity (all components, advecting velocity
 * chosen by the Godunov rule) and xi of every solid */
static void bar_states(orc_grid* g) {
  const double h = g->h, dt = g->dt;
  for (int e = 0; e < 3; e++) {
    int ext[3] = {g->n[0], g->n[1], g->n[2]};
    ext[e] += 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < ext[2]; k++)
      for (int j = 0; j < ext[1]; j++)
        for (int i = 0; i < ext[0]; i++) {
          long f = fidx(g, e, i, j, k);
          int fi = e == 0 ? i : (e == 1 ? j : k);
          int lo[3] = {i, j, k};
          lo[e] -= 1; /* cell below (D), (i,j,k) is the cell above (U) */
          if (is_wall_face(g, e, fi)) {
            int face = fi == 0 ? 2 * e : 2 * e + 1;
            for (int a = 0; a < 3; a++) g->ub[e][a][f] = g->d.wall_u[face][a];
            g->vadv[e][f] = g->d.wall_u[face][e];
            for (int m = 0; m < g->nsol; m++) g->sol[m].xbok[e][f] = 0;
            continue;
          }
          double uD = uval(g, e, lo[0], lo[1], lo[2]), uU = uval(g, e, i, j, k);
          double qD[3], qU[3];
          for (int a = 0; a < 3; a++) {
            qD[a] = uval(g, a, lo[0], lo[1], lo[2]) + (0.5 * h - 0.5 * dt * uD) * slope_u(g, a, e, lo[0], lo[1], lo[2]);
            qU[a] = uval(g, a, i, j, k) - (0.5 * h + 0.5 * dt * uU) * slope_u(g, a, e, i, j, k);
          }
          double va = orc_godunov_normal(qD[e], qU[e], g->utol);
          g->vadv[e][f] = va;
          for (int a = 0; a < 3; a++) g->ub[e][a][f] = orc_upwind(qD[a], qU[a], va, g->utol);
          for (int m = 0; m < g->nsol; m++) {
            solid* S = &g->sol[m];
            double xD[3], xU[3];
            int ok = 1;
            for (int a = 0; a < 3; a++) {
              ok &= xval(g, S->xi, S->lay, a, lo[0], lo[1], lo[2], &xD[a]);
              ok &= xval(g, S->xi, S->lay, a, i, j, k, &xU[a]);
            }
            S->xbok[e][f] = (signed char)ok;
            if (!ok) continue;
            for (int a = 0; a < 3; a++) {
              double sD = slope_x(g, S->xi, S->lay, a, e, lo[0], lo[1], lo[2]);
              double sU = slope_x(g, S->xi, S->lay, a, e, i, j, k);
              double bD = xD[a] + (0.5 * h - 0.5 * dt * uD) * sD;
              double bU = xU[a] - (0.5 * h + 0.5 * dt * uU) * sU;
              S->xb[e][a][f] = orc_upwind(bD, bU, va, g->utol);
            }
          }
        }
  }
}

/* face indices of cell (i,j,k) along e: low face = cell index, high face = +1 */
static void efaces(const orc_grid* g, int e, int i, int j, int k, long* flo, long* fhi) {
  int ii[3] = {i, j, k};
  *flo = fidx(g, e, ii[0], ii[1], ii[2]);
  ii[e] += 1;
  *fhi = fidx(g, e, ii[0], ii[1], ii[2]);
}

/* tangential term sum_{e != d} avg(v_adv) * (qbar(+) - qbar(-)) / h at cell (i,j,k) for the
 * velocity component a (SI "Tangential derivatives") */
static double trans_u(const orc_grid* g, int d, int a, int i, int j, int k) {
  double t = 0.0;
  for (int e = 0; e < 3; e++) {
    if (e == d) continue;
    long fl, fh;
    efaces(g, e, i, j, k, &fl, &fh);
    t += 0.5 * (g->vadv[e][fl] + g->vadv[e][fh]) * (g->ub[e][a][fh] - g->ub[e][a][fl]) / g->h;
  }
  return t;
}
/* same for xi; Reading: a transverse term whose bar state is missing (band edge) is zero */
static double trans_x(const orc_grid* g, const solid* S, int d, int a, int i, int j, int k) {
  double t = 0.0;
  for (int e = 0; e < 3; e++) {
    if (e == d) continue;
    long fl, fh;
    efaces(g, e, i, j, k, &fl, &fh);
    if (!S->xbok[e][fl] || !S->xbok[e][fh]) continue;
    t += 0.5 * (g->vadv[e][fl] + g->vadv[e][fh]) * (S->xb[e][a][fh] - S->xb[e][a][fl]) / g->h;
  }
  return t;
}

/* normal-face states u^{n+1/2} (all components) and xi^{n+1/2} at every d-face
 * (eqs. taylor_left, time_partial, left_final, right_final, xi_taylor_final) */
/* ------------------------------------------------------------------------------- */
/* wall repulsion (SI "Contact with a wall")                                         */
/* ------------------------------------------------------------------------------- */

double orc_rep_accel(double V, double U, double dw, double Lmin, double rho_s, double rho_f, double gmag,
                     double Usafe) {
  const double vrep = dw * Lmin * Lmin;           /* conservative contact volume */
  const double a_safe = Usafe * Usafe / dw;
  const double a_stop = V * U * U / (2.0 * dw * vrep);
  const double a_hold = fabs(rho_s - rho_f) * V * gmag / (rho_s * vrep);
  double a = a_safe;
  if (a_stop > a) a = a_stop;
  if (a_hold > a) a = a_hold;
  return a;
}

/* Acceleration a_rep at every cell from the bodies' level sets (which = 0: phi^n with the
 * layers of step n; which = 1: phi^{n+1/2} with the layers of step n+1).  For a no-slip wall
 * alpha with inward normal n_alpha, the cells whose centre is nearer than d_w to it get, from
 * every body present there, A_rep n_alpha times the transition factor of eq. wall_acc in the
 * body's phi with width Delta h_alpha = h; walls add up, and (Reading) so do bodies. */
static void rep_accel(orc_grid* g, int which, double* out[3]) {
  const double h = g->h, dw = g->d.wall_dw > 0.0 ? g->d.wall_dw : h;
  for (int a = 0; a < 3; a++) memset(out[a], 0, sizeof(double) * g->N);
  int any = 0;
  for (int m = 0; m < g->nsol; m++) any |= g->sol[m].d.rep_A != 0.0;
  if (!any) return;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->n[2]; k++)
    for (int j = 0; j < g->n[1]; j++)
      for (int i = 0; i < g->n[0]; i++) {
        const int ii[3] = {i, j, k};
        double nsum[3] = {0.0, 0.0, 0.0};
        int near = 0;
        for (int d = 0; d < 3; d++) {
          if (g->per[d]) continue;
          const double dlo = (ii[d] + 0.5) * h, dhi = (g->n[d] - ii[d] - 0.5) * h;
          if (dlo < dw) { nsum[d] += 1.0; near = 1; }  /* wall at lo: inward normal +e_d */
          if (dhi < dw) { nsum[d] -= 1.0; near = 1; }  /* wall at hi: inward normal -e_d */
        }
        if (!near) continue;
        const long c = cidx(g, i, j, k);
        for (int m = 0; m < g->nsol; m++) {
          const solid* S = &g->sol[m];
          if (S->d.rep_A == 0.0) continue;
          const signed char* L = which == 0 ? S->lay : S->layn;
          if (L[c] < 0) continue;
          const double ph = which == 0 ? S->phi[c] : S->phih[c];
          double f;
          if (ph <= -h) f = 1.0;
          else if (ph < h) f = 0.5 - ph / (2.0 * h);
          else f = 0.0;
          for (int a = 0; a < 3; a++) out[a][c] += f * S->d.rep_A * nsum[a];
        }
      }
}

static void face_states(orc_grid* g) {
  const double h = g->h, dt = g->dt;
  const long N = g->N;
  /* forcing F = -grad p^{n-1/2} + div tau^n + b^n at cells; Reading: b = (rho - rho_f) g
   * plus rho a_rep (wall repulsion, from phi^n) */
  double* F[3];
  double* A[3];
  for (int a = 0; a < 3; a++) { F[a] = dalloc(N); A[a] = dalloc(N); }
  rep_accel(g, 0, A);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->n[2]; k++)
    for (int j = 0; j < g->n[1]; j++)
      for (int i = 0; i < g->n[0]; i++) {
        long c = cidx(g, i, j, k);
        double gp[3];
        grad_at_cell(g, g->p, i, j, k, gp);
        for (int a = 0; a < 3; a++)
          F[a][c] = -gp[a] + g->divtau_n[a][c] + (g->rho[c] - g->d.rho_f) * g->d.gravity[a] + g->rho[c] * A[a][c];
      }
  for (int a = 0; a < 3; a++) free(A[a]);
  for (int d = 0; d < 3; d++) {
    int ext[3] = {g->n[0], g->n[1], g->n[2]};
    ext[d] += 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < ext[2]; k++)
      for (int j = 0; j < ext[1]; j++)
        for (int i = 0; i < ext[0]; i++) {
          long f = fidx(g, d, i, j, k);
          int fi = d == 0 ? i : (d == 1 ? j : k);
          int ia[3] = {i, j, k};
          ia[d] -= 1;
          if (is_wall_face(g, d, fi)) {
            int face = fi == 0 ? 2 * d : 2 * d + 1;
            for (int a = 0; a < 3; a++) g->uf[d][a][f] = g->d.wall_u[face][a];
          }
          long ca = -1, cb = -1;
          int has_a = cellw(g, ia[0], ia[1], ia[2], &ca);
          int has_b = cellw(g, i, j, k, &cb);
          int wa[3] = {0, 0, 0}, wb[3] = {0, 0, 0};
          if (has_a) { wrap1(g, 0, ia[0], &wa[0]); wrap1(g, 1, ia[1], &wa[1]); wrap1(g, 2, ia[2], &wa[2]); }
          if (has_b) { wrap1(g, 0, i, &wb[0]); wrap1(g, 1, j, &wb[1]); wrap1(g, 2, k, &wb[2]); }
          double un = 0.0;
          if (!is_wall_face(g, d, fi)) {
            double Lq[3], Rq[3];
            double ua = g->u[d][ca], ubv = g->u[d][cb];
            for (int a = 0; a < 3; a++) {
              Lq[a] = g->u[a][ca] + (0.5 * h - 0.5 * dt * ua) * slope_u(g, a, d, wa[0], wa[1], wa[2]) -
                      0.5 * dt * trans_u(g, d, a, wa[0], wa[1], wa[2]) + 0.5 * dt / g->rho[ca] * F[a][ca];
              Rq[a] = g->u[a][cb] - (0.5 * h + 0.5 * dt * ubv) * slope_u(g, a, d, wb[0], wb[1], wb[2]) -
                      0.5 * dt * trans_u(g, d, a, wb[0], wb[1], wb[2]) + 0.5 * dt / g->rho[cb] * F[a][cb];
            }
            un = orc_godunov_normal(Lq[d], Rq[d], g->utol);
            for (int a = 0; a < 3; a++) g->uf[d][a][f] = (a == d) ? un : orc_upwind(Lq[a], Rq[a], un, g->utol);
          }
          /* xi faces: both sides -> upwind with the same normal velocity; one side -> that side
           * (Reading; this is also the wall-face rule) */
          for (int m = 0; m < g->nsol; m++) {
            solid* S = &g->sol[m];
            int okA = has_a && S->lay[ca] >= 0, okB = has_b && S->lay[cb] >= 0;
            S->xfok[d][f] = (signed char)(okA || okB);
            if (!okA && !okB) continue;
            for (int a = 0; a < 3; a++) {
              double Lx = 0, Rx = 0;
              if (okA)
                Lx = S->xi[a][ca] + (0.5 * h - 0.5 * dt * g->u[d][ca]) * slope_x(g, S->xi, S->lay, a, d, wa[0], wa[1], wa[2]) -
                     0.5 * dt * trans_x(g, S, d, a, wa[0], wa[1], wa[2]);
              if (okB)
                Rx = S->xi[a][cb] - (0.5 * h + 0.5 * dt * g->u[d][cb]) * slope_x(g, S->xi, S->lay, a, d, wb[0], wb[1], wb[2]) -
                     0.5 * dt * trans_x(g, S, d, a, wb[0], wb[1], wb[2]);
              S->xf[d][a][f] = (okA && okB) ? orc_upwind(Lx, Rx, un, g->utol) : (okA ? Lx : Rx);
            }
          }
        }
  }
  for (int a = 0; a < 3; a++) free(F[a]);
}

/* ------------------------------------------------------------------------------- */
/* linear solvers: conjugate gradients on the mean-free subspace                     */
/* ------------------------------------------------------------------------------- */

typedef void (*opfn)(orc_grid*, const double*, const double*, double*);

/* Sums over fixed chunks of SUM_CHUNK entries, the chunk totals added in order: the same
 * result for any number of threads. */
#define SUM_CHUNK 4096L
static double chunked_sum(const double* a, const double* b, long n) {
  const long nch = (n + SUM_CHUNK - 1) / SUM_CHUNK;
  double* part = dalloc(nch);
#pragma omp parallel for schedule(static)
  for (long q = 0; q < nch; q++) {
    const long i1 = (q + 1) * SUM_CHUNK < n ? (q + 1) * SUM_CHUNK : n;
    double s = 0.0;
    for (long i = q * SUM_CHUNK; i < i1; i++) s += b ? a[i] * b[i] : a[i];
    part[q] = s;
  }
  double s = 0.0;
  for (long q = 0; q < nch; q++) s += part[q];
  free(part);
  return s;
}
static double dotp(const double* a, const double* b, long n) { return chunked_sum(a, b, n); }
static void demean(double* a, long n) {
  double s = chunked_sum(a, NULL, n);
  s /= (double)n;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; i++) a[i] -= s;
}

/* solves A x = b for the symmetric positive semi-definite A whose null space is the
 * constants; b is made mean-free first; returns the iteration count or -1 */
static int cg(orc_grid* g, opfn A, const double* coef, const double* b_in, double* x, long n) {
  double *r = dalloc(n), *pv = dalloc(n), *Ap = dalloc(n), *b = dalloc(n);
  memcpy(b, b_in, sizeof(double) * n);
  demean(b, n);
  for (long i = 0; i < n; i++) x[i] = 0.0;
  memcpy(r, b, sizeof(double) * n);
  memcpy(pv, r, sizeof(double) * n);
  double bn = sqrt(dotp(b, b, n));
  double rr = dotp(r, r, n);
  int it = 0, maxit = g->d.solve_max_iter > 0 ? g->d.solve_max_iter : 20000;
  double tol = g->d.solve_rtol > 0 ? g->d.solve_rtol : 1e-14;
  if (bn == 0.0) goto done;
  while (sqrt(rr) > tol * bn && it < maxit) {
    A(g, coef, pv, Ap);
    double pAp = dotp(pv, Ap, n);
    if (!(pAp > 0.0)) break;
    double al = rr / pAp;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) { x[i] += al * pv[i]; r[i] -= al * Ap[i]; }
    it++;
    if (it % 50 == 0) {
      /* residual replacement: keep the recursive residual equal to the true one */
      A(g, coef, x, Ap);
#pragma omp parallel for schedule(static)
      for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    }
    demean(r, n);
    double rr2 = dotp(r, r, n);
    double be = rr2 / rr;
    rr = rr2;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) pv[i] = r[i] + be * pv[i];
  }
done:
  demean(x, n);
  /* true relative residual of the returned solution */
  A(g, coef, x, Ap);
  for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
  g->last_true_rel = bn > 0.0 ? sqrt(dotp(r, r, n)) / bn : 0.0;
  free(r); free(pv); free(Ap); free(b);
  return (bn == 0.0 || sqrt(rr) <= tol * bn) ? it : -1;
}

/* MAC operator (negated so it is positive semi-definite):
 * (A q)_c = -(1/h^2) sum_d [ beta_{d,+}(q_{c+e_d} - q_c) - beta_{d,-}(q_c - q_{c-e_d}) ],
 * beta = 1/rho_face with rho_face the mean of the two cells (Reading), zero on walls. */
static void mac_apply(orc_grid* g, const double* rho, const double* q, double* out) {
  const double h2 = g->h * g->h;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->n[2]; k++)
    for (int j = 0; j < g->n[1]; j++)
      for (int i = 0; i < g->n[0]; i++) {
        long c = cidx(g, i, j, k);
        double s = 0.0;
        for (int d = 0; d < 3; d++)
          for (int sgn_ = -1; sgn_ <= 1; sgn_ += 2) {
            int ii[3] = {i, j, k};
            ii[d] += sgn_;
            long nb;
            if (!cellw(g, ii[0], ii[1], ii[2], &nb)) continue; /* wall face: no flux */
            double beta = 2.0 / (rho[c] + rho[nb]);
            s += beta * (q[nb] - q[c]);
          }
        out[c] = -s / h2;
      }
}

/* MAC projection (SI eq. mac_proj): solve div(rho^-1 grad q) = div(u_face)/(dt/2), then
 * subtract (dt/2) rho^-1 grad q from the normal face velocities. */
int orc_mac_project(orc_grid* g, const double* rho, double* ufx, double* ufy, double* ufz, double dt, double* q_out) {
  double* U[3] = {ufx, ufy, ufz};
  double* rhs = dalloc(g->N);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->n[2]; k++)
    for (int j = 0; j < g->n[1]; j++)
      for (int i = 0; i < g->n[0]; i++) {
        double dv = 0.0;
        for (int d = 0; d < 3; d++) {
          long fl, fh;
          efaces(g, d, i, j, k, &fl, &fh);
          dv += (U[d][fh] - U[d][fl]) / g->h;
        }
        /* A = -L, so A q = -rhs */
        rhs[cidx(g, i, j, k)] = -dv / (0.5 * dt);
      }
  int it = cg(g, mac_apply, rho, rhs, q_out, g->N);
  g->iters[0] = it;
  g->true_rel[0] = g->last_true_rel;
  for (int d = 0; d < 3; d++) {
    int ext[3] = {g->n[0], g->n[1], g->n[2]};
    ext[d] += 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < ext[2]; k++)
      for (int j = 0; j < ext[1]; j++)
        for (int i = 0; i < ext[0]; i++) {
          int fi = d == 0 ? i : (d == 1 ? j : k);
          if (is_wall_face(g, d, fi)) continue;
          int ia[3] = {i, j, k};
          ia[d] -= 1;
          long ca, cb;
          cellw(g, ia[0], ia[1], ia[2], &ca);
          cellw(g, i, j, k, &cb);
          double beta = 2.0 / (rho[ca] + rho[cb]);
          U[d][fidx(g, d, i, j, k)] -= 0.5 * dt * beta * (q_out[cb] - q_out[ca]) / g->h;
        }
  }
  free(rhs);
  return it < 0 ? ENOCONV_ : OK;
}

/* Trilinear finite-element stiffness (SI "Approximate pressure-Poisson projection";
 * Almgren et al. 1996): K_ij = sum_cells beta_c int_c grad N_i . grad N_j.  On a cube of
 * side h the element matrix is (h/12) * {4 same node, 0 edge, -1 face diagonal,
 * -1 body diagonal}.  beta lives on cells. */
/* The element loops below add each cell's contributions into its 8 nodes.  They visit the
 * cells in 8 colours of (i, j, k) parity: two cells of one colour share no node (on a periodic
 * axis when its cell count is even), so a colour runs in parallel and every node's sum is
 * taken in the same order for any number of threads. */
static int colour_parallel(const orc_grid* g) {
  for (int d = 0; d < 3; d++)
    if (g->per[d] && (g->n[d] & 1)) return 0;
  return 1;
}
void orc_fe_apply(orc_grid* g, const double* beta, const double* psi, double* out) {
  for (long i = 0; i < g->NN; i++) out[i] = 0.0;
  const int par = colour_parallel(g);
  for (int col = 0; col < 8; col++)
#pragma omp parallel for collapse(2) schedule(static) if (par)
  for (int k = (col >> 2) & 1; k < g->n[2]; k += 2)
    for (int j = (col >> 1) & 1; j < g->n[1]; j += 2)
      for (int i = col & 1; i < g->n[0]; i += 2) {
        long nd[8];
        double v[8];
        for (int q = 0; q < 8; q++) {
          nodew(g, i + (q & 1), j + ((q >> 1) & 1), k + ((q >> 2) & 1), &nd[q]);
          v[q] = psi[nd[q]];
        }
        double s = beta[cidx(g, i, j, k)] * g->h / 12.0;
        for (int a = 0; a < 8; a++) {
          double acc = 0.0;
          for (int b = 0; b < 8; b++) {
            int diff = __builtin_popcount((unsigned)(a ^ b));
            double w = diff == 0 ? 4.0 : (diff == 1 ? 0.0 : -1.0);
            acc += w * v[b];
          }
          out[nd[a]] += s * acc;
        }
      }
}
static void fe_apply_op(orc_grid* g, const double* beta, const double* x, double* out) { orc_fe_apply(g, beta, x, out); }

/* weak divergence: f_i = sum_c int_c V_c . grad N_i = sum_c (h^2/4) sum_d sigma_d V_{c,d},
 * sigma_d = +1 when node i is on the high side of cell c along d, -1 otherwise */
void orc_fe_weak_div(orc_grid* g, const double* V, double* out) {
  for (long i = 0; i < g->NN; i++) out[i] = 0.0;
  const double s = g->h * g->h / 4.0;
  const int par = colour_parallel(g);
  for (int col = 0; col < 8; col++)
#pragma omp parallel for collapse(2) schedule(static) if (par)
  for (int k = (col >> 2) & 1; k < g->n[2]; k += 2)
    for (int j = (col >> 1) & 1; j < g->n[1]; j += 2)
      for (int i = col & 1; i < g->n[0]; i += 2) {
        long c = cidx(g, i, j, k);
        for (int q = 0; q < 8; q++) {
          int a = q & 1, b = (q >> 1) & 1, e = (q >> 2) & 1;
          long nd;
          nodew(g, i + a, j + b, k + e, &nd);
          double v = (a ? V[c] : -V[c]) + (b ? V[g->N + c] : -V[g->N + c]) + (e ? V[2 * g->N + c] : -V[2 * g->N + c]);
          out[nd] += s * v;
        }
      }
}

int orc_fe_solve(orc_grid* g, const double* rho, const double* V, double* psi_out) {
  double* beta = dalloc(g->N);
  double* f = dalloc(g->NN);
  for (long c = 0; c < g->N; c++) beta[c] = 1.0 / rho[c];
  orc_fe_weak_div(g, V, f);
  int it = cg(g, fe_apply_op, beta, f, psi_out, g->NN);
  g->iters[1] = it;
  g->true_rel[1] = g->last_true_rel;
  free(beta); free(f);
  return it < 0 ? ENOCONV_ : OK;
}

/* ------------------------------------------------------------------------------- */
/* initialisation and timestep                                                      */
/* ------------------------------------------------------------------------------- */

/* Reading: dt = min(0.2 h, 0.8 rho_min h^2 / (6 mu_max), 0.5 h / sqrt(G_max / rho_min)) when
 * the caller gives none (explicit viscous and elastic-wave limits). */
static double pick_dt(orc_grid* g) {
  if (g->d.dt > 0.0) return g->d.dt;
  double rmin = g->d.rho_f, mumax = g->d.mu, gmax = 0.0, h = g->h;
  for (int m = 0; m < g->nsol; m++) {
    const orc_solid_desc* s = &g->sol[m].d;
    if (s->rho_s < rmin) rmin = s->rho_s;
    double ma = s->mu_a * (1.0 + s->gamma_t);
    if (ma > mumax) mumax = ma;
    if (s->G > gmax) gmax = s->G;
  }
  double dt = 0.2 * h;
  double dv = 0.8 * rmin * h * h / (6.0 * mumax);
  if (dv < dt) dt = dv;
  if (gmax > 0.0) {
    double de = 0.5 * h / sqrt(gmax / rmin);
    if (de < dt) dt = de;
  }
  return dt;
}

/* SI "Initialization": xi^0 = x in the solids, extrapolation, phi, rho^0.
 * Reading: on a periodic axis the reference coordinate is the periodic image of x
 * nearest to the body's centre. */
static void init_solid(orc_grid* g, solid* S) {
  signed char* cand = calloc8(g->N);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->n[2]; k++)
    for (int j = 0; j < g->n[1]; j++)
      for (int i = 0; i < g->n[0]; i++) {
        long c = cidx(g, i, j, k);
        double x[3];
        cell_center(g, i, j, k, x);
        for (int d = 0; d < 3; d++)
          if (g->per[d]) {
            double L = g->d.hi[d] - g->d.lo[d];
            x[d] += L * floor((S->d.center[d] - x[d]) / L + 0.5);
          }
        for (int a = 0; a < 3; a++) S->xi[a][c] = x[a];
        cand[c] = 1;
      }
  extrapolate(g, S, S->xi, S->phi, S->lay, cand);
  free(cand);
}

static void ensure_init(orc_grid* g) {
  if (g->inited) return;
  g->inited = 1;
  g->dt = pick_dt(g);
  g->utol = 1e-12 * g->h / g->dt;
  for (int m = 0; m < g->nsol; m++) init_solid(g, &g->sol[m]);
  mix_density(g, 0, g->rho);
}

static int one_step(orc_grid* g) {
  const long N = g->N;
  const double dt = g->dt, h = g->h;
  int rc = OK;
  /* 1. tau^n and its divergence */
  stress_divergence(g, 0, g->t, g->divtau_n);
  /* 2. Godunov face states (transverse bar states first) */
  bar_states(g);
  face_states(g);
  /* 3. MAC projection of the normal face velocities */
  for (int d = 0; d < 3; d++) memcpy(g->umac[d], g->uf[d][d], sizeof(double) * g->NF[d]);
  if (orc_mac_project(g, g->rho, g->umac[0], g->umac[1], g->umac[2], dt, g->q) != OK) rc = ENOCONV_;
  /* 4. advective terms (eq. adv_terms) and 5. predictor of xi (eq. dis_xi_adv) */
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->n[2]; k++)
    for (int j = 0; j < g->n[1]; j++)
      for (int i = 0; i < g->n[0]; i++) {
        long c = cidx(g, i, j, k);
        double acc[3] = {0, 0, 0};
        for (int d = 0; d < 3; d++) {
          long fl, fh;
          efaces(g, d, i, j, k, &fl, &fh);
          /* the normal component is the MAC-corrected one; the others are the upwinded states */
          double vavg = 0.5 * (g->umac[d][fl] + g->umac[d][fh]);
          for (int a = 0; a < 3; a++) {
            const double* Q = a == d ? g->umac[d] : g->uf[d][a];
            acc[a] += vavg * (Q[fh] - Q[fl]) / h;
          }
        }
        for (int a = 0; a < 3; a++) g->adv[a][c] = acc[a];
      }
  for (int m = 0; m < g->nsol; m++) {
    solid* S = &g->sol[m];
    signed char* cand = calloc8(N);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->n[2]; k++)
      for (int j = 0; j < g->n[1]; j++)
        for (int i = 0; i < g->n[0]; i++) {
          long c = cidx(g, i, j, k);
          S->xn[0][c] = S->xn[1][c] = S->xn[2][c] = NAN;
          /* Reading: the predictor runs on the cells of layers 0 and 1 (the interface moves
           * less than a cell per step) whose six faces carry xi^{n+1/2} */
          if (S->lay[c] < 0 || S->lay[c] > 1) continue;
          int ok = 1;
          double acc[3] = {0, 0, 0};
          for (int d = 0; d < 3 && ok; d++) {
            long fl, fh;
            efaces(g, d, i, j, k, &fl, &fh);
            if (!S->xfok[d][fl] || !S->xfok[d][fh]) { ok = 0; break; }
            double vavg = 0.5 * (g->umac[d][fl] + g->umac[d][fh]);
            for (int a = 0; a < 3; a++) acc[a] += vavg * (S->xf[d][a][fh] - S->xf[d][a][fl]) / h;
          }
          if (!ok) continue;
          for (int a = 0; a < 3; a++) S->xn[a][c] = S->xi[a][c] - dt * acc[a];
          cand[c] = 1;
        }
    /* 6. re-classify and extrapolate the predictor */
    extrapolate(g, S, S->xn, S->phin, S->layn, cand);
    free(cand);
    /* 7. corrector xi^{n+1/2} = (xi^n + xi^{n+1})/2 on every cell holding both.
     * Reading: a cell new to the band (no xi^n) gets xi^{n+1/2} by the same WLS
     * extrapolation, layer by layer (band of step n+1), from the corrected values of the
     * lower layers; this keeps affine maps exact. */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; c++) {
      if (S->layn[c] < 0 || S->lay[c] < 0) { S->xh[0][c] = S->xh[1][c] = S->xh[2][c] = NAN; continue; }
      for (int a = 0; a < 3; a++) S->xh[a][c] = 0.5 * (S->xi[a][c] + S->xn[a][c]);
    }
    for (int l = 1; l <= g->d.band_layers; l++) {
      int bad = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(+ : bad)
      for (int k = 0; k < g->n[2]; k++)
        for (int j = 0; j < g->n[1]; j++)
          for (int i = 0; i < g->n[0]; i++) {
            long c = cidx(g, i, j, k);
            if (S->layn[c] != l || S->lay[c] >= 0) continue;
            double out[3];
            if (!wls_cell(g, S, S->xh, S->layn, i, j, k, l, out)) {
              /* cannot happen when the same cell was extrapolated at step 6 from a superset */
              out[0] = S->xn[0][c]; out[1] = S->xn[1][c]; out[2] = S->xn[2][c];
              bad++;
            }
            S->xh[0][c] = out[0]; S->xh[1][c] = out[1]; S->xh[2][c] = out[2];
          }
      g->degenerate += bad;
    }
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; c++) {
      if (S->layn[c] < 0) { S->phih[c] = NAN; continue; }
      double xv[3] = {S->xh[0][c], S->xh[1][c], S->xh[2][c]};
      S->phih[c] = orc_phi0(&S->d, xv);
    }
  }
  /* 8. tau^{n+1/2} (solid stress from xi^{n+1/2}, viscous parts from u^n) */
  stress_divergence(g, 1, g->t + 0.5 * dt, g->divtau_h);
  /* 9. rho^{n+1/2} */
  mix_density(g, 1, g->rho_h);
  /* 10. u* (Reading of the garbled item: eq. dis_full_mmt with p^{n-1/2}); the wall
   * repulsion joins b^{n+1/2} as rho a_rep, from phi^{n+1/2} */
  rep_accel(g, 1, g->rep);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < g->n[2]; k++)
    for (int j = 0; j < g->n[1]; j++)
      for (int i = 0; i < g->n[0]; i++) {
        long c = cidx(g, i, j, k);
        double gp[3];
        grad_at_cell(g, g->p, i, j, k, gp);
        for (int a = 0; a < 3; a++)
          g->ustar[a][c] = g->u[a][c] - dt * g->adv[a][c] +
                           dt / g->rho_h[c] * (g->divtau_h[a][c] - gp[a] + (g->rho_h[c] - g->d.rho_f) * g->d.gravity[a] +
                                               g->rho_h[c] * g->rep[a][c]);
      }
  /* 11. approximate projection of (u* - u^n)/dt, u^{n+1}, p^{n+1/2} */
  {
    double* V = dalloc(3 * N);
    for (int a = 0; a < 3; a++)
      for (long c = 0; c < N; c++) V[a * N + c] = (g->ustar[a][c] - g->u[a][c]) / dt;
    if (orc_fe_solve(g, g->rho_h, V, g->psi) != OK) rc = ENOCONV_;
    free(V);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->n[2]; k++)
      for (int j = 0; j < g->n[1]; j++)
        for (int i = 0; i < g->n[0]; i++) {
          long c = cidx(g, i, j, k);
          double gp[3];
          grad_at_cell(g, g->psi, i, j, k, gp);
          for (int a = 0; a < 3; a++) g->u[a][c] = g->ustar[a][c] - dt / g->rho_h[c] * gp[a];
        }
    for (long i = 0; i < g->NN; i++) g->p[i] += g->psi[i];
  }
  /* 12. xi <- xi^{n+1}; 13. rho^{n+1} (Reading: from phi_0(xi^{n+1})) */
  for (int m = 0; m < g->nsol; m++) {
    solid* S = &g->sol[m];
    for (int a = 0; a < 3; a++) memcpy(S->xi[a], S->xn[a], sizeof(double) * N);
    memcpy(S->phi, S->phin, sizeof(double) * N);
    memcpy(S->lay, S->layn, (size_t)N);
  }
  mix_density(g, 0, g->rho);
  g->t += dt;
  g->step++;
  return rc;
}

/* Initial pressure iterations (SI "Initialization" item 2): a timestep from the initial state
 * is run with the current estimate of p^{-1/2}; its p^{1/2} becomes the next estimate and
 * every other change is discarded.  Reading of the stopping test (the paper names a tolerance
 * on the divergence of u^0, which the iterations do not change): stop once the estimate moves
 * by at most tol relative, ||p_k - p_{k-1}||_2 <= tol ||p_k||_2, or after max_iters
 * iterations.  The projection computes pressure increments (p += psi), the variant the paper
 * asks for. */
int orc_init_pressure(orc_grid* g, int max_iters, double tol, int* iters_out) {
  if (!g || max_iters < 0) return EINVAL_;
  ensure_init(g);
  if (g->step != 0) return ESTATE_;
  const long N = g->N, NN = g->NN;
  double* u0[3];
  for (int a = 0; a < 3; a++) { u0[a] = dalloc(N); memcpy(u0[a], g->u[a], sizeof(double) * N); }
  double* rho0 = dalloc(N);
  memcpy(rho0, g->rho, sizeof(double) * N);
  double** xi0 = (double**)calloc((size_t)(g->nsol > 0 ? g->nsol : 1) * 4, sizeof(double*));
  signed char** lay0 = (signed char**)calloc((size_t)(g->nsol > 0 ? g->nsol : 1), sizeof(signed char*));
  for (int m = 0; m < g->nsol; m++) {
    solid* S = &g->sol[m];
    for (int a = 0; a < 3; a++) { xi0[4 * m + a] = dalloc(N); memcpy(xi0[4 * m + a], S->xi[a], sizeof(double) * N); }
    xi0[4 * m + 3] = dalloc(N);
    memcpy(xi0[4 * m + 3], S->phi, sizeof(double) * N);
    lay0[m] = calloc8(N);
    memcpy(lay0[m], S->lay, (size_t)N);
  }
  double* prev = dalloc(NN);
  int it = 0, rc = OK;
  const int degen0 = g->degenerate;
  while (it < max_iters) {
    memcpy(prev, g->p, sizeof(double) * NN);
    rc = one_step(g);
    it++;
    /* keep p^{1/2}; restore everything else */
    for (int a = 0; a < 3; a++) memcpy(g->u[a], u0[a], sizeof(double) * N);
    memcpy(g->rho, rho0, sizeof(double) * N);
    for (int m = 0; m < g->nsol; m++) {
      solid* S = &g->sol[m];
      for (int a = 0; a < 3; a++) memcpy(S->xi[a], xi0[4 * m + a], sizeof(double) * N);
      memcpy(S->phi, xi0[4 * m + 3], sizeof(double) * N);
      memcpy(S->lay, lay0[m], (size_t)N);
    }
    g->t = 0.0;
    g->step = 0;
    if (rc != OK) break;
    double dn = 0.0, pn = 0.0;
    for (long i = 0; i < NN; i++) {
      const double dv = g->p[i] - prev[i];
      dn += dv * dv;
      pn += g->p[i] * g->p[i];
    }
    if (dn <= tol * tol * pn) break;
  }
  g->degenerate = degen0 > g->degenerate ? degen0 : g->degenerate;
  for (int a = 0; a < 3; a++) free(u0[a]);
  free(rho0);
  for (int m = 0; m < g->nsol; m++) {
    for (int q = 0; q < 4; q++) free(xi0[4 * m + q]);
    free(lay0[m]);
  }
  free(xi0);
  free(lay0);
  free(prev);
  if (iters_out) *iters_out = it;
  if (rc != OK) snprintf(g->err, sizeof g->err, "linear solve did not converge in the initial pressure iterations");
  return rc;
}

/* Diagnostics of one body at the current step (main text "Swimming"; SI "Swimming
 * statistics"; SI "Pre-stretched sphere", eq. elas): out[0..2] the centroid velocity, out[3]
 * the active power P = -int sigma_a : grad u dV, out[4] the body's volume, out[5] its elastic
 * energy int Phi_elas dV with Phi_elas = G/2 (tr(F^T F) - 3 - 2 ln J), out[6] the RMS of
 * J - 1 over the body.  Reading (the paper defines neither the centroid velocity nor the solid
 * region of the integrals on the grid): every sum weights a cell by the body's solid fraction
 * 1 - H_eps(phi) (the blending weight of its stress), over the cells holding the body's xi;
 * grad xi and grad u are centred differences over the two neighbouring cells (velocity ghosts
 * at walls), F = (grad xi)^-1 and J = det F; a cell whose grad xi is missing or has det <= 0
 * adds to the centroid velocity and the volume only; sigma_a is the active stress of the
 * stress calculation evaluated at the cell centre at the current time. */
int orc_body_stats(orc_grid* g, int sid, double* out) {
  if (!g || !out || sid < 0) return EINVAL_;
  ensure_init(g);
  if (sid >= g->nsol) return EINVAL_;
  const solid* S = &g->sol[sid];
  const double h = g->h, G = S->d.G;
  double wu[3] = {0.0, 0.0, 0.0}, ws = 0.0, pw = 0.0, en = 0.0, wj = 0.0, jj = 0.0;
  for (int k = 0; k < g->n[2]; k++)
    for (int j = 0; j < g->n[1]; j++)
      for (int i = 0; i < g->n[0]; i++) {
        const long c = cidx(g, i, j, k);
        if (S->lay[c] < 0) continue;
        const double w = 1.0 - orc_heaviside(S->phi[c], g->eps);
        if (!(w > 0.0)) continue;
        for (int a = 0; a < 3; a++) wu[a] += w * g->u[a][c];
        ws += w;
        /* grad xi at the cell: A[3a+d] = d xi_a / d x_d */
        double A[9];
        int ok = 1;
        const int ii[3] = {i, j, k};
        for (int d = 0; d < 3 && ok; d++) {
          int p[3] = {ii[0], ii[1], ii[2]}, m[3] = {ii[0], ii[1], ii[2]};
          p[d]++; m[d]--;
          double xp[3], xm[3];
          if (!xval(g, S->xi, S->lay, 0, p[0], p[1], p[2], &xp[0]) || !xval(g, S->xi, S->lay, 0, m[0], m[1], m[2], &xm[0])) {
            ok = 0;
            break;
          }
          for (int a = 1; a < 3; a++) {
            xval(g, S->xi, S->lay, a, p[0], p[1], p[2], &xp[a]);
            xval(g, S->xi, S->lay, a, m[0], m[1], m[2], &xm[a]);
          }
          for (int a = 0; a < 3; a++) A[3 * a + d] = (xp[a] - xm[a]) / (2.0 * h);
        }
        if (!ok) continue;
        const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                           A[2] * (A[3] * A[7] - A[4] * A[6]);
        if (!(det > 0.0)) continue;
        double F[9];
        F[0] = (A[4] * A[8] - A[5] * A[7]) / det;
        F[1] = (A[2] * A[7] - A[1] * A[8]) / det;
        F[2] = (A[1] * A[5] - A[2] * A[4]) / det;
        F[3] = (A[5] * A[6] - A[3] * A[8]) / det;
        F[4] = (A[0] * A[8] - A[2] * A[6]) / det;
        F[5] = (A[2] * A[3] - A[0] * A[5]) / det;
        F[6] = (A[3] * A[7] - A[4] * A[6]) / det;
        F[7] = (A[1] * A[6] - A[0] * A[7]) / det;
        F[8] = (A[0] * A[4] - A[1] * A[3]) / det;
        /* eq. elas: tr(C) = sum of the squares of F's entries; J = det F = 1 / det(grad xi) */
        double trC = 0.0;
        for (int q = 0; q < 9; q++) trC += F[q] * F[q];
        const double J = 1.0 / det;
        en += w * 0.5 * G * (trC - 3.0 - 2.0 * log(J));
        wj += w;
        jj += w * (J - 1.0) * (J - 1.0);
        if (S->d.active_A == 0.0) continue;
        const double* R = S->d.rot;
        const double r[3] = {S->xi[0][c] - S->d.center[0], S->xi[1][c] - S->d.center[1], S->xi[2][c] - S->d.center[2]};
        const double Xb = R[0] * r[0] + R[3] * r[1] + R[6] * r[2];
        const double Zb = R[2] * r[0] + R[5] * r[1] + R[8] * r[2];
        const double s0 = S->d.active_A * sin(2.0 * M_PI * Xb / S->d.active_len - S->d.active_omega * g->t);
        const double EX[3] = {R[0], R[3], R[6]};
        double f[3];
        for (int a = 0; a < 3; a++) f[a] = F[3 * a] * EX[0] + F[3 * a + 1] * EX[1] + F[3 * a + 2] * EX[2];
        const double fn = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        const double amp = 1.5 * Zb * s0;
        /* grad u at the cell: gu[3a+d] = d u_a / d x_d */
        double sg = 0.0;
        for (int a = 0; a < 3; a++)
          for (int d = 0; d < 3; d++) {
            int p[3] = {ii[0], ii[1], ii[2]}, m[3] = {ii[0], ii[1], ii[2]};
            p[d]++; m[d]--;
            const double gu = (uval(g, a, p[0], p[1], p[2]) - uval(g, a, m[0], m[1], m[2])) / (2.0 * h);
            const double sig = amp * ((f[a] / fn) * (f[d] / fn) - (a == d ? 1.0 / 3.0 : 0.0));
            sg += sig * gu;
          }
        pw += w * sg;
      }
  const double dv = h * h * h;
  for (int a = 0; a < 3; a++) out[a] = ws > 0.0 ? wu[a] / ws : 0.0;
  out[3] = -pw * dv;
  out[4] = ws * dv;
  out[5] = en * dv;
  out[6] = wj > 0.0 ? sqrt(jj / wj) : 0.0;
  return OK;
}

int orc_step(orc_grid* g, int nsteps) {
  if (!g) return EINVAL_;
  ensure_init(g);
  for (int s = 0; s < nsteps; s++) {
    int rc = one_step(g);
    if (rc != OK) { snprintf(g->err, sizeof g->err, "linear solve did not converge at step %ld", g->step); return rc; }
  }
  if (g->degenerate) { snprintf(g->err, sizeof g->err, "%d degenerate extrapolations", g->degenerate); return EDEGEN_; }
  return OK;
}

/* ------------------------------------------------------------------------------- */
/* field access                                                                     */
/* ------------------------------------------------------------------------------- */

long orc_field_len(orc_grid* g, int field) {
  switch (field) {
    case ORC_F_U: case ORC_F_XI: case ORC_F_DIVTAU_N: case ORC_F_DIVTAU_H: case ORC_F_ADV_U:
    case ORC_F_USTAR: case ORC_F_XI_HALF: case ORC_F_REPULSION: return 3 * g->N;
    case ORC_F_P: case ORC_F_PSI: return g->NN;
    case ORC_F_RHO: case ORC_F_PHI: case ORC_F_LAYER: case ORC_F_MAC_Q: case ORC_F_RHO_HALF: return g->N;
    case ORC_F_UFACE_X: return 3 * g->NF[0];
    case ORC_F_UFACE_Y: return 3 * g->NF[1];
    case ORC_F_UFACE_Z: return 3 * g->NF[2];
    case ORC_F_UMAC_X: return g->NF[0];
    case ORC_F_UMAC_Y: return g->NF[1];
    case ORC_F_UMAC_Z: return g->NF[2];
  }
  return -1;
}

int orc_read(orc_grid* g, int field, int sid, double* dst, long n) {
  if (!g) return EINVAL_;
  ensure_init(g);
  long len = orc_field_len(g, field);
  if (len < 0 || n < len) return EINVAL_;
  const long N = g->N;
  solid* S = NULL;
  if (field == ORC_F_XI || field == ORC_F_PHI || field == ORC_F_LAYER || field == ORC_F_XI_HALF) {
    if (sid < 0 || sid >= g->nsol) return EINVAL_;
    S = &g->sol[sid];
  }
  switch (field) {
    case ORC_F_U: for (int a = 0; a < 3; a++) memcpy(dst + a * N, g->u[a], sizeof(double) * N); break;
    case ORC_F_P: memcpy(dst, g->p, sizeof(double) * g->NN); break;
    case ORC_F_RHO: memcpy(dst, g->rho, sizeof(double) * N); break;
    case ORC_F_XI: for (int a = 0; a < 3; a++) memcpy(dst + a * N, S->xi[a], sizeof(double) * N); break;
    case ORC_F_PHI: memcpy(dst, S->phi, sizeof(double) * N); break;
    case ORC_F_LAYER: for (long c = 0; c < N; c++) dst[c] = S->lay[c]; break;
    case ORC_F_XI_HALF: for (int a = 0; a < 3; a++) memcpy(dst + a * N, S->xh[a], sizeof(double) * N); break;
    case ORC_F_DIVTAU_N: for (int a = 0; a < 3; a++) memcpy(dst + a * N, g->divtau_n[a], sizeof(double) * N); break;
    case ORC_F_DIVTAU_H: for (int a = 0; a < 3; a++) memcpy(dst + a * N, g->divtau_h[a], sizeof(double) * N); break;
    case ORC_F_ADV_U: for (int a = 0; a < 3; a++) memcpy(dst + a * N, g->adv[a], sizeof(double) * N); break;
    case ORC_F_USTAR: for (int a = 0; a < 3; a++) memcpy(dst + a * N, g->ustar[a], sizeof(double) * N); break;
    case ORC_F_REPULSION: for (int a = 0; a < 3; a++) memcpy(dst + a * N, g->rep[a], sizeof(double) * N); break;
    case ORC_F_PSI: memcpy(dst, g->psi, sizeof(double) * g->NN); break;
    case ORC_F_MAC_Q: memcpy(dst, g->q, sizeof(double) * N); break;
    case ORC_F_RHO_HALF: memcpy(dst, g->rho_h, sizeof(double) * N); break;
    case ORC_F_UFACE_X: case ORC_F_UFACE_Y: case ORC_F_UFACE_Z: {
      int d = field - ORC_F_UFACE_X;
      for (int a = 0; a < 3; a++) memcpy(dst + a * g->NF[d], g->uf[d][a], sizeof(double) * g->NF[d]);
      break;
    }
    case ORC_F_UMAC_X: case ORC_F_UMAC_Y: case ORC_F_UMAC_Z: {
      int d = field - ORC_F_UMAC_X;
      memcpy(dst, g->umac[d], sizeof(double) * g->NF[d]);
      break;
    }
    default: return EINVAL_;
  }
  return OK;
}

/* Writes U, P, or the reference map of one solid.  Writing XI re-runs classification,
 * layer marking and extrapolation with every cell holding a finite xi as a candidate
 * primary value, then re-blends rho (as after SI Initialization item 4-6). */
int orc_write(orc_grid* g, int field, int sid, const double* src, long n) {
  if (!g) return EINVAL_;
  ensure_init(g);
  const long N = g->N;
  if (field == ORC_F_U) {
    if (n < 3 * N) return EINVAL_;
    for (int a = 0; a < 3; a++) memcpy(g->u[a], src + a * N, sizeof(double) * N);
    return OK;
  }
  if (field == ORC_F_P) {
    if (n < g->NN) return EINVAL_;
    memcpy(g->p, src, sizeof(double) * g->NN);
    return OK;
  }
  if (field == ORC_F_XI) {
    if (n < 3 * N || sid < 0 || sid >= g->nsol) return EINVAL_;
    solid* S = &g->sol[sid];
    signed char* cand = calloc8(N);
    for (long c = 0; c < N; c++) {
      for (int a = 0; a < 3; a++) S->xi[a][c] = src[a * N + c];
      cand[c] = isfinite(src[c]) && isfinite(src[N + c]) && isfinite(src[2 * N + c]);
    }
    extrapolate(g, S, S->xi, S->phi, S->lay, cand);
    free(cand);
    mix_density(g, 0, g->rho);
    return g->degenerate ? EDEGEN_ : OK;
  }
  return EINVAL_;
}
