/*
 * rmt_oracle.h -- plain, slow, FP64 CPU oracle of the per-timestep update of the
 * 3D reference map technique (Lin, Derr & Rycroft, arXiv 2104.00095).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists so that the tests, the smoke check
 * and the CPU-baseline leg of the benchmark can compare the CUDA path against an
 * independent statement of the scheme.  It shares no source with the CUDA library
 * and the product path never calls it.
 *
 * Every function follows a passage of the paper (cited beside it in the .c file):
 *   SI "Timestepping algorithm" (13 steps), SI "Initialization", main text
 *   "Extrapolation of xi", SI "Weighting scheme", SI "Stress calculations",
 *   SI "Evaluating the advective term", SI "MAC projection",
 *   SI "Approximate pressure-Poisson projection", eqs. blend / sm_heavi /
 *   mixed_stresses / mod_heaviside.
 * Where the paper is silent or garbled the oracle takes the readings listed in the
 * design notes; each such place is marked "Reading:" in the source.
 *
 * Layouts: cell fields x fastest, then y, then z ([nz][ny][nx]); vector fields are
 * three such blocks.  Nodal fields use nn_d = n_d+1 nodes on a wall axis and n_d on
 * a periodic axis.  Face fields of direction d use n_d+1 faces along d.
 */
#ifndef RMT_ORACLE_H
#define RMT_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_NOSLIP = 0, ORC_BC_PERIODIC = 1 };
enum { ORC_SHAPE_SPHERE = 0, ORC_SHAPE_ELLIPSOID = 1 };

typedef struct {
  int n[3];
  double lo[3], hi[3];
  int bc[6];               /* -x,+x,-y,+y,-z,+z */
  double wall_u[6][3];     /* wall velocity per face (tangential only) */
  double rho_f, mu;
  double eps_h;            /* half blur width in cells */
  int band_layers;         /* maximum extrapolation layer */
  double dt;               /* > 0 required by the oracle */
  double gravity[3];
  double solve_rtol;       /* CG relative residual target */
  int solve_max_iter;
  double wall_dw;          /* wall-repulsion threshold distance (<= 0: one grid spacing) */
} orc_grid_desc;

typedef struct {
  int shape;
  double center[3], semi_axes[3], rot[9]; /* rot: body -> world, row-major */
  double rho_s, G, mu_a, gamma_t;
  double active_A, active_omega, active_len;
  double rep_A;            /* wall-repulsion acceleration magnitude (0: none) */
} orc_solid_desc;

typedef struct orc_grid orc_grid;

/* field ids for orc_read / orc_write (same numbering as the CUDA library) */
enum {
  ORC_F_U = 1, ORC_F_P = 2, ORC_F_RHO = 3, ORC_F_XI = 4, ORC_F_PHI = 5, ORC_F_LAYER = 6,
  /* intermediates of the last step */
  ORC_F_DIVTAU_N = 20, ORC_F_DIVTAU_H = 21, ORC_F_UFACE_X = 22, ORC_F_UFACE_Y = 23,
  ORC_F_UFACE_Z = 24, ORC_F_MAC_Q = 25, ORC_F_ADV_U = 26, ORC_F_USTAR = 27,
  ORC_F_PSI = 28, ORC_F_RHO_HALF = 29, ORC_F_XI_HALF = 30, ORC_F_UMAC_X = 31,
  ORC_F_UMAC_Y = 32, ORC_F_UMAC_Z = 33,
  ORC_F_REPULSION = 34     /* wall-repulsion acceleration of the last step's u* (3 N) */
};

int  orc_create(const orc_grid_desc* d, orc_grid** out);
int  orc_add_solid(orc_grid* g, const orc_solid_desc* s, int* id);
int  orc_step(orc_grid* g, int nsteps);
/* initial pressure iterations before the first step; iters_out receives the count */
int  orc_init_pressure(orc_grid* g, int max_iters, double tol, int* iters_out);
/* diagnostics of one body: centroid velocity (3), active power, volume, elastic energy,
 * RMS of J - 1 */
int  orc_body_stats(orc_grid* g, int solid, double* out7);
long orc_field_len(orc_grid* g, int field);
int  orc_read(orc_grid* g, int field, int solid, double* dst, long n);
int  orc_write(orc_grid* g, int field, int solid, const double* src, long n);
void orc_destroy(orc_grid* g);
double orc_dt(orc_grid* g);
int  orc_last_iters(orc_grid* g, int which);   /* 0: MAC CG iterations, 1: FE CG iterations */
double orc_last_true_residual(orc_grid* g, int which); /* true relative residual of that solve */
const char* orc_error(orc_grid* g);

/* Building blocks exposed for the pin tests. */
/* A_rep of SI "Contact with a wall": the largest of U_safe^2/d_w (safety floor), V U^2 /
 * (2 d_w^2 L_min^2) (stops a body of volume V approaching at U within d_w, with the
 * conservative contact volume d_w L_min^2) and |rho_s - rho_f| V g / (rho_s d_w L_min^2)
 * (carries the body's weight at rest). */
double orc_rep_accel(double V, double U, double dw, double Lmin, double rho_s, double rho_f, double gmag,
                     double Usafe);
double orc_heaviside(double phi, double eps);
double orc_dheaviside(double phi, double eps);
double orc_limited_slope(const double q[5], const int ok[5], double h);
double orc_godunov_normal(double L, double R, double tol);
double orc_upwind(double L, double R, double un, double tol);
double orc_phi0(const orc_solid_desc* s, const double X[3]);
/* Neo-Hookean deviatoric stress (3x3 row-major) from A = grad xi (row-major). */
int  orc_neohookean(const double A[9], double G, double tau[9]);
/* Mixing rule: H and normalised weights from per-object H_m (eq. mod_heaviside). */
double orc_mix_weights(int S, const double* Hm, double* w_out);
/* Stand-alone projections on a fresh grid (for the projection pins):
 * MAC: face velocities in (layout of ORC_F_UFACE_*), rho at cells; returns q and corrected faces.
 * FE:  cell field V (3 blocks), rho at cells; returns psi (nodal) and the cell gradient. */
int  orc_mac_project(orc_grid* g, const double* rho, double* ufx, double* ufy, double* ufz,
                     double dt, double* q_out);
int  orc_fe_solve(orc_grid* g, const double* rho, const double* V, double* psi_out);
void orc_fe_apply(orc_grid* g, const double* beta, const double* psi, double* out);
void orc_fe_weak_div(orc_grid* g, const double* V, double* out);
void orc_cell_grad(orc_grid* g, const double* nodal, double* out);

#ifdef __cplusplus
}
#endif
#endif
