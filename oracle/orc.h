/*
 * TEST INFRASTRUCTURE ONLY.  Plain FP64 CPU oracle of the per-RK-stage
 * right-hand side of arXiv 2303.10785 (MEG6 + HLLC + alpha-damping on
 * curvilinear, possibly moving, structured meshes).  Only tests/, the smoke
 * check and bench.py's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Layouts (all arrays C-contiguous doubles, i fastest):
 *   nodes   [ndim][Nk][Nj][Ni] with N_d = n_d + 1 on periodic axes and
 *           n_d + 1 + 2*ghost_nodes on non-periodic axes (ghost layers first).
 *   state   [nv][nk][nj][ni]  (nv = ndim + 2; conserved rho, rho u.., E)
 *   faces   [..][n_other...][n_d + 1] along direction d: face index f = 0..n_d
 *           is the interface i+1/2 with i = f - 1 (so f = 0 is the low boundary
 *           face).  The face arrays are laid out like a cell array whose extent
 *           along d is n_d + 1.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_ZEROGRAD = 1, ORC_BC_INFLOW = 2, ORC_BC_WALL = 3 };

typedef struct {
  int ndim;              /* 2 or 3 */
  int n[3];              /* cells per axis; n[2] = 1 when ndim == 2 */
  int periodic[3];       /* 1 = periodic axis */
  int ghost_nodes;       /* node layers supplied beyond each non-periodic side (>= 10), or 0:
                            the non-periodic axes end at walls and their metrics take the
                            one-sided formulas of App. C */
  int bc[3][2];          /* non-periodic sides: ORC_BC_ZEROGRAD, ORC_BC_INFLOW (x-low only) or
                            ORC_BC_WALL (slip wall) */
  int metric_scheme;     /* 0 = conservative metrics with the MEG6 operator (Sec. 7),
                            1 = non-conservative metrics with E4 (App. D, negative control) */
  double gamma, prandtl;
  double reynolds;       /* <= 0: Euler (no viscous flux); mu_ref = 1/reynolds */
  double sutherland_s;   /* S / T_ref; <= 0: constant viscosity mu_ref */
  double t_ref;          /* reference temperature (T = p/rho units) for Sutherland */
  double alpha_damping;  /* alpha^D of Eq. (AD-eqn1); paper: 4 */
  double mp_alpha, mp_beta, mp_eps;  /* App. E limiter constants */
  int gradient_scheme;   /* 0 = MEG6: explicit E6 gradients (Eq. E6_grads);
                            1 = MIG4: implicit IG4 gradients (Eq. IG4_grads), cyclic on periodic
                            axes, explicit end rows on open lines */
} orc_params;

typedef struct orc_solver orc_solver;

/* 0 on success, nonzero on invalid input (message via orc_last_error). */
int  orc_create(const orc_params* p, const double* nodes, const double* node_vel, orc_solver** out);
int  orc_set_nodes(orc_solver* s, const double* nodes, const double* node_vel);
/* xc_ext: [ndim][ek][ej][ei] cell centroids on the extended box [-10, n+10) per active axis. */
int  orc_set_centroids(orc_solver* s, const double* xc_ext, const double* vc_ext);
void orc_destroy(orc_solver* s);
const char* orc_last_error(void);
int  orc_ext_pad(void);

/* geometry read-back */
void orc_get_cell_metrics(const orc_solver* s, double* mh /*[nd][nd][cells]*/, double* det /*[cells]*/);
void orc_get_cell_time_metrics(const orc_solver* s, double* mt /*[nd][cells]*/);
void orc_get_face_metrics(const orc_solver* s, int d, double* fh /*[nd][faces]*/,
                          double* fu /*[nd][nd][faces] or NULL*/, double* ft /*[faces] or NULL*/);
void orc_get_gcl(const orc_solver* s, double* gcl /*[cells]*/);

/* jet-type boundary data */
void orc_set_inflow(orc_solver* s, const double* prim /*[nv][nk][nj]*/);
void orc_set_sponge(orc_solver* s, const double* sigma /*[cells]*/, const double* q_amb /*[nv]*/);

/* right-hand side pieces */
int  orc_rhs(orc_solver* s, const double* q, double* L /*[nv][cells]*/);
int  orc_residual(orc_solver* s, const double* q, double* res /*[nv][cells]*/);
int  orc_face_flux(orc_solver* s, const double* q, int d, double* g /*[nv][faces]*/);
int  orc_primitives(orc_solver* s, const double* q, double* prim /*[nv][cells]*/);
double orc_dt(orc_solver* s, const double* q, double cfl);
/* Sec. 2: dynamic viscosity mu(T) of the solver's parameters (T = p/rho units). */
double orc_viscosity(const orc_solver* s, double T);
/* One SSP-RK3 step in place.  stage_nodes/stage_vel: NULL for a static mesh,
   else 3 node sets (and velocities) at t, t+dt, t+dt/2. */
int  orc_rk3(orc_solver* s, double* q, double dt,
             const double* const* stage_nodes, const double* const* stage_vel);

/* small pieces for pin tests */
void orc_op1d(int kind, int n, const double* f, double* out); /* periodic line; kind 0:E6 1:second 2:face 3:D 4:E4 */
void orc_eigen(int nd, const double* nh, double rho, double p, double gamma, double* R, double* Rinv);
void orc_hllc(int nd, const double* PL, const double* PR, const double* nh, double nt, double gamma, double* F);
double orc_mp_limit(double wface, double w_up, double w_base, double w_down,
                    double d_up, double d_base, double d_down, double alpha, double beta, double eps);

/* counting build only (-DORC_COUNTING): operation tallies since the last reset */
void orc_count_reset(void);
void orc_count_get(unsigned long long* add, unsigned long long* mul,
                   unsigned long long* div, unsigned long long* sqrt_);
/* phase: 0 time step / RK combination, 1 primitives, 2 gradients, 3 interface
   fluxes, 4 divergence and source terms, 5 geometry; -1 = all */
void orc_count_get_phase(int phase, unsigned long long* add, unsigned long long* mul,
                         unsigned long long* div, unsigned long long* sqrt_);
int  orc_is_counting(void);
int  orc_threads(void);
void orc_set_threads(int n); /* OpenMP threads of the following calls (n > 0) */

#ifdef __cplusplus
}
#endif
#endif
