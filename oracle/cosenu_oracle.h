/*
 * COSEnu oracle: a plain, slow, FP64 CPU solver of the two-flavour neutrino
 * quantum kinetic equations on a periodic z grid x midpoint v bins.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * (the CUDA library and its Python binding) never calls it, and shares no
 * code, header, table or helper with it.
 *
 * What it computes, and the passage of arXiv:2203.12866 each part follows:
 *   - equations of motion (d_t + v d_z) rho = -i[H, rho], same for rhobar:
 *     Sec. 2, Eq. (eom), density matrix Eq. (rho);
 *   - Hamiltonian H = H_vac + mu int dv' (1 - v v') [rho(v') - alpha rhobar*(v')],
 *     Hbar = H_vac - mu int dv' (1 - v v') [rho*(v') - alpha rhobar(v')]:
 *     Sec. 2, Eq. (ham) with the printed H_vac;
 *   - v grid: N_v bins on [-1,1], beam at bin midpoint, Riemann sum: Sec. 3;
 *     or vertex points with the trapezoid or Simpson rule: Sec. 3.1;
 *   - FD: 4th-order central difference + Kreiss-Oliger dissipation (r = 2,
 *     or r = 3 from the general form of Q), method of lines: Sec. 3.1;
 *   - FV: cell-average update Eq. (cell_av) with 7th-order WENO flux,
 *     Eqs. (fn_w_lin_comb), (weight), Appendix A Eqs. (f7), (f4s), (Si4),
 *     Algorithm 1;
 *   - RK4 time integration: Sec. 1 and Sec. 3;
 *   - periodic boundaries in z: Sec. 4;
 *   - conserved quantities: Sec. 2 (P0, |P|), Sec. 5 (M0, delta P).
 *
 * Readings taken where the paper is silent or inconsistent (each is also
 * listed in the design notes of the repository):
 *   R1 WENO7 linear weights: the printed d_r list is in reverse order with
 *      respect to the printed sub-stencil labels; solving Eq. (fn_lin_comb)
 *      with Eqs. (f7), (f4s) gives d_0 = 4/35 for S_0 = {i..i+3},
 *      d_1 = 18/35, d_2 = 12/35, d_3 = 1/35 for S_3 = {i-3..i}.
 *   R2 SI_r is used exactly as printed in Eq. (Si4) (no 1/240 factor),
 *      with epsilon from Eq. (weight) and exponent 2.
 *   R3 upwinding: the flux f = v u is reconstructed at i+1/2 from the
 *      left-biased stencil {i-3..i+3} for v > 0 and from its mirror image
 *      {i+4..i-2} for v < 0 ("similar procedure", end of Appendix A).
 *   R4 Kreiss-Oliger: the paper adds Q u to the time-derivative side
 *      (d_t u -> d_t u + Q u), so the right-hand side receives -Q u; for
 *      r = 2 that is -(eps_ko / (16 dz)) (u_{-2} - 4u_{-1} + 6u_0 - 4u_{+1} + u_{+2}),
 *      which is dissipative; for r = 3 it is
 *      +(eps_ko / (64 dz)) (u_{-3} - 6u_{-2} + 15u_{-1} - 20u_0 + 15u_{+1} - 6u_{+2} + u_{+3}),
 *      also dissipative.  h = dz.
 *   R5 alpha is absorbed into the stored antineutrino state (Sbar = alpha g rhobar),
 *      so the code's Hamiltonian uses Sbar where Eq. (ham) has alpha rhobar.
 *   R6 an optional constant matter potential lambda enters as diag(lambda,0)
 *      for neutrinos and -diag(lambda,0) for antineutrinos (the sign that the
 *      frame rotation of the footnote of Sec. 2 removes); lambda = 0 is the
 *      paper's setting.
 *   R7 FV: the source term is evaluated on the cell values; both schemes
 *      store point/cell values on the same grid.
 *
 * State layout, shared by every function here: double [2][4][nz][nv],
 * species (nu, nubar) x component (rho_ee, rho_xx, Re rho_ex, Im rho_ex)
 * x z x v, v fastest.
 */
#ifndef COSENU_ORACLE_H
#define COSENU_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int64_t nz;        /* z cells, periodic, z in [-L/2, L/2) */
  int32_t nv;        /* v bins on [-1, 1] */
  double L;          /* domain length */
  int32_t scheme;    /* 0 = FD4 + Kreiss-Oliger r = 2, 1 = FV WENO7, 2 = FD4 + Kreiss-Oliger r = 3 */
  int32_t hmode;     /* 0 = O(Nv) quadrature per beam (Eq. ham as written), 1 = separable moments */
  double mu, omega, theta, lambda;
  double ko_eps;     /* Kreiss-Oliger strength (0.1 in the paper) */
  double weno_eps;   /* epsilon of Eq. (weight) (1e-6 in the paper) */
  double dt;
  int32_t vgrid;     /* velocity quadrature: 0 midpoint bins, 1 trapezoid, 2 Simpson (oracle_vgrid_q) */
} oracle_params;

/* v_j = -1 + (j + 1/2) dv, w_j = dv = 2 / nv. */
void oracle_vgrid(int32_t nv, double* v, double* w);

/* Velocity grid and weights of quadrature `mode`: 0 as oracle_vgrid; 1 vertex
 * grid v_j = -1 + j h, h = 2 / (nv - 1), trapezoid rule; 2 the same grid,
 * composite Simpson rule (the 1/3 rule on pairs of intervals; with an odd
 * number of intervals the last three take the 3/8 rule).  Returns -1 for an
 * unknown mode or too few points (trapezoid nv >= 2, Simpson nv >= 3). */
int oracle_vgrid_q(int32_t nv, int32_t mode, double* v, double* w);

/* Per-beam Hamiltonian, out layout [2 species][3][nz][nv]: (H_ee - H_xx, Re H_ex, Im H_ex). */
int oracle_hamiltonian(const oracle_params* p, const double* u, double* out);

/* Right-hand side k = F(u) of the semi-discrete system (advection + commutator). */
int oracle_rhs(const oracle_params* p, const double* u, double* k);

/* nsteps classic RK4 steps in place on y. */
int oracle_step(const oracle_params* p, double* y, int64_t nsteps);

/* One WENO7 reconstruction at i+1/2 from f[0..6] = f_{i-3..i+3}.
 * detail (may be NULL) receives f4[4], SI[4], wbar[4]. Returns the reconstructed value. */
double oracle_weno7_face(const double* f, double eps, double* detail);

/* Diagnostics.  out[0..9] = Tr_nu, Tr_nubar, M1, M2, M3, M_vac, dP_max, dP_mean, 0, 0.
 * Sums are sum_{z,v} w dz (...).  dP is |P|/P0 - 1 per cell with P0 = trace. */
int oracle_conserved(const oracle_params* p, const double* u, double* out);

/* z-averaged state [2][4][nv] and per-z v-moments [nz][6]
 * (D3_0, D3_1, Dr_0, Dr_1, Di_0, Di_1); either pointer may be NULL. */
int oracle_moments(const oracle_params* p, const double* u, double* zavg, double* vmom);

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int oracle_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
