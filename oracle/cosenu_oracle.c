/*
 * COSEnu oracle -- plain FP64 CPU reference of the method of arXiv:2203.12866.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.  See cosenu_oracle.h for the passage each part follows
 * and for the readings R1..R7 taken where the paper is silent or inconsistent.
 *
 * Everything is written out in the most direct form: 2x2 complex matrices
 * for the commutator, the integral of Eq. (ham) as a Riemann sum per beam,
 * the difference operators D+ and D- of Sec. 3.1 applied literally, and
 * the WENO7 steps of Algorithm 1 in order.  Nothing is fused or blocked;
 * the only parallelism is an OpenMP loop over independent z cells.
 */
#include "cosenu_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { NU = 0, NUBAR = 1 };
enum { EE = 0, XX = 1, EXR = 2, EXI = 3 };

static inline int64_t idx(const oracle_params* p, int s, int c, int64_t z, int32_t v) {
  return (((int64_t)(s * 4 + c)) * p->nz + z) * p->nv + v;
}

static inline int64_t wrap(int64_t z, int64_t nz) {
  int64_t r = z % nz;
  return r < 0 ? r + nz : r;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sec. 3: N_v bins of width dv on [-1, 1]; every beam in [v_j, v_j + dv) is
 * represented by v_j + dv/2; integrals over v are simple Riemann sums. */
void oracle_vgrid(int32_t nv, double* v, double* w) {
  const double dv = 2.0 / nv;
  for (int32_t j = 0; j < nv; ++j) {
    v[j] = -1.0 + j * dv + 0.5 * dv;
    w[j] = dv;
  }
}

/* Sec. 3.1: vertex-centred points on [-1, 1], v_j = -1 + j h, integrals by the
 * trapezoid rule (mode 1) or Simpson's rule (mode 2).  The weights are built
 * panel by panel: trapezoid panels [j, j+1] add h/2 to both ends; Simpson
 * panels [k, k+2] add h/3 (1, 4, 1); an odd interval count ends with one 3/8
 * panel [n-3, n] adding 3h/8 (1, 3, 3, 1). */
int oracle_vgrid_q(int32_t nv, int32_t mode, double* v, double* w) {
  if (mode == 0) {
    oracle_vgrid(nv, v, w);
    return 0;
  }
  if ((mode == 1 && nv < 2) || (mode == 2 && nv < 3) || (mode != 1 && mode != 2)) return -1;
  const int32_t n = nv - 1; /* intervals */
  const double h = 2.0 / n;
  for (int32_t j = 0; j < nv; ++j) {
    v[j] = -1.0 + j * h;
    w[j] = 0.0;
  }
  if (mode == 1) {
    for (int32_t j = 0; j < n; ++j) {
      w[j] += h / 2.0;
      w[j + 1] += h / 2.0;
    }
    return 0;
  }
  const int32_t n13 = (n % 2 == 0) ? n : n - 3; /* intervals covered by the 1/3 rule */
  for (int32_t k = 0; k + 2 <= n13; k += 2) {
    w[k] += h / 3.0;
    w[k + 1] += 4.0 * h / 3.0;
    w[k + 2] += h / 3.0;
  }
  if (n13 < n) {
    w[n - 3] += 3.0 * h / 8.0;
    w[n - 2] += 9.0 * h / 8.0;
    w[n - 1] += 9.0 * h / 8.0;
    w[n] += 3.0 * h / 8.0;
  }
  return 0;
}

static int check(const oracle_params* p) {
  if (!p || p->nz < 1 || p->nv < 1 || !(p->L > 0.0)) return -1;
  if (p->scheme < 0 || p->scheme > 2) return -1;
  if (p->hmode != 0 && p->hmode != 1) return -1;
  if (p->vgrid < 0 || p->vgrid > 2 || (p->vgrid > 0 && p->nv < 3)) return -1;
  return 0;
}

/* ---------------------------------------------------------------------------
 * Hamiltonian, Eq. (ham).
 *
 * With S = g rho and Sbar = alpha g rhobar stored (reading R5):
 *   H(v)    = H_vac + H_m + mu sum_j w_j (1 - v v_j) [S(v_j) - Sbar(v_j)^*]
 *   Hbar(v) = H_vac - H_m - mu sum_j w_j (1 - v v_j) [S(v_j)^* - Sbar(v_j)]
 * H_vac = (omega/2) [[-cos 2theta, sin 2theta], [sin 2theta, cos 2theta]],
 * H_m = diag(lambda, 0) (reading R6).
 * The result is written as 2x2 complex matrices hm[s][v][2][2] for one z.
 * ------------------------------------------------------------------------- */
static void build_h(const oracle_params* p, const double* u, int64_t z, const double* vg,
                    const double* wg, cplx* hm /* [2][nv][2][2] */) {
  const int32_t nv = p->nv;
  const double c2 = cos(2.0 * p->theta), s2 = sin(2.0 * p->theta);
  cplx hvac[2][2] = {{-0.5 * p->omega * c2, 0.5 * p->omega * s2},
                     {0.5 * p->omega * s2, 0.5 * p->omega * c2}};
  cplx hmat[2][2] = {{p->lambda, 0.0}, {0.0, 0.0}};

  /* density matrices of this z for both species */
  cplx* rho = (cplx*)malloc(sizeof(cplx) * 2 * nv * 4);
  for (int s = 0; s < 2; ++s)
    for (int32_t j = 0; j < nv; ++j) {
      double a = u[idx(p, s, EE, z, j)], b = u[idx(p, s, XX, z, j)];
      double cr = u[idx(p, s, EXR, z, j)], ci = u[idx(p, s, EXI, z, j)];
      cplx* r = rho + (s * nv + j) * 4;
      r[0] = a;             /* ee */
      r[1] = cr + I * ci;   /* ex */
      r[2] = cr - I * ci;   /* xe = ex^* (Hermitian, Eq. (rho)) */
      r[3] = b;             /* xx */
    }

  /* the two velocity moments of D = S - Sbar^*; used by hmode 1 */
  cplx m0[4] = {0, 0, 0, 0}, m1[4] = {0, 0, 0, 0};
  if (p->hmode == 1) {
    for (int32_t j = 0; j < nv; ++j) {
      const cplx* r = rho + (0 * nv + j) * 4;
      const cplx* rb = rho + (1 * nv + j) * 4;
      for (int e = 0; e < 4; ++e) {
        cplx d = r[e] - conj(rb[e]);
        m0[e] += wg[j] * d;
        m1[e] += wg[j] * vg[j] * d;
      }
    }
  }

  for (int32_t i = 0; i < nv; ++i) {
    cplx hnn[4] = {0, 0, 0, 0};
    if (p->hmode == 0) {
      /* int dv' (1 - v v') [S(v') - Sbar^*(v')] as a Riemann sum over beams */
      for (int32_t j = 0; j < nv; ++j) {
        const cplx* r = rho + (0 * nv + j) * 4;
        const cplx* rb = rho + (1 * nv + j) * 4;
        const double ker = wg[j] * (1.0 - vg[i] * vg[j]);
        for (int e = 0; e < 4; ++e) hnn[e] += ker * (r[e] - conj(rb[e]));
      }
    } else {
      /* the same integral split as int D dv' - v int v' D dv' */
      for (int e = 0; e < 4; ++e) hnn[e] = m0[e] - vg[i] * m1[e];
    }
    cplx* h = hm + (0 * nv + i) * 4;
    cplx* hb = hm + (1 * nv + i) * 4;
    for (int e = 0; e < 4; ++e) {
      const int a = e / 2, b = e % 2;
      h[e] = hvac[a][b] + hmat[a][b] + p->mu * hnn[e];
      /* Hbar = H_vac - H_m - mu [S^* - Sbar] integral = H_vac - H_m - (mu hnn)^* */
      hb[e] = hvac[a][b] - hmat[a][b] - p->mu * conj(hnn[e]);
    }
  }
  free(rho);
}

int oracle_hamiltonian(const oracle_params* p, const double* u, double* out) {
  if (check(p)) return -1;
  const int32_t nv = p->nv;
  double* vg = (double*)malloc(sizeof(double) * nv);
  double* wg = (double*)malloc(sizeof(double) * nv);
  oracle_vgrid_q(nv, p->vgrid, vg, wg);
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < p->nz; ++z) {
    cplx* hm = (cplx*)malloc(sizeof(cplx) * 2 * nv * 4);
    build_h(p, u, z, vg, wg, hm);
    for (int s = 0; s < 2; ++s)
      for (int32_t i = 0; i < nv; ++i) {
        const cplx* h = hm + (s * nv + i) * 4;
        out[(((int64_t)(s * 3 + 0)) * p->nz + z) * nv + i] = creal(h[0] - h[3]);
        out[(((int64_t)(s * 3 + 1)) * p->nz + z) * nv + i] = creal(h[1]);
        out[(((int64_t)(s * 3 + 2)) * p->nz + z) * nv + i] = cimag(h[1]);
      }
    free(hm);
  }
  free(vg);
  free(wg);
  return 0;
}

/* ---------------------------------------------------------------------------
 * WENO7 reconstruction at i+1/2, Appendix A and Algorithm 1.
 * f[0..6] = fbar_{i-3}, ..., fbar_{i+3}.
 * ------------------------------------------------------------------------- */
double oracle_weno7_face(const double* f, double eps, double* detail) {
  const double fm3 = f[0], fm2 = f[1], fm1 = f[2], f0 = f[3], fp1 = f[4], fp2 = f[5], fp3 = f[6];

  /* step 2: 4th-order values on S_0 = {i..i+3}, S_1 = {i-1..i+2},
   * S_2 = {i-2..i+1}, S_3 = {i-3..i}, Eq. (f4s) */
  double f4[4];
  f4[0] = (3.0 / 12.0) * f0 + (13.0 / 12.0) * fp1 + (-5.0 / 12.0) * fp2 + (1.0 / 12.0) * fp3;
  f4[1] = (-1.0 / 12.0) * fm1 + (7.0 / 12.0) * f0 + (7.0 / 12.0) * fp1 + (-1.0 / 12.0) * fp2;
  f4[2] = (1.0 / 12.0) * fm2 + (-5.0 / 12.0) * fm1 + (13.0 / 12.0) * f0 + (3.0 / 12.0) * fp1;
  f4[3] = (-3.0 / 12.0) * fm3 + (13.0 / 12.0) * fm2 + (-23.0 / 12.0) * fm1 + (25.0 / 12.0) * f0;

  /* step 3: smoothness indices, Eq. (Si4), as printed (reading R2) */
  double si[4];
  si[0] = f0 * (2107.0 * f0 - 9402.0 * fp1 + 7042.0 * fp2 - 1854.0 * fp3)
        + fp1 * (11003.0 * fp1 - 17246.0 * fp2 + 4642.0 * fp3)
        + fp2 * (7043.0 * fp2 - 3882.0 * fp3) + 547.0 * fp3 * fp3;
  si[1] = fm1 * (547.0 * fm1 - 2522.0 * f0 + 1922.0 * fp1 - 494.0 * fp2)
        + f0 * (3443.0 * f0 - 5966.0 * fp1 + 1602.0 * fp2)
        + fp1 * (2843.0 * fp1 - 1642.0 * fp2) + 267.0 * fp2 * fp2;
  si[2] = fm2 * (267.0 * fm2 - 1642.0 * fm1 + 1602.0 * f0 - 494.0 * fp1)
        + fm1 * (2843.0 * fm1 - 5966.0 * f0 + 1922.0 * fp1)
        + f0 * (3443.0 * f0 - 2522.0 * fp1) + 547.0 * fp1 * fp1;
  si[3] = fm3 * (547.0 * fm3 - 3882.0 * fm2 + 4642.0 * fm1 - 1854.0 * f0)
        + fm2 * (7043.0 * fm2 - 17246.0 * fm1 + 7042.0 * f0)
        + fm1 * (11003.0 * fm1 - 9402.0 * f0) + 2107.0 * f0 * f0;

  /* step 4: w_r = d_r / (SI_r + eps)^2, Eq. (weight); d_r per reading R1 */
  const double d[4] = {4.0 / 35.0, 18.0 / 35.0, 12.0 / 35.0, 1.0 / 35.0};
  double w[4], wsum = 0.0;
  for (int r = 0; r < 4; ++r) {
    w[r] = d[r] / ((si[r] + eps) * (si[r] + eps));
    wsum += w[r];
  }
  /* steps 5-6: normalised weights and the weighted combination, Eq. (fn_w_lin_comb) */
  double out = 0.0;
  for (int r = 0; r < 4; ++r) out += (w[r] / wsum) * f4[r];
  if (detail) {
    for (int r = 0; r < 4; ++r) {
      detail[r] = f4[r];
      detail[4 + r] = si[r];
      detail[8 + r] = w[r] / wsum;
    }
  }
  return out;
}

/* ---------------------------------------------------------------------------
 * Right-hand side of the semi-discrete system: for every real component q of
 * both species, dq/dt = -v dq/dz (discretised) + [-i[H, rho]]_q.
 * ------------------------------------------------------------------------- */
int oracle_rhs(const oracle_params* p, const double* u, double* k) {
  if (check(p)) return -1;
  const int64_t nz = p->nz;
  const int32_t nv = p->nv;
  const double h = p->L / (double)nz;
  double* vg = (double*)malloc(sizeof(double) * nv);
  double* wg = (double*)malloc(sizeof(double) * nv);
  oracle_vgrid_q(nv, p->vgrid, vg, wg);

#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < nz; ++z) {
    cplx* hm = (cplx*)malloc(sizeof(cplx) * 2 * nv * 4);
    build_h(p, u, z, vg, wg, hm);

    for (int s = 0; s < 2; ++s)
      for (int32_t j = 0; j < nv; ++j) {
        /* -i [H, rho] with 2x2 complex matrices, Eq. (eom) */
        const cplx* H = hm + (s * nv + j) * 4;
        const double a = u[idx(p, s, EE, z, j)], b = u[idx(p, s, XX, z, j)];
        const double cr = u[idx(p, s, EXR, z, j)], ci = u[idx(p, s, EXI, z, j)];
        const cplx R[4] = {a, cr + I * ci, cr - I * ci, b};
        cplx C[4];
        for (int r = 0; r < 2; ++r)
          for (int c = 0; c < 2; ++c) {
            cplx hr = 0.0, rh = 0.0;
            for (int m = 0; m < 2; ++m) {
              hr += H[r * 2 + m] * R[m * 2 + c];
              rh += R[r * 2 + m] * H[m * 2 + c];
            }
            C[r * 2 + c] = -I * (hr - rh);
          }
        const double comm[4] = {creal(C[0]), creal(C[3]), creal(C[1]), cimag(C[1])};

        for (int c = 0; c < 4; ++c) {
          double adv;
          if (p->scheme == 0 || p->scheme == 2) {
            /* Sec. 3.1: 4th-order central difference for d/dz */
            const double um2 = u[idx(p, s, c, wrap(z - 2, nz), j)];
            const double um1 = u[idx(p, s, c, wrap(z - 1, nz), j)];
            const double u0 = u[idx(p, s, c, z, j)];
            const double up1 = u[idx(p, s, c, wrap(z + 1, nz), j)];
            const double up2 = u[idx(p, s, c, wrap(z + 2, nz), j)];
            const double dudz = (um2 - 8.0 * um1 + 8.0 * up1 - up2) / (12.0 * h);
            double Qu;
            if (p->scheme == 0) {
              /* Kreiss-Oliger, r = 2: Q = eps (-1)^r h^(2r-1) (D+)^r (D-)^r / 2^(2r);
               * D+D- u_i = (u_{i+1} - 2u_i + u_{i-1}) / h^2 applied twice. */
              const double dd_m1 = (u0 - 2.0 * um1 + um2) / (h * h);
              const double dd_0 = (up1 - 2.0 * u0 + um1) / (h * h);
              const double dd_p1 = (up2 - 2.0 * up1 + u0) / (h * h);
              const double dddd = (dd_p1 - 2.0 * dd_0 + dd_m1) / (h * h);
              Qu = p->ko_eps * 1.0 /* (-1)^2 */ * (h * h * h) * dddd / 16.0;
            } else {
              /* Kreiss-Oliger, r = 3 (the general form of Sec. 3.1 with r = 3):
               * Q = eps (-1)^3 h^5 (D+)^3 (D-)^3 / 2^6; D+D- applied three times
               * to u_{z-3..z+3}, each pass shortening the row by one on each side. */
              double dd[7];
              for (int m = -3; m <= 3; ++m) dd[m + 3] = u[idx(p, s, c, wrap(z + m, nz), j)];
              for (int pass = 0, len = 7; pass < 3; ++pass, len -= 2)
                for (int i = 0; i + 2 < len; ++i)
                  dd[i] = (dd[i + 2] - 2.0 * dd[i + 1] + dd[i]) / (h * h);
              Qu = p->ko_eps * -1.0 /* (-1)^3 */ * (h * h * h * h * h) * dd[0] / 64.0;
            }
            /* d_t u + Q u = ... (reading R4) */
            adv = -vg[j] * dudz - Qu;
          } else {
            /* Eq. (cell_av): -(F_{i+1/2} - F_{i-1/2}) / dz with F = v u by WENO7 */
            double F[2];
            for (int side = 0; side < 2; ++side) {
              const int64_t i = z - 1 + side; /* interface i+1/2 for i = z-1, z */
              double f[7];
              for (int m = -3; m <= 3; ++m) {
                /* v > 0: left-biased stencil i-3..i+3; v < 0: mirror, f_{i+m} -> f_{i+1-m} (R3) */
                const int64_t src = vg[j] > 0.0 ? i + m : i + 1 - m;
                f[m + 3] = vg[j] * u[idx(p, s, c, wrap(src, nz), j)];
              }
              F[side] = oracle_weno7_face(f, p->weno_eps, NULL);
            }
            adv = -(F[1] - F[0]) / h;
          }
          k[idx(p, s, c, z, j)] = adv + comm[c];
        }
      }
    free(hm);
  }
  free(vg);
  free(wg);
  return 0;
}

/* Classic fourth-order Runge-Kutta (Sec. 1, Sec. 3):
 *   k1 = F(y), k2 = F(y + dt/2 k1), k3 = F(y + dt/2 k2), k4 = F(y + dt k3),
 *   y <- y + dt/6 (k1 + 2 k2 + 2 k3 + k4). */
int oracle_step(const oracle_params* p, double* y, int64_t nsteps) {
  if (check(p)) return -1;
  const int64_t n = 8 * p->nz * (int64_t)p->nv;
  const double dt = p->dt;
  double* k1 = (double*)malloc(sizeof(double) * n);
  double* k2 = (double*)malloc(sizeof(double) * n);
  double* k3 = (double*)malloc(sizeof(double) * n);
  double* k4 = (double*)malloc(sizeof(double) * n);
  double* t = (double*)malloc(sizeof(double) * n);
  if (!k1 || !k2 || !k3 || !k4 || !t) {
    free(k1); free(k2); free(k3); free(k4); free(t);
    return -2;
  }
  for (int64_t step = 0; step < nsteps; ++step) {
    oracle_rhs(p, y, k1);
    for (int64_t e = 0; e < n; ++e) t[e] = y[e] + 0.5 * dt * k1[e];
    oracle_rhs(p, t, k2);
    for (int64_t e = 0; e < n; ++e) t[e] = y[e] + 0.5 * dt * k2[e];
    oracle_rhs(p, t, k3);
    for (int64_t e = 0; e < n; ++e) t[e] = y[e] + dt * k3[e];
    oracle_rhs(p, t, k4);
    for (int64_t e = 0; e < n; ++e)
      y[e] = y[e] + (dt / 6.0) * (k1[e] + 2.0 * k2[e] + 2.0 * k3[e] + k4[e]);
  }
  free(k1); free(k2); free(k3); free(k4); free(t);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Diagnostics (Sec. 2: P0 and |P| of rho = (P0 + P.sigma)/2; Sec. 5: M0, delta P).
 * For a 2x2 density matrix d: P0 = d_ee + d_xx, P1 = 2 Re d_ex, P2 = -2 Im d_ex,
 * P3 = d_ee - d_xx.  M is sum_{z,v} w dz P(S - Sbar^*).
 * ------------------------------------------------------------------------- */
int oracle_conserved(const oracle_params* p, const double* u, double* out) {
  if (check(p)) return -1;
  const int64_t nz = p->nz;
  const int32_t nv = p->nv;
  const double h = p->L / (double)nz;
  double* vg = (double*)malloc(sizeof(double) * nv);
  double* wg = (double*)malloc(sizeof(double) * nv);
  oracle_vgrid_q(nv, p->vgrid, vg, wg);
  double tr[2] = {0, 0}, M[3] = {0, 0, 0}, dpmax = 0.0, dpnum = 0.0, dpden = 0.0;
  for (int64_t z = 0; z < nz; ++z)
    for (int32_t j = 0; j < nv; ++j) {
      double P[2][4];
      for (int s = 0; s < 2; ++s) {
        const double a = u[idx(p, s, EE, z, j)], b = u[idx(p, s, XX, z, j)];
        const double cr = u[idx(p, s, EXR, z, j)], ci = u[idx(p, s, EXI, z, j)];
        P[s][0] = a + b;
        P[s][1] = 2.0 * cr;
        P[s][2] = -2.0 * ci;
        P[s][3] = a - b;
        tr[s] += wg[j] * h * P[s][0];
        const double len = sqrt(P[s][1] * P[s][1] + P[s][2] * P[s][2] + P[s][3] * P[s][3]);
        if (P[s][0] > 0.0) {
          const double dp = fabs(len / P[s][0] - 1.0);
          if (dp > dpmax) dpmax = dp;
          if (s == NU) {
            dpnum += wg[j] * h * dp * P[s][0];
            dpden += wg[j] * h * P[s][0];
          }
        }
      }
      /* P of Sbar^*: conjugation flips the sign of Im, i.e. of P2 */
      M[0] += wg[j] * h * (P[0][1] - P[1][1]);
      M[1] += wg[j] * h * (P[0][2] + P[1][2]);
      M[2] += wg[j] * h * (P[0][3] - P[1][3]);
    }
  out[0] = tr[0];
  out[1] = tr[1];
  out[2] = M[0];
  out[3] = M[1];
  out[4] = M[2];
  out[5] = sin(2.0 * p->theta) * M[0] - cos(2.0 * p->theta) * M[2];
  out[6] = dpmax;
  out[7] = dpden > 0.0 ? dpnum / dpden : 0.0;
  out[8] = 0.0;
  out[9] = 0.0;
  free(vg);
  free(wg);
  return 0;
}

int oracle_moments(const oracle_params* p, const double* u, double* zavg, double* vmom) {
  if (check(p)) return -1;
  const int64_t nz = p->nz;
  const int32_t nv = p->nv;
  double* vg = (double*)malloc(sizeof(double) * nv);
  double* wg = (double*)malloc(sizeof(double) * nv);
  oracle_vgrid_q(nv, p->vgrid, vg, wg);
  if (zavg) {
    for (int s = 0; s < 2; ++s)
      for (int c = 0; c < 4; ++c)
        for (int32_t j = 0; j < nv; ++j) {
          double acc = 0.0;
          for (int64_t z = 0; z < nz; ++z) acc += u[idx(p, s, c, z, j)];
          zavg[(s * 4 + c) * nv + j] = acc / (double)nz;
        }
  }
  if (vmom) {
    for (int64_t z = 0; z < nz; ++z) {
      double m[6] = {0, 0, 0, 0, 0, 0};
      for (int32_t j = 0; j < nv; ++j) {
        const double d3 = (u[idx(p, NU, EE, z, j)] - u[idx(p, NU, XX, z, j)])
                        - (u[idx(p, NUBAR, EE, z, j)] - u[idx(p, NUBAR, XX, z, j)]);
        const double dr = u[idx(p, NU, EXR, z, j)] - u[idx(p, NUBAR, EXR, z, j)];
        const double di = u[idx(p, NU, EXI, z, j)] + u[idx(p, NUBAR, EXI, z, j)];
        m[0] += wg[j] * d3;
        m[1] += wg[j] * vg[j] * d3;
        m[2] += wg[j] * dr;
        m[3] += wg[j] * vg[j] * dr;
        m[4] += wg[j] * di;
        m[5] += wg[j] * vg[j] * di;
      }
      for (int e = 0; e < 6; ++e) vmom[z * 6 + e] = m[e];
    }
  }
  free(vg);
  free(wg);
  return 0;
}
