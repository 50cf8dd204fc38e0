/*
 * Input synthesis for the density-fitting hot path: the two- and three-centre
 * Coulomb integrals over normalised s-type Gaussian primitives that the DF
 * tensor is built from (Section 2.1, Eqs. df and cderi take them as given).
 *
 * This file is part of the seeded input generator, not of the method: the
 * hot path (split, slice GEMMs, rho/J, energies) starts from the DF tensor B.
 * It is plain C with an OpenMP loop over the auxiliary index so that the
 * 120- and 240-atom molecules can be generated in seconds.
 *
 *   (c|ab) = N_c N_a N_b K_ab 2 pi^{5/2} / (g p sqrt(g+p)) F0(g p/(g+p) |C-P|^2)
 *   (c|d)  = N_c N_d 2 pi^{5/2} / (g d sqrt(g+d)) F0(g d/(g+d) |C-D|^2)
 * with p = a+b, P = (aA+bB)/p, K_ab = exp(-ab/p |A-B|^2), N(a) = (2a/pi)^{3/4}
 * and F0(T) = sqrt(pi/T) erf(sqrt T)/2 (series 1 - T/3 + T^2/10 below 1e-10).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>

static const double kPi = 3.14159265358979323846;

static double boys0(double t) {
  if (t < 1e-10) return 1.0 - t / 3.0 + t * t / 10.0;
  double r = sqrt(t);
  return 0.5 * sqrt(kPi / t) * erf(r);
}

static double norm_s(double a) { return pow(2.0 * a / kPi, 0.75); }

/* out[P][mu][nu], row-major, for nao AO and naux auxiliary primitives.
 * The Gaussian-product quantities of every AO pair are formed once; the loop
 * over P then only evaluates the Boys factor. */
void gen_int3c(int nao, int naux, const double *ao_xyz, const double *ao_exp,
               const double *aux_xyz, const double *aux_exp, double *out) {
  const double two_pi52 = 2.0 * pow(kPi, 2.5);
  const size_t npair = (size_t)nao * (nao + 1) / 2;
  double *pp = (double *)malloc(sizeof(double) * npair * 5);
  int *pm = (int *)malloc(sizeof(int) * npair * 2);
  size_t q = 0;
  for (int m = 0; m < nao; ++m) {
    const double a = ao_exp[m];
    const double ax = ao_xyz[3 * m], ay = ao_xyz[3 * m + 1], az = ao_xyz[3 * m + 2];
    for (int n = 0; n <= m; ++n, ++q) {
      const double b = ao_exp[n];
      const double bx = ao_xyz[3 * n], by = ao_xyz[3 * n + 1], bz = ao_xyz[3 * n + 2];
      const double p = a + b;
      const double dx = ax - bx, dy = ay - by, dz = az - bz;
      const double kab = exp(-a * b / p * (dx * dx + dy * dy + dz * dz));
      pp[5 * q + 0] = p;
      pp[5 * q + 1] = (a * ax + b * bx) / p;
      pp[5 * q + 2] = (a * ay + b * by) / p;
      pp[5 * q + 3] = (a * az + b * bz) / p;
      pp[5 * q + 4] = norm_s(a) * norm_s(b) * kab;
      pm[2 * q] = m;
      pm[2 * q + 1] = n;
    }
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int P = 0; P < naux; ++P) {
    const double g = aux_exp[P];
    const double cx = aux_xyz[3 * P], cy = aux_xyz[3 * P + 1], cz = aux_xyz[3 * P + 2];
    const double nc = norm_s(g);
    double *row = out + (size_t)P * nao * nao;
    for (size_t k = 0; k < npair; ++k) {
      const double *e = pp + 5 * k;
      const double p = e[0];
      const double ex = e[1] - cx, ey = e[2] - cy, ez = e[3] - cz;
      const double t = g * p / (g + p) * (ex * ex + ey * ey + ez * ez);
      const double v = nc * e[4] * two_pi52 / (g * p * sqrt(g + p)) * boys0(t);
      const int m = pm[2 * k], n = pm[2 * k + 1];
      row[(size_t)m * nao + n] = v;
      row[(size_t)n * nao + m] = v;
    }
  }
  free(pp);
  free(pm);
}

/* out[P][Q], the Coulomb metric of the auxiliary primitives. */
void gen_metric(int naux, const double *aux_xyz, const double *aux_exp, double *out) {
  const double two_pi52 = 2.0 * pow(kPi, 2.5);
#pragma omp parallel for schedule(dynamic, 4)
  for (int P = 0; P < naux; ++P) {
    const double g = aux_exp[P];
    for (int Q = 0; Q <= P; ++Q) {
      const double d = aux_exp[Q];
      const double dx = aux_xyz[3 * P] - aux_xyz[3 * Q];
      const double dy = aux_xyz[3 * P + 1] - aux_xyz[3 * Q + 1];
      const double dz = aux_xyz[3 * P + 2] - aux_xyz[3 * Q + 2];
      const double t = g * d / (g + d) * (dx * dx + dy * dy + dz * dz);
      const double v = norm_s(g) * norm_s(d) * two_pi52 / (g * d * sqrt(g + d)) * boys0(t);
      out[(size_t)P * naux + Q] = v;
      out[(size_t)Q * naux + P] = v;
    }
  }
}

/* One-electron integrals over the AO primitives, for an SCF loop around the
 * build: overlap S, kinetic energy T and attraction V to nuclei of charge
 * Z[C] at nuc_xyz[C] (all [nao][nao], row-major):
 *   S_ab = N_a N_b (pi/p)^{3/2} K_ab
 *   T_ab = (ab/p) (3 - 2 (ab/p) |A-B|^2) S_ab
 *   V_ab = -sum_C Z_C N_a N_b (2 pi/p) K_ab F0(p |P-C|^2)                  */
void gen_oneel(int nao, const double *ao_xyz, const double *ao_exp, int nnuc, const double *nuc_xyz,
               const double *Z, double *S, double *T, double *V) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int a = 0; a < nao; ++a) {
    const double ea = ao_exp[a];
    for (int b = 0; b <= a; ++b) {
      const double eb = ao_exp[b];
      const double p = ea + eb, mu = ea * eb / p;
      const double dx = ao_xyz[3 * a] - ao_xyz[3 * b];
      const double dy = ao_xyz[3 * a + 1] - ao_xyz[3 * b + 1];
      const double dz = ao_xyz[3 * a + 2] - ao_xyz[3 * b + 2];
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double nk = norm_s(ea) * norm_s(eb) * exp(-mu * r2);
      const double s = nk * pow(kPi / p, 1.5);
      const double t = mu * (3.0 - 2.0 * mu * r2) * s;
      const double px = (ea * ao_xyz[3 * a] + eb * ao_xyz[3 * b]) / p;
      const double py = (ea * ao_xyz[3 * a + 1] + eb * ao_xyz[3 * b + 1]) / p;
      const double pz = (ea * ao_xyz[3 * a + 2] + eb * ao_xyz[3 * b + 2]) / p;
      double v = 0.0;
      for (int c = 0; c < nnuc; ++c) {
        const double cx = px - nuc_xyz[3 * c], cy = py - nuc_xyz[3 * c + 1], cz = pz - nuc_xyz[3 * c + 2];
        v -= Z[c] * boys0(p * (cx * cx + cy * cy + cz * cz));
      }
      v *= nk * 2.0 * kPi / p;
      S[(size_t)a * nao + b] = S[(size_t)b * nao + a] = s;
      T[(size_t)a * nao + b] = T[(size_t)b * nao + a] = t;
      V[(size_t)a * nao + b] = V[(size_t)b * nao + a] = v;
    }
  }
}
