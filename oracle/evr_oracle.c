/*
 * evr_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Reinbacher, Graber, Pock, "Real-Time Intensity-Image Reconstruction for Event
 * Cameras Using Manifold Regularisation", BMVC 2016.  Each function below follows
 * one passage of the paper, in the paper's order and notation, with one loop per
 * step and no blocking or fusion, so that it can be checked against the paper by
 * eye.  Built with -O2 -ffp-contract=off (no fused multiply-add).
 *
 * The per-pixel loops of one step carry "omp parallel for": their iterations are
 * independent (each writes only its own pixel, reading the previous step's arrays),
 * so a build with -fopenmp computes the same bits on any number of threads; without
 * -fopenmp the pragmas are ignored.  Only the CPU-baseline timing uses that build.
 *
 * Readings taken where the paper is silent (all are parameters, shared with the
 * CUDA library by value, never by code):
 *  - t(x,y) is the time since the pixel's last event (Sec. 3.1), scaled by
 *    time_scale and clamped at t_max_us; never-fired pixels count from t_init.
 *  - L_x, L_y are forward differences whose last column/row is zero; L_g^* is
 *    the exact adjoint, written here as -div_g.
 *  - f is the previous reconstruction stepped by c1 or c2 once per event at the
 *    event's pixel (Eq. intensity_update); pixels without events keep the
 *    previous reconstruction (data_mode 0), or f persists (data_mode 1).
 *  - primal step first, then the dual step on 2u_{k+1}-u_k (Eq. cont_iterates),
 *    warm-started from the previous packet's (u, p).
 *  - optional: the L2 data term of Eq. 7 instead of the KL term, and anisotropic
 *    TV-L1 denoising of the time surface before the metric (Sec. 4).
 */
#include "evr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Discrete derivatives (Sec. 3.1 "Discrete Energy": L_x, L_y are first-order
 * finite differences after Chambolle 2004: forward difference, zero on the last
 * column for L_x and on the last row for L_y). */
void orc_grad(int W, int H, const double* a, double* ax, double* ay) {
#pragma omp parallel for
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      int i = y * W + x;
      ax[i] = (x < W - 1) ? a[i + 1] - a[i] : 0.0;
      ay[i] = (y < H - 1) ? a[i + W] - a[i] : 0.0;
    }
  }
}

/* Metric of the graph surface phi(x,y) = (x, y, t(x,y)) (Eqs. 1, 2):
 * phi_x = (1,0,t_x), phi_y = (0,1,t_y), g = [[1+t_x^2, t_x t_y],[t_x t_y, 1+t_y^2]],
 * G = det g = 1 + t_x^2 + t_y^2, with t_x = L_x t, t_y = L_y t (after Eq. 3). */
void orc_metric(int W, int H, const double* t, double* tx, double* ty, double* G) {
  orc_grad(W, H, t, tx, ty);
#pragma omp parallel for
  for (int i = 0; i < W * H; ++i) G[i] = 1.0 + tx[i] * tx[i] + ty[i] * ty[i];
}

/* Eq. 3: the three components of L_g u at each pixel, from L_x t, L_y t, L_x u,
 * L_y u and G. */
void orc_Lg(int W, int H, const double* tx, const double* ty, const double* G,
            const double* u, double* g1, double* g2, double* g3) {
  int n = W * H;
  double* ux = (double*)malloc(sizeof(double) * (size_t)n);
  double* uy = (double*)malloc(sizeof(double) * (size_t)n);
  orc_grad(W, H, u, ux, uy);
#pragma omp parallel for
  for (int i = 0; i < n; ++i) {
    double a = tx[i], b = ty[i];
    g1[i] = ((1.0 + b * b) * ux[i] - a * b * uy[i]) / G[i];
    g2[i] = ((1.0 + a * a) * uy[i] - a * b * ux[i]) / G[i];
    g3[i] = (a * ux[i] + b * uy[i]) / G[i];
  }
  free(ux);
  free(uy);
}

/* div_g p = -L_g^* p.  Eq. 3 writes L_g u = M (L_x u, L_y u) with the per-pixel
 * 3x2 matrix M = (1/G) [[1+t_y^2, -t_x t_y], [-t_x t_y, 1+t_x^2], [t_x, t_y]].
 * Hence <L_g u, p> = <(L_x u, L_y u), M^T p> = -<u, div(M^T p)>, where div is
 * the negative adjoint of the forward differences:
 *   (div q)(x,y) = q1(x,y)[x<W-1] - q1(x-1,y)[x>0] + q2(x,y)[y<H-1] - q2(x,y-1)[y>0]. */
void orc_divg(int W, int H, const double* tx, const double* ty, const double* G,
              const double* p1, const double* p2, const double* p3, double* out) {
  int n = W * H;
  double* q1 = (double*)malloc(sizeof(double) * (size_t)n);
  double* q2 = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp parallel for
  for (int i = 0; i < n; ++i) {
    double a = tx[i], b = ty[i];
    /* column 1 and column 2 of M, dotted with (p1, p2, p3) */
    q1[i] = ((1.0 + b * b) * p1[i] - a * b * p2[i] + a * p3[i]) / G[i];
    q2[i] = (-a * b * p1[i] + (1.0 + a * a) * p2[i] + b * p3[i]) / G[i];
  }
#pragma omp parallel for
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      int i = y * W + x;
      double d = 0.0;
      if (x < W - 1) d += q1[i];
      if (x > 0) d -= q1[i - 1];
      if (y < H - 1) d += q2[i];
      if (y > 0) d -= q2[i - W];
      out[i] = d;
    }
  }
  free(q1);
  free(q2);
}

/* Eq. update_rules, first line: the minimiser of (u - v)^2/(2 tau) +
 * tau-scaled KL term is the positive root 1/2 (v - beta + sqrt((v-beta)^2 + 4 beta f)),
 * beta = tau lambda sqrt(G), clamped to [u_min, u_max]. */
double orc_prox_kl(double v, double beta, double f, double u_min, double u_max) {
  double d = v - beta;
  double r = 0.5 * (d + sqrt(d * d + 4.0 * beta * f));
  if (r < u_min) r = u_min;
  if (r > u_max) r = u_max;
  return r;
}

/* Eq. update_rules, second line: p / max(1, ||p|| / sqrt(G)). */
void orc_project(double p1, double p2, double p3, double sqrtG, double* out3) {
  double nrm = sqrt(p1 * p1 + p2 * p2 + p3 * p3);
  double den = nrm / sqrtG;
  if (den < 1.0) den = 1.0;
  out3[0] = p1 / den;
  out3[1] = p2 / den;
  out3[2] = p3 / den;
}

/* Eq. 7 data term: (u - v)^2/(2 tau) + (lambda/2) sqrt(G)(u - f)^2 is minimal at
 * (v + beta f)/(1 + beta), beta = tau lambda sqrt(G). */
double orc_prox_l2(double v, double beta, double f) { return (v + beta * f) / (1.0 + beta); }

/* TV-L1 on the time surface (Sec. 4), anisotropic: min_s sum |L_x s| + |L_y s| +
 * lam sum |s - t0|, Chambolle-Pock with tau = sigma = 1/sqrt(8) (||grad||^2 <= 8):
 *   s_{k+1} = t0 + shrink(s_k + tau div q_k - t0, tau lam)
 *   q_{k+1} = clip(q_k + sigma grad(2 s_{k+1} - s_k), -1, 1)   (each component)
 * shrink(d, a) = sign(d) max(|d| - a, 0); div is the negative adjoint of grad. */
void orc_tvl1(int W, int H, const double* t0, int K, double lam, double* out) {
  int n = W * H;
  size_t bytes = sizeof(double) * (size_t)n;
  double st = 1.0 / sqrt(8.0);
  double* q1 = (double*)calloc((size_t)n, sizeof(double));
  double* q2 = (double*)calloc((size_t)n, sizeof(double));
  double* sb = (double*)malloc(bytes);
  double* gx = (double*)malloc(bytes);
  double* gy = (double*)malloc(bytes);
  memcpy(out, t0, bytes);
  for (int k = 0; k < K; ++k) {
    for (int y = 0; y < H; ++y) {
      for (int x = 0; x < W; ++x) {
        int i = y * W + x;
        double div = 0.0;
        if (x < W - 1) div += q1[i];
        if (x > 0) div -= q1[i - 1];
        if (y < H - 1) div += q2[i];
        if (y > 0) div -= q2[i - W];
        double d = out[i] + st * div - t0[i];
        double a = st * lam;
        double sh = (d > a) ? d - a : ((d < -a) ? d + a : 0.0);
        double s_new = t0[i] + sh;
        sb[i] = 2.0 * s_new - out[i];
        out[i] = s_new;
      }
    }
    orc_grad(W, H, sb, gx, gy);
    for (int i = 0; i < n; ++i) {
      double a = q1[i] + st * gx[i], b = q2[i] + st * gy[i];
      q1[i] = a > 1.0 ? 1.0 : (a < -1.0 ? -1.0 : a);
      q2[i] = b > 1.0 ? 1.0 : (b < -1.0 ? -1.0 : b);
    }
  }
  free(q1);
  free(q2);
  free(sb);
  free(gx);
  free(gy);
}

/* Eq. cont_iterates:
 *   u_{k+1} = prox_{tau D}(u_k - tau L_g^* p_k) = prox_{tau D}(u_k + tau div_g p_k)
 *   p_{k+1} = prox_{sigma R^*}(p_k + sigma L_g(2 u_{k+1} - u_k))
 * with the closed-form proximal maps of Eq. update_rules. */
void orc_pd_iterations(int W, int H, const double* tx, const double* ty, const double* G,
                       const double* f, double* u, double* p1, double* p2, double* p3,
                       int K, double tau, double sigma, double lambda,
                       double u_min, double u_max) {
  orc_pd_iterations_dt(W, H, tx, ty, G, f, u, p1, p2, p3, K, tau, sigma, lambda, u_min, u_max,
                       0);
}

void orc_pd_iterations_dt(int W, int H, const double* tx, const double* ty, const double* G,
                          const double* f, double* u, double* p1, double* p2, double* p3,
                          int K, double tau, double sigma, double lambda, double u_min,
                          double u_max, int data_term) {
  int n = W * H;
  size_t bytes = sizeof(double) * (size_t)n;
  double* dv = (double*)malloc(bytes);
  double* un = (double*)malloc(bytes);
  double* ub = (double*)malloc(bytes);
  double* g1 = (double*)malloc(bytes);
  double* g2 = (double*)malloc(bytes);
  double* g3 = (double*)malloc(bytes);
  for (int k = 0; k < K; ++k) {
    /* primal: argument u_k - tau L_g^* p_k */
    orc_divg(W, H, tx, ty, G, p1, p2, p3, dv);
#pragma omp parallel for
    for (int i = 0; i < n; ++i) {
      double v = u[i] + tau * dv[i];
      double beta = tau * lambda * sqrt(G[i]);
      un[i] = data_term ? orc_prox_l2(v, beta, f[i]) : orc_prox_kl(v, beta, f[i], u_min, u_max);
    }
    /* over-relaxation 2 u_{k+1} - u_k */
#pragma omp parallel for
    for (int i = 0; i < n; ++i) ub[i] = 2.0 * un[i] - u[i];
    /* dual: ascent on L_g of the extrapolated primal, then projection */
    orc_Lg(W, H, tx, ty, G, ub, g1, g2, g3);
#pragma omp parallel for
    for (int i = 0; i < n; ++i) {
      double out[3];
      orc_project(p1[i] + sigma * g1[i], p2[i] + sigma * g2[i], p3[i] + sigma * g3[i],
                  sqrt(G[i]), out);
      p1[i] = out[0];
      p2[i] = out[1];
      p3[i] = out[2];
    }
#pragma omp parallel for
    for (int i = 0; i < n; ++i) u[i] = un[i];
  }
  free(dv);
  free(un);
  free(ub);
  free(g1);
  free(g2);
  free(g3);
}

/* Reverse mode through Eq. cont_iterates.  One forward iteration maps (u, p) to
 *   d  = div_g p = div(M^T p)             (= -L_g^T p)
 *   v  = u + tau d
 *   r  = 1/2 (v - beta + sqrt((v - beta)^2 + 4 beta f)),  beta = tau lambda sqrt(G)
 *   u' = clamp(r, u_min, u_max)
 *   ub = 2 u' - u
 *   pt = p + sigma L_g ub
 *   p' = pt / max(1, |pt| / sqrt(G))
 * and the adjoint walks these steps backwards with the chain rule:
 *   a_pt = J_proj a_p'   (J = identity inside the ball, else
 *                         (sqrt G/|pt|)(I - pt pt^T/|pt|^2))
 *   a_p += a_pt;  a_ub = L_g^T (sigma a_pt) = -div_g(sigma a_pt)
 *   a_u' += 2 a_ub;  a_u = -a_ub
 *   a_r = a_u' [clamp inactive];  a_v = a_r dr/dv;  a_beta = a_r dr/dbeta;
 *   a_f += a_r dr/df;  a_lambda += a_beta tau sqrt(G)
 *   a_u += a_v;  a_p += -L_g (tau a_v)     (d = -L_g^T p)
 * with dr/dv = (1 + (v-beta)/s)/2, dr/dbeta = (-1 + (2f - v + beta)/s)/2,
 * dr/df = beta/s, s = sqrt((v-beta)^2 + 4 beta f). */
void orc_pd_grad(int W, int H, const double* tx, const double* ty, const double* G,
                 const double* f, const double* u0, const double* p0, int K, double tau,
                 double sigma, double lambda, double u_min, double u_max, const double* gu_K,
                 double* gu0, double* gp0, double* gf, double* glambda) {
  int n = W * H;
  size_t bytes = sizeof(double) * (size_t)n;
  /* tape: (u_k, p_k) for k = 0..K */
  double* tu = (double*)malloc(bytes * (size_t)(K + 1));
  double* tp = (double*)malloc(3 * bytes * (size_t)(K + 1));
  memcpy(tu, u0, bytes);
  memcpy(tp, p0, 3 * bytes);
  for (int k = 0; k < K; ++k) {
    memcpy(tu + (size_t)(k + 1) * n, tu + (size_t)k * n, bytes);
    memcpy(tp + (size_t)(k + 1) * 3 * n, tp + (size_t)k * 3 * n, 3 * bytes);
    double* pk = tp + (size_t)(k + 1) * 3 * n;
    orc_pd_iterations(W, H, tx, ty, G, f, tu + (size_t)(k + 1) * n, pk, pk + n, pk + 2 * n, 1,
                      tau, sigma, lambda, u_min, u_max);
  }
  double* au = (double*)malloc(bytes);
  double* ap = (double*)malloc(3 * bytes);
  double* d = (double*)malloc(bytes);
  double* v = (double*)malloc(bytes);
  double* un = (double*)malloc(bytes);
  double* ub = (double*)malloc(bytes);
  double* g = (double*)malloc(3 * bytes);
  double* apt = (double*)malloc(3 * bytes);
  double* aub = (double*)malloc(bytes);
  double* av = (double*)malloc(bytes);
  double* lv = (double*)malloc(3 * bytes);
  memcpy(au, gu_K, bytes);
  memset(ap, 0, 3 * bytes);
  memset(gf, 0, bytes);
  double gl = 0.0;
  for (int k = K - 1; k >= 0; --k) {
    const double* u = tu + (size_t)k * n;
    const double* p = tp + (size_t)k * 3 * n;
    /* recompute the iteration's intermediates */
    orc_divg(W, H, tx, ty, G, p, p + n, p + 2 * n, d);
    for (int i = 0; i < n; ++i) {
      v[i] = u[i] + tau * d[i];
      un[i] = orc_prox_kl(v[i], tau * lambda * sqrt(G[i]), f[i], u_min, u_max);
      ub[i] = 2.0 * un[i] - u[i];
    }
    orc_Lg(W, H, tx, ty, G, ub, g, g + n, g + 2 * n);
    /* dual step backwards */
    for (int i = 0; i < n; ++i) {
      double pt[3] = {p[i] + sigma * g[i], p[n + i] + sigma * g[n + i],
                      p[2 * n + i] + sigma * g[2 * n + i]};
      double nrm = sqrt(pt[0] * pt[0] + pt[1] * pt[1] + pt[2] * pt[2]);
      double sG = sqrt(G[i]);
      double a[3] = {ap[i], ap[n + i], ap[2 * n + i]};
      if (nrm > sG) {
        double dot = (pt[0] * a[0] + pt[1] * a[1] + pt[2] * a[2]) / (nrm * nrm);
        for (int c = 0; c < 3; ++c) a[c] = (sG / nrm) * (a[c] - pt[c] * dot);
      }
      for (int c = 0; c < 3; ++c) {
        apt[c * n + i] = a[c];
        ap[c * n + i] = a[c]; /* a_p (from pt = p + ...) */
        lv[c * n + i] = sigma * a[c];
      }
    }
    orc_divg(W, H, tx, ty, G, lv, lv + n, lv + 2 * n, aub); /* div_g(sigma a_pt) */
    for (int i = 0; i < n; ++i) aub[i] = -aub[i];            /* L_g^T = -div_g */
    /* over-relaxation and primal step backwards */
    for (int i = 0; i < n; ++i) {
      double aun = au[i] + 2.0 * aub[i];
      double anew_u = -aub[i];
      double beta = tau * lambda * sqrt(G[i]);
      double dd = v[i] - beta;
      double s = sqrt(dd * dd + 4.0 * beta * f[i]);
      double r = 0.5 * (dd + s);
      double ar = (r < u_min || r > u_max) ? 0.0 : aun;
      double drdv = 0.5 * (1.0 + dd / s);
      double drdb = 0.5 * (-1.0 + (2.0 * f[i] - v[i] + beta) / s);
      double drdf = beta / s;
      av[i] = ar * drdv;
      gf[i] += ar * drdf;
      gl += ar * drdb * tau * sqrt(G[i]);
      au[i] = anew_u + av[i];
      lv[i] = tau * av[i];
    }
    orc_Lg(W, H, tx, ty, G, lv, g, g + n, g + 2 * n); /* L_g(tau a_v) */
    for (int c = 0; c < 3; ++c)
      for (int i = 0; i < n; ++i) ap[c * n + i] -= g[c * n + i];
  }
  memcpy(gu0, au, bytes);
  memcpy(gp0, ap, 3 * bytes);
  *glambda = gl;
  free(tu);
  free(tp);
  free(au);
  free(ap);
  free(d);
  free(v);
  free(un);
  free(ub);
  free(g);
  free(apt);
  free(aub);
  free(av);
  free(lv);
}

/* Primal energy, Eq. 5: ||L_g u||_g + lambda sum (u - f log u) sqrt(G), with the
 * g-tensor norm ||A||_g = sum_ij sqrt(G_ij sum_l A_ijl^2).
 * Dual function of Eq. primal_dual_energy for feasible p (R^* = 0):
 *   min_{u in box} D(u,f) + <L_g u, p> = sum_ij min_{u in box} [a (u - f log u) - u div_g p],
 * a = lambda sqrt(G).  The per-pixel minimiser is clamp(a f / (a + w)) with
 * w = -div_g p when a + w > 0, and u_max otherwise (the objective then decreases). */
void orc_energy(int W, int H, const double* tx, const double* ty, const double* G,
                const double* f, const double* u, const double* p1, const double* p2,
                const double* p3, double lambda, double u_min, double u_max,
                double* primal, double* dual) {
  int n = W * H;
  size_t bytes = sizeof(double) * (size_t)n;
  if (primal) {
    double* g1 = (double*)malloc(bytes);
    double* g2 = (double*)malloc(bytes);
    double* g3 = (double*)malloc(bytes);
    orc_Lg(W, H, tx, ty, G, u, g1, g2, g3);
    double reg = 0.0, dat = 0.0;
    for (int i = 0; i < n; ++i) {
      reg += sqrt(G[i] * (g1[i] * g1[i] + g2[i] * g2[i] + g3[i] * g3[i]));
      double lg = (f[i] == 0.0) ? 0.0 : f[i] * log(u[i]);
      dat += (u[i] - lg) * sqrt(G[i]);
    }
    *primal = reg + lambda * dat;
    free(g1);
    free(g2);
    free(g3);
  }
  if (dual) {
    double* dv = (double*)malloc(bytes);
    orc_divg(W, H, tx, ty, G, p1, p2, p3, dv);
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      double a = lambda * sqrt(G[i]);
      double w = -dv[i];
      double us = (a + w > 0.0) ? a * f[i] / (a + w) : u_max;
      if (us < u_min) us = u_min;
      if (us > u_max) us = u_max;
      double lg = (f[i] == 0.0) ? 0.0 : f[i] * log(us);
      acc += a * (us - lg) + w * us;
    }
    *dual = acc;
    free(dv);
  }
}

void orc_energy_l2(int W, int H, const double* tx, const double* ty, const double* G,
                   const double* f, const double* u, const double* p1, const double* p2,
                   const double* p3, double lambda, double* primal, double* dual) {
  int n = W * H;
  size_t bytes = sizeof(double) * (size_t)n;
  if (primal) {
    double* g1 = (double*)malloc(bytes);
    double* g2 = (double*)malloc(bytes);
    double* g3 = (double*)malloc(bytes);
    orc_Lg(W, H, tx, ty, G, u, g1, g2, g3);
    double reg = 0.0, dat = 0.0;
    for (int i = 0; i < n; ++i) {
      reg += sqrt(G[i] * (g1[i] * g1[i] + g2[i] * g2[i] + g3[i] * g3[i]));
      dat += 0.5 * (u[i] - f[i]) * (u[i] - f[i]) * sqrt(G[i]);
    }
    *primal = reg + lambda * dat;
    free(g1);
    free(g2);
    free(g3);
  }
  if (dual) {
    double* dv = (double*)malloc(bytes);
    orc_divg(W, H, tx, ty, G, p1, p2, p3, dv);
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      double w = -dv[i];
      acc += w * f[i] - w * w / (2.0 * lambda * sqrt(G[i]));
    }
    *dual = acc;
    free(dv);
  }
}

/* ------------------------------------------------------------------------ */
/* Stream: the state carried from packet to packet. */
struct orc_stream {
  int W, H;
  orc_params prm;
  int64_t* t_last;  /* surface of active events: most recent timestamp per pixel */
  int32_t* n_pos;   /* positive events at the pixel since the last solve */
  int32_t* n_neg;   /* negative events at the pixel since the last solve */
  int64_t t_ref;    /* stream clock: the latest timestamp seen */
  int64_t t_init;
  int have_t_init;
  double *u, *p1, *p2, *p3, *f;
  double *tau, *tx, *ty, *G; /* last solve's time surface and metric */
};

static int prm_valid(const orc_params* p) {
  if (!(p->lambda > 0.0) || !(p->delta_pos > 0.0) || !(p->delta_neg > 0.0)) return 0;
  if (!(p->u_min > 0.0) || !(p->u_min < p->u_max)) return 0;
  if (!(p->u_init > 0.0)) return 0;
  if (!(p->tau > 0.0) || !(p->sigma > 0.0) || !(p->time_scale >= 0.0)) return 0;
  if (p->data_mode != 0 && p->data_mode != 1) return 0;
  if (p->data_term != 0 && p->data_term != 1) return 0;
  if (p->tvl1_iters < 0 || (p->tvl1_iters > 0 && !(p->tvl1_lambda > 0.0))) return 0;
  return 1;
}

orc_stream* orc_create(int W, int H, const orc_params* prm) {
  if (W <= 0 || H <= 0 || W > 65536 || H > 65536 || !prm || !prm_valid(prm)) return NULL;
  orc_stream* s = (orc_stream*)calloc(1, sizeof(orc_stream));
  if (!s) return NULL;
  size_t n = (size_t)W * (size_t)H;
  s->W = W;
  s->H = H;
  s->prm = *prm;
  s->t_last = (int64_t*)malloc(sizeof(int64_t) * n);
  s->n_pos = (int32_t*)calloc(n, sizeof(int32_t));
  s->n_neg = (int32_t*)calloc(n, sizeof(int32_t));
  double** planes[] = {&s->u, &s->p1, &s->p2, &s->p3, &s->f, &s->tau, &s->tx, &s->ty, &s->G};
  for (int k = 0; k < 9; ++k) *planes[k] = (double*)calloc(n, sizeof(double));
  if (!s->t_last || !s->n_pos || !s->n_neg || !s->G) {
    orc_destroy(s);
    return NULL;
  }
  s->have_t_init = prm->t_init_first ? 0 : 1;
  s->t_init = prm->t_init_first ? 0 : prm->t_init_us;
  s->t_ref = s->t_init;
  for (size_t i = 0; i < n; ++i) {
    s->t_last[i] = s->t_init;
    s->u[i] = prm->u_init;
    s->f[i] = prm->u_init;
    s->G[i] = 1.0;
  }
  return s;
}

void orc_destroy(orc_stream* s) {
  if (!s) return;
  free(s->t_last);
  free(s->n_pos);
  free(s->n_neg);
  free(s->u);
  free(s->p1);
  free(s->p2);
  free(s->p3);
  free(s->f);
  free(s->tau);
  free(s->tx);
  free(s->ty);
  free(s->G);
  free(s);
}

/* Events e^n = {x^n, y^n, theta^n, t^n}, theta in {-1, 1}, timestamps increasing
 * (Sec. 3, first paragraph; equal timestamps are accepted).  The surface of active
 * events records the most recent timestamp of each pixel (Sec. 3.1). */
int orc_push(orc_stream* s, const uint16_t* x, const uint16_t* y, const int64_t* t,
             const int8_t* pol, size_t n) {
  if (!s) return ORC_ERR_INVALID_ARG;
  if (n == 0) return ORC_OK;
  if (!x || !y || !t || !pol) return ORC_ERR_INVALID_ARG;
  /* validate the whole packet before touching the state */
  int have_clock = s->have_t_init;
  int64_t clock = s->t_ref;
  for (size_t i = 0; i < n; ++i) {
    if ((int)x[i] >= s->W || (int)y[i] >= s->H) return ORC_ERR_OUT_OF_RANGE;
    if (pol[i] == 0) return ORC_ERR_BAD_POLARITY;
    if (have_clock && t[i] < clock) return ORC_ERR_NONMONOTONIC;
    have_clock = 1;
    clock = t[i];
  }
  /* commit */
  if (!s->have_t_init) {
    s->t_init = t[0];
    s->t_ref = t[0];
    s->have_t_init = 1;
    for (int i = 0; i < s->W * s->H; ++i) s->t_last[i] = s->t_init;
  }
  for (size_t i = 0; i < n; ++i) {
    int k = (int)y[i] * s->W + (int)x[i];
    if (t[i] > s->t_last[k]) s->t_last[k] = t[i];
    if (pol[i] > 0)
      s->n_pos[k] += 1;
    else
      s->n_neg[k] += 1;
    if (t[i] > s->t_ref) s->t_ref = t[i];
  }
  return ORC_OK;
}

int orc_solve(orc_stream* s, int K) {
  if (!s || K < 0) return ORC_ERR_INVALID_ARG;
  const orc_params* pr = &s->prm;
  int n = s->W * s->H;
  /* time surface: time since the pixel's last event (Sec. 3.1), in manifold units */
  for (int i = 0; i < n; ++i) {
    if (!pr->manifold) {
      s->tau[i] = 0.0; /* t = const switches the manifold off (Sec. 4.2) */
      continue;
    }
    int64_t d = s->t_ref - s->t_last[i];
    if (pr->t_max_us > 0 && d > pr->t_max_us) d = pr->t_max_us;
    s->tau[i] = pr->time_scale * (double)d;
  }
  if (pr->tvl1_iters > 0) { /* denoise the surface first (Sec. 4) */
    double* t0 = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(t0, s->tau, sizeof(double) * (size_t)n);
    orc_tvl1(s->W, s->H, t0, pr->tvl1_iters, pr->tvl1_lambda, s->tau);
    free(t0);
  }
  orc_metric(s->W, s->H, s->tau, s->tx, s->ty, s->G);
  /* data image: Eq. intensity_update applied once per event, starting from the
   * previous reconstruction u^{n-1} (data_mode 0) or the previous f (data_mode 1);
   * c1 = exp(Delta+), c2 = exp(-Delta-). */
  double c1 = exp(pr->delta_pos), c2 = exp(-pr->delta_neg);
  for (int i = 0; i < n; ++i) {
    double v = (pr->data_mode == 0) ? s->u[i] : s->f[i];
    for (int e = 0; e < s->n_pos[i]; ++e) v = v * c1;
    for (int e = 0; e < s->n_neg[i]; ++e) v = v * c2;
    s->f[i] = v;
    s->n_pos[i] = 0;
    s->n_neg[i] = 0;
  }
  orc_pd_iterations_dt(s->W, s->H, s->tx, s->ty, s->G, s->f, s->u, s->p1, s->p2, s->p3, K,
                       pr->tau, pr->sigma, pr->lambda, pr->u_min, pr->u_max, pr->data_term);
  return ORC_OK;
}

static size_t plane_bytes(const orc_stream* s, int which) {
  size_t n = (size_t)s->W * (size_t)s->H;
  switch (which) {
    case ORC_U: case ORC_P1: case ORC_P2: case ORC_P3: case ORC_F: case ORC_TAU:
    case ORC_G: case ORC_TX: case ORC_TY:
      return n * sizeof(double);
    case ORC_TLAST: return n * sizeof(int64_t);
    case ORC_NPOS: case ORC_NNEG: return n * sizeof(int32_t);
    case ORC_TREF: case ORC_TINIT: return sizeof(int64_t);
    default: return 0;
  }
}

static void* plane_ptr(const orc_stream* s, int which) {
  switch (which) {
    case ORC_U: return s->u;
    case ORC_P1: return s->p1;
    case ORC_P2: return s->p2;
    case ORC_P3: return s->p3;
    case ORC_F: return s->f;
    case ORC_TAU: return s->tau;
    case ORC_G: return s->G;
    case ORC_TX: return s->tx;
    case ORC_TY: return s->ty;
    case ORC_TLAST: return s->t_last;
    case ORC_NPOS: return s->n_pos;
    case ORC_NNEG: return s->n_neg;
    case ORC_TREF: return (void*)&s->t_ref;
    case ORC_TINIT: return (void*)&s->t_init;
    default: return NULL;
  }
}

int orc_get(const orc_stream* s, int which, void* out) {
  if (!s || !out) return ORC_ERR_INVALID_ARG;
  size_t b = plane_bytes(s, which);
  if (!b) return ORC_ERR_INVALID_ARG;
  memcpy(out, plane_ptr(s, which), b);
  return ORC_OK;
}

int orc_set(orc_stream* s, int which, const void* in) {
  if (!s || !in) return ORC_ERR_INVALID_ARG;
  size_t b = plane_bytes(s, which);
  if (!b) return ORC_ERR_INVALID_ARG;
  memcpy(plane_ptr(s, which), in, b);
  if (which == ORC_TINIT) s->have_t_init = 1;
  return ORC_OK;
}

int orc_stream_energy(const orc_stream* s, double* primal, double* dual) {
  if (!s) return ORC_ERR_INVALID_ARG;
  if (s->prm.data_term)
    orc_energy_l2(s->W, s->H, s->tx, s->ty, s->G, s->f, s->u, s->p1, s->p2, s->p3,
                  s->prm.lambda, primal, dual);
  else
    orc_energy(s->W, s->H, s->tx, s->ty, s->G, s->f, s->u, s->p1, s->p2, s->p3,
               s->prm.lambda, s->prm.u_min, s->prm.u_max, primal, dual);
  return ORC_OK;
}
