/*
 * evr_oracle.h -- plain FP64 CPU oracle for event-camera intensity reconstruction
 * on the event manifold (Reinbacher, Graber, Pock, BMVC 2016, arXiv:1607.06283).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle is what the CUDA library is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA path (paper_1607_06283_gb300/csrc, include/evr.h), and it never calls it.
 *
 * Every floating-point quantity is double precision; integer state (timestamps,
 * event counts) stays integer.  Arrays are dense row-major H x W with index
 * y*W + x, x the column and y the row (the paper's (i,j) on an M x M grid,
 * Sec. 3.1 "Discrete Energy", generalised to W x H).
 *
 * Functions return 0 on success or one of the negative ORC_ERR_* codes.
 */
#ifndef EVR_ORACLE_H
#define EVR_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG (-1)
#define ORC_ERR_OUT_OF_RANGE (-2)
#define ORC_ERR_BAD_POLARITY (-3)
#define ORC_ERR_NONMONOTONIC (-4)
#define ORC_ERR_OOM (-5)

/* Model and solver parameters (Sec. 3, Eqs. 5, intensity update, update rules). */
typedef struct {
  double lambda;      /* data weight lambda of Eq. 5 */
  double delta_pos;   /* Delta+ : log-intensity step of a positive event (Sec. 3) */
  double delta_neg;   /* Delta- : log-intensity step of a negative event (Sec. 3) */
  double u_min;       /* box [u_min, u_max] of the data term (Eq. data_term) */
  double u_max;
  double u_init;      /* u^0, the initial image */
  double tau;         /* primal step tau (Sec. 3.2) */
  double sigma;       /* dual step sigma (Sec. 3.2) */
  double time_scale;  /* manifold height units per microsecond */
  int64_t t_max_us;   /* clamp of the time since the last event; <= 0 disables */
  int64_t t_init_us;  /* timestamp of never-fired pixels (used if t_init_first == 0) */
  int t_init_first;   /* 1: never-fired pixels take the first pushed timestamp */
  int data_mode;      /* 0: f = previous u stepped at event pixels; 1: persistent f */
  int manifold;       /* 1: t from the events; 0: t = const (manifold switched off) */
  int data_term;      /* 0: generalised KL with box (Eq. data_term); 1: L2 / ROF (Eq. 7) */
  int tvl1_iters;     /* TV-L1 iterations on the time surface before the metric; 0 = off */
  double tvl1_lambda; /* data weight of that TV-L1 denoising */
} orc_params;

/* ---- stateless operators (each cites the passage it implements) ---- */

/* Forward differences with a zero last row/column (Sec. 3.1, "simple first order
 * finite difference approximations", cited to Chambolle 2004). */
void orc_grad(int W, int H, const double* a, double* ax, double* ay);

/* Metric of the surface t(x,y): tx = L_x t, ty = L_y t, G = 1 + tx^2 + ty^2
 * (Eq. 2 and the text after Eq. 3). */
void orc_metric(int W, int H, const double* t, double* tx, double* ty, double* G);

/* Discrete manifold gradient L_g u, three output planes (Eq. 3). */
void orc_Lg(int W, int H, const double* tx, const double* ty, const double* G,
            const double* u, double* g1, double* g2, double* g3);

/* div_g p = -L_g^* p, the negative adjoint of L_g (Eq. cont_iterates uses L_g^*). */
void orc_divg(int W, int H, const double* tx, const double* ty, const double* G,
              const double* p1, const double* p2, const double* p3, double* out);

/* Closed-form KL proximal root with clamping (Eq. update_rules, first line). */
double orc_prox_kl(double v, double beta, double f, double u_min, double u_max);

/* Proximal map of the L2 data term of Eq. 7 (ROF on the manifold): the minimiser of
 * (u - v)^2/(2 tau) + (lambda/2) sqrt(G) (u - f)^2 is (v + beta f)/(1 + beta),
 * beta = tau lambda sqrt(G); no box constraint. */
double orc_prox_l2(double v, double beta, double f);

/* TV-L1 denoising of the time surface (Sec. 4: a few iterations of a TV-L1 method
 * before the surface is used): min_s sum |L_x s| + |L_y s| + lam sum |s - t0|
 * (anisotropic TV), K Chambolle-Pock iterations from s = t0, q = 0 with steps
 * 1/sqrt(8).  out[W*H] receives s. */
void orc_tvl1(int W, int H, const double* t0, int K, double lam, double* out);

/* Projection onto the metric ball ||p|| <= sqrt(G) (Eq. update_rules, second line). */
void orc_project(double p1, double p2, double p3, double sqrtG, double* out3);

/* K primal-dual iterations (Eq. cont_iterates with the update rules), in place on
 * u, p1, p2, p3.  beta = tau * lambda * sqrt(G). */
void orc_pd_iterations(int W, int H, const double* tx, const double* ty, const double* G,
                       const double* f, double* u, double* p1, double* p2, double* p3,
                       int K, double tau, double sigma, double lambda,
                       double u_min, double u_max);

/* As orc_pd_iterations with the data term chosen by data_term (0 KL with box, 1 L2). */
void orc_pd_iterations_dt(int W, int H, const double* tx, const double* ty, const double* G,
                          const double* f, double* u, double* p1, double* p2, double* p3,
                          int K, double tau, double sigma, double lambda, double u_min,
                          double u_max, int data_term);

/* Primal energy of Eq. 5 and the dual function of the saddle form (Eq.
 * primal_dual_energy) at a feasible p.  Either output pointer may be NULL. */
void orc_energy(int W, int H, const double* tx, const double* ty, const double* G,
                const double* f, const double* u, const double* p1, const double* p2,
                const double* p3, double lambda, double u_min, double u_max,
                double* primal, double* dual);

/* Energy and dual value for the L2 data term of Eq. 7: primal ||L_g u||_g +
 * (lambda/2) sum sqrt(G)(u - f)^2; dual sum min_u (lambda/2) sqrt(G)(u - f)^2 + w u =
 * sum w f - w^2 / (2 lambda sqrt(G)), w = -div_g p. */
void orc_energy_l2(int W, int H, const double* tx, const double* ty, const double* G,
                   const double* f, const double* u, const double* p1, const double* p2,
                   const double* p3, double lambda, double* primal, double* dual);

/* Reverse-mode derivative of orc_pd_iterations (K iterations from (u0, p0) with
 * fixed metric and f) for a loss L with given dL/du_K (gu_K[W*H]).  Outputs:
 * gu0[W*H] = dL/du0, gp0[3*W*H] = dL/dp0 (planes p1, p2, p3), gf[W*H] = dL/df,
 * *glambda = dL/dlambda.  Clamped pixels and the projection's kink are
 * differentiated on their active side (derivative 0 through an active clamp).
 * Every intermediate (u, p) is kept (plain full tape). */
void orc_pd_grad(int W, int H, const double* tx, const double* ty, const double* G,
                 const double* f, const double* u0, const double* p0, int K, double tau,
                 double sigma, double lambda, double u_min, double u_max, const double* gu_K,
                 double* gu0, double* gp0, double* gf, double* glambda);

/* ---- a stream: events in, one image per packet out ---- */
typedef struct orc_stream orc_stream;

orc_stream* orc_create(int W, int H, const orc_params* prm);
void orc_destroy(orc_stream* s);

/* Validate a whole packet of events, then integrate it (Sec. 3, event definition
 * and Eq. intensity_update; surface of active events, Sec. 3.1).  A rejected
 * packet leaves the state unchanged; the code is that of the first bad event. */
int orc_push(orc_stream* s, const uint16_t* x, const uint16_t* y, const int64_t* t,
             const int8_t* pol, size_t n);

/* Per-packet solve: time surface, metric, data image f, then K iterations. */
int orc_solve(orc_stream* s, int K);

/* State planes that can be read or (for teacher-forced checks) written. */
#define ORC_U 0        /* double[W*H] */
#define ORC_P1 1       /* double[W*H] */
#define ORC_P2 2
#define ORC_P3 3
#define ORC_F 4        /* double[W*H], f of the last solve */
#define ORC_TAU 5      /* double[W*H], time surface of the last solve */
#define ORC_G 6        /* double[W*H], G of the last solve */
#define ORC_TLAST 7    /* int64[W*H], never-fired pixels hold t_init */
#define ORC_NPOS 8     /* int32[W*H] */
#define ORC_NNEG 9     /* int32[W*H] */
#define ORC_TREF 10    /* int64[1] */
#define ORC_TINIT 11   /* int64[1] */
#define ORC_TX 12      /* double[W*H], L_x t of the last solve */
#define ORC_TY 13      /* double[W*H], L_y t of the last solve */
int orc_get(const orc_stream* s, int which, void* out);
int orc_set(orc_stream* s, int which, const void* in);

/* Energy and dual value of the current (u, p) under the last solve's metric and f. */
int orc_stream_energy(const orc_stream* s, double* primal, double* dual);

#ifdef __cplusplus
}
#endif
#endif
