/*
 * _sim.c -- inner loop of the synthetic event-camera simulator.
 *
 * Input generation only: renders moving texture layers at every pixel centre and
 * emits an event each time a pixel's log intensity crosses its reference level
 * by the contrast threshold C.  It contains none of the reconstruction method.
 *
 * Each layer is a wrap-padded (DH+1) x (DW+1) row-major texture on a toroidal
 * domain.  Pixel (x, y) at time t (seconds) samples layer l at
 *   q = R(omega_l t) ((x+0.5, y+0.5) - c) + c + v_l t - (0.5, 0.5),  c = (W/2, H/2),
 * bilinearly, wrapped into [0, DW) x [0, DH).  The sensor sees the sum of layers.
 */
#include <math.h>
#include <stdint.h>

typedef struct {
  double c, s, ox, oy;
} frame_pose;

/* Per-layer rotation and offset at time ts (seconds). */
static void poses(int W, int H, int nl, const double* vx, const double* vy,
                  const double* omega, double ts, frame_pose* out) {
  for (int l = 0; l < nl; ++l) {
    double th = omega[l] * ts;
    out[l].c = cos(th);
    out[l].s = sin(th);
    out[l].ox = W / 2.0 + vx[l] * ts - 0.5;
    out[l].oy = H / 2.0 + vy[l] * ts - 0.5;
  }
}

static double sample_px(int W, int H, int nl, const double* const* tex, const int* DW,
                        const int* DH, const frame_pose* fp, int x, int y) {
  double px = x + 0.5 - W / 2.0, py = y + 0.5 - H / 2.0;
  double acc = 0.0;
  for (int l = 0; l < nl; ++l) {
    double qx = fp[l].c * px - fp[l].s * py + fp[l].ox;
    double qy = fp[l].s * px + fp[l].c * py + fp[l].oy;
    qx -= DW[l] * floor(qx * (1.0 / DW[l]));
    qy -= DH[l] * floor(qy * (1.0 / DH[l]));
    int fx = (int)qx, fy = (int)qy;
    if (fx > DW[l] - 1) fx = DW[l] - 1;
    if (fy > DH[l] - 1) fy = DH[l] - 1;
    double ax = qx - fx, ay = qy - fy;
    const double* T = tex[l];
    int P = DW[l] + 1;
    double t0 = T[fy * P + fx] + ax * (T[fy * P + fx + 1] - T[fy * P + fx]);
    double t1 = T[(fy + 1) * P + fx] + ax * (T[(fy + 1) * P + fx + 1] - T[(fy + 1) * P + fx]);
    acc += t0 + ay * (t1 - t0);
  }
  return acc;
}

#define MAX_LAYERS 64

/* Sample the whole sensor at time t_us into out[W*H]. */
void evsim_sample(int W, int H, int nl, const double* const* tex, const int* DW,
                  const int* DH, const double* vx, const double* vy, const double* omega,
                  double t_us, double* out) {
  frame_pose fp[MAX_LAYERS];
  if (nl > MAX_LAYERS) return;
  poses(W, H, nl, vx, vy, omega, t_us * 1e-6, fp);
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) out[y * W + x] = sample_px(W, H, nl, tex, DW, DH, fp, x, y);
}

/*
 * Advance the simulation of sensor rows [y0, y1) frame by frame (step dt_us) from
 * *t_us while the next frame ends at or before t_stop_us, with per-pixel reference
 * levels ref[] and last samples Lprev[] (full-sensor arrays, updated in place for
 * the rows simulated).  Stops early when the next frame could exceed the output
 * capacity ((y1-y0)*W*max_per_px events per frame).  Event times are linear
 * interpolations of the crossing inside the step, floored to whole microseconds.
 * Returns the number of events written (>= 0), or -1 when one pixel crossed more
 * than max_per_px levels in a single frame (or there are more than MAX_LAYERS layers).
 */
int64_t evsim_run(int W, int H, int y0, int y1, int nl, const double* const* tex,
                  const int* DW, const int* DH, const double* vx, const double* vy,
                  const double* omega, double C, double dt_us, double t_stop_us, int64_t cap,
                  int max_per_px, double* ref, double* Lprev, double* t_us, uint16_t* ox,
                  uint16_t* oy, int64_t* ot, int8_t* op) {
  int64_t n = 0;
  int64_t npx = (int64_t)W * (y1 - y0);
  frame_pose fp[MAX_LAYERS];
  if (nl > MAX_LAYERS || y0 < 0 || y1 > H || y0 > y1) return -1;
  while (*t_us + dt_us <= t_stop_us && n + npx * max_per_px <= cap) {
    double ta = *t_us, tb = ta + dt_us;
    poses(W, H, nl, vx, vy, omega, tb * 1e-6, fp);
    for (int y = y0; y < y1; ++y) {
      for (int x = 0; x < W; ++x) {
        int i = y * W + x;
        double Lb = sample_px(W, H, nl, tex, DW, DH, fp, x, y);
        double La = Lprev[i];
        double d = Lb - ref[i];
        int sign = 0;
        int cnt = 0;
        if (d >= C) {
          sign = 1;
          cnt = (int)floor(d / C);
        } else if (-d >= C) {
          sign = -1;
          cnt = (int)floor(-d / C);
        }
        if (cnt > max_per_px) return -1;
        for (int k = 1; k <= cnt; ++k) {
          double level = ref[i] + sign * k * C;
          double den = Lb - La;
          double alpha = (den != 0.0) ? (level - La) / den : 1.0;
          if (alpha < 0.0) alpha = 0.0;
          if (alpha > 1.0) alpha = 1.0;
          ox[n] = (uint16_t)x;
          oy[n] = (uint16_t)y;
          ot[n] = (int64_t)floor(ta + alpha * dt_us);
          op[n] = (int8_t)sign;
          ++n;
        }
        ref[i] += sign * cnt * C;
        Lprev[i] = Lb;
      }
    }
    *t_us = tb;
  }
  return n;
}
