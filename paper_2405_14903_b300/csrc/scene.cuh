// Analytic solid geometry on the device (Sec. 2.2; Sec. 2.3.1, Projection;
// Sec. 2.3.3). phi > 0 in the fluid; unions of fluid pieces take the max.
// Every SDF here is 1-Lipschitz, which the rasteriser's early exit relies on.
#pragma once

#include "nf_internal.cuh"

namespace nf {

template <class R>
__device__ __forceinline__ R box_sdf(R px, R py, R pz, R hx, R hy, R hz) {
  R qx = fabs(px) - hx, qy = fabs(py) - hy, qz = fabs(pz) - hz;
  R mx = fmax(qx, R(0)), my = fmax(qy, R(0)), mz = fmax(qz, R(0));
  R out = sqrt(mx * mx + my * my + mz * mz);
  R in = fmin(fmax(qx, fmax(qy, qz)), R(0));
  return out + in;
}

// Gradient of box_sdf with respect to p.
__device__ __forceinline__ void box_sdf_grad(double px, double py, double pz,
                                             double hx, double hy, double hz,
                                             double &gx, double &gy,
                                             double &gz) {
  double qx = fabs(px) - hx, qy = fabs(py) - hy, qz = fabs(pz) - hz;
  double sx = px >= 0 ? 1.0 : -1.0, sy = py >= 0 ? 1.0 : -1.0,
         sz = pz >= 0 ? 1.0 : -1.0;
  double mx = fmax(qx, 0.0), my = fmax(qy, 0.0), mz = fmax(qz, 0.0);
  double n = sqrt(mx * mx + my * my + mz * mz);
  if (n > 0.0) {
    gx = sx * mx / n;
    gy = sy * my / n;
    gz = sz * mz / n;
    return;
  }
  gx = gy = gz = 0.0;
  if (qx >= qy && qx >= qz)
    gx = sx;
  else if (qy >= qz)
    gy = sy;
  else
    gz = sz;
}

// sqrt(v) to near FP64 accuracy from the FP32 root and one Newton step in
// FP64 (a few FP64 multiply-adds instead of the FP64 square root, which is
// slow on a part whose FP64 rate is 1/64 of FP32). v >= 0.
__device__ __forceinline__ double fsqrt_refined(double v) {
  const float r0 = sqrtf((float)v);
  if (!(r0 > 0.f)) return 0.0;
  const double r = (double)r0;
  return r + (v - r * r) * (double)(0.5f / r0);
}

// The same gradient in FP32 (the narrow-band sub-samples of the FP32 path).
__device__ __forceinline__ void box_sdf_grad_f(float px, float py, float pz, float hx,
                                               float hy, float hz, float &gx, float &gy,
                                               float &gz) {
  const float qx = fabsf(px) - hx, qy = fabsf(py) - hy, qz = fabsf(pz) - hz;
  const float sx = px >= 0.f ? 1.f : -1.f, sy = py >= 0.f ? 1.f : -1.f,
              sz = pz >= 0.f ? 1.f : -1.f;
  const float mx = fmaxf(qx, 0.f), my = fmaxf(qy, 0.f), mz = fmaxf(qz, 0.f);
  const float n = sqrtf(mx * mx + my * my + mz * mz);
  if (n > 0.f) {
    gx = sx * mx / n;
    gy = sy * my / n;
    gz = sz * mz / n;
    return;
  }
  gx = gy = gz = 0.f;
  if (qx >= qy && qx >= qz)
    gx = sx;
  else if (qy >= qz)
    gy = sy;
  else
    gz = sz;
}

// A scene parameter in the evaluator's precision R: the FP32 mirror for
// float, the double itself otherwise.
template <class R>
__device__ __forceinline__ R P(double d, float f) {
  if constexpr (sizeof(R) == 4)
    return f;
  else
    return d;
}

// ------------------------------------------ extruded polar-Bezier shapes ----
// App. A: a closed 2D curve of N cubic Bezier segments around a centre c;
// segment i spans the polar angles [2 pi i / N, 2 pi (i + 1) / N], its inner
// control points sit at the radii rho1_i, rho2_i at 2 pi / (3N) in from each
// end of that range, and the shared endpoints are the midpoints of the two
// control points around them (G1 continuity). A 3D shape extrudes the
// cross-section along its local z between z0 and z1; the n key sections
// (evenly spaced in u = (z - z0) / (z1 - z0)) are interpolated by the
// polynomial through them (the inverse Vandermonde coefficients are formed
// on the host), applied to the centre and every radius. The distance to a
// cross-section is the distance to the closest point of the curve, found per
// segment from the nearest of 24 evenly spaced parameters by 5 Newton steps
// on (B - x) . B' = 0; its side comes from the outward normal there. The
// slab z0 <= z <= z1 caps it, and shapes combine by CSG union (the minimum
// of the outside-positive distances). Sec. 2.2.
//
// Table (FP64, one block per shape at bz_off[s]):
//   [0] n keys, [1] N segments, [2] z0, [3] z1, [4] has frame,
//   [5..7] frame origin, [8..16] frame axes (row r: local axis r in world
//   coordinates), [17..32] coeff[m][k] (4 x 4: W_k = sum_m u^m coeff[m][k]),
//   [33 .. 33 + 4N) per segment cos a0, sin a0, cos a1, sin a1,
//   then per key: centre (2), radii rho1_0, rho2_0, rho1_1, ... (2N).
constexpr int kBzHead = 33;

struct BzHit {
  double out;          // capped outside-positive distance
  double d, w;         // cross-section signed distance, slab term
  double dist;         // unsigned distance to the curve
  double nv[2];        // unit vector from the closest point to the point
  double sb;           // closest parameter
  double W[kBzMaxKeys];
  double X[3];         // the point in the shape's frame
  int seg, n, N;
  bool inside;
};

__device__ __forceinline__ void bz_bern(double s, double b[4]) {
  const double u = 1.0 - s;
  b[0] = u * u * u;
  b[1] = 3.0 * u * u * s;
  b[2] = 3.0 * u * s * s;
  b[3] = s * s * s;
}

// radius j (0 .. 2N-1, wrapped) of the cross-section with weights W
__device__ __forceinline__ double bz_radius(const double *kb, int n, int N, const double *W,
                                            double scale, int j) {
  j = (j + 2 * N) % (2 * N);
  double r = 0.0;
  for (int k = 0; k < n; ++k) r += W[k] * (scale * kb[k * (2 + 2 * N) + 2 + j]);
  return r;
}

// control polygon of segment i (e0, p0, p1, e1) of the cross-section
__device__ __forceinline__ void bz_polygon(const double *t, const double *kb, int n, int N,
                                           const double *W, const double c[2], double scale,
                                           int i, double P[4][2]) {
  const int im = (i + N - 1) % N, ip = (i + 1) % N;
  const double *tr = t + kBzHead;
  const double r1 = bz_radius(kb, n, N, W, scale, 2 * i);
  const double r2 = bz_radius(kb, n, N, W, scale, 2 * i + 1);
  const double r2m = bz_radius(kb, n, N, W, scale, 2 * im + 1);
  const double r1p = bz_radius(kb, n, N, W, scale, 2 * ip);
  const double p0x = c[0] + r1 * tr[4 * i], p0y = c[1] + r1 * tr[4 * i + 1];
  const double p1x = c[0] + r2 * tr[4 * i + 2], p1y = c[1] + r2 * tr[4 * i + 3];
  const double q1x = c[0] + r2m * tr[4 * im + 2], q1y = c[1] + r2m * tr[4 * im + 3];
  const double q0x = c[0] + r1p * tr[4 * ip], q0y = c[1] + r1p * tr[4 * ip + 1];
  P[0][0] = 0.5 * (q1x + p0x);
  P[0][1] = 0.5 * (q1y + p0y);
  P[1][0] = p0x;
  P[1][1] = p0y;
  P[2][0] = p1x;
  P[2][1] = p1y;
  P[3][0] = 0.5 * (p1x + q0x);
  P[3][1] = 0.5 * (p1y + q0y);
}

// Point of shape sh at its local position; Lagrange weights and centre.
__device__ __forceinline__ void bz_frame(const SceneDev &s, int sh, double x, double y, double z,
                                         BzHit &h, double c[2]) {
  const double *t = s.bz + s.bz_off[sh];
  const int n = (int)t[0], N = (int)t[1];
  h.n = n;
  h.N = N;
  if (t[4] != 0.0) {
    const double a = x - t[5], b = y - t[6], e = z - t[7];
    for (int r = 0; r < 3; ++r) h.X[r] = a * t[8 + 3 * r] + b * t[9 + 3 * r] + e * t[10 + 3 * r];
  } else {
    h.X[0] = x;
    h.X[1] = y;
    h.X[2] = z;
  }
  const double z0 = t[2], z1 = t[3];
  const double u = fmin(fmax((h.X[2] - z0) / (z1 - z0), 0.0), 1.0);
  double pw[kBzMaxKeys];
  pw[0] = 1.0;
  for (int m = 1; m < kBzMaxKeys; ++m) pw[m] = pw[m - 1] * u;
  for (int k = 0; k < kBzMaxKeys; ++k) {
    double w = 0.0;
    for (int m = 0; m < n; ++m) w += pw[m] * t[17 + 4 * m + k];
    h.W[k] = k < n ? w : 0.0;
  }
  const double *kb = t + kBzHead + 4 * N;
  c[0] = c[1] = 0.0;
  for (int k = 0; k < n; ++k) {
    c[0] += h.W[k] * kb[k * (2 + 2 * N)];
    c[1] += h.W[k] * kb[k * (2 + 2 * N) + 1];
  }
}

// Outside-positive distance of (x, y, z) to shape sh, with what the
// gradient needs.
__device__ inline void bz_shape(const SceneDev &s, int sh, double x, double y, double z,
                                BzHit &h) {
  double c[2];
  bz_frame(s, sh, x, y, z, h, c);
  const double *t = s.bz + s.bz_off[sh];
  const int n = h.n, N = h.N;
  const double *kb = t + kBzHead + 4 * N;
  const double scale = (s.bz_mode == kBzPulse && sh == s.bz_pulse) ? s.bz_k : 1.0;
  const double X0 = h.X[0], X1 = h.X[1];
  double best = 1.0e300, bs = 0.0;
  int bi = 0;
  for (int i = 0; i < N; ++i) {
    double P[4][2];
    bz_polygon(t, kb, n, N, h.W, c, scale, i, P);
    // nearest of 24 evenly spaced parameters (the first of equals)
    double sv = 0.0, dmin = 1.0e300;
    for (int q = 0; q < 24; ++q) {
      const double sq = q == 23 ? 1.0 : q * (1.0 / 23.0);
      double b[4];
      bz_bern(sq, b);
      const double px = b[0] * P[0][0] + b[1] * P[1][0] + b[2] * P[2][0] + b[3] * P[3][0];
      const double py = b[0] * P[0][1] + b[1] * P[1][1] + b[2] * P[2][1] + b[3] * P[3][1];
      const double dd = (px - X0) * (px - X0) + (py - X1) * (py - X1);
      if (dd < dmin) {
        dmin = dd;
        sv = sq;
      }
    }
    for (int it = 0; it < 5; ++it) {
      const double u = 1.0 - sv;
      double Bv[2], d1[2], d2[2];
      for (int a = 0; a < 2; ++a) {
        Bv[a] = (u * u * u) * P[0][a] + (3.0 * u * u * sv) * P[1][a] +
                (3.0 * u * sv * sv) * P[2][a] + (sv * sv * sv) * P[3][a];
        d1[a] = (3.0 * u * u) * (P[1][a] - P[0][a]) + (6.0 * u * sv) * (P[2][a] - P[1][a]) +
                (3.0 * sv * sv) * (P[3][a] - P[2][a]);
        d2[a] = (6.0 * u) * (P[2][a] - 2.0 * P[1][a] + P[0][a]) +
                (6.0 * sv) * (P[3][a] - 2.0 * P[2][a] + P[1][a]);
      }
      const double rx = Bv[0] - X0, ry = Bv[1] - X1;
      const double f1 = rx * d1[0] + ry * d1[1];
      const double f2 = (d1[0] * d1[0] + d1[1] * d1[1]) + (rx * d2[0] + ry * d2[1]);
      const double step = f2 > 0.0 ? f1 / f2 : 0.0;
      sv = fmin(fmax(sv - step, 0.0), 1.0);
    }
    double b[4];
    bz_bern(sv, b);
    const double fx = b[0] * P[0][0] + b[1] * P[1][0] + b[2] * P[2][0] + b[3] * P[3][0];
    const double fy = b[0] * P[0][1] + b[1] * P[1][1] + b[2] * P[2][1] + b[3] * P[3][1];
    const double dist = sqrt((fx - X0) * (fx - X0) + (fy - X1) * (fy - X1));
    if (dist < best) {
      best = dist;
      bi = i;
      bs = sv;
    }
  }
  // side from the outward normal (right of the counter-clockwise tangent)
  double P[4][2];
  bz_polygon(t, kb, n, N, h.W, c, scale, bi, P);
  const double u = 1.0 - bs;
  double b[4];
  bz_bern(bs, b);
  const double fx = b[0] * P[0][0] + b[1] * P[1][0] + b[2] * P[2][0] + b[3] * P[3][0];
  const double fy = b[0] * P[0][1] + b[1] * P[1][1] + b[2] * P[2][1] + b[3] * P[3][1];
  const double tx = (3.0 * u * u) * (P[1][0] - P[0][0]) + (6.0 * u * bs) * (P[2][0] - P[1][0]) +
                    (3.0 * bs * bs) * (P[3][0] - P[2][0]);
  const double ty = (3.0 * u * u) * (P[1][1] - P[0][1]) + (6.0 * u * bs) * (P[2][1] - P[1][1]) +
                    (3.0 * bs * bs) * (P[3][1] - P[2][1]);
  h.inside = (X0 - fx) * ty + (X1 - fy) * (-tx) < 0.0;
  h.dist = best;
  h.seg = bi;
  h.sb = bs;
  h.nv[0] = best > 0.0 ? (X0 - fx) / best : 0.0;
  h.nv[1] = best > 0.0 ? (X1 - fy) / best : 0.0;
  h.d = h.inside ? -best : best;
  const double zm = 0.5 * (t[2] + t[3]), hh = 0.5 * (t[3] - t[2]);
  h.w = fabs(h.X[2] - zm) - hh;
  const double nrm = hypot(fmax(h.d, 0.0), fmax(h.w, 0.0));
  h.out = fmin(fmax(h.d, h.w), 0.0) + nrm;
}

// Fluid-positive phi of the union; *arg receives the nearest shape.
__device__ inline double bz_phi(const SceneDev &s, double x, double y, double z, int *arg,
                                BzHit *hit) {
  double best = 1.0e300;
  int a = 0;
  for (int sh = 0; sh < s.bz_n; ++sh) {
    BzHit h;
    bz_shape(s, sh, x, y, z, h);
    if (h.out < best) {
      best = h.out;
      a = sh;
      if (hit) *hit = h;
    }
  }
  if (arg) *arg = a;
  return s.bz_inside ? -best : best;
}

// d phi / d theta (K values): the envelope derivative of the nearest
// shape's distance with respect to its radii (moved along their radial unit
// vectors), times the capping factor; radii mode maps it onto theta,
// pulse mode contracts it with the base radii into d / d k and k's knots.
__device__ inline void bz_dphi(const SceneDev &s, double x, double y, double z, double *out) {
  for (int q = 0; q < kMaxParams; ++q) out[q] = 0.0;
  if (s.bz_mode == kBzFixed) return;
  int a = 0;
  BzHit h;
  bz_phi(s, x, y, z, &a, &h);
  const double *t = s.bz + s.bz_off[a];
  const int n = h.n, N = h.N, seg = h.seg;
  const double *tr = t + kBzHead;
  const double *kb = tr + 4 * N;
  double bw[4];
  bz_bern(h.sb, bw);
  const int pm = (seg + N - 1) % N, nx = (seg + 1) % N;
  // the radii of the closest segment's polygon and their envelope factors
  const int js[4] = {2 * pm + 1, 2 * seg, 2 * seg + 1, 2 * nx};
  double g2[4];
  for (int q = 0; q < 4; ++q) {
    const int j = js[q], i = j >> 1;
    const double ux = (j & 1) ? tr[4 * i + 2] : tr[4 * i], uy = (j & 1) ? tr[4 * i + 3] : tr[4 * i + 1];
    const double nu = h.nv[0] * ux + h.nv[1] * uy;
    double g = 0.0;
    if (q == 0) g -= nu * bw[0] * 0.5;                 // e0 (with rho2_{seg-1})
    if (q == 1) {
      g -= nu * bw[0] * 0.5;                           // e0 (with rho1_seg)
      g -= nu * bw[1];                                 // p0
    }
    if (q == 2) {
      g -= nu * bw[2];                                 // p1
      g -= nu * bw[3] * 0.5;                           // e1 (with rho1_{seg+1})
    }
    if (q == 3) g -= nu * bw[3] * 0.5;                 // e1
    g2[q] = h.inside ? -g : g;
  }
  const bool both_in = h.d <= 0.0 && h.w <= 0.0;
  const double nrm = hypot(fmax(h.d, 0.0), fmax(h.w, 0.0));
  const double dd = both_in ? (h.d >= h.w ? 1.0 : 0.0) : fmax(h.d, 0.0) / (nrm > 0.0 ? nrm : 1.0);
  const double sgn = s.bz_inside ? -1.0 : 1.0;
  if (s.bz_mode == kBzRadii) {
    for (int k = 0; k < n; ++k)
      for (int q = 0; q < 4; ++q) {
        const int idx = s.bz_theta0[a] + k * 2 * N + js[q];
        if (idx < kMaxParams) out[idx] += sgn * ((dd * h.W[k]) * g2[q]);
      }
    return;
  }
  if (a != s.bz_pulse) return;
  double v = 0.0;
  for (int k = 0; k < n; ++k)
    for (int q = 0; q < 4; ++q) v += ((dd * h.W[k]) * g2[q]) * kb[k * (2 + 2 * N) + 2 + js[q]];
  for (int q = 0; q < 4; ++q) out[q] = sgn * v * s.bz_dk[q];
}

// Solid velocity (and d/d theta) of the pulsing shape where it is the
// nearest shape: the velocity (kdot / k) (p - c(z)) of its uniform
// contraction about the cross-section centre, across its local z.
__device__ inline double bz_us(const SceneDev &s, int d, double x, double y, double z,
                               double *dout) {
  if (dout)
    for (int q = 0; q < kMaxParams; ++q) dout[q] = 0.0;
  if (s.bz_mode != kBzPulse) return 0.0;
  int a = 0;
  bz_phi(s, x, y, z, &a, nullptr);
  if (a != s.bz_pulse) return 0.0;
  BzHit h;
  double c[2];
  bz_frame(s, a, x, y, z, h, c);
  const double *t = s.bz + s.bz_off[a];
  const double r0 = h.X[0] - c[0], r1 = h.X[1] - c[1];
  const double dir = t[4] != 0.0 ? r0 * t[8 + d] + r1 * t[11 + d] : (d == 0 ? r0 : (d == 1 ? r1 : 0.0));
  if (dout) {
    const double k = s.bz_k, kd = s.bz_kdot;
    for (int q = 0; q < 4; ++q) dout[q] = dir * ((s.bz_dkdot[q] * k - kd * s.bz_dk[q]) / (k * k));
  }
  return (s.bz_kdot / s.bz_k) * dir;
}

// Fluid-positive level set phi(x) of the scene at its time. kBz = false
// compiles the polar-Bezier case out (kernels launched for the other scene
// kinds then keep their own register budget).
template <class R, bool kBz = true>
__device__ __forceinline__ R scene_phi(const SceneDev &s, R x, R y, R z) {
  switch (s.kind) {
    case NF_SCENE_SPHERE: {
      R dx = x - P<R>(s.sc[0], s.f_sc[0]), dy = y - P<R>(s.sc[1], s.f_sc[1]), dz = z - P<R>(s.sc[2], s.f_sc[2]);
      return sqrt(dx * dx + dy * dy + dz * dz) - P<R>(s.sr, s.f_sr);
    }
    case NF_SCENE_SPHERES: {
      R best = R(1.0e3);
      for (int i = 0; i < s.nspheres; ++i) {
        const double *p = s.spheres + 4 * i;
        R dx = x - R(p[0]), dy = y - R(p[1]), dz = z - R(p[2]);
        best = fmin(best, sqrt(dx * dx + dy * dy + dz * dz) - R(p[3]));
      }
      return best;
    }
    case NF_SCENE_CHAMBER: {
      R ex = (x - P<R>(s.cc[0], s.f_cc[0])) * P<R>(s.cinva[0], s.finva[0]), ey = (y - P<R>(s.cc[1], s.f_cc[1])) * P<R>(s.cinva[1], s.finva[1]),
        ez = (z - P<R>(s.cc[2], s.f_cc[2])) * P<R>(s.cinva[2], s.finva[2]);
      R pe = P<R>(s.camin, s.f_camin) * (P<R>(s.cs, s.f_cs) - sqrt(ex * ex + ey * ey + ez * ez));
      R pd = -box_sdf<R>(x - P<R>(s.dc[0], s.f_dc[0]), y - P<R>(s.dc[1], s.f_dc[1]), z - P<R>(s.dc[2], s.f_dc[2]),
                         P<R>(s.dh[0], s.f_dh[0]), P<R>(s.dh[1], s.f_dh[1]), P<R>(s.dh[2], s.f_dh[2]));
      return fmax(pe, pd);
    }
    case NF_SCENE_PLATE: {
      R rx = x - P<R>(s.pc[0], s.f_pc[0]), ry = y - P<R>(s.pc[1], s.f_pc[1]), rz = z - P<R>(s.pc[2], s.f_pc[2]);
      R c = P<R>(s.pcos, s.f_pcos), sn = P<R>(s.psin, s.f_psin);
      return box_sdf<R>(c * rx + sn * ry, -sn * rx + c * ry, rz, P<R>(s.ph[0], s.f_ph[0]),
                        P<R>(s.ph[1], s.f_ph[1]), P<R>(s.ph[2], s.f_ph[2]));
    }
    case NF_SCENE_EXTRUDED:
      if constexpr (kBz) return R(bz_phi(s, (double)x, (double)y, (double)z, nullptr, nullptr));
      return R(1.0e3);
    default:
      return R(1.0e3);
  }
}

// Chamber: is the ellipsoid the active piece of the union at x?
template <class R>
__device__ __forceinline__ bool chamber_ell_active(const SceneDev &s, R x, R y,
                                                   R z) {
  R ex = (x - P<R>(s.cc[0], s.f_cc[0])) * P<R>(s.cinva[0], s.finva[0]), ey = (y - P<R>(s.cc[1], s.f_cc[1])) * P<R>(s.cinva[1], s.finva[1]),
    ez = (z - P<R>(s.cc[2], s.f_cc[2])) * P<R>(s.cinva[2], s.finva[2]);
  R pe = P<R>(s.camin, s.f_camin) * (P<R>(s.cs, s.f_cs) - sqrt(ex * ex + ey * ey + ez * ez));
  R pd = -box_sdf<R>(x - P<R>(s.dc[0], s.f_dc[0]), y - P<R>(s.dc[1], s.f_dc[1]), z - P<R>(s.dc[2], s.f_dc[2]),
                     P<R>(s.dh[0], s.f_dh[0]), P<R>(s.dh[1], s.f_dh[1]), P<R>(s.dh[2], s.f_dh[2]));
  return pe >= pd;
}

// Component d of the solid velocity at x, in precision R.
template <class R, bool kBz = true>
__device__ __forceinline__ R scene_us(const SceneDev &s, int d, R x, R y,
                                      R z) {
  switch (s.kind) {
    case NF_SCENE_SPHERE:
      return P<R>(s.sv[d], s.f_sv[d]);
    case NF_SCENE_CHAMBER: {
      if (!chamber_ell_active<R>(s, x, y, z)) return R(0);
      R r = d == 0 ? x - P<R>(s.cc[0], s.f_cc[0]) : (d == 1 ? y - P<R>(s.cc[1], s.f_cc[1]) : z - P<R>(s.cc[2], s.f_cc[2]));
      return P<R>(s.crate, s.f_crate) * r;
    }
    case NF_SCENE_PLATE: {
      if (d == 0) return -P<R>(s.pomega, s.f_pomega) * (y - P<R>(s.pc[1], s.f_pc[1]));
      if (d == 1) return P<R>(s.pomega, s.f_pomega) * (x - P<R>(s.pc[0], s.f_pc[0]));
      return R(0);
    }
    case NF_SCENE_EXTRUDED:
      if constexpr (kBz) return R(bz_us(s, d, (double)x, (double)y, (double)z, nullptr));
      return R(0);
    default:
      return R(0);
  }
}

// d phi / d theta at x (K values).
template <bool kBz = true>
__device__ __forceinline__ void scene_dphi(const SceneDev &s, double x,
                                           double y, double z, double *out) {
  switch (s.kind) {
    case NF_SCENE_SPHERE: {
      double dx = x - s.sc[0], dy = y - s.sc[1], dz = z - s.sc[2];
      double n = sqrt(dx * dx + dy * dy + dz * dz);
      double inv = n > 0.0 ? 1.0 / n : 0.0;
      out[0] = -s.t * dx * inv;
      out[1] = -s.t * dy * inv;
      out[2] = -s.t * dz * inv;
      return;
    }
    case NF_SCENE_CHAMBER: {
      bool e = chamber_ell_active<double>(s, x, y, z);
      for (int k = 0; k < 8; ++k) out[k] = e ? s.camin * s.cds[k] : 0.0;
      return;
    }
    case NF_SCENE_PLATE: {
      double rx = x - s.pc[0], ry = y - s.pc[1], rz = z - s.pc[2];
      double px = s.pcos * rx + s.psin * ry, py = -s.psin * rx + s.pcos * ry;
      double gx, gy, gz;
      box_sdf_grad(px, py, rz, s.ph[0], s.ph[1], s.ph[2], gx, gy, gz);
      double dang = gx * py - gy * px;
      for (int k = 0; k < 4; ++k) out[k] = dang * s.pdang[k];
      return;
    }
    case NF_SCENE_EXTRUDED:
      if constexpr (kBz) {
        bz_dphi(s, x, y, z, out);
        return;
      }
      [[fallthrough]];
    default:
#pragma unroll
      for (int k = 0; k < kMaxParams; ++k) out[k] = 0.0;
  }
}

// d u_s,d / d theta at x (K values), FP32 (selector and factors only).
template <bool kBz = true>
__device__ __forceinline__ void scene_dus_f(const SceneDev &s, int d, float x,
                                            float y, float z, float *out) {
  switch (s.kind) {
    case NF_SCENE_SPHERE:
      for (int k = 0; k < 3; ++k) out[k] = (k == d) ? 1.f : 0.f;
      return;
    case NF_SCENE_CHAMBER: {
      const bool e = chamber_ell_active<float>(s, x, y, z);
      const float r = d == 0 ? x - s.f_cc[0] : (d == 1 ? y - s.f_cc[1] : z - s.f_cc[2]);
      for (int k = 0; k < 8; ++k) out[k] = e ? s.f_cdus[k] * r : 0.f;
      return;
    }
    case NF_SCENE_PLATE: {
      const float f = d == 0 ? -(y - s.f_pc[1]) : (d == 1 ? (x - s.f_pc[0]) : 0.f);
      for (int k = 0; k < 4; ++k) out[k] = f * s.f_pdomega[k];
      return;
    }
    case NF_SCENE_EXTRUDED:
      if constexpr (kBz) {
        double tmp[kMaxParams];
        bz_us(s, d, (double)x, (double)y, (double)z, tmp);
        for (int k = 0; k < kMaxParams; ++k) out[k] = (float)tmp[k];
        return;
      }
      [[fallthrough]];
    default:
#pragma unroll
      for (int k = 0; k < kMaxParams; ++k) out[k] = 0.f;
  }
}

// d u_s,d / d theta at x (K values).
template <bool kBz = true>
__device__ __forceinline__ void scene_dus(const SceneDev &s, int d, double x,
                                          double y, double z, double *out) {
  switch (s.kind) {
    case NF_SCENE_SPHERE:
      for (int k = 0; k < 3; ++k) out[k] = (k == d) ? 1.0 : 0.0;
      return;
    case NF_SCENE_CHAMBER: {
      bool e = chamber_ell_active<double>(s, x, y, z);
      double r = d == 0 ? x - s.cc[0] : (d == 1 ? y - s.cc[1] : z - s.cc[2]);
      for (int k = 0; k < 8; ++k) out[k] = e ? s.cdus[k] * r : 0.0;
      return;
    }
    case NF_SCENE_PLATE: {
      double f = d == 0 ? -(y - s.pc[1]) : (d == 1 ? (x - s.pc[0]) : 0.0);
      for (int k = 0; k < 4; ++k) out[k] = f * s.pdomega[k];
      return;
    }
    case NF_SCENE_EXTRUDED:
      if constexpr (kBz) {
        bz_us(s, d, x, y, z, out);
        return;
      }
      [[fallthrough]];
    default:
#pragma unroll
      for (int k = 0; k < kMaxParams; ++k) out[k] = 0.0;
  }
}

}  // namespace nf

namespace nf {

// --------------------------------------------------- narrow-band phi -----
// phi at points x_f + delta near a face centre x_f, with |delta| <= dx:
// the centre quantities are formed in FP64 once, the increments in FP32
// without cancellation, e.g. |d + delta| - |d| = (2 d.delta + |delta|^2) /
// (|d + delta| + |d|) and, per box axis, |p + delta| - |p| = sign(p) delta
// when |p| > |delta|. Near the interface every retained quantity is O(dx),
// so the FP32 result carries an absolute error of ~1e-7 dx while the bulk
// of the arithmetic (64 samples per face) is FP32.
struct LocalSdf {
  int kind;
  // sphere(s): offset of the face centre from the centre, its norm, radius
  float d[4][3], dn[4], r[4];
  int nsph;
  // chamber ellipsoid: e = (x_f - c0) / a, rho_c = |e|, 1 / a, amin, s
  float e[3], rho, inva[3], amin;
  double phic_ell;
  float phic_f;         // phic_ell rounded once
  // per-face constants of d phi / d theta, rounded to FP32 once: chamber
  // amin * ds/dtheta_k, plate dangle/dtheta_k, sphere -t
  float dscale[8];
  float bh[3];          // box half extents (plate gradient)
  // boxes (duct of the chamber, plate): per-axis p and q = |p| - h at the
  // centre, and the rotation (plate) taking offsets into the box frame
  float bp[3], bq[3], rc, rs;
  bool has_box;
  bool overflow;  // more candidate spheres than kept: evaluate in FP64

  __device__ void init(const SceneDev &s, double x, double y, double z,
                       double dx) {
    kind = s.kind;
    has_box = false;
    overflow = false;
    nsph = 0;
    rc = 1.f;
    rs = 0.f;
    if (kind == NF_SCENE_SPHERE) {
      const double a = x - s.sc[0], b = y - s.sc[1], c = z - s.sc[2];
      nsph = 1;
      d[0][0] = (float)a;
      d[0][1] = (float)b;
      d[0][2] = (float)c;
      const double n = fsqrt_refined(a * a + b * b + c * c);
      dn[0] = (float)n;
      r[0] = (float)(n - s.sr);  // phi at the centre
      dscale[0] = s.fdscale[0];
    } else if (kind == NF_SCENE_SPHERES) {
      // candidate spheres: within 1.6 dx (twice the control-volume radius)
      // of the best centre value can be the minimum somewhere in the volume
      double best = 1.0e3;
      for (int i = 0; i < s.nspheres; ++i) {
        const double *p = s.spheres + 4 * i;
        const double a = x - p[0], b = y - p[1], c = z - p[2];
        best = fmin(best, sqrt(a * a + b * b + c * c) - p[3]);
      }
      for (int i = 0; i < s.nspheres; ++i) {
        const double *p = s.spheres + 4 * i;
        const double a = x - p[0], b = y - p[1], c = z - p[2];
        const double n = sqrt(a * a + b * b + c * c);
        if (n - p[3] > best + 1.6 * dx) continue;
        if (nsph == 4) {  // too many candidates: caller evaluates in FP64
          overflow = true;
          break;
        }
        d[nsph][0] = (float)a;
        d[nsph][1] = (float)b;
        d[nsph][2] = (float)c;
        dn[nsph] = (float)n;
        r[nsph] = (float)(n - p[3]);
        ++nsph;
      }
    } else if (kind == NF_SCENE_CHAMBER) {
      const double ex = (x - s.cc[0]) * s.cinva[0], ey = (y - s.cc[1]) * s.cinva[1],
                   ez = (z - s.cc[2]) * s.cinva[2];
      const double rr = fsqrt_refined(ex * ex + ey * ey + ez * ez);
      e[0] = (float)ex;
      e[1] = (float)ey;
      e[2] = (float)ez;
      rho = (float)rr;
      inva[0] = s.finva[0];
      inva[1] = s.finva[1];
      inva[2] = s.finva[2];
      amin = s.f_camin;
      phic_ell = s.camin * (s.cs - rr);
      phic_f = (float)phic_ell;
#pragma unroll
      for (int k = 0; k < 8; ++k) dscale[k] = s.fdscale[k];
      box_init(x - s.dc[0], y - s.dc[1], z - s.dc[2], s.dh);
    } else if (kind == NF_SCENE_EXTRUDED) {
      overflow = true;  // polar-Bezier shapes: evaluated in FP64 throughout
    } else if (kind == NF_SCENE_PLATE) {
      const double rx = x - s.pc[0], ry = y - s.pc[1], rz = z - s.pc[2];
      rc = s.f_pcos;
      rs = s.f_psin;
      box_init(s.pcos * rx + s.psin * ry, -s.psin * rx + s.pcos * ry, rz, s.ph);
#pragma unroll
      for (int k = 0; k < 4; ++k) dscale[k] = s.fdscale[k];
      for (int a = 0; a < 3; ++a) bh[a] = s.f_ph[a];
    }
  }

  __device__ void box_init(double px, double py, double pz, const double *h) {
    has_box = true;
    const double p[3] = {px, py, pz};
    for (int a = 0; a < 3; ++a) {
      bp[a] = (float)p[a];
      bq[a] = (float)(fabs(p[a]) - h[a]);
    }
  }

  // |p + o| - |p| without cancellation.
  __device__ static float absdiff(float p, float o) {
    if (fabsf(p) >= fabsf(o)) return p >= 0.f ? o : -o;
    return fabsf(p + o) - fabsf(p);
  }

  // box SDF (positive outside) at the centre offset by o (box frame)
  __device__ float box(float ox, float oy, float oz) const {
    const float qx = bq[0] + absdiff(bp[0], ox);
    const float qy = bq[1] + absdiff(bp[1], oy);
    const float qz = bq[2] + absdiff(bp[2], oz);
    const float mx = fmaxf(qx, 0.f), my = fmaxf(qy, 0.f), mz = fmaxf(qz, 0.f);
    return sqrtf(mx * mx + my * my + mz * mz) + fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f);
  }

  // phi at x_f + (ox, oy, oz) (world offsets, |o| <= dx)
  __device__ float phi(float ox, float oy, float oz) const {
    switch (kind) {
      case NF_SCENE_SPHERE:
      case NF_SCENE_SPHERES: {
        float best = 1.0e3f;
        for (int i = 0; i < nsph; ++i) {
          const float a = d[i][0] + ox, b = d[i][1] + oy, c = d[i][2] + oz;
          const float num = 2.f * (d[i][0] * ox + d[i][1] * oy + d[i][2] * oz) +
                            (ox * ox + oy * oy + oz * oz);
          const float den = sqrtf(a * a + b * b + c * c) + dn[i];
          best = fminf(best, r[i] + (den > 0.f ? num / den : 0.f));
        }
        return best;
      }
      case NF_SCENE_CHAMBER: {
        const float ex = ox * inva[0], ey = oy * inva[1], ez = oz * inva[2];
        const float a = e[0] + ex, b = e[1] + ey, c = e[2] + ez;
        const float num = 2.f * (e[0] * ex + e[1] * ey + e[2] * ez) +
                          (ex * ex + ey * ey + ez * ez);
        const float den = sqrtf(a * a + b * b + c * c) + rho;
        const float pe = phic_f - amin * (den > 0.f ? num / den : 0.f);
        return fmaxf(pe, -box(ox, oy, oz));
      }
      case NF_SCENE_PLATE:
        return box(rc * ox + rs * oy, -rs * ox + rc * oy, oz);
      default:
        return 1.0e3f;
    }
  }

  // d phi / d theta at x_f + o (K values, FP32); xs are world coordinates
  __device__ void dphi(const SceneDev &s, float ox, float oy, float oz,
                       float *out) const {
    switch (kind) {
      case NF_SCENE_SPHERE: {
        const float a = d[0][0] + ox, b = d[0][1] + oy, c = d[0][2] + oz;
        const float n = sqrtf(a * a + b * b + c * c);
        const float inv = n > 0.f ? dscale[0] / n : 0.f;
        out[0] = a * inv;
        out[1] = b * inv;
        out[2] = c * inv;
        return;
      }
      case NF_SCENE_CHAMBER: {
        const float ex = ox * inva[0], ey = oy * inva[1], ez = oz * inva[2];
        const float a = e[0] + ex, b = e[1] + ey, c = e[2] + ez;
        const float num = 2.f * (e[0] * ex + e[1] * ey + e[2] * ez) +
                          (ex * ex + ey * ey + ez * ez);
        const float den = sqrtf(a * a + b * b + c * c) + rho;
        const float pe = phic_f - amin * (den > 0.f ? num / den : 0.f);
        const bool ell = pe >= -box(ox, oy, oz);
        for (int k = 0; k < 8; ++k) out[k] = ell ? dscale[k] : 0.f;
        return;
      }
      case NF_SCENE_PLATE: {
        const float px = bp[0] + (rc * ox + rs * oy), py = bp[1] + (-rs * ox + rc * oy),
                    pz = bp[2] + oz;
        float gx, gy, gz;
        box_sdf_grad_f(px, py, pz, bh[0], bh[1], bh[2], gx, gy, gz);
        const float dang = gx * py - gy * px;
        for (int k = 0; k < 4; ++k) out[k] = dang * dscale[k];
        return;
      }
      default:
  #pragma unroll
      for (int k = 0; k < kMaxParams; ++k) out[k] = 0.f;
    }
  }
};

}  // namespace nf
