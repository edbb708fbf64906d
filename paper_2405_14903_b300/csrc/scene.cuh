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

// Fluid-positive level set phi(x) of the scene at its time.
template <class R>
__device__ __forceinline__ R scene_phi(const SceneDev &s, R x, R y, R z) {
  switch (s.kind) {
    case NF_SCENE_SPHERE: {
      R dx = x - R(s.sc[0]), dy = y - R(s.sc[1]), dz = z - R(s.sc[2]);
      return sqrt(dx * dx + dy * dy + dz * dz) - R(s.sr);
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
      R ex = (x - R(s.cc[0])) / R(s.ca[0]), ey = (y - R(s.cc[1])) / R(s.ca[1]),
        ez = (z - R(s.cc[2])) / R(s.ca[2]);
      R pe = R(s.camin) * (R(s.cs) - sqrt(ex * ex + ey * ey + ez * ez));
      R pd = -box_sdf<R>(x - R(s.dc[0]), y - R(s.dc[1]), z - R(s.dc[2]),
                         R(s.dh[0]), R(s.dh[1]), R(s.dh[2]));
      return fmax(pe, pd);
    }
    case NF_SCENE_PLATE: {
      R rx = x - R(s.pc[0]), ry = y - R(s.pc[1]), rz = z - R(s.pc[2]);
      R c = R(s.pcos), sn = R(s.psin);
      return box_sdf<R>(c * rx + sn * ry, -sn * rx + c * ry, rz, R(s.ph[0]),
                        R(s.ph[1]), R(s.ph[2]));
    }
    default:
      return R(1.0e3);
  }
}

// Chamber: is the ellipsoid the active piece of the union at x?
template <class R>
__device__ __forceinline__ bool chamber_ell_active(const SceneDev &s, R x, R y,
                                                   R z) {
  R ex = (x - R(s.cc[0])) / R(s.ca[0]), ey = (y - R(s.cc[1])) / R(s.ca[1]),
    ez = (z - R(s.cc[2])) / R(s.ca[2]);
  R pe = R(s.camin) * (R(s.cs) - sqrt(ex * ex + ey * ey + ez * ez));
  R pd = -box_sdf<R>(x - R(s.dc[0]), y - R(s.dc[1]), z - R(s.dc[2]),
                     R(s.dh[0]), R(s.dh[1]), R(s.dh[2]));
  return pe >= pd;
}

// Component d of the solid velocity at x, in precision R.
template <class R>
__device__ __forceinline__ R scene_us(const SceneDev &s, int d, R x, R y,
                                      R z) {
  switch (s.kind) {
    case NF_SCENE_SPHERE:
      return R(s.sv[d]);
    case NF_SCENE_CHAMBER: {
      if (!chamber_ell_active<R>(s, x, y, z)) return R(0);
      R r = d == 0 ? x - R(s.cc[0]) : (d == 1 ? y - R(s.cc[1]) : z - R(s.cc[2]));
      return R(s.csdot / s.cs) * r;
    }
    case NF_SCENE_PLATE: {
      if (d == 0) return -R(s.pomega) * (y - R(s.pc[1]));
      if (d == 1) return R(s.pomega) * (x - R(s.pc[0]));
      return R(0);
    }
    default:
      return R(0);
  }
}

// d phi / d theta at x (K values).
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
    default:
      for (int k = 0; k < s.K; ++k) out[k] = 0.0;
  }
}

// d u_s,d / d theta at x (K values).
__device__ __forceinline__ void scene_dus(const SceneDev &s, int d, double x,
                                          double y, double z, double *out) {
  switch (s.kind) {
    case NF_SCENE_SPHERE:
      for (int k = 0; k < 3; ++k) out[k] = (k == d) ? 1.0 : 0.0;
      return;
    case NF_SCENE_CHAMBER: {
      bool e = chamber_ell_active<double>(s, x, y, z);
      double r = d == 0 ? x - s.cc[0] : (d == 1 ? y - s.cc[1] : z - s.cc[2]);
      double inv = 1.0 / (s.cs * s.cs);
      for (int k = 0; k < 8; ++k)
        out[k] = e ? (s.cdsdot[k] * s.cs - s.csdot * s.cds[k]) * inv * r : 0.0;
      return;
    }
    case NF_SCENE_PLATE: {
      double f = d == 0 ? -(y - s.pc[1]) : (d == 1 ? (x - s.pc[0]) : 0.0);
      for (int k = 0; k < 4; ++k) out[k] = f * s.pdomega[k];
      return;
    }
    default:
      for (int k = 0; k < s.K; ++k) out[k] = 0.0;
  }
}

}  // namespace nf
