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

// Fluid-positive level set phi(x) of the scene at its time.
template <class R>
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
template <class R>
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
#pragma unroll
      for (int k = 0; k < kMaxParams; ++k) out[k] = 0.0;
  }
}

// d u_s,d / d theta at x (K values), FP32 (selector and factors only).
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
    default:
#pragma unroll
      for (int k = 0; k < kMaxParams; ++k) out[k] = 0.f;
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
      for (int k = 0; k < 8; ++k) out[k] = e ? s.cdus[k] * r : 0.0;
      return;
    }
    case NF_SCENE_PLATE: {
      double f = d == 0 ? -(y - s.pc[1]) : (d == 1 ? (x - s.pc[0]) : 0.0);
      for (int k = 0; k < 4; ++k) out[k] = f * s.pdomega[k];
      return;
    }
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
