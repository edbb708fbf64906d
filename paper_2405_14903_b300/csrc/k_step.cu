// Step kernels: rasterisation (Sec. 2.3.1, Projection), RK2 semi-Lagrangian
// advection (Eq. advection_matrix; Appendix B, Eqs. advection_1/2), the
// right-hand side of Eq. projection_matrix, the blended velocity update
// (Eq. u_next_matrix, read as U = S (U^ - c G P) + (I - S) U_s), the losses,
// and the adjoint kernels of Sec. 2.3.2 / 2.3.3.
//
// All kernels are HBM-bound stencils or gathers (no dense contraction), so
// they are plain CUDA-core code: one thread per face or cell, x fastest so
// that warps read contiguous rows.
#include <algorithm>

#include "kernels.h"
#include "scene.cuh"

namespace nf {

// ------------------------------------------------------------ helpers -----

// Split a flat index over the three face arrays into (component, face).
__device__ __forceinline__ bool split_face(const GridDev &g, int64_t t, int &d,
                                           int64_t &f) {
  const int64_t n0 = g.nface(0), n1 = g.nface(1), n2 = g.nface(2);
  if (t < n0) {
    d = 0;
    f = t;
    return true;
  }
  t -= n0;
  if (t < n1) {
    d = 1;
    f = t;
    return true;
  }
  t -= n1;
  if (t < n2) {
    d = 2;
    f = t;
    return true;
  }
  return false;
}

// Grid-unit position of face (d; i, j, k): integer part plus 1/2 off-axis.
__device__ __forceinline__ void face_pos(int d, int i, int j, int k, double &X,
                                         double &Y, double &Z) {
  X = i + (d == 0 ? 0.0 : 0.5);
  Y = j + (d == 1 ? 0.0 : 0.5);
  Z = k + (d == 2 ? 0.0 : 0.5);
}

// One axis of a clamped linear interpolation on a lattice of n points, at
// position base + o (o small). Returns the left index, fraction, and the
// clamp slope (1 inside [0, n-1], 0 outside).
template <class R>
__device__ __forceinline__ void axis_w(int base, R o, int n, int &i0, R &fr,
                                       R &slope) {
  if (n == 1) {  // a one-point lattice (the 2D slab's z axis): constant
    i0 = 0;
    fr = R(0);
    slope = R(0);
    return;
  }
  const R fl = floor(o);
  const int i = base + (int)fl;
  const R f = o - fl;
  // below the lattice: the first point, slope 0; at or past the last point:
  // the last interval at weight 1, slope 0 past it and 1 exactly on it;
  // inside: the interval's own weight (selects, no branches)
  const bool below = i < 0, top = i >= n - 1;
  const bool past = i > n - 1 || (i == n - 1 && f > R(0));
  i0 = below ? 0 : (top ? n - 2 : i);
  fr = below ? R(0) : (top ? R(1) : f);
  slope = (below || past) ? R(0) : R(1);
}

// Lattice offsets (h_d - s_e) of a component-d face in component e's lattice.
__device__ __forceinline__ float lat_off(int d, int e, int a) {
  if (a == d && a != e) return -0.5f;
  if (a == e && a != d) return 0.5f;
  return 0.0f;
}

template <class R>
struct Interp {
  int idx[8];
  R w[8];
  R dw[3][8];
};

// Trilinear interpolation of component e at base + o (grid units, e's
// lattice coordinates). Optionally records corners and weight derivatives.
// Indices are 32-bit: an episode has fewer than 2^31 faces per component.
template <class T, class R, bool kStencil>
__device__ __forceinline__ R trilerp(const GridDev &g, const T *U, int e,
                                     int bi, int bj, int bk, R ox, R oy, R oz,
                                     Interp<R> *st = nullptr) {
  const int nx = g.nx + (e == 0), ny = g.ny + (e == 1), nz = g.nz + (e == 2);
  int i0, j0, k0;
  R fx, fy, fz, sx, sy, sz;
  axis_w<R>(bi, ox, nx, i0, fx, sx);
  axis_w<R>(bj, oy, ny, j0, fy, sy);
  axis_w<R>(bk, oz, nz, k0, fz, sz);
  const int base = (k0 * ny + j0) * nx + i0;
  // steps to the upper corner along each axis (0 on a one-point axis, whose
  // upper corner has weight 0: its load stays in bounds)
  const int sx1 = nx > 1 ? 1 : 0, sy1 = ny > 1 ? nx : 0, sz1 = nz > 1 ? nx * ny : 0;
  const R c000 = (R)U[base], c100 = (R)U[base + sx1];
  const R c010 = (R)U[base + sy1], c110 = (R)U[base + sy1 + sx1];
  const R c001 = (R)U[base + sz1], c101 = (R)U[base + sz1 + sx1];
  const R c011 = (R)U[base + sz1 + sy1], c111 = (R)U[base + sz1 + sy1 + sx1];
  const R gx = R(1) - fx, gy = R(1) - fy, gz = R(1) - fz;
  const R v = gz * (gy * (gx * c000 + fx * c100) + fy * (gx * c010 + fx * c110)) +
              fz * (gy * (gx * c001 + fx * c101) + fy * (gx * c011 + fx * c111));
  if (kStencil) {
    const int id[8] = {base,             base + sx1,       base + sy1,
                           base + sy1 + sx1, base + sz1,       base + sz1 + sx1,
                           base + sz1 + sy1, base + sz1 + sy1 + sx1};
    const R wx[2] = {gx, fx}, wy[2] = {gy, fy}, wz[2] = {gz, fz};
    const R ddx[2] = {-sx, sx}, ddy[2] = {-sy, sy}, ddz[2] = {-sz, sz};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
      st->idx[c] = id[c];
      st->w[c] = wx[cx] * wy[cy] * wz[cz];
      st->dw[0][c] = ddx[cx] * wy[cy] * wz[cz];
      st->dw[1][c] = wx[cx] * ddy[cy] * wz[cz];
      st->dw[2][c] = wx[cx] * wy[cy] * ddz[cz];
    }
  }
  return v;
}

template <class T>
__device__ __forceinline__ const T *comp(const Fields<T> &u, int e) {
  return e == 0 ? u.x : (e == 1 ? u.y : u.z);
}
template <class T>
__device__ __forceinline__ T *comp(FieldsMut<T> &u, int e) {
  return e == 0 ? u.x : (e == 1 ? u.y : u.z);
}

// ------------------------------------------------ corner (area) fractions --
// The paper's face fraction (Sec. 2.3.1, Projection), the grid option
// NF_FRACTIONS_CORNER: phi at the face's four corners, in the cyclic order
// (0,0), (1,0), (1,1), (0,1) of its tangential axes (d+1)%3 and (d+2)%3; on
// each edge whose end values differ in sign (phi >= 0 is fluid) the zero
// crossing by linear interpolation; alpha = the area of the polygon through
// the fluid corners and the crossings in walking order (shoelace formula),
// which keeps the fluid connected where only two diagonal corners are fluid.

// Physical position of corner c of face (d; i, j, k).
__device__ __forceinline__ void face_corner(int d, int i, int j, int k, int c,
                                            double dx, double p[3]) {
  face_pos(d, i, j, k, p[0], p[1], p[2]);
  p[(d + 1) % 3] += (c == 1 || c == 2) ? 0.5 : -0.5;
  p[(d + 2) % 3] += (c >= 2) ? 0.5 : -0.5;
  p[0] *= dx;
  p[1] *= dx;
  p[2] *= dx;
}

// alpha from the corner values, and d alpha / d phi_c into da.
__device__ double corner_area(const double ph[4], double da[4]) {
  const double cs[4] = {0.0, 1.0, 1.0, 0.0}, ct[4] = {0.0, 0.0, 1.0, 1.0};
  double vx[8], vy[8], w0[8], w1[8];
  int ve[8];  // edge (its first corner) of a crossing vertex, -1 for a corner
  int m = 0;
  for (int c = 0; c < 4; ++c) {
    const int n = (c + 1) & 3;
    const bool fc = ph[c] >= 0.0, fn = ph[n] >= 0.0;
    da[c] = 0.0;
    if (fc) {
      vx[m] = cs[c];
      vy[m] = ct[c];
      ve[m] = -1;
      ++m;
    }
    if (fc != fn) {
      const double den = ph[c] - ph[n], t = ph[c] / den;
      vx[m] = cs[c] + t * (cs[n] - cs[c]);
      vy[m] = ct[c] + t * (ct[n] - ct[c]);
      ve[m] = c;
      w0[m] = -ph[n] / (den * den);  // dt / dphi_c
      w1[m] = ph[c] / (den * den);   // dt / dphi_n
      ++m;
    }
  }
  double area = 0.0;
  for (int a = 0; a < m; ++a) {
    const int b = a + 1 < m ? a + 1 : 0;
    area += 0.5 * (vx[a] * vy[b] - vx[b] * vy[a]);
  }
  // dA/dv_a = 1/2 (y_next - y_prev, x_prev - x_next); a crossing moves along
  // its edge as t changes
  for (int a = 0; a < m; ++a) {
    if (ve[a] < 0) continue;
    const int nx = a + 1 < m ? a + 1 : 0, pv = a > 0 ? a - 1 : m - 1;
    const int c = ve[a], n = (c + 1) & 3;
    const double gdt = 0.5 * (vy[nx] - vy[pv]) * (cs[n] - cs[c]) +
                       0.5 * (vx[pv] - vx[nx]) * (ct[n] - ct[c]);
    da[c] += gdt * w0[a];
    da[n] += gdt * w1[a];
  }
  return area;
}

// ---------------------------------------------------------- rasterise -----
// alpha of a band face centred at (x, y, z), by the 32 lanes of a warp
// together: lane l takes subsamples l and l + 32 (x fastest, then y, z),
// the warp sums them. FP32 fields use the face's narrow-band evaluator L
// unless it overflowed, FP64 fields evaluate phi directly in FP64. Every lane
// returns the face's value in the field precision.
template <class T, bool kBz>
__device__ __forceinline__ T band_fraction_warp(const GridDev &g, const SceneDev &s,
                                                     const LocalSdf *L, double x, double y,
                                                     double z, int lane) {
  constexpr unsigned kAll = 0xffffffffu;
  if (sizeof(T) == 4 && !L->overflow) {
    // saturated samples are counted exactly; only the samples inside the
    // ramp are summed in FP32
    const float inv_w = g.finvw, h = g.fdx;
    int full = 0;
    float part = 0.f;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int sm = lane + 32 * half;
      const float ox = (((sm & 3) + 0.5f) * 0.25f - 0.5f) * h;
      const float oy = ((((sm >> 2) & 3) + 0.5f) * 0.25f - 0.5f) * h;
      const float oz = (((sm >> 4) + 0.5f) * 0.25f - 0.5f) * h;
      const float hv = 0.5f + L->phi(ox, oy, oz) * inv_w;
      if (hv >= 1.f)
        ++full;
      else if (hv > 0.f)
        part += hv;
    }
    full = __reduce_add_sync(kAll, full);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kAll, part, o);
    // (full + part) / 64 rounded once to FP32: the sum is formed exactly
    // before its one rounding (full <= 64, part a float), so FP32 arithmetic
    // gives the bits that the FP64 sum rounded to FP32 would
    return T(((float)full + part) * (1.0f / 64.0f));
  }
  const double inv_w = g.invw;
  double acc = 0.0;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int sm = lane + 32 * half;
    const double xx = x + (((sm & 3) + 0.5) * 0.25 - 0.5) * g.dx;
    const double yy = y + ((((sm >> 2) & 3) + 0.5) * 0.25 - 0.5) * g.dx;
    const double zz = z + (((sm >> 4) + 0.5) * 0.25 - 0.5) * g.dx;
    const double hv = 0.5 + scene_phi<double, kBz>(s, xx, yy, zz) * inv_w;
    acc += fmin(fmax(hv, 0.0), 1.0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kAll, acc, o);
  return T(acc * (1.0 / 64.0));
}

// Threads per block of the rasteriser: one narrow-band evaluator slot in
// shared memory per thread.
constexpr int kRastBlock = 128;

// alpha_f = (1/64) sum over 4x4x4 cell-centred subsamples of the face's
// dx^3 control volume of H(phi), H = clamp(1/2 + phi / (dx/4), 0, 1).
// Faces whose centre is farther than 0.8 dx from the interface are saturated
// (subsamples lie within 0.65 dx of the centre and phi is 1-Lipschitz), so
// only the narrow band evaluates the 64 samples. Each lane classifies its own
// face and, for a band face, sets up its narrow-band evaluator (the FP64
// centre terms, all band lanes at once); the band faces of a warp (sparse:
// one lane per band face would leave the others idle through 64 samples)
// are then summed one after another by the whole warp. kBz: the scene may
// be polar-Bezier shapes (else that case is compiled out).
template <class T, bool kCorner, bool kBz>
__global__ void __launch_bounds__(kRastBlock, 8)
k_rasterize(GridDev g, SceneDev s, FieldsMut<T> alpha) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  __shared__ LocalSdf sdf[kCorner ? 1 : kRastBlock];
  bool band = false;
  double X = 0.0, Y = 0.0, Z = 0.0;
  T *a = alpha.x;
  int64_t f = 0;
  do {
    int d;
    if (!split_face(g, t, d, f)) break;
    int i, j, k;
    g.face_ijk(d, f, i, j, k);
    a = comp(alpha, d);
    if (g.boundary(d, i, j, k)) {
      a[f] = g.outlet_face(d, i, j, k) ? T(1) : T(0);
      break;
    }
    const float hf = g.fdx;
    const float pc = scene_phi<float, kBz>(s, (i + (d == 0 ? 0.f : 0.5f)) * hf,
                                           (j + (d == 1 ? 0.f : 0.5f)) * hf,
                                           (k + (d == 2 ? 0.f : 0.5f)) * hf);
    // corners lie within 0.71 dx and subsamples within 0.65 dx of the centre
    const float margin = (kCorner ? 0.75f : 0.8f) * hf;
    if (pc > margin) {
      a[f] = T(1);
      break;
    }
    if (pc < -margin) {
      a[f] = T(0);
      break;
    }
    if (kCorner) {
      double ph[4], da[4], p[3];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        face_corner(d, i, j, k, c, g.dx, p);
        ph[c] = scene_phi<double, kBz>(s, p[0], p[1], p[2]);
      }
      a[f] = T(corner_area(ph, da));
      break;
    }
    face_pos(d, i, j, k, X, Y, Z);
    X *= g.dx;
    Y *= g.dx;
    Z *= g.dx;
    if (sizeof(T) == 4) sdf[threadIdx.x].init(s, X, Y, Z, g.dx);
    band = true;
  } while (false);
  if (kCorner) return;
  __syncwarp();  // the band lanes' evaluators are visible to the whole warp
  unsigned todo = __ballot_sync(0xffffffffu, band);
  while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1;
    const double bx = __shfl_sync(0xffffffffu, X, src);
    const double by = __shfl_sync(0xffffffffu, Y, src);
    const double bz = __shfl_sync(0xffffffffu, Z, src);
    const T v = band_fraction_warp<T, kBz>(g, s, &sdf[(threadIdx.x & ~31) + src], bx, by, bz,
                                           lane);
    if (lane == src) a[f] = v;
  }
}


// ------------------------------------------------------------- advect -----
// Positions are carried as (integer lattice base, small fractional offset)
// so that the interpolation weights keep full precision at every grid size.
// Component e of the velocity at the centre of face (d; i, j, k): the
// clamped trilinear interpolant there, whose weights are 1/2 or 1 (a face
// of component d sits half a cell off component e's lattice along d and e):
// the face's own value for e = d, else the mean of the two e-faces across
// it along e, averaged over the two cells beside it along d (one at the
// box walls, where the interpolant clamps).
template <class T>
__device__ __forceinline__ T face_velocity(const GridDev &g, const T *U, int e, int d, int i,
                                           int j, int k) {
  const int nx = g.nx + (e == 0), ny = g.ny + (e == 1);
  if (e == d) return U[(k * ny + j) * nx + i];
  const int nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);  // e's points along d
  const int id = d == 0 ? i : (d == 1 ? j : k);
  const int se = e == 0 ? 1 : (e == 1 ? nx : nx * ny);
  const int sd = d == 0 ? 1 : (d == 1 ? nx : nx * ny);
  // lattice point (i, j, k) of component e with the d index moved to id - 1
  const int base = (k * ny + j) * nx + i - sd;
  const int lo = id > 0 ? -1 : 0;            // d neighbours, clamped at the walls
  const int hi = id < nd ? 0 : -1;
  const T a = T(0.5) * (U[base + (lo + 1) * sd] + U[base + (lo + 1) * sd + se]);
  const T b = T(0.5) * (U[base + (hi + 1) * sd] + U[base + (hi + 1) * sd + se]);
  return T(0.5) * (a + b);
}

// r = dt / dx is formed on the host (an FP64 division per thread occupied
// the FP64 pipe, 1/64 of the FP32 rate here, for 45 % of the kernel).
template <class T>
__global__ void k_advect(GridDev g, Fields<T> u, FieldsMut<T> out, int order, T rdt) {
  pdl_wait();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int d;
  int64_t f;
  if (!split_face(g, t, d, f)) return;
  int i, j, k;
  g.face_ijk(d, f, i, j, k);
  typedef T R;
  const R r = rdt;
  R v0[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) v0[e] = face_velocity<T>(g, comp(u, e), e, d, i, j, k);
  R db[3];
  if (order == 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) db[a] = -r * v0[a];
  } else {
    R dm[3], v1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) dm[a] = R(-0.5) * r * v0[a];
#pragma unroll
    for (int e = 0; e < 3; ++e)
      v1[e] = trilerp<T, R, false>(g, comp(u, e), e, i, j, k,
                                   R(lat_off(d, e, 0)) + dm[0],
                                   R(lat_off(d, e, 1)) + dm[1],
                                   R(lat_off(d, e, 2)) + dm[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) db[a] = -r * v1[a];
  }
  comp(out, d)[f] =
      trilerp<T, R, false>(g, comp(u, d), d, i, j, k, db[0], db[1], db[2]);
}

// Adjoint of k_advect: scatter dJ/dU~ back to dJ/dU^n through the
// interpolation weights at x_b, x_m, x_f and through the positions
// (Sec. 2.3.2, the dB/dU U term). gu must be zeroed; float atomics make the
// summation order (not the set of terms) scheduling dependent.
template <class T>
__global__ void k_advect_adjoint(GridDev g, Fields<T> u, Fields<T> gut,
                                 FieldsMut<T> gu, int order, T rdt) {
  pdl_wait();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int d;
  int64_t f;
  if (!split_face(g, t, d, f)) return;
  const T gval = comp(gut, d)[f];
  if (gval == T(0)) return;
  int i, j, k;
  g.face_ijk(d, f, i, j, k);
  typedef T R;
  const R r = rdt;
  Interp<R> st;
  R v0[3], v1[3], dm[3], db[3];
#pragma unroll
  for (int e = 0; e < 3; ++e)
    v0[e] = trilerp<T, R, false>(g, comp(u, e), e, i, j, k, R(lat_off(d, e, 0)),
                                 R(lat_off(d, e, 1)), R(lat_off(d, e, 2)));
  if (order == 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) db[a] = -r * v0[a];
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) dm[a] = R(-0.5) * r * v0[a];
#pragma unroll
    for (int e = 0; e < 3; ++e)
      v1[e] = trilerp<T, R, false>(g, comp(u, e), e, i, j, k,
                                   R(lat_off(d, e, 0)) + dm[0],
                                   R(lat_off(d, e, 1)) + dm[1],
                                   R(lat_off(d, e, 2)) + dm[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) db[a] = -r * v1[a];
  }
  // u~_d = I_d(u_d; x_b)
  trilerp<T, R, true>(g, comp(u, d), d, i, j, k, db[0], db[1], db[2], &st);
  T *gd = comp(gu, d);
  const T *ud = comp(u, d);
  R gxb[3] = {0, 0, 0};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    atomicAdd(gd + st.idx[c], (T)(gval * st.w[c]));
    const R uc = (R)ud[st.idx[c]];
#pragma unroll
    for (int a = 0; a < 3; ++a) gxb[a] += st.dw[a][c] * uc;
  }
  R gv0[3];
  if (order == 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) gv0[a] = -r * gval * gxb[a];
  } else {
    R gxm[3] = {0, 0, 0};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const R gv1 = -r * gval * gxb[e];
      trilerp<T, R, true>(g, comp(u, e), e, i, j, k, R(lat_off(d, e, 0)) + dm[0],
                          R(lat_off(d, e, 1)) + dm[1],
                          R(lat_off(d, e, 2)) + dm[2], &st);
      T *ge = comp(gu, e);
      const T *ue = comp(u, e);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        atomicAdd(ge + st.idx[c], (T)(gv1 * st.w[c]));
        const R uc = (R)ue[st.idx[c]];
#pragma unroll
        for (int a = 0; a < 3; ++a) gxm[a] += gv1 * st.dw[a][c] * uc;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) gv0[a] = R(-0.5) * r * gxm[a];
  }
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    trilerp<T, R, true>(g, comp(u, e), e, i, j, k, R(lat_off(d, e, 0)),
                        R(lat_off(d, e, 1)), R(lat_off(d, e, 2)), &st);
    T *ge = comp(gu, e);
#pragma unroll
    for (int c = 0; c < 8; ++c) atomicAdd(ge + st.idx[c], (T)(gv0[e] * st.w[c]));
  }
}

// ----------------------------------------------------- face helpers -------
// Solid velocity of a component-d face (0 on the box boundary but for an
// inflow patch's faces, which carry the inflow speed), evaluated in
// the field precision T (positions formed in T: no FP64 for FP32 fields).
template <class T, bool kBz>
__device__ __forceinline__ T face_us(const GridDev &g, const SceneDev &s,
                                     int d, int i, int j, int k) {
  // box walls: at rest, except the faces of an inflow patch
  if (g.boundary(d, i, j, k)) return g.inlet_face(d, i, j, k) ? T(g.ispeed) : T(0);
  if (s.kind == NF_SCENE_NONE || s.kind == NF_SCENE_SPHERES) return T(0);
  const T h = sizeof(T) == 4 ? T(g.fdx) : T(g.dx);
  const T X = (T(i) + (d == 0 ? T(0) : T(0.5))) * h;
  const T Y = (T(j) + (d == 1 ? T(0) : T(0.5))) * h;
  const T Z = (T(k) + (d == 2 ? T(0) : T(0.5))) * h;
  return scene_us<T, kBz>(s, d, X, Y, Z);
}

// Sum of the six face fractions of cell (i, j, k).
template <class T>
__device__ __forceinline__ T cell_diag(const GridDev &g, const Fields<T> &a,
                                       int i, int j, int k) {
  return a.x[g.face(0, i, j, k)] + a.x[g.face(0, i + 1, j, k)] +
         a.y[g.face(1, i, j, k)] + a.y[g.face(1, i, j + 1, k)] +
         a.z[g.face(2, i, j, k)] + a.z[g.face(2, i, j, k + 1)];
}

// Cells on the two sides of face (d; i, j, k); -1 outside the box.
__device__ __forceinline__ void face_cells(const GridDev &g, int d, int i,
                                           int j, int k, int64_t &cL,
                                           int64_t &cR) {
  const int n = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
  const int o = d == 0 ? i : (d == 1 ? j : k);
  cR = o < n ? g.cell(i, j, k) : -1;
  cL = o > 0 ? g.cell(i - (d == 0), j - (d == 1), k - (d == 2)) : -1;
}

// ---------------------------------------------------------- viscosity -----
// Explicit viscosity (Eq. viscosity_matrix): out = in - kv G^T G in on each
// component's own face lattice, kv = nu h / dx^2. G differences the values
// across every edge between two neighbouring lattice points inside the box,
// so a face at the end of a lattice row has no neighbour past it (-G^T G is
// the lattice's graph Laplacian). G^T G is symmetric, so the same kernel maps
// dJ/dU^ to dJ/dU~ in the adjoint (Sec. 2.3.2, Viscosity and Advection).
//
// One thread per (i, j) lattice column of component blockIdx.z marches
// kViscZ planes (z-chunk blockIdx.y), carrying the values below, at and
// above the current plane in registers, so each value comes from DRAM once;
// the x and y neighbours are L1/L2 hits of the same plane. The unrolled
// loop lets the loads of every plane of the chunk be in flight together.
// in and out must not overlap.
constexpr int kViscZ = 8;

template <class T>
__global__ void __launch_bounds__(kBlock)
k_viscosity(GridDev g, Fields<T> in, FieldsMut<T> out, T kv) {
  const int d = blockIdx.z;
  const int nx = g.fnx(d), ny = g.fny(d), nz = g.fnz(d);
  const int64_t plane = (int64_t)nx * ny;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int k0 = blockIdx.y * kViscZ;
  if (p >= plane || k0 >= nz) return;
  const int j = (int)((uint32_t)p / (uint32_t)nx);
  const int i = (int)(p - (int64_t)j * nx);
  const bool xl = i > 0, xh = i + 1 < nx, yl = j > 0, yh = j + 1 < ny;
  const T *__restrict__ u = comp(in, d) + p;
  T *__restrict__ o = comp(out, d) + p;
  if (k0 + kViscZ < nz) {
    // a whole chunk with a plane above it: the column's kViscZ + 2 values
    // are loaded up front (all in flight at once)
    T v[kViscZ + 2];
    v[0] = k0 > 0 ? u[(int64_t)(k0 - 1) * plane] : T(0);
#pragma unroll
    for (int s = 0; s <= kViscZ; ++s) v[s + 1] = u[(int64_t)(k0 + s) * plane];
#pragma unroll
    for (int s = 0; s < kViscZ; ++s) {
      const int64_t q = (int64_t)(k0 + s) * plane;
      const T c = v[s + 1];
      T acc = v[s + 2] - c;
      if (k0 + s > 0) acc += v[s] - c;
      if (xl) acc += u[q - 1] - c;
      if (xh) acc += u[q + 1] - c;
      if (yl) acc += u[q - nx] - c;
      if (yh) acc += u[q + nx] - c;
      o[q] = c + kv * acc;
    }
    return;
  }
  T below = k0 > 0 ? u[(int64_t)(k0 - 1) * plane] : T(0);
  T c = u[(int64_t)k0 * plane];
#pragma unroll
  for (int s = 0; s < kViscZ; ++s) {
    const int k = k0 + s;
    if (k < nz) {
      const int64_t q = (int64_t)k * plane;
      const T above = k + 1 < nz ? u[q + plane] : T(0);
      T acc = T(0);
      if (xl) acc += u[q - 1] - c;
      if (xh) acc += u[q + 1] - c;
      if (yl) acc += u[q - nx] - c;
      if (yh) acc += u[q + nx] - c;
      if (k > 0) acc += below - c;
      if (k + 1 < nz) acc += above - c;
      o[q] = c + kv * acc;
      below = c;
      c = above;
    }
  }
}

// --------------------------------------------------------------- rhs ------
// b = G^T (S U^ + (I - S) U_s) / c on active cells (sum alpha > 0), else 0.
// G^T v at a cell is v(low face) - v(high face), summed over the axes. The
// division by c = dt / (rho dx) lets the solver use the unit-scale operator
// G^T S G, whose coefficients do not depend on the step length. Four blocks
// per SM (at most 64 registers) keep the kRedBlocks grid to one wave.
template <class T, class S, bool kBz>
__global__ void __launch_bounds__(kBlock, 4)
k_rhs(GridDev g, SceneDev s, Fields<T> alpha, Fields<T> uh, S *b, RedScratch rs,
      double *bnorm2) {
  pdl_wait();
  const double inv_c = g.invc;
  double v[1] = {0.0};
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       c < g.ncell(); c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    g.cell_ijk(c, i, j, k);
    const T dg = cell_diag(g, alpha, i, j, k);
    double acc = 0.0;
    if (dg > T(0)) {
      const int I[2] = {i, i + 1}, J[2] = {j, j + 1}, K[2] = {k, k + 1};
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const double sg = side == 0 ? 1.0 : -1.0;
        const int64_t fx = g.face(0, I[side], j, k), fy = g.face(1, i, J[side], k),
                      fz = g.face(2, i, j, K[side]);
        const T ax = alpha.x[fx], ay = alpha.y[fy], az = alpha.z[fz];
        // the solid velocity only where it has weight (fluid faces skip the scene)
        const T usx = ax < T(1) ? face_us<T, kBz>(g, s, 0, I[side], j, k) : T(0);
        const T usy = ay < T(1) ? face_us<T, kBz>(g, s, 1, i, J[side], k) : T(0);
        const T usz = az < T(1) ? face_us<T, kBz>(g, s, 2, i, j, K[side]) : T(0);
        acc += sg * (double)(ax * uh.x[fx] + (T(1) - ax) * usx);
        acc += sg * (double)(ay * uh.y[fy] + (T(1) - ay) * usy);
        acc += sg * (double)(az * uh.z[fz] + (T(1) - az) * usz);
      }
      acc *= inv_c;
    }
    b[c] = (S)acc;
    v[0] += acc * acc;
  }
  double tot[1];
  if (grid_sum<1>(v, rs, tot) && threadIdx.x == 0) *bnorm2 = tot[0];
}

// ------------------------------------------------------------- update -----
// U = alpha (U^ - c G P) + (1 - alpha) U_s, with ghost P = 0 outside.
template <class T, class S, bool kBz>
__global__ void k_update(GridDev g, SceneDev s, Fields<T> alpha, Fields<T> uh,
                         const S *P, FieldsMut<T> u, T cT) {
  pdl_wait();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int d;
  int64_t f;
  if (!split_face(g, t, d, f)) return;
  int i, j, k;
  g.face_ijk(d, f, i, j, k);
  int64_t cL, cR;
  face_cells(g, d, i, j, k, cL, cR);
  const S pR = cR >= 0 ? P[cR] : S(0);
  const S pL = cL >= 0 ? P[cL] : S(0);
  const T gp = cT * narrow<T>(pR - pL);
  const T a = comp(alpha, d)[f];
  // the solid velocity only where it has weight (fluid faces skip the scene)
  const T us = a < T(1) ? face_us<T, kBz>(g, s, d, i, j, k) : T(0);
  comp(u, d)[f] = a * (comp(uh, d)[f] - gp) + (T(1) - a) * us;
}

// -------------------------------------------------------------- losses ----
template <class T>
__global__ void k_loss_kinetic(GridDev g, Fields<T> u, FieldsMut<T> gu,
                               bool want_grad, RedScratch rs, double *J) {
  const double vol = g.dx * g.dx * g.dx;
  double v[1] = {0.0};
  const int64_t n = g.nface(0) + g.nface(1) + g.nface(2);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int d;
    int64_t f;
    split_face(g, t, d, f);
    const T x = comp(u, d)[f];
    v[0] += (double)x * (double)x;
    if (want_grad) comp(gu, d)[f] = (T)(vol * (double)x);
  }
  double tot[1];
  if (grid_sum<1>(v, rs, tot) && threadIdx.x == 0) *J = 0.5 * vol * tot[0];
}

template <class T>
__global__ void k_loss_outflow(GridDev g, Fields<T> u, FieldsMut<T> gu,
                               bool want_grad, RedScratch rs, double *J) {
  const double area = g.dx * g.dx;
  double v[1] = {0.0};
  const int64_t n = g.nface(0) + g.nface(1) + g.nface(2);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int d;
    int64_t f;
    split_face(g, t, d, f);
    int i, j, k;
    g.face_ijk(d, f, i, j, k);
    const bool o = g.outlet_face(d, i, j, k);
    if (o) v[0] += (double)comp(u, d)[f];
    if (want_grad) comp(gu, d)[f] = o ? (T)area : T(0);
  }
  double tot[1];
  if (grid_sum<1>(v, rs, tot) && threadIdx.x == 0) *J = area * tot[0];
}

// ------------------------------------------------------------ adjoint -----
// The 64-sample ramp derivative of one band face shared by a warp: lane l
// evaluates samples l and l + 32 with the narrow-band evaluator L (FP32
// fields; initialised once per face by one lane) or directly in FP64; out
// receives this lane's part of sum_samples (4 / dx) d phi / d theta, to be
// summed over the warp.
template <class T, bool kBz>
__device__ __forceinline__ void band_dalpha_lanes(const GridDev &g, const SceneDev &s,
                                                  const LocalSdf *L, double x, double y,
                                                  double z, int lane, T *out) {
#pragma unroll
  for (int q = 0; q < kMaxParams; ++q) out[q] = T(0);
  if (sizeof(T) == 4 && !L->overflow) {
    const float inv_w = g.finvw, h = g.fdx;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int sm = lane + 32 * half;
      const float ox = (((sm & 3) + 0.5f) * 0.25f - 0.5f) * h;
      const float oy = ((((sm >> 2) & 3) + 0.5f) * 0.25f - 0.5f) * h;
      const float oz = (((sm >> 4) + 0.5f) * 0.25f - 0.5f) * h;
      const float hv = 0.5f + L->phi(ox, oy, oz) * inv_w;
      if (hv > 0.f && hv < 1.f) {
        float tmp[kMaxParams];
        L->dphi(s, ox, oy, oz, tmp);
#pragma unroll
        for (int p = 0; p < kMaxParams; ++p)
          if (p < s.K) out[p] += (T)(inv_w * tmp[p]);
      }
    }
    return;
  }
  const double inv_w = g.invw;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int sm = lane + 32 * half;
    const double xx = x + (((sm & 3) + 0.5) * 0.25 - 0.5) * g.dx;
    const double yy = y + ((((sm >> 2) & 3) + 0.5) * 0.25 - 0.5) * g.dx;
    const double zz = z + (((sm >> 4) + 0.5) * 0.25 - 0.5) * g.dx;
    const double hv = 0.5 + scene_phi<double, kBz>(s, xx, yy, zz) * inv_w;
    if (hv > 0.0 && hv < 1.0) {
      double tmp[kMaxParams];
      scene_dphi<kBz>(s, xx, yy, zz, tmp);
#pragma unroll
      for (int p = 0; p < kMaxParams; ++p)
        if (p < s.K) out[p] += (T)(inv_w * tmp[p]);
    }
  }
}

// gP / c = -G^T (S gU) on active cells (dJ/dP of the update, divided by c
// for the unit-scale solver operator, like the forward right-hand side).
template <class T, class S>
__global__ void k_adj_gp(GridDev g, Fields<T> alpha, Fields<T> gu, S *gp,
                         RedScratch rs, double *norm2) {
  pdl_wait();
  double v[1] = {0.0};
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       c < g.ncell(); c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    g.cell_ijk(c, i, j, k);
    double acc = 0.0;
    if (cell_diag(g, alpha, i, j, k) > T(0)) {
      const int64_t f0 = g.face(0, i, j, k), f1 = g.face(1, i, j, k),
                    f2 = g.face(2, i, j, k);
      const int64_t f0p = f0 + 1, f1p = g.face(1, i, j + 1, k),
                    f2p = g.face(2, i, j, k + 1);
      acc = (double)(alpha.x[f0] * gu.x[f0]) - (double)(alpha.x[f0p] * gu.x[f0p]) +
            (double)(alpha.y[f1] * gu.y[f1]) - (double)(alpha.y[f1p] * gu.y[f1p]) +
            (double)(alpha.z[f2] * gu.z[f2]) - (double)(alpha.z[f2p] * gu.z[f2p]);
      acc = -acc;
    }
    gp[c] = (S)acc;
    v[0] += acc * acc;
  }
  double tot[1];
  if (grid_sum<1>(v, rs, tot) && threadIdx.x == 0) *norm2 = tot[0];
}

// Per face, with GP and Gy from the pressure and the adjoint variable:
//   gS   = gU (U^ - c GP - U_s) + Gy (U^ - U_s) - c Gy GP
//   gU^  = alpha (gU + Gy),   gU_s = (1 - alpha)(gU + Gy)
// and the parameter gradient  sum_f gS_f dalpha_f/dtheta + gU_s,f du_s,f/dtheta
// (Sec. 2.3.3), with dalpha/dtheta from the subsample ramps (narrow band).
// Threads per block of k_adj_face: one narrow-band evaluator slot in shared
// memory per thread.
constexpr int kAdjBlock = 128;

template <class T, class S, bool kCorner, bool kBz>
__global__ void __launch_bounds__(kAdjBlock, 4)
k_adj_face(GridDev g, SceneDev s, Fields<T> alpha, Fields<T> uh, const S *P, const S *y,
           Fields<T> gu, FieldsMut<T> guh, RedScratch rs, double *gtheta) {
  pdl_wait();
  // per-thread partial sums in the field precision (each thread adds a few
  // dozen faces), block and grid sums in FP64
  T acc[kMaxParams];
#pragma unroll
  for (int q = 0; q < kMaxParams; ++q) acc[q] = T(0);
  const int64_t n = g.nface(0) + g.nface(1) + g.nface(2);
  const T cT = sizeof(T) == 4 ? T(g.fc) : T(g.c), h = sizeof(T) == 4 ? T(g.fdx) : T(g.dx);
  const float margin = 0.8f * g.fdx;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  __shared__ LocalSdf sdf[kCorner ? 1 : kAdjBlock];
  // Each warp takes 32 consecutive faces at a time: every lane does its own
  // face's per-face work, a band face's lane also the FP64 centre terms of
  // its narrow-band evaluator (all band lanes at once); then the whole warp
  // evaluates the 64-sample derivative of each band face of the chunk in
  // turn (band faces are sparse, so one lane per band face would leave the
  // others idle).
  for (int64_t base = warp * 32; base < n; base += nwarps * 32) {
    const int64_t t = base + lane;
    bool band = false;
    T gS = T(0);
    double Xd = 0.0, Yd = 0.0, Zd = 0.0;
    do {
      if (t >= n) break;
      int d;
      int64_t f;
      split_face(g, t, d, f);
      int i, j, k;
      g.face_ijk(d, f, i, j, k);
      int64_t cL, cR;
      face_cells(g, d, i, j, k, cL, cR);
      // differences of the pressure-precision fields, the rest in T
      const T Gy = (T)((cR >= 0 ? y[cR] : S(0)) - (cL >= 0 ? y[cL] : S(0)));
      const T a = comp(alpha, d)[f];
      const T gU = comp(gu, d)[f];
      comp(guh, d)[f] = a * (gU + Gy);
      if (s.K == 0 || g.boundary(d, i, j, k)) break;
      const T X = (T(i) + (d == 0 ? T(0) : T(0.5))) * h;
      const T Y = (T(j) + (d == 1 ? T(0) : T(0.5))) * h;
      const T Z = (T(k) + (d == 2 ? T(0) : T(0.5))) * h;
      // solid-velocity term: its weight (1 - alpha) is exactly 0 where a = 1
      const T gUs = (T(1) - a) * (gU + Gy);
      if (gUs != T(0) && s.kind != NF_SCENE_SPHERES) {
        if (sizeof(T) == 4) {
          float tmp[kMaxParams];
          scene_dus_f<kBz>(s, d, (float)X, (float)Y, (float)Z, tmp);
#pragma unroll
          for (int q = 0; q < kMaxParams; ++q)
            if (q < s.K) acc[q] += gUs * (T)tmp[q];
        } else {
          double tmp[kMaxParams];
          scene_dus<kBz>(s, d, (double)X, (double)Y, (double)Z, tmp);
#pragma unroll
          for (int q = 0; q < kMaxParams; ++q)
            if (q < s.K) acc[q] += gUs * (T)tmp[q];
        }
      }
      // fraction term: d alpha / d theta vanishes off the narrow band (the
      // rasteriser's own test)
      const float pc = scene_phi<float, kBz>(s, (float)X, (float)Y, (float)Z);
      if (pc > margin || pc < -margin) break;
      const T GP = (T)((cR >= 0 ? P[cR] : S(0)) - (cL >= 0 ? P[cL] : S(0)));
      const T Uh = comp(uh, d)[f];
      const T us = face_us<T, kBz>(g, s, d, i, j, k);
      gS = gU * (Uh - cT * GP - us) + Gy * (Uh - us) - cT * Gy * GP;
      if (gS == T(0)) break;
      if (kCorner) {
        // d alpha / d theta = sum_c d alpha / d phi_c d phi_c / d theta,
        // four corners evaluated by this lane
        double ph[4], da[4], p[4][3];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          face_corner(d, i, j, k, c, g.dx, p[c]);
          ph[c] = scene_phi<double, kBz>(s, p[c][0], p[c][1], p[c][2]);
        }
        corner_area(ph, da);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (da[c] == 0.0) continue;
          double tmp[kMaxParams];
          scene_dphi<kBz>(s, p[c][0], p[c][1], p[c][2], tmp);
#pragma unroll
          for (int q = 0; q < kMaxParams; ++q)
            if (q < s.K) acc[q] += gS * (T)(da[c] * tmp[q]);
        }
        break;
      }
      face_pos(d, i, j, k, Xd, Yd, Zd);
      if (sizeof(T) == 4) sdf[threadIdx.x].init(s, Xd * g.dx, Yd * g.dx, Zd * g.dx, g.dx);
      band = true;
    } while (false);
    __syncwarp();  // the band lanes' evaluators are visible to the whole warp
    unsigned todo = __ballot_sync(0xffffffffu, band);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const double bx = __shfl_sync(0xffffffffu, Xd, src) * g.dx;
      const double by = __shfl_sync(0xffffffffu, Yd, src) * g.dx;
      const double bz = __shfl_sync(0xffffffffu, Zd, src) * g.dx;
      const T gSb = __shfl_sync(0xffffffffu, gS, src);
      const LocalSdf *L = &sdf[(threadIdx.x & ~31) + src];
      T part[kMaxParams];
      band_dalpha_lanes<T, kBz>(g, s, L, bx, by, bz, lane, part);
#pragma unroll
      for (int q = 0; q < kMaxParams; ++q) {
        T v = part[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && q < s.K) acc[q] += gSb * (v * T(1.0 / 64.0));
      }
    }
    __syncwarp();  // the slots are rewritten for the next chunk
  }
  double dacc[kMaxParams];
#pragma unroll
  for (int q = 0; q < kMaxParams; ++q) dacc[q] = (double)acc[q];
  double tot[kMaxParams];
  if (grid_sum<kMaxParams>(dacc, rs, tot) && threadIdx.x == 0)
    for (int q = 0; q < kMaxParams; ++q) gtheta[q] = tot[q];
}

// max |u| over every face (CFL rule), as the bits of a non-negative double
// (their integer order is the numeric order, so atomicMax is exact).
template <class T>
__global__ void k_absmax_faces(GridDev g, Fields<T> u, unsigned long long *out) {
  double m = 0.0;
  const int64_t n = g.nface(0) + g.nface(1) + g.nface(2);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int d;
    int64_t f;
    split_face(g, t, d, f);
    m = fmax(m, fabs((double)comp(u, d)[f]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// ------------------------------------------------------------ launchers ---
template <class T>
void launch_absmax_faces(const Launch &L, const GridDev &g, Fields<T> u,
                         unsigned long long *out) {
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), L.s);
  ProfScope _ps(L, NF_K_LOSS);
  k_absmax_faces<T><<<kRedBlocks, kBlock, 0, L.s>>>(g, u, out);
  ++*L.counter;
}

template <class T>
void launch_rasterize(const Launch &L, const GridDev &g, const SceneDev &s,
                      FieldsMut<T> alpha) {
  const int64_t n = g.nface(0) + g.nface(1) + g.nface(2);
  ProfScope _ps(L, NF_K_RASTERIZE);
  const bool corner = g.frac == NF_FRACTIONS_CORNER, bz = s.kind == NF_SCENE_EXTRUDED;
  const unsigned nb = nblocks(n, kRastBlock);
  if (corner && bz)
    k_rasterize<T, true, true><<<nb, kRastBlock, 0, L.s>>>(g, s, alpha);
  else if (corner)
    k_rasterize<T, true, false><<<nb, kRastBlock, 0, L.s>>>(g, s, alpha);
  else if (bz)
    k_rasterize<T, false, true><<<nb, kRastBlock, 0, L.s>>>(g, s, alpha);
  else
    k_rasterize<T, false, false><<<nb, kRastBlock, 0, L.s>>>(g, s, alpha);
  ++*L.counter;
}

template <class T>
void launch_advect(const Launch &L, const GridDev &g, Fields<T> u,
                   FieldsMut<T> out, int order) {
  const int64_t n = g.nface(0) + g.nface(1) + g.nface(2);
  ProfScope _ps(L, NF_K_ADVECT);
  launch_pdl(k_advect<T>, nblocks(n), kBlock, 0, L.s, g, u, out, order, (T)(g.dt / g.dx));
  ++*L.counter;
}

template <class T>
void launch_advect_adjoint(const Launch &L, const GridDev &g, Fields<T> u,
                           Fields<T> gut, FieldsMut<T> gu, int order) {
  const int64_t n = g.nface(0) + g.nface(1) + g.nface(2);
  cudaMemsetAsync(gu.x, 0, g.nface(0) * sizeof(T), L.s);
  cudaMemsetAsync(gu.y, 0, g.nface(1) * sizeof(T), L.s);
  cudaMemsetAsync(gu.z, 0, g.nface(2) * sizeof(T), L.s);
  ProfScope _ps(L, NF_K_ADJ_ADVECT);
  launch_pdl(k_advect_adjoint<T>, nblocks(n), kBlock, 0, L.s, g, u, gut, gu, order,
             (T)(g.dt / g.dx));
  ++*L.counter;
}

template <class T>
void launch_viscosity(const Launch &L, const GridDev &g, Fields<T> in,
                      FieldsMut<T> out) {
  // the largest lattice plane (x by y points) and depth over the components
  const int64_t plane = std::max({(int64_t)(g.nx + 1) * g.ny, (int64_t)g.nx * (g.ny + 1),
                                  (int64_t)g.nx * g.ny});
  const dim3 grid((unsigned)((plane + kBlock - 1) / kBlock),
                  (unsigned)((g.nz + 1 + kViscZ - 1) / kViscZ), 3);
  const double kv = g.nu * g.dt / (g.dx * g.dx);
  ProfScope _ps(L, NF_K_VISCOSITY);
  k_viscosity<T><<<grid, kBlock, 0, L.s>>>(g, in, out, T(kv));
  ++*L.counter;
}

template <class T, class S>
void launch_rhs(const Launch &L, const GridDev &g, const SceneDev &s,
                Fields<T> alpha, Fields<T> uh, S *b, const RedScratch &rs,
                double *bnorm2) {
  ProfScope _ps(L, NF_K_RHS);
  if (s.kind == NF_SCENE_EXTRUDED)
    launch_pdl(k_rhs<T, S, true>, kRedBlocks, kBlock, 0, L.s, g, s, alpha, uh, b, rs, bnorm2);
  else
    launch_pdl(k_rhs<T, S, false>, kRedBlocks, kBlock, 0, L.s, g, s, alpha, uh, b, rs, bnorm2);
  ++*L.counter;
}

template <class T, class S>
void launch_update(const Launch &L, const GridDev &g, const SceneDev &s,
                   Fields<T> alpha, Fields<T> uh, const S *P, FieldsMut<T> u) {
  const int64_t n = g.nface(0) + g.nface(1) + g.nface(2);
  ProfScope _ps(L, NF_K_UPDATE);
  if (s.kind == NF_SCENE_EXTRUDED)
    launch_pdl(k_update<T, S, true>, nblocks(n), kBlock, 0, L.s, g, s, alpha, uh, P, u, (T)g.c);
  else
    launch_pdl(k_update<T, S, false>, nblocks(n), kBlock, 0, L.s, g, s, alpha, uh, P, u, (T)g.c);
  ++*L.counter;
}

template <class T>
void launch_loss(const Launch &L, const GridDev &g, int kind, Fields<T> u,
                 FieldsMut<T> gu, bool want_grad, const RedScratch &rs,
                 double *J) {
  ProfScope _ps(L, NF_K_LOSS);
  if (kind == NF_LOSS_KINETIC)
    k_loss_kinetic<T><<<kRedBlocks, kBlock, 0, L.s>>>(g, u, gu, want_grad, rs, J);
  else
    k_loss_outflow<T><<<kRedBlocks, kBlock, 0, L.s>>>(g, u, gu, want_grad, rs, J);
  ++*L.counter;
}

template <class T, class S>
void launch_adj_gp(const Launch &L, const GridDev &g, Fields<T> alpha,
                   Fields<T> gu, S *gp, const RedScratch &rs, double *norm2) {
  ProfScope _ps(L, NF_K_ADJ_GP);
  launch_pdl(k_adj_gp<T, S>, kRedBlocks, kBlock, 0, L.s, g, alpha, gu, gp, rs, norm2);
  ++*L.counter;
}

template <class T, class S>
void launch_adj_face(const Launch &L, const GridDev &g, const SceneDev &s,
                     Fields<T> alpha, Fields<T> uh, const S *P, const S *y,
                     Fields<T> gu, FieldsMut<T> guh, const RedScratch &rs,
                     double *gtheta) {
  ProfScope _ps(L, NF_K_ADJ_FACE);
  const bool corner = g.frac == NF_FRACTIONS_CORNER, bz = s.kind == NF_SCENE_EXTRUDED;
  if (corner && bz)
    launch_pdl(k_adj_face<T, S, true, true>, kRedBlocks, kAdjBlock, 0, L.s, g, s, alpha, uh, P, y,
               gu, guh, rs, gtheta);
  else if (corner)
    launch_pdl(k_adj_face<T, S, true, false>, kRedBlocks, kAdjBlock, 0, L.s, g, s, alpha, uh, P, y,
               gu, guh, rs, gtheta);
  else if (bz)
    launch_pdl(k_adj_face<T, S, false, true>, kRedBlocks, kAdjBlock, 0, L.s, g, s, alpha, uh, P, y,
               gu, guh, rs, gtheta);
  else
    launch_pdl(k_adj_face<T, S, false, false>, kRedBlocks, kAdjBlock, 0, L.s, g, s, alpha, uh, P,
               y, gu, guh, rs, gtheta);
  ++*L.counter;
}

#define NF_INST_T(T)                                                          \
  template void launch_rasterize<T>(const Launch &, const GridDev &,        \
                                    const SceneDev &, FieldsMut<T>);         \
  template void launch_advect<T>(const Launch &, const GridDev &, Fields<T>,\
                                 FieldsMut<T>, int);                         \
  template void launch_advect_adjoint<T>(const Launch &, const GridDev &,   \
                                         Fields<T>, Fields<T>, FieldsMut<T>, \
                                         int);                               \
  template void launch_viscosity<T>(const Launch &, const GridDev &,        \
                                    Fields<T>, FieldsMut<T>);                \
  template void launch_loss<T>(const Launch &, const GridDev &, int,        \
                               Fields<T>, FieldsMut<T>, bool,                \
                               const RedScratch &, double *);                \
  template void launch_absmax_faces<T>(const Launch &, const GridDev &,     \
                                       Fields<T>, unsigned long long *);
#define NF_INST_TS(T, S)                                                      \
  template void launch_rhs<T, S>(const Launch &, const GridDev &,           \
                                 const SceneDev &, Fields<T>, Fields<T>, S *,\
                                 const RedScratch &, double *);              \
  template void launch_update<T, S>(const Launch &, const GridDev &,        \
                                    const SceneDev &, Fields<T>, Fields<T>,  \
                                    const S *, FieldsMut<T>);                \
  template void launch_adj_gp<T, S>(const Launch &, const GridDev &,        \
                                    Fields<T>, Fields<T>, S *,               \
                                    const RedScratch &, double *);           \
  template void launch_adj_face<T, S>(const Launch &, const GridDev &,      \
                                      const SceneDev &, Fields<T>, Fields<T>,\
                                      const S *, const S *, Fields<T>,       \
                                      FieldsMut<T>, const RedScratch &,      \
                                      double *);
NF_INST_T(float)
NF_INST_T(double)
NF_INST_TS(float, float)
NF_INST_TS(float, double)
NF_INST_TS(double, double)

}  // namespace nf
