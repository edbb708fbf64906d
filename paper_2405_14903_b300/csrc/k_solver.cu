// Solver kernels for A P = b, A = c G^T S G (Sec. 2.3.1, Eq.
// projection_matrix): the matrix-free 7-point alpha-weighted apply, fused CG
// vector updates with deterministic FP64 reductions, and the geometric
// multigrid V-cycle used as the CG preconditioner (red-black Gauss-Seidel
// smoothing, trilinear prolongation, restriction R = P^T / 4, coarse
// fractions = mean of the four fine sub-faces, operator rediscretised with
// c_l = dt / (rho dx_l)).
#include <cmath>

#include <cooperative_groups.h>

#include "kernels.h"
#include "util.h"

namespace nf {

// ---------------------------------------------------- level indexing -----
struct Lv {
  int nx, ny, nz;
  __device__ __forceinline__ int64_t fx(int i, int j, int k) const {
    return ((int64_t)k * ny + j) * (nx + 1) + i;
  }
  __device__ __forceinline__ int64_t fy(int i, int j, int k) const {
    return ((int64_t)k * (ny + 1) + j) * nx + i;
  }
  __device__ __forceinline__ int64_t fz(int i, int j, int k) const {
    return ((int64_t)k * ny + j) * nx + i;
  }
};

// Fractions of the six faces of a cell, in arithmetic type R.
template <class R>
struct Six {
  R xm, xp, ym, yp, zm, zp;
  __device__ __forceinline__ R diag() const { return xm + xp + ym + yp + zm + zp; }
};
template <class R, class TA>
__device__ __forceinline__ Six<R> six(const LevelView<TA> &lv, int i, int j,
                                      int k) {
  Lv L{lv.nx, lv.ny, lv.nz};
  Six<R> s;
  s.xm = (R)ld(lv.ax + L.fx(i, j, k));
  s.xp = (R)ld(lv.ax + L.fx(i + 1, j, k));
  s.ym = (R)ld(lv.ay + L.fy(i, j, k));
  s.yp = (R)ld(lv.ay + L.fy(i, j + 1, k));
  s.zm = (R)ld(lv.az + L.fz(i, j, k));
  s.zp = (R)ld(lv.az + L.fz(i, j, k + 1));
  return s;
}

// Weighted neighbour sum sum_f alpha_f x_nb(f) (ghost x = 0 outside).
template <class R, class X>
__device__ __forceinline__ R nbsum(const Six<R> &s, const X *x, int nx, int ny,
                                   int nz, int i, int j, int k, int64_t c) {
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  R acc = R(0);
  if (i > 0) acc += s.xm * (R)x[c - 1];
  if (i < nx - 1) acc += s.xp * (R)x[c + 1];
  if (j > 0) acc += s.ym * (R)x[c - sy];
  if (j < ny - 1) acc += s.yp * (R)x[c + sy];
  if (k > 0) acc += s.zm * (R)x[c - sz];
  if (k < nz - 1) acc += s.zp * (R)x[c + sz];
  return acc;
}

// ------------------------------------------------- per-cell operations -----
// (A x)_c = c (diag x_c - sum_f alpha_f x_nb), 0 on inactive cells. The
// arithmetic type is the vector type V.
template <class V, class TA>
__device__ __forceinline__ V apply_cell(const LevelView<TA> &lv, const V *x,
                                        int i, int j, int k, int64_t c) {
  const Six<V> s = six<V>(lv, i, j, k);
  const V dg = s.diag();
  if (!(dg > V(0))) return V(0);
  const V nb = nbsum<V>(s, x, lv.nx, lv.ny, lv.nz, i, j, k, c);
  return V(lv.c) * (dg * x[c] - nb);
}

// Multigrid residual b - A x, zero on inactive cells: the restriction is
// R = P^T / 4 with the prolongation P masked to active fine cells, so the
// residual it restricts must vanish where P is masked (keeps M symmetric).
template <class V, class TA>
__device__ __forceinline__ V residual_cell(const LevelView<TA> &lv, const V *x,
                                           const V *b, int i, int j, int k,
                                           int64_t c) {
  const Six<V> s = six<V>(lv, i, j, k);
  const V dg = s.diag();
  if (!(dg > V(0))) return V(0);
  const V nb = nbsum<V>(s, x, lv.nx, lv.ny, lv.nz, i, j, k, c);
  return b[c] - V(lv.c) * (dg * x[c] - nb);
}

// Gauss-Seidel update of one cell: x = (b + c nb) / (c diag); 0 if inactive.
template <class V, class TA>
__device__ __forceinline__ V gs_cell(const LevelView<TA> &lv, const V *x,
                                     const V *b, int i, int j, int k,
                                     int64_t c) {
  const Six<V> s = six<V>(lv, i, j, k);
  const V dg = s.diag();
  if (!(dg > V(0))) return V(0);
  const V cc = V(lv.c);
  const V nb = nbsum<V>(s, x, lv.nx, lv.ny, lv.nz, i, j, k, c);
  return (b[c] + cc * nb) / (cc * dg);
}

// 1D restriction weights (R = P^T / 4 with clamped trilinear P) for coarse
// index I of n coarse cells: fine offsets 2I-1 .. 2I+2.
__device__ __forceinline__ void rweights(int I, int n, float w[4]) {
  w[0] = 0.25f;
  w[1] = 0.75f;
  w[2] = 0.75f;
  w[3] = 0.25f;
  if (I == 0) {
    w[0] = 0.f;
    w[1] = 1.f;
  }
  if (I == n - 1) {
    w[3] = 0.f;
    w[2] = 1.f;
  }
}

// Transfer modes between levels: kTransferTrilinear (P trilinear, clamped
// at the box; R = P^T / 4) or kTransferConstant (P copies the parent, R is
// the mean of the eight children: with that pair the coarse operator built
// from the mean sub-face fractions and c / 2 is exactly the Galerkin
// operator R A P, so the coarse correction is an A-orthogonal projection).
[[maybe_unused]] constexpr int kTransferTrilinear = 0;
constexpr int kTransferConstant = 1;

template <class V>
__device__ __forceinline__ V restrict_cell(int fnx, int fny, int fnz, int cnx,
                                           int cny, int cnz, const V *rf, int I,
                                           int J, int K, int mode) {
  if (mode == kTransferConstant) {
    V acc = V(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const V *row = rf + ((int64_t)(2 * K + c) * fny + (2 * J + b)) * fnx + 2 * I;
        acc += row[0];
        acc += row[1];
      }
    return V(0.125) * acc;
  }
  // fine offsets 2I-1 .. 2I+2 per axis; an offset outside the fine grid has
  // weight 0 and reads a clamped (valid) index, so all 64 loads are
  // unconditional and can be issued together
  float wx[4], wy[4], wz[4];
  rweights(I, cnx, wx);
  rweights(J, cny, wy);
  rweights(K, cnz, wz);
  int ix[4], iy[4], iz[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = 2 * I - 1 + a, j = 2 * J - 1 + a, k = 2 * K - 1 + a;
    if (i < 0 || i >= fnx) wx[a] = 0.f;
    if (j < 0 || j >= fny) wy[a] = 0.f;
    if (k < 0 || k >= fnz) wz[a] = 0.f;
    ix[a] = min(max(i, 0), fnx - 1);
    iy[a] = min(max(j, 0), fny - 1);
    iz[a] = min(max(k, 0), fnz - 1);
  }
  V acc = V(0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const V wzy = V(wz[c] * wy[b]);
      const V *row = rf + ((int64_t)iz[c] * fny + iy[b]) * fnx;
#pragma unroll
      for (int a = 0; a < 4; ++a) acc += wzy * V(wx[a]) * row[ix[a]];
    }
  }
  return V(0.25) * acc;
}

// Trilinear (clamped) prolongation of the coarse correction to fine cell
// (i, j, k).
template <class V>
__device__ __forceinline__ V prolong_cell(int cnx, int cny, int cnz,
                                          const V *xc, int i, int j, int k,
                                          int mode) {
  if (mode == kTransferConstant)
    return xc[((int64_t)(k >> 1) * cny + (j >> 1)) * cnx + (i >> 1)];
  int I[2], J[2], K[2];
  auto ax = [](int f, int n, int *C) {
    const int c0 = f >> 1;
    int c1 = (f & 1) ? c0 + 1 : c0 - 1;
    if (c1 < 0 || c1 >= n) c1 = c0;
    C[0] = c0;
    C[1] = c1;
  };
  ax(i, cnx, I);
  ax(j, cny, J);
  ax(k, cnz, K);
  const V w[2] = {V(0.75), V(0.25)};
  V acc = V(0);
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a)
        acc += w[c] * w[b] * w[a] * xc[((int64_t)K[c] * cny + J[b]) * cnx + I[a]];
  return acc;
}

__device__ __forceinline__ bool stopped(const CGState *st) {
  return st != nullptr && *(volatile const int *)&st->done != 0;
}
// The same flag for kernels that check it late: the load is issued first,
// the kernel issues its first data loads, and only its first store waits
// for the flag (one L2 round trip less per block). Blocks of one launch all
// read the same value: the flag changes only at the end of a grid reduction,
// after every block of that launch has read it.
__device__ __forceinline__ int stop_flag(const CGState *st) {
  return st != nullptr ? *(volatile const int *)&st->done : 0;
}

// ------------------------------------------------------------- ILP ------
// Grid-stride kernels walk cells in batches of ILP cells per thread (cells
// c0, c0 + stride, ...): every load of a batch is issued before its results
// are used or stored, so a thread keeps several cells' loads in flight
// instead of one (the compiler may not move a load above a store through a
// possibly aliasing pointer). Per-thread accumulation still runs over cells
// in increasing order, so reductions are unchanged.
constexpr int kIlpStream = 4;   // streaming vector kernels (stencils: one cell per step)

// The 13 operands of one cell's 7-point operator: the six face fractions,
// the six neighbour values (0 outside the grid) and the centre value.
template <class R>
struct Nb7 {
  R xm, xp, ym, yp, zm, zp;
  R vxm, vxp, vym, vyp, vzm, vzp, vc;
  __device__ __forceinline__ R diag() const { return xm + xp + ym + yp + zm + zp; }
  // sum_f alpha_f x_nb(f) in the order x-, x+, y-, y+, z-, z+
  __device__ __forceinline__ R nb() const {
    R acc = R(0);
    acc += xm * vxm;
    acc += xp * vxp;
    acc += ym * vym;
    acc += yp * vyp;
    acc += zm * vzm;
    acc += zp * vzp;
    return acc;
  }
};
template <class R, class TA, class X>
__device__ __forceinline__ void gather7(Nb7<R> &g, const LevelView<TA> &lv,
                                        const X *x, int i, int j, int k,
                                        int64_t c) {
  const Six<R> s = six<R>(lv, i, j, k);
  g.xm = s.xm;
  g.xp = s.xp;
  g.ym = s.ym;
  g.yp = s.yp;
  g.zm = s.zm;
  g.zp = s.zp;
  const int64_t sy = lv.nx, sz = (int64_t)lv.nx * lv.ny;
  g.vxm = i > 0 ? (R)x[c - 1] : R(0);
  g.vxp = i < lv.nx - 1 ? (R)x[c + 1] : R(0);
  g.vym = j > 0 ? (R)x[c - sy] : R(0);
  g.vyp = j < lv.ny - 1 ? (R)x[c + sy] : R(0);
  g.vzm = k > 0 ? (R)x[c - sz] : R(0);
  g.vzp = k < lv.nz - 1 ? (R)x[c + sz] : R(0);
  g.vc = (R)x[c];
}

// ------------------------------------------------------------ rows ------
// Stencil kernels walk the grid by rows (j, k): one warp per row in a
// grid-stride loop over rows, lanes along x. A row costs one integer
// division; every face index follows from the cell index c with adds
// (ax: c + row, ay: c + k nx, az: c) in 32-bit arithmetic (episodes are
// limited to fewer than 2^31 faces per component).
struct RowWalk {
  int lane, warp, nwarps;
  __device__ __forceinline__ RowWalk() {
    lane = threadIdx.x & 31;
    warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  }
};

// A fraction widened to the arithmetic type R (FP32 fractions into the FP64
// outer residual by f2d: that kernel is bound by the FP64 pipe).
template <class R, class TA>
__device__ __forceinline__ R widen(const TA *p) {
  return (R)ld(p);
}
template <>
__device__ __forceinline__ double widen<double, float>(const float *p) {
  return f2d(*p);
}
// A V value widened to FP64 (FP32 by f2d).
__device__ __forceinline__ double widen_v(float v) { return f2d(v); }
__device__ __forceinline__ double widen_v(double v) { return v; }

template <class R, class TA, class X>
__device__ __forceinline__ void gather7r(Nb7<R> &g, const LevelView<TA> &lv,
                                         const X *x, int i, int j, int k, int c,
                                         int row) {
  const int nx = lv.nx, nxy = lv.nx * lv.ny;
  const int fy = c + k * nx;
  g.xm = widen<R>(lv.ax + c + row);
  g.xp = widen<R>(lv.ax + c + row + 1);
  g.ym = widen<R>(lv.ay + fy);
  g.yp = widen<R>(lv.ay + fy + nx);
  g.zm = widen<R>(lv.az + c);
  g.zp = widen<R>(lv.az + c + nxy);
  g.vxm = i > 0 ? (R)x[c - 1] : R(0);
  g.vxp = i < nx - 1 ? (R)x[c + 1] : R(0);
  g.vym = j > 0 ? (R)x[c - nx] : R(0);
  g.vyp = j < lv.ny - 1 ? (R)x[c + nx] : R(0);
  g.vzm = k > 0 ? (R)x[c - nxy] : R(0);
  g.vzp = k < lv.nz - 1 ? (R)x[c + nxy] : R(0);
  g.vc = (R)x[c];
}

// Blocks of kBlock threads giving one warp per row (at most kRedBlocks * 8).
inline unsigned row_blocks(int nrows) {
  const unsigned w = kBlock / 32;
  const unsigned b = (unsigned)((nrows + w - 1) / w);
  return b < (unsigned)kRedBlocks * 8 ? b : (unsigned)kRedBlocks * 8;
}

// ------------------------------------------------------ outer residual -----
// r = b - A x in FP64 arithmetic, scaled into rin (V), and ||r||^2 (FP64
// per-thread partials, block and grid sums).
template <class S, class T, class V>
__global__ void k_residual_outer(LevelView<T> lv, const S *b, const S *x,
                                 V *rin, double scale, RedScratch rs,
                                 double *norm2) {
  double v[1] = {0.0};
  const RowWalk w;
  const int nrows = lv.ny * lv.nz;
  for (int row = w.warp; row < nrows; row += w.nwarps) {
    const int k = row / lv.ny, j = row - k * lv.ny;
    const int base = row * lv.nx;
    for (int i = w.lane; i < lv.nx; i += 32) {
      const int c = base + i;
      Nb7<double> g;
      gather7r(g, lv, x, i, j, k, c, row);
      const double dg = g.diag();
      double rv = 0.0;
      if (dg > 0.0) rv = (double)b[c] - lv.c * (dg * g.vc - g.nb());
      rin[c] = (V)(rv * scale);
      v[0] += rv * rv;
    }
  }
  double tot[1];
  if (grid_sum<1>(v, rs, tot) && threadIdx.x == 0) *norm2 = tot[0];
}

// The same residual for S = double, T = V = float without FP64 arithmetic
// (FP64 runs at 1/64 of the FP32 rate on this part, and every float-double
// conversion is an FP64 instruction): each FP64 value of x and b is split
// by integer operations on its bits into a float pair h + l (48 bits),
// scaled by 2^es so that the values are of unit size, and
// r = b - sum_f alpha_f (x_c - x_nb) is formed with error-free float
// transformations (two-sum, FMA two-product). The absolute error is about
// 2^-44 max|x|, far below the refinement tolerance. c must be 1 (the solver's
// finest level is unit scale).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// d 2^es = h + l; values below 2^-74 after scaling become 0, values at or
// above 2^128 infinity (the solve then reports divergence), NaN stays NaN.
__device__ __forceinline__ void split_f64(double d, int es, float &h, float &l) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned sign = hi & 0x80000000u;
  const int ef = e - (1023 - 127) + es;  // float biased exponent of h
  if (e == 0x7ff) {
    h = __int_as_float((int)(sign | 0x7fc00000u));
    l = 0.f;
    return;
  }
  if (e == 0 || ef <= 0) {
    h = 0.f;
    l = 0.f;
    return;
  }
  if (ef >= 255) {
    h = __int_as_float((int)(sign | 0x7f800000u));
    l = 0.f;
    return;
  }
  // h: the leading 24 significant bits (truncated); l: the other 29, whose
  // unit is 2^(ef - 127 - 52)
  h = __int_as_float((int)(sign | ((unsigned)ef << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29)));
  const int pe = ef - 52;
  const float m = pe > 0 ? __uint2float_rn(lo & 0x1fffffffu) * __int_as_float(pe << 23) : 0.f;
  l = sign ? -m : m;
}

__global__ void k_residual_outer_df(LevelView<float> lv, const double *b,
                                    const double *x, float *rin, int es,
                                    float rscale, double scale, RedScratch rs,
                                    double *norm2) {
  pdl_wait();
  float acc = 0.f;
  const RowWalk w;
  const int nrows = lv.ny * lv.nz;
  const int nx = lv.nx, nxy = lv.nx * lv.ny;
  for (int row = w.warp; row < nrows; row += w.nwarps) {
    const int k = row / lv.ny, j = row - k * lv.ny;
    const int base = row * nx;
    for (int i = w.lane; i < nx; i += 32) {
      const int c = base + i;
      const int fy = c + k * nx;
      const float a[6] = {ld(lv.ax + c + row), ld(lv.ax + c + row + 1), ld(lv.ay + fy),
                          ld(lv.ay + fy + nx), ld(lv.az + c), ld(lv.az + c + nxy)};
      const bool has[6] = {i > 0, i < nx - 1, j > 0, j < lv.ny - 1, k > 0, k < lv.nz - 1};
      const int nb[6] = {c - 1, c + 1, c - nx, c + nx, c - nxy, c + nxy};
      float rv = 0.f;
      if (a[0] + a[1] + a[2] + a[3] + a[4] + a[5] > 0.f) {
        float ch, cl;
        split_f64(x[c], es, ch, cl);
        float S = 0.f, E = 0.f;  // sum_f alpha_f (x_c - x_nb) = S + E
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          if (a[f] == 0.f) continue;
          float nh = 0.f, nl = 0.f;
          if (has[f]) split_f64(x[nb[f]], es, nh, nl);
          float d, t;  // x_c - x_nb = d + t
          two_sum(ch, -nh, d, t);
          t = __fadd_rn(t, __fsub_rn(cl, nl));
          const float p = __fmul_rn(a[f], d);
          const float q = __fmaf_rn(a[f], t, __fmaf_rn(a[f], d, -p));
          float s2, e2;
          two_sum(S, p, s2, e2);
          S = s2;
          E = __fadd_rn(E, __fadd_rn(e2, q));
        }
        float bh, bl;
        split_f64(b[c], es, bh, bl);
        float rh, re;
        two_sum(bh, -S, rh, re);
        rv = __fadd_rn(rh, __fadd_rn(re, __fsub_rn(bl, E)));
      }
      const float ri = __fmul_rn(rv, rscale);
      rin[c] = ri;
      acc = __fmaf_rn(ri, ri, acc);
    }
  }
  double v[1] = {(double)acc}, tot[1];
  if (grid_sum<1>(v, rs, tot) && threadIdx.x == 0) *norm2 = tot[0] / (scale * scale);
}

template <class S, class V>
__global__ void __launch_bounds__(kBlock, sizeof(S) + sizeof(V) <= 12 ? 8 : 6)
k_axpy_outer(int64_t n, S *x, const V *e, double inv) {
  pdl_wait();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int U = kIlpStream;
  for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c0 < n;
       c0 += U * stride) {
    S xv[U];
    V ev[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) {
        xv[u] = x[c];
        ev[u] = e[c];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) x[c] = (S)((double)xv[u] + inv * widen_v(ev[u]));
    }
  }
}

// ------------------------------------------------------------------ CG -----
// Dots. Each thread accumulates its few grid-stride terms (2M cells over
// 151k threads: ~14), then the block and grid sums are FP64 in fixed order.
// FP32 vectors: every product is kept exactly as a float pair (p, e) with
// p + e = a b (FMA residual), and the thread's sum is compensated (two-sum,
// the rounding errors gathered in a second float), so a thread's partial
// carries about 48 significant bits, the error of an FP64 sum of these few
// terms, using FP32 instructions only: this part runs FP64 arithmetic (and
// float-to-double conversion) at 1/64 of the FP32 rate, and an FP64
// accumulation per element doubled the time of the dot kernels. The error
// of a partial is below 2^-46 of the sum of its terms' magnitudes. FP64
// vectors accumulate in FP64.
template <class V>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);  // a b = p + e exactly
    const float t = __fadd_rn(s, p);      // two-sum: s + p = t + err exactly
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <class V>
__global__ void __launch_bounds__(kBlock, 4) k_cg_init(int64_t n, const V *r, const V *z, V *d, CGState *st,
                          RedScratch rs) {
  pdl_wait();
  DotAcc<V> p0, p1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int U = kIlpStream;
  for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c0 < n;
       c0 += U * stride) {
    V rv[U], zv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) {
        rv[u] = r[c];
        zv[u] = z[c];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) {
        d[c] = zv[u];
        p0.add(rv[u], zv[u]);
        p1.add(rv[u], rv[u]);
      }
    }
  }
  double v[2] = {p0.value(), p1.value()};
  double tot[2];
  if (grid_sum<2>(v, rs, tot) && threadIdx.x == 0) {
    st->rz = tot[0];
    st->rr = tot[1];
    st->stop2 = st->tol * st->tol * tot[1];
    st->iters = 0;
    st->alpha = st->beta = st->dq = 0.0;
    st->done = (tot[1] == 0.0) ? 1 : (isfinite(tot[0]) && isfinite(tot[1]) ? 0 : 3);
    if (st->done == 0 && !(tot[0] > 0.0)) st->done = 2;
  }
}

template <class V>
__global__ void __launch_bounds__(kBlock, 4) k_cg_continue(int64_t n, const V *r, const V *z, CGState *st,
                              RedScratch rs) {
  pdl_wait();
  DotAcc<V> p0, p1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int U = kIlpStream;
  for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c0 < n;
       c0 += U * stride) {
    V rv[U], zv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) {
        rv[u] = r[c];
        zv[u] = z[c];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) {
        p0.add(rv[u], zv[u]);
        p1.add(rv[u], rv[u]);
      }
    }
  }
  double v[2] = {p0.value(), p1.value()};
  double tot[2];
  if (grid_sum<2>(v, rs, tot) && threadIdx.x == 0) {
    const double s = st->ratio, rz_old = st->rz * s * s;
    st->rr = tot[1];
    st->stop2 = st->tol * st->tol * tot[1];
    st->iters = 0;
    st->alpha = st->dq = 0.0;
    st->done = (tot[1] == 0.0) ? 1 : (isfinite(tot[0]) && isfinite(tot[1]) ? 0 : 3);
    if (st->done == 0 && !(tot[0] > 0.0 && rz_old > 0.0)) st->done = 2;
    // d = z + (s beta) d brings the old direction to the new scale
    st->beta = st->done == 0 ? tot[0] / rz_old * s : 0.0;
    st->rz = tot[0];
  }
}

template <class V, class TA>
__global__ void k_apply_dot(LevelView<TA> lv, const V *d, V *q, CGState *st,
                            RedScratch rs) {
  pdl_wait();
  const int stop = stop_flag(st);
  DotAcc<V> p;
  const RowWalk w;
  const int nrows = lv.ny * lv.nz;
  const V cc = V(lv.c);
  for (int row = w.warp; row < nrows; row += w.nwarps) {
    const int k = row / lv.ny, j = row - k * lv.ny;
    const int base = row * lv.nx;
    for (int i = w.lane; i < lv.nx; i += 32) {
      const int c = base + i;
      Nb7<V> g;
      gather7r(g, lv, d, i, j, k, c, row);
      const V dg = g.diag();
      const V qc = dg > V(0) ? cc * (dg * g.vc - g.nb()) : V(0);
      if (stop) return;
      q[c] = qc;
      p.add(g.vc, qc);
    }
  }
  if (stop) return;  // every thread of every block (none reaches the grid sum)
  double v[1] = {p.value()};
  double tot[1];
  if (grid_sum<1>(v, rs, tot) && threadIdx.x == 0) {
    st->dq = tot[0];
    if (tot[0] > 0.0 && isfinite(tot[0]))
      st->alpha = st->rz / tot[0];
    else
      st->done = isfinite(tot[0]) ? 2 : 3;
  }
}

template <class V>
__global__ void __launch_bounds__(kBlock, 4) k_cg_xr(int64_t n, V *x, V *r, const V *d, const V *q,
                        CGState *st, RedScratch rs, bool preconditioned, int loop,
                        LoopHandles h) {
  pdl_wait();
  const int stop = stop_flag(st);
  const V a = (V)st->alpha;
  DotAcc<V> p;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int U = kIlpStream;
  for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c0 < n;
       c0 += U * stride) {
    V xv[U], rv[U], dv[U], qv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) {
        xv[u] = x[c];
        rv[u] = r[c];
        dv[u] = d[c];
        qv[u] = q[c];
      }
    }
    if (stop) return;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) {
        x[c] = xv[u] + a * dv[u];
        const V rc = rv[u] - a * qv[u];
        r[c] = rc;
        p.add(rc, rc);
      }
    }
  }
  if (stop) return;  // every thread of every block (none reaches the grid sum)
  double v[1] = {p.value()};
  double tot[1];
  if (grid_sum<1>(v, rs, tot) && threadIdx.x == 0) {
    st->rr = tot[0];
    st->iters += 1;
    if (!isfinite(tot[0])) {
      st->done = 3;
    } else if (tot[0] <= st->stop2) {
      st->done = 1;
    } else if (!preconditioned) {
      st->beta = tot[0] / st->rz;
      st->rz = tot[0];
    }
    if (loop) {
      // in the device-side loop: the rest of the body runs only while the
      // solve runs; a finished (or abandoned) solve also ends the loop
      if (st->done || st->err) {
        cudaGraphSetConditional(h.body, 0u);
        cudaGraphSetConditional(h.tail, 0u);
      } else {
        cudaGraphSetConditional(h.tail, 1u);
      }
    }
  }
}

template <class V>
__global__ void __launch_bounds__(kBlock, 4) k_cg_rz(int64_t n, const V *r, const V *z, CGState *st,
                        RedScratch rs) {
  pdl_wait();
  const int stop = stop_flag(st);
  DotAcc<V> p;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int U = kIlpStream;
  for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c0 < n;
       c0 += U * stride) {
    V rv[U], zv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) {
        rv[u] = r[c];
        zv[u] = z[c];
      }
    }
    if (stop) return;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (c0 + u * stride < n) p.add(rv[u], zv[u]);
  }
  if (stop) return;  // every thread of every block (none reaches the grid sum)
  double v[1] = {p.value()};
  double tot[1];
  if (grid_sum<1>(v, rs, tot) && threadIdx.x == 0) {
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
      st->done = isfinite(tot[0]) ? 2 : 3;
    } else {
      st->beta = tot[0] / st->rz;
      st->rz = tot[0];
    }
  }
}

template <class V>
__global__ void __launch_bounds__(kBlock, 4) k_dot(int64_t n, const V *a, const V *b,
                                                   RedScratch rs, double *out) {
  DotAcc<V> p;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int U = kIlpStream;
  for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c0 < n;
       c0 += U * stride) {
    V av[U], bv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) {
        av[u] = a[c];
        bv[u] = b[c];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (c0 + u * stride < n) p.add(av[u], bv[u]);
  }
  double v[1] = {p.value()};
  double tot[1];
  if (grid_sum<1>(v, rs, tot) && threadIdx.x == 0) *out = tot[0];
}

template <class V>
__global__ void __launch_bounds__(kBlock, sizeof(V) == 4 ? 8 : 6) k_cg_d(int64_t n, const V *z, V *d, CGState *st, int loop,
                       cudaGraphConditionalHandle handle) {
  pdl_wait();
  const int stop = stop_flag(st);
  const V b = (V)st->beta;
  if (loop && blockIdx.x == 0 && threadIdx.x == 0) {
    // end of a body of the device-side loop: continue while the solve runs,
    // under its iteration budget, and the bodies stay below max_it + 4 (so
    // the loop ends even if no iteration is counted)
    const int loops = ++st->loops;
    const bool more = st->done == 0 && st->err == 0 && st->iters < st->max_it &&
                      loops < st->max_it + 4;
    cudaGraphSetConditional(handle, more ? 1u : 0u);
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int U = kIlpStream;
  for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c0 < n;
       c0 += U * stride) {
    V zv[U], dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) {
        zv[u] = z[c];
        dv[u] = d[c];
      }
    }
    if (stop) return;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * stride;
      if (c < n) d[c] = zv[u] + b * dv[u];
    }
  }
}

// ----------------------------------------------------------- multigrid -----
template <class TI, class TO>
__global__ void k_mg_coarsen(LevelView<TI> f, int cnx, int cny, int cnz, TO *ax,
                             TO *ay, TO *az) {
  const int64_t n0 = (int64_t)(cnx + 1) * cny * cnz;
  const int64_t n1 = (int64_t)cnx * (cny + 1) * cnz;
  const int64_t n2 = (int64_t)cnx * cny * (cnz + 1);
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  Lv F{f.nx, f.ny, f.nz};
  if (t < n0) {
    int I, J, K;
    GridDev::decomp(t, cnx + 1, cny, I, J, K);
    float s = 0.f;
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) s += (float)ld(f.ax + F.fx(2 * I, 2 * J + a, 2 * K + b));
    ax[t] = cvt<TO>(0.25 * s);
    return;
  }
  t -= n0;
  if (t < n1) {
    int I, J, K;
    GridDev::decomp(t, cnx, cny + 1, I, J, K);
    float s = 0.f;
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) s += (float)ld(f.ay + F.fy(2 * I + a, 2 * J, 2 * K + b));
    ay[t] = cvt<TO>(0.25 * s);
    return;
  }
  t -= n1;
  if (t < n2) {
    int I, J, K;
    GridDev::decomp(t, cnx, cny, I, J, K);
    float s = 0.f;
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) s += (float)ld(f.az + F.fz(2 * I + a, 2 * J + b, 2 * K));
    az[t] = cvt<TO>(0.25 * s);
  }
}

// ------------------------------------------------------ boundary band -----
// Cells next to the solid (an own face with alpha < 1) and their active
// neighbours get extra Gauss-Seidel sweeps: the coarse-grid correction is
// weakest there (cut cells, small fractions), so smoothing them alone buys
// most of what more full sweeps would.
template <class TA>
__global__ void k_band_mark(LevelView<TA> lv, unsigned char *m) {
  const int64_t n = lv.ncell();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    GridDev::decomp(c, lv.nx, lv.ny, i, j, k);
    const Six<float> s = six<float>(lv, i, j, k);
    const bool cut = s.xm < 1.f || s.xp < 1.f || s.ym < 1.f || s.yp < 1.f ||
                     s.zm < 1.f || s.zp < 1.f;
    m[c] = (s.diag() > 0.f && cut) ? 1 : 0;
  }
}

// Active cells marked or next to a marked cell, appended to the list of
// their colour (order does not matter: cells of one colour update
// independently).
template <class TA>
__global__ void k_band_collect(LevelView<TA> lv, const unsigned char *m,
                               int *list0, int *list1, int *count) {
  const int64_t n = lv.ncell();
  const int64_t sy = lv.nx, sz = (int64_t)lv.nx * lv.ny;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    GridDev::decomp(c, lv.nx, lv.ny, i, j, k);
    bool in = m[c] != 0;
    if (!in) {
      if (!(six<float>(lv, i, j, k).diag() > 0.f)) continue;
      in = (i > 0 && m[c - 1]) || (i < lv.nx - 1 && m[c + 1]) ||
           (j > 0 && m[c - sy]) || (j < lv.ny - 1 && m[c + sy]) ||
           (k > 0 && m[c - sz]) || (k < lv.nz - 1 && m[c + sz]);
    }
    if (!in) continue;
    const int col = (i + j + k) & 1;
    const int at = atomicAdd(count + col, 1);
    (col ? list1 : list0)[at] = (int)c;
  }
}

// Gauss-Seidel update of the band cells of one colour.
template <class V, class TA>
__global__ void k_band_smooth(LevelView<TA> lv, V *x, const V *b,
                              const int *list, const int *count,
                              const CGState *st) {
  if (stopped(st)) return;
  const int n = *count;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += gridDim.x * blockDim.x) {
    const int64_t c = list[t];
    int i, j, k;
    GridDev::decomp(c, lv.nx, lv.ny, i, j, k);
    x[c] = gs_cell<V, TA>(lv, x, b, i, j, k, c);
  }
}

// Neighbour values plus the prolonged coarse correction w x_c of their
// parents (constant transfer; the neighbours that exist).
template <class V>
__device__ __forceinline__ void add_fold(Nb7<V> &g, const Fold<V> &f, int nx, int ny,
                                         int nz, int i, int j, int k) {
  const int cxy = f.cnx * f.cny;
  const int pc = ((k >> 1) * f.cny + (j >> 1)) * f.cnx + (i >> 1);
  if (i > 0) g.vxm += f.xc[(i & 1) ? pc : pc - 1] * f.w;
  if (i < nx - 1) g.vxp += f.xc[(i & 1) ? pc + 1 : pc] * f.w;
  if (j > 0) g.vym += f.xc[(j & 1) ? pc : pc - f.cnx] * f.w;
  if (j < ny - 1) g.vyp += f.xc[(j & 1) ? pc + f.cnx : pc] * f.w;
  if (k > 0) g.vzm += f.xc[(k & 1) ? pc : pc - cxy] * f.w;
  if (k < nz - 1) g.vzp += f.xc[(k & 1) ? pc + cxy : pc] * f.w;
}

// New value of cell c = (i, j, k) (row = k ny + j) under a half sweep.
template <class V, class TA, int MODE>
__device__ __forceinline__ V sweep_cell(const LevelView<TA> &lv, const V *x,
                                        const V *b, int i, int j, int k, int c,
                                        int row, V cc, const Fold<V> &f) {
  if (MODE == kSweepZero) {
    const int nx = lv.nx, nxy = lv.nx * lv.ny, fy = c + k * nx;
    const V dg = (V)ld(lv.ax + c + row) + (V)ld(lv.ax + c + row + 1) + (V)ld(lv.ay + fy) +
                 (V)ld(lv.ay + fy + nx) + (V)ld(lv.az + c) + (V)ld(lv.az + c + nxy);
    return dg > V(0) ? b[c] / (cc * dg) : V(0);
  }
  Nb7<V> g;
  gather7r(g, lv, x, i, j, k, c, row);
  if (MODE == kSweepProlong) add_fold(g, f, lv.nx, lv.ny, lv.nz, i, j, k);
  const V dg = g.diag();
  return dg > V(0) ? (b[c] + cc * g.nb()) / (cc * dg) : V(0);
}

// Half sweep over the rows of a level, one warp per row (warps warp,
// warp + nwarps, ...; lanes along x).
template <class V, class TA, int MODE>
__device__ __forceinline__ void sweep_rows(const LevelView<TA> &lv, V *x,
                                           const V *b, int color,
                                           const Fold<V> &f, int warp,
                                           int nwarps, int lane, int stop = 0) {
  const int nrows = lv.ny * lv.nz;
  const int hx = (lv.nx + 1) >> 1;
  const V cc = V(lv.c);
  for (int row = warp; row < nrows; row += nwarps) {
    const int k = row / lv.ny, j = row - k * lv.ny;
    const int base = row * lv.nx;
    const int p = (j + k + color) & 1;
    for (int m = lane; m < hx; m += 32) {
      const int i = 2 * m + p;
      if (i >= lv.nx) continue;
      const int c = base + i;
      const V v = sweep_cell<V, TA, MODE>(lv, x, b, i, j, k, c, row, cc, f);
      if (stop) return;
      x[c] = v;
    }
  }
}

// Constant-transfer restriction of the residual of coarse cell (I, J, K)
// after pre-smoothing: the sum over its eight children of (b - A x). The
// last pre-smoothing half sweep updated the odd cells ((i + j + k) odd) from
// their even neighbours, which it did not change, so the residual of every
// odd cell is zero (up to the rounding of that update) and only the four
// even children are summed (inactive children add 0).
template <class V, class TA>
__device__ __forceinline__ V resrestrict_cell(const LevelView<TA> &lv,
                                              const V *x, const V *b, int I,
                                              int J, int K, V cc) {
  V acc = V(0);
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    // even children (a, b, c) = (0,0,0), (1,1,0), (1,0,1), (0,1,1)
    const int a = (ch == 1 || ch == 2), bb = (ch == 1 || ch == 3), cz = (ch >= 2);
    const int i = 2 * I + a, j = 2 * J + bb, k = 2 * K + cz;
    const int frow = k * lv.ny + j;
    const int c = frow * lv.nx + i;
    Nb7<V> g;
    gather7r(g, lv, x, i, j, k, c, frow);
    const V dg = g.diag();
    if (dg > V(0)) acc += b[c] - cc * (dg * g.vc - g.nb());
  }
  return acc;
}

// b_c = pn / 8 sum_children (b - A x) over the coarse rows of a level.
template <class V, class TA>
__device__ __forceinline__ void resrestrict_rows(const LevelView<TA> &lv,
                                                 const V *x, const V *b,
                                                 int cnx, int cny, int cnz,
                                                 V *bc, float pn, int warp,
                                                 int nwarps, int lane, int stop = 0) {
  const int nrows = cny * cnz;
  const V cc = V(lv.c);
  for (int row = warp; row < nrows; row += nwarps) {
    const int K = row / cny, J = row - K * cny;
    for (int I = lane; I < cnx; I += 32) {
      const V v = V(0.125) * V(pn) * resrestrict_cell<V, TA>(lv, x, b, I, J, K, cc);
      if (stop) return;
      bc[row * cnx + I] = v;
    }
  }
}

// Red-black Gauss-Seidel half sweep over cells with (i + j + k) % 2 == color.
template <class V, class TA, int MODE>
__global__ void k_mg_smooth(LevelView<TA> lv, V *x, const V *b, int color,
                            Fold<V> f, const CGState *st) {
  pdl_wait();
  const int stop = stop_flag(st);
  const RowWalk w;
  sweep_rows<V, TA, MODE>(lv, x, b, color, f, w.warp, w.nwarps, w.lane, stop);
}

// ------------------------------------------ fused red-black sweep pair -----
// One launch applies two half sweeps of a level: colour c1 in mode MODE
// (zero start, x as stored, or x with the folded constant prolongation),
// then colour 1 - c1 (x as just updated). Each block owns a TX x TY column
// of cells and marches up a chunk of planes, ZB planes per step, with the
// operands staged in shared memory:
//   - x (other colour of c1) over the tile plus a halo of two cells, read
//     once from xin (not at all in zero-start mode);
//   - b and the three fraction arrays over the tile plus one cell;
//   - in each step the loaded planes are written to shared memory, the next
//     ZB planes are requested into registers (their latency hides under the
//     sweeps), the first half sweep runs one plane behind the newest plane
//     over the tile plus one cell, and the second half sweep one plane
//     further behind over the tile, storing both colours of its planes.
// Both half sweeps read only the other colour, so cells of the halo are
// recomputed by each block that needs them (no exchange between blocks),
// and the result goes to xout (never xin: a neighbour block still reads
// the input halo). The per-cell arithmetic is that of sweep_cell, in the
// same order, so the pair equals two k_mg_smooth launches bit for bit.
// Loads: x 4 (x halo), b 4 + fractions 3 sizeof(TA) (halo 1); stores: x 4.
template <class V, class TA, int TX, int TY, int ZB>
struct RbPair {
  static constexpr int NT = 256;                   // threads per block
  static constexpr int XW = TX + 4, XH = TY + 4;   // x region (halo 2)
  static constexpr int BW = TX + 2, BH = TY + 2;   // b and z-face region (halo 1)
  static constexpr int AXW = TX + 3;               // x faces: one more column
  static constexpr int AYH = TY + 3;               // y faces: one more row
  static constexpr int NX = XW * XH, NB = BW * BH, NAX = AXW * BH, NAY = BW * AYH;
  static constexpr int DX = ZB + 3;                // planes of x kept
  static constexpr int DA = ZB + 2;                // planes of b and fractions kept
  // per-thread register slots of one batch of ZB planes
  static constexpr int MX = (ZB * NX + NT - 1) / NT;
  static constexpr int MB = (ZB * NB + NT - 1) / NT;
  static constexpr int MAX = (ZB * NAX + NT - 1) / NT;
  static constexpr int MAY = (ZB * NAY + NT - 1) / NT;
  static constexpr size_t off_b = (size_t)DX * NX * sizeof(V);
  static constexpr size_t off_ax = off_b + (size_t)DA * NB * sizeof(V);
  static constexpr size_t off_ay = off_ax + (size_t)DA * NAX * sizeof(TA);
  static constexpr size_t off_az = off_ay + (size_t)DA * NAY * sizeof(TA);
  static constexpr size_t bytes = off_az + (size_t)DA * NB * sizeof(TA);
  static_assert(TX % 2 == 0, "cells are swept in x pairs");
};

template <class V, class TA, int MODE, int TX, int TY, int ZB>
__global__ void __launch_bounds__(256, 2)
k_mg_rb_pair(LevelView<TA> lv, const V *xin, V *xout, const V *b, int c1, int zc,
             Fold<V> f, const CGState *st) {
  using C = RbPair<V, TA, TX, TY, ZB>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *sx = (V *)smem_raw;
  V *sb = (V *)(smem_raw + C::off_b);
  TA *sax = (TA *)(smem_raw + C::off_ax);
  TA *say = (TA *)(smem_raw + C::off_ay);
  TA *saz = (TA *)(smem_raw + C::off_az);
  pdl_wait();
  if (stop_flag(st)) return;  // every thread of the block

  const int nx = lv.nx, ny = lv.ny, nz = lv.nz, nxy = nx * ny;
  const int nbx = (nx + TX - 1) / TX, nby = (ny + TY - 1) / TY;
  const int bxi = blockIdx.x % nbx, rest = blockIdx.x / nbx;
  const int byi = rest % nby, bzi = rest / nby;
  const int x0 = bxi * TX, y0 = byi * TY, z0 = bzi * zc;
  const int z1 = min(z0 + zc, nz);
  const int c2 = c1 ^ 1;
  const V cc = V(lv.c);
  // ring slot of plane p (p >= -2 - ZB)
  auto slx = [](int p) { return (p + 4 * C::DX) % C::DX; };
  auto sla = [](int p) { return (p + 4 * C::DA) % C::DA; };

  // registers of one batch of planes [p0, p0 + ZB)
  V rx[C::MX], rb[C::MB];
  TA rax[C::MAX], ray[C::MAY], raz[C::MB];

  auto fetch = [&](int p0) {
    if (MODE != kSweepZero) {
#pragma unroll
      for (int m = 0; m < C::MX; ++m) {
        const int e = threadIdx.x + m * C::NT;
        V v = V(0);
        if (e < ZB * C::NX) {
          const int pz = e / C::NX, rem = e - pz * C::NX;
          const int r = rem / C::XW, col = rem - r * C::XW;
          const int gi = x0 - 2 + col, gj = y0 - 2 + r, gk = p0 + pz;
          // only the other colour of the first half sweep is read
          if (gi >= 0 && gi < nx && gj >= 0 && gj < ny && gk >= 0 && gk < nz &&
              ((gi + gj + gk) & 1) == c2) {
            v = xin[gk * nxy + gj * nx + gi];
            if (MODE == kSweepProlong)
              v += f.xc[((gk >> 1) * f.cny + (gj >> 1)) * f.cnx + (gi >> 1)] * f.w;
          }
        }
        rx[m] = v;
      }
    }
#pragma unroll
    for (int m = 0; m < C::MB; ++m) {
      const int e = threadIdx.x + m * C::NT;
      V v = V(0);
      TA a = TA(0.f);
      if (e < ZB * C::NB) {
        const int pz = e / C::NB, rem = e - pz * C::NB;
        const int r = rem / C::BW, col = rem - r * C::BW;
        const int gi = x0 - 1 + col, gj = y0 - 1 + r, gk = p0 + pz;
        if (gi >= 0 && gi < nx && gj >= 0 && gj < ny && gk >= 0 && gk <= nz) {
          if (gk < nz) v = b[gk * nxy + gj * nx + gi];
          a = lv.az[gk * nxy + gj * nx + gi];
        }
      }
      rb[m] = v;
      raz[m] = a;
    }
#pragma unroll
    for (int m = 0; m < C::MAX; ++m) {
      const int e = threadIdx.x + m * C::NT;
      TA a = TA(0.f);
      if (e < ZB * C::NAX) {
        const int pz = e / C::NAX, rem = e - pz * C::NAX;
        const int r = rem / C::AXW, col = rem - r * C::AXW;
        const int gi = x0 - 1 + col, gj = y0 - 1 + r, gk = p0 + pz;
        if (gi >= 0 && gi <= nx && gj >= 0 && gj < ny && gk >= 0 && gk < nz)
          a = lv.ax[(gk * ny + gj) * (nx + 1) + gi];
      }
      rax[m] = a;
    }
#pragma unroll
    for (int m = 0; m < C::MAY; ++m) {
      const int e = threadIdx.x + m * C::NT;
      TA a = TA(0.f);
      if (e < ZB * C::NAY) {
        const int pz = e / C::NAY, rem = e - pz * C::NAY;
        const int r = rem / C::BW, col = rem - r * C::BW;
        const int gi = x0 - 1 + col, gj = y0 - 1 + r, gk = p0 + pz;
        if (gi >= 0 && gi < nx && gj >= 0 && gj <= ny && gk >= 0 && gk < nz)
          a = lv.ay[(gk * (ny + 1) + gj) * nx + gi];
      }
      ray[m] = a;
    }
  };

  auto stage = [&](int p0) {
    if (MODE != kSweepZero) {
#pragma unroll
      for (int m = 0; m < C::MX; ++m) {
        const int e = threadIdx.x + m * C::NT;
        if (e < ZB * C::NX) {
          const int pz = e / C::NX, rem = e - pz * C::NX;
          sx[slx(p0 + pz) * C::NX + rem] = rx[m];
        }
      }
    } else {
      // zero start: the other colour is 0 wherever the first half sweep reads it
      for (int e = threadIdx.x; e < ZB * C::NX; e += C::NT) {
        const int pz = e / C::NX, rem = e - pz * C::NX;
        sx[slx(p0 + pz) * C::NX + rem] = V(0);
      }
    }
#pragma unroll
    for (int m = 0; m < C::MB; ++m) {
      const int e = threadIdx.x + m * C::NT;
      if (e < ZB * C::NB) {
        const int pz = e / C::NB, rem = e - pz * C::NB;
        sb[sla(p0 + pz) * C::NB + rem] = rb[m];
        saz[sla(p0 + pz) * C::NB + rem] = raz[m];
      }
    }
#pragma unroll
    for (int m = 0; m < C::MAX; ++m) {
      const int e = threadIdx.x + m * C::NT;
      if (e < ZB * C::NAX) {
        const int pz = e / C::NAX, rem = e - pz * C::NAX;
        sax[sla(p0 + pz) * C::NAX + rem] = rax[m];
      }
    }
#pragma unroll
    for (int m = 0; m < C::MAY; ++m) {
      const int e = threadIdx.x + m * C::NT;
      if (e < ZB * C::NAY) {
        const int pz = e / C::NAY, rem = e - pz * C::NAY;
        say[sla(p0 + pz) * C::NAY + rem] = ray[m];
      }
    }
  };

  // The 13 operands of cell (gi, gj, q) from shared memory; neighbours
  // outside the level read the staged zeros (ghost x = 0), as gather7r.
  auto gather = [&](Nb7<V> &g, V &bc, int gi, int gj, int q) {
    const int lx = gi - (x0 - 2), ly = gj - (y0 - 2);
    const int bx = gi - (x0 - 1), by = gj - (y0 - 1);
    const int a0 = sla(q), a1 = sla(q + 1);
    g.xm = (V)ld(sax + a0 * C::NAX + by * C::AXW + bx);
    g.xp = (V)ld(sax + a0 * C::NAX + by * C::AXW + bx + 1);
    g.ym = (V)ld(say + a0 * C::NAY + by * C::BW + bx);
    g.yp = (V)ld(say + a0 * C::NAY + (by + 1) * C::BW + bx);
    g.zm = (V)ld(saz + a0 * C::NB + by * C::BW + bx);
    g.zp = (V)ld(saz + a1 * C::NB + by * C::BW + bx);
    const V *xq = sx + slx(q) * C::NX + ly * C::XW + lx;
    g.vxm = xq[-1];
    g.vxp = xq[1];
    g.vym = xq[-C::XW];
    g.vyp = xq[C::XW];
    g.vzm = sx[slx(q - 1) * C::NX + ly * C::XW + lx];
    g.vzp = sx[slx(q + 1) * C::NX + ly * C::XW + lx];
    bc = sb[a0 * C::NB + by * C::BW + bx];
  };

  const int s1lo = max(z0 - 1, 0), s1hi = min(z1, nz - 1);  // first half sweep planes
  fetch(z0 - 2);
  for (int p0 = z0 - 2; p0 - 2 < z1; p0 += ZB) {
    __syncthreads();  // the previous step's sweeps are done with the slots reused here
    stage(p0);
    __syncthreads();
    if (p0 + ZB <= z1 + 1) fetch(p0 + ZB);
    // first half sweep: colour c1 on planes p0 - 1 .. p0 + ZB - 2, tile + 1
    for (int e = threadIdx.x; e < ZB * C::BH * (C::BW / 2); e += C::NT) {
      const int pz = e / (C::BH * (C::BW / 2)), rem = e - pz * (C::BH * (C::BW / 2));
      const int r = rem / (C::BW / 2), m = rem - r * (C::BW / 2);
      const int q = p0 - 1 + pz, gj = y0 - 1 + r;
      const int gi = x0 - 1 + 2 * m + ((c1 + x0 + 1 + gj + q) & 1);
      if (q < s1lo || q > s1hi || gj < 0 || gj >= ny || gi < 0 || gi >= nx) continue;
      Nb7<V> g;
      V bc;
      gather(g, bc, gi, gj, q);
      const V dg = g.diag();
      V v;
      if (MODE == kSweepZero)
        v = dg > V(0) ? bc / (cc * dg) : V(0);
      else
        v = dg > V(0) ? (bc + cc * g.nb()) / (cc * dg) : V(0);
      sx[slx(q) * C::NX + (gj - (y0 - 2)) * C::XW + (gi - (x0 - 2))] = v;
    }
    __syncthreads();
    // second half sweep: colour c2 on planes p0 - 2 .. p0 + ZB - 3, tile;
    // each thread stores one cell pair of a row
    for (int e = threadIdx.x; e < ZB * TY * (TX / 2); e += C::NT) {
      const int pz = e / (TY * (TX / 2)), rem = e - pz * (TY * (TX / 2));
      const int r = rem / (TX / 2), m = rem - r * (TX / 2);
      const int q = p0 - 2 + pz, gj = y0 + r;
      if (q < z0 || q >= z1 || gj >= ny) continue;
      const int par = (c2 + x0 + gj + q) & 1;
      const int gi2 = x0 + 2 * m + par, gi1 = x0 + 2 * m + (par ^ 1);
      V v = V(0);
      if (gi2 < nx) {
        Nb7<V> g;
        V bc;
        gather(g, bc, gi2, gj, q);
        const V dg = g.diag();
        v = dg > V(0) ? (bc + cc * g.nb()) / (cc * dg) : V(0);
      }
      const int row = q * nxy + gj * nx;
      if (gi1 < nx)
        xout[row + gi1] = sx[slx(q) * C::NX + (gj - (y0 - 2)) * C::XW + (gi1 - (x0 - 2))];
      if (gi2 < nx) xout[row + gi2] = v;
    }
  }
}

// Prolongation normaliser of fine cell (i, j, k): 1 / (sum of the trilinear
// weights of its active coarse cells), 0 if none is active. The V-cycle uses
// P' = N P and R' = P'^T / 4 = P^T N / 4: near a Neumann (solid) boundary the
// plain trilinear P would mix in inactive coarse cells, whose value is 0, and
// damp the correction as if the wall were a zero-pressure boundary.
template <class TC>
__device__ __forceinline__ float pnorm_cell(const LevelView<TC> &cv, int i,
                                            int j, int k) {
  int I[2], J[2], K[2];
  auto ax = [](int f, int n, int *C) {
    const int c0 = f >> 1;
    int c1 = (f & 1) ? c0 + 1 : c0 - 1;
    if (c1 < 0 || c1 >= n) c1 = c0;
    C[0] = c0;
    C[1] = c1;
  };
  ax(i, cv.nx, I);
  ax(j, cv.ny, J);
  ax(k, cv.nz, K);
  const float w[2] = {0.75f, 0.25f};
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a)
        if (six<float>(cv, I[a], J[b], K[c]).diag() > 0.f) s += w[c] * w[b] * w[a];
  return s > 0.f ? 1.f / s : 0.f;
}

template <class TC>
__global__ void k_mg_pnorm(int fnx, int fny, int fnz, LevelView<TC> cv, float *pn,
                           float scale) {
  const int64_t n = (int64_t)fnx * fny * fnz;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    GridDev::decomp(c, fnx, fny, i, j, k);
    pn[c] = scale * pnorm_cell(cv, i, j, k);
  }
}

template <class V, class TA>
__global__ void k_mg_residual(LevelView<TA> lv, const V *x, const V *b, V *r,
                              const float *pn, const CGState *st) {
  if (stopped(st)) return;
  const RowWalk w;
  const int nrows = lv.ny * lv.nz;
  const V cc = V(lv.c);
  for (int row = w.warp; row < nrows; row += w.nwarps) {
    const int k = row / lv.ny, j = row - k * lv.ny;
    const int base = row * lv.nx;
    for (int i = w.lane; i < lv.nx; i += 32) {
      const int c = base + i;
      Nb7<V> g;
      gather7r(g, lv, x, i, j, k, c, row);
      const V dg = g.diag();
      const V rv = dg > V(0) ? b[c] - cc * (dg * g.vc - g.nb()) : V(0);
      r[c] = pn ? rv * V(pn[c]) : rv;
    }
  }
}

template <class V>
__global__ void k_mg_restrict(int fnx, int fny, int fnz, int cnx, int cny,
                              int cnz, const V *rf, V *bc, int mode,
                              const CGState *st) {
  if (stopped(st)) return;
  const RowWalk w;
  const int nrows = cny * cnz;
  for (int row = w.warp; row < nrows; row += w.nwarps) {
    const int K = row / cny, J = row - K * cny;
    const int base = row * cnx;
    for (int I = w.lane; I < cnx; I += 32) {
      if (mode == kTransferConstant) {
        // mean of the eight children (fine dims are twice the coarse ones)
        const int f0 = ((2 * K) * fny + 2 * J) * fnx + 2 * I;
        const int sy = fnx, sz = fnx * fny;
        const V s = rf[f0] + rf[f0 + 1] + rf[f0 + sy] + rf[f0 + sy + 1] + rf[f0 + sz] +
                    rf[f0 + sz + 1] + rf[f0 + sz + sy] + rf[f0 + sz + sy + 1];
        bc[base + I] = V(0.125) * s;
      } else {
        bc[base + I] = restrict_cell<V>(fnx, fny, fnz, cnx, cny, cnz, rf, I, J, K, mode);
      }
    }
  }
}

// Fused residual and restriction for the constant transfer: every coarse
// cell adds the residuals of its eight children (times the normaliser pn,
// here the uniform sqrt of the coarse weight) without storing the fine
// residual: b_c = pn / 8 sum_children (b - A x).
template <class V, class TA>
__global__ void k_mg_resrestrict(LevelView<TA> lv, const V *x, const V *b,
                                 int cnx, int cny, int cnz, V *bc, float pn,
                                 const CGState *st) {
  pdl_wait();
  const int stop = stop_flag(st);
  const RowWalk w;
  resrestrict_rows<V, TA>(lv, x, b, cnx, cny, cnz, bc, pn, w.warp, w.nwarps, w.lane, stop);
}

// x_f += P x_c on active fine cells.
template <class V, class TF>
__global__ void k_mg_prolong(LevelView<TF> f, int cnx, int cny, int cnz,
                             const V *xc, V *xf, const float *pn, int mode,
                             const CGState *st) {
  if (stopped(st)) return;
  const RowWalk w;
  const int nrows = f.ny * f.nz;
  const int nx = f.nx, nxy = f.nx * f.ny;
  for (int row = w.warp; row < nrows; row += w.nwarps) {
    const int k = row / f.ny, j = row - k * f.ny;
    const int base = row * nx;
    for (int i = w.lane; i < nx; i += 32) {
      const int c = base + i;
      const int fy = c + k * nx;
      const float dg = (float)ld(f.ax + c + row) + (float)ld(f.ax + c + row + 1) +
                       (float)ld(f.ay + fy) + (float)ld(f.ay + fy + nx) +
                       (float)ld(f.az + c) + (float)ld(f.az + c + nxy);
      if (!(dg > 0.f)) continue;
      V add = prolong_cell<V>(cnx, cny, cnz, xc, i, j, k, mode);
      if (pn) add *= V(pn[c]);
      xf[c] += add;
    }
  }
}

// One thread block runs the V-cycle on all small levels of the chain. Global
// memory writes are made visible to the block by __syncthreads().
template <class V, class TA>
__device__ void blk_smooth(const LevelView<TA> &lv, V *x, const V *b,
                           int color) {
  const int hx = (lv.nx + 1) >> 1;
  const int n = hx * lv.ny * lv.nz;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int ii = t % hx, q = t / hx;
    const int j = q % lv.ny, k = q / lv.ny;
    const int i = 2 * ii + ((j + k + color) & 1);
    if (i >= lv.nx) continue;
    const int64_t c = ((int64_t)k * lv.ny + j) * lv.nx + i;
    x[c] = gs_cell<V, TA>(lv, x, b, i, j, k, c);
  }
  __syncthreads();
}

template <class V, class TA>
__global__ void __launch_bounds__(1024, 1)
k_mg_coarse_chain(CoarseChain<V, TA> ch, const CGState *st) {
  if (stopped(st)) return;
  const int last = ch.nlev - 1;
  for (int l = ch.first; l <= last; ++l) {
    const LevelView<TA> &lv = ch.lv[l];
    const int n = (int)lv.ncell();
    for (int t = threadIdx.x; t < n; t += blockDim.x) ch.x[l][t] = V(0);
    __syncthreads();
    if (l == last) break;
    for (int s = 0; s < ch.smooth; ++s) {
      blk_smooth(lv, ch.x[l], ch.b[l], 0);
      blk_smooth(lv, ch.x[l], ch.b[l], 1);
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int i = t % lv.nx, q = t / lv.nx;
      const int j = q % lv.ny, k = q / lv.ny;
      ch.r[l][t] = residual_cell<V, TA>(lv, ch.x[l], ch.b[l], i, j, k, t) * V(ch.pn[l][t]);
    }
    __syncthreads();
    const LevelView<TA> &cv = ch.lv[l + 1];
    const int nc = (int)cv.ncell();
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
      const int I = t % cv.nx, q = t / cv.nx;
      const int J = q % cv.ny, K = q / cv.ny;
      ch.b[l + 1][t] = restrict_cell<V>(lv.nx, lv.ny, lv.nz, cv.nx, cv.ny,
                                        cv.nz, ch.r[l], I, J, K, ch.transfer);
    }
    __syncthreads();
  }
  {
    const LevelView<TA> &lv = ch.lv[last];
    for (int s = 0; s < ch.coarsest_sweeps; ++s) {
      blk_smooth(lv, ch.x[last], ch.b[last], 0);
      blk_smooth(lv, ch.x[last], ch.b[last], 1);
    }
    for (int s = 0; s < ch.coarsest_sweeps; ++s) {
      blk_smooth(lv, ch.x[last], ch.b[last], 1);
      blk_smooth(lv, ch.x[last], ch.b[last], 0);
    }
  }
  for (int l = last - 1; l >= ch.first; --l) {
    const LevelView<TA> &lv = ch.lv[l];
    const LevelView<TA> &cv = ch.lv[l + 1];
    const int n = (int)lv.ncell();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int i = t % lv.nx, q = t / lv.nx;
      const int j = q % lv.ny, k = q / lv.ny;
      if (six<float>(lv, i, j, k).diag() > 0.f)
        ch.x[l][t] += prolong_cell<V>(cv.nx, cv.ny, cv.nz, ch.x[l + 1], i, j, k,
                                      ch.transfer) *
                      V(ch.pn[l][t]);
    }
    __syncthreads();
    for (int s = 0; s < ch.smooth; ++s) {
      blk_smooth(lv, ch.x[l], ch.b[l], 1);
      blk_smooth(lv, ch.x[l], ch.b[l], 0);
    }
  }
}

// Shared-memory version of the chain: every array of the chain levels (x, b,
// the fractions, the inverse diagonal, and r for the trilinear transfer)
// lives in shared memory for the whole sub-V-cycle; global memory is read
// once (fractions, b of the first chain level) and written once (x of the
// first chain level).
// Fractions keep their storage type in shared memory, so that they arrive
// by bulk copies (converted at every read, one instruction for BF16).
template <class TA>
struct ChainFA {
  using type = TA;
};

// Byte offsets of x, b, r, ax, ay, az and the inverse diagonal of every
// chain level; returns the total.
template <class V, class TA>
__host__ __device__ inline size_t chain_layout(const CoarseChain<V, TA> &ch,
                                               size_t off[kMaxLevels][7]) {
  using FA = typename ChainFA<TA>::type;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o += (bytes + 15) & ~(size_t)15;
    return at;
  };
  const bool need_r = ch.transfer != kTransferConstant;  // the fused restriction needs none
  for (int l = ch.first; l < ch.nlev; ++l) {
    const LevelView<TA> &v = ch.lv[l];
    const size_t nc = (size_t)v.nx * v.ny * v.nz;
    off[l][0] = take(nc * sizeof(V));
    off[l][1] = take(nc * sizeof(V));
    off[l][2] = take(need_r && l + 1 < ch.nlev ? nc * sizeof(V) : 0);
    off[l][3] = take((size_t)(v.nx + 1) * v.ny * v.nz * sizeof(FA));
    off[l][4] = take((size_t)v.nx * (v.ny + 1) * v.nz * sizeof(FA));
    off[l][5] = take((size_t)v.nx * v.ny * (v.nz + 1) * sizeof(FA));
    off[l][6] = take(nc * sizeof(V));
  }
  return o;
}

// t / d for t < 2^17 and d < 2^15 as a multiply-high: with m = ceil(2^32 / d)
// the error term t (m d - 2^32) / 2^32 stays below 1 / d.
struct UDiv {
  unsigned d, m;
  __device__ __forceinline__ unsigned q(unsigned t) const {
    return d == 1u ? t : __umulhi(t, m);
  }
};
__device__ __forceinline__ UDiv make_udiv(unsigned d) {
  return UDiv{d, d == 1u ? 0u : 0xFFFFFFFFu / d + 1u};
}

// One block-resident chain level: arrays in shared memory (the fractions
// as FA), the inverse diagonal 1 / (c dg) (0 on inactive cells) and the
// divisions of its index arithmetic.
template <class V, class FA>
struct CLev {
  LevelView<FA> lv;
  V *x, *b, *dinv;
  UDiv hx, ny;  // half row (cells of one colour per row), rows per plane
};

// Half sweep of a chain level over the cells t0, t0 + stride, ... of one
// colour: x = (b + c nb) / (c dg) with the division replaced by dinv.
template <class V, class FA, int MODE>
__device__ __forceinline__ void csweep_cells(const CLev<V, FA> &L, int color,
                                             const Fold<V> &f, unsigned t0,
                                             unsigned stride) {
  const unsigned n = L.hx.d * L.ny.d * (unsigned)L.lv.nz;
  const V cc = V(L.lv.c);
  for (unsigned t = t0; t < n; t += stride) {
    const unsigned row = L.hx.q(t), m = t - row * L.hx.d;
    const unsigned k = L.ny.q(row), j = row - k * L.ny.d;
    const int i = (int)(2 * m + ((j + k + color) & 1));
    if (i >= L.lv.nx) continue;
    const int c = (int)row * L.lv.nx + i;
    if (MODE == kSweepZero) {
      L.x[c] = L.b[c] * L.dinv[c];
      continue;
    }
    Nb7<V> g;
    gather7r(g, L.lv, L.x, i, (int)j, (int)k, c, (int)row);
    if (MODE == kSweepProlong) add_fold(g, f, L.lv.nx, L.lv.ny, L.lv.nz, i, (int)j, (int)k);
    L.x[c] = (L.b[c] + cc * g.nb()) * L.dinv[c];
  }
}
template <class V, class FA, int MODE>
__device__ __forceinline__ void blk_sweep(const CLev<V, FA> &L, int color,
                                          const Fold<V> &f) {
  csweep_cells<V, FA, MODE>(L, color, f, threadIdx.x, blockDim.x);
  __syncthreads();
}

// b_c = pn / 8 sum_children (b - A x) for every cell of a block-resident
// coarse level (even children only: see resrestrict_cell).
template <class V, class FA>
__device__ void blk_resrestrict(const CLev<V, FA> &L, int cnx, int cny, int cnz, V *bc,
                                float pn) {
  const UDiv ux = make_udiv((unsigned)cnx), uy = make_udiv((unsigned)cny);
  const unsigned n = (unsigned)cnx * cny * cnz;
  const V cc = V(L.lv.c);
  for (unsigned t = threadIdx.x; t < n; t += blockDim.x) {
    const unsigned q = ux.q(t), I = t - q * cnx;
    const unsigned K = uy.q(q), J = q - K * cny;
    bc[t] = V(0.125) * V(pn) * resrestrict_cell<V, FA>(L.lv, L.x, L.b, (int)I, (int)J, (int)K, cc);
  }
  __syncthreads();
}

// The coarsest level's symmetric sweeps when each colour has at most 32
// cells: one warp, each lane keeps its cell of each colour (fractions,
// neighbour indices, dinv, b) in registers; only x lives in shared memory.
template <class V, class FA>
__device__ void warp_coarsest(const CLev<V, FA> &L, int sweeps) {
  const unsigned lane = threadIdx.x & 31u;
  const int nx = L.lv.nx, ny = L.lv.ny, nz = L.lv.nz, nxy = nx * ny;
  const unsigned n = L.hx.d * L.ny.d * (unsigned)nz;
  const V cc = V(L.lv.c);
  int cell[2], nb[2][6];
  V a[2][6], di[2], bv[2];
#pragma unroll
  for (int col = 0; col < 2; ++col) {
    cell[col] = -1;
    const unsigned t = lane;
    const unsigned row = L.hx.q(t), m = t - row * L.hx.d;
    const unsigned k = L.ny.q(row), j = row - k * L.ny.d;
    const int i = (int)(2 * m + ((j + k + col) & 1));
    if (t < n && i < nx) {
      const int c = (int)row * nx + i, fy = c + (int)k * nx;
      cell[col] = c;
      a[col][0] = (V)ld(L.lv.ax + c + row);
      a[col][1] = (V)ld(L.lv.ax + c + row + 1);
      a[col][2] = (V)ld(L.lv.ay + fy);
      a[col][3] = (V)ld(L.lv.ay + fy + nx);
      a[col][4] = (V)ld(L.lv.az + c);
      a[col][5] = (V)ld(L.lv.az + c + nxy);
      nb[col][0] = i > 0 ? c - 1 : -1;
      nb[col][1] = i < nx - 1 ? c + 1 : -1;
      nb[col][2] = (int)j > 0 ? c - nx : -1;
      nb[col][3] = (int)j < ny - 1 ? c + nx : -1;
      nb[col][4] = (int)k > 0 ? c - nxy : -1;
      nb[col][5] = (int)k < nz - 1 ? c + nxy : -1;
      di[col] = L.dinv[c];
      bv[col] = L.b[c];
    }
  }
  auto update = [&](int col, bool zero) {
    if (cell[col] < 0) return;
    V acc = V(0);
    if (!zero) {
#pragma unroll
      for (int q = 0; q < 6; ++q) acc += a[col][q] * (nb[col][q] >= 0 ? L.x[nb[col][q]] : V(0));
    }
    L.x[cell[col]] = (bv[col] + cc * acc) * di[col];
  };
  for (int s = 0; s < sweeps; ++s) {
    update(0, s == 0);
    __syncwarp();
    update(1, false);
    __syncwarp();
  }
  for (int s = 0; s < sweeps; ++s) {
    update(1, false);
    __syncwarp();
    update(0, false);
    __syncwarp();
  }
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Every bounded wait on the device (grid barriers, mbarriers) gives up
// after this long.
constexpr unsigned long long kBarrierNs = 1000000000ull;

// Bounded wait for phase `parity` of an mbarrier: true once it completed;
// after kBarrierNs sets *err (when given) and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned mb, unsigned parity, int *err) {
  unsigned long long t0 = 0;
  unsigned spins = 0;
  for (;;) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((++spins & 255u) == 0) {
      const unsigned long long t = globaltimer_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > kBarrierNs) {
        if (err) atomicExch(err, 1);
        return false;
      }
    }
  }
}

// The chain's whole sub-V-cycle by one thread block in `smem` (at least
// mg_chain_smem_bytes). Reads b of the first chain level and writes its x
// (global memory); every other array stays in shared memory. With the
// constant transfer the residual is restricted in one pass and the
// prolongation is folded into the first post-smoothing half sweep.
template <class V, class TA>
__device__ void chain_body(const CoarseChain<V, TA> &ch, unsigned char *smem) {
  using FA = typename ChainFA<TA>::type;
  // a bounded wait expired: the solve is being abandoned (decided by the
  // whole block, since another block may set the word meanwhile)
  if (__syncthreads_or(ch.err != nullptr && *(volatile int *)ch.err != 0)) return;
  __shared__ unsigned soff[kMaxLevels][7];
  __shared__ UDiv sdiv[kMaxLevels][2];
  __shared__ const TA *seg_src[3 * kMaxLevels];
  __shared__ unsigned seg_dst[3 * kMaxLevels], seg_end[3 * kMaxLevels];
  const int first = ch.first, last = ch.nlev - 1;
  const int nseg = 3 * (last - first + 1);
  if (threadIdx.x == 0) {
    size_t off[kMaxLevels][7];
    chain_layout(ch, off);
    unsigned e = 0;
    for (int l = first; l <= last; ++l) {
      const LevelView<TA> &g = ch.lv[l];
      for (int q = 0; q < 7; ++q) soff[l][q] = (unsigned)off[l][q];
      sdiv[l][0] = make_udiv((unsigned)(g.nx + 1) >> 1);
      sdiv[l][1] = make_udiv((unsigned)g.ny);
      const int s0 = 3 * (l - first);
      const TA *src[3] = {g.ax, g.ay, g.az};
      const unsigned cnt[3] = {(unsigned)((g.nx + 1) * g.ny * g.nz),
                               (unsigned)(g.nx * (g.ny + 1) * g.nz),
                               (unsigned)(g.nx * g.ny * (g.nz + 1))};
      for (int q = 0; q < 3; ++q) {
        seg_src[s0 + q] = src[q];
        seg_dst[s0 + q] = soff[l][3 + q];
        e += cnt[q];
        seg_end[s0 + q] = e;
      }
    }
  }
  __syncthreads();
  const bool fused = ch.transfer == kTransferConstant;
  auto lev = [&](int l) {
    const LevelView<TA> &g = ch.lv[l];
    CLev<V, FA> L;
    L.lv = LevelView<FA>{g.nx, g.ny, g.nz, g.c, (const FA *)(smem + soff[l][3]),
                         (const FA *)(smem + soff[l][4]), (const FA *)(smem + soff[l][5])};
    L.x = (V *)(smem + soff[l][0]);
    L.b = (V *)(smem + soff[l][1]);
    L.dinv = (V *)(smem + soff[l][6]);
    L.hx = sdiv[l][0];
    L.ny = sdiv[l][1];
    return L;
  };
  auto R = [&](int l) { return (V *)(smem + soff[l][2]); };
  const Fold<V> none{nullptr, 0, 0, V(0)};
  // global -> shared: thread 0 issues a bulk copy of every 16-byte-aligned
  // array (b of the first level, the fractions of every level), tracked by
  // one mbarrier; ragged tails and unaligned arrays are copied by plain
  // loads meanwhile
  {
    __shared__ __align__(8) unsigned long long mbar;
    const unsigned mb = (unsigned)__cvta_generic_to_shared(&mbar);
    const int nb0 = (int)ch.lv[first].ncell();
    V *bs = (V *)(smem + soff[first][1]);
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // bytes a bulk copy takes: both addresses 16-byte aligned, a multiple of 16
    auto bulk_bytes = [](const void *dst, const void *src, unsigned bytes) {
      return (((uintptr_t)src | (uintptr_t)__cvta_generic_to_shared(dst)) & 15u) ? 0u
                                                                               : (bytes & ~15u);
    };
    if (threadIdx.x == 0) {
      unsigned tx = bulk_bytes(bs, ch.b[first], (unsigned)(nb0 * sizeof(V))) + 16u * ch.stall;
      for (int sg = 0; sg < nseg; ++sg) {
        const unsigned cnt = seg_end[sg] - (sg ? seg_end[sg - 1] : 0u);
        tx += bulk_bytes(smem + seg_dst[sg], seg_src[sg], cnt * (unsigned)sizeof(TA));
      }
      // b may have been written by other CTAs of a cluster (generic stores
      // made visible by a cluster barrier): order them before the copies
      asm volatile("fence.proxy.async.global;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(tx)
                   : "memory");
      auto issue = [&](void *dst, const void *src, unsigned bytes) {
        const unsigned nbulk = bulk_bytes(dst, src, bytes);
        if (nbulk == 0) return;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
            "l"(src), "r"(nbulk), "r"(mb)
            : "memory");
      };
      issue(bs, ch.b[first], (unsigned)(nb0 * sizeof(V)));
      for (int sg = 0; sg < nseg; ++sg) {
        const unsigned cnt = seg_end[sg] - (sg ? seg_end[sg - 1] : 0u);
        issue(smem + seg_dst[sg], seg_src[sg], cnt * (unsigned)sizeof(TA));
      }
    }
    {
      const unsigned done0 = bulk_bytes(bs, ch.b[first], (unsigned)(nb0 * sizeof(V))) / sizeof(V);
      for (int t = (int)done0 + threadIdx.x; t < nb0; t += blockDim.x) bs[t] = ch.b[first][t];
      for (int sg = 0; sg < nseg; ++sg) {
        const unsigned cnt = seg_end[sg] - (sg ? seg_end[sg - 1] : 0u);
        TA *dst = (TA *)(smem + seg_dst[sg]);
        const unsigned done = bulk_bytes(dst, seg_src[sg], cnt * (unsigned)sizeof(TA)) / sizeof(TA);
        for (unsigned t = done + threadIdx.x; t < cnt; t += blockDim.x) dst[t] = seg_src[sg][t];
      }
    }
    // the block decides together (a wait that expired in one thread ends the
    // chain in all of them); copies still in flight land (bounded) first
    const bool landed = mbar_wait(mb, 0, ch.err);
    if (!__syncthreads_and(landed)) {
      mbar_wait(mb, 0, nullptr);
      return;
    }
  }
  // inverse diagonals of every chain level
  for (int l = first; l <= last; ++l) {
    const CLev<V, FA> L = lev(l);
    const UDiv ux = make_udiv((unsigned)L.lv.nx);
    const unsigned n = (unsigned)L.lv.ncell();
    const V cc = V(L.lv.c);
    for (unsigned t = threadIdx.x; t < n; t += blockDim.x) {
      const unsigned row = ux.q(t), i = t - row * L.lv.nx;
      const unsigned k = L.ny.q(row), j = row - k * L.ny.d;
      const Six<V> sx = six<V>(L.lv, (int)i, (int)j, (int)k);
      const V dg = sx.diag();
      L.dinv[t] = dg > V(0) ? V(1) / (cc * dg) : V(0);
    }
  }
  __syncthreads();
  for (int l = first; l < last; ++l) {
    const CLev<V, FA> L = lev(l);
    for (int s = 0; s < ch.smooth; ++s) {
      if (s == 0)
        blk_sweep<V, FA, kSweepZero>(L, 0, none);
      else
        blk_sweep<V, FA, kSweepPlain>(L, 0, none);
      blk_sweep<V, FA, kSweepPlain>(L, 1, none);
    }
    const LevelView<TA> &cv = ch.lv[l + 1];
    V *bc = (V *)(smem + soff[l + 1][1]);
    if (fused) {
      blk_resrestrict<V, FA>(L, cv.nx, cv.ny, cv.nz, bc, ch.pnu);
      continue;
    }
    const int n = (int)L.lv.ncell();
    V *r = R(l);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int i = t % L.lv.nx, q = t / L.lv.nx;
      const int j = q % L.lv.ny, k = q / L.lv.ny;
      r[t] = residual_cell<V, FA>(L.lv, L.x, L.b, i, j, k, t) * V(ch.pn[l][t]);
    }
    __syncthreads();
    const int nc = (int)cv.ncell();
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
      const int I = t % cv.nx, q = t / cv.nx;
      const int J = q % cv.ny, K = q / cv.ny;
      bc[t] = restrict_cell<V>(L.lv.nx, L.lv.ny, L.lv.nz, cv.nx, cv.ny, cv.nz, r, I, J, K,
                               ch.transfer);
    }
    __syncthreads();
  }
  {
    const CLev<V, FA> L = lev(last);
    if (L.hx.d * L.ny.d * (unsigned)L.lv.nz <= 32u) {
      if (threadIdx.x < 32) warp_coarsest<V, FA>(L, ch.coarsest_sweeps);
      __syncthreads();
    } else {
      for (int s = 0; s < ch.coarsest_sweeps; ++s) {
        if (s == 0)
          blk_sweep<V, FA, kSweepZero>(L, 0, none);
        else
          blk_sweep<V, FA, kSweepPlain>(L, 0, none);
        blk_sweep<V, FA, kSweepPlain>(L, 1, none);
      }
      for (int s = 0; s < ch.coarsest_sweeps; ++s) {
        blk_sweep<V, FA, kSweepPlain>(L, 1, none);
        blk_sweep<V, FA, kSweepPlain>(L, 0, none);
      }
    }
  }
  for (int l = last - 1; l >= first; --l) {
    const CLev<V, FA> L = lev(l);
    const LevelView<TA> &cv = ch.lv[l + 1];
    const V *xc = (const V *)(smem + soff[l + 1][0]);
    if (fused) {
      const Fold<V> f{xc, cv.nx, cv.ny, V(ch.pnu)};
      for (int s = 0; s < ch.smooth; ++s) {
        if (s == 0)
          blk_sweep<V, FA, kSweepProlong>(L, 1, f);
        else
          blk_sweep<V, FA, kSweepPlain>(L, 1, none);
        blk_sweep<V, FA, kSweepPlain>(L, 0, none);
      }
      continue;
    }
    const int n = (int)L.lv.ncell();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int i = t % L.lv.nx, q = t / L.lv.nx;
      const int j = q % L.lv.ny, k = q / L.lv.ny;
      if (six<float>(L.lv, i, j, k).diag() > 0.f)
        L.x[t] += prolong_cell<V>(cv.nx, cv.ny, cv.nz, xc, i, j, k, ch.transfer) *
                  V(ch.pn[l][t]);
    }
    __syncthreads();
    for (int s = 0; s < ch.smooth; ++s) {
      blk_sweep<V, FA, kSweepPlain>(L, 1, none);
      blk_sweep<V, FA, kSweepPlain>(L, 0, none);
    }
  }
  {
    const int n = (int)ch.lv[first].ncell();
    const V *x = (const V *)(smem + soff[first][0]);
    for (int t = threadIdx.x; t < n; t += blockDim.x) ch.x[first][t] = x[t];
  }
}

template <class V, class TA>
__global__ void __launch_bounds__(1024, 1)
k_mg_chain_smem(CoarseChain<V, TA> ch, const CGState *st) {
  pdl_wait();
  if (stopped(st)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  chain_body<V, TA>(ch, smem);
}


// --------------------------------------------- coarse levels on a cluster ---
// The levels just above the local chain (at 128^3: 32^3 and 16^3) split into
// z-slabs over the kClusterCtas CTAs of one thread-block cluster: each CTA
// keeps its slab's x, b and fractions (and, for levels that the per-launch
// path sweeps inside the chain, the inverse diagonal) in shared memory,
// reads the x planes just across its slab boundaries from its neighbours'
// shared memory, and the phases are separated by the cluster's hardware
// barrier instead of kernel launches. Slabs of consecutive levels line up
// (an even number of planes per CTA), so restriction outputs and
// prolongation parents stay in the CTA. CTA 0 runs the local chain between
// the down and the up sweeps. Every CTA passes the same barriers in the same
// order (the only early exit, the stop flag, is read before the first one
// and is the same for all), so no CTA can be left waiting. Per cell the
// arithmetic is the per-launch path's: division for the levels it sweeps as
// grid kernels, the inverse diagonal for those it sweeps in the chain, and
// the prolongation as an explicit pass that stores the values the folded
// sweep forms on the fly.
namespace cgr = cooperative_groups;

template <class V, class TA>
struct Slab {
  int nx, ny, nz, P, z0;
  double c;
  V *x, *b, *dinv;           // dinv null: sweep by division
  const TA *ax, *ay, *az;    // faces of the slab's cells (az: P + 1 planes)
  const V *xdn, *xup;        // x of the CTAs below and above (null at the ends)
};

template <class V, class TA>
__device__ __forceinline__ void slab_gather(Nb7<V> &g, const Slab<V, TA> &S, int i, int j,
                                            int kk, int c) {
  const int row = kk * S.ny + j, nx = S.nx, nxy = S.nx * S.ny, k = S.z0 + kk;
  g.xm = (V)ld(S.ax + c + row);
  g.xp = (V)ld(S.ax + c + row + 1);
  g.ym = (V)ld(S.ay + c + kk * nx);
  g.yp = (V)ld(S.ay + c + kk * nx + nx);
  g.zm = (V)ld(S.az + c);
  g.zp = (V)ld(S.az + c + nxy);
  g.vxm = i > 0 ? S.x[c - 1] : V(0);
  g.vxp = i < nx - 1 ? S.x[c + 1] : V(0);
  g.vym = j > 0 ? S.x[c - nx] : V(0);
  g.vyp = j < S.ny - 1 ? S.x[c + nx] : V(0);
  g.vzm = k > 0 ? (kk > 0 ? S.x[c - nxy] : S.xdn[c + (S.P - 1) * nxy]) : V(0);
  g.vzp = k < S.nz - 1 ? (kk < S.P - 1 ? S.x[c + nxy] : S.xup[c - (S.P - 1) * nxy]) : V(0);
  g.vc = S.x[c];
}

// Half sweep of colour `color` over the slab (zero: x = 0 before it).
template <class V, class TA, bool ZERO>
__device__ void slab_sweep(const Slab<V, TA> &S, int color) {
  const int hx = S.nx >> 1;
  const int n = S.P * S.ny * hx;
  const V cc = V(S.c);
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int row = t / hx, m = t - row * hx;
    const int kk = row / S.ny, j = row - kk * S.ny;
    const int i = 2 * m + ((j + S.z0 + kk + color) & 1);
    const int c = row * S.nx + i;
    V v;
    if (S.dinv) {
      if (ZERO) {
        v = S.b[c] * S.dinv[c];
      } else {
        Nb7<V> g;
        slab_gather(g, S, i, j, kk, c);
        v = (S.b[c] + cc * g.nb()) * S.dinv[c];
      }
    } else if (ZERO) {
      const int nx = S.nx, nxy = S.nx * S.ny;
      const V dg = (V)ld(S.ax + c + row) + (V)ld(S.ax + c + row + 1) +
                   (V)ld(S.ay + c + kk * nx) + (V)ld(S.ay + c + kk * nx + nx) +
                   (V)ld(S.az + c) + (V)ld(S.az + c + nxy);
      v = dg > V(0) ? S.b[c] / (cc * dg) : V(0);
    } else {
      Nb7<V> g;
      slab_gather(g, S, i, j, kk, c);
      const V dg = g.diag();
      v = dg > V(0) ? (S.b[c] + cc * g.nb()) / (cc * dg) : V(0);
    }
    S.x[c] = v;
  }
}

// Restriction of the slab's residual (four even children, as
// resrestrict_cell) into the coarse slab: bc indexed locally, or globally
// (the level below is the local chain's) when `global`.
template <class V, class TA>
__device__ void slab_resrestrict(const Slab<V, TA> &F, V *bc, bool global, float pn) {
  const int cnx = F.nx >> 1, cny = F.ny >> 1, cP = F.P >> 1, cz0 = F.z0 >> 1;
  const int n = cP * cny * cnx;
  const V cc = V(F.c);
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int q = t / cnx, I = t - q * cnx;
    const int KK = q / cny, J = q - KK * cny;
    V acc = V(0);
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      const int a = (ch == 1 || ch == 2), bb = (ch == 1 || ch == 3), cz = (ch >= 2);
      const int i = 2 * I + a, j = 2 * J + bb, kk = 2 * KK + cz;
      const int c = (kk * F.ny + j) * F.nx + i;
      Nb7<V> g;
      slab_gather(g, F, i, j, kk, c);
      const V dg = g.diag();
      if (dg > V(0)) acc += F.b[c] - cc * (dg * g.vc - g.nb());
    }
    const int out = global ? ((cz0 + KK) * cny + J) * cnx + I : t;
    bc[out] = V(0.125) * V(pn) * acc;
  }
}

// x += w x_c(parent) on the slab's active cells; the parents are the coarse
// slab (local indices) or the local chain's first level (global indices).
template <class V, class TA>
__device__ void slab_prolong(const Slab<V, TA> &S, const V *xc, bool global, V w) {
  const int cnx = S.nx >> 1, cny = S.ny >> 1;
  const int n = S.P * S.ny * S.nx;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const int row = c / S.nx, i = c - row * S.nx;
    const int kk = row / S.ny, j = row - kk * S.ny;
    const int nx = S.nx, nxy = S.nx * S.ny;
    const float dg = (float)ld(S.ax + c + row) + (float)ld(S.ax + c + row + 1) +
                     (float)ld(S.ay + c + kk * nx) + (float)ld(S.ay + c + kk * nx + nx) +
                     (float)ld(S.az + c) + (float)ld(S.az + c + nxy);
    if (!(dg > 0.f)) continue;
    const int K = global ? (S.z0 + kk) >> 1 : kk >> 1;
    S.x[c] += xc[(K * cny + (j >> 1)) * cnx + (i >> 1)] * w;
  }
}

template <class V, class TA>
__global__ void __launch_bounds__(1024, 1)
k_mg_cluster(ClusterSpan<V, TA> m, CoarseChain<V, TA> ch, const CGState *st) {
  if (stopped(st)) return;  // the same value in every CTA: no barrier is passed
  cgr::cluster_group cl = cgr::this_cluster();
  const int r = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smem[];
  auto slab = [&](int l) {
    const LevelView<TA> &g = m.lv[l];
    Slab<V, TA> S;
    S.nx = g.nx;
    S.ny = g.ny;
    S.nz = g.nz;
    S.P = g.nz / kClusterCtas;
    S.z0 = r * S.P;
    S.c = g.c;
    S.x = (V *)(smem + m.off[l][0]);
    S.b = (V *)(smem + m.off[l][1]);
    S.dinv = m.use_dinv[l] ? (V *)(smem + m.off[l][5]) : nullptr;
    S.ax = (const TA *)(smem + m.off[l][2]);
    S.ay = (const TA *)(smem + m.off[l][3]);
    S.az = (const TA *)(smem + m.off[l][4]);
    S.xdn = r > 0 ? cl.map_shared_rank(S.x, r - 1) : nullptr;
    S.xup = r < kClusterCtas - 1 ? cl.map_shared_rank(S.x, r + 1) : nullptr;
    return S;
  };
  // the slabs' fractions (and b of the first level) from global memory:
  // thread 0 issues bulk copies of the contiguous slab arrays on one
  // mbarrier, the other threads copy any part a bulk copy cannot take
  {
    __shared__ __align__(8) unsigned long long mbar;
    const unsigned mb = (unsigned)__cvta_generic_to_shared(&mbar);
    struct Seg {
      void *dst;
      const void *src;
      unsigned bytes;
    };
    Seg seg[3 * kMaxLevels + 1];
    int ns = 0;
    for (int l = m.lo; l < m.hi; ++l) {
      const LevelView<TA> &g = m.lv[l];
      const int P = g.nz / kClusterCtas, z0 = r * P;
      const size_t nxy = (size_t)g.nx * g.ny;
      seg[ns++] = {smem + m.off[l][2], g.ax + (size_t)z0 * g.ny * (g.nx + 1),
                   (unsigned)(P * g.ny * (g.nx + 1) * sizeof(TA))};
      seg[ns++] = {smem + m.off[l][3], g.ay + (size_t)z0 * (g.ny + 1) * g.nx,
                   (unsigned)(P * (g.ny + 1) * g.nx * sizeof(TA))};
      seg[ns++] = {smem + m.off[l][4], g.az + (size_t)z0 * nxy,
                   (unsigned)((P + 1) * nxy * sizeof(TA))};
    }
    {
      const LevelView<TA> &g = m.lv[m.lo];
      const size_t n = (size_t)(g.nz / kClusterCtas) * g.nx * g.ny;
      seg[ns++] = {smem + m.off[m.lo][1], m.b_lo + (size_t)r * n, (unsigned)(n * sizeof(V))};
    }
    // bytes a bulk copy takes: both addresses 16-byte aligned, a multiple of 16
    auto bulk = [](const Seg &q) {
      return (((uintptr_t)q.src | (uintptr_t)__cvta_generic_to_shared(q.dst)) & 15u)
                 ? 0u
                 : (q.bytes & ~15u);
    };
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned tx = 0;
      for (int q = 0; q < ns; ++q) tx += bulk(seg[q]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(tx)
                   : "memory");
      for (int q = 0; q < ns; ++q) {
        const unsigned nb = bulk(seg[q]);
        if (nb == 0) continue;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"((unsigned)__cvta_generic_to_shared(seg[q].dst)),
            "l"(seg[q].src), "r"(nb), "r"(mb)
            : "memory");
      }
    }
    for (int q = 0; q < ns; ++q) {
      const unsigned done = bulk(seg[q]);
      for (unsigned t = done + threadIdx.x; t < seg[q].bytes; t += blockDim.x)
        ((unsigned char *)seg[q].dst)[t] = ((const unsigned char *)seg[q].src)[t];
    }
    // an expired wait (error word set, the solve reports NF_E_TIMEOUT) still
    // passes every barrier below, after the copies had a second bound to land
    if (!mbar_wait(mb, 0, ch.err)) mbar_wait(mb, 0, nullptr);
  }
  __syncthreads();
  // inverse diagonals (the chain's formula) where the per-launch path uses them
  for (int l = m.lo; l < m.hi; ++l) {
    if (!m.use_dinv[l]) continue;
    const Slab<V, TA> S = slab(l);
    const LevelView<TA> lvs{S.nx, S.ny, S.P, S.c, S.ax, S.ay, S.az};
    const V cc = V(S.c);
    const int n = S.P * S.ny * S.nx;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int row = c / S.nx, i = c - row * S.nx;
      const int kk = row / S.ny, j = row - kk * S.ny;
      const V dg = six<V>(lvs, i, j, kk).diag();
      S.dinv[c] = dg > V(0) ? V(1) / (cc * dg) : V(0);
    }
  }
  __syncthreads();
  for (int l = m.lo; l < m.hi; ++l) {
    const Slab<V, TA> S = slab(l);
    for (int s = 0; s < m.smooth; ++s) {
      if (s == 0)
        slab_sweep<V, TA, true>(S, 0);
      else
        slab_sweep<V, TA, false>(S, 0);
      cl.sync();
      slab_sweep<V, TA, false>(S, 1);
      cl.sync();
    }
    if (l + 1 < m.hi)
      slab_resrestrict<V, TA>(S, (V *)(smem + m.off[l + 1][1]), false, m.w);
    else
      slab_resrestrict<V, TA>(S, m.b_hi, true, m.w);
    cl.sync();
  }
  if (r == 0) chain_body<V, TA>(ch, smem + m.chain_off);
  cl.sync();
  for (int l = m.hi - 1; l >= m.lo; --l) {
    const Slab<V, TA> S = slab(l);
    if (l + 1 < m.hi)
      slab_prolong<V, TA>(S, (const V *)(smem + m.off[l + 1][0]), false, V(m.w));
    else
      slab_prolong<V, TA>(S, m.x_hi, true, V(m.w));
    cl.sync();
    for (int s = 0; s < m.smooth; ++s) {
      slab_sweep<V, TA, false>(S, 1);
      cl.sync();
      slab_sweep<V, TA, false>(S, 0);
      cl.sync();
    }
  }
  {
    const LevelView<TA> &g = m.lv[m.lo];
    const int n = (g.nz / kClusterCtas) * g.nx * g.ny;
    const V *src = (const V *)(smem + m.off[m.lo][0]);
    V *dst = m.x_lo + (size_t)r * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = src[t];
  }
}

// ------------------------------------------------ persistent mid levels ---
// Levels too small to fill the GPU with one launch per half sweep (each
// launch costs a few microseconds of issue and tail) and too large for one
// thread block run inside one cooperative kernel: every phase (half sweep,
// fused residual-restriction, the first post-smoothing half sweep with the
// prolongation folded in) is a grid-stride loop over rows, consecutive
// phases are separated by a grid-wide barrier, and between the down and the
// up sweep block 0 runs the shared-memory chain while the others wait.

// Grid-wide barrier of a cooperative launch: after the block's threads meet,
// thread 0 adds one to *bar with release semantics (the block's writes,
// ordered before it by the CTA barrier, become visible with the arrival)
// and spins with acquire loads until *bar reaches target (phases so far x
// blocks). Each wait is bounded: every 256 polls it checks *err and the
// clock, and after kBarrierNs it sets *err; every block then leaves at its
// next barrier. Returns false (the same in all threads of the block) when
// the kernel must stop.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned target,
                                             int *err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    unsigned long long t0 = 0;
    unsigned spins = 0;
    int e = 0;
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if ((++spins & 255u) == 0) {
        if (*(volatile int *)err != 0) {
          e = 1;
          break;
        }
        const unsigned long long t = globaltimer_ns();
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > kBarrierNs) {
          atomicExch(err, 1);
          e = 1;
          break;
        }
      }
    }
    ok = e == 0;
  }
  __syncthreads();
  return ok != 0;
}

template <class V, class TA>
__global__ void __launch_bounds__(1024, 1)
k_mg_mid(MidSpan<V, TA> m, CoarseChain<V, TA> ch, const CGState *st) {
  const int stop = stop_flag(st) | *(volatile int *)m.err;
  extern __shared__ __align__(16) unsigned char smem[];
  const RowWalk rw;
  const Fold<V> none{nullptr, 0, 0, V(0)};
  unsigned phase = 0;
  auto sync = [&]() { return grid_barrier(m.bar, ++phase * gridDim.x + m.stall, m.err); };
  for (int l = m.lo; l < m.hi; ++l) {
    const LevelView<TA> lv = m.lv[l];
    V *x = m.x[l];
    const V *b = m.b[l];
    for (int s = 0; s < m.smooth; ++s) {
      if (s == 0)
        sweep_rows<V, TA, kSweepZero>(lv, x, b, 0, none, rw.warp, rw.nwarps, rw.lane,
                                      l == m.lo ? stop : 0);
      else
        sweep_rows<V, TA, kSweepPlain>(lv, x, b, 0, none, rw.warp, rw.nwarps, rw.lane);
      if (stop) return;  // (the same in every block: no barrier is left waiting)
      if (!sync()) return;
      sweep_rows<V, TA, kSweepPlain>(lv, x, b, 1, none, rw.warp, rw.nwarps, rw.lane);
      if (!sync()) return;
    }
    const LevelView<TA> cv = m.lv[l + 1];
    resrestrict_rows<V, TA>(lv, x, b, cv.nx, cv.ny, cv.nz, m.b[l + 1], m.w, rw.warp,
                            rw.nwarps, rw.lane);
    if (!sync()) return;
  }
  if (blockIdx.x == 0) chain_body<V, TA>(ch, smem);
  if (!sync()) return;
  for (int l = m.hi - 1; l >= m.lo; --l) {
    const LevelView<TA> lv = m.lv[l];
    V *x = m.x[l];
    const V *b = m.b[l];
    const Fold<V> f{m.x[l + 1], m.lv[l + 1].nx, m.lv[l + 1].ny, V(m.w)};
    for (int s = 0; s < m.smooth; ++s) {
      if (s == 0)
        sweep_rows<V, TA, kSweepProlong>(lv, x, b, 1, f, rw.warp, rw.nwarps, rw.lane);
      else
        sweep_rows<V, TA, kSweepPlain>(lv, x, b, 1, none, rw.warp, rw.nwarps, rw.lane);
      if (!sync()) return;
      sweep_rows<V, TA, kSweepPlain>(lv, x, b, 0, none, rw.warp, rw.nwarps, rw.lane);
      // the end of the kernel orders the last phase before the next launch
      if (l > m.lo || s + 1 < m.smooth)
        if (!sync()) return;
    }
  }
}

// ------------------------------------------------------------ launchers ---

// Grid-stride streaming kernels: at most one wave (148 SMs x 8 blocks of
// kBlock threads; their launch bounds keep 8 blocks resident), so every
// block pays its start-up latency once.
static inline unsigned gs_blocks(int64_t n) {
  const unsigned b = nblocks(n), wave = 148u * 8u;
  return b < wave ? b : wave;
}

template <class S, class T, class V>
void launch_residual_outer(const Launch &L, const LevelView<T> &lv, const S *b,
                           const S *x, V *rin, double scale, int es, bool split,
                           const RedScratch &rs, double *norm2) {
  ProfScope _ps(L, NF_K_RESIDUAL64);
  if constexpr (sizeof(S) == 8 && sizeof(T) == 4 && sizeof(V) == 4) {
    // split arithmetic needs c = 1 and the scale of rin in float range
    const double rscale = std::ldexp(scale, -es);
    if (split && lv.c == 1.0 && rscale >= 0x1p-120 && rscale <= 0x1p120) {
      launch_pdl(k_residual_outer_df, kRedBlocks, kBlock, 0, L.s, lv, b, x, rin, es,
                 (float)rscale, scale, rs, norm2);
      ++*L.counter;
      return;
    }
  }
  k_residual_outer<S, T, V><<<kRedBlocks, kBlock, 0, L.s>>>(lv, b, x, rin, scale, rs, norm2);
  ++*L.counter;
}
template <class S, class V>
__global__ void __launch_bounds__(kBlock, 8) k_scale_rhs(int64_t n, const S *b, V *rin,
                                                         double scale) {
  pdl_wait();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    rin[c] = (V)((double)b[c] * scale);
}
template <class S, class V>
void launch_scale_rhs(const Launch &L, int64_t n, const S *b, V *rin, double scale) {
  ProfScope _ps(L, NF_K_RESIDUAL64);
  launch_pdl(k_scale_rhs<S, V>, gs_blocks(n), kBlock, 0, L.s, n, b, rin, scale);
  ++*L.counter;
}
template <class S, class V>
void launch_axpy_outer(const Launch &L, int64_t n, S *x, const V *e, double inv) {
  ProfScope _ps(L, NF_K_AXPY64);
  launch_pdl(k_axpy_outer<S, V>, gs_blocks(n), kBlock, 0, L.s, n, x, e, inv);
  ++*L.counter;
}
template <class V>
void launch_cg_init(const Launch &L, int64_t n, const V *r, const V *z, V *d,
                    CGState *st, const RedScratch &rs) {
  ProfScope _ps(L, NF_K_CG_INIT);
  launch_pdl(k_cg_init<V>, kRedBlocks, kBlock, 0, L.s, n, r, z, d, st, rs);
  ++*L.counter;
}
template <class V>
void launch_cg_continue(const Launch &L, int64_t n, const V *r, const V *z,
                        CGState *st, const RedScratch &rs) {
  ProfScope _ps(L, NF_K_CG_INIT);
  launch_pdl(k_cg_continue<V>, kRedBlocks, kBlock, 0, L.s, n, r, z, st, rs);
  ++*L.counter;
}
template <class V, class TA>
void launch_apply_dot(const Launch &L, const LevelView<TA> &lv, const V *d,
                      V *q, CGState *st, const RedScratch &rs) {
  ProfScope _ps(L, NF_K_APPLY_DOT);
  launch_pdl(k_apply_dot<V, TA>, kRedBlocks, kBlock, 0, L.s, lv, d, q, st, rs);
  ++*L.counter;
}
template <class V>
void launch_cg_xr(const Launch &L, int64_t n, V *x, V *r, const V *d,
                  const V *q, CGState *st, const RedScratch &rs,
                  bool preconditioned, const LoopHandles *loop) {
  ProfScope _ps(L, NF_K_CG_XR);
  launch_pdl(k_cg_xr<V>, kRedBlocks, kBlock, 0, L.s, n, x, r, d, q, st, rs, preconditioned,
             (int)(loop != nullptr), loop ? *loop : LoopHandles{});
  ++*L.counter;
}
template <class V>
void launch_cg_rz(const Launch &L, int64_t n, const V *r, const V *z,
                  CGState *st, const RedScratch &rs) {
  ProfScope _ps(L, NF_K_CG_RZ);
  launch_pdl(k_cg_rz<V>, kRedBlocks, kBlock, 0, L.s, n, r, z, st, rs);
  ++*L.counter;
}
template <class V>
void launch_dot(const Launch &L, int64_t n, const V *a, const V *b,
                const RedScratch &rs, double *out) {
  k_dot<V><<<kRedBlocks, kBlock, 0, L.s>>>(n, a, b, rs, out);
  ++*L.counter;
}
template <class V>
void launch_cg_d(const Launch &L, int64_t n, const V *z, V *d, CGState *st,
                 const cudaGraphConditionalHandle *loop) {
  ProfScope _ps(L, NF_K_CG_D);
  launch_pdl(k_cg_d<V>, gs_blocks(n), kBlock, 0, L.s, n, z, d, st, (int)(loop != nullptr),
             loop ? *loop : cudaGraphConditionalHandle{});
  ++*L.counter;
}
template <class TI, class TO>
void launch_mg_coarsen(const Launch &L, const LevelView<TI> &fine, int cnx,
                       int cny, int cnz, TO *ax, TO *ay, TO *az) {
  const int64_t n = (int64_t)(cnx + 1) * cny * cnz + (int64_t)cnx * (cny + 1) * cnz +
                    (int64_t)cnx * cny * (cnz + 1);
  ProfScope _ps(L, NF_K_MG_COARSEN);
  k_mg_coarsen<TI, TO><<<nblocks(n), kBlock, 0, L.s>>>(fine, cnx, cny, cnz, ax, ay, az);
  ++*L.counter;
}
template <class V, class TA>
void launch_mg_smooth(const Launch &L, const LevelView<TA> &lv, V *x,
                      const V *b, int color, int mode, const Fold<V> &f,
                      const CGState *st, int kclass) {
  ProfScope _ps(L, kclass);
  const unsigned nb = row_blocks(lv.ny * lv.nz);
  if (mode == kSweepZero)
    launch_pdl(k_mg_smooth<V, TA, kSweepZero>, nb, kBlock, 0, L.s, lv, x, b, color, f, st);
  else if (mode == kSweepProlong)
    launch_pdl(k_mg_smooth<V, TA, kSweepProlong>, nb, kBlock, 0, L.s, lv, x, b, color, f, st);
  else
    launch_pdl(k_mg_smooth<V, TA, kSweepPlain>, nb, kBlock, 0, L.s, lv, x, b, color, f, st);
  ++*L.counter;
}
// Tile shapes of the fused pair: 32 x 8 cells per block, 4 planes per step
// for FP32 vectors (46 KB of shared memory), 2 for FP64 (62 KB).
template <class V, class TA, int MODE>
static void rb_pair_kernel(const Launch &L, const LevelView<TA> &lv, const V *xin, V *xout,
                           const V *b, int c1, const Fold<V> &f, const CGState *st) {
  constexpr int TX = 32, TY = 8, ZB = sizeof(V) == 4 ? 4 : 2;
  using C = RbPair<V, TA, TX, TY, ZB>;
  auto kernel = k_mg_rb_pair<V, TA, MODE, TX, TY, ZB>;
  static bool ready = false;  // one attribute call per instantiation
  if (!ready) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::bytes);
    ready = true;
  }
  const int nbx = (lv.nx + TX - 1) / TX, nby = (lv.ny + TY - 1) / TY;
  // planes per block: 32, halved (to 8 at least) until there are two blocks
  // per SM
  int zc = 32;
  while (zc > 8 && (int64_t)nbx * nby * ((lv.nz + zc - 1) / zc) < 2 * 148) zc /= 2;
  const unsigned nb = (unsigned)(nbx * nby * ((lv.nz + zc - 1) / zc));
  launch_pdl(kernel, nb, (unsigned)C::NT, C::bytes, L.s, lv, xin, xout, b, c1, zc, f, st);
}
template <class V, class TA>
void launch_mg_rb_pair(const Launch &L, const LevelView<TA> &lv, const V *xin, V *xout,
                       const V *b, int c1, int mode, const Fold<V> &f, const CGState *st,
                       int kclass) {
  ProfScope _ps(L, kclass);
  if (mode == kSweepZero)
    rb_pair_kernel<V, TA, kSweepZero>(L, lv, xin, xout, b, c1, f, st);
  else if (mode == kSweepProlong)
    rb_pair_kernel<V, TA, kSweepProlong>(L, lv, xin, xout, b, c1, f, st);
  else
    rb_pair_kernel<V, TA, kSweepPlain>(L, lv, xin, xout, b, c1, f, st);
  ++*L.counter;
}
template <class TA>
void launch_band_build(const Launch &L, const LevelView<TA> &lv,
                       unsigned char *mark, int *list0, int *list1, int *count) {
  ProfScope _ps(L, NF_K_MG_COARSEN);
  cudaMemsetAsync(count, 0, 2 * sizeof(int), L.s);
  k_band_mark<TA><<<gs_blocks(lv.ncell()), kBlock, 0, L.s>>>(lv, mark);
  k_band_collect<TA><<<gs_blocks(lv.ncell()), kBlock, 0, L.s>>>(lv, mark, list0,
                                                                list1, count);
  *L.counter += 2;
}
template <class V, class TA>
void launch_band_smooth(const Launch &L, const LevelView<TA> &lv, V *x,
                        const V *b, const int *list, const int *count,
                        const CGState *st) {
  ProfScope _ps(L, NF_K_MG_SMOOTH0);
  k_band_smooth<V, TA><<<kRedBlocks, kBlock, 0, L.s>>>(lv, x, b, list, count, st);
  ++*L.counter;
}
template <class V, class TA>
void launch_mg_residual(const Launch &L, const LevelView<TA> &lv, const V *x,
                        const V *b, V *r, const float *pn, const CGState *st) {
  ProfScope _ps(L, NF_K_MG_RESIDUAL);
  k_mg_residual<V, TA><<<row_blocks(lv.ny * lv.nz), kBlock, 0, L.s>>>(lv, x, b, r, pn, st);
  ++*L.counter;
}
template <class V, class TA>
void launch_mg_resrestrict(const Launch &L, const LevelView<TA> &fine, const V *x,
                           const V *b, int cnx, int cny, int cnz, V *bc, float pn,
                           const CGState *st) {
  ProfScope _ps(L, NF_K_MG_RESTRICT);
  launch_pdl(k_mg_resrestrict<V, TA>, row_blocks(cny * cnz), kBlock, 0, L.s, fine, x, b, cnx, cny,
             cnz, bc, pn, st);
  ++*L.counter;
}
template <class V, class TA>
void launch_mg_restrict(const Launch &L, const LevelView<TA> &fine,
                        const LevelView<TA> &coarse, const V *rf, V *bc,
                        int mode, const CGState *st) {
  ProfScope _ps(L, NF_K_MG_RESTRICT);
  k_mg_restrict<V><<<row_blocks(coarse.ny * coarse.nz), kBlock, 0, L.s>>>(
      fine.nx, fine.ny, fine.nz, coarse.nx, coarse.ny, coarse.nz, rf, bc, mode, st);
  ++*L.counter;
}
template <class V, class TF, class TC>
void launch_mg_prolong(const Launch &L, const LevelView<TF> &fine,
                       const LevelView<TC> &coarse, const V *xc, V *xf,
                       const float *pn, int mode, const CGState *st) {
  ProfScope _ps(L, NF_K_MG_PROLONG);
  k_mg_prolong<V, TF><<<row_blocks(fine.ny * fine.nz), kBlock, 0, L.s>>>(
      fine, coarse.nx, coarse.ny, coarse.nz, xc, xf, pn, mode, st);
  ++*L.counter;
}
__global__ void k_fill(int64_t n, float *p, float v) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    p[c] = v;
}
void launch_mg_fill(const Launch &L, int64_t n, float *p, float v) {
  k_fill<<<gs_blocks(n), kBlock, 0, L.s>>>(n, p, v);
  ++*L.counter;
}
template <class TC>
void launch_mg_pnorm(const Launch &L, int fnx, int fny, int fnz,
                     const LevelView<TC> &coarse, float *pn, float scale) {
  ProfScope _ps(L, NF_K_MG_COARSEN);
  const int64_t n = (int64_t)fnx * fny * fnz;
  k_mg_pnorm<TC><<<gs_blocks(n), kBlock, 0, L.s>>>(fnx, fny, fnz, coarse, pn, scale);
  ++*L.counter;
}
template <class V, class TA>
size_t mg_chain_smem_bytes(const CoarseChain<V, TA> &ch) {
  size_t off[kMaxLevels][7];
  return chain_layout(ch, off);
}
// Allow a kernel the opt-in shared memory left beside its static shared
// variables as dynamic shared memory.
template <class K>
static cudaError_t allow_dynamic_smem(K kernel, int smem_limit) {
  cudaFuncAttributes a{};
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_limit - (int)a.sharedSizeBytes);
}
template <class V, class TA>
int prepare_mg_chain(int smem_limit) {
  const cudaError_t e = allow_dynamic_smem(k_mg_chain_smem<V, TA>, smem_limit);
  return e == cudaSuccess ? NF_OK : cuda_fail(e, "cudaFuncSetAttribute(chain)");
}
template <class V, class TA>
int prepare_mg_mid(int smem_limit, int smem) {
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      allow_dynamic_smem(k_mg_mid<V, TA>, smem_limit) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mg_mid<V, TA>, 1024, smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return coop ? per_sm * sms : 0;
}
template <class V, class TA>
bool prepare_mg_cluster(int smem_limit, int smem) {
  if (allow_dynamic_smem(k_mg_cluster<V, TA>, smem_limit) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kClusterCtas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, (void *)k_mg_cluster<V, TA>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters >= 1;
}
template <class V, class TA>
int launch_mg_cluster(const Launch &L, const ClusterSpan<V, TA> &m,
                      const CoarseChain<V, TA> &ch, const CGState *st, int smem) {
  ProfScope _ps(L, NF_K_MG_CHAIN);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = L.s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kClusterCtas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_mg_cluster<V, TA>, m, ch, st);
  ++*L.counter;
  return e == cudaSuccess ? NF_OK : cuda_fail(e, "cluster launch (k_mg_cluster)");
}
template <class V, class TA>
int launch_mg_mid(const Launch &L, const MidSpan<V, TA> &m,
                  const CoarseChain<V, TA> &ch, const CGState *st, int blocks) {
  ProfScope _ps(L, NF_K_MG_MID);
  cudaMemsetAsync(m.bar, 0, sizeof(unsigned), L.s);
  MidSpan<V, TA> a0 = m;
  CoarseChain<V, TA> a1 = ch;
  const CGState *a2 = st;
  void *args[] = {(void *)&a0, (void *)&a1, (void *)&a2};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_mg_mid<V, TA>, dim3(blocks),
                                                    dim3(1024), args, (size_t)ch.smem_bytes, L.s);
  ++*L.counter;
  return e == cudaSuccess ? NF_OK : cuda_fail(e, "cooperative launch (k_mg_mid)");
}
template <class V, class TA>
void launch_mg_coarse_chain(const Launch &L, const CoarseChain<V, TA> &ch,
                            const CGState *st) {
  ProfScope _ps(L, NF_K_MG_CHAIN);
  if (ch.smem_bytes > 0)
    launch_pdl(k_mg_chain_smem<V, TA>, 1u, 1024u, (size_t)ch.smem_bytes, L.s, ch, st);
  else
    k_mg_coarse_chain<V, TA><<<1, 1024, 0, L.s>>>(ch, st);
  ++*L.counter;
}

#define NF_INST_V(V)                                                           \
  template void launch_cg_init<V>(const Launch &, int64_t, const V *,        \
                                  const V *, V *, CGState *,                  \
                                  const RedScratch &);                        \
  template void launch_cg_continue<V>(const Launch &, int64_t, const V *,    \
                                      const V *, CGState *,                   \
                                      const RedScratch &);                    \
  template void launch_cg_xr<V>(const Launch &, int64_t, V *, V *, const V *,\
                                const V *, CGState *, const RedScratch &,     \
                                bool, const LoopHandles *);                   \
  template void launch_cg_rz<V>(const Launch &, int64_t, const V *,          \
                                const V *, CGState *, const RedScratch &);    \
  template void launch_cg_d<V>(const Launch &, int64_t, const V *, V *,      \
                               CGState *, const cudaGraphConditionalHandle *);\
  template void launch_dot<V>(const Launch &, int64_t, const V *, const V *, \
                              const RedScratch &, double *);
#define NF_INST_VA(V, TA)                                                      \
  template void launch_apply_dot<V, TA>(const Launch &, const LevelView<TA> &,\
                                        const V *, V *, CGState *,            \
                                        const RedScratch &);                  \
  template void launch_mg_smooth<V, TA>(const Launch &, const LevelView<TA> &,\
                                        V *, const V *, int, int,             \
                                        const Fold<V> &, const CGState *, int);\
  template void launch_mg_rb_pair<V, TA>(const Launch &, const LevelView<TA> &,\
                                         const V *, V *, const V *, int, int, \
                                         const Fold<V> &, const CGState *, int);\
  template void launch_band_smooth<V, TA>(const Launch &,                    \
                                          const LevelView<TA> &, V *,         \
                                          const V *, const int *,             \
                                          const int *, const CGState *);      \
  template void launch_mg_residual<V, TA>(const Launch &,                    \
                                          const LevelView<TA> &, const V *,   \
                                          const V *, V *, const float *,      \
                                          const CGState *);                   \
  template void launch_mg_resrestrict<V, TA>(const Launch &,                 \
                                             const LevelView<TA> &, const V *,\
                                             const V *, int, int, int, V *,   \
                                             float, const CGState *);         \
  template void launch_mg_restrict<V, TA>(const Launch &,                    \
                                          const LevelView<TA> &,              \
                                          const LevelView<TA> &, const V *,   \
                                          V *, int, const CGState *);              \
  template void launch_mg_coarse_chain<V, TA>(const Launch &,                \
                                              const CoarseChain<V, TA> &,     \
                                              const CGState *);               \
  template size_t mg_chain_smem_bytes<V, TA>(const CoarseChain<V, TA> &);    \
  template int prepare_mg_chain<V, TA>(int);                                 \
  template int prepare_mg_mid<V, TA>(int, int);                              \
  template bool prepare_mg_cluster<V, TA>(int, int);                         \
  template int launch_mg_cluster<V, TA>(const Launch &,                      \
                                        const ClusterSpan<V, TA> &,           \
                                        const CoarseChain<V, TA> &,           \
                                        const CGState *, int);                \
  template int launch_mg_mid<V, TA>(const Launch &, const MidSpan<V, TA> &,  \
                                    const CoarseChain<V, TA> &,               \
                                    const CGState *, int);
NF_INST_V(float)
NF_INST_V(double)
template void launch_band_build<float>(const Launch &, const LevelView<float> &,
                                       unsigned char *, int *, int *, int *);
template void launch_band_build<double>(const Launch &, const LevelView<double> &,
                                        unsigned char *, int *, int *, int *);
NF_INST_VA(float, float)
NF_INST_VA(float, __nv_bfloat16)
NF_INST_VA(double, double)

template void launch_mg_prolong<float, float, float>(const Launch &, const LevelView<float> &, const LevelView<float> &, const float *, float *, const float *, int, const CGState *);
template void launch_mg_prolong<float, float, __nv_bfloat16>(const Launch &, const LevelView<float> &, const LevelView<__nv_bfloat16> &, const float *, float *, const float *, int, const CGState *);
template void launch_mg_prolong<float, __nv_bfloat16, __nv_bfloat16>(const Launch &, const LevelView<__nv_bfloat16> &, const LevelView<__nv_bfloat16> &, const float *, float *, const float *, int, const CGState *);
template void launch_mg_prolong<double, double, double>(const Launch &, const LevelView<double> &, const LevelView<double> &, const double *, double *, const float *, int, const CGState *);
template void launch_mg_pnorm<float>(const Launch &, int, int, int, const LevelView<float> &, float *, float);
template void launch_mg_pnorm<__nv_bfloat16>(const Launch &, int, int, int, const LevelView<__nv_bfloat16> &, float *, float);
template void launch_mg_pnorm<double>(const Launch &, int, int, int, const LevelView<double> &, float *, float);

template void launch_mg_coarsen<float, float>(const Launch &, const LevelView<float> &, int, int, int, float *, float *, float *);
template void launch_mg_coarsen<float, __nv_bfloat16>(const Launch &, const LevelView<float> &, int, int, int, __nv_bfloat16 *, __nv_bfloat16 *, __nv_bfloat16 *);
template void launch_mg_coarsen<__nv_bfloat16, __nv_bfloat16>(const Launch &, const LevelView<__nv_bfloat16> &, int, int, int, __nv_bfloat16 *, __nv_bfloat16 *, __nv_bfloat16 *);
template void launch_mg_coarsen<double, double>(const Launch &, const LevelView<double> &, int, int, int, double *, double *, double *);

template void launch_residual_outer<double, float, float>(const Launch &, const LevelView<float> &, const double *, const double *, float *, double, int, bool, const RedScratch &, double *);
template void launch_residual_outer<float, float, float>(const Launch &, const LevelView<float> &, const float *, const float *, float *, double, int, bool, const RedScratch &, double *);
template void launch_residual_outer<double, double, double>(const Launch &, const LevelView<double> &, const double *, const double *, double *, double, int, bool, const RedScratch &, double *);
template void launch_scale_rhs<double, float>(const Launch &, int64_t, const double *, float *, double);
template void launch_scale_rhs<float, float>(const Launch &, int64_t, const float *, float *, double);
template void launch_scale_rhs<double, double>(const Launch &, int64_t, const double *, double *, double);
template void launch_axpy_outer<double, float>(const Launch &, int64_t, double *, const float *, double);
template void launch_axpy_outer<float, float>(const Launch &, int64_t, float *, const float *, double);
template void launch_axpy_outer<double, double>(const Launch &, int64_t, double *, const double *, double);

}  // namespace nf
