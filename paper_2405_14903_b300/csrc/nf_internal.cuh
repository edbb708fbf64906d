// Internal definitions shared by the libnf translation units.
//
// Layout (device): face component d of a grid with nx*ny*nz cells is a dense
// array with x fastest; the own axis of component d has one extra sample.
// Cell (i, j, k) has linear index (k*ny + j)*nx + i.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/nf.h"

namespace nf {

constexpr int kMaxLevels = 12;
constexpr int kBlock = 256;          // threads per block of the stencil kernels
constexpr int kRedBlocks = 148 * 4;  // blocks of grid-stride reduction kernels

struct GridDev {
  int nx, ny, nz;
  double dx, dt, rho, c;  // c = dt / (rho dx)
  double nu;              // kinematic viscosity (0: inviscid)
  int frac;               // NF_FRACTIONS_* rule of the face fractions
  int outlet, oj0, ok0, ow, oh;
  int inlet, iside, ij0, ik0, iw, ih;  // inflow patch on an x wall (side -1 / +1)
  double ispeed;                       // its normal velocity (along +x)
  // Derived on the host by set_derived(): a division or an FP32/FP64
  // conversion per thread would occupy the FP64 pipe, which runs at 1/64 of
  // the FP32 rate on this part.
  double invc;           // 1 / c
  double invw;           // 4 / dx, the slope of the fraction ramp
  float fdx, finvw, fc;  // dx, 4 / dx and c rounded to FP32

  void set_derived() {
    invc = c != 0.0 ? 1.0 / c : 0.0;
    invw = 4.0 / dx;
    fdx = (float)dx;
    finvw = (float)invw;
    fc = (float)c;
  }

  __host__ __device__ int64_t ncell() const { return (int64_t)nx * ny * nz; }
  __host__ __device__ int fnx(int d) const { return nx + (d == 0); }
  __host__ __device__ int fny(int d) const { return ny + (d == 1); }
  __host__ __device__ int fnz(int d) const { return nz + (d == 2); }
  __host__ __device__ int64_t nface(int d) const {
    return (int64_t)fnx(d) * fny(d) * fnz(d);
  }
  __host__ __device__ int64_t cell(int i, int j, int k) const {
    return ((int64_t)k * ny + j) * nx + i;
  }
  __host__ __device__ int64_t face(int d, int i, int j, int k) const {
    return ((int64_t)k * fny(d) + j) * fnx(d) + i;
  }
  // Linear face index -> (i, j, k) of component d. Arrays hold fewer than
  // 2^32 entries, so the decode uses 32-bit unsigned division (64-bit
  // integer division is a long instruction sequence on the GPU).
  __host__ __device__ void face_ijk(int d, int64_t f, int &i, int &j,
                                    int &k) const {
    decomp(f, fnx(d), fny(d), i, j, k);
  }
  __host__ __device__ void cell_ijk(int64_t c, int &i, int &j, int &k) const {
    decomp(c, nx, ny, i, j, k);
  }
  __host__ __device__ static void decomp(int64_t c, int nx, int ny, int &i,
                                         int &j, int &k) {
    const uint32_t u = (uint32_t)c, q = u / (uint32_t)nx;
    i = (int)(u - q * (uint32_t)nx);
    const uint32_t kk = q / (uint32_t)ny;
    j = (int)(q - kk * (uint32_t)ny);
    k = (int)kk;
  }
  // Is face (d; i, j, k) on the box boundary?
  __host__ __device__ bool boundary(int d, int i, int j, int k) const {
    int o = d == 0 ? i : (d == 1 ? j : k);
    int n = d == 0 ? nx : (d == 1 ? ny : nz);
    return o == 0 || o == n;
  }
  __host__ __device__ bool inlet_face(int d, int i, int j, int k) const {
    return inlet && d == 0 && i == (iside > 0 ? nx : 0) && j >= ij0 && j < ij0 + iw &&
           k >= ik0 && k < ik0 + ih;
  }
  __host__ __device__ bool outlet_face(int d, int i, int j, int k) const {
    return outlet && d == 0 && i == nx && j >= oj0 && j < oj0 + ow &&
           k >= ok0 && k < ok0 + oh;
  }
};

// Scene state at one time t (built on the host in double precision).
struct SceneDev {
  int kind;
  int K;
  double t;
  // sphere: centre c(t) = c0 + v t, radius, velocity v = theta
  double sc[3], sr, sv[3];
  // chamber: centre, axes, min axis, radius s(t), rate sdot(t) and their
  // theta derivatives; duct box centre and half extents (fluid inside)
  double cc[3], ca[3], camin, cs, csdot, crate, cds[8], cdsdot[8];  // crate = sdot / s
  double cdus[8];  // d(sdot / s) / d theta
  double cinva[3]; // 1 / ca (no divisions on the device)
  // FP32 copies for the narrow-band evaluator: the derivative scales of
  // d phi / d theta (chamber amin ds/dtheta_k, plate dangle/dtheta_k, sphere
  // -t) and the chamber's 1 / ca
  float fdscale[8], finva[3];
  // FP32 mirrors of the fields the FP32 evaluators read (rounded once per
  // scene state on the host: a double-to-float conversion per evaluation
  // runs on the FP64 pipe)
  float f_sc[3], f_sr, f_sv[3], f_cc[3], f_camin, f_cs, f_crate, f_dc[3], f_dh[3], f_cdus[8];
  float f_pc[3], f_ph[3], f_pcos, f_psin, f_pomega, f_pdomega[4];
  double dc[3], dh[3];
  // plate: centre, half extents, angle, cos/sin, rate, theta derivatives
  double pc[3], ph[3], pang, pcos, psin, pomega, pdang[4], pdomega[4];
  // static spheres (device array of nspheres x 4 doubles)
  const double *spheres;
  int nspheres;
  // extruded polar-Bezier shapes (App. A): device table (layout in
  // scene.cuh, bz_*), shape count, fluid inside (1) or outside (0) their
  // union, theta mode (kBzRadii, kBzPulse, kBzFixed), the pulsing shape and
  // its contraction k(t), rate and their theta derivatives
  const double *bz;
  int bz_n, bz_inside, bz_mode, bz_pulse;
  int bz_off[4];       // table offset of each shape
  int bz_theta0[4];    // first theta index of each shape's radii (kBzRadii)
  double bz_k, bz_kdot, bz_dk[4], bz_dkdot[4];
};
constexpr int kBzRadii = 0, kBzPulse = 1, kBzFixed = 2;
constexpr int kBzMaxShapes = 4, kBzMaxKeys = 4, kBzMaxSeg = 8;

// ------------------------------------------------------------ launches ----
struct Prof;  // CUDA-event timing of one kernel class (util.h)
void prof_begin(Prof *p, int kclass, cudaStream_t s, int *slot);
void prof_end(Prof *p, int slot, cudaStream_t s);

struct Launch {
  cudaStream_t s;
  int64_t *counter;  // host-side count of kernels issued
  Prof *prof;        // null unless nf_profile is active
};

// Brackets one launch with CUDA events when its class is being profiled.
struct ProfScope {
  Prof *p;
  cudaStream_t s;
  int slot = -1;
  ProfScope(const Launch &L, int kclass) : p(L.prof), s(L.s) {
    if (p) prof_begin(p, kclass, s, &slot);
  }
  ~ProfScope() {
    if (p && slot >= 0) prof_end(p, slot, s);
  }
};

// Programmatic dependent launch: kernels launched by launch_pdl may start
// while their predecessor in the stream finishes. Each such kernel first
// waits until the predecessor has completed and its writes are visible,
// then lets its own successor's blocks be scheduled (they wait the same
// way). Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch with programmatic dependent launch allowed (the kernel calls
// pdl_wait() before reading anything its predecessor wrote).
template <class... P, class... A>
inline void launch_pdl(void (*kernel)(P...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, (P)args...);
}

inline unsigned nblocks(int64_t n, int b = kBlock) {
  return (unsigned)((n + b - 1) / b);
}

// ----------------------------------------------------------- reductions ----
// Deterministic grid reduction: every block writes its partial sums, the
// last block to finish adds them in fixed block order. Results do not depend
// on scheduling, so a recomputed forward reproduces the same bits.
struct RedScratch {
  double *partials;      // kRedBlocks * kMaxWidth
  unsigned int *ticket;  // one counter, reset by the last block
};
constexpr int kMaxWidth = 16;

template <int W>
__device__ inline void block_sum(double (&v)[W], double *smem /*W*32*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    double x = v[w];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) smem[w * 32 + warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      double x = lane < nw ? smem[w * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[w] = x;  // valid in thread 0
    }
  }
  __syncthreads();
}

// Write this block's partials; returns true in every thread of the block that
// finishes last, after which `tot` holds the fixed-order grand totals.
template <int W>
__device__ inline bool grid_sum(double (&v)[W], const RedScratch &rs,
                                double (&tot)[W]) {
  __shared__ double smem[W * 32];
  __shared__ bool last;
  block_sum<W>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) rs.partials[blockIdx.x * W + w] = v[w];
    __threadfence();
    unsigned t = atomicAdd(rs.ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[W];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[w] = 0.0;
  // fixed order: thread t sums blocks t, t + blockDim, ... The partials are
  // read past L1 (the scratch is reused by every reduction, so this SM's L1
  // may hold an older kernel's values) and without volatile, so a thread's
  // loads are all in flight before its sums.
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] += __ldcg(&rs.partials[b * W + w]);
  }
  block_sum<W>(acc, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) smem[w] = acc[w];
    *rs.ticket = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int w = 0; w < W; ++w) tot[w] = smem[w];
  __syncthreads();
  return true;
}

// ---------------------------------------------------------- conversions ----
// float -> double by integer operations on the bits (exact): a conversion
// between FP32 and FP64 issues on the FP64 pipe, which runs at 1/64 of the
// FP32 rate on this part. Zero and normal values take the integer path;
// subnormal, infinite and NaN values the conversion instruction.
__device__ __forceinline__ double f2d(float v) {
  const unsigned u = __float_as_uint(v), a = u & 0x7fffffffu, e = a >> 23;
  if (a != 0u && (e == 0u || e == 0xffu)) return (double)v;
  const unsigned sign = u & 0x80000000u;
  const unsigned hi = a == 0u ? sign : (sign | ((e + 896u) << 20) | ((a & 0x7fffffu) >> 3));
  const unsigned lo = a == 0u ? 0u : (u << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// double -> float, rounded to nearest even, by integer operations on the
// bits (the same result as the conversion instruction). Zero takes the
// integer path; values outside the normal FP32 range, infinities and NaN the
// conversion instruction.
__device__ __forceinline__ float d2f(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(u >> 32), sign = hi & 0x80000000u;
  if ((u << 1) == 0ull) return __uint_as_float(sign);
  const int ef = (int)((hi >> 20) & 0x7ffu) - 896;  // FP32 biased exponent
  if (ef <= 0 || ef >= 255) return (float)v;
  const unsigned long long m = u & 0xfffffffffffffull;
  const unsigned keep = (unsigned)(m >> 29), rem = (unsigned)(m & 0x1fffffffull);
  unsigned f = sign | ((unsigned)ef << 23) | keep;
  f += (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u))) ? 1u : 0u;  // may carry
  return __uint_as_float(f);                                                // into the exponent
}
// A value of precision S in the field precision T.
template <class T, class S>
__device__ __forceinline__ T narrow(S v) {
  return (T)v;
}
template <>
__device__ __forceinline__ float narrow<float, double>(double v) {
  return d2f(v);
}
__device__ __forceinline__ float ld(const float *p) { return *p; }
__device__ __forceinline__ double ld(const double *p) { return *p; }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) {
  return __bfloat162float(*p);
}
template <class T>
__device__ __forceinline__ T cvt(double x);
template <>
__device__ __forceinline__ float cvt<float>(double x) { return (float)x; }
template <>
__device__ __forceinline__ double cvt<double>(double x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(double x) {
  return __float2bfloat16((float)x);
}

}  // namespace nf
