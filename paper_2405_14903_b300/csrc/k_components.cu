// Connected fluid components of the active cells and the gauge of the
// components that touch no open face (Sec. 2.3.1, Projection: the cut-cell
// system is singular on such a component, with the constants as null space).
//
// Labelling: lock-free union-find. A union hooks the larger root under the
// smaller one with compare-and-swap, retrying if another thread moved the
// root first, so roots only ever decrease and no cycle can form. Two levels:
// every 8x8x8 tile first unions the faces inside it in shared memory (its
// local root, the smallest local index, is also the smallest global index of
// the tile component: both orders are lexicographic in (k, j, i)); then the
// faces on tile borders are unioned in global memory over that much smaller
// forest, and a last pass points every cell at its root. The root of a
// component is its smallest cell index, so the labels do not depend on
// scheduling.
//
// Gauge: on every floating component the field is shifted to zero mean. The
// per-component sums are accumulated as 64-bit fixed-point integers (scale
// 2^(62 - bits) / max|v| with 2^bits >= the cell count, so no sum overflows),
// whose atomic additions are exact and order independent, so a recomputed
// forward reproduces the same bits.
#include "components.h"

namespace nf {

template <class T>
__device__ __forceinline__ bool active_cell(const GridDev &g, const Fields<T> &a,
                                            int i, int j, int k) {
  return (a.x[g.face(0, i, j, k)] + a.x[g.face(0, i + 1, j, k)] +
          a.y[g.face(1, i, j, k)] + a.y[g.face(1, i, j + 1, k)] +
          a.z[g.face(2, i, j, k)] + a.z[g.face(2, i, j, k + 1)]) > T(0);
}

__device__ __forceinline__ int cc_find(const int *lab, int x) {
  const volatile int *l = lab;
  for (;;) {
    const int p = l[x];
    if (p == x) return x;
    x = p;
  }
}

// Root of x, halving the path on the way (every cell visited is pointed at
// its grandparent, still an ancestor: benign under concurrent updates).
__device__ __forceinline__ int cc_find_halve(int *lab, int x) {
  volatile int *l = lab;
  int p = l[x];
  while (p != x) {
    const int g = l[p];
    if (g != p) l[x] = g;
    x = p;
    p = g;
  }
  return x;
}

__device__ __forceinline__ void cc_union(int *lab, int a, int b);

constexpr int kCcTile = 8;

template <class T>
__global__ void __launch_bounds__(kCcTile * kCcTile * kCcTile)
k_cc_tile(GridDev g, Fields<T> a, int *lab) {
  __shared__ int par[kCcTile * kCcTile * kCcTile];
  const int li = threadIdx.x, lj = threadIdx.y, lk = threadIdx.z;
  const int i0 = blockIdx.x * kCcTile, j0 = blockIdx.y * kCcTile, k0 = blockIdx.z * kCcTile;
  const int i = i0 + li, j = j0 + lj, k = k0 + lk;
  const int t = (lk * kCcTile + lj) * kCcTile + li;
  const bool in = i < g.nx && j < g.ny && k < g.nz;
  const bool act = in && active_cell(g, a, i, j, k);
  par[t] = act ? t : -1;
  __syncthreads();
  if (act) {
    for (int d = 0; d < 3; ++d) {
      const int ni = i + (d == 0), nj = j + (d == 1), nk = k + (d == 2);
      const int mi = li + (d == 0), mj = lj + (d == 1), mk = lk + (d == 2);
      if (mi >= kCcTile || mj >= kCcTile || mk >= kCcTile) continue;
      if (ni >= g.nx || nj >= g.ny || nk >= g.nz) continue;
      const T af = d == 0 ? a.x[g.face(0, ni, j, k)]
                          : (d == 1 ? a.y[g.face(1, i, nj, k)] : a.z[g.face(2, i, j, nk)]);
      if (!(af > T(0))) continue;
      cc_union(par, t, (mk * kCcTile + mj) * kCcTile + mi);
    }
  }
  __syncthreads();
  if (!in) return;
  int root = -1;
  if (act) {
    const int r = cc_find(par, t);
    root = (int)g.cell(i0 + r % kCcTile, j0 + (r / kCcTile) % kCcTile,
                       k0 + r / (kCcTile * kCcTile));
  }
  lab[g.cell(i, j, k)] = root;
}

// Union across tile borders: the faces from a tile's last layer to the next
// tile, in the forest of tile roots. The lanes of a warp hold consecutive
// cells, and across a tile border plane the neighbouring lanes' cells mostly
// carry the same pair of tile labels: a lane whose pair (its label, its
// neighbour's label, as read) equals the previous lane's leaves the union to
// that lane (the two unions join the same two sets, since labels only ever
// point at ancestors). That cuts the contended unions on the tile roots by
// up to the tile width; the labels that result are the same (a component's
// root is its smallest cell index whatever the order of the unions).
template <class T>
__global__ void k_cc_merge(GridDev g, Fields<T> a, int *lab) {
  const int lane = threadIdx.x & 31;
  const int64_t n = g.ncell();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane; base < n;
       base += stride) {
    const int64_t c = base + lane;
    int i = 0, j = 0, k = 0;
    bool bx = false, by = false, bz = false, live = false;
    if (c < n) {
      g.cell_ijk(c, i, j, k);
      bx = (i % kCcTile) == kCcTile - 1;
      by = (j % kCcTile) == kCcTile - 1;
      bz = (k % kCcTile) == kCcTile - 1;
      live = (bx || by || bz) && ((const volatile int *)lab)[c] >= 0;
    }
    for (int d = 0; d < 3; ++d) {
      int la = -1, lb = -1;
      if (live && (d == 0 ? bx : (d == 1 ? by : bz))) {
        const int ni = i + (d == 0), nj = j + (d == 1), nk = k + (d == 2);
        if (ni < g.nx && nj < g.ny && nk < g.nz) {
          const T af = d == 0 ? a.x[g.face(0, ni, j, k)]
                              : (d == 1 ? a.y[g.face(1, i, nj, k)] : a.z[g.face(2, i, j, nk)]);
          if (af > T(0)) {
            la = ((const volatile int *)lab)[c];
            lb = ((const volatile int *)lab)[g.cell(ni, nj, nk)];
          }
        }
      }
      const int pa = __shfl_up_sync(0xffffffffu, la, 1), pb = __shfl_up_sync(0xffffffffu, lb, 1);
      const bool dup = lane > 0 && pa == la && pb == lb;
      if (la >= 0 && lb >= 0 && la != lb && !dup) cc_union(lab, la, lb);
    }
  }
}

__device__ __forceinline__ void cc_union(int *lab, int a, int b) {
  int ra = cc_find_halve(lab, a), rb = cc_find_halve(lab, b);
  while (ra != rb) {
    if (ra > rb) {
      const int t = ra;
      ra = rb;
      rb = t;
    }
    // hook the larger root rb under ra if rb is still a root
    const int old = atomicCAS(lab + rb, rb, ra);
    if (old == rb) return;
    rb = cc_find_halve(lab, old);
    ra = cc_find_halve(lab, ra);
  }
}



__global__ void k_cc_compress(int64_t n, int *lab) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    if (lab[c] >= 0) lab[c] = cc_find(lab, (int)c);
  }
}

// ground[root] = 1 for components with an open box face: a face of the box
// boundary with alpha > 0 (walls and inflow patches have alpha = 0, outlet
// faces 1). For one episode this is the outlet patch; for episodes stacked
// along z (a batched solve) it finds every member's own outlet.
template <class T>
__global__ void k_cc_ground_open(GridDev g, Fields<T> a, const int *lab, int *ground) {
  const int64_t nxw = 2 * (int64_t)g.ny * g.nz, nyw = 2 * (int64_t)g.nx * g.nz,
                nzw = 2 * (int64_t)g.nx * g.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nxw + nyw + nzw;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    T af;
    if (t < nxw) {
      const int hi = (int)(t & 1);
      const int64_t q = t >> 1;
      j = (int)(q % g.ny);
      k = (int)(q / g.ny);
      af = a.x[g.face(0, hi ? g.nx : 0, j, k)];
      i = hi ? g.nx - 1 : 0;
    } else if (t < nxw + nyw) {
      const int64_t u = t - nxw;
      const int hi = (int)(u & 1);
      const int64_t q = u >> 1;
      i = (int)(q % g.nx);
      k = (int)(q / g.nx);
      af = a.y[g.face(1, i, hi ? g.ny : 0, k)];
      j = hi ? g.ny - 1 : 0;
    } else {
      const int64_t u = t - nxw - nyw;
      const int hi = (int)(u & 1);
      const int64_t q = u >> 1;
      i = (int)(q % g.nx);
      j = (int)(q / g.nx);
      af = a.z[g.face(2, i, j, hi ? g.nz : 0)];
      k = hi ? g.nz - 1 : 0;
    }
    if (!(af > T(0))) continue;
    const int r = lab[g.cell(i, j, k)];
    if (r >= 0) ground[r] = 1;
  }
}

// Counts the floating roots into *nfloat and gives each a slot.
__global__ void k_cc_count(int64_t n, const int *lab, const int *ground,
                           int *nfloat, int *fslot) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    if (lab[c] == (int)c && !ground[c]) fslot[c] = atomicAdd(nfloat, 1);
}

// Cells per floating slot (warp-aggregated: the lanes of a warp usually
// share one component).
__global__ void k_cc_fcount(int64_t n, const int *lab, const int *ground,
                            const int *fslot, int *fcnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x; c0 < n;
       c0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = c0 + threadIdx.x;
    int slot = -1;
    if (c < n) {
      const int r = lab[c];
      if (r >= 0 && !ground[r]) slot = fslot[r];
    }
    const unsigned same = __match_any_sync(0xffffffffu, slot);
    if (slot >= 0 && lane == __ffs(same) - 1) atomicAdd(fcnt + slot, __popc(same));
  }
}

__device__ __forceinline__ bool floating(const int *lab, const int *ground,
                                         int64_t c, int &r) {
  r = lab[c];
  return r >= 0 && !ground[r];
}

template <class S>
__global__ void k_gauge_max(int64_t n, const int *lab, const int *ground,
                            const S *v, unsigned long long *mx) {
  double m = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    int r;
    if (floating(lab, ground, c, r)) m = fmax(m, fabs((double)v[c]));
  }
  // bit patterns of non-negative doubles order like their values
  if (m > 0.0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

__device__ __forceinline__ double fixed_scale(unsigned long long mxbits,
                                              int bits) {
  const double mx = __longlong_as_double((long long)mxbits);
  int e = 0;
  frexp(mx > 0.0 ? mx : 1.0, &e);  // mx < 2^e
  return ldexp(1.0, 62 - bits - e);
}

template <class S>
__global__ void k_gauge_sum(int64_t n, const int *lab, const int *ground,
                            const S *v, const unsigned long long *mx, int bits,
                            unsigned long long *csum, int *ccnt) {
  const double sc = fixed_scale(*mx, bits);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    int r;
    if (!floating(lab, ground, c, r)) continue;
    const long long q = llrint((double)v[c] * sc);
    atomicAdd(csum + r, (unsigned long long)q);
    atomicAdd(ccnt + r, 1);
  }
}

template <class S>
__global__ void k_gauge_sub(int64_t n, const int *lab, const int *ground, S *v,
                            const unsigned long long *mx, int bits,
                            const unsigned long long *csum, const int *ccnt,
                            RedScratch rs, double *norm2) {
  const double sc = fixed_scale(*mx, bits);
  double acc[1] = {0.0};
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    int r;
    double x = (double)v[c];
    if (floating(lab, ground, c, r)) {
      const double mean = (double)(long long)csum[r] / sc / (double)ccnt[r];
      x -= mean;
      v[c] = (S)x;
    }
    acc[0] += x * x;
  }
  double tot[1];
  if (grid_sum<1>(acc, rs, tot) && threadIdx.x == 0) *norm2 = tot[0];
}

// ------------------------------------------- projection inside the solve ---
// v -= mean per floating component, with the component sums accumulated in
// 64-bit fixed point (exact, order independent) and combined per warp before
// the atomics: on a domain that floats as a whole every cell has one slot.
template <class V>
__global__ void k_proj_max(int64_t n, const int *lab, const int *ground,
                           const int *nfloat, const V *v, unsigned long long *mx) {
  if (*(volatile const int *)nfloat == 0) return;
  double m = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int r = lab[c];
    if (r >= 0 && !ground[r]) m = fmax(m, fabs((double)v[c]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_proj_zero(const int *nfloat, unsigned long long *fsum) {
  const int nf = *(volatile const int *)nfloat;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nf; s += gridDim.x * blockDim.x)
    fsum[s] = 0ull;
}

template <class V>
__global__ void k_proj_sum(int64_t n, const int *lab, const int *ground,
                           const int *nfloat, const int *fslot, const V *v,
                           const unsigned long long *mx, int bits,
                           unsigned long long *fsum) {
  if (*(volatile const int *)nfloat == 0) return;
  const double sc = fixed_scale(*mx, bits);
  const int lane = threadIdx.x & 31;
  for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x; c0 < n;
       c0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = c0 + threadIdx.x;
    int slot = -1;
    long long q = 0;
    if (c < n) {
      const int r = lab[c];
      if (r >= 0 && !ground[r]) {
        slot = fslot[r];
        q = llrint((double)v[c] * sc);
      }
    }
    const unsigned same = __match_any_sync(0xffffffffu, slot);
    if (same == 0xffffffffu) {
      // one slot for the whole warp: add the 64-bit values in registers
      for (int o = 16; o > 0; o >>= 1) q += __shfl_down_sync(0xffffffffu, q, o);
      if (lane == 0 && slot >= 0) atomicAdd(fsum + slot, (unsigned long long)q);
    } else if (slot >= 0) {
      atomicAdd(fsum + slot, (unsigned long long)q);
    }
  }
}

template <class V>
__global__ void k_proj_sub(int64_t n, const int *lab, const int *ground,
                           const int *nfloat, const int *fslot, V *v,
                           const unsigned long long *mx, int bits,
                           const unsigned long long *fsum, const int *fcnt) {
  if (*(volatile const int *)nfloat == 0) return;
  const double sc = fixed_scale(*mx, bits);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int r = lab[c];
    if (r < 0 || ground[r]) continue;
    const int s = fslot[r];
    v[c] = (V)((double)v[c] - (double)(long long)fsum[s] / sc / (double)fcnt[s]);
  }
}

// ------------------------------------------------------------ launchers ---
static inline unsigned cc_blocks(int64_t n) {
  const unsigned b = nblocks(n);
  return b < 148u * 16u ? b : 148u * 16u;
}

template <class T>
int Components::label(Ctx *ctx, const GridDev &g, Fields<T> alpha) {
  Launch L = ctx->launch();
  const int64_t n = g.ncell();
  int h[2] = {0, 0};
  {
    ProfScope _ps(L, NF_K_GAUGE);
    const dim3 tiles((g.nx + kCcTile - 1) / kCcTile, (g.ny + kCcTile - 1) / kCcTile,
                     (g.nz + kCcTile - 1) / kCcTile);
    k_cc_tile<T><<<tiles, dim3(kCcTile, kCcTile, kCcTile), 0, L.s>>>(g, alpha, lab);
    k_cc_merge<T><<<cc_blocks(n), kBlock, 0, L.s>>>(g, alpha, lab);
    k_cc_compress<<<cc_blocks(n), kBlock, 0, L.s>>>(n, lab);
    *L.counter += 3;
  }
  cudaMemsetAsync(ground, 0, n * sizeof(int), L.s);
  cudaMemsetAsync((int *)scal + 1, 0, sizeof(int), L.s);
  {
    ProfScope _ps(L, NF_K_GAUGE);
    const int64_t nw = 2 * ((int64_t)g.ny * g.nz + (int64_t)g.nx * g.nz + (int64_t)g.nx * g.ny);
    k_cc_ground_open<T><<<cc_blocks(nw), kBlock, 0, L.s>>>(g, alpha, lab, ground);
    k_cc_count<<<cc_blocks(n), kBlock, 0, L.s>>>(n, lab, ground, (int *)scal + 1, fslot);
    *L.counter += 2;
  }
  ctx->read_bytes(h, scal, 2 * sizeof(int));
  nfloat = h[1];
  if (nfloat > 0) {
    cudaMemsetAsync(fcnt, 0, (size_t)nfloat * sizeof(int), L.s);
    ProfScope _ps(L, NF_K_GAUGE);
    k_cc_fcount<<<cc_blocks(n), kBlock, 0, L.s>>>(n, lab, ground, fslot, fcnt);
    ++*L.counter;
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NF_OK : cuda_fail(e, "component labelling");
}

template <class S>
double Components::gauge(Ctx *ctx, int64_t n, S *v, double norm2) {
  if (nfloat == 0) return norm2;
  Launch L = ctx->launch();
  unsigned long long *mx = (unsigned long long *)((char *)scal + 16);
  double *nrm = (double *)((char *)scal + 24);
  cudaMemsetAsync(mx, 0, sizeof(unsigned long long), L.s);
  cudaMemsetAsync(csum, 0, n * sizeof(unsigned long long), L.s);
  cudaMemsetAsync(ccnt, 0, n * sizeof(int), L.s);
  int bits = 1;
  while (bits < 40 && ((int64_t)1 << bits) < n) ++bits;
  ProfScope _ps(L, NF_K_GAUGE);
  k_gauge_max<S><<<cc_blocks(n), kBlock, 0, L.s>>>(n, lab, ground, v, mx);
  k_gauge_sum<S><<<cc_blocks(n), kBlock, 0, L.s>>>(n, lab, ground, v, mx, bits, csum,
                                                   ccnt);
  k_gauge_sub<S><<<kRedBlocks, kBlock, 0, L.s>>>(n, lab, ground, v, mx, bits, csum, ccnt,
                                                 ctx->rs, nrm);
  *L.counter += 3;
  return ctx->read_double(nrm);
}

template <class V>
void Components::project(const Launch &L, int64_t n, V *v) {
  const int *nf = (const int *)scal + 1;
  unsigned long long *mx = (unsigned long long *)((char *)scal + 32);
  int bits = 1;
  while (bits < 40 && ((int64_t)1 << bits) < n) ++bits;
  cudaMemsetAsync(mx, 0, sizeof(unsigned long long), L.s);
  ProfScope _ps(L, NF_K_GAUGE);
  k_proj_max<V><<<cc_blocks(n), kBlock, 0, L.s>>>(n, lab, ground, nf, v, mx);
  k_proj_zero<<<64, kBlock, 0, L.s>>>(nf, fsum);
  k_proj_sum<V><<<cc_blocks(n), kBlock, 0, L.s>>>(n, lab, ground, nf, fslot, v, mx, bits,
                                                  fsum);
  k_proj_sub<V><<<cc_blocks(n), kBlock, 0, L.s>>>(n, lab, ground, nf, fslot, v, mx, bits,
                                                  fsum, fcnt);
  *L.counter += 4;
}

int Components::init(Alloc &A, int64_t n) {
  CKS(A.get(&lab, n * sizeof(int)));
  CKS(A.get(&ground, n * sizeof(int)));
  CKS(A.get(&ccnt, n * sizeof(int)));
  CKS(A.get(&csum, n * sizeof(unsigned long long)));
  CKS(A.get(&fslot, n * sizeof(int)));
  CKS(A.get(&fcnt, n * sizeof(int)));
  CKS(A.get(&fsum, n * sizeof(unsigned long long)));
  CKS(A.get(&scal, 64));
  return NF_OK;
}

template void Components::project<float>(const Launch &, int64_t, float *);
template void Components::project<double>(const Launch &, int64_t, double *);

template int Components::label<float>(Ctx *, const GridDev &, Fields<float>);
template int Components::label<double>(Ctx *, const GridDev &, Fields<double>);
template double Components::gauge<float>(Ctx *, int64_t, float *, double);
template double Components::gauge<double>(Ctx *, int64_t, double *, double);

}  // namespace nf
