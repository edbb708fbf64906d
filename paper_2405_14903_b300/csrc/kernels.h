// Host-side launchers of the libnf kernels (explicitly instantiated in the
// .cu files for the precisions the library uses).
#pragma once

#include "nf_internal.cuh"

namespace nf {

constexpr int kMaxParams = NF_MAX_PARAMS;

template <class T>
struct Fields {
  const T *x, *y, *z;
};
template <class T>
struct FieldsMut {
  T *x, *y, *z;
  operator Fields<T>() const { return Fields<T>{x, y, z}; }
};

// Device-resident state of one conjugate-gradient solve. Every iteration
// kernel returns immediately once `done` is set, so the host may enqueue
// iterations in batches and poll rarely without changing the result.
struct CGState {
  double tol;    // relative tolerance of the inner solve (set by the host)
  double ratio;  // scale of this pass's r over the previous pass's (host)
  int max_it;    // iterations this pass may take (host)
  int loops;     // iteration bodies the device loop ran this pass (host zeroes)
  double rz;     // <r, z>
  double dq;     // <d, A d>
  double rr;     // <r, r>
  double alpha, beta;
  double stop2;  // stop when <r, r> <= stop2
  int iters;
  int done;      // 0 running, 1 converged, 2 breakdown, 3 non-finite
  int err;       // set by the device when a bounded wait expired (host resets)
};

// One multigrid level: dimensions, operator scale c = dt / (rho dx_l) and
// face fractions (component arrays) of type TA.
template <class TA>
struct LevelView {
  int nx, ny, nz;
  double c;
  const TA *ax, *ay, *az;
  __host__ __device__ int64_t ncell() const { return (int64_t)nx * ny * nz; }
};

// ------------------------------------------------------------- step ops ---
template <class T>
void launch_rasterize(const Launch &L, const GridDev &g, const SceneDev &s,
                      FieldsMut<T> alpha);
template <class T>
void launch_advect(const Launch &L, const GridDev &g, Fields<T> u,
                   FieldsMut<T> out, int order);
template <class T>
void launch_advect_adjoint(const Launch &L, const GridDev &g, Fields<T> u,
                           Fields<T> gut, FieldsMut<T> gu, int order);
// Explicit viscosity out = (I - nu h / dx^2 G^T G) in, h = g.dt (also the
// adjoint map: G^T G is symmetric). in and out must not overlap.
template <class T>
void launch_viscosity(const Launch &L, const GridDev &g, Fields<T> in,
                      FieldsMut<T> out);
template <class T, class S>
void launch_rhs(const Launch &L, const GridDev &g, const SceneDev &s,
                Fields<T> alpha, Fields<T> uh, S *b, const RedScratch &rs,
                double *bnorm2);
template <class T, class S>
void launch_update(const Launch &L, const GridDev &g, const SceneDev &s,
                   Fields<T> alpha, Fields<T> uh, const S *P, FieldsMut<T> u);
template <class T>
void launch_loss(const Launch &L, const GridDev &g, int kind, Fields<T> u,
                 FieldsMut<T> gu, bool want_grad, const RedScratch &rs,
                 double *J);
// max |u| over all faces into *out (the bits of a double).
template <class T>
void launch_absmax_faces(const Launch &L, const GridDev &g, Fields<T> u,
                         unsigned long long *out);
template <class T, class S>
void launch_adj_gp(const Launch &L, const GridDev &g, Fields<T> alpha,
                   Fields<T> gu, S *gp, const RedScratch &rs, double *norm2);
template <class T, class S>
void launch_adj_face(const Launch &L, const GridDev &g, const SceneDev &s,
                     Fields<T> alpha, Fields<T> uh, const S *P, const S *y,
                     Fields<T> gu, FieldsMut<T> guh, const RedScratch &rs,
                     double *gtheta);

// ----------------------------------------------------------- solver ops ---
// r = b - A x (fine operator with fractions of type T, x and b of type S),
// written as scale * r converted to V into rin, and ||r||^2 (unscaled).
// scale is a power of two that brings rin to unit size, so that the V-typed
// inner solve neither underflows nor overflows; 2^es is a power of two that
// brings b to unit size (used by the split-float MIXED variant, taken when
// `split` and S = double, T = V = float).
template <class S, class T, class V>
void launch_residual_outer(const Launch &L, const LevelView<T> &lv,
                           const S *b, const S *x, V *rin, double scale, int es,
                           bool split, const RedScratch &rs, double *norm2);
// x += inv * e (V -> S); inv undoes the scale of the inner system.
template <class S, class V>
void launch_axpy_outer(const Launch &L, int64_t n, S *x, const V *e, double inv);
// rin = scale * b (S -> V): the residual of the zero start, b - A 0 = b,
// rounded as the residual kernel rounds its output.
template <class S, class V>
void launch_scale_rhs(const Launch &L, int64_t n, const S *b, V *rin, double scale);

// d = z, <r, z>, <r, r>; stop when <r, r> <= st->tol^2 <r0, r0>.
template <class V>
void launch_cg_init(const Launch &L, int64_t n, const V *r, const V *z, V *d,
                    CGState *st, const RedScratch &rs);
// Continue the previous pass's search direction after its residual was
// replaced by the true one (reliable update): with s = st->ratio,
// beta = <r, z> / (s^2 <r, z>_old) and, through launch_cg_d, d = z + s beta d.
template <class V>
void launch_cg_continue(const Launch &L, int64_t n, const V *r, const V *z,
                        CGState *st, const RedScratch &rs);
template <class V, class TA>
void launch_apply_dot(const Launch &L, const LevelView<TA> &lv, const V *d,
                      V *q, CGState *st, const RedScratch &rs);
// The conditional handles of the device-side CG loop: `body` (WHILE: run
// another iteration) and `tail` (IF: run the rest of this iteration after
// the x, r update).
struct LoopHandles {
  cudaGraphConditionalHandle body, tail;
};
// x += alpha d, r -= alpha q, <r, r>, done when <r, r> <= stop2. With `loop`
// it also sets the loop's conditions: a finished solve skips the rest of the
// iteration and ends the loop.
template <class V>
void launch_cg_xr(const Launch &L, int64_t n, V *x, V *r, const V *d,
                  const V *q, CGState *st, const RedScratch &rs,
                  bool preconditioned, const LoopHandles *loop = nullptr);
template <class V>
void launch_cg_rz(const Launch &L, int64_t n, const V *r, const V *z,
                  CGState *st, const RedScratch &rs);
// *out = <a, b> over n entries, with the dot arithmetic of the CG kernels
// (per-thread partials, fixed-order FP64 block and grid sums).
template <class V>
void launch_dot(const Launch &L, int64_t n, const V *a, const V *b,
                const RedScratch &rs, double *out);
// d = z + beta d. With `loop` (the WHILE handle of the device-side CG loop,
// whose body this launch ends) block 0 also decides whether the loop runs
// another iteration.
template <class V>
void launch_cg_d(const Launch &L, int64_t n, const V *z, V *d, CGState *st,
                 const cudaGraphConditionalHandle *loop = nullptr);

// Multigrid pieces.
// What a red-black half sweep folds into the x it reads (all three give
// the same cell values as the separate passes they replace):
//  kSweepPlain   x as stored;
//  kSweepZero    x = 0 before the sweep: the first half sweep of a level
//                from a zero guess reads no x and needs no zeroing pass (the
//                cells of the other colour are written by the next half
//                sweep, which does not read them);
//  kSweepProlong x += w P x_c before the sweep, P the constant transfer on
//                active cells: only the other colour's prolonged values are
//                read (the swept colour is overwritten without being read,
//                and the next half sweep overwrites the other colour), so
//                the correction is added on the fly and never stored. An
//                inactive neighbour has a zero fraction towards the cell, so
//                adding its correction changes nothing.
constexpr int kSweepPlain = 0, kSweepZero = 1, kSweepProlong = 2;
template <class V>
struct Fold {
  const V *xc;  // coarse correction (kSweepProlong)
  int cnx, cny;
  V w;          // uniform normaliser (sqrt of the coarse-correction weight)
};

template <class TI, class TO>
void launch_mg_coarsen(const Launch &L, const LevelView<TI> &fine,
                       int cnx, int cny, int cnz, TO *ax, TO *ay, TO *az);
// Two half sweeps in one launch: colour c1 in mode kSweep* (fold f), then
// colour 1 - c1 as stored; reads xin (unused in zero-start mode), writes
// every cell of xout (xout != xin). Equal, bit for bit, to the two
// launch_mg_smooth calls on one array.
template <class V, class TA>
void launch_mg_rb_pair(const Launch &L, const LevelView<TA> &lv, const V *xin, V *xout,
                       const V *b, int c1, int mode, const Fold<V> &f, const CGState *st,
                       int kclass);
// Red-black half sweep of colour `color`; mode kSweep* with its fold f.
template <class V, class TA>
void launch_mg_smooth(const Launch &L, const LevelView<TA> &lv, V *x,
                      const V *b, int color, int mode, const Fold<V> &f,
                      const CGState *st, int kclass);
// r = N (b - A x) with N the prolongation normaliser pn (null: N = I).
template <class V, class TA>
void launch_mg_residual(const Launch &L, const LevelView<TA> &lv, const V *x,
                        const V *b, V *r, const float *pn, const CGState *st);
// Constant transfer, fused: b_c = pn / 8 * sum over the eight children of
// (b - A x), without storing the fine residual.
template <class V, class TA>
void launch_mg_resrestrict(const Launch &L, const LevelView<TA> &fine, const V *x,
                           const V *b, int cnx, int cny, int cnz, V *bc, float pn,
                           const CGState *st);
// b_c = R r_f; mode 0: R = P^T / 4 with trilinear P, 1: mean of the eight
// children (P copies the parent).
template <class V, class TA>
void launch_mg_restrict(const Launch &L, const LevelView<TA> &fine,
                        const LevelView<TA> &coarse, const V *rf, V *bc,
                        int mode, const CGState *st);
// x_f += N P x_c on active fine cells (pn null: N = I).
template <class V, class TF, class TC>
void launch_mg_prolong(const Launch &L, const LevelView<TF> &fine,
                       const LevelView<TC> &coarse, const V *xc, V *xf,
                       const float *pn, int mode, const CGState *st);
// pn = N: 1 / (sum of the trilinear prolongation weights of the active
// coarse cells) per fine cell, 0 where none is active.
void launch_mg_fill(const Launch &L, int64_t n, float *p, float v);
template <class TC>
void launch_mg_pnorm(const Launch &L, int fnx, int fny, int fnz,
                     const LevelView<TC> &coarse, float *pn, float scale);

// The levels at and below `first` handled by one thread block: a whole
// V-cycle on the small grids (levels first .. nlev-1), x zeroed inside.
template <class V, class TA>
struct CoarseChain {
  int first, nlev;
  LevelView<TA> lv[kMaxLevels];
  V *x[kMaxLevels];
  V *b[kMaxLevels];
  V *r[kMaxLevels];
  const float *pn[kMaxLevels];  // prolongation normaliser of each level
  int transfer;                 // 0 trilinear, 1 constant (see restrict)
  int smooth;         // sweeps per level
  int coarsest_sweeps;
  int smem_bytes;     // > 0: run the chain in that much dynamic shared memory
  float pnu;          // constant transfer: the uniform normaliser (pn's value)
  int *err;           // set to 1 when a bounded wait of the chain expired
  int stall;          // test hook: expect 16 bytes more than the copies bring
};
template <class V, class TA>
void launch_mg_coarse_chain(const Launch &L, const CoarseChain<V, TA> &ch,
                            const CGState *st);
// Levels lo .. hi-1 of a V-cycle run as phases of one cooperative kernel
// (k_mg_mid), level hi and below by its block 0 as the shared-memory chain.
// Constant transfer only. x of level lo is not read (the first half sweep
// starts from zero); x of level lo holds the post-smoothed correction after.
template <class V, class TA>
struct MidSpan {
  int lo, hi;
  int smooth;         // sweeps per level
  float w;            // uniform normaliser of the constant transfer
  LevelView<TA> lv[kMaxLevels];
  V *x[kMaxLevels];
  V *b[kMaxLevels];
  unsigned *bar;      // barrier counter (zeroed by the launcher)
  int *err;           // set to 1 when a barrier wait expired
  int stall;          // test hook: every barrier waits for one block more
};
// Levels lo .. hi-1 of a V-cycle split into z-slabs over the CTAs of one
// thread-block cluster (k_mg_cluster; each level's nz a multiple of
// 2 kClusterCtas, FP32 data, constant transfer), level hi and below (the
// local chain) on CTA 0. x of level lo is written to x_lo at the end; b of
// level lo is read from b_lo.
constexpr int kClusterCtas = 8;
template <class V, class TA>
struct ClusterSpan {
  int lo, hi;
  int smooth;         // sweeps per level
  float w;            // uniform normaliser of the constant transfer
  LevelView<TA> lv[kMaxLevels];
  int use_dinv[kMaxLevels];  // 1: sweep with the inverse diagonal (as in the chain)
  unsigned off[kMaxLevels][6];  // per-CTA shared memory: x, b, ax, ay, az, dinv
  unsigned chain_off;           // CTA 0's chain region
  V *x_lo;
  const V *b_lo;
  V *b_hi;            // the local chain's b (global), written by the restriction
  const V *x_hi;      // the local chain's x (global), read by the prolongation
};
// Launches k_mg_cluster (one cluster of kClusterCtas CTAs of 1024 threads,
// `smem` bytes of dynamic shared memory each); NF_OK or NF_E_CUDA.
template <class V, class TA>
int launch_mg_cluster(const Launch &L, const ClusterSpan<V, TA> &m,
                      const CoarseChain<V, TA> &ch, const CGState *st, int smem);
// Allows k_mg_cluster `smem` bytes and returns whether one cluster fits.
template <class V, class TA>
bool prepare_mg_cluster(int smem_limit, int smem);

// Launches k_mg_mid cooperatively on `blocks` blocks of 1024 threads with
// the chain's shared memory; returns NF_OK or NF_E_CUDA.
template <class V, class TA>
int launch_mg_mid(const Launch &L, const MidSpan<V, TA> &m,
                  const CoarseChain<V, TA> &ch, const CGState *st, int blocks);
// Co-resident blocks of k_mg_mid with `smem` bytes of dynamic shared memory
// on the current device (0: the cooperative path is unavailable).
template <class V, class TA>
int prepare_mg_mid(int smem_limit, int smem);

// Boundary band of the finest level: active cells with a face alpha < 1 and
// their active neighbours, listed per colour (count[0], count[1]).
template <class TA>
void launch_band_build(const Launch &L, const LevelView<TA> &lv,
                       unsigned char *mark, int *list0, int *list1, int *count);
// Gauss-Seidel update of the listed cells of one colour.
template <class V, class TA>
void launch_band_smooth(const Launch &L, const LevelView<TA> &lv, V *x,
                        const V *b, const int *list, const int *count,
                        const CGState *st);
// Shared memory the chain needs with every level resident (bytes).
template <class V, class TA>
size_t mg_chain_smem_bytes(const CoarseChain<V, TA> &ch);
// Allow the shared-memory chain kernel up to smem_limit bytes (call once per
// device, outside stream capture).
template <class V, class TA>
int prepare_mg_chain(int smem_limit);

// The integer-bit conversions beside the conversion instructions (a check).
void launch_check_conversions(const Launch &L, const double *in, int64_t n, float *out_f,
                              double *out_d, unsigned long long *mismatches);

}  // namespace nf
