// Host orchestration of the pressure solve A P = b (Eq. projection_matrix).
//
// Outer loop: iterative refinement in precision S, r = b - A P computed with
// FP64 arithmetic (k_residual_outer); inner loop: CG (plain or V-cycle
// preconditioned) in precision V on A e = r, then P += e. With S = V the
// inner solve targets the final tolerance and the outer loop only confirms
// it; with S = double, V = float (MIXED) each inner solve reduces the
// residual by `inner_tol`. A pass that follows a converged pass keeps its
// search direction (reliable update: the recurrence residual is replaced by
// the true FP64 one and CG continues) while the two residuals agree, so the
// Krylov space is not lost at every refinement.
//
// Iteration kernels stop themselves once the device-side CGState says the
// solve is done, so iterations are enqueued in batches and the host polls
// the state once per batch.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "components.h"
#include "kernels.h"
#include "util.h"

namespace nf {

struct SolveStats {
  int iters = 0;
  int outer = 0;
  double rel = 0.0;
  int status = NF_OK;
};

template <class T, class S, class V, class TA>
class Solver {
 public:
  // The operator is the unit-scale G^T S G (c = 1 on the finest level,
  // c_l = 2^-l below); callers pass b / c for A = c G^T S G.
  Solver(Ctx *ctx, const GridDev &g, const nf_config &cfg)
      : ctx_(ctx), g_(g), cfg_(cfg) {
    g_.c = 1.0;
    // NF_GRAPHS=0: launch every kernel directly (for profilers that cannot
    // follow stream capture); the kernels and results are the same
    const char *env = std::getenv("NF_GRAPHS");
    if (env && std::strcmp(env, "0") == 0) graphs_ok_ = false;
    // NF_TEST_STALL_WAITS=1: the device's bounded waits (grid barriers,
    // the chain's mbarrier) wait for something that never comes, so that
    // a test sees them expire into NF_E_TIMEOUT
    const char *stall = std::getenv("NF_TEST_STALL_WAITS");
    stall_ = stall && std::strcmp(stall, "1") == 0 ? 1 : 0;
  }

  // At most this many multigrid levels (a batched solve keeps every level
  // of the stacked grid aligned with its members' own levels).
  void set_max_levels(int n) { max_levels_ = std::max(1, std::min(n, kMaxLevels)); }

  // Allocates the hierarchy. Returns NF_OK or an error status.
  int init(Alloc &A) {
    n_ = g_.ncell();
    CKS(A.get(&rin_, n_ * sizeof(V)));
    CKS(A.get(&e_, n_ * sizeof(V)));
    CKS(A.get(&z_, n_ * sizeof(V)));
    CKS(A.get(&d_, n_ * sizeof(V)));
    CKS(A.get(&q_, n_ * sizeof(V)));
    CKS(A.get(&st_, sizeof(CGState)));
    CKS(A.get(&norm2_, 2 * sizeof(double)));
    mg_ = cfg_.solver == NF_SOLVER_MGPCG;
    // level 0 uses the episode's fractions (type T); levels >= 1 own TA arrays
    int nx = g_.nx, ny = g_.ny, nz = g_.nz;
    double c = g_.c;
    levels_.clear();
    levels_.push_back(Level{nx, ny, nz, c});
    if (mg_) {
      const int mn = std::max(2, cfg_.mg_coarsest);
      while (nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0 && nx / 2 >= mn &&
             ny / 2 >= mn && nz / 2 >= mn && (int)levels_.size() < max_levels_) {
        nx /= 2;
        ny /= 2;
        nz /= 2;
        c *= 0.5;  // c_l = dt / (rho dx_l), dx_l = 2 dx_{l-1}
        levels_.push_back(Level{nx, ny, nz, c});
      }
      for (size_t l = 0; l < levels_.size(); ++l) {
        Level &L = levels_[l];
        const int64_t nc = (int64_t)L.nx * L.ny * L.nz;
        if (l > 0) {
          CKS(A.get(&L.ax, (int64_t)(L.nx + 1) * L.ny * L.nz * sizeof(TA)));
          CKS(A.get(&L.ay, (int64_t)L.nx * (L.ny + 1) * L.nz * sizeof(TA)));
          CKS(A.get(&L.az, (int64_t)L.nx * L.ny * (L.nz + 1) * sizeof(TA)));
          CKS(A.get(&L.x, nc * sizeof(V)));
          CKS(A.get(&L.b, nc * sizeof(V)));
        }
        CKS(A.get(&L.r, nc * sizeof(V)));
        CKS(A.get(&L.pn, nc * sizeof(float)));
      }
      if (cfg_.mg_band_sweeps > 0 && levels_.size() > 1) {
        CKS(A.get(&band_mark_, n_));
        CKS(A.get(&band_list_[0], (n_ / 2 + 1) * sizeof(int)));
        CKS(A.get(&band_list_[1], (n_ / 2 + 1) * sizeof(int)));
        CKS(A.get(&band_count_, 2 * sizeof(int)));
      }
      // first level handled inside the one-block chain kernel
      first_chain_ = (int)levels_.size() - 1;
      while (first_chain_ > 0) {
        const Level &L = levels_[first_chain_ - 1];
        if ((int64_t)L.nx * L.ny * L.nz > kChainCells) break;
        --first_chain_;
      }
      // run the chain from shared memory when all of its levels fit
      const int nl = (int)levels_.size();
      const int down = std::min(std::max(1, first_chain_), nl - 1);
      int limit = 0;
      if (nl > 1) {
        int dev = 0;
        CKC(cudaGetDevice(&dev));
        CKC(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        // (headroom for the kernels' few static shared variables)
        const size_t need = mg_chain_smem_bytes(chain(down));
        if (need + 1024 <= (size_t)limit) {
          const int rc = prepare_mg_chain<V, TA>(limit);
          if (rc != NF_OK) return rc;
          chain_smem_ = (int)need;
        }
      }
      // the small grid levels above the chain (at most kMidCells cells)
      // run, with the chain, inside one cooperative kernel: one warp per row
      // of the largest of them, capped at the co-resident blocks
      if (cfg_.mg_persistent && cfg_.mg_transfer == 1 && chain_smem_ > 0 && nl > 2) {
        int lo = down;
        while (lo > 1 && (int64_t)levels_[lo - 1].nx * levels_[lo - 1].ny * levels_[lo - 1].nz <=
                             kMidCells)
          --lo;
        if (lo < down) {
          const int cap = prepare_mg_mid<V, TA>(limit, chain_smem_);
          const int want = (levels_[lo].ny * levels_[lo].nz + 31) / 32;
          if (cap > 0) {
            CKS(A.get(&bar_, sizeof(unsigned)));
            mid_lo_ = lo;
            mid_blocks_ = std::min(cap, std::max(1, want));
          }
        }
      }
      // otherwise the levels just above an 8^3-or-smaller local chain whose
      // planes split evenly (an even number per CTA) run on one thread-block
      // cluster, the local chain on its CTA 0
      if (cfg_.mg_cluster && !mid_lo_ && sizeof(V) == 4 && cfg_.mg_transfer == 1 && nl > 2 &&
          chain_smem_ > 0) {
        int lo = -1, hi = -1;
        for (int l = 1; l < nl - 1; ++l) {
          const Level &L = levels_[l];
          const int64_t nc = (int64_t)L.nx * L.ny * L.nz;
          const bool ok = nc > 512 && nc <= kClusterCells && L.nz % (2 * kClusterCtas) == 0;
          if (ok && lo < 0) lo = l;
          if (lo >= 0) {
            if (!ok) break;
            hi = l + 1;
          }
        }
        if (lo >= 1 && hi > lo && hi < nl) {
          size_t o = 0;
          auto take = [&o](size_t bytes) {
            const size_t at = o;
            o += (bytes + 15) & ~(size_t)15;
            return (unsigned)at;
          };
          for (int l = lo; l < hi; ++l) {
            const Level &L = levels_[l];
            const size_t P = (size_t)L.nz / kClusterCtas, nxy = (size_t)L.nx * L.ny;
            cl_off_[l][0] = take(P * nxy * sizeof(V));
            cl_off_[l][1] = take(P * nxy * sizeof(V));
            cl_off_[l][2] = take(P * L.ny * (L.nx + 1) * sizeof(TA));
            cl_off_[l][3] = take(P * (L.ny + 1) * L.nx * sizeof(TA));
            cl_off_[l][4] = take((P + 1) * nxy * sizeof(TA));
            cl_off_[l][5] = l >= down ? take(P * nxy * sizeof(V)) : 0u;
          }
          cl_chain_off_ = (unsigned)o;
          const size_t total = o + mg_chain_smem_bytes(chain(hi));
          if (total + 1024 <= (size_t)limit && prepare_mg_cluster<V, TA>(limit, (int)total)) {
            cl_lo_ = lo;
            cl_hi_ = hi;
            cl_smem_ = (int)total;
          }
        }
      }
    }
    return NF_OK;
  }

  // New fractions for level 0 (device arrays of type T): rebuild coarse
  // fractions (mean of the four fine sub-faces).
  void set_fractions(const T *ax, const T *ay, const T *az) {
    ax0_ = ax;
    ay0_ = ay;
    az0_ = az;
    if (!mg_) return;
    Launch L = ctx_->launch();
    if (band_count_)
      launch_band_build<T>(L, view0(), (unsigned char *)band_mark_, (int *)band_list_[0],
                           (int *)band_list_[1], (int *)band_count_);
    for (size_t l = 1; l < levels_.size(); ++l) {
      Level &C = levels_[l];
      if (l == 1)
        launch_mg_coarsen<T, TA>(L, view0(), C.nx, C.ny, C.nz, (TA *)C.ax,
                                 (TA *)C.ay, (TA *)C.az);
      else
        launch_mg_coarsen<TA, TA>(L, viewc(l - 1), C.nx, C.ny, C.nz,
                                  (TA *)C.ax, (TA *)C.ay, (TA *)C.az);
    }
    for (size_t l = 0; l + 1 < levels_.size(); ++l) {
      const Level &F = levels_[l];
      const float w = coarse_w();
      if (cfg_.mg_transfer == 0)
        launch_mg_pnorm<TA>(L, F.nx, F.ny, F.nz, viewc(l + 1), (float *)F.pn, w);
      else  // a constant P needs no normaliser
        launch_mg_fill(L, (int64_t)F.nx * F.ny * F.nz, (float *)F.pn, w);
    }
  }

  // Solve A x = b (x overwritten). bnorm2 is ||b||^2 already on the host.
  // The tolerance is relative to tol_norm2 when given (> 0), else to
  // bnorm2: a batched solve of stacked, decoupled systems stops when
  // ||r|| <= tol min_e ||b_e||, which bounds every member's own residual.
  SolveStats solve(const S *b, S *x, double bnorm2, double tol_norm2 = 0.0) {
    SolveStats out;
    Launch L = ctx_->launch();
    cudaMemsetAsync(x, 0, n_ * sizeof(S), L.s);
    cudaMemsetAsync(&((CGState *)st_)->err, 0, sizeof(int), L.s);
    if (!(bnorm2 > 0.0)) {
      out.rel = 0.0;
      if (!std::isfinite(bnorm2)) out.status = NF_E_DIVERGED;
      return out;
    }
    const double tol = cfg_.tol;
    const bool mixed = sizeof(S) != sizeof(V);
    proj_now_ = mg_ && proj_ != nullptr && proj_->nfloat > 0;
    // the inner system is solved for scale * r, scale a power of two close
    // to 1 / ||r||: tiny right-hand sides (an adjoint far from its loss)
    // would otherwise underflow in the V-typed dots
    double scale = unit_scale(std::sqrt(bnorm2));
    es_ = std::max(-900, std::min(900, -std::ilogb(std::sqrt(bnorm2))));
    const double tn2 = tol_norm2 > 0.0 ? tol_norm2 : bnorm2;
    // r = b - A 0 = b: the scaled right-hand side, no stencil evaluation
    launch_scale_rhs<S, V>(L, n_, b, (V *)rin_, scale);
    double rn2 = bnorm2;
    out.rel = std::sqrt(rn2 / tn2);
    int total = 0;
    double prev_scale = scale;
    bool can_cont = false;
    for (int pass = 0; pass < kMaxOuter && out.rel > tol; ++pass) {
      if (!std::isfinite(rn2)) {
        out.status = NF_E_DIVERGED;
        break;
      }
      double inner = mixed ? std::max(cfg_.inner_tol, 0.5 * tol / out.rel)
                           : 0.5 * tol / out.rel;
      inner = std::min(inner, 0.5);
      int it = 0, done = 0;
      double rr_in = 0.0;
      const bool cont = pass > 0 && can_cont;
      inner_solve(inner, cfg_.max_iters - total, &it, &done, &rr_in, cont,
                  scale / prev_scale);
      if (cont && done == 2 && it == 0)  // no usable direction: start afresh
        inner_solve(inner, cfg_.max_iters - total, &it, &done, &rr_in, false, 1.0);
      prev_scale = scale;
      total += it;
      out.outer += 1;
      if (done == 5) {  // a bounded device wait expired
        out.status = NF_E_TIMEOUT;
        break;
      }
      launch_axpy_outer<S, V>(L, n_, x, (const V *)e_, 1.0 / scale);
      // next scale from the inner recurrence's final residual (unscaled),
      // floored at the V rounding level of the current residual
      const double rn = std::sqrt(rn2);
      const double pred = std::max(std::sqrt(rr_in) / scale, 1e-7 * rn);
      scale = unit_scale(pred);
      rn2 = residual(b, x, scale);
      out.rel = std::sqrt(rn2 / tn2);
      // the next pass may keep the search direction only while the
      // recurrence residual still tracks the true one (it drifts below it
      // once V rounding stalls the true residual)
      can_cont = done == 1 && std::sqrt(rn2) <= 2.0 * std::sqrt(rr_in) / prev_scale;
      if (done == 3 || !std::isfinite(rn2)) {
        out.status = NF_E_DIVERGED;
        break;
      }
      if (total >= cfg_.max_iters) break;
      if (done == 2 && it == 0) break;  // no progress possible
    }
    out.iters = total;
    if (out.status == NF_OK && out.rel > tol) out.status = NF_E_NOT_CONVERGED;
    return out;
  }

  int levels() const { return (int)levels_.size(); }

  // Components of the episode, whose floating part the preconditioner
  // projects out (labels must be current when solve() is called).
  void set_projector(Components *c) { proj_ = c; }

 private:
  struct Level {
    int nx, ny, nz;
    double c;
    void *ax = nullptr, *ay = nullptr, *az = nullptr;
    void *x = nullptr, *b = nullptr, *r = nullptr;
    void *pn = nullptr;  // prolongation normaliser (levels with a coarser one)
  };
  static constexpr int kMaxOuter = 12;
  int max_levels_ = kMaxLevels;
  static constexpr int kChainCells = 16 * 16 * 16;
  static constexpr int64_t kMidCells = 64 * 64 * 64;
  static constexpr int64_t kClusterCells = 32 * 32 * 32;
  static constexpr int kBatch = 4;
  int coarsest_sweeps() const {
    return cfg_.mg_coarsest_sweeps > 0 ? cfg_.mg_coarsest_sweeps : 8;
  }
  // sqrt of the coarse-correction weight, applied on each side (P' = w P,
  // R' = w R) so that R' = P'^T / 8 stays the transpose pair
  float coarse_w() const {
    return (float)std::sqrt(cfg_.mg_coarse_weight > 0 ? cfg_.mg_coarse_weight : 1.0);
  }
  int nu_coarse() const {
    return cfg_.mg_smooth_coarse > 0 ? cfg_.mg_smooth_coarse : std::max(1, cfg_.mg_smooth);
  }

  LevelView<T> view0() const {
    return LevelView<T>{g_.nx, g_.ny, g_.nz, g_.c, ax0_, ay0_, az0_};
  }
  LevelView<TA> viewc(size_t l) const {
    const Level &L = levels_[l];
    return LevelView<TA>{L.nx, L.ny, L.nz, L.c, (const TA *)L.ax,
                         (const TA *)L.ay, (const TA *)L.az};
  }

  // 2^-e with 2^e within a factor 2 of v (1 when v is 0 or not finite)
  static double unit_scale(double v) {
    if (!(v > 0.0) || !std::isfinite(v)) return 1.0;
    return std::ldexp(1.0, -std::ilogb(v));
  }

  double residual(const S *b, const S *x, double scale) {
    Launch L = ctx_->launch();
    launch_residual_outer<S, T, V>(L, view0(), b, x, (V *)rin_, scale, es_,
                                   cfg_.residual_fp64 == 0, ctx_->rs, (double *)norm2_);
    return ctx_->read_double((double *)norm2_);
  }

  void smooth(int l, V *x, const V *b, int color, const CGState *st,
              int mode = kSweepPlain, const Fold<V> &f = Fold<V>{nullptr, 0, 0, V(0)}) {
    Launch L = ctx_->launch();
    if (l == 0)
      launch_mg_smooth<V, T>(L, view0(), x, b, color, mode, f, st, NF_K_MG_SMOOTH0);
    else
      launch_mg_smooth<V, TA>(L, viewc(l), x, b, color, mode, f, st, NF_K_MG_SMOOTH);
  }

  // Extra sweeps on the finest level's boundary band: red-black before the
  // pre-smoothing (first = 0), black-red after the post-smoothing (first =
  // 1), so the V-cycle stays symmetric.
  void band(V *x, const V *b, int first, const CGState *st) {
    if (!band_count_) return;
    Launch L = ctx_->launch();
    const int *cnt = (const int *)band_count_;
    for (int s = 0; s < cfg_.mg_band_sweeps; ++s) {
      launch_band_smooth<V, T>(L, view0(), x, b, (const int *)band_list_[first], cnt + first, st);
      launch_band_smooth<V, T>(L, view0(), x, b, (const int *)band_list_[first ^ 1],
                               cnt + (first ^ 1), st);
    }
  }

  // Prolongation normaliser of level l for the grid kernels (null: none).
  const float *pnorm(int l) const {
    const bool unit = cfg_.mg_transfer != 0 &&
                      (cfg_.mg_coarse_weight == 1.0 || cfg_.mg_coarse_weight == 0.0);
    return unit ? nullptr : (const float *)levels_[l].pn;
  }

  CoarseChain<V, TA> chain(int first) const {
    CoarseChain<V, TA> ch;
    ch.first = first;
    ch.nlev = (int)levels_.size();
    for (int l = first; l < ch.nlev; ++l) {
      ch.lv[l] = viewc(l);
      ch.x[l] = (V *)levels_[l].x;
      ch.b[l] = (V *)levels_[l].b;
      ch.r[l] = (V *)levels_[l].r;
      ch.pn[l] = (const float *)levels_[l].pn;
    }
    ch.transfer = cfg_.mg_transfer;
    ch.smooth = nu_coarse();
    ch.coarsest_sweeps = coarsest_sweeps();
    ch.smem_bytes = chain_smem_;
    ch.pnu = coarse_w();
    ch.err = &((CGState *)st_)->err;
    ch.stall = stall_;
    return ch;
  }

  ClusterSpan<V, TA> cluster() const {
    ClusterSpan<V, TA> m{};
    m.lo = cl_lo_;
    m.hi = cl_hi_;
    m.smooth = nu_coarse();
    m.w = coarse_w();
    const int down = std::min(std::max(1, first_chain_), (int)levels_.size() - 1);
    for (int l = cl_lo_; l <= cl_hi_; ++l) m.lv[l] = viewc(l);
    for (int l = cl_lo_; l < cl_hi_; ++l) {
      m.use_dinv[l] = l >= down ? 1 : 0;
      for (int q = 0; q < 6; ++q) m.off[l][q] = cl_off_[l][q];
    }
    m.chain_off = cl_chain_off_;
    m.x_lo = (V *)levels_[cl_lo_].x;
    m.b_lo = (const V *)levels_[cl_lo_].b;
    m.b_hi = (V *)levels_[cl_hi_].b;
    m.x_hi = (const V *)levels_[cl_hi_].x;
    return m;
  }

  MidSpan<V, TA> mid(int lo, int hi) const {
    MidSpan<V, TA> m{};
    m.lo = lo;
    m.hi = hi;
    m.smooth = nu_coarse();
    m.w = coarse_w();
    for (int l = lo; l <= hi; ++l) {
      m.lv[l] = viewc(l);
      m.x[l] = (V *)levels_[l].x;
      m.b[l] = (V *)levels_[l].b;
    }
    m.bar = (unsigned *)bar_;
    m.err = &((CGState *)st_)->err;
    m.stall = stall_;
    return m;
  }

  // z = M r: one symmetric V-cycle (red-black pre-smoothing, black-red
  // post-smoothing) from z = 0. Levels above kChainCells cells run as grid
  // kernels, the small ones inside one thread block.
  // z = P M r with P the zero-mean projection of every floating component
  // (when the system has one): on a singular system the V-cycle's coarse
  // sweeps add a null-space constant that grows once rounding makes r
  // slightly inconsistent, and P keeps the preconditioner on the range.
  void precondition(const V *r, V *z, const CGState *st) {
    vcycle(r, z, st);
    if (proj_now_) proj_->project<V>(ctx_->launch(), n_, z);
  }

  void vcycle(const V *r, V *z, const CGState *st) {
    Launch L = ctx_->launch();
    const int nl = (int)levels_.size();
    if (nl == 1) {
      // no coarser grid: symmetric Gauss-Seidel sweeps only
      cudaMemsetAsync(z, 0, n_ * sizeof(V), L.s);
      for (int s = 0; s < coarsest_sweeps(); ++s) {
        smooth(0, z, r, 0, st);
        smooth(0, z, r, 1, st);
      }
      for (int s = 0; s < coarsest_sweeps(); ++s) {
        smooth(0, z, r, 1, st);
        smooth(0, z, r, 0, st);
      }
      return;
    }
    const int F = std::max(1, first_chain_);  // level 0 always on grid kernels
    const int down = std::min(F, nl - 1);     // levels with a coarser level
    // levels [0, gl) as one launch per phase; [gl, down) and the chain in
    // one cooperative kernel when that is set up, else per phase too
    const int gl = mid_lo_ > 0 ? mid_lo_ : (cl_lo_ > 0 ? cl_lo_ : down);
    down_levels(0, gl, r, z, st);
    bool done = false;
    if (mid_lo_ > 0) {
      if (launch_mg_mid<V, TA>(L, mid(gl, down), chain(down), st, mid_blocks_) == NF_OK) {
        done = true;
      } else {  // no cooperative launch here: per-phase launches from now on
        cudaGetLastError();
        mid_lo_ = 0;
      }
    } else if (cl_lo_ > 0) {
      if (launch_mg_cluster<V, TA>(L, cluster(), chain(cl_hi_), st, cl_smem_) == NF_OK) {
        done = true;
      } else {  // no cluster launch here: per-phase launches from now on
        cudaGetLastError();
        cl_lo_ = 0;
      }
    }
    if (!done) {
      down_levels(gl, down, r, z, st);
      launch_mg_coarse_chain<V, TA>(L, chain(down), st);
      up_levels(gl, down, r, z, st);
    }
    up_levels(0, gl, r, z, st);
  }

  // Pre-smoothing and restriction of levels lo .. hi-1 (level 0: x = z,
  // b = r), one launch per phase. x starts from zero: the first half sweep
  // reads no x, unless the boundary band sweeps first.
  // Sweep pairs as fused launches (constant transfer): level 0 with
  // mg_fused >= 1 (and no band sweeps), the coarser grid levels with
  // mg_fused = 2. Pair m of a level's 2 nu pairs writes the level's x (z on
  // level 0) when 2 nu - 1 - m is even and the level's spare vector (r,
  // unused by the constant transfer) otherwise, and reads pair m - 1's
  // output, so the last pre-smoothing pair's output is what the restriction
  // reads and the last pair leaves the result in x.
  bool fused(int l) const {
    if (!mg_ || cfg_.mg_transfer != 1 || levels_.size() < 2 || cfg_.mg_fused < 1) return false;
    return l == 0 ? !band_count_ : cfg_.mg_fused >= 2;
  }
  int nu_at(int l) const { return l == 0 ? std::max(1, cfg_.mg_smooth) : nu_coarse(); }
  V *pair_out(int l, V *z, int m) const {
    V *x = l == 0 ? z : (V *)levels_[l].x;
    return ((2 * nu_at(l) - 1 - m) & 1) ? (V *)levels_[l].r : x;
  }
  void pair(int l, const V *in, V *out, const V *b, int c1, int mode, const Fold<V> &f,
            const CGState *st) {
    Launch L = ctx_->launch();
    if (l == 0)
      launch_mg_rb_pair<V, T>(L, view0(), in, out, b, c1, mode, f, st, NF_K_MG_SMOOTH0);
    else
      launch_mg_rb_pair<V, TA>(L, viewc(l), in, out, b, c1, mode, f, st, NF_K_MG_SMOOTH);
  }

  void down_levels(int lo, int hi, const V *r, V *z, const CGState *st) {
    Launch L = ctx_->launch();
    for (int l = lo; l < hi; ++l) {
      V *x = l == 0 ? z : (V *)levels_[l].x;
      const V *b = l == 0 ? r : (const V *)levels_[l].b;
      const bool banded = l == 0 && band_count_;
      if (banded) {
        const int64_t nc = (int64_t)levels_[l].nx * levels_[l].ny * levels_[l].nz;
        cudaMemsetAsync(x, 0, nc * sizeof(V), L.s);
        band(x, b, 0, st);
      }
      const int nu = l == 0 ? std::max(1, cfg_.mg_smooth) : nu_coarse();
      if (fused(l)) {
        for (int s = 0; s < nu; ++s) {
          x = pair_out(l, z, s);
          pair(l, s == 0 ? nullptr : pair_out(l, z, s - 1), x, b, 0,
               s == 0 ? kSweepZero : kSweepPlain, Fold<V>{nullptr, 0, 0, V(0)}, st);
        }
      } else {
        for (int s = 0; s < nu; ++s) {
          smooth(l, x, b, 0, st, s == 0 && !banded ? kSweepZero : kSweepPlain);
          smooth(l, x, b, 1, st);
        }
      }
      const Level &C = levels_[l + 1];
      if (cfg_.mg_transfer == 1) {
        // constant transfer: residual and restriction in one pass
        const float w = coarse_w();
        if (l == 0)
          launch_mg_resrestrict<V, T>(L, view0(), x, b, C.nx, C.ny, C.nz, (V *)C.b, w, st);
        else
          launch_mg_resrestrict<V, TA>(L, viewc(l), x, b, C.nx, C.ny, C.nz, (V *)C.b, w, st);
      } else {
        if (l == 0)
          launch_mg_residual<V, T>(L, view0(), x, b, (V *)levels_[0].r, pnorm(0), st);
        else
          launch_mg_residual<V, TA>(L, viewc(l), x, b, (V *)levels_[l].r, pnorm(l), st);
        const LevelView<TA> f{levels_[l].nx, levels_[l].ny, levels_[l].nz, 0.0,
                              nullptr, nullptr, nullptr};
        launch_mg_restrict<V, TA>(L, f, viewc(l + 1), (const V *)levels_[l].r, (V *)C.b,
                                  cfg_.mg_transfer, st);
      }
    }
  }

  // Prolongation and post-smoothing of levels hi-1 .. lo. With the constant
  // transfer the prolongation is folded into the first half sweep.
  void up_levels(int lo, int hi, const V *r, V *z, const CGState *st) {
    Launch L = ctx_->launch();
    for (int l = hi - 1; l >= lo; --l) {
      V *x = l == 0 ? z : (V *)levels_[l].x;
      const V *b = l == 0 ? r : (const V *)levels_[l].b;
      const Level &C = levels_[l + 1];
      const int nu = l == 0 ? std::max(1, cfg_.mg_smooth) : nu_coarse();
      int s = 0;
      if (fused(l)) {
        const Fold<V> f{(const V *)C.x, C.nx, C.ny, V(coarse_w())};
        for (int m = nu; m < 2 * nu; ++m)
          pair(l, pair_out(l, z, m - 1), pair_out(l, z, m), b, 1,
               m == nu ? kSweepProlong : kSweepPlain, m == nu ? f : Fold<V>{nullptr, 0, 0, V(0)},
               st);
        continue;
      }
      if (cfg_.mg_transfer == 1) {
        const Fold<V> f{(const V *)C.x, C.nx, C.ny, V(coarse_w())};
        smooth(l, x, b, 1, st, kSweepProlong, f);
        smooth(l, x, b, 0, st);
        s = 1;
      } else if (l == 0) {
        launch_mg_prolong<V, T, TA>(L, view0(), viewc(l + 1), (const V *)C.x, x, pnorm(0),
                                    cfg_.mg_transfer, st);
      } else {
        launch_mg_prolong<V, TA, TA>(L, viewc(l), viewc(l + 1), (const V *)C.x, x, pnorm(l),
                                     cfg_.mg_transfer, st);
      }
      for (; s < nu; ++s) {
        smooth(l, x, b, 1, st);
        smooth(l, x, b, 0, st);
      }
      if (l == 0) band(x, b, 1, st);
    }
  }

  // ------------------------------------------------------------ graphs --
  // The per-solve setup (e = 0, z = M r, d = z, dots) and a batch of kBatch
  // CG iterations are captured once per solver and replayed: every kernel
  // argument is fixed (pointers, level sizes, unit-scale coefficients; the
  // inner tolerance lives in CGState), so one capture serves every solve.
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;  // kernel launches per replay
    int gen = -1;     // profiling generation the capture was made under
    GraphEvents ev;   // event pairs of profiled kernels (when profiling)
  };

  void init_body() {
    Launch L = ctx_->launch();
    CGState *st = (CGState *)st_;
    V *r = (V *)rin_, *z = (V *)z_, *d = (V *)d_, *e = (V *)e_;
    ctx_->prof.capture_iter = 0;
    cudaMemsetAsync(e, 0, n_ * sizeof(V), L.s);
    if (mg_) {
      precondition(r, z, nullptr);
      launch_cg_init<V>(L, n_, r, z, d, st, ctx_->rs);
    } else {
      launch_cg_init<V>(L, n_, r, r, d, st, ctx_->rs);
    }
  }

  // Continuation of a converged pass after the true residual replaced the
  // recurrence one: e = 0, z = M r, beta from the rescaled old <r, z>,
  // d = z + beta d.
  void cont_body() {
    Launch L = ctx_->launch();
    CGState *st = (CGState *)st_;
    V *r = (V *)rin_, *z = (V *)z_, *d = (V *)d_, *e = (V *)e_;
    ctx_->prof.capture_iter = 0;
    cudaMemsetAsync(e, 0, n_ * sizeof(V), L.s);
    if (mg_) {
      precondition(r, z, nullptr);
      launch_cg_continue<V>(L, n_, r, z, st, ctx_->rs);
      launch_cg_d<V>(L, n_, z, d, st);
    } else {
      launch_cg_continue<V>(L, n_, r, r, st, ctx_->rs);
      launch_cg_d<V>(L, n_, r, d, st);
    }
  }

  void iterations(int count) {
    for (int b = 0; b < count; ++b) {
      ctx_->prof.capture_iter = b;
      iteration_head(nullptr);
      iteration_tail(nullptr);
    }
  }
  // One CG iteration in two parts: q = A d, alpha, x and r updates (with
  // `loop`: setting the device loop's conditions) ...
  void iteration_head(const LoopHandles *loop) {
    Launch L = ctx_->launch();
    CGState *st = (CGState *)st_;
    V *r = (V *)rin_, *d = (V *)d_, *q = (V *)q_, *e = (V *)e_;
    launch_apply_dot<V, T>(L, view0(), d, q, st, ctx_->rs);
    launch_cg_xr<V>(L, n_, e, r, d, q, st, ctx_->rs, mg_, loop);
  }
  // ... and z = M r, beta, d = z + beta d (with `loop`: deciding whether the
  // device loop runs another iteration).
  void iteration_tail(const LoopHandles *loop) {
    Launch L = ctx_->launch();
    CGState *st = (CGState *)st_;
    V *r = (V *)rin_, *z = (V *)z_, *d = (V *)d_;
    const cudaGraphConditionalHandle *body = loop ? &loop->body : nullptr;
    if (mg_) {
      precondition(r, z, st);
      launch_cg_rz<V>(L, n_, r, z, st, ctx_->rs);
      launch_cg_d<V>(L, n_, z, d, st, body);
    } else {
      launch_cg_d<V>(L, n_, r, d, st, body);
    }
  }

  // The device-side iteration loop: a graph whose WHILE node runs one CG
  // iteration per body, continued by its last kernel until the solve is
  // done or its budget is spent, so a pass needs one launch and one
  // read-back. Inside the body an IF node holds everything after the x, r
  // update: the iteration that meets the tolerance skips its V-cycle (the
  // update kernel clears both conditions). Not used while profiling (event
  // nodes may not live in a conditional body) or if the capture fails.
  struct Loop {
    cudaGraphExec_t exec = nullptr;
    int head = 0, tail = 0;  // kernel launches of the two parts of a body
  };
  bool ensure_loop(Loop &G) {
    if (!graphs_ok_ || !loops_ok_ || ctx_->prof.kclass != -2) return false;
    if (G.exec) return true;
    if (!cap_ && cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      loops_ok_ = false;
      return false;
    }
    // graph: WHILE { head; IF { tail } }
    cudaGraph_t g = nullptr;
    LoopHandles h{};
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h.body, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h.body;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp);
    cudaGraph_t body = e == cudaSuccess ? wp.conditional.phGraph_out[0] : nullptr;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h.tail, body, 1, cudaGraphCondAssignDefault);
    const int64_t before = ctx_->launches;
    int64_t mid = before;
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(cap_, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      ctx_->capture = cap_;
      iteration_head(&h);
      mid = ctx_->launches;
      ctx_->capture = nullptr;
      cudaGraph_t out = nullptr;
      e = cudaStreamEndCapture(cap_, &out);
    }
    // the head is a chain: its one node without dependents precedes the IF
    cudaGraphNode_t leaf = nullptr;
    if (e == cudaSuccess) {
      size_t n = 0;
      e = cudaGraphGetNodes(body, nullptr, &n);
      std::vector<cudaGraphNode_t> nodes(n);
      if (e == cudaSuccess && n > 0) e = cudaGraphGetNodes(body, nodes.data(), &n);
      int leaves = 0;
      for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
        size_t nd = 0;
        e = cudaGraphNodeGetDependentNodes(nodes[i], nullptr, nullptr, &nd);
        if (e == cudaSuccess && nd == 0) {
          leaf = nodes[i];
          ++leaves;
        }
      }
      if (e == cudaSuccess && leaves != 1) e = cudaErrorInvalidValue;
    }
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h.tail;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&inode, body, &leaf, nullptr, 1, &ip);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(cap_, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      ctx_->capture = cap_;
      iteration_tail(&h);
      ctx_->capture = nullptr;
      cudaGraph_t out = nullptr;
      e = cudaStreamEndCapture(cap_, &out);
    }
    G.head = (int)(mid - before);
    G.tail = (int)(ctx_->launches - mid);
    ctx_->launches = before;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      G.exec = nullptr;
      loops_ok_ = false;
      return false;
    }
    return true;
  }

  template <class F>
  bool ensure_graph(Graph &G, F body) {
    if (!graphs_ok_) return false;
    if (G.exec && G.gen == ctx_->prof.gen) return true;
    if (G.exec) {
      cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
    }
    G.ev.clear();
    if (!cap_ && cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      graphs_ok_ = false;
      return false;
    }
    const int64_t before = ctx_->launches;
    ctx_->capture = cap_;
    if (ctx_->prof.kclass != -2) ctx_->prof.capture_ev = &G.ev;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      body();
      e = cudaStreamEndCapture(cap_, &graph);
    }
    ctx_->capture = nullptr;
    ctx_->prof.capture_ev = nullptr;
    G.kernels = (int)(ctx_->launches - before);
    ctx_->launches = before;  // counted at every replay instead
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      G.exec = nullptr;
      graphs_ok_ = false;
      return false;
    }
    G.gen = ctx_->prof.gen;
    return true;
  }

  void replay(Graph &G) {
    cudaGraphLaunch(G.exec, ctx_->stream);
    ctx_->launches += G.kernels;
  }

  void inner_solve(double rel_tol, int max_it, int *iters, int *done,
                   double *rr, bool cont, double ratio) {
    CGState *st = (CGState *)st_;
    // tolerance and scale ratio go to device memory through a pinned slot
    // that no earlier copy still reads (every pass synchronised the stream)
    double *slot = (double *)((char *)ctx_->pinned + 2048);
    slot[0] = rel_tol;
    slot[1] = ratio;
    int *islot = (int *)(slot + 2);
    islot[0] = max_it;
    islot[1] = 0;
    static_assert(offsetof(CGState, ratio) == offsetof(CGState, tol) + sizeof(double) &&
                      offsetof(CGState, max_it) == offsetof(CGState, tol) + 2 * sizeof(double) &&
                      offsetof(CGState, loops) == offsetof(CGState, max_it) + sizeof(int),
                  "tol, ratio, max_it and loops are copied together");
    cudaMemcpyAsync(&st->tol, slot, 2 * sizeof(double) + 2 * sizeof(int), cudaMemcpyHostToDevice,
                    ctx_->stream);
    const int pv = proj_now_ ? 1 : 0;
    Graph &G0 = cont ? cont_g_[pv] : init_g_[pv];
    const bool g_init = cont ? ensure_graph(cont_g_[pv], [&] { cont_body(); })
                             : ensure_graph(init_g_[pv], [&] { init_body(); });
    if (g_init)
      replay(G0);
    else if (cont)
      cont_body();
    else
      init_body();
    CGState hs{};
    bool looped = false;
    if (g_init && ensure_loop(loop_g_[pv])) {
      looped = cudaGraphLaunch(loop_g_[pv].exec, ctx_->stream) == cudaSuccess;
      if (!looped) {  // not launchable here: the batches below continue the pass
        cudaGetLastError();
        loops_ok_ = false;
      }
    }
    if (looped) {
      ctx_->read_bytes(&hs, st, sizeof(CGState));
      // bodies that ran the tail are counted on the device; a converged
      // solve ran one more body without it
      const int64_t bodies = hs.loops + (hs.done == 1 ? 1 : 0);
      ctx_->launches += bodies * loop_g_[pv].head + (int64_t)hs.loops * loop_g_[pv].tail;
      *iters = hs.iters;
      *done = hs.err ? 5 : hs.done;
      *rr = hs.rr;
      return;
    }
    int issued = 0, seen = 0;
    bool init_collected = !g_init;
    while (issued < max_it) {
      const bool full = max_it - issued >= kBatch;
      const bool g_batch = full && ensure_graph(batch_g_[pv], [&] { iterations(kBatch); });
      if (g_batch)
        replay(batch_g_[pv]);
      else
        iterations(full ? kBatch : max_it - issued);
      issued += full ? kBatch : max_it - issued;
      ctx_->read_bytes(&hs, st, sizeof(CGState));
      if (!init_collected) {
        ctx_->prof.collect(G0.ev, 1);
        init_collected = true;
      }
      if (g_batch) {
        // iterations of this replay that ran to the end (the one that met
        // the tolerance skipped its preconditioner)
        const int ran = hs.iters - seen - (hs.done ? 1 : 0);
        ctx_->prof.collect(batch_g_[pv].ev, ran > 0 ? ran : 0);
      }
      seen = hs.iters;
      if (hs.done || hs.err) break;
    }
    *iters = hs.iters;
    *done = hs.err ? 5 : hs.done;
    *rr = hs.rr;
  }

  Ctx *ctx_;
  GridDev g_;
  nf_config cfg_;
  int64_t n_ = 0;
  bool mg_ = false;
  int first_chain_ = 0;
  int chain_smem_ = 0;  // dynamic shared memory of the chain kernel (0: global)
  int cl_lo_ = 0, cl_hi_ = 0;  // levels on the thread-block cluster (0: none)
  int cl_smem_ = 0;
  unsigned cl_off_[kMaxLevels][6] = {};
  unsigned cl_chain_off_ = 0;
  int mid_lo_ = 0;      // first level inside the cooperative kernel (0: none)
  int mid_blocks_ = 0;  // its grid
  void *bar_ = nullptr; // its barrier counter
  void *band_mark_ = nullptr, *band_list_[2] = {nullptr, nullptr}, *band_count_ = nullptr;
  std::vector<Level> levels_;
  const T *ax0_ = nullptr, *ay0_ = nullptr, *az0_ = nullptr;
  int es_ = 0;  // 2^es_ brings the current right-hand side to unit size
  void *rin_ = nullptr, *e_ = nullptr, *z_ = nullptr,
       *d_ = nullptr, *q_ = nullptr, *st_ = nullptr, *norm2_ = nullptr;
  cudaStream_t cap_ = nullptr;
  bool graphs_ok_ = true;
  bool loops_ok_ = true;
  int stall_ = 0;  // test hook (NF_TEST_STALL_WAITS)
  Graph init_g_[2], cont_g_[2], batch_g_[2];  // [1]: with the projection
  Loop loop_g_[2];
  Components *proj_ = nullptr;  // the episode's components (null: none)
  bool proj_now_ = false;       // this solve's system has a floating part

 public:
  ~Solver() {
    for (int p = 0; p < 2; ++p) {
      if (loop_g_[p].exec) cudaGraphExecDestroy(loop_g_[p].exec);
      if (init_g_[p].exec) cudaGraphExecDestroy(init_g_[p].exec);
      if (cont_g_[p].exec) cudaGraphExecDestroy(cont_g_[p].exec);
      if (batch_g_[p].exec) cudaGraphExecDestroy(batch_g_[p].exec);
    }
    if (cap_) cudaStreamDestroy(cap_);
  }
};

}  // namespace nf
