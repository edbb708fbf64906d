// Episode implementation: the forward step (Sec. 2.3.1), the checkpointed
// rollout tape, and the adjoint step (Sec. 2.3.2 / 2.3.3).
//
// Rollout tape: the velocity U^{mC} is saved before every C-th step. To
// revert step m the library restores U^{sC} (s = m / C), recomputes the
// segment's steps storing (U^k, U^k hat, P^k, alpha^k) for each, then runs the
// adjoint of the segment's steps in reverse. The forward kernels are
// deterministic (no float atomics, fixed-order reductions), so the recomputed
// segment reproduces the recorded rollout bit for bit.
//
// Sub-stepping: with cfl_max > 0 every frame of length dt is split into m
// equal steps, m = ceil(max|U| dt / (dx cfl_max)) from the velocity at the
// frame start (the CFL rule the paper applies between frames, Table 1). The
// time t_{k+1} and length h_k of every step are kept in the tape, so the
// recomputation and the adjoint replay the same schedule.
//
// Gauge: on a fluid component that touches no open face A is singular with
// the constants on the component as null space. There the right-hand side is
// projected to zero mean (a no-op for consistent data, the least-squares
// reading otherwise) and the pressure is returned with zero mean; the
// adjoint does the same for dJ/dP and the adjoint variable y, so the
// parameter gradient is the derivative of that reading. Components are
// labelled on the device after every rasterisation that precedes a solve.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "components.h"
#include "episode.h"
#include "kernels.h"
#include "solver.cuh"

namespace nf {

// ------------------------------------------------------------- scenes -----

static int scene_K(const nf_scene &sc) {
  switch (sc.kind) {
    case NF_SCENE_SPHERE:
      return 3;
    case NF_SCENE_CHAMBER:
      return 8;
    case NF_SCENE_PLATE:
      return 4;
    case NF_SCENE_EXTRUDED:
      return sc.K;
    default:
      return 0;
  }
}

// ------------------------------------------------ extruded shapes (host) ---
// Caller's table (nf.h): per shape 17 header values, then n keys of 2 + 2N.
std::string bz_check(const nf_scene &s) {
  const int ns = (int)s.consts[0], mode = (int)s.consts[2];
  if (ns < 1 || ns > kBzMaxShapes) return "1 to 4 shapes";
  if (!s.shapes || s.nshape_values <= 0) return "shape table missing";
  if (mode < kBzRadii || mode > kBzFixed) return "unknown theta mode";
  int o = 0, radii = 0;
  for (int sh = 0; sh < ns; ++sh) {
    if (o + 17 > s.nshape_values) return "shape table too short";
    const double *h = s.shapes + o;
    const int n = (int)h[0], N = (int)h[1];
    if (n < 1 || n > kBzMaxKeys || N < 1 || N > kBzMaxSeg || h[0] != n || h[1] != N)
      return "1 to 4 keys and 1 to 8 segments per shape";
    if (!(h[3] > h[2])) return "z1 must exceed z0";
    for (int v = 2; v < 17; ++v)
      if (!std::isfinite(h[v])) return "non-finite shape header";
    o += 17 + n * (2 + 2 * N);
    radii += n * 2 * N;
    if (o > s.nshape_values) return "shape table too short";
  }
  if (o != s.nshape_values) return "shape table size does not match its shapes";
  for (int v = 0; v < o; ++v)
    if (!std::isfinite(s.shapes[v])) return "non-finite shape table entry";
  const int want = mode == kBzRadii ? radii : (mode == kBzPulse ? 4 : 0);
  if (mode == kBzRadii && radii > NF_MAX_PARAMS) return "more radii than NF_MAX_PARAMS";
  if (s.K != want) return "K does not match the theta mode";
  if (mode == kBzPulse &&
      ((int)s.consts[3] < 0 || (int)s.consts[3] >= ns || !(s.consts[4] > 0.0)))
    return "pulse shape index or period invalid";
  return std::string();
}

// Device table of scene.cuh: header with the inverse Vandermonde
// coefficients of the key interpolation and the segments' unit vectors,
// keys with the radii (theta's in radii mode).
void bz_build(const nf_scene &s, const std::vector<double> &src, BzInfo &out) {
  out.n = (int)s.consts[0];
  out.inside = s.consts[1] != 0.0 ? 1 : 0;
  out.mode = (int)s.consts[2];
  out.pulse = (int)s.consts[3];
  out.period = s.consts[4];
  out.table.clear();
  int o = 0, th = 0;
  out.radii = 0;
  for (int sh = 0; sh < out.n; ++sh) {
    const double *h = src.data() + o;
    const int n = (int)h[0], N = (int)h[1];
    out.off[sh] = (int)out.table.size();
    out.theta0[sh] = th;
    for (int v = 0; v < 17; ++v) out.table.push_back(h[v]);
    // coeff = V^-1, V[k][m] = u_k^m, u_k = k / (n - 1): W = powers(u) coeff
    double V[kBzMaxKeys][2 * kBzMaxKeys] = {};
    for (int k = 0; k < n; ++k) {
      const double uk = n > 1 ? (double)k / (double)(n - 1) : 0.0;
      double p = 1.0;
      for (int m = 0; m < n; ++m) {
        V[k][m] = p;
        p *= uk;
      }
      V[k][n + k] = 1.0;
    }
    for (int c = 0; c < n; ++c) {  // Gauss-Jordan with partial pivoting
      int piv = c;
      for (int r = c + 1; r < n; ++r)
        if (std::fabs(V[r][c]) > std::fabs(V[piv][c])) piv = r;
      for (int m = 0; m < 2 * n; ++m) std::swap(V[c][m], V[piv][m]);
      const double inv = 1.0 / V[c][c];
      for (int m = 0; m < 2 * n; ++m) V[c][m] *= inv;
      for (int r = 0; r < n; ++r) {
        if (r == c) continue;
        const double f = V[r][c];
        for (int m = 0; m < 2 * n; ++m) V[r][m] -= f * V[c][m];
      }
    }
    // the inverse: coeff[m][k] = (V^-1)[m][k], rows m of the right half
    for (int m = 0; m < kBzMaxKeys; ++m)
      for (int k = 0; k < kBzMaxKeys; ++k)
        out.table.push_back(m < n && k < n ? V[m][n + k] : 0.0);
    for (int i = 0; i < N; ++i) {
      const double base = 2.0 * M_PI * i / N;
      const double a0 = base + 2.0 * M_PI / (3.0 * N), a1 = base + 4.0 * M_PI / (3.0 * N);
      out.table.push_back(std::cos(a0));
      out.table.push_back(std::sin(a0));
      out.table.push_back(std::cos(a1));
      out.table.push_back(std::sin(a1));
    }
    const double *kb = h + 17;
    for (int k = 0; k < n; ++k) {
      out.table.push_back(kb[k * (2 + 2 * N)]);
      out.table.push_back(kb[k * (2 + 2 * N) + 1]);
      for (int j = 0; j < 2 * N; ++j)
        out.table.push_back(out.mode == kBzRadii ? s.theta[th + j]
                                                 : kb[k * (2 + 2 * N) + 2 + j]);
      th += 2 * N;
    }
    out.radii += n * 2 * N;
    o += 17 + n * (2 + 2 * N);
  }
}

// Scene state at time t (host, double precision).
static SceneDev scene_at(const nf_scene &sc, double t, const double *d_spheres,
                         const BzInfo *bz = nullptr) {
  SceneDev s;
  std::memset(&s, 0, sizeof(s));
  s.kind = sc.kind;
  s.K = scene_K(sc);
  s.t = t;
  const double *c = sc.consts;
  const double *th = sc.theta;
  switch (sc.kind) {
    case NF_SCENE_SPHERE:
      for (int a = 0; a < 3; ++a) {
        s.sv[a] = th[a];
        s.sc[a] = c[a] + th[a] * t;
      }
      s.sr = c[3];
      s.fdscale[0] = (float)(-t);
      break;
    case NF_SCENE_CHAMBER: {
      for (int a = 0; a < 3; ++a) {
        s.cc[a] = c[a];
        s.ca[a] = c[3 + a];
      }
      s.camin = std::min(s.ca[0], std::min(s.ca[1], s.ca[2]));
      for (int a = 0; a < 3; ++a) s.cinva[a] = 1.0 / s.ca[a];
      const double T = c[6];
      double r = 1.0, rd = 0.0;
      for (int k = 1; k <= 4; ++k) {
        const double w = 2.0 * M_PI * k / T;
        const double cs = std::cos(w * t), sn = std::sin(w * t);
        const double a = th[k - 1], b = th[3 + k];
        r += a * cs + b * sn;
        rd += w * (-a * sn + b * cs);
        s.cds[k - 1] = cs;
        s.cds[3 + k] = sn;
        s.cdsdot[k - 1] = -w * sn;
        s.cdsdot[3 + k] = w * cs;
      }
      s.cs = r;
      s.csdot = rd;
      s.crate = rd / r;
      for (int k = 0; k < 8; ++k) s.cdus[k] = (s.cdsdot[k] * r - rd * s.cds[k]) / (r * r);
      for (int k = 0; k < 8; ++k) s.fdscale[k] = (float)(s.camin * s.cds[k]);
      for (int a = 0; a < 3; ++a) s.finva[a] = (float)s.cinva[a];
      const double x0 = c[7], hw = c[8];
      s.dc[0] = 0.5 * (x0 + 2.0);
      s.dc[1] = c[1];
      s.dc[2] = c[2];
      s.dh[0] = 0.5 * (2.0 - x0);
      s.dh[1] = hw;
      s.dh[2] = hw;
      break;
    }
    case NF_SCENE_PLATE: {
      for (int a = 0; a < 3; ++a) {
        s.pc[a] = c[a];
        s.ph[a] = c[3 + a];
      }
      const double L = c[6] / 3.0;
      int seg = (int)std::floor(t / L);
      seg = std::max(0, std::min(2, seg));
      const double tau = (t - seg * L) / L;
      s.pang = th[seg] * (1.0 - tau) + th[seg + 1] * tau;
      s.pomega = (th[seg + 1] - th[seg]) / L;
      s.pcos = std::cos(s.pang);
      s.psin = std::sin(s.pang);
      for (int k = 0; k < 4; ++k) s.pdang[k] = s.pdomega[k] = 0.0;
      s.pdang[seg] = 1.0 - tau;
      s.pdang[seg + 1] = tau;
      for (int k = 0; k < 4; ++k) s.fdscale[k] = (float)s.pdang[k];
      s.pdomega[seg] = -1.0 / L;
      s.pdomega[seg + 1] = 1.0 / L;
      break;
    }
    case NF_SCENE_SPHERES:
      s.spheres = d_spheres;
      s.nspheres = sc.nspheres;
      break;
    case NF_SCENE_EXTRUDED: {
      s.bz = bz->dev;
      s.bz_n = bz->n;
      s.bz_inside = bz->inside;
      s.bz_mode = bz->mode;
      s.bz_pulse = bz->pulse;
      for (int a = 0; a < kBzMaxShapes; ++a) {
        s.bz_off[a] = bz->off[a];
        s.bz_theta0[a] = bz->theta0[a];
      }
      s.bz_k = 1.0;
      if (bz->mode == kBzPulse) {
        // k(t) piecewise linear through the 4 knots at 0, T/3, 2T/3, T
        const double L = bz->period / 3.0;
        int seg = (int)std::floor(t / L);
        seg = std::max(0, std::min(2, seg));
        const double tau = (t - seg * L) / L;
        s.bz_k = th[seg] * (1.0 - tau) + th[seg + 1] * tau;
        s.bz_kdot = (th[seg + 1] - th[seg]) / L;
        for (int k = 0; k < 4; ++k) s.bz_dk[k] = s.bz_dkdot[k] = 0.0;
        s.bz_dk[seg] = 1.0 - tau;
        s.bz_dk[seg + 1] = tau;
        s.bz_dkdot[seg] = -1.0 / L;
        s.bz_dkdot[seg + 1] = 1.0 / L;
      }
      break;
    }
    default:
      break;
  }
  for (int a = 0; a < 3; ++a) {
    s.f_sc[a] = (float)s.sc[a];
    s.f_sv[a] = (float)s.sv[a];
    s.f_cc[a] = (float)s.cc[a];
    s.f_dc[a] = (float)s.dc[a];
    s.f_dh[a] = (float)s.dh[a];
    s.f_pc[a] = (float)s.pc[a];
    s.f_ph[a] = (float)s.ph[a];
    s.finva[a] = (float)s.cinva[a];
  }
  s.f_sr = (float)s.sr;
  s.f_camin = (float)s.camin;
  s.f_cs = (float)s.cs;
  s.f_crate = (float)s.crate;
  s.f_pcos = (float)s.pcos;
  s.f_psin = (float)s.psin;
  s.f_pomega = (float)s.pomega;
  for (int k = 0; k < 8; ++k) s.f_cdus[k] = (float)s.cdus[k];
  for (int k = 0; k < 4; ++k) s.f_pdomega[k] = (float)s.pdomega[k];
  return s;
}

// -------------------------------------------------------- conversions -----
template <class A, class B>
__global__ void k_cast(int64_t n, const A *in, B *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (B)in[i];
}

// out = f in (f a power of two: exact).
template <class A>
__global__ void k_scaled_copy(int64_t n, const A *in, A *out, double f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (A)((double)in[i] * f);
}
template <class A>
static void scaled_copy(const Launch &L, int64_t n, const A *in, A *out, double f) {
  unsigned nb = nblocks(n);
  if (nb > 148u * 32u) nb = 148u * 32u;
  k_scaled_copy<A><<<nb, kBlock, 0, L.s>>>(n, in, out, f);
  ++*L.counter;
}

template <class A, class B>
static void cast(const Launch &L, int64_t n, const A *in, B *out) {
  unsigned nb = nblocks(n);
  if (nb > 148u * 32u) nb = 148u * 32u;
  ProfScope _ps(L, NF_K_CAST);
  k_cast<A, B><<<nb, kBlock, 0, L.s>>>(n, in, out);
  ++*L.counter;
}

static size_t dtype_size(int dtype) { return dtype == NF_F64 ? 8 : 4; }

// --------------------------------------------------------------- impl -----
template <class T, class S, class V, class TA>
class EpisodeImpl : public EpisodeBase {
 public:
  EpisodeImpl(Ctx *ctx, const nf_grid &gr, const nf_scene &sc)
      : ctx_(ctx), g_(make_grid(gr)), sc_(sc), solver_(ctx, make_grid(gr), ctx->cfg) {
    A_.stream = ctx->stream;
    sc_.K = scene_K(sc);
    sc_.spheres = nullptr;
    sc_.shapes = nullptr;  // kept in bz_src_ by init
  }

  static GridDev make_grid(const nf_grid &gr) {
    GridDev g;
    g.nx = gr.nx;
    g.ny = gr.ny;
    g.nz = gr.nz;
    g.dx = gr.dx;
    g.dt = gr.dt;
    g.rho = gr.rho > 0 ? gr.rho : 1.0;
    g.c = g.dt / (g.rho * g.dx);
    g.nu = gr.nu;
    g.frac = gr.fractions;
    g.outlet = gr.outlet;
    g.oj0 = gr.outlet_j0;
    g.ok0 = gr.outlet_k0;
    g.ow = gr.outlet_w;
    g.oh = gr.outlet_h;
    g.inlet = gr.inlet;
    g.iside = gr.inlet_side;
    g.ij0 = gr.inlet_j0;
    g.ik0 = gr.inlet_k0;
    g.iw = gr.inlet_w;
    g.ih = gr.inlet_h;
    g.ispeed = gr.inlet_speed;
    g.set_derived();
    return g;
  }

  int init(const nf_scene &sc) {
    nfaces_ = g_.nface(0) + g_.nface(1) + g_.nface(2);
    ncell_ = g_.ncell();
    CKS(faces(&U_));
    CKS(faces(&Uh_));
    CKS(faces(&alpha_));
    CKS(faces(&gU_));
    CKS(faces(&gUb_));
    CKS(faces(&gUh_));
    if (g_.nu > 0.0) CKS(faces(&Ut_));  // U~ before viscosity, dJ/dU~ after
    CKS(A_.get(&P_, ncell_ * sizeof(S)));
    CKS(A_.get(&b_, ncell_ * sizeof(S)));
    CKS(A_.get(&gP_, ncell_ * sizeof(S)));
    CKS(A_.get(&y_, ncell_ * sizeof(S)));
    const int64_t mf = std::max(g_.nface(0), std::max(g_.nface(1), g_.nface(2)));
    CKS(A_.get(&stage_, std::max(mf, ncell_) * sizeof(double)));
    CKS(A_.get(&dscal_, 64 * sizeof(double)));
    if (sc.kind == NF_SCENE_SPHERES && sc.nspheres > 0) {
      CKS(A_.get(&dsph_, (size_t)sc.nspheres * 4 * sizeof(double)));
      CKC(cudaMemcpyAsync(dsph_, sc.spheres, (size_t)sc.nspheres * 4 * sizeof(double),
                          cudaMemcpyHostToDevice, ctx_->stream));
      CKC(cudaStreamSynchronize(ctx_->stream));  // the host list is the caller's
    }
    if (sc.kind == NF_SCENE_EXTRUDED) {
      bz_src_.assign(sc.shapes, sc.shapes + sc.nshape_values);
      CKS(upload_bz());
    }
    CKS(solver_.init(A_));
    CKS(cc_.init(A_, ncell_));
    solver_.set_projector(&cc_);
    Launch L = ctx_->launch();
    CKC(cudaMemsetAsync(U_, 0, nfaces_ * sizeof(T), L.s));
    CKC(cudaMemsetAsync(P_, 0, ncell_ * sizeof(S), L.s));
    CKC(cudaMemsetAsync(Uh_, 0, nfaces_ * sizeof(T), L.s));
    // fractions of the initial geometry (t = 0) so queries are meaningful
    launch_rasterize<T>(L, g_, scene_at(sc_, 0.0, dsph_, &bz_), mut(alpha_));
    return check_launch();
  }

  size_t bytes() const override { return A_.bytes; }
  int step_index() const override { return n_; }

  int set_params(const double *theta, int K) override {
    if (K != sc_.K) return invalid("set_params: expected %d parameters", sc_.K);
    for (int k = 0; k < K; ++k) sc_.theta[k] = theta[k];
    clear_tape();
    if (sc_.kind == NF_SCENE_EXTRUDED) CKS(upload_bz());  // radii mode: new radii
    return NF_OK;
  }

  // The extruded scene's device table from the kept caller table and theta.
  int upload_bz() {
    bz_build(sc_, bz_src_, bz_);
    const size_t bytes = bz_.table.size() * sizeof(double);
    if (!bz_dev_) CKS(A_.get(&bz_dev_, bytes));
    CKC(cudaMemcpyAsync(bz_dev_, bz_.table.data(), bytes, cudaMemcpyHostToDevice, ctx_->stream));
    CKC(cudaStreamSynchronize(ctx_->stream));  // bz_.table is rebuilt by the next call
    bz_.dev = bz_dev_;
    return NF_OK;
  }

  int set_velocity(const void *const u[3], int dtype, int mem, int project,
                   nf_step_stats *st) override {
    for (int d = 0; d < 3; ++d)
      CKS(copy_in(comp(U_, d), u[d], g_.nface(d), dtype, mem));
    clear_tape();
    nf_step_stats s{};
    int rc = NF_OK;
    if (project) {
      if (!Uinit_) {
        CKS(faces(&Uinit_));
        CKS(A_.get(&Pinit_, ncell_ * sizeof(S)));
      }
      Launch L = ctx_->launch();
      CKC(cudaMemcpyAsync(Uinit_, U_, nfaces_ * sizeof(T), cudaMemcpyDeviceToDevice, L.s));
      const SceneDev sd = scene_at(sc_, 0.0, dsph_, &bz_);
      launch_rasterize<T>(L, g_, sd, mut(alpha_));
      SolveStats ss;
      Eng e = eng();
      CKS(project_faces(e, g_, sd, Uinit_, Pinit_, U_, &ss));
      CKC(cudaMemcpyAsync(Uh_, Uinit_, nfaces_ * sizeof(T), cudaMemcpyDeviceToDevice, L.s));
      CKC(cudaMemcpyAsync(P_, Pinit_, ncell_ * sizeof(S), cudaMemcpyDeviceToDevice, L.s));
      acc_stats(&s, ss);
      init_proj_ = true;
      rc = ss.status;
    }
    if (st) *st = s;
    CKS(check_launch());
    return rc;
  }

  int step(int nsteps, nf_step_stats *st) override {
    if (nsteps < 0) return invalid("step: nsteps < 0%s", "");
    nf_step_stats s{};
    int worst = NF_OK;
    const double cfl = ctx_->cfg.cfl_max;
    for (int i = 0; i < nsteps && worst != NF_E_DIVERGED; ++i) {
      int m = 1;
      if (cfl > 0.0) {
        const double umax = max_speed();
        if (!std::isfinite(umax)) return diverged("step: non-finite velocity");
        m = std::max(1, (int)std::ceil(umax * g_.dt / (g_.dx * cfl)));
      }
      for (int sub = 0; sub < m; ++sub) {
        CKS(begin_substep(sub, m));
        SolveStats ss;
        Eng e = eng();
        CKS(forward_step(e, n_, U_, U_, Uh_, P_, &ss));
        acc_stats(&s, ss);
        s.steps += 1;
        if (ss.status != NF_OK && worst == NF_OK) worst = ss.status;
        if (ss.status == NF_E_DIVERGED) {
          worst = NF_E_DIVERGED;
          break;
        }
        end_substep();
      }
      ++frames_;
    }
    if (st) *st = s;
    CKS(check_launch());
    return worst;
  }

  int loss(int kind, double *J, void *const gU[3], int dtype, int mem) override {
    if (kind != NF_LOSS_KINETIC && kind != NF_LOSS_OUTFLOW)
      return invalid("loss: unknown kind %d", kind);
    if (kind == NF_LOSS_OUTFLOW && !g_.outlet)
      return invalid("loss: outflow needs an outlet%s", "");
    Launch L = ctx_->launch();
    const bool want = gU != nullptr;
    launch_loss<T>(L, g_, kind, cview(U_), mut(gUh_), want, ctx_->rs, dscal_ + 1);
    if (J) *J = ctx_->read_double(dscal_ + 1);
    if (want)
      for (int d = 0; d < 3; ++d)
        CKS(copy_out(gU[d], comp(gUh_, d), g_.nface(d), dtype, mem));
    return check_launch();
  }

  int backward_step(const void *const gU_next[3], void *const gU_prev[3],
                    int dtype, int mem, double *g_theta,
                    nf_step_stats *st) override {
    if (n_rev_ == 0 && !(init_proj_ && !init_reverted_))
      return state_err("backward_step: nothing left to revert");
    for (int d = 0; d < 3; ++d)
      CKS(copy_in(comp(gU_, d), gU_next[d], g_.nface(d), dtype, mem));
    nf_step_stats s{};
    double gth[kMaxParams] = {0};
    const int rc = revert_one(gth, &s);
    if (rc != NF_OK && rc != NF_E_NOT_CONVERGED) return rc;
    if (g_theta)
      for (int k = 0; k < sc_.K; ++k) g_theta[k] += gth[k];
    if (gU_prev)
      for (int d = 0; d < 3; ++d)
        if (gU_prev[d]) CKS(copy_out(gU_prev[d], comp(gU_, d), g_.nface(d), dtype, mem));
    if (st) *st = s;
    CKS(check_launch());
    return rc;
  }

  int backward(const void *const gU_final[3], void *const gU0[3], int dtype,
               int mem, double *g_theta, nf_step_stats *st) override {
    if (n_rev_ == 0 && !(init_proj_ && !init_reverted_))
      return state_err("backward: no recorded step to revert");
    for (int d = 0; d < 3; ++d)
      CKS(copy_in(comp(gU_, d), gU_final[d], g_.nface(d), dtype, mem));
    return backward_from_gU(gU0, dtype, mem, g_theta, st);
  }

  int loss_backward(int kind, double *J, double *g_theta, nf_step_stats *st) override {
    if (kind != NF_LOSS_KINETIC && kind != NF_LOSS_OUTFLOW)
      return invalid("loss_backward: unknown kind %d", kind);
    if (kind == NF_LOSS_OUTFLOW && !g_.outlet)
      return invalid("loss_backward: outflow needs an outlet%s", "");
    if (n_rev_ == 0 && !(init_proj_ && !init_reverted_))
      return state_err("loss_backward: no recorded step to revert");
    Launch L = ctx_->launch();
    launch_loss<T>(L, g_, kind, cview(U_), mut(gU_), true, ctx_->rs, dscal_ + 1);
    if (J) *J = ctx_->read_double(dscal_ + 1);
    return backward_from_gU(nullptr, NF_F32, NF_MEM_DEVICE, g_theta, st);
  }

  // BPTT from dJ/dU^final already in gU_.
  int backward_from_gU(void *const gU0[3], int dtype, int mem, double *g_theta,
                       nf_step_stats *st) {
    nf_step_stats s{};
    double gth[kMaxParams] = {0};
    int worst = NF_OK;
    overlap_now_ = overlap_ok();
    while (n_rev_ > 0 || (init_proj_ && !init_reverted_)) {
      const int rc = revert_one(gth, &s);
      if (rc != NF_OK && rc != NF_E_NOT_CONVERGED) {
        overlap_now_ = false;
        if (helper_seg_ >= 0) {  // a helper still running: wait, drop its segment
          helper_seg_ = -1;
          if (helper_->th.joinable()) helper_->th.join();
        }
        return rc;
      }
      if (rc != NF_OK && worst == NF_OK) worst = rc;
    }
    overlap_now_ = false;
    if (helper_seg_ >= 0) {
      helper_seg_ = -1;
      if (helper_->th.joinable()) helper_->th.join();
    }
    if (g_theta)
      for (int k = 0; k < sc_.K; ++k) g_theta[k] = gth[k];
    if (gU0)
      for (int d = 0; d < 3; ++d)
        if (gU0[d]) CKS(copy_out(gU0[d], comp(gU_, d), g_.nface(d), dtype, mem));
    if (st) *st = s;
    CKS(check_launch());
    return worst;
  }

  int get_faces(int which, void *const dst[3], int dtype, int mem) override {
    const T *src = which == 0 ? U_ : (which == 1 ? Uh_ : alpha_);
    for (int d = 0; d < 3; ++d)
      CKS(copy_out(dst[d], comp(src, d), g_.nface(d), dtype, mem));
    return check_launch();
  }

  int get_pressure(void *dst, int dtype, int mem) override {
    return copy_out_t<S>(dst, P_, ncell_, dtype, mem);
  }

  // Resume format: a header (magic, version, field size, grid, frame
  // clock, theta) and the face velocity in the episode's field type.
  struct StateHeader {
    char magic[8];
    int32_t version, field_bytes, nx, ny, nz, K, kind, pad;
    int64_t frames;
    double dx, dt, theta[NF_MAX_PARAMS];
  };
  static constexpr char kMagic[8] = {'N', 'F', 'E', 'P', 'I', 'S', 'O', '1'};

  int export_state(void *buf, size_t *bytes) override {
    const size_t need = sizeof(StateHeader) + nfaces_ * sizeof(T);
    if (!buf) {
      *bytes = need;
      return NF_OK;
    }
    if (*bytes < need) return invalid("episode_export: buffer of %zu bytes is too small", *bytes);
    StateHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.field_bytes = (int32_t)sizeof(T);
    h.nx = g_.nx;
    h.ny = g_.ny;
    h.nz = g_.nz;
    h.K = sc_.K;
    h.kind = sc_.kind;
    h.frames = frames_;
    h.dx = g_.dx;
    h.dt = g_.dt;
    for (int k = 0; k < NF_MAX_PARAMS; ++k) h.theta[k] = sc_.theta[k];
    std::memcpy(buf, &h, sizeof(h));
    CKC(cudaMemcpyAsync((char *)buf + sizeof(h), U_, nfaces_ * sizeof(T), cudaMemcpyDeviceToHost,
                        ctx_->stream));
    CKC(cudaStreamSynchronize(ctx_->stream));
    *bytes = need;
    return NF_OK;
  }

  int import_state(const void *buf, size_t bytes) override {
    StateHeader h{};
    if (!buf || bytes < sizeof(h)) return invalid("episode_import: buffer too short%s", "");
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 1)
      return invalid("episode_import: not an exported episode state%s", "");
    if (h.field_bytes != (int32_t)sizeof(T) || h.nx != g_.nx || h.ny != g_.ny || h.nz != g_.nz ||
        h.K != sc_.K || h.kind != sc_.kind || h.dx != g_.dx || h.dt != g_.dt || h.frames < 0)
      return invalid("episode_import: state of another grid, scene or precision%s", "");
    if (bytes != sizeof(h) + nfaces_ * sizeof(T))
      return invalid("episode_import: size does not match the grid%s", "");
    CKC(cudaMemcpyAsync(U_, (const char *)buf + sizeof(h), nfaces_ * sizeof(T),
                        cudaMemcpyHostToDevice, ctx_->stream));
    CKC(cudaStreamSynchronize(ctx_->stream));  // the caller's buffer is borrowed
    for (int k = 0; k < sc_.K; ++k) sc_.theta[k] = h.theta[k];
    clear_tape();
    if (sc_.kind == NF_SCENE_EXTRUDED) CKS(upload_bz());
    frames_ = (int)h.frames;  // the clock resumes; the tape starts here
    return NF_OK;
  }

 private:
  // ---------------------------------------------------------- helpers ----
  int faces(T **p) { return A_.get(p, nfaces_ * sizeof(T)); }
  T *comp(T *base, int d) const {
    return base + (d == 0 ? 0 : (d == 1 ? g_.nface(0) : g_.nface(0) + g_.nface(1)));
  }
  const T *comp(const T *base, int d) const {
    return base + (d == 0 ? 0 : (d == 1 ? g_.nface(0) : g_.nface(0) + g_.nface(1)));
  }
  FieldsMut<T> mut(T *base) const {
    return FieldsMut<T>{comp(base, 0), comp(base, 1), comp(base, 2)};
  }
  Fields<T> cview(const T *base) const {
    return Fields<T>{comp(base, 0), comp(base, 1), comp(base, 2)};
  }
  int invalid(const char *fmt, int v) {
    char buf[256];
    snprintf(buf, sizeof buf, fmt, v);
    set_error(buf);
    return NF_E_INVALID;
  }
  int invalid(const char *fmt, const char *v) {
    char buf[256];
    snprintf(buf, sizeof buf, fmt, v);
    set_error(buf);
    return NF_E_INVALID;
  }
  int state_err(const char *msg) {
    set_error(msg);
    return NF_E_STATE;
  }
  int diverged(const char *msg) {
    set_error(msg);
    return NF_E_DIVERGED;
  }
  // max |U| over all faces (synchronises the stream)
  double max_speed() {
    Launch L = ctx_->launch();
    unsigned long long *mx = (unsigned long long *)(dscal_ + 2);
    launch_absmax_faces<T>(L, g_, cview(U_), mx);
    unsigned long long bits = 0;
    ctx_->read_bytes(&bits, mx, sizeof(bits));
    double v;
    std::memcpy(&v, &bits, sizeof(v));
    return v;
  }
  // Grid description of a step of length h (advection and operator scale).
  GridDev grid_h(double h) const {
    GridDev g = g_;
    g.dt = h;
    g.c = h / (g_.rho * g_.dx);
    g.set_derived();
    return g;
  }
  int check_launch() {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return NF_OK;
  }
  void acc_stats(nf_step_stats *s, const SolveStats &ss) {
    s->solves += 1;
    s->iters += ss.iters;
    s->max_iters = std::max(s->max_iters, ss.iters);
    s->outer += ss.outer;
    s->rel_residual = std::max(s->rel_residual, ss.rel);
  }

  template <class D>
  int copy_in_t(D *dst, const void *src, int64_t n, int dtype, int mem) {
    if (!src) return invalid("null input array%s", "");
    Launch L = ctx_->launch();
    const size_t es = dtype_size(dtype);
    const bool same = es == sizeof(D);
    if (mem == NF_MEM_DEVICE && same) {
      CKC(cudaMemcpyAsync(dst, src, n * es, cudaMemcpyDeviceToDevice, L.s));
      return NF_OK;
    }
    const void *dsrc = src;
    if (mem == NF_MEM_HOST) {
      void *target = same ? (void *)dst : stage_;
      CKC(cudaMemcpyAsync(target, src, n * es, cudaMemcpyHostToDevice, L.s));
      if (same) return NF_OK;
      dsrc = stage_;
    }
    if (dtype == NF_F64)
      cast<double, D>(L, n, (const double *)dsrc, dst);
    else
      cast<float, D>(L, n, (const float *)dsrc, dst);
    return NF_OK;
  }
  int copy_in(T *dst, const void *src, int64_t n, int dtype, int mem) {
    return copy_in_t<T>(dst, src, n, dtype, mem);
  }

  template <class D>
  int copy_out_t(void *dst, const D *src, int64_t n, int dtype, int mem) {
    if (!dst) return invalid("null output array%s", "");
    Launch L = ctx_->launch();
    const size_t es = dtype_size(dtype);
    const bool same = es == sizeof(D);
    const void *from = src;
    if (!same) {
      void *target = mem == NF_MEM_DEVICE ? dst : stage_;
      if (dtype == NF_F64)
        cast<D, double>(L, n, src, (double *)target);
      else
        cast<D, float>(L, n, src, (float *)target);
      if (mem == NF_MEM_DEVICE) return NF_OK;
      from = stage_;
    }
    CKC(cudaMemcpyAsync(dst, from, n * es,
                        mem == NF_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                             : cudaMemcpyDeviceToHost,
                        L.s));
    if (mem == NF_MEM_HOST) CKC(cudaStreamSynchronize(L.s));
    return NF_OK;
  }
  int copy_out(void *dst, const T *src, int64_t n, int dtype, int mem) {
    return copy_out_t<T>(dst, src, n, dtype, mem);
  }

  void clear_tape() {
    std::fill(tapeA_ok_.begin(), tapeA_ok_.end(), 0);
    n_ = 0;
    frames_ = 0;
    ts_.clear();
    hs_.clear();
    n_rev_ = 0;
    init_proj_ = false;
    init_reverted_ = false;
    seg_start_ = -1;
  }

  // Zero mean on every floating component; returns ||v||^2 afterwards.
  double gauge(S *v, double n2) { return cc_.gauge<S>(ctx_, ncell_, v, n2); }

  // What one forward step works with: a context (stream, reduction
  // scratch), fraction and right-hand-side scratch, components, a solver.
  // The episode's own engine serves every call; a second one (its own
  // stream) lets the backward pass recompute the next segment while it
  // reverts the current one.
  struct Eng {
    Ctx *ctx;
    T *alpha;
    S *b;
    Components *cc;
    Solver<T, S, V, TA> *solver;
    T *Ut;
    double *dscal;
  };
  Eng eng() { return Eng{ctx_, alpha_, b_, &cc_, &solver_, Ut_, dscal_}; }

  // ----------------------------------------------------------- forward ----
  // Right-hand side, solve and blended update for fractions e.alpha (already
  // rasterised for scene state sd): uh -> P, u_out.
  int project_faces(Eng &e, const GridDev &g, const SceneDev &sd, const T *uh, S *P,
                    T *u_out, SolveStats *ss) {
    NvtxRange nv("nf.project");
    Launch L = e.ctx->launch();
    CKS(e.cc->template label<T>(e.ctx, g, cview(e.alpha)));
    launch_rhs<T, S>(L, g, sd, cview(e.alpha), cview(uh), e.b, e.ctx->rs, e.dscal);
    e.solver->set_fractions(comp(e.alpha, 0), comp(e.alpha, 1), comp(e.alpha, 2));
    const double bn2 = e.cc->template gauge<S>(e.ctx, ncell_, e.b, e.ctx->read_double(e.dscal));
    {
      NvtxRange nvs("nf.solve");
      *ss = e.solver->solve(e.b, P, bn2);
    }
    e.cc->template gauge<S>(e.ctx, ncell_, P, 0.0);
    launch_update<T, S>(L, g, sd, cview(e.alpha), cview(uh), P, mut(u_out));
    return NF_OK;
  }

  // Substep sub of m of the current frame: its time and length on the
  // tape, and a checkpoint of U every checkpoint_every steps.
  int begin_substep(int sub, int m) {
    // t = (f + (sub + 1) / m) dt, exact for m = 1
    const double h = g_.dt / m;
    const double t1 = (double)(frames_ * (int64_t)m + sub + 1) * h;
    const int C = std::max(1, ctx_->cfg.checkpoint_every);
    if (n_ % C == 0) {
      const int idx = n_ / C;
      while ((int)ckpt_.size() <= idx) {
        T *p = nullptr;
        CKS(faces(&p));
        ckpt_.push_back(p);
      }
      CKC(cudaMemcpyAsync(ckpt_[idx], U_, nfaces_ * sizeof(T), cudaMemcpyDeviceToDevice,
                          ctx_->stream));
    }
    ts_.resize(n_ + 1);
    hs_.resize(n_ + 1);
    ts_[n_] = t1;
    hs_[n_] = h;
    return NF_OK;
  }
  void end_substep() {
    ++n_;
    n_rev_ = n_;
    init_reverted_ = false;  // a later backward covers the whole history
    seg_start_ = -1;         // a new step invalidates the cached segment
  }

  // Step m (from ts_[m] - hs_[m] to ts_[m]): u_in -> uh, P, u_out (u_out
  // may alias u_in).
  int forward_step(Eng &e, int m, const T *u_in, T *u_out, T *uh, S *P, SolveStats *ss) {
    NvtxRange nv("nf.step");
    const GridDev g = grid_h(hs_[m]);
    const SceneDev sd = scene_at(sc_, ts_[m], dsph_, &bz_);
    CKS(geometry_and_advect(e, m, g, sd, u_in, uh));
    return project_faces(e, g, sd, uh, P, u_out, ss);
  }

  // Step m up to the projection: fractions at its end time (taped or
  // rasterised), then U^ from u_in by advection and viscosity.
  int geometry_and_advect(Eng &e, int m, const GridDev &g, const SceneDev &sd, const T *u_in,
                          T *uh) {
    Launch L = e.ctx->launch();
    bool joined = true;
    if (m < (int)tapeA_.size() && tapeA_[m] && tapeA_ok_[m]) {
      // recomputed step: the fractions kept by the first pass (bit-identical
      // to rasterising them again)
      CKC(cudaMemcpyAsync(e.alpha, tapeA_[m], nfaces_ * sizeof(T), cudaMemcpyDeviceToDevice, L.s));
    } else {
      NvtxRange nvr("nf.rasterize");
      const bool tape = e.ctx == ctx_ && ctx_->cfg.tape_fractions;  // (the first pass only)
      if (tape) {
        if ((int)tapeA_.size() <= m) {
          tapeA_.resize(m + 1, nullptr);
          tapeA_ok_.resize(m + 1, 0);
        }
        if (!tapeA_[m]) CKS(faces(&tapeA_[m]));
      }
      // The fractions (and their tape copy) go to a side stream and overlap
      // the advection below, which does not read them: both kernels are
      // latency-bound and leave most of the GPU idle. The context stream
      // waits for them before the projection. The episode's own engine only,
      // and not while kernel classes are being timed.
      Launch Lr = L;
      if (e.ctx == ctx_ && ctx_->prof.kclass == -2 && L.s == ctx_->stream) {
        CKS(side_.ensure());
        CKC(cudaEventRecord(side_.fork, L.s));
        CKC(cudaStreamWaitEvent(side_.s, side_.fork, 0));
        Lr = Launch{side_.s, L.counter, nullptr};
        joined = false;
      }
      launch_rasterize<T>(Lr, g, sd, mut(e.alpha));
      if (tape) {
        CKC(cudaMemcpyAsync(tapeA_[m], e.alpha, nfaces_ * sizeof(T), cudaMemcpyDeviceToDevice,
                            Lr.s));
        tapeA_ok_[m] = 1;
      }
    }
    NvtxRange nva("nf.advect");
    if (e.Ut) {
      // U~ = B(U) U, then U^ = (I - nu h / dx^2 G^T G) U~ (Sec. 2.3.1)
      launch_advect<T>(L, g, cview(u_in), mut(e.Ut), ctx_->cfg.advect_order);
      launch_viscosity<T>(L, g, cview(e.Ut), mut(uh));
    } else {
      launch_advect<T>(L, g, cview(u_in), mut(uh), ctx_->cfg.advect_order);
    }
    if (!joined) {
      CKC(cudaEventRecord(side_.join, side_.s));
      CKC(cudaStreamWaitEvent(L.s, side_.join, 0));
    }
    return NF_OK;
  }

 public:
  // ------------------------------------------------ batched substeps -----
  // nf_step_batch: the members' substeps run up to the right-hand side on
  // their own, the projections of one substep as one stacked solve, then
  // each member's blended update.
  int batch_before(int sub, int m, GridDev *g, SceneDev *sd, double *bn2) {
    CKS(begin_substep(sub, m));
    *g = grid_h(hs_[n_]);
    *sd = scene_at(sc_, ts_[n_], dsph_, &bz_);
    Eng e = eng();
    CKS(geometry_and_advect(e, n_, *g, *sd, U_, Uh_));
    Launch L = ctx_->launch();
    launch_rhs<T, S>(L, *g, *sd, cview(alpha_), cview(Uh_), b_, ctx_->rs, dscal_);
    *bn2 = ctx_->read_double(dscal_);
    return check_launch();
  }
  int batch_after(const GridDev &g, const SceneDev &sd) {
    Launch L = ctx_->launch();
    launch_update<T, S>(L, g, sd, cview(alpha_), cview(Uh_), P_, mut(U_));
    end_substep();
    return check_launch();
  }
  void batch_end_frame() { ++frames_; }
  int substeps_now(int *m) {
    *m = 1;
    if (ctx_->cfg.cfl_max > 0.0) {
      const double umax = max_speed();
      if (!std::isfinite(umax)) return diverged("step: non-finite velocity");
      *m = std::max(1, (int)std::ceil(umax * g_.dt / (g_.dx * ctx_->cfg.cfl_max)));
    }
    return NF_OK;
  }
  const GridDev &grid() const { return g_; }
  bool batchable_with(EpisodeBase *const *eps, int n) const override {
    for (int i = 0; i < n; ++i) {
      const auto *o = static_cast<const EpisodeImpl *>(eps[i]);
      if (o->g_.nx != g_.nx || o->g_.ny != g_.ny || o->g_.nz != g_.nz ||
          o->solver_.levels() != solver_.levels())
        return false;
    }
    return true;
  }
  const T *alpha() const { return alpha_; }
  const S *rhs() const { return b_; }
  S *pressure_buf() { return P_; }
  int levels() const { return solver_.levels(); }
  void acc(nf_step_stats *s, const SolveStats &ss) { acc_stats(s, ss); }

 private:

  // ---------------------------------------------------------- backward ----
  // A recomputed segment: per step the velocity entering it, U^, the
  // fractions, the pressure and whether a component floats.
  struct Seg {
    std::vector<T *> U, Uh, A;
    std::vector<S *> P;
    std::vector<int> Float;
    T *tmpU = nullptr;
    int start = -1;  // first step held (-1: none)
  };

  int ensure_segment_buffers(Seg &sg, int C) {
    while ((int)sg.U.size() < C) {
      T *a = nullptr, *b = nullptr, *f = nullptr;
      S *p = nullptr;
      CKS(faces(&a));
      CKS(faces(&b));
      CKS(faces(&f));
      CKS(A_.get(&p, ncell_ * sizeof(S)));
      sg.U.push_back(a);
      sg.Uh.push_back(b);
      sg.A.push_back(f);
      sg.P.push_back(p);
      sg.Float.push_back(-1);
    }
    if (!sg.tmpU) CKS(faces(&sg.tmpU));
    return NF_OK;
  }

  // Recompute segment s from its checkpoint with engine e into sg.
  int recompute_into(Eng &e, Seg &sg, int s, nf_step_stats *st) {
    NvtxRange nv("nf.recompute");
    const int C = std::max(1, ctx_->cfg.checkpoint_every);
    const int start = s * C, end = std::min(start + C, n_);
    CKC(cudaMemcpyAsync(sg.U[0], ckpt_[s], nfaces_ * sizeof(T), cudaMemcpyDeviceToDevice,
                        e.ctx->stream));
    for (int m = start; m < end; ++m) {
      const int k = m - start;
      T *out = (k + 1 < end - start) ? sg.U[k + 1] : sg.tmpU;
      SolveStats ss;
      CKS(forward_step(e, m, sg.U[k], out, sg.Uh[k], sg.P[k], &ss));
      // keep the step's fractions for its adjoint (saves a rasterisation)
      // and whether any component floats (if none, the adjoint needs no
      // labels: its gauge is the identity)
      CKC(cudaMemcpyAsync(sg.A[k], e.alpha, nfaces_ * sizeof(T), cudaMemcpyDeviceToDevice,
                          e.ctx->stream));
      sg.Float[k] = e.cc->nfloat;
      acc_stats(st, ss);
    }
    sg.start = start;
    return NF_OK;
  }

  // Segment s on the episode's own engine.
  int recompute_segment(int s, nf_step_stats *st) {
    CKS(ensure_segment_buffers(seg_, std::max(1, ctx_->cfg.checkpoint_every)));
    Eng e = eng();
    CKS(recompute_into(e, seg_, s, st));
    seg_start_ = seg_.start;
    return NF_OK;
  }

  // ------------------------------------------- overlapped recompute -----
  // While the backward pass reverts segment s on the context's stream, a
  // helper thread recomputes segment s - 1 on a stream of its own, with its
  // own solver, components and scratch, into a second segment set; the two
  // are swapped at the segment boundary. Both are latency-bound chains of
  // small launches, so their kernels fill each other's gaps. Results are
  // those of the sequential order (the same kernels on the same data).
  struct Helper {
    Ctx ctx;
    std::unique_ptr<Solver<T, S, V, TA>> solver;
    Components cc;
    T *alpha = nullptr, *Ut = nullptr;
    S *b = nullptr;
    double *dscal = nullptr;
    Seg seg;
    std::thread th;
    int rc = NF_OK;
    nf_step_stats st{};
    bool ready = false;
    ~Helper() {
      if (th.joinable()) th.join();
      if (ctx.stream) cudaStreamDestroy(ctx.stream);
      if (ctx.rs.partials) cudaFree(ctx.rs.partials);
      if (ctx.rs.ticket) cudaFree(ctx.rs.ticket);
      if (ctx.pinned) cudaFreeHost(ctx.pinned);
    }
  };

  bool overlap_ok() const {
    if (!ctx_->cfg.recompute_overlap || ctx_->prof.kclass != -2) return false;
    // the taped fractions must cover every step (a recompute that rasterises
    // would write the tape from the helper thread)
    if (ctx_->cfg.tape_fractions)
      for (int m = 0; m < n_; ++m)
        if (m >= (int)tapeA_.size() || !tapeA_[m] || !tapeA_ok_[m]) return false;
    return true;
  }

  int helper_init() {
    if (helper_) return NF_OK;
    auto h = std::make_unique<Helper>();
    h->ctx.device = ctx_->device;
    h->ctx.cfg = ctx_->cfg;
    h->ctx.prof.kclass = -2;
    CKC(cudaStreamCreateWithFlags(&h->ctx.stream, cudaStreamNonBlocking));
    CKC(cudaMalloc(&h->ctx.rs.partials, sizeof(double) * kRedBlocks * kMaxWidth));
    CKC(cudaMalloc(&h->ctx.rs.ticket, sizeof(unsigned int)));
    CKC(cudaMemset(h->ctx.rs.ticket, 0, sizeof(unsigned int)));
    CKC(cudaMallocHost(&h->ctx.pinned, 4096));
    CKS(faces(&h->alpha));
    if (g_.nu > 0.0) CKS(faces(&h->Ut));
    CKS(A_.get(&h->b, ncell_ * sizeof(S)));
    CKS(A_.get(&h->dscal, 64 * sizeof(double)));
    h->solver = std::make_unique<Solver<T, S, V, TA>>(&h->ctx, g_, ctx_->cfg);
    CKS(h->solver->init(A_));
    CKS(h->cc.init(A_, ncell_));
    h->solver->set_projector(&h->cc);
    CKS(ensure_segment_buffers(h->seg, std::max(1, ctx_->cfg.checkpoint_every)));
    CKC(cudaStreamSynchronize(ctx_->stream));  // allocations are ordered on this stream
    helper_ = std::move(h);
    return NF_OK;
  }

  // Start recomputing segment s on the helper (context stream's work so far
  // comes first: the checkpoints and buffers it reads).
  int helper_start(int s) {
    Helper &h = *helper_;
    cudaEvent_t ev;
    CKC(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CKC(cudaEventRecord(ev, ctx_->stream));
    CKC(cudaStreamWaitEvent(h.ctx.stream, ev, 0));
    CKC(cudaEventDestroy(ev));
    h.rc = NF_OK;
    h.st = nf_step_stats{};
    h.ready = false;
    const int dev = ctx_->device;
    h.th = std::thread([this, &h, s, dev] {
      cudaSetDevice(dev);
      Eng e{&h.ctx, h.alpha, h.b, &h.cc, h.solver.get(), h.Ut, h.dscal};
      int rc = recompute_into(e, h.seg, s, &h.st);
      const cudaError_t ce = cudaStreamSynchronize(h.ctx.stream);
      if (rc == NF_OK && ce != cudaSuccess) rc = cuda_fail(ce, "recompute helper");
      h.rc = rc;
    });
    return NF_OK;
  }

  // Wait for the helper; on success its segment becomes the current one.
  int helper_join(nf_step_stats *st) {
    Helper &h = *helper_;
    if (!h.th.joinable()) return NF_OK;
    h.th.join();
    ctx_->launches += h.ctx.launches;
    h.ctx.launches = 0;
    if (h.rc != NF_OK && h.rc != NF_E_NOT_CONVERGED) return h.rc;
    st->solves += h.st.solves;
    st->iters += h.st.iters;
    st->outer += h.st.outer;
    st->max_iters = std::max(st->max_iters, h.st.max_iters);
    st->rel_residual = std::max(st->rel_residual, h.st.rel_residual);
    std::swap(seg_, h.seg);
    seg_start_ = seg_.start;
    return NF_OK;
  }

  // Adjoint of one projection (fractions alpha_ for scene state sd) with
  // the forward's U^ = uh and pressure P: gU_ -> gUh_, theta gradient.
  int adjoint_projection(const GridDev &g, const SceneDev &sd, const T *uh,
                         const S *P, double *gth, nf_step_stats *st,
                         bool relabel = true) {
    NvtxRange nv("nf.adjoint_projection");
    Launch L = ctx_->launch();
    if (relabel)
      CKS(cc_.label<T>(ctx_, g, cview(alpha_)));
    else
      cc_.nfloat = 0;
    solver_.set_fractions(comp(alpha_, 0), comp(alpha_, 1), comp(alpha_, 2));
    launch_adj_gp<T, S>(L, g, cview(alpha_), cview(gU_), gP_, ctx_->rs, dscal_);
    const double n2 = gauge(gP_, ctx_->read_double(dscal_));
    const SolveStats ss = solver_.solve(gP_, y_, n2);
    gauge(y_, 0.0);
    acc_stats(st, ss);
    launch_adj_face<T, S>(L, g, sd, cview(alpha_), cview(uh), P, y_, cview(gU_),
                          mut(gUh_), ctx_->rs, dscal_ + 8);
    if (sd.K > 0) {
      double h[kMaxParams];
      ctx_->read_bytes(h, dscal_ + 8, sizeof(h));
      for (int k = 0; k < sd.K; ++k) gth[k] += h[k];
    }
    return ss.status;
  }

  // Revert the most recent unreverted step (or the initial projection).
  int revert_one(double *gth, nf_step_stats *st) {
    NvtxRange nv("nf.backward_step");
    Launch L = ctx_->launch();
    if (n_rev_ == 0) {
      if (!init_proj_ || init_reverted_)
        return state_err("backward_step: nothing left to revert");
      const SceneDev sd = scene_at(sc_, 0.0, dsph_, &bz_);
      launch_rasterize<T>(L, g_, sd, mut(alpha_));
      const int rc = adjoint_projection(g_, sd, Uinit_, Pinit_, gth, st);
      CKC(cudaMemcpyAsync(gU_, gUh_, nfaces_ * sizeof(T), cudaMemcpyDeviceToDevice, L.s));
      init_reverted_ = true;
      return rc;
    }
    const int m = n_rev_ - 1;
    const int C = std::max(1, ctx_->cfg.checkpoint_every);
    const int s = m / C;
    if (seg_start_ != s * C && helper_ && helper_seg_ == s) {
      helper_seg_ = -1;
      CKS(helper_join(st));
    }
    if (seg_start_ != s * C) CKS(recompute_segment(s, st));
    // the segment before this one, on the helper, while this one is reverted
    if (overlap_now_ && s >= 1 && helper_seg_ < 0) {
      CKS(helper_init());
      CKS(helper_start(s - 1));
      helper_seg_ = s - 1;
    }
    const int k = m - seg_start_;
    const GridDev g = grid_h(hs_[m]);
    const SceneDev sd = scene_at(sc_, ts_[m], dsph_, &bz_);
    // the step's fractions, kept by the recompute (the solver's captured
    // graphs read alpha_, so they are copied back rather than pointed to)
    CKC(cudaMemcpyAsync(alpha_, seg_.A[k], nfaces_ * sizeof(T), cudaMemcpyDeviceToDevice, L.s));
    const int rc = adjoint_projection(g, sd, seg_.Uh[k], seg_.P[k], gth, st, seg_.Float[k] != 0);
    const T *gUt = gUh_;
    if (Ut_) {
      // dJ/dU~ = (I - nu h / dx^2 G^T G) dJ/dU^ (Sec. 2.3.2; the map is
      // symmetric). Ut_ is free here: the recompute above is done with it.
      launch_viscosity<T>(L, g, cview(gUh_), mut(Ut_));
      gUt = Ut_;
    }
    {
      NvtxRange nva("nf.advect_adjoint");
      launch_advect_adjoint<T>(L, g, cview(seg_.U[k]), cview(gUt), mut(gUb_),
                               ctx_->cfg.advect_order);
    }
    std::swap(gU_, gUb_);
    n_rev_ = m;
    st->steps += 1;
    return rc;
  }

  Ctx *ctx_;
  GridDev g_;
  nf_scene sc_;
  Solver<T, S, V, TA> solver_;
  Components cc_;
  Alloc A_;
  int64_t nfaces_ = 0, ncell_ = 0;
  T *U_ = nullptr, *Uh_ = nullptr, *alpha_ = nullptr;
  T *gU_ = nullptr, *gUb_ = nullptr, *gUh_ = nullptr;
  T *Ut_ = nullptr;  // viscous grids only: U~ (forward), dJ/dU~ (adjoint)
  S *P_ = nullptr, *b_ = nullptr, *gP_ = nullptr, *y_ = nullptr;
  void *stage_ = nullptr;
  double *dscal_ = nullptr;  // [0] norms, [1] loss, [8..16) dJ/dtheta
  double *dsph_ = nullptr;
  std::vector<double> bz_src_;  // the caller's shape table (extruded scenes)
  BzInfo bz_;
  double *bz_dev_ = nullptr;
  // tape
  int n_ = 0, n_rev_ = 0, frames_ = 0;
  std::vector<double> ts_, hs_;  // end time and length of every step
  bool init_proj_ = false, init_reverted_ = false;
  T *Uinit_ = nullptr;
  S *Pinit_ = nullptr;
  std::vector<T *> ckpt_;
  int seg_start_ = -1;
  Seg seg_;                          // the segment the backward pass reverts
  std::unique_ptr<Helper> helper_;   // overlapped recompute (backward)
  // A second stream of the episode and its fork / join events (the
  // forward's rasterisation beside the advection), made on first use.
  struct Side {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int ensure() {
      if (s) return NF_OK;
      CKC(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      CKC(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
      CKC(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
      return NF_OK;
    }
    ~Side() {
      if (fork) cudaEventDestroy(fork);
      if (join) cudaEventDestroy(join);
      if (s) cudaStreamDestroy(s);
    }
  };
  Side side_;
  int helper_seg_ = -1;              // segment the helper is recomputing
  bool overlap_now_ = false;         // inside a whole-rollout backward pass
  std::vector<T *> tapeA_;     // fractions of every step (tape_fractions)
  std::vector<char> tapeA_ok_; // tapeA_[m] holds step m of the current tape
};

size_t episode_base_bytes(const nf_config &cfg, const nf_grid &g) {
  const size_t nf = (size_t)(g.nx + 1) * g.ny * g.nz + (size_t)g.nx * (g.ny + 1) * g.nz +
                    (size_t)g.nx * g.ny * (g.nz + 1);
  const size_t nc = (size_t)g.nx * g.ny * g.nz;
  const size_t t = cfg.precision == NF_PREC_FP64 ? 8 : 4;
  const size_t s = cfg.precision == NF_PREC_FP32 ? 4 : 8;
  const size_t v = cfg.precision == NF_PREC_FP64 ? 8 : 4;
  size_t b = (g.nu > 0.0 ? 7 : 6) * nf * t + 4 * nc * s + nc * 8;  // fields, scalars, staging
  b += nc * 20;                                  // component labels, gauge
  b += nc * s + 5 * nc * v;                      // solver vectors
  b += (nc * (2 * v + 3 * t)) * 2 / 7 + nc * v;  // hierarchy (approx.)
  return b;
}

// ------------------------------------------------------ batched solve -----
// B same-size episodes stacked along z into one grid of nx x ny x (B nz)
// cells. Each member keeps its own closed z walls (alpha = 0 on the planes
// between members), so the stacked operator is block diagonal: one solve
// of the stack is B independent projections, and every kernel of the
// solver (smoothing, restriction, the coarse chain, the CG updates and dots,
// the FP64 residual) runs once for all members. The stacked hierarchy is
// capped at the members' own level count, so coarse cells never straddle
// two members. Members' CG iterates share their step lengths (one Krylov
// process): the result of each member differs from its solve alone within
// the solver tolerance, which the stopping rule keeps for every member.
template <class T, class S, class V, class TA>
struct BatchProj : BatchBase {
  Ctx *ctx;
  GridDev gs;  // stacked grid, unit operator scale
  GridDev ge;  // one member's grid
  int B;
  Alloc A;
  Solver<T, S, V, TA> solver;
  Components cc;
  T *alpha = nullptr;
  S *b = nullptr, *P = nullptr;
  std::vector<double> scale_;  // each member's right-hand-side scale

  static GridDev stacked(const GridDev &g, int B) {
    GridDev s = g;
    s.nz = g.nz * B;
    s.c = 1.0;
    s.outlet = 0;  // open faces are found from the fractions
    s.inlet = 0;
    s.set_derived();
    return s;
  }
  BatchProj(Ctx *c, const GridDev &g, int nb)
      : ctx(c), gs(stacked(g, nb)), ge(g), B(nb), solver(c, stacked(g, nb), c->cfg),
        scale_(nb, 1.0) {
    A.stream = c->stream;
  }
  ~BatchProj() override { A.free_all(); }
  size_t bytes() const override { return A.bytes; }

  int init(int levels) {
    const int64_t nf = gs.nface(0) + gs.nface(1) + gs.nface(2);
    CKS(A.get(&alpha, nf * sizeof(T)));
    CKS(A.get(&b, gs.ncell() * sizeof(S)));
    CKS(A.get(&P, gs.ncell() * sizeof(S)));
    solver.set_max_levels(levels);
    CKS(solver.init(A));
    CKS(cc.init(A, gs.ncell()));
    solver.set_projector(&cc);
    return NF_OK;
  }

  // Gather the members' fractions and right-hand sides (slot e of the
  // stack; a null member leaves its slot empty: no active cell), solve,
  // scatter the pressures. bn2[e] = ||b_e||^2 of each member.
  template <class E>
  SolveStats solve(E *const *mem, const double *bn2) {
    Launch L = ctx->launch();
    const int64_t fx = ge.nface(0), fy = ge.nface(1), nc = ge.ncell();
    const int64_t zplane = (int64_t)ge.nx * ge.ny;
    T *ax = alpha, *ay = alpha + gs.nface(0), *az = alpha + gs.nface(0) + gs.nface(1);
    double total = 0.0, tmin = 0.0;
    for (int e = 0; e < B; ++e) {
      if (!mem[e]) {
        cudaMemsetAsync(ax + e * fx, 0, fx * sizeof(T), L.s);
        cudaMemsetAsync(ay + e * fy, 0, fy * sizeof(T), L.s);
        cudaMemsetAsync(az + e * nc, 0, nc * sizeof(T), L.s);
        cudaMemsetAsync(b + e * nc, 0, nc * sizeof(S), L.s);
        continue;
      }
      const T *a = mem[e]->alpha();
      cudaMemcpyAsync(ax + e * fx, a, fx * sizeof(T), cudaMemcpyDeviceToDevice, L.s);
      cudaMemcpyAsync(ay + e * fy, a + fx, fy * sizeof(T), cudaMemcpyDeviceToDevice, L.s);
      // z faces: the member's planes 0 .. nz - 1 (its top wall is the next
      // member's bottom wall, alpha = 0 in both)
      cudaMemcpyAsync(az + e * nc, a + fx + fy, nc * sizeof(T), cudaMemcpyDeviceToDevice, L.s);
      // each member's right-hand side scaled by a power of two to norm in
      // [1/2, 2) (exact, undone on its pressure): the stacked stopping rule
      // then asks every member for about the same relative residual
      const double sb = bn2[e] > 0.0 ? std::ldexp(1.0, -std::ilogb(std::sqrt(bn2[e]))) : 1.0;
      scale_[e] = sb;
      scaled_copy<S>(L, nc, mem[e]->rhs(), b + e * nc, sb);
      const double n2 = bn2[e] * sb * sb;
      total += n2;
      if (n2 > 0.0 && (tmin == 0.0 || n2 < tmin)) tmin = n2;
    }
    cudaMemsetAsync(az + (int64_t)B * nc, 0, zplane * sizeof(T), L.s);  // the stack's top wall
    SolveStats ss;
    if (cc.label<T>(ctx, gs, Fields<T>{ax, ay, az}) != NF_OK) {
      ss.status = NF_E_CUDA;
      return ss;
    }
    solver.set_fractions(ax, ay, az);
    const double bn = cc.gauge<S>(ctx, gs.ncell(), b, total);
    ss = solver.solve(b, P, bn, tmin);
    cc.gauge<S>(ctx, gs.ncell(), P, 0.0);
    for (int e = 0; e < B; ++e)
      if (mem[e]) scaled_copy<S>(L, nc, P + e * nc, mem[e]->pressure_buf(), 1.0 / scale_[e]);
    return ss;
  }
};

template <class T, class S, class V, class TA>
static int step_batch_t(Ctx *ctx, BatchCache &cache, EpisodeBase *const *base, int n,
                        int nframes, nf_step_stats *st, int *stat) {
  using E = EpisodeImpl<T, S, V, TA>;
  std::vector<E *> eps(n);
  for (int i = 0; i < n; ++i) eps[i] = static_cast<E *>(base[i]);
  const GridDev &g0 = eps[0]->grid();
  const std::array<int, 4> key = {g0.nx, g0.ny, g0.nz, n};
  auto it = cache.find(key);
  if (it == cache.end()) {
    auto *bp = new BatchProj<T, S, V, TA>(ctx, g0, n);
    const int rc = bp->init(eps[0]->levels());
    if (rc != NF_OK) {
      delete bp;
      return rc;
    }
    it = cache.emplace(key, std::unique_ptr<BatchBase>(bp)).first;
  }
  auto *bp = static_cast<BatchProj<T, S, V, TA> *>(it->second.get());
  std::vector<nf_step_stats> s(n);
  std::vector<int> status(n, NF_OK), m(n);
  std::vector<GridDev> gh(n);
  std::vector<SceneDev> sd(n);
  std::vector<double> bn2(n);
  std::vector<E *> mem(n);
  for (int f = 0; f < nframes; ++f) {
    int M = 0;
    for (int i = 0; i < n; ++i) {
      m[i] = 0;
      if (status[i] == NF_E_DIVERGED) continue;
      const int rc = eps[i]->substeps_now(&m[i]);
      if (rc != NF_OK) {
        status[i] = rc;
        m[i] = 0;
      }
      M = std::max(M, m[i]);
    }
    for (int sub = 0; sub < M; ++sub) {
      for (int i = 0; i < n; ++i) {
        mem[i] = nullptr;
        if (sub >= m[i]) continue;
        CKS(eps[i]->batch_before(sub, m[i], &gh[i], &sd[i], &bn2[i]));
        if (!std::isfinite(bn2[i])) {  // this member diverged: out of the batch
          status[i] = NF_E_DIVERGED;
          m[i] = 0;
          continue;
        }
        mem[i] = eps[i];
      }
      const SolveStats ss = bp->solve(mem.data(), bn2.data());
      for (int i = 0; i < n; ++i) {
        if (!mem[i]) continue;
        eps[i]->acc(&s[i], ss);
        s[i].steps += 1;
        if (ss.status != NF_OK && status[i] == NF_OK) status[i] = ss.status;
        CKS(eps[i]->batch_after(gh[i], sd[i]));
      }
    }
    for (int i = 0; i < n; ++i)
      if (status[i] != NF_E_DIVERGED) eps[i]->batch_end_frame();
  }
  int worst = NF_OK;
  for (int i = 0; i < n; ++i) {
    if (st) st[i] = s[i];
    if (stat) stat[i] = status[i];
    if (status[i] != NF_OK && worst == NF_OK) worst = status[i];
    if (status[i] == NF_E_DIVERGED) worst = NF_E_DIVERGED;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batched step");
  return worst;
}

int step_batch(Ctx *ctx, BatchCache &cache, EpisodeBase *const *eps, int n, int nframes,
               nf_step_stats *st, int *status) {
  switch (ctx->cfg.precision) {
    case NF_PREC_FP64:
      return step_batch_t<double, double, double, double>(ctx, cache, eps, n, nframes, st,
                                                          status);
    case NF_PREC_FP32:
      return step_batch_t<float, float, float, float>(ctx, cache, eps, n, nframes, st, status);
    default:
      return step_batch_t<float, double, float, __nv_bfloat16>(ctx, cache, eps, n, nframes, st,
                                                               status);
  }
}

template <class T, class S, class V, class TA>
static int make(Ctx *ctx, const nf_grid *g, const nf_scene *s, EpisodeBase **out) {
  auto *e = new EpisodeImpl<T, S, V, TA>(ctx, *g, *s);
  const int rc = e->init(*s);
  if (rc != NF_OK) {
    delete e;
    return rc;
  }
  *out = e;
  return NF_OK;
}

int create_episode(Ctx *ctx, const nf_grid *g, const nf_scene *s,
                   EpisodeBase **out) {
  *out = nullptr;
  switch (ctx->cfg.precision) {
    case NF_PREC_FP64:
      return make<double, double, double, double>(ctx, g, s, out);
    case NF_PREC_FP32:
      return make<float, float, float, float>(ctx, g, s, out);
    default:
      return make<float, double, float, __nv_bfloat16>(ctx, g, s, out);
  }
}

}  // namespace nf
