// The C ABI of libnf (declared in include/nf.h): argument checking, context
// and episode bookkeeping, HBM admission, kernel-class profiling and error
// plumbing. No exception crosses the ABI; every entry point returns a status.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "episode.h"
#include "kernels.h"
#include "util.h"

namespace nf {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }
const std::string &get_error() { return g_err; }
int cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? NF_E_OOM : NF_E_CUDA;
}

int Alloc::get(void **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 16;
  // stream-ordered: unlike cudaMalloc / cudaFree this never synchronises
  // the device, so episodes created or destroyed while others run (the
  // serving slots) do not stall the other streams
  const cudaError_t e = cudaMallocAsync(p, n, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return cuda_fail(e, "cudaMallocAsync");
  }
  ptrs.push_back(*p);
  bytes += n;
  return NF_OK;
}

void Alloc::free_all() {
  for (void *p : ptrs) cudaFreeAsync(p, stream);
  ptrs.clear();
  bytes = 0;
}

// ------------------------------------------------------------ profiling ---
static constexpr size_t kProfSlots = 4096;

static constexpr int kGraphSlot = 1 << 30;

void GraphEvents::clear() {
  for (auto &e : ev) cudaEventDestroy(e);
  ev.clear();
  cls.clear();
  iter.clear();
}

void prof_begin(Prof *p, int kclass, cudaStream_t s, int *slot) {
  *slot = -1;
  if (p->kclass != -1 && p->kclass != kclass) return;
  if (p->capture_ev) {
    GraphEvents &ge = *p->capture_ev;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    ge.ev.push_back(a);
    ge.ev.push_back(b);
    ge.cls.push_back(kclass);
    ge.iter.push_back(p->capture_iter);
    cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
    *slot = kGraphSlot | (int)(ge.cls.size() - 1);
    return;
  }
  if (p->ev.empty()) {
    p->ev.resize(2 * kProfSlots);
    p->cls.resize(kProfSlots);
    for (auto &e : p->ev) cudaEventCreate(&e);
  }
  if (p->used == kProfSlots) p->drain(s);
  *slot = (int)p->used++;
  p->cls[*slot] = kclass;
  cudaEventRecord(p->ev[2 * *slot], s);
}

void prof_end(Prof *p, int slot, cudaStream_t s) {
  if (slot & kGraphSlot) {
    cudaEventRecordWithFlags(p->capture_ev->ev[2 * (slot & ~kGraphSlot) + 1], s,
                             cudaEventRecordExternal);
    return;
  }
  cudaEventRecord(p->ev[2 * slot + 1], s);
}

void Prof::collect(const GraphEvents &ge, int iters) {
  for (size_t i = 0; i < ge.cls.size(); ++i) {
    if (ge.iter[i] >= iters) continue;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ge.ev[2 * i], ge.ev[2 * i + 1]) == cudaSuccess) {
      launches[ge.cls[i]] += 1;
      ms[ge.cls[i]] += t;
    } else {
      cudaGetLastError();
    }
  }
}

void Prof::drain(cudaStream_t s) {
  cudaStreamSynchronize(s);
  for (size_t i = 0; i < used; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
      launches[cls[i]] += 1;
      ms[cls[i]] += t;
    } else {
      cudaGetLastError();
    }
  }
  used = 0;
}

void Prof::reset() {
  used = 0;
  for (int k = 0; k < NF_K_COUNT; ++k) {
    launches[k] = 0;
    ms[k] = 0.0;
  }
}

Prof::~Prof() {
  for (auto &e : ev) cudaEventDestroy(e);
}

double Ctx::read_double(const double *dptr) {
  double *h = (double *)pinned;
  cudaMemcpyAsync(h, dptr, sizeof(double), cudaMemcpyDeviceToHost, stream);
  cudaStreamSynchronize(stream);
  return *h;
}

void Ctx::read_bytes(void *host, const void *dev, size_t n) {
  cudaMemcpyAsync(pinned, dev, n, cudaMemcpyDeviceToHost, stream);
  cudaStreamSynchronize(stream);
  memcpy(host, pinned, n);
}

}  // namespace nf


using nf::set_error;

#define GUARD(ctx)                                                    \
  do {                                                                \
    if (!(ctx)) {                                                     \
      set_error("null context");                                      \
      return NF_E_INVALID;                                            \
    }                                                                 \
    cudaError_t _e = cudaSetDevice((ctx)->c.device);                  \
    if (_e != cudaSuccess) return nf::cuda_fail(_e, "cudaSetDevice"); \
  } while (0)

static nf::EpisodeBase *find(nf_ctx *ctx, int64_t id) {
  auto it = ctx->eps.find(id);
  if (it == ctx->eps.end()) {
    set_error("unknown episode id " + std::to_string(id));
    return nullptr;
  }
  return it->second.get();
}

#define EPISODE(ctx, id, e)           \
  GUARD(ctx);                         \
  nf::EpisodeBase *e = find(ctx, id); \
  if (!e) return NF_E_INVALID;

static bool valid_dtype(int dt) { return dt == NF_F32 || dt == NF_F64; }
static bool valid_mem(int m) { return m == NF_MEM_DEVICE || m == NF_MEM_HOST; }

extern "C" {

int nf_config_default(nf_config *cfg) {
  if (!cfg) return NF_E_INVALID;
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->precision = NF_PREC_MIXED;
  cfg->solver = NF_SOLVER_MGPCG;
  cfg->tol = 1e-6;
  cfg->max_iters = 500;
  cfg->inner_tol = 1e-3;
  cfg->mg_smooth = 2;
  cfg->mg_coarsest = 4;
  cfg->advect_order = 2;
  cfg->checkpoint_every = 10;
  cfg->hbm_budget = 0;
  cfg->cfl_max = 0.0;
  cfg->mg_coarsest_sweeps = 8;
  cfg->mg_band_sweeps = 0;
  cfg->mg_transfer = 1;
  cfg->mg_coarse_weight = 1.9;
  cfg->mg_smooth_coarse = 0;
  cfg->tape_fractions = 0;
  cfg->mg_persistent = 0;
  cfg->mg_cluster = 0;
  cfg->residual_fp64 = 1;
  cfg->mg_fused = 0;
  cfg->recompute_overlap = 1;
  return NF_OK;
}

const char *nf_status_string(int s) {
  switch (s) {
    case NF_OK: return "ok";
    case NF_E_INVALID: return "invalid argument";
    case NF_E_OOM: return "out of device memory or over the HBM budget";
    case NF_E_NOT_CONVERGED: return "solver did not converge";
    case NF_E_DIVERGED: return "non-finite value in a residual";
    case NF_E_TIMEOUT: return "bounded device wait expired";
    case NF_E_CUDA: return "CUDA runtime error";
    case NF_E_STATE: return "call invalid in the current state";
    case NF_E_CANCELED: return "request cancelled before it started";
    default: return "unknown status";
  }
}

const char *nf_last_error(nf_ctx *) { return nf::get_error().c_str(); }

int nf_create(nf_ctx **out, const nf_config *cfg) {
  if (!out || !cfg) {
    set_error("nf_create: null argument");
    return NF_E_INVALID;
  }
  *out = nullptr;
  if (cfg->precision < NF_PREC_FP64 || cfg->precision > NF_PREC_MIXED ||
      (cfg->solver != NF_SOLVER_CG && cfg->solver != NF_SOLVER_MGPCG) ||
      !(cfg->tol > 0) || cfg->max_iters <= 0 ||
      (cfg->advect_order != 1 && cfg->advect_order != 2) ||
      cfg->checkpoint_every <= 0 || cfg->mg_smooth < 0 || !(cfg->cfl_max >= 0.0) ||
      cfg->mg_coarsest_sweeps < 0 || cfg->mg_band_sweeps < 0 ||
      (cfg->mg_transfer != 0 && cfg->mg_transfer != 1) ||
      !(cfg->mg_coarse_weight >= 0.0 && cfg->mg_coarse_weight < 2.0) ||
      cfg->mg_smooth_coarse < 0 || (cfg->tape_fractions != 0 && cfg->tape_fractions != 1) ||
      (cfg->mg_persistent != 0 && cfg->mg_persistent != 1) ||
      (cfg->residual_fp64 != 0 && cfg->residual_fp64 != 1) ||
      cfg->mg_fused < 0 || cfg->mg_fused > 2 ||
      (cfg->recompute_overlap != 0 && cfg->recompute_overlap != 1) ||
      (cfg->mg_cluster != 0 && cfg->mg_cluster != 1)) {
    set_error("nf_create: invalid configuration");
    return NF_E_INVALID;
  }
  nf_ctx *ctx = new (std::nothrow) nf_ctx();
  if (!ctx) return NF_E_OOM;
  ctx->c.cfg = *cfg;
  if (!(ctx->c.cfg.inner_tol > 0 && ctx->c.cfg.inner_tol < 1)) ctx->c.cfg.inner_tol = 1e-3;
  ctx->c.device = cfg->device;
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) {
    delete ctx;
    return nf::cuda_fail(e, "cudaSetDevice");
  }
  {
    // episode memory comes from this process's default pool of the device
    // (stream-ordered); keep freed blocks for reuse instead of returning
    // them at every synchronisation
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, cfg->device) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  if (cfg->stream) {
    ctx->c.stream = (cudaStream_t)cfg->stream;
  } else {
    e = cudaStreamCreateWithFlags(&ctx->c.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete ctx;
      return nf::cuda_fail(e, "cudaStreamCreate");
    }
    ctx->c.own_stream = true;
  }
  e = cudaMalloc(&ctx->c.rs.partials, sizeof(double) * nf::kRedBlocks * nf::kMaxWidth);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->c.rs.ticket, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(ctx->c.rs.ticket, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->c.pinned, 4096);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->c.dscal, sizeof(double));
  if (e != cudaSuccess) {
    const int rc = nf::cuda_fail(e, "nf_create allocation");
    nf_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return NF_OK;
}

int nf_destroy(nf_ctx *ctx) {
  if (!ctx) return NF_E_INVALID;
  cudaSetDevice(ctx->c.device);
  if (ctx->c.stream) cudaStreamSynchronize(ctx->c.stream);
  ctx->eps.clear();
  ctx->batches.clear();  // frees on the context's stream, before it goes
  if (ctx->c.rs.partials) cudaFree(ctx->c.rs.partials);
  if (ctx->c.rs.ticket) cudaFree(ctx->c.rs.ticket);
  if (ctx->c.pinned) cudaFreeHost(ctx->c.pinned);
  if (ctx->c.dscal) cudaFree(ctx->c.dscal);
  if (ctx->c.own_stream && ctx->c.stream) cudaStreamDestroy(ctx->c.stream);
  delete ctx;
  return NF_OK;
}

int nf_synchronize(nf_ctx *ctx) {
  GUARD(ctx);
  const cudaError_t e = cudaStreamSynchronize(ctx->c.stream);
  if (e != cudaSuccess) return nf::cuda_fail(e, "cudaStreamSynchronize");
  return NF_OK;
}

int nf_episode_create(nf_ctx *ctx, const nf_grid *g, const nf_scene *s,
                      int64_t *id) {
  GUARD(ctx);
  if (!g || !s || !id) {
    set_error("nf_episode_create: null argument");
    return NF_E_INVALID;
  }
  // the kernels index face arrays with 32-bit integers
  const int64_t max_faces = std::max({(int64_t)(g->nx + 1) * g->ny * g->nz,
                                      (int64_t)g->nx * (g->ny + 1) * g->nz,
                                      (int64_t)g->nx * g->ny * (g->nz + 1)});
  // nz = 1: the 2D variant as a one-cell slab between closed z walls
  if (g->nx < 4 || g->ny < 4 || (g->nz < 4 && g->nz != 1) || !(g->dx > 0) || !(g->dt > 0) ||
      max_faces > (int64_t)INT32_MAX) {
    set_error("nf_episode_create: grid must have >= 4 cells in x and y, nz >= 4 or nz = 1 "
              "(a 2D slab), dx > 0, dt > 0 and fewer than 2^31 faces per component");
    return NF_E_INVALID;
  }
  if (g->fractions != NF_FRACTIONS_SUPERSAMPLE && g->fractions != NF_FRACTIONS_CORNER) {
    set_error("nf_episode_create: unknown fraction rule");
    return NF_E_INVALID;
  }
  if (!(g->nu >= 0.0) || !std::isfinite(g->nu)) {
    set_error("nf_episode_create: viscosity nu must be finite and >= 0");
    return NF_E_INVALID;
  }
  if (g->outlet && (g->outlet_j0 < 0 || g->outlet_k0 < 0 || g->outlet_w <= 0 ||
                    g->outlet_h <= 0 || g->outlet_j0 + g->outlet_w > g->ny ||
                    g->outlet_k0 + g->outlet_h > g->nz)) {
    set_error("nf_episode_create: outlet patch outside the high-x wall");
    return NF_E_INVALID;
  }
  if (g->inlet) {
    const bool inside = (g->inlet_side == 1 || g->inlet_side == -1) && g->inlet_j0 >= 0 &&
                        g->inlet_k0 >= 0 && g->inlet_w > 0 && g->inlet_h > 0 &&
                        g->inlet_j0 + g->inlet_w <= g->ny && g->inlet_k0 + g->inlet_h <= g->nz;
    const bool overlap = g->outlet && g->inlet_side == 1 &&
                         g->inlet_j0 < g->outlet_j0 + g->outlet_w &&
                         g->outlet_j0 < g->inlet_j0 + g->inlet_w &&
                         g->inlet_k0 < g->outlet_k0 + g->outlet_h &&
                         g->outlet_k0 < g->inlet_k0 + g->inlet_h;
    if (!inside || overlap || !std::isfinite(g->inlet_speed)) {
      set_error("nf_episode_create: inflow patch outside an x wall, over the outlet, or "
                "with a non-finite speed");
      return NF_E_INVALID;
    }
  }
  if (s->kind < NF_SCENE_NONE || s->kind > NF_SCENE_EXTRUDED) {
    set_error("nf_episode_create: unknown scene kind");
    return NF_E_INVALID;
  }
  if (s->kind == NF_SCENE_EXTRUDED) {
    const std::string why = nf::bz_check(*s);
    if (!why.empty()) {
      set_error("nf_episode_create: extruded scene: " + why);
      return NF_E_INVALID;
    }
  }
  const int want = s->kind == NF_SCENE_SPHERE ? 3 : s->kind == NF_SCENE_CHAMBER ? 8
                   : s->kind == NF_SCENE_PLATE ? 4 : s->kind == NF_SCENE_EXTRUDED ? s->K : 0;
  if (s->K != want) {
    set_error("nf_episode_create: scene expects " + std::to_string(want) + " parameters");
    return NF_E_INVALID;
  }
  if (s->kind == NF_SCENE_SPHERES && (s->nspheres < 0 || (s->nspheres > 0 && !s->spheres))) {
    set_error("nf_episode_create: spheres array missing");
    return NF_E_INVALID;
  }
  const size_t need = nf::episode_base_bytes(ctx->c.cfg, *g);
  if (ctx->c.cfg.hbm_budget && ctx->c.bytes_in_use + need > ctx->c.cfg.hbm_budget) {
    set_error("nf_episode_create: HBM budget exceeded (admission refused)");
    return NF_E_OOM;
  }
  nf::EpisodeBase *e = nullptr;
  const int rc = nf::create_episode(&ctx->c, g, s, &e);
  if (rc != NF_OK) return rc;
  const int64_t eid = ctx->next_id++;
  ctx->c.bytes_in_use += e->bytes();
  ctx->eps[eid].reset(e);
  *id = eid;
  return NF_OK;
}

int nf_episode_destroy(nf_ctx *ctx, int64_t id) {
  EPISODE(ctx, id, e);
  cudaStreamSynchronize(ctx->c.stream);
  const size_t b = e->bytes();
  ctx->c.bytes_in_use -= std::min(b, ctx->c.bytes_in_use);
  ctx->eps.erase(id);
  return NF_OK;
}

int nf_episode_bytes(nf_ctx *ctx, int64_t id, size_t *bytes) {
  EPISODE(ctx, id, e);
  if (!bytes) return NF_E_INVALID;
  *bytes = e->bytes();
  return NF_OK;
}

int nf_set_params(nf_ctx *ctx, int64_t id, const double *theta, int K) {
  EPISODE(ctx, id, e);
  if (K > 0 && !theta) return NF_E_INVALID;
  return e->set_params(theta, K);
}

int nf_set_velocity(nf_ctx *ctx, int64_t id, const void *const u[3], int dtype,
                    int mem, int project, nf_step_stats *st) {
  EPISODE(ctx, id, e);
  if (!u || !valid_dtype(dtype) || !valid_mem(mem)) {
    set_error("nf_set_velocity: bad arguments");
    return NF_E_INVALID;
  }
  return e->set_velocity(u, dtype, mem, project, st);
}

int nf_step(nf_ctx *ctx, int64_t id, int nsteps, nf_step_stats *st) {
  EPISODE(ctx, id, e);
  return e->step(nsteps, st);
}

int nf_loss(nf_ctx *ctx, int64_t id, int loss_kind, double *J,
            void *const gU[3], int dtype, int mem) {
  EPISODE(ctx, id, e);
  if (!valid_dtype(dtype) || !valid_mem(mem)) return NF_E_INVALID;
  return e->loss(loss_kind, J, gU, dtype, mem);
}

int nf_backward_step(nf_ctx *ctx, int64_t id, const void *const gU_next[3],
                     void *const gU_prev[3], int dtype, int mem,
                     double *g_theta, nf_step_stats *st) {
  EPISODE(ctx, id, e);
  if (!gU_next || !valid_dtype(dtype) || !valid_mem(mem)) return NF_E_INVALID;
  return e->backward_step(gU_next, gU_prev, dtype, mem, g_theta, st);
}

int nf_backward(nf_ctx *ctx, int64_t id, const void *const gU_final[3],
                void *const gU0[3], int dtype, int mem, double *g_theta,
                nf_step_stats *st) {
  EPISODE(ctx, id, e);
  if (!gU_final || !valid_dtype(dtype) || !valid_mem(mem)) return NF_E_INVALID;
  return e->backward(gU_final, gU0, dtype, mem, g_theta, st);
}

int nf_get_velocity(nf_ctx *ctx, int64_t id, void *const u[3], int dtype, int mem) {
  EPISODE(ctx, id, e);
  if (!u || !valid_dtype(dtype) || !valid_mem(mem)) return NF_E_INVALID;
  return e->get_faces(0, u, dtype, mem);
}

int nf_get_advected(nf_ctx *ctx, int64_t id, void *const u[3], int dtype, int mem) {
  EPISODE(ctx, id, e);
  if (!u || !valid_dtype(dtype) || !valid_mem(mem)) return NF_E_INVALID;
  return e->get_faces(1, u, dtype, mem);
}

int nf_get_fractions(nf_ctx *ctx, int64_t id, void *const a[3], int dtype, int mem) {
  EPISODE(ctx, id, e);
  if (!a || !valid_dtype(dtype) || !valid_mem(mem)) return NF_E_INVALID;
  return e->get_faces(2, a, dtype, mem);
}

int nf_get_pressure(nf_ctx *ctx, int64_t id, void *p, int dtype, int mem) {
  EPISODE(ctx, id, e);
  if (!p || !valid_dtype(dtype) || !valid_mem(mem)) return NF_E_INVALID;
  return e->get_pressure(p, dtype, mem);
}

int nf_step_batch(nf_ctx *ctx, const int64_t *ids, int n, int nframes, nf_step_stats *st,
                  int *status) {
  GUARD(ctx);
  if (!ids || n < 1 || n > 64 || nframes < 0) {
    set_error("nf_step_batch: need 1 to 64 episode ids and nframes >= 0");
    return NF_E_INVALID;
  }
  std::vector<nf::EpisodeBase *> eps(n);
  for (int i = 0; i < n; ++i) {
    auto it = ctx->eps.find(ids[i]);
    if (it == ctx->eps.end()) {
      set_error("nf_step_batch: unknown episode id");
      return NF_E_INVALID;
    }
    for (int j = 0; j < i; ++j)
      if (ids[j] == ids[i]) {
        set_error("nf_step_batch: an episode appears twice");
        return NF_E_INVALID;
      }
    eps[i] = it->second.get();
  }
  if (n == 1) {
    const int rc = eps[0]->step(nframes, st);
    if (status) status[0] = rc;
    return rc;
  }
  if (!eps[0]->batchable_with(eps.data(), n)) {
    set_error("nf_step_batch: members must share their cell counts and multigrid depth");
    return NF_E_INVALID;
  }
  return nf::step_batch(&ctx->c, ctx->batches, eps.data(), n, nframes, st, status);
}

int nf_episode_export(nf_ctx *ctx, int64_t id, void *buf, size_t *bytes) {
  EPISODE(ctx, id, e);
  if (!bytes) return NF_E_INVALID;
  return e->export_state(buf, bytes);
}

int nf_episode_import(nf_ctx *ctx, int64_t id, const void *buf, size_t bytes) {
  EPISODE(ctx, id, e);
  return e->import_state(buf, bytes);
}

int nf_get_step(nf_ctx *ctx, int64_t id, int *n) {
  EPISODE(ctx, id, e);
  if (!n) return NF_E_INVALID;
  *n = e->step_index();
  return NF_OK;
}

int nf_dot(nf_ctx *ctx, const void *a, const void *b, int64_t n, int dtype,
           double *out) {
  GUARD(ctx);
  if (!a || !b || !out || n < 0 || !valid_dtype(dtype)) {
    set_error("nf_dot: bad arguments");
    return NF_E_INVALID;
  }
  cudaSetDevice(ctx->c.device);
  nf::Launch L = ctx->c.launch();
  if (dtype == NF_F64)
    nf::launch_dot<double>(L, n, (const double *)a, (const double *)b, ctx->c.rs, ctx->c.dscal);
  else
    nf::launch_dot<float>(L, n, (const float *)a, (const float *)b, ctx->c.rs, ctx->c.dscal);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nf::cuda_fail(e, "nf_dot");
  *out = ctx->c.read_double(ctx->c.dscal);
  return NF_OK;
}

int nf_check_conversions(nf_ctx *ctx, const double *in, int64_t n, float *out_f,
                         double *out_d, int64_t *mismatches) {
  GUARD(ctx);
  if (n < 0 || n > ((int64_t)1 << 24) || !mismatches || (n > 0 && (!in || !out_f || !out_d))) {
    set_error("nf_check_conversions: bad arguments");
    return NF_E_INVALID;
  }
  cudaSetDevice(ctx->c.device);
  *mismatches = 0;
  if (n == 0) return NF_OK;
  void *dev = nullptr;
  const size_t bytes = (size_t)n * (sizeof(double) + sizeof(float) + sizeof(double)) + 16;
  cudaError_t e = cudaMalloc(&dev, bytes);
  if (e != cudaSuccess) return nf::cuda_fail(e, "nf_check_conversions");
  double *din = (double *)dev;
  double *dd = din + n;
  unsigned long long *dm = (unsigned long long *)(dd + n);
  float *df = (float *)(dm + 1);
  const cudaStream_t st = ctx->c.stream;
  e = cudaMemcpyAsync(din, in, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dm, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    nf::launch_check_conversions(ctx->c.launch(), din, n, df, dd, dm);
    e = cudaGetLastError();
  }
  unsigned long long m = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_f, df, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_d, dd, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&m, dm, sizeof(m), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dev);
  if (e != cudaSuccess) return nf::cuda_fail(e, "nf_check_conversions");
  *mismatches = (int64_t)m;
  return NF_OK;
}

int nf_launch_count(nf_ctx *ctx, int64_t *count) {
  if (!ctx || !count) return NF_E_INVALID;
  *count = ctx->c.launches;
  return NF_OK;
}

int nf_profile(nf_ctx *ctx, int kclass) {
  GUARD(ctx);
  if (kclass < -2 || kclass >= NF_K_COUNT) return NF_E_INVALID;
  if (ctx->c.prof.used) ctx->c.prof.drain(ctx->c.stream);
  ctx->c.prof.reset();
  ctx->c.prof.kclass = kclass;
  ctx->c.prof.gen += 1;  // graphs are re-captured with (or without) events
  return NF_OK;
}

int nf_profile_read(nf_ctx *ctx, int kclass, int64_t *launches, double *ms) {
  GUARD(ctx);
  if (kclass < 0 || kclass >= NF_K_COUNT || !launches || !ms) return NF_E_INVALID;
  if (ctx->c.prof.used) ctx->c.prof.drain(ctx->c.stream);
  *launches = ctx->c.prof.launches[kclass];
  *ms = ctx->c.prof.ms[kclass];
  return NF_OK;
}

}  // extern "C"
