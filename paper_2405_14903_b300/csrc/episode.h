// Episode: one simulated grid with its scene, fields, solver hierarchy and
// rollout tape. Precision-specific implementations live in episode.cu.
#pragma once

#include <array>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "util.h"

namespace nf {

class EpisodeBase {
 public:
  virtual ~EpisodeBase() {}
  virtual int set_params(const double *theta, int K) = 0;
  virtual int set_velocity(const void *const u[3], int dtype, int mem,
                           int project, nf_step_stats *st) = 0;
  virtual int step(int nsteps, nf_step_stats *st) = 0;
  virtual int loss(int kind, double *J, void *const gU[3], int dtype,
                   int mem) = 0;
  virtual int backward_step(const void *const gU_next[3],
                            void *const gU_prev[3], int dtype, int mem,
                            double *g_theta, nf_step_stats *st) = 0;
  virtual int backward(const void *const gU_final[3], void *const gU0[3],
                       int dtype, int mem, double *g_theta,
                       nf_step_stats *st) = 0;
  // The loss of the current velocity and dJ/dtheta by BPTT over the whole
  // recorded rollout, with dJ/dU kept on the device.
  virtual int loss_backward(int kind, double *J, double *g_theta,
                            nf_step_stats *st) = 0;
  // which: 0 velocity, 1 advected velocity, 2 fractions
  virtual int get_faces(int which, void *const dst[3], int dtype, int mem) = 0;
  virtual int get_pressure(void *dst, int dtype, int mem) = 0;
  virtual int step_index() const = 0;
  virtual size_t bytes() const = 0;
  // Resumable state (velocity, frame clock, theta) to / from host bytes.
  virtual int export_state(void *buf, size_t *bytes) = 0;
  virtual int import_state(const void *buf, size_t bytes) = 0;
  // Can these n episodes (this one among them) be stepped as one batch?
  virtual bool batchable_with(EpisodeBase *const *eps, int n) const = 0;
};

// Extruded polar-Bezier scenes: the device table of scene.cuh built from
// the caller's table (nf.h, NF_SCENE_EXTRUDED) and theta, and the per-shape
// offsets. bz_check validates a scene (empty string when valid).
struct BzInfo {
  int n = 0, inside = 0, mode = 0, pulse = 0;
  double period = 0.0;
  int off[4] = {0, 0, 0, 0}, theta0[4] = {0, 0, 0, 0};
  int radii = 0;                 // radii in the table (all shapes and keys)
  const double *dev = nullptr;   // device copy of `table`
  std::vector<double> table;
};
std::string bz_check(const nf_scene &s);
void bz_build(const nf_scene &s, const std::vector<double> &src, BzInfo &out);

// Stacked projections of a batch of same-size episodes (nf_step_batch),
// cached per context by (nx, ny, nz, members).
struct BatchBase {
  virtual ~BatchBase() {}
  virtual size_t bytes() const = 0;
};
using BatchCache = std::map<std::array<int, 4>, std::unique_ptr<BatchBase>>;

// Advances n episodes of one context (same cell counts) by nframes frames
// each; every substep's projections are solved as one stacked system.
// st and status (n entries each, may be null) receive each member's
// statistics and status.
int step_batch(Ctx *ctx, BatchCache &cache, EpisodeBase *const *eps, int n, int nframes,
               nf_step_stats *st, int *status);

// Creates an episode in the precision of ctx->cfg. Returns a status.
int create_episode(Ctx *ctx, const nf_grid *g, const nf_scene *s,
                   EpisodeBase **out);

// Device bytes an episode of this grid would hold before any rollout tape.
size_t episode_base_bytes(const nf_config &cfg, const nf_grid &g);

}  // namespace nf
