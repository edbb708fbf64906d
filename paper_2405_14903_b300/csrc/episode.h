// Episode: one simulated grid with its scene, fields, solver hierarchy and
// rollout tape. Precision-specific implementations live in episode.cu.
#pragma once

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
};

// Creates an episode in the precision of ctx->cfg. Returns a status.
int create_episode(Ctx *ctx, const nf_grid *g, const nf_scene *s,
                   EpisodeBase **out);

// Device bytes an episode of this grid would hold before any rollout tape.
size_t episode_base_bytes(const nf_config &cfg, const nf_grid &g);

}  // namespace nf
