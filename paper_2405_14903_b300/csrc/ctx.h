// The nf_ctx handle of the C ABI: a device context (stream, reduction
// scratch, profiler) and the episodes created in it.
#pragma once

#include <map>
#include <memory>

#include "episode.h"
#include "util.h"

struct nf_ctx {
  nf::Ctx c;
  std::map<int64_t, std::unique_ptr<nf::EpisodeBase>> eps;
  nf::BatchCache batches;  // stacked solvers of nf_step_batch
  int64_t next_id = 1;
};
