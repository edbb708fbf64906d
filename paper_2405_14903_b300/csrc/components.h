// Connected fluid components of an episode's active cells and the zero-mean
// gauge of the components without an open face (k_components.cu).
#pragma once

#include "kernels.h"
#include "util.h"

namespace nf {

struct Components {
  int *lab = nullptr;      // root cell of each active cell, -1 if inactive
  int *ground = nullptr;   // per root: 1 if the component has an open face
  int *ccnt = nullptr;     // per root: cell count (gauge scratch)
  unsigned long long *csum = nullptr;  // per root: fixed-point sum
  void *scal = nullptr;    // [1] floating count, +16 max, +24 norm
  int nfloat = 0;          // floating components found by the last label()

  int init(Alloc &A, int64_t ncell);
  // Label the components of the cells with sum alpha > 0 and find those
  // with an open face. Synchronises the stream once (the floating count).
  template <class T>
  int label(Ctx *ctx, const GridDev &g, Fields<T> alpha);
  // Shift v to zero mean on every floating component; returns ||v||^2
  // afterwards (or norm2 unchanged when nothing floats).
  template <class S>
  double gauge(Ctx *ctx, int64_t n, S *v, double norm2);
};

}  // namespace nf
