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
  int *fslot = nullptr;    // per floating root: its slot 0..nfloat-1
  int *fcnt = nullptr;     // per slot: cells of the floating component
  unsigned long long *fsum = nullptr;  // per slot: fixed-point sum (project)
  void *scal = nullptr;    // [1] floating count, +16 max, +24 norm, +32 max
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
  // The same zero-mean projection without a readback, for use inside a
  // captured solver graph: the kernels read the floating count on the device
  // and do nothing when no component floats.
  template <class V>
  void project(const Launch &L, int64_t n, V *v);
};

}  // namespace nf
