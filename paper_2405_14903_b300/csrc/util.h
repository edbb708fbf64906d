// Context, allocation tracking, profiling and error plumbing of libnf (host).
#pragma once

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nf_internal.cuh"

namespace nf {

// Last error message of the calling thread (set by every failing call).
void set_error(const std::string &msg);
const std::string &get_error();
int cuda_fail(cudaError_t e, const char *what);

#define CKS(x)                  \
  do {                          \
    int _s = (x);               \
    if (_s != NF_OK) return _s; \
  } while (0)
#define CKC(x)                                             \
  do {                                                     \
    cudaError_t _e = (x);                                  \
    if (_e != cudaSuccess) return ::nf::cuda_fail(_e, #x); \
  } while (0)

// Event pairs recorded inside a captured graph (external event-record
// nodes around the profiled kernels), tagged with the iteration of the
// captured batch they belong to.
struct GraphEvents {
  std::vector<cudaEvent_t> ev;  // 2 per pair
  std::vector<int> cls, iter;
  void clear();
  ~GraphEvents() { clear(); }
};

// CUDA-event timing of the launches of one kernel class (or all classes).
// Direct launches use event pairs from a fixed pool; a full pool is drained
// (stream synchronised, elapsed times accumulated) and reused. Launches
// inside graphs use the graph's own pairs, read after each replay.
struct Prof {
  int kclass = -2;              // -2 off, -1 every class, else one NF_K_*
  std::vector<cudaEvent_t> ev;  // 2 per slot
  std::vector<int> cls;         // class of each used slot
  size_t used = 0;
  int64_t launches[NF_K_COUNT] = {};
  double ms[NF_K_COUNT] = {};
  GraphEvents *capture_ev = nullptr;  // set while a graph is being captured
  int capture_iter = 0;               // iteration tag of captured launches
  int gen = 0;                        // bumped by nf_profile
  void drain(cudaStream_t s);
  void reset();
  // Add the pairs of a completed replay whose iteration tag is < iters.
  void collect(const GraphEvents &ge, int iters);
  ~Prof();
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  nf_config cfg{};
  RedScratch rs{};
  int64_t launches = 0;
  void *pinned = nullptr;  // small pinned host buffer for status readback
  double *dscal = nullptr; // one device double (diagnostic results)
  size_t bytes_in_use = 0;
  Prof prof;
  cudaStream_t capture = nullptr;  // set while a graph is being captured

  Launch launch() {
    return Launch{capture ? capture : stream, &launches,
                  prof.kclass == -2 ? nullptr : &prof};
  }
  // Synchronous readback of a small device value (synchronises the stream).
  double read_double(const double *dptr);
  void read_bytes(void *host, const void *dev, size_t n);
};

// Device allocations of one owner (an episode), stream-ordered on `stream`
// (the owner's stream: memory is used in that stream's order); freed
// together.
struct Alloc {
  std::vector<void *> ptrs;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  int get(void **p, size_t n);
  template <class P>
  int get(P **p, size_t n) {
    void *v = nullptr;
    int s = get(&v, n);
    *p = (P *)v;
    return s;
  }
  void free_all();
  ~Alloc() { free_all(); }
};

// A named host range for profilers (NVTX: nsys and ncu group the launches
// of a phase under it). Header-only; without an attached tool each range
// costs a pointer test.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace nf
