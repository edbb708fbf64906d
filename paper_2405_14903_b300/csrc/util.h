// Context, allocation tracking, profiling and error plumbing of libnf (host).
#pragma once

#include <string>
#include <vector>

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

// CUDA-event timing of the launches of one kernel class (or all classes).
// Event pairs come from a fixed pool; a full pool is drained (stream
// synchronised, elapsed times accumulated) and reused.
struct Prof {
  int kclass = -2;              // -2 off, -1 every class, else one NF_K_*
  std::vector<cudaEvent_t> ev;  // 2 per slot
  std::vector<int> cls;         // class of each used slot
  size_t used = 0;
  int64_t launches[NF_K_COUNT] = {};
  double ms[NF_K_COUNT] = {};
  void drain(cudaStream_t s);
  void reset();
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
  size_t bytes_in_use = 0;
  Prof prof;

  Launch launch() {
    return Launch{stream, &launches, prof.kclass == -2 ? nullptr : &prof};
  }
  // Synchronous readback of a small device value (synchronises the stream).
  double read_double(const double *dptr);
  void read_bytes(void *host, const void *dev, size_t n);
};

// Device allocations of one owner (an episode); freed together.
struct Alloc {
  std::vector<void *> ptrs;
  size_t bytes = 0;
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

}  // namespace nf
