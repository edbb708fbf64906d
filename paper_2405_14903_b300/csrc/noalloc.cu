// nf_loss_noalloc: the loss reduction of nf_loss on a caller's velocity with
// its scratch in a file-scope device array instead of context memory. Nothing
// here allocates: no cudaMalloc/cudaFree, no host or device pools.
#include <mutex>

#include "kernels.h"
#include "util.h"

namespace nf {
namespace {

// Layout of the scratch: kRedBlocks block partials (one double each), the
// reduction's ticket counter, the result.
constexpr size_t kPartialBytes = sizeof(double) * kRedBlocks;
constexpr size_t kTicketOff = 4864;
constexpr size_t kResultOff = 4992;
static_assert(kPartialBytes <= kTicketOff, "partials overlap the ticket");
static_assert(kTicketOff + sizeof(unsigned int) <= kResultOff, "ticket overlaps the result");
static_assert(kResultOff + sizeof(double) <= NF_NOALLOC_SCRATCH_BYTES, "scratch too small");

__device__ __align__(256) unsigned char g_scratch[NF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once).
int scratch_address(void **out) {
  int dev = 0;
  CKC(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("nf_loss_noalloc: device index out of range");
    return NF_E_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    CKC(cudaGetSymbolAddress(&p, g_scratch));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NF_OK;
}

int invalid(const char *msg) {
  set_error(std::string("nf_loss_noalloc: ") + msg);
  return NF_E_INVALID;
}

// Device (or managed) memory of device `dev`, the device the call runs on:
// a pointer into another GPU's memory would be dereferenced by this
// device's kernel.
bool on_device(const void *p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of the query
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == dev;
  return a.type == cudaMemoryTypeManaged;
}

template <class T>
int run(const GridDev &g, int kind, const void *const u[3], void *const gU[3],
        double *J, cudaStream_t s, void *scratch) {
  char *base = (char *)scratch;
  RedScratch rs{(double *)base, (unsigned int *)(base + kTicketOff)};
  double *res = (double *)(base + kResultOff);
  CKC(cudaMemsetAsync(rs.ticket, 0, sizeof(unsigned int), s));
  int64_t launches = 0;
  Launch L{s, &launches, nullptr};
  Fields<T> uf{(const T *)u[0], (const T *)u[1], (const T *)u[2]};
  FieldsMut<T> gf{gU ? (T *)gU[0] : nullptr, gU ? (T *)gU[1] : nullptr,
                  gU ? (T *)gU[2] : nullptr};
  launch_loss<T>(L, g, kind, uf, gf, gU != nullptr, rs, res);
  CKC(cudaGetLastError());
  CKC(cudaMemcpyAsync(J, res, sizeof(double), cudaMemcpyDeviceToHost, s));
  CKC(cudaStreamSynchronize(s));
  return NF_OK;
}

}  // namespace
}  // namespace nf

extern "C" int nf_loss_noalloc(const nf_grid *gr, int loss_kind,
                               const void *const u[3], void *const gU[3],
                               int dtype, double *J, void *stream) {
  using namespace nf;
  if (!gr || !u || !J) return invalid("null argument");
  if (dtype != NF_F32 && dtype != NF_F64) return invalid("dtype must be NF_F32 or NF_F64");
  if (loss_kind != NF_LOSS_KINETIC && loss_kind != NF_LOSS_OUTFLOW)
    return invalid("unknown loss kind");
  if (gr->nx < 1 || gr->ny < 1 || gr->nz < 1 || !(gr->dx > 0.0))
    return invalid("grid needs nx, ny, nz >= 1 and dx > 0");
  GridDev g{};
  g.nx = gr->nx;
  g.ny = gr->ny;
  g.nz = gr->nz;
  g.dx = gr->dx;
  g.dt = gr->dt;
  g.rho = gr->rho > 0 ? gr->rho : 1.0;
  g.c = 0.0;
  g.outlet = gr->outlet;
  g.oj0 = gr->outlet_j0;
  g.ok0 = gr->outlet_k0;
  g.ow = gr->outlet_w;
  g.oh = gr->outlet_h;
  g.set_derived();
  for (int d = 0; d < 3; ++d)
    if (g.nface(d) > NF_NOALLOC_MAX_FACES)
      return invalid("grid too large: a face component exceeds NF_NOALLOC_MAX_FACES entries");
  if (loss_kind == NF_LOSS_OUTFLOW &&
      (!g.outlet || g.ow < 1 || g.oh < 1 || g.oj0 < 0 || g.ok0 < 0 ||
       g.oj0 + g.ow > g.ny || g.ok0 + g.oh > g.nz))
    return invalid("outflow loss needs an outlet patch inside the high-x wall");
  int dev = 0;
  CKC(cudaGetDevice(&dev));
  for (int d = 0; d < 3; ++d) {
    if (!u[d] || !on_device(u[d], dev))
      return invalid("u must be three device arrays of the current device");
    if (gU && (!gU[d] || !on_device(gU[d], dev)))
      return invalid("gU must be NULL or three device arrays of the current device");
  }
  void *scratch = nullptr;
  CKS(scratch_address(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == NF_F64 ? run<double>(g, loss_kind, u, gU, J, s, scratch)
                         : run<float>(g, loss_kind, u, gU, J, s, scratch);
}
