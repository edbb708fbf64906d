// Check of the integer-bit conversions between FP32 and FP64 (f2d, d2f of
// nf_internal.cuh) against the conversion instructions, for nf_check_conversions.
#include "kernels.h"

namespace nf {

__global__ void k_check_conversions(const double *in, int64_t n, float *out_f, double *out_d,
                                    unsigned long long *mismatches) {
  unsigned long long bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = in[i];
    const float a = d2f(v), r = __double2float_rn(v);
    const bool same_f = __float_as_uint(a) == __float_as_uint(r) || (isnan(a) && isnan(r));
    const double wa = f2d(r), wr = (double)r;
    const bool same_d =
        __double_as_longlong(wa) == __double_as_longlong(wr) || (isnan(wa) && isnan(wr));
    out_f[i] = a;
    out_d[i] = wa;
    bad += (same_f && same_d) ? 0ull : 1ull;
  }
  if (bad) atomicAdd(mismatches, bad);
}

void launch_check_conversions(const Launch &L, const double *in, int64_t n, float *out_f,
                              double *out_d, unsigned long long *mismatches) {
  const int64_t want = (n + kBlock - 1) / kBlock;
  const unsigned nb = (unsigned)(want < 1 ? 1 : (want > 4096 ? 4096 : want));
  k_check_conversions<<<nb, kBlock, 0, L.s>>>(in, n, out_f, out_d, mismatches);
  ++*L.counter;
}

}  // namespace nf
