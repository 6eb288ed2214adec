// Checks the setup stage's correctly rounded quotient (div_rn_by: a / w from the correctly
// rounded reciprocal of w, by Markstein's correction) against the IEEE division __fdiv_rn,
// bit for bit. Test code: compiled by tests/test_gpu_division.py.
#include "lr_common.cuh"

namespace {

// For every mantissa of w in [1, 2) scaled by 2^w_exp: every numerator in as[0, na).
__global__ void k_div_check(const float* as, int na, int w_exp, unsigned long long* mismatches,
                            unsigned long long* first) {
  const unsigned m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (1u << 23)) return;
  const float w = ldexpf(__uint_as_float(0x3f800000u | m), w_exp);
  const float y = __frcp_rn(w);
  unsigned long long bad = 0;
  for (int i = 0; i < na; ++i) {
    const float a = as[i];
    const float got = lr::div_rn_by(a, w, y), want = __fdiv_rn(a, w);
    if (__float_as_uint(got) != __float_as_uint(want)) {
      ++bad;
      atomicCAS(first, 0ull, ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(w));
    }
  }
  if (bad) atomicAdd(mismatches, bad);
}

}  // namespace

extern "C" int lr_test_div_check(const float* as, int na, int w_exp, unsigned long long* mismatches,
                                 unsigned long long* first) {
  k_div_check<<<(1 << 23) / 256, 256>>>(as, na, w_exp, mismatches, first);
  return (int)cudaGetLastError();
}
