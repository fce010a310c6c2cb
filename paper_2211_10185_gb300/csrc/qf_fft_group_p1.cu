// Complex-FP32 four-pass kernels with the second radix plan (tile variants 2 and 3: the
// plan's first stage is radix 16 with 16 elements per thread), grouped launches, for the
// sizes that have one; selected per N by the autotuner.  Compiled apart from variants 0
// and 1 so the three build in parallel.
#include "qf_fft_impl.cuh"

namespace qf {

// Every radix plan the library compiles: the radices multiply to N, each divides the
// elements per thread, and the per-stage twiddle table has N - 1 entries (the sizes
// the lattice workspaces and the allocation-free scratch reserve).
constexpr bool plan_valid(int n, int p) {
  int prod = 1;
  for (int s = 0; s < plan_stages(n, p); ++s) {
    const int r = plan_radix(n, s, p);
    if (r < 2 || plan_ept(n, p) % r != 0) return false;
    prod *= r;
  }
  return plan_stages(n, p) > 0 && prod == n && plan_tw_size(n, p) == n - 1;
}
constexpr bool all_plans_valid() {
  constexpr int sizes[] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512};
  for (int n : sizes) {
    if (!plan_valid(n, 0)) return false;
    if (has_alt_plan(n) && (!plan_valid(n, 1) || plan_ept(n, 1) != 16 || plan_radix(n, 0, 1) != 16)) return false;
  }
  return true;
}
static_assert(all_plans_valid(), "radix plans");

template <int N>
static cudaError_t p1_pass(int variant, int pass, const FftGroup<float>& g, cudaStream_t st) {
  static_assert(has_alt_plan(N), "no second plan for this size");
  // the second plan's table follows the first in every member's twiddle region
  FftGroup<float> gp = g;
  for (int i = 0; i < gp.count; ++i) gp.a[i].twiddle += plan_tw_size(N, 0);
  return variant == 2 ? group_pass_n<float, N, 2>(pass, gp, st) : group_pass_n<float, N, 3>(pass, gp, st);
}

cudaError_t launch_fft_group_pass_p1(int n, int variant, int pass, const FftGroup<float>& g, cudaStream_t st) {
  if (variant != 2 && variant != 3) return cudaErrorInvalidValue;
  if (g.count < 0 || g.count > kGroupMax) return cudaErrorInvalidValue;
  switch (n) {
    case 32: return p1_pass<32>(variant, pass, g, st);
    case 64: return p1_pass<64>(variant, pass, g, st);
    case 512: return p1_pass<512>(variant, pass, g, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qf
