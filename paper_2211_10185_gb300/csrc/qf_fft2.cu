// The two-pass FFT step for N = 256 (the N = 128 instantiation is in qf_fft2_n128.cu, a
// translation unit of its own so that the two compile in parallel), and the size dispatch.
#include "qf_fft2_launch.cuh"

namespace qf {

template cudaError_t launch_fft2_pass_n<256>(int, const FftGroup<float>&, cudaStream_t);
extern template cudaError_t launch_fft2_pass_n<128>(int, const FftGroup<float>&, cudaStream_t);

bool fft2_supported(int n) { return n == 128 || n == 256; }
int fft2_final_blocks(int n) { return n == 128 ? F2G<128>::AC_BLOCKS : F2G<256>::AC_BLOCKS; }
// partial rows of a measure (passes 3 and 4): pass A rows, then pass B rows
int fft2_measure_blocks(int n) {
  return n == 128 ? F2G<128>::AC_BLOCKS + F2G<128>::B_BLOCKS : F2G<256>::AC_BLOCKS + F2G<256>::B_BLOCKS;
}

cudaError_t launch_fft2_group_pass(int n, int pass, const FftGroup<float>& g, cudaStream_t st) {
  if (n == 256) return launch_fft2_pass_n<256>(pass, g, st);
  if (n == 128) return launch_fft2_pass_n<128>(pass, g, st);
  return cudaErrorInvalidValue;
}

}  // namespace qf
