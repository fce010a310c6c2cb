// The two-pass FFT step for N = 128 lattices (kernels in qf_fft2.cuh).
#include "qf_fft2_launch.cuh"

namespace qf {

template cudaError_t launch_fft2_pass_n<128>(int, const FftGroup<float>&, cudaStream_t);

}  // namespace qf
