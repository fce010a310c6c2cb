// Grouped (many lattices per launch) complex FP32 instantiation of the fused FFT step;
// the kernels are in qf_fft_impl.cuh.
#include "qf_fft_impl.cuh"

namespace qf {

template cudaError_t launch_fft_group_pass<float>(int, int, const FftGroup<float>&, cudaStream_t);

}  // namespace qf
