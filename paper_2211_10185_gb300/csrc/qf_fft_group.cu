// Complex-FP32 instantiation of the fused FFT step: grouped launches (many lattices per
// launch) and single lattices, which run the same grouped kernels with one member.
#include "qf_fft_impl.cuh"

namespace qf {

template cudaError_t launch_fft_group_pass<float>(int, int, const FftGroup<float>&, cudaStream_t, bool);
template cudaError_t launch_fft_pass<float>(int, int, FftPassArgs<float>, cpx<float>*, cudaStream_t, int*, bool);

}  // namespace qf
