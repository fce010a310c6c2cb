// Complex-FP32 four-pass kernels with tile variant 1 (half-size tiles, more blocks per
// SM), grouped launches; selected per N by the autotuner.  Compiled apart from variant 0
// (qf_fft_group.cu) so the two build in parallel.
#include "qf_fft_impl.cuh"

namespace qf {

cudaError_t launch_fft_group_pass_t1(int n, int pass, const FftGroup<float>& g, cudaStream_t st) {
  switch (n) {
#define QF_CASE(NN) \
  case NN:          \
    return group_pass_n<float, NN, 1>(pass, g, st);
    QF_CASE(8) QF_CASE(12) QF_CASE(16) QF_CASE(24) QF_CASE(32) QF_CASE(48) QF_CASE(64) QF_CASE(96)
    QF_CASE(128) QF_CASE(192) QF_CASE(256) QF_CASE(384) QF_CASE(512)
#undef QF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace qf
