// qf_fft_step_static: one imaginary-time FFT step on caller-owned device arrays that
// allocates no device memory at all.
//
// Who needs it: code that owns no allocator of its own and may not take device memory
// from anyone else at call time -- a plugin living inside a host application whose
// allocator has already reserved the GPU, a solver loop that must not be able to fail
// with out-of-memory halfway through, or a caller that reaches this library through a
// plain C interface with nothing but raw device pointers.  Such callers cannot size and
// hand over a workspace the way qf_create_lattice requires.
//
// How: the step needs scratch beyond its input and output (the transformed field, the
// per-block partial sums, the twiddle and kinetic tables, a few scalars).  Here that
// scratch is one file-scope __device__ array of fixed size, so it exists on every GPU
// that loads the library, from load until process exit, and the largest lattice is
// capped (N <= 64).  All calls share that one array and it keeps whatever the previous
// call left in it: everything a call reads is written earlier in the same call, and two
// calls whose GPU work overlaps (different streams, or different host threads on the
// same device) race on it.
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/qfdtd.h"
#include "qf_common.cuh"

namespace qf {
namespace {

constexpr int kStaticMaxN = 64;
constexpr size_t kStaticField = (size_t)kStaticMaxN * kStaticMaxN * kStaticMaxN * sizeof(cpx<float>);  // 2 MiB
constexpr size_t kStaticPartialsOff = kStaticField;
constexpr size_t kStaticPartialsBytes = 64 * 1024;  // >= blocks of the reducing pass x 8 doubles
constexpr size_t kStaticTwOff = kStaticPartialsOff + kStaticPartialsBytes;
constexpr size_t kStaticTwBytes = 2 * sizeof(float) * kStaticMaxN;
constexpr size_t kStaticSymOff = kStaticTwOff + 1024;
constexpr size_t kStaticSymBytes = sizeof(float) * kStaticMaxN;
constexpr size_t kStaticScOff = kStaticSymOff + 1024;
constexpr size_t kStaticBytes = kStaticScOff + 1024;
static_assert(kStaticTwBytes <= 1024 && kStaticSymBytes <= 1024 && sizeof(DevScalars) <= 1024, "layout");

// The scratch itself.  In host code this name is only a handle for the runtime, not an
// address a kernel may use: kernels get the device address from cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Per-call tables, passed by value in the kernel's parameter space and written into the
// scratch array on the device: no host buffer has to outlive the call.
struct StaticTables {
  float tw[2 * kStaticMaxN];  // per-stage twiddles (re, im), fft_twiddle_count(n) pairs
  float sym[kStaticMaxN];     // per-axis kinetic symbol
  double out_scale;
  int tw_count, n;
};

__global__ void static_tables_kernel(const __grid_constant__ StaticTables t, float* tw, float* sym,
                                     DevScalars* sc) {
  for (int i = threadIdx.x; i < 2 * t.tw_count; i += blockDim.x) tw[i] = t.tw[i];
  for (int i = threadIdx.x; i < t.n; i += blockDim.x) sym[i] = t.sym[i];
  if (threadIdx.x == 0) {
    DevScalars z{};
    z.scale[0] = t.out_scale;
    z.scale[1] = t.out_scale;
    *sc = z;
  }
}

}  // namespace
}  // namespace qf

using namespace qf;

extern "C" qf_status qf_fft_step_static(int n, double a, int kinetic, double mass, double dtau, void* psi,
                                        const void* v, int v_complex, double out_scale, double* sums,
                                        void* cuda_stream) {
  if (n < 8 || n > kStaticMaxN || !fft_supported(n)) return QF_EINVAL;
  if (kinetic < QF_KIN_FFT_NAIVE || kinetic > QF_KIN_FFT_REL) return QF_EINVAL;
  if (!(a > 0) || !(mass > 0) || !(dtau > 0) || !isfinite(out_scale) || !psi || !v) return QF_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* base_v = nullptr;
  if (scratch_address(&base_v) != cudaSuccess) return QF_ECUDA;
  char* base = static_cast<char*>(base_v);

  // tables of this call (the array holds the previous call's): per-stage twiddles, the
  // per-axis symbol and the output scale, written on the device by the first launch
  StaticTables tab{};
  double twd[2 * kStaticMaxN];
  const int cnt = fft_twiddle_count(n);
  fft_twiddles(n, twd);
  for (int i = 0; i < 2 * cnt; ++i) tab.tw[i] = (float)twd[i];
  for (int j = 0; j < n; ++j) {
    const double k = 2.0 * M_PI * (double)(j <= n / 2 ? j : j - n) / (double)n;
    tab.sym[j] = (float)(kinetic == QF_KIN_FFT_NAIVE ? k * k : 4.0 * sin(0.5 * k) * sin(0.5 * k));
  }
  tab.out_scale = out_scale;
  tab.tw_count = cnt;
  tab.n = n;
  float* tw_dev = reinterpret_cast<float*>(base + kStaticTwOff);
  float* sym_dev = reinterpret_cast<float*>(base + kStaticSymOff);
  DevScalars* sc_dev = reinterpret_cast<DevScalars*>(base + kStaticScOff);
  void* targs[] = {&tab, &tw_dev, &sym_dev, &sc_dev};
  // (cudaLaunchKernel returns this launch's own status, not an earlier error of the thread)
  if (cudaLaunchKernel((const void*)static_tables_kernel, dim3(1), dim3(128), targs, 0, st) != cudaSuccess)
    return QF_ECUDA;

  DevScalars* dsc = reinterpret_cast<DevScalars*>(base + kStaticScOff);
  double* partials = reinterpret_cast<double*>(base + kStaticPartialsOff);
  const double n3 = (double)n * n * n;
  FftPassArgs<float> p{};
  p.twiddle = reinterpret_cast<const cpx<float>*>(base + kStaticTwOff);
  p.symbol = reinterpret_cast<const float*>(base + kStaticSymOff);
  p.kinetic = kinetic;
  p.tcoef = (float)(kinetic == QF_KIN_FFT_REL ? 1.0 / (a * n3) : 1.0 / (2.0 * a * a * mass * n3));
  p.am2 = (float)((a * mass) * (a * mass));
  p.psi = static_cast<cpx<float>*>(psi);
  p.v = v;
  p.v_real = v_complex ? 0 : 1;
  p.half_dtau = (float)(0.5 * dtau);
  p.dtau = (float)dtau;
  p.scale = &dsc->scale[0];
  p.partials = partials;
  p.write_psi = 1;
  p.reduce = sums ? 1 : 0;
  cpx<float>* tmp = reinterpret_cast<cpx<float>*>(base);
  int nb = 0;
  for (int pass = 0; pass < kFftPasses; ++pass)
    // (its twiddle scratch holds the first radix plan's table only)
    if (launch_fft_pass<float>(n, pass, p, tmp, st, &nb, false) != cudaSuccess) return QF_ECUDA;
  if (sums) {
    if (launch_finish(partials, nb, dsc, 0, st) != cudaSuccess) return QF_ECUDA;
    if (cudaMemcpyAsync(sums, dsc->sums, kNumSums * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return QF_ECUDA;
  }
  return QF_OK;
}
