// Launcher of the two-pass FFT step's passes for one lattice size N (kernels in
// qf_fft2.cuh).  Every launch is a group (blockIdx.y = member); a lone lattice is a group
// of one, so it runs the same machine code alone and in a batch.
#pragma once
#include "qf_fft2.cuh"

namespace qf {

template <int N, int OP, bool VREAL, bool NEXT>
static void f2_attr_c() {
  cudaFuncSetAttribute(fft2_c_kernel<N, OP, VREAL, NEXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)F2G<N>::SMEM_AC);
}

template <int N>
static bool f2_set_attrs() {
  using G = F2G<N>;
  cudaFuncSetAttribute(fft2_a_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_AC);
  cudaFuncSetAttribute(fft2_a_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_AC);
  cudaFuncSetAttribute(fft2_b_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_B);
  cudaFuncSetAttribute(fft2_b_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_B);
  f2_attr_c<N, OP_FINAL, true, true>();
  f2_attr_c<N, OP_FINAL, true, false>();
  f2_attr_c<N, OP_FINAL, false, true>();
  f2_attr_c<N, OP_FINAL, false, false>();
  f2_attr_c<N, OP_FINAL_SUMS, true, true>();
  f2_attr_c<N, OP_FINAL_SUMS, true, false>();
  f2_attr_c<N, OP_FINAL_SUMS, false, true>();
  f2_attr_c<N, OP_FINAL_SUMS, false, false>();
  f2_attr_c<N, OP_SUMS, true, false>();
  f2_attr_c<N, OP_SUMS, false, false>();
  return true;
}

// Launch with or without programmatic stream serialization (the kernels wait for the
// previous kernel before their first dependent read: f2_grid_dependency).
template <typename... KArgs, typename... Args>
static cudaError_t f2_launch(void (*kern)(KArgs...), dim3 grid, int threads, size_t smem, cudaStream_t st, bool pdl,
                             Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Steady-state passes B and C start during the previous pass's last wave at N = 256
// (measured 218 -> 211 us per B + C in a CUDA graph); at N = 128 both grids fit one
// wave and early blocks only take slots (26.0 -> 27.0 us), so it stays off there.
template <int N>
constexpr bool kF2Pdl = N == 256;

// pass 0: natural field -> S (members' src); 1: S in place; 2: S -> update / sums (+ the
// next step's pass 0 when emit_next).  The pass-2 variant follows member 0.  Energy of a
// field that is not stepped: 3 = pass 0 with <v|v>, <v|V v> sums, 4 = forward half of
// pass 1 with the k-space <v|H_K v> sums (nothing written back).
template <int N>
cudaError_t launch_fft2_pass_n(int pass, const FftGroup<float>& g, cudaStream_t st) {
  using G = F2G<N>;
  static const bool attrs = f2_set_attrs<N>();
  (void)attrs;
  if (g.count < 1 || g.count > kGroupMax) return cudaErrorInvalidValue;
  const dim3 grid_b(G::B_BLOCKS, g.count), grid_ac(G::AC_BLOCKS, g.count);
  const bool vreal = g.a[0].v_real != 0, sums = g.a[0].reduce != 0, write = g.a[0].write_psi != 0;
  const bool next = write && g.a[0].emit_next != 0;
  cudaError_t e = cudaSuccess;
  switch (pass) {
    case 0: fft2_a_kernel<N, false><<<grid_ac, G::AC_THREADS, G::SMEM_AC, st>>>(g); break;
    case 1: e = f2_launch(fft2_b_kernel<N, false>, grid_b, G::B_THREADS, G::SMEM_B, st, kF2Pdl<N>, g, 0); break;
    case 3: fft2_a_kernel<N, true><<<grid_ac, G::AC_THREADS, G::SMEM_AC, st>>>(g); break;
    case 4: fft2_b_kernel<N, true><<<grid_b, G::B_THREADS, G::SMEM_B, st>>>(g, G::AC_BLOCKS); break;
    case 2:
#define F2_C(OP, VR, NX) \
  e = f2_launch(fft2_c_kernel<N, OP, VR, NX>, grid_ac, G::AC_THREADS, G::SMEM_AC, st, kF2Pdl<N>, g)
      if (!write) {
        if (vreal) F2_C(OP_SUMS, true, false);
        else F2_C(OP_SUMS, false, false);
      } else if (sums) {
        if (vreal) { if (next) F2_C(OP_FINAL_SUMS, true, true); else F2_C(OP_FINAL_SUMS, true, false); }
        else { if (next) F2_C(OP_FINAL_SUMS, false, true); else F2_C(OP_FINAL_SUMS, false, false); }
      } else {
        if (vreal) { if (next) F2_C(OP_FINAL, true, true); else F2_C(OP_FINAL, true, false); }
        else { if (next) F2_C(OP_FINAL, false, true); else F2_C(OP_FINAL, false, false); }
      }
#undef F2_C
      break;
    default: return cudaErrorInvalidValue;
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace qf
