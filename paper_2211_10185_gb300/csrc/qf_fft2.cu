// Launchers of the two-pass FFT step for N = 256 complex-FP32 lattices (kernels in
// qf_fft2.cuh).  Every launch is a group (blockIdx.y = member); a lone lattice is a group
// of one, so it runs the same machine code alone and in a batch.
#include "qf_fft2.cuh"

namespace qf {

// y_lo values per pass-A/C block: 2 makes each block's scratch accesses whole 32-byte
// sectors (1 measured 12 % slower per step)
constexpr int kF2YL = 2;

bool fft2_supported(int n) { return n == F2_N; }
int fft2_final_blocks() { return F2AC<kF2YL>::BLOCKS; }
// partial rows of a measure (passes 3 and 4): pass A rows, then pass B rows
int fft2_measure_blocks() { return F2AC<kF2YL>::BLOCKS + F2_BLOCKS; }

template <int OP, bool VREAL, bool NEXT>
static void f2_attr_c() {
  cudaFuncSetAttribute(fft2_c_kernel<kF2YL, OP, VREAL, NEXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)F2AC<kF2YL>::SMEM);
}

// pass 0: natural field -> S (members' src); 1: S in place; 2: S -> update / sums (+ the
// next step's pass 0 when emit_next).  The pass-2 variant follows member 0.  Energy of a
// field that is not stepped: 3 = pass 0 with <v|v>, <v|V v> sums, 4 = forward half of
// pass 1 with the k-space <v|H_K v> sums (nothing written back).
cudaError_t launch_fft2_group_pass(int pass, const FftGroup<float>& g, cudaStream_t st) {
  using AC = F2AC<kF2YL>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(fft2_a_kernel<kF2YL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AC::SMEM);
    cudaFuncSetAttribute(fft2_a_kernel<kF2YL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AC::SMEM);
    cudaFuncSetAttribute(fft2_b_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F2_SMEM_B);
    cudaFuncSetAttribute(fft2_b_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F2_SMEM_B);
    f2_attr_c<OP_FINAL, true, true>();
    f2_attr_c<OP_FINAL, true, false>();
    f2_attr_c<OP_FINAL, false, true>();
    f2_attr_c<OP_FINAL, false, false>();
    f2_attr_c<OP_FINAL_SUMS, true, true>();
    f2_attr_c<OP_FINAL_SUMS, true, false>();
    f2_attr_c<OP_FINAL_SUMS, false, true>();
    f2_attr_c<OP_FINAL_SUMS, false, false>();
    f2_attr_c<OP_SUMS, true, false>();
    f2_attr_c<OP_SUMS, false, false>();
    attr_done = true;
  }
  if (g.count < 1 || g.count > kGroupMax) return cudaErrorInvalidValue;
  const dim3 grid_b(F2_BLOCKS, g.count), grid_ac(AC::BLOCKS, g.count);
  const bool vreal = g.a[0].v_real != 0, sums = g.a[0].reduce != 0, write = g.a[0].write_psi != 0;
  const bool next = write && g.a[0].emit_next != 0;
  switch (pass) {
    case 0: fft2_a_kernel<kF2YL, false><<<grid_ac, AC::THREADS, AC::SMEM, st>>>(g); break;
    case 1: fft2_b_kernel<false><<<grid_b, F2_THREADS, F2_SMEM_B, st>>>(g, 0); break;
    case 3: fft2_a_kernel<kF2YL, true><<<grid_ac, AC::THREADS, AC::SMEM, st>>>(g); break;
    case 4: fft2_b_kernel<true><<<grid_b, F2_THREADS, F2_SMEM_B, st>>>(g, AC::BLOCKS); break;
    case 2:
#define F2_C(OP, VR, NX) fft2_c_kernel<kF2YL, OP, VR, NX><<<grid_ac, AC::THREADS, AC::SMEM, st>>>(g)
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
  return cudaGetLastError();
}

}  // namespace qf
