// FDTD kinetic step (Eq. HK0) fused with the imaginary-time update: launchers of the
// TMA-staged kernel in qf_stencil_tma.cuh.
//
// (H_K^(0) psi)(r) = -1/(2 m a^2) sum over the six neighbours of (psi(nbr) - psi(r)), with
// psi pinned to 0 on the Dirichlet planes (any index 0; a neighbour index N wraps onto
// the plane 0).  One pass: read psi and V, write psi' = s (coef_A psi - coef_B dtau H psi)
// into the other buffer, plus the FP64 partial sums of <psi|psi>, <psi|H_K psi>,
// <psi|V psi> on check steps.  A lone lattice is a group of one, so it runs the same
// code alone and inside a batch.
#include <cudaTypedefs.h>

#include <mutex>

#include "qf_stencil_tb.cuh"

namespace qf {

// Partial-sum rows of one launch with z-chunk zc (the most over all chunks when zc <= 0).
template <typename R>
int stencil_blocks(int n, int zc) {
  if (zc <= 0) zc = kStencilZChunkMin;
  return stencil_member_blocks(n, zc);
}

template <typename R>
cudaError_t launch_stencil_tma(const StencilTmaGroup<R>& g, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(stencil_tma_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)stencil_tma_smem<R>());
    attr = true;
  }
  if (g.count < 1 || g.count > kGroupMax) return cudaErrorInvalidValue;
  // the block table: member i's blocks follow member i-1's
  StencilTmaGroup<R> gl = g;
  long long total = 0;
  for (int i = 0; i < g.count; ++i) {
    if (g.zcm[i] < 1 || g.nm[i] < 2) return cudaErrorInvalidValue;
    gl.start[i] = (int)total;
    total += stencil_member_blocks(g.nm[i], g.zcm[i]);
  }
  if (total > (1LL << 30)) return cudaErrorInvalidValue;
  gl.start[g.count] = (int)total;
  stencil_tma_kernel<R><<<(unsigned)total, dim3(TS_X, TS_Y / TS_ROWS), stencil_tma_smem<R>(), st>>>(gl);
  return cudaGetLastError();
}

cudaError_t launch_stencil_tb(const StencilTbArgs& g, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(stencil_tb_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stencil_tb_smem());
    cudaFuncSetAttribute(stencil_tb_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)stencil_tb_smem());
    attr = true;
  }
  const int n = g.n;
  if (g.nzb < 1 || g.nzb > n) return cudaErrorInvalidValue;
  dim3 grid((n + TB_X - 1) / TB_X, (n + TB_Y - 1) / TB_Y, g.nzb);
  if (g.v_real) stencil_tb_kernel<true><<<grid, TB_THREADS, stencil_tb_smem(), st>>>(g);
  else stencil_tb_kernel<false><<<grid, TB_THREADS, stencil_tb_smem(), st>>>(g);
  return cudaGetLastError();
}

// Two steps for every member of g (any sizes, one kind of potential) in one launch.
cudaError_t launch_stencil_tb_group(const StencilTbGroup& g, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(stencil_tb_group_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)stencil_tb_smem());
    cudaFuncSetAttribute(stencil_tb_group_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)stencil_tb_smem());
    attr = true;
  }
  if (g.count < 1 || g.count > kGroupMax) return cudaErrorInvalidValue;
  StencilTbGroup gl = g;
  long long total = 0;
  for (int i = 0; i < g.count; ++i) {
    const StencilTbArgs& m = g.m[i];
    if (m.n < 2 || m.nzb < 1 || m.nzb > m.n || m.v_real != g.m[0].v_real) return cudaErrorInvalidValue;
    gl.start[i] = (int)total;
    total += stencil_tb_member_blocks(m.n, m.nzb);
  }
  if (total > (1LL << 30)) return cudaErrorInvalidValue;
  gl.start[g.count] = (int)total;
  if (g.m[0].v_real) stencil_tb_group_kernel<true><<<(unsigned)total, TB_THREADS, stencil_tb_smem(), st>>>(gl);
  else stencil_tb_group_kernel<false><<<(unsigned)total, TB_THREADS, stencil_tb_smem(), st>>>(gl);
  return cudaGetLastError();
}

// Tensor map of an N^3 complex field for plane boxes of box_w x box_h 8-byte elements
// (one complex FP32 or one FP64 component).
static bool encode_field_map(CUtensorMap* map, void* field, int n, bool c64, unsigned box_w, unsigned box_h) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!encode) return false;
  const cuuint64_t w = c64 ? (cuuint64_t)n : 2 * (cuuint64_t)n;
  const cuuint64_t dims[3] = {w, (cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t strides[2] = {w * 8, w * 8 * (cuuint64_t)n};
  const cuuint32_t box[3] = {box_w, box_h, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(map, c64 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, field,
                            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// boxes of the single-step kernel: the tile plus a one-site halo (x rounded to 16 bytes)
bool encode_stencil_map(CUtensorMap* map, void* field, int n, bool c64) {
  return encode_field_map(map, field, n, c64, c64 ? TmaTile<float>::W : TmaTile<double>::W, TS_Y + 2);
}

// boxes of the two-step kernel (complex FP32): the tile plus a two-site halo
bool encode_tb_map(CUtensorMap* map, void* field, int n) { return encode_field_map(map, field, n, true, TB_W0, TB_H0); }

// Self-test of the bounded waits: an mbarrier that expects bytes nobody sends never
// completes, so every thread's bounded wait runs out and the block reports it.
__global__ void bounded_wait_probe(int* err) {
  __shared__ alignas(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    mbar_expect_tx(&bar, 16);  // no copy follows
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0);
  if (__syncthreads_and(ok) == 0 && threadIdx.x == 0) atomicExch(err, 1);
}

cudaError_t launch_bounded_wait_probe(int* err, cudaStream_t st) {
  bounded_wait_probe<<<1, 32, 0, st>>>(err);
  return cudaGetLastError();
}

template int stencil_blocks<float>(int, int);
template int stencil_blocks<double>(int, int);
template cudaError_t launch_stencil_tma<float>(const StencilTmaGroup<float>&, cudaStream_t);
template cudaError_t launch_stencil_tma<double>(const StencilTmaGroup<double>&, cudaStream_t);

}  // namespace qf
