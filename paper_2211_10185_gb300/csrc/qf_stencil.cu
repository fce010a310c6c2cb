// FDTD kinetic step (Eq. HK0) fused with the imaginary-time update, sm_103a.
//
// (H_K^(0) psi)(r) = -1/(2 m a^2) sum over the six neighbours of (psi(nbr) - psi(r)), with
// psi pinned to 0 on the Dirichlet planes (any index 0; a neighbour index N wraps onto
// the plane 0).  One pass: read psi and V, write psi' = s (coef_A psi - coef_B dtau H psi)
// into the other buffer, plus the FP64 partial sums of <psi|psi>, <psi|H_K psi>,
// <psi|V psi> on check steps.
//
// Each block owns a BX x BY column tile and marches in z, keeping psi(z-1), psi(z),
// psi(z+1) of its column in registers; the x/y neighbours come from the cache
// hierarchy (they are read by the neighbouring threads of the same block).
#include "qf_common.cuh"

namespace qf {

constexpr int ST_BX = 32, ST_BY = 4, ST_ZC = 16;

template <typename R>
__device__ __forceinline__ cpx<R> ld_masked(const cpx<R>* __restrict__ p, int n, int ix, int iy, int iz) {
  // sites on the Dirichlet planes (index 0, or N = the plane 0 seen across the wrap) are 0
  if (ix == 0 || iy == 0 || iz == 0 || ix == n || iy == n || iz == n) return mk<R>(R(0), R(0));
  return p[((long long)iz * n + iy) * n + ix];
}

template <typename R>
__device__ __forceinline__ void stencil_body(const StencilArgs<R>& a, const int n, const int bzi) {
  __shared__ double red_s[32 * kNumSums];
  const int ix = blockIdx.x * ST_BX + threadIdx.x;
  const int iy = blockIdx.y * ST_BY + threadIdx.y;
  const int z0 = bzi * ST_ZC;
  const int z1 = min(n, z0 + ST_ZC);
  const bool active = ix < n && iy < n;
  CheckSums<R> cs;
  if (active) {
    const R sc = R(*a.scale);
    cpx<R> zm = ld_masked<R>(a.in, n, ix, iy, z0 - 1 < 0 ? 0 : z0 - 1);
    cpx<R> c = ld_masked<R>(a.in, n, ix, iy, z0);
    for (int iz = z0; iz < z1; ++iz) {
      const cpx<R> zp = ld_masked<R>(a.in, n, ix, iy, iz + 1);
      const long long site = ((long long)iz * n + iy) * n + ix;
      const bool interior = ix != 0 && iy != 0 && iz != 0;
      if (interior) {
        const cpx<R> xm = ld_masked<R>(a.in, n, ix - 1, iy, iz), xp = ld_masked<R>(a.in, n, ix + 1, iy, iz);
        const cpx<R> ym = ld_masked<R>(a.in, n, ix, iy - 1, iz), yp = ld_masked<R>(a.in, n, ix, iy + 1, iz);
        const cpx<R> nb = ((xm + xp) + (ym + yp)) + (zm + zp);
        // H psi = -kcoef (sum nbr - 6 psi)
        const cpx<R> h = mk<R>(-a.kcoef * (nb.x - R(6) * c.x), -a.kcoef * (nb.y - R(6) * c.y));
        cpx<R> vv;
        if (a.v_real) vv = mk<R>(reinterpret_cast<const R*>(a.v)[site], R(0));
        else vv = reinterpret_cast<const cpx<R>*>(a.v)[site];
        if (a.reduce) cs.add(c, h, vv);
        if (a.write_psi) {
          const cpx<R> d = mk<R>(R(1) + a.half_dtau * vv.x, a.half_dtau * vv.y);
          const cpx<R> num = cmul<R>(mk<R>(R(2) - d.x, -d.y), c) - cscale<R>(h, a.dtau);
          const R inv = sc / (d.x * d.x + d.y * d.y);
          a.out[site] = cscale<R>(cmulc<R>(num, d), inv);
        }
      } else if (a.write_psi) {
        a.out[site] = mk<R>(R(0), R(0));
      }
      zm = c;
      c = zp;
    }
  }
  if (a.reduce) {
    double acc[kNumSums];
    cs.to(acc);
    const int bid = (bzi * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    // flatten the 2D thread index for the block reduction
    double* out = a.partials + (long long)bid * kPartialStride;
    // block_sum_store uses threadIdx.x as the linear id: remap through a local copy
    const int tid = threadIdx.y * ST_BX + threadIdx.x;
    // warp-level: threads of one warp share threadIdx.y (BX = 32)
    warp_sum<kNumSums>(acc);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
      for (int i = 0; i < kNumSums; ++i) red_s[warp * kNumSums + i] = acc[i];
    __syncthreads();
    if (warp == 0) {
      double t[kNumSums];
      for (int i = 0; i < kNumSums; ++i) t[i] = lane < ST_BY ? red_s[lane * kNumSums + i] : 0.0;
      warp_sum<kNumSums>(t);
      if (lane == 0)
        for (int i = 0; i < kNumSums; ++i) out[i] = t[i];
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(ST_BX* ST_BY) stencil_kernel(StencilArgs<R> a, int n) {
  stencil_body<R>(a, n, blockIdx.z);
}

// A group of lattices of the same n: blockIdx.z = member * z-chunks + z-chunk.
template <typename R>
__global__ void __launch_bounds__(ST_BX* ST_BY) stencil_group_kernel(const __grid_constant__ StencilGroup<R> g, int n) {
  const int nzb = (n + ST_ZC - 1) / ST_ZC;
  stencil_body<R>(g.a[blockIdx.z / nzb], n, blockIdx.z % nzb);
}

template cudaError_t launch_stencil_group<float>(int, const StencilGroup<float>&, cudaStream_t);

template <typename R>
int stencil_blocks(int n) {
  return ((n + ST_BX - 1) / ST_BX) * ((n + ST_BY - 1) / ST_BY) * ((n + ST_ZC - 1) / ST_ZC);
}

template <typename R>
cudaError_t launch_stencil_group(int n, const StencilGroup<R>& g, cudaStream_t st) {
  dim3 grid((n + ST_BX - 1) / ST_BX, (n + ST_BY - 1) / ST_BY, ((n + ST_ZC - 1) / ST_ZC) * g.count);
  stencil_group_kernel<R><<<grid, dim3(ST_BX, ST_BY), 0, st>>>(g, n);
  return cudaGetLastError();
}
// Complex-FP32 lattices run the grouped kernel (a lone lattice is a group of one) so a
// lattice executes the same machine code alone and inside a batch.
template <typename R>
cudaError_t launch_stencil(int n, StencilArgs<R> a, cudaStream_t st, int* nblocks) {
  dim3 grid((n + ST_BX - 1) / ST_BX, (n + ST_BY - 1) / ST_BY, (n + ST_ZC - 1) / ST_ZC);
  dim3 block(ST_BX, ST_BY);
  if (nblocks) *nblocks = grid.x * grid.y * grid.z;
  if constexpr (sizeof(R) == 4) {
    StencilGroup<R> g;
    g.count = 1;
    g.a[0] = a;
    return launch_stencil_group<R>(n, g, st);
  } else {
    stencil_kernel<R><<<grid, block, 0, st>>>(a, n);
    return cudaGetLastError();
  }
}

template int stencil_blocks<float>(int);
template int stencil_blocks<double>(int);
template cudaError_t launch_stencil<float>(int, StencilArgs<float>, cudaStream_t, int*);
template cudaError_t launch_stencil<double>(int, StencilArgs<double>, cudaStream_t, int*);

}  // namespace qf
