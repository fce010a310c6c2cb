// TMA-staged FDTD step (Eq. HK0), sm_103a.
//
// A block owns a 32 x 32 column tile of the output (each thread 4 rows) and marches through
// a chunk of z, prefetching V one plane ahead into registers.  One
// thread streams the halo-extended z-planes of the tile (x0-2 .. x0+33 or x0-1 .. x0+32,
// y0-1 .. y0+32) from global memory into a ring of six shared-memory buffers with
// cp.async.bulk.tensor; each buffer has an mbarrier that completes when its bytes have
// landed.  While plane z is computed (it needs planes z-1, z, z+1) the planes z+2 .. z+4
// are in flight.  Coordinates outside the lattice are filled with zeros by the copy
// engine; the Dirichlet planes (index 0) are masked when read.
//
// Every wait is bounded.  If a buffer does not complete within the limit, the block
// agrees on it (__syncthreads_and), records the failure in *err, waits a bounded time
// for its own copies still in flight and returns; the host reports QF_ETIMEOUT.
#pragma once
#include <cuda.h>

#include "qf_common.cuh"

namespace qf {

constexpr int TS_X = 32, TS_Y = 32, TS_ROWS = 4, TS_BUF = 6;  // 32 x 8 threads
// z-chunk per block: runtime (StencilTmaGroup::zc), picked by the autotuner from these
constexpr int kStencilZChunks[3] = {8, 16, 32};
constexpr int kStencilZChunkMin = 8;
constexpr unsigned kTmaSpinLimit = 1u << 24;

// words of 8 bytes per tile row: c64 x0-2 .. x0+33 (36 complex); c128 x0-1 .. x0+32 as
// 68 doubles
template <typename R>
struct TmaTile {
  static constexpr int W = sizeof(R) == 4 ? TS_X + 4 : 2 * (TS_X + 2);
  static constexpr int PLANE_WORDS = (TS_Y + 2) * W;            // one box
  static constexpr int STRIDE_WORDS = (PLANE_WORDS + 15) / 16 * 16;  // buffers start on 128 B
  static constexpr unsigned BYTES = PLANE_WORDS * 8u;
};

// Members of one launch may have different lattice sizes: member i runs
// tiles(n_i) x ceil(n_i / zc_i) blocks, numbered from start[i] in a one-dimensional grid
// (tile x fastest, then tile y, then z-chunk), exactly the blocks it runs alone.
template <typename R>
struct alignas(64) StencilTmaGroup {
  CUtensorMap map[kGroupMax];  // input field of member i, 3D (x, y, z), 8-byte elements
  StencilArgs<R> a[kGroupMax];
  int nm[kGroupMax];           // lattice size of member i
  int zcm[kGroupMax];          // planes per block (z-chunk) of member i
  int start[kGroupMax + 1];    // first block of member i; start[count] = blocks in all
  int count;
  int* err;                    // set to 1 when a bounded wait ran out
};

// Blocks member i of a stencil group runs (tiles x z-chunks).
__host__ __device__ __forceinline__ int stencil_member_blocks(int n, int zc) {
  return ((n + TS_X - 1) / TS_X) * ((n + TS_Y - 1) / TS_Y) * ((n + zc - 1) / zc);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for phase `parity` of a buffer's barrier
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (unsigned it = 0; it < kTmaSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// plane p of member tile -> buffer; coordinates in elements of the tensor map
template <typename R>
__device__ __forceinline__ void tma_plane(const CUtensorMap* map, unsigned long long* bar, void* dst, int x0, int y0,
                                          int z) {
  const int cx = sizeof(R) == 4 ? x0 - 2 : 2 * (x0 - 1);  // x start: 16-byte aligned
  const int cy = y0 - 1;
  mbar_expect_tx(bar, TmaTile<R>::BYTES);
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(cx), "r"(cy), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// ---- the per-site FDTD update, shared by every kernel that computes a site ------------
// Each operation is rounded explicitly (no contraction left to the compiler), so the
// single-step kernel and the temporally blocked kernel produce the same bits for a site.
template <typename R> __device__ __forceinline__ R add_rn(R a, R b);
template <typename R> __device__ __forceinline__ R mul_rn(R a, R b);
template <typename R> __device__ __forceinline__ R fma_rn(R a, R b, R c);
template <typename R> __device__ __forceinline__ R scaled_inverse(R s, R d);
template <> __device__ __forceinline__ float add_rn<float>(float a, float b) { return __fadd_rn(a, b); }
template <> __device__ __forceinline__ double add_rn<double>(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
// s / d: FP32 through the fast hardware division (about 2 ulp, no branch); FP64 through
// the correctly rounded reciprocal
template <> __device__ __forceinline__ float scaled_inverse<float>(float s, float d) { return __fdividef(s, d); }
template <> __device__ __forceinline__ double scaled_inverse<double>(double s, double d) {
  return __dmul_rn(s, __drcp_rn(d));
}

// sum of the six neighbours in the fixed order ((x- + x+) + (y- + y+)) + (z- + z+)
template <typename R>
__device__ __forceinline__ cpx<R> six_sum(cpx<R> xm, cpx<R> xp, cpx<R> ym, cpx<R> yp, cpx<R> zm, cpx<R> zp) {
  return mk<R>(add_rn<R>(add_rn<R>(add_rn<R>(xm.x, xp.x), add_rn<R>(ym.x, yp.x)), add_rn<R>(zm.x, zp.x)),
               add_rn<R>(add_rn<R>(add_rn<R>(xm.y, xp.y), add_rn<R>(ym.y, yp.y)), add_rn<R>(zm.y, zp.y)));
}

// lap = sum of neighbours - 6 psi, so that H_K^(0) psi = -kcoef * lap (Eq. HK0)
template <typename R>
__device__ __forceinline__ cpx<R> lap_of(cpx<R> c, cpx<R> nbs) {
  return mk<R>(fma_rn<R>(R(-6), c.x, nbs.x), fma_rn<R>(R(-6), c.y, nbs.y));
}

// psi' = s (coef_A psi - coef_B dtau H_K psi) with d = 1 + dtau V / 2:
// psi' = s ((2 - d) psi + kd lap) conj(d) / |d|^2, kd = dtau * kcoef.  For real V,
// conj(d)/|d|^2 = 1/d.
template <typename R>
__device__ __forceinline__ cpx<R> fdtd_update(cpx<R> c, cpx<R> lap, cpx<R> v, bool v_real, R half_dtau, R kd, R sc) {
  const R dx = fma_rn<R>(half_dtau, v.x, R(1));
  const R tx = add_rn<R>(R(2), -dx);
  if (v_real) {
    const R inv = scaled_inverse<R>(sc, dx);
    return mk<R>(mul_rn<R>(fma_rn<R>(kd, lap.x, mul_rn<R>(tx, c.x)), inv),
                 mul_rn<R>(fma_rn<R>(kd, lap.y, mul_rn<R>(tx, c.y)), inv));
  }
  const R dy = mul_rn<R>(half_dtau, v.y);
  // (2 - d) psi = (tx - i dy) psi
  const R ax = fma_rn<R>(tx, c.x, mul_rn<R>(dy, c.y));
  const R ay = fma_rn<R>(tx, c.y, -mul_rn<R>(dy, c.x));
  const R nx = fma_rn<R>(kd, lap.x, ax), ny = fma_rn<R>(kd, lap.y, ay);
  const R inv = scaled_inverse<R>(sc, fma_rn<R>(dx, dx, mul_rn<R>(dy, dy)));
  return mk<R>(mul_rn<R>(fma_rn<R>(nx, dx, mul_rn<R>(ny, dy)), inv),
               mul_rn<R>(fma_rn<R>(ny, dx, -mul_rn<R>(nx, dy)), inv));
}

template <typename R>
__device__ __forceinline__ cpx<R> tile_at(const unsigned long long* buf, int ix, int iy, int x0, int y0) {
  const int row = iy - y0 + 1;
  if constexpr (sizeof(R) == 4) {
    const cpx<float>* b = reinterpret_cast<const cpx<float>*>(buf);
    const cpx<float> v = b[row * TmaTile<R>::W + (ix - x0 + 2)];
    return mk<R>(R(v.x), R(v.y));
  } else {
    const cpx<double>* b = reinterpret_cast<const cpx<double>*>(buf);
    const cpx<double> v = b[(row * TmaTile<R>::W) / 2 + (ix - x0 + 1)];
    return mk<R>(R(v.x), R(v.y));
  }
}

template <typename R>
__global__ void __launch_bounds__(TS_X*(TS_Y / TS_ROWS), sizeof(R) == 4 ? 3 : 2) stencil_tma_kernel(const __grid_constant__ StencilTmaGroup<R> g) {
  extern __shared__ __align__(128) unsigned long long planes_dyn[];
  unsigned long long(*planes)[TmaTile<R>::STRIDE_WORDS] =
      reinterpret_cast<unsigned long long(*)[TmaTile<R>::STRIDE_WORDS]>(planes_dyn);
  __shared__ alignas(8) unsigned long long bars[TS_BUF];
  __shared__ double red_s[32 * kNumSums];
  // member of this block (last i with start[i] <= block), then its tile and z-chunk
  int member = 0;
  {
    int hi = g.count - 1;
    while (member < hi) {
      const int mid = (member + hi + 1) >> 1;
      if (g.start[mid] <= (int)blockIdx.x) member = mid;
      else hi = mid - 1;
    }
  }
  const int n = g.nm[member];
  const int zc = g.zcm[member];
  const int nbx = (n + TS_X - 1) / TS_X, nby = (n + TS_Y - 1) / TS_Y;
  const int local = (int)blockIdx.x - g.start[member];
  const int bx = local % nbx, by = (local / nbx) % nby, zb = local / (nbx * nby);
  const StencilArgs<R>& a = g.a[member];
  const CUtensorMap* map = &g.map[member];
  const int tid = threadIdx.y * TS_X + threadIdx.x;
  const int x0 = bx * TS_X, y0 = by * TS_Y;
  const int ix = x0 + threadIdx.x;
  const int z0 = zb * zc, z1 = min(n, z0 + zc);
  const int pfirst = z0 - 1, plast = z1;  // planes needed (inclusive)
  if (tid == 0) {
    for (int b = 0; b < TS_BUF; ++b) mbar_init(&bars[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  int issued = pfirst - 1;  // last plane whose copy was issued
  if (tid == 0)
    for (int p = pfirst; p <= plast && p < pfirst + TS_BUF; ++p) {
      tma_plane<R>(map, &bars[(p - pfirst) % TS_BUF], planes[(p - pfirst) % TS_BUF], x0, y0, p);
      issued = p;
    }
  // V of this thread's sites, one plane ahead
  auto load_v = [&](int iz, int k) {
    const int iy = y0 + threadIdx.y + (TS_Y / TS_ROWS) * k;
    if (ix >= n || iy >= n || iz >= z1) return mk<R>(R(0), R(0));
    const long long site = ((long long)iz * n + iy) * n + ix;
    return a.v_real ? mk<R>(reinterpret_cast<const R*>(a.v)[site], R(0)) : reinterpret_cast<const cpx<R>*>(a.v)[site];
  };
  cpx<R> vnext[TS_ROWS];
#pragma unroll
  for (int k = 0; k < TS_ROWS; ++k) vnext[k] = load_v(z0, k);
  int waited = pfirst - 1;  // last plane whose buffer this thread has seen complete
  bool ok = true;
  const R sc = R(*a.scale);
  CheckSums<R> cs;
  for (int iz = z0; iz < z1 && ok; ++iz) {
    cpx<R> vcur[TS_ROWS];
#pragma unroll
    for (int k = 0; k < TS_ROWS; ++k) {
      vcur[k] = vnext[k];
      vnext[k] = load_v(iz + 1, k);
    }
    // planes iz-1, iz, iz+1 must have landed: thread 0 polls (bounded), the block learns
    // the outcome at the barrier, then every thread observes the completed phases itself
    bool mine = true;
    if (tid == 0)
      while (waited < iz + 1 && mine) {
        const int u = waited + 1 - pfirst;
        mine = mbar_wait_bounded(&bars[u % TS_BUF], (unsigned)((u / TS_BUF) & 1));
        if (mine) ++waited;
      }
    ok = __syncthreads_and(mine) != 0;
    if (!ok) break;
    if (tid != 0)
      for (; waited < iz + 1; ++waited) {
        const int u = waited + 1 - pfirst;
        mbar_try_wait(&bars[u % TS_BUF], (unsigned)((u / TS_BUF) & 1));  // completed: returns at once
      }
    const unsigned long long* bm = planes[(iz - 1 - pfirst) % TS_BUF];
    const unsigned long long* bc = planes[(iz - pfirst) % TS_BUF];
    const unsigned long long* bp = planes[(iz + 1 - pfirst) % TS_BUF];
    // blocks away from the boundaries read neighbours without masks
    const bool inner = x0 > 0 && y0 > 0 && x0 + TS_X < n && y0 + TS_Y < n && iz > 1 && iz + 1 < n;
#pragma unroll
    for (int k = 0; k < TS_ROWS; ++k) {
      const int iy = y0 + threadIdx.y + (TS_Y / TS_ROWS) * k;
      if (ix >= n || iy >= n) continue;
      const long long site = ((long long)iz * n + iy) * n + ix;
      const bool interior = ix != 0 && iy != 0 && iz != 0;
      if (interior) {
        cpx<R> c, xm, xp, ym, yp, zm, zp;
        c = tile_at<R>(bc, ix, iy, x0, y0);
        if (inner) {
          xm = tile_at<R>(bc, ix - 1, iy, x0, y0);
          xp = tile_at<R>(bc, ix + 1, iy, x0, y0);
          ym = tile_at<R>(bc, ix, iy - 1, x0, y0);
          yp = tile_at<R>(bc, ix, iy + 1, x0, y0);
          zm = tile_at<R>(bm, ix, iy, x0, y0);
          zp = tile_at<R>(bp, ix, iy, x0, y0);
        } else {
          // a neighbour index 0 (the Dirichlet plane) or n (outside, zero-filled) reads 0
          auto nb_at = [&](const unsigned long long* b, int x, int y) {
            return (x == 0 || y == 0 || x == n || y == n) ? mk<R>(R(0), R(0)) : tile_at<R>(b, x, y, x0, y0);
          };
          xm = nb_at(bc, ix - 1, iy);
          xp = nb_at(bc, ix + 1, iy);
          ym = nb_at(bc, ix, iy - 1);
          yp = nb_at(bc, ix, iy + 1);
          zm = (iz - 1 == 0) ? mk<R>(R(0), R(0)) : tile_at<R>(bm, ix, iy, x0, y0);
          zp = (iz + 1 == n) ? mk<R>(R(0), R(0)) : tile_at<R>(bp, ix, iy, x0, y0);
        }
        const cpx<R> lap = lap_of<R>(c, six_sum<R>(xm, xp, ym, yp, zm, zp));
        const cpx<R> vv = vcur[k];
        if (a.reduce) cs.add(c, mk<R>(mul_rn<R>(-a.kcoef, lap.x), mul_rn<R>(-a.kcoef, lap.y)), vv);
        if (a.write_psi) a.out[site] = fdtd_update<R>(c, lap, vv, a.v_real != 0, a.half_dtau, a.kd, sc);
      } else if (a.write_psi) {
        a.out[site] = mk<R>(R(0), R(0));
      }
    }
    __syncthreads();  // every thread is done with plane iz-1's buffer
    if (tid == 0 && issued < plast) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      const int p = issued + 1;
      tma_plane<R>(map, &bars[(p - pfirst) % TS_BUF], planes[(p - pfirst) % TS_BUF], x0, y0, p);
      issued = p;
    }
  }
  if (!ok) {
    if (tid == 0) {
      atomicExch(g.err, 1);
      // copies already issued may still land in this block's shared memory
      for (int p = waited + 1; p <= issued; ++p) {
        const int u = p - pfirst;
        mbar_wait_bounded(&bars[u % TS_BUF], (unsigned)((u / TS_BUF) & 1));
      }
    }
    return;
  }
  if (a.reduce) {
    double acc[kNumSums];
    cs.to(acc);
    const int bid = local;  // (zb * nby + by) * nbx + bx: the member's own partial row
    warp_sum<kNumSums>(acc);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
      for (int i = 0; i < kNumSums; ++i) red_s[warp * kNumSums + i] = acc[i];
    __syncthreads();
    if (warp == 0) {
      double t[kNumSums];
      for (int i = 0; i < kNumSums; ++i) t[i] = lane < (TS_X * TS_Y / TS_ROWS) / 32 ? red_s[lane * kNumSums + i] : 0.0;
      warp_sum<kNumSums>(t);
      if (lane == 0)
        for (int i = 0; i < kNumSums; ++i) a.partials[(long long)bid * kPartialStride + i] = t[i];
    }
  }
}

// dynamic shared memory of the plane ring
template <typename R>
constexpr size_t stencil_tma_smem() {
  return (size_t)TS_BUF * TmaTile<R>::STRIDE_WORDS * 8;
}

}  // namespace qf
