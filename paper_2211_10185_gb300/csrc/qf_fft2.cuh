// Two-pass imaginary-time FFT step for N = 256 complex-FP32 lattices (Eqs. HK1-HK3 and
// the update of Sec. 2), sm_103a.
//
// The 3D transform is reorganised so that a steady-state step reads and writes HBM in two
// passes instead of four.  The y transform of length 256 is split four-step fashion,
// y = y_lo + 16 y_hi and k_y = k_lo + 16 k_hi:
//   Y(k_lo + 16 k_hi) = sum_{y_lo} w16^{y_lo k_hi} [ w256^{y_lo k_lo}
//                        sum_{y_hi} w16^{y_hi k_lo} f(y_lo + 16 y_hi) ],
// and each half is attached to a pass that already holds the needed elements:
//   pass A  x forward + the inner 16-point DFTs over y_hi (+ twiddle), from a field in
//           natural order, into the scratch field S;
//   pass B  the outer 16-point DFTs over y_lo, z forward, T(k), z inverse, the outer
//           inverse DFTs, S in place;
//   pass C  the inner inverse DFTs (+ conjugate twiddle), x inverse, the update of psi
//           (and the FP64 check sums), then pass A on psi_{t+1} for the next step.
// Steady state: B + C = 16 + (8 + 8 + 4 + 8 + 8) B per site (real V) instead of 84.
//
// S layout (the scratch field, 2^24 elements): [kx_hi 128][k_lo 16][y_lo 16][z 256][kx_lo 2]
// with kx = 2 kx_hi + kx_lo.  A pass-B block owns one (kx_hi, k_lo): 8192 contiguous
// elements, and reads its outer y DFTs' inputs straight from global memory (a warp reads
// 256 contiguous bytes per y_lo).  A pass-A/C block owns one y_lo and the two z-planes
// z0, z0 + 1: the 32 lines y = y_lo + 16 y_hi of both planes, and in S one 32-byte
// sector (2 z x 2 kx_lo) per (kx_hi, k_lo).
//
// Shared-memory layouts are padded for conflict-free access: the A/C line tile has pitch
// 280 (line 2 y_hi + (z - z0), one pad element per 16); pass B exchanges through a
// [k_hi][z][kx_lo] tile and per-warp buffers of pitch 280 (one pad element per 16).
#pragma once
#include "qf_fft_impl.cuh"

namespace qf {

constexpr int F2_N = 256;
constexpr int F2_THREADS = 512;                       // pass B block
constexpr int F2_BLOCKS = 2048;                       // pass B blocks per lattice
constexpr int F2_PL = 280;                            // A/C tile line pitch
constexpr int F2_BPAD = 280;                          // B per-(warp, kx_lo) buffer pitch
constexpr int F2_TW = plan_tw_size(F2_N);             // 255 per-stage twiddles
constexpr int F2_TW1 = plan_tw_off(F2_N, 1);          // stage-1 block: w256^{k r}
constexpr int F2_TWB = (F2_TW * 8 + 15) / 16 * 16;    // twiddle bytes in shared memory
constexpr int F2_BTILE = 16 * 2 * F2_BPAD;            // B tile elements (exchange buffers)
constexpr size_t F2_SMEM_B = F2_TWB + F2_N * 4 + (size_t)F2_BTILE * 8 + 32 * kNumSums * 8;
constexpr long long F2_SKLO = (long long)F2_N * 32;   // S stride of k_lo

// pass A / C geometry: YL = 2 z-planes of one y_lo per block
template <int YL>
struct F2AC {
  static_assert(YL == 2, "a pass-A/C block holds two z-planes");
  static constexpr int THREADS = 256 * YL;
  static constexpr int LINES = 16 * YL;
  static constexpr int BLOCKS = 4096 / YL;
  static constexpr size_t SMEM = F2_TWB + (size_t)LINES * F2_PL * 8 + 32 * kNumSums * 8;
};

// w256^{y_lo k_lo} (forward) from the stage-1 twiddle block
__device__ __forceinline__ cpx<float> f2_tw(const cpx<float>* tw_s, int ylo, int klo) {
  return klo == 0 ? mk<float>(1.f, 0.f) : tw_s[F2_TW1 + ylo * 15 + klo - 1];
}

__device__ __forceinline__ int f2_tile(int line, int e) { return line * F2_PL + e + (e >> 4); }
// B exchange buffer position: one pad element per 16 (pitch 280 = 8 mod 16 between the
// two kx_lo buffers of a warp), so both Stockham access patterns are conflict-free
__device__ __forceinline__ int f2_bpad(int p) { return p + (p >> 4); }

// Blocks are dispatched roughly in index order, two per SM at a time, so block b + 2 x
// (SM count) runs about one wave after block b: passes A and B pull that block's inputs
// into L2 while they work, and the next wave finds them there instead of waiting on HBM.
__device__ __forceinline__ int f2_next_wave_block() {
  unsigned nsm;
  asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
  return (int)blockIdx.x + 2 * (int)nsm;
}
__device__ __forceinline__ void f2_prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// Offset of line `line` of pass-A/C block blk in a natural-order field: the block holds
// y_lo = blk mod 16 of the z-planes 2 (blk / 16) and 2 (blk / 16) + 1; line = 2 y_hi + dz.
template <int YL>
__device__ __forceinline__ long long f2_row(int blk, int line) {
  const int z = 2 * (blk >> 4) + (line & 1), y = (blk & 15) + 16 * (line >> 1);
  return ((long long)z * F2_N + y) * F2_N;
}

// x transform of the 16 elements v[r] = line element g + 16 r of this thread's line
// (positions g + 16 r in and out), through the line tile for the stage exchange.  A line
// belongs to 16 lanes of one warp and its tile row to those lanes alone (callers
// separate block-wide tile use with __syncthreads), so the exchange needs only warp
// synchronisation.
template <bool INV>
__device__ __forceinline__ void f2_x_transform(cpx<float> (&v)[16], int line, int g, cpx<float>* tile,
                                               const cpx<float>* tw_s) {
  stage_compute<float, F2_N, 0, INV>(v, g, tw_s);
  __syncwarp();  // the line's earlier reads of its tile row are done
#pragma unroll
  for (int r = 0; r < 16; ++r) tile[f2_tile(line, 16 * g + r)] = v[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = tile[f2_tile(line, g + 16 * r)];
  stage_compute<float, F2_N, 1, INV>(v, g, tw_s);
}

// Thread roles in a pass-A/C block (one y_lo, z-planes z0 and z0 + 1).
template <int YL>
struct F2Roles {
  int z0, ylo;            // the block's first z-plane and its y_lo
  int line, g;            // x role: line 2 y_hi + s, element group g
  int kx, s;              // cross role: column kx of the lines of z-plane z0 + s
  long long row;          // natural offset of line `line`
  long long sbase;        // S offset of (kx_hi, k_lo = 0, y_lo, z0 + s, kx_lo)
  __device__ __forceinline__ F2Roles(int blk) {
    z0 = 2 * (blk >> 4);
    ylo = blk & 15;
    const int tid = threadIdx.x;
    line = tid >> 4;
    g = tid & 15;
    row = f2_row<YL>(blk, line);
    const int kxlo = tid & 1;
    s = (tid >> 1) & 1;
    const int kxhi = tid >> 2;
    kx = 2 * kxhi + kxlo;
    sbase = ((long long)kxhi * 16 * 16 + ylo) * (2 * F2_N) + 2 * (z0 + s) + kxlo;
  }
};

// Cross stage forward: line tile (x-transformed) -> 16-point DFTs over y_hi, twiddle,
// store into S.
template <int YL>
__device__ __forceinline__ void f2_cross_fwd(const F2Roles<YL>& q, const cpx<float>* tile, const cpx<float>* tw_s,
                                             cpx<float>* S) {
  cpx<float> u[16];
#pragma unroll
  for (int yh = 0; yh < 16; ++yh) u[yh] = tile[f2_tile(YL * yh + q.s, q.kx)];
  dft16<float, false>(u);
#pragma unroll
  for (int k = 0; k < 16; ++k) S[q.sbase + k * F2_SKLO] = cmul<float>(u[k], f2_tw(tw_s, q.ylo, k));
}

// Pass A: field `src` (natural order) -> S.  With SUMS (energy of a field that is not
// stepped): also <src|src> and <src|V src> of its sites into partial row blockIdx.x; the
// kinetic part comes from pass B in k-space.
template <int YL, bool SUMS = false>
__global__ void __launch_bounds__(F2AC<YL>::THREADS, 4 / YL) fft2_a_kernel(const __grid_constant__ FftGroup<float> gr) {
  const FftPassArgs<float>& a = gr.a[blockIdx.y];
  extern __shared__ __align__(16) unsigned char f2_smem[];
  cpx<float>* tw_s = reinterpret_cast<cpx<float>*>(f2_smem);
  cpx<float>* tile = reinterpret_cast<cpx<float>*>(f2_smem + F2_TWB);
  const F2Roles<YL> q(blockIdx.x);
  const cpx<float>* __restrict__ src = a.src ? a.src : a.psi;
  cpx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = src[q.row + q.g + 16 * r];
  CheckSums<float> cs;
  if constexpr (SUMS) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const long long site = q.row + q.g + 16 * r;
      const cpx<float> vi = a.v_real ? mk<float>(reinterpret_cast<const float*>(a.v)[site], 0.f)
                                     : reinterpret_cast<const cpx<float>*>(a.v)[site];
      cs.add(v[r], mk<float>(0.f, 0.f), vi);
    }
  }
  {
    const int nb = f2_next_wave_block();
    if (nb < (int)gridDim.x && threadIdx.x < F2AC<YL>::LINES)
      f2_prefetch_l2(src + f2_row<YL>(nb, threadIdx.x), F2_N * 8);
  }
  for (int i = threadIdx.x; i < F2_TW; i += F2AC<YL>::THREADS) tw_s[i] = a.twiddle[i];
  __syncthreads();
  f2_x_transform<false>(v, q.line, q.g, tile, tw_s);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) tile[f2_tile(q.line, q.g + 16 * r)] = v[r];
  __syncthreads();
  f2_cross_fwd<YL>(q, tile, tw_s, a.data);
  if constexpr (SUMS) {
    double acc[kNumSums];
    cs.to(acc);
    block_sum_store<kNumSums>(acc, reinterpret_cast<double*>(tile + F2AC<YL>::LINES * F2_PL),
                              a.partials + (long long)blockIdx.x * kPartialStride);
  }
}

// Pass B: S in place, one (kx_hi, k_lo) block of 8192 contiguous elements [y_lo][z][kx_lo].
//   outer y DFTs: thread (z, kx_lo) = (tid / 2, tid % 2) reads its 16 y_lo values straight
//     from global memory (a warp reads 256 contiguous bytes per y_lo) -> natural k_hi;
//   exchange 1 through the [k_hi][z][kx_lo] tile to the z role: warp = k_hi, lane =
//     (z1, kx_lo) = (lane / 2, lane % 2), holding z = z1 + 16 r;
//   z forward, T(k), z inverse: Stockham stages with warp-local exchanges through the
//     warp's two padded buffers (which reuse the tile);
//   exchange 2 back to (z, kx_lo), inverse outer y DFTs, written straight to global memory.
// Four shared-memory round trips per element.  With SUMS (energy of a field that is not
// stepped): after the z forward transform, <v|H_K v> = sum_k T(k)/N^3 |v^(k)|^2
// (Parseval) into partial row row0 + blockIdx.x, and nothing is written back.
template <bool SUMS = false>
__global__ void __launch_bounds__(F2_THREADS, 2) fft2_b_kernel(const __grid_constant__ FftGroup<float> gr,
                                                               int row0 = 0) {
  const FftPassArgs<float>& a = gr.a[blockIdx.y];
  extern __shared__ __align__(16) unsigned char f2_smem[];
  cpx<float>* tw_s = reinterpret_cast<cpx<float>*>(f2_smem);
  float* sym_s = reinterpret_cast<float*>(f2_smem + F2_TWB);
  cpx<float>* tile = reinterpret_cast<cpx<float>*>(reinterpret_cast<unsigned char*>(sym_s) + F2_N * 4);
  const int blk = blockIdx.x, kxhi = blk >> 4, klo = blk & 15;
  const int tid = threadIdx.x;
  cpx<float>* base = a.data + (long long)blk * 8192;
  {
    const int nb = f2_next_wave_block();
    if (nb < (int)gridDim.x && tid < 4) f2_prefetch_l2(a.data + (long long)nb * 8192 + tid * 2048, 2048 * 8);
  }
  cpx<float> u[16];
#pragma unroll
  for (int y = 0; y < 16; ++y) u[y] = base[y * 512 + tid];
  for (int i = tid; i < F2_TW; i += F2_THREADS) tw_s[i] = a.twiddle[i];
  for (int i = tid; i < F2_N; i += F2_THREADS) sym_s[i] = a.symbol[i];
  dft16<float, false>(u);
#pragma unroll
  for (int k = 0; k < 16; ++k) tile[k * 512 + tid] = u[k];
  __syncthreads();
  // z role
  const int w = tid >> 5, lane = tid & 31, kxl = lane & 1, z1 = lane >> 1;
  cpx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = tile[w * 512 + lane + 32 * r];
  __syncthreads();  // the tile becomes the per-warp exchange buffers
  cpx<float>* wb = tile + (2 * w + kxl) * F2_BPAD;
  stage_compute<float, F2_N, 0, false>(v, z1, tw_s);
#pragma unroll
  for (int r = 0; r < 16; ++r) wb[f2_bpad(16 * z1 + r)] = v[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = wb[f2_bpad(z1 + 16 * r)];
  stage_compute<float, F2_N, 1, false>(v, z1, tw_s);
  // natural-order kz = z1 + 16 r; T(kx, ky, kz)/N^3 with ky = k_lo + 16 k_hi
  {
    const int kx = 2 * kxhi + kxl, ky = klo + 16 * w;
    const float sxy = sym_s[kx] + sym_s[ky];
    if constexpr (SUMS) {
      CheckSums<float> cs;
#pragma unroll
      for (int r = 0; r < 16; ++r)
        cs.add(v[r], cscale<float>(v[r], kin_mult<float>(a.kinetic, sxy, sym_s[z1 + 16 * r], a.tcoef, a.am2)),
               mk<float>(0.f, 0.f));
      double acc[kNumSums];
      cs.to(acc);
      acc[0] = acc[3] = acc[4] = 0.0;  // norm and potential terms come from pass A
      block_sum_store<kNumSums>(acc, reinterpret_cast<double*>(tile + F2_BTILE),
                                a.partials + (long long)(row0 + blockIdx.x) * kPartialStride);
      return;
    }
#pragma unroll
    for (int r = 0; r < 16; ++r)
      v[r] = cscale<float>(v[r], kin_mult<float>(a.kinetic, sxy, sym_s[z1 + 16 * r], a.tcoef, a.am2));
  }
  stage_compute<float, F2_N, 0, true>(v, z1, tw_s);
  __syncwarp();  // (the buffer's own lanes are its only readers)
#pragma unroll
  for (int r = 0; r < 16; ++r) wb[f2_bpad(16 * z1 + r)] = v[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = wb[f2_bpad(z1 + 16 * r)];
  stage_compute<float, F2_N, 1, true>(v, z1, tw_s);
  __syncthreads();  // every warp is done with its buffers
#pragma unroll
  for (int r = 0; r < 16; ++r) tile[w * 512 + lane + 32 * r] = v[r];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 16; ++k) u[k] = tile[k * 512 + tid];
  dft16<float, true>(u);
#pragma unroll
  for (int y = 0; y < 16; ++y) base[y * 512 + tid] = u[y];
}

// Pass C: S -> inverse inner y DFTs, x inverse -> H_K psi; update / sums; with NEXT, pass A
// on psi_{t+1} into S.  OP: OP_FINAL (write), OP_FINAL_SUMS (write + sums), OP_SUMS.
// Everything of pass C after the scratch values u (this thread's 16 k_lo values of its
// cross-role column) are in registers: block `item`.
template <int YL, int OP, bool VREAL, bool NEXT>
__device__ __forceinline__ void f2_c_body(const FftPassArgs<float>& a, const F2Roles<YL>& q, cpx<float> (&u)[16],
                                          cpx<float>* tile, const cpx<float>* tw_s, double* red_s, int item) {
  constexpr bool WRITE = (OP == OP_FINAL || OP == OP_FINAL_SUMS);
  constexpr bool SUMS = (OP == OP_FINAL_SUMS || OP == OP_SUMS);
#pragma unroll
  for (int k = 0; k < 16; ++k) u[k] = cmulc<float>(u[k], f2_tw(tw_s, q.ylo, k));
  dft16<float, true>(u);
#pragma unroll
  for (int yh = 0; yh < 16; ++yh) tile[f2_tile(YL * yh + q.s, q.kx)] = u[yh];
  __syncthreads();
  cpx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = tile[f2_tile(q.line, q.g + 16 * r)];
  f2_x_transform<true>(v, q.line, q.g, tile, tw_s);
  // v[r] = H_K psi at x = g + 16 r of row `row` (1/N^3 inside T); psi and V are read
  // site by site (registers are the limit)
  CheckSums<float> cs;
  const float sc = WRITE ? float(*a.scale) : 1.f;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const long long site = q.row + q.g + 16 * r;
    const cpx<float> pv = a.psi[site];
    cpx<float> vi;
    if constexpr (VREAL) vi = mk<float>(reinterpret_cast<const float*>(a.v)[site], 0.f);
    else vi = reinterpret_cast<const cpx<float>*>(a.v)[site];
    if constexpr (SUMS) cs.add(pv, v[r], vi);
    if constexpr (WRITE) {
      // d = 1 + dtau V/2; coef_B = 1/d; coef_A = (2 - d)/d
      if constexpr (VREAL) {
        const float d = 1.f + a.half_dtau * vi.x;
        const cpx<float> num = cscale<float>(pv, 2.f - d) - cscale<float>(v[r], a.dtau);
        v[r] = cscale<float>(num, __fdividef(sc, d));  // psi_{t+1}
      } else {
        const cpx<float> d = mk<float>(1.f + a.half_dtau * vi.x, a.half_dtau * vi.y);
        const cpx<float> num = cmul<float>(mk<float>(2.f - d.x, -d.y), pv) - cscale<float>(v[r], a.dtau);
        const float inv = __fdividef(sc, d.x * d.x + d.y * d.y);
        v[r] = cscale<float>(cmulc<float>(num, d), inv);  // psi_{t+1}
      }
      a.psi[site] = v[r];
    }
  }
  if constexpr (SUMS) {
    double acc[kNumSums];
    cs.to(acc);
    block_sum_store<kNumSums>(acc, red_s, a.partials + ((long long)item) * kPartialStride);
  }
  if constexpr (WRITE && NEXT) {
    f2_x_transform<false>(v, q.line, q.g, tile, tw_s);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) tile[f2_tile(q.line, q.g + 16 * r)] = v[r];
    __syncthreads();
    f2_cross_fwd<YL>(q, tile, tw_s, a.data);
  }
}

// L2 prefetch of psi and V of the output rows of pass-C block `item` (threads < 4 YL 16).
template <int YL, bool VREAL>
__device__ __forceinline__ void f2_prefetch_psi_v(const FftPassArgs<float>& a, int item) {
  constexpr int LINES = F2AC<YL>::LINES;
  if (threadIdx.x < 2 * LINES) {
    const long long row = f2_row<YL>(item, threadIdx.x % LINES);
    if (threadIdx.x < LINES) f2_prefetch_l2(a.psi + row, F2_N * 8);
    else if (VREAL) f2_prefetch_l2(reinterpret_cast<const float*>(a.v) + row, F2_N * 4);
    else f2_prefetch_l2(reinterpret_cast<const cpx<float>*>(a.v) + row, F2_N * 8);
  }
}

template <int YL, int OP, bool VREAL, bool NEXT>
__global__ void __launch_bounds__(F2AC<YL>::THREADS, 4 / YL) fft2_c_kernel(const __grid_constant__ FftGroup<float> gr) {
  constexpr int LINES = F2AC<YL>::LINES;
  const FftPassArgs<float>& a = gr.a[blockIdx.y];
  extern __shared__ __align__(16) unsigned char f2_smem[];
  cpx<float>* tw_s = reinterpret_cast<cpx<float>*>(f2_smem);
  cpx<float>* tile = reinterpret_cast<cpx<float>*>(f2_smem + F2_TWB);
  double* red_s = reinterpret_cast<double*>(tile + LINES * F2_PL);
  const F2Roles<YL> q(blockIdx.x);
  // psi and V of the output rows are needed only after the transforms: start pulling them
  // into L2 now, one bulk prefetch per row.  (Measured slower: prefetching the next
  // wave's rows or scratch sectors here as well, this pass already moving 36 B per site;
  // and a persistent form with one block per SM that stages the next item's sectors with
  // cp.async while computing, 16 warps per SM being too few for the transforms.)
  f2_prefetch_psi_v<YL, VREAL>(a, blockIdx.x);
  for (int i = threadIdx.x; i < F2_TW; i += F2AC<YL>::THREADS) tw_s[i] = a.twiddle[i];
  cpx<float> u[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) u[k] = a.data[q.sbase + k * F2_SKLO];
  __syncthreads();
  f2_c_body<YL, OP, VREAL, NEXT>(a, q, u, tile, tw_s, red_s, blockIdx.x);
}

}  // namespace qf
