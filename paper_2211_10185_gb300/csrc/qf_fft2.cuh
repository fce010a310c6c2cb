// Two-pass imaginary-time FFT step for complex-FP32 lattices of N = 128 and N = 256
// (Eqs. HK1-HK3 and the update of Sec. 2), sm_103a.
//
// The 3D transform is reorganised so that a steady-state step reads and writes HBM in two
// passes instead of four.  The y transform of length N = 16 L (L = N / 16: 16 for N = 256,
// 8 for N = 128) is split four-step fashion, y = y_lo + L y_hi and k_y = k_lo + 16 k_hi
// (y_lo, k_hi < L; y_hi, k_lo < 16):
//   Y(k_lo + 16 k_hi) = sum_{y_lo} wL^{y_lo k_hi} [ wN^{y_lo k_lo}
//                        sum_{y_hi} w16^{y_hi k_lo} f(y_lo + L y_hi) ],
// and each half is attached to a pass that already holds the needed elements:
//   pass A  x forward + the inner 16-point DFTs over y_hi (+ twiddle), from a field in
//           natural order, into the scratch field S;
//   pass B  the outer L-point DFTs over y_lo, z forward, T(k), z inverse, the outer
//           inverse DFTs, S in place;
//   pass C  the inner inverse DFTs (+ conjugate twiddle), x inverse, the update of psi
//           (and the FP64 check sums), then pass A on psi_{t+1} for the next step.
// Steady state: B + C = 16 + (8 + 8 + 4 + 8 + 8) B per site (real V) instead of 84.
//
// S layout (the scratch field, N^3 elements): [kx_hi N/2][k_lo 16][y_lo L][z N][kx_lo 2]
// with kx = 2 kx_hi + kx_lo.  A pass-B block owns one (kx_hi, k_lo): 2 L N contiguous
// elements, and reads its outer y DFTs' inputs straight from global memory (a warp reads
// 256 contiguous bytes per y_lo).  A pass-A/C block owns one y_lo and the two z-planes
// z0, z0 + 1: the 32 lines y = y_lo + L y_hi of both planes, and in S one 32-byte
// sector (2 z x 2 kx_lo) per (kx_hi, k_lo).
//
// Every 1D transform of length N runs on TL = N / 16 threads with 16 elements each, in
// the two Stockham stages of the radix plan (16 x 16 for N = 256, 16 x 8 for N = 128).
// Register m of a thread holds position g + TL m before the first stage; after the last
// stage register i holds position g + TL f2_pos(i): the same positions in another order.
//
// Shared-memory layouts are padded for conflict-free access: the A/C line tile and the
// pass-B per-column buffers have a pitch of 8 (mod 16) elements with one pad element per
// 16; pass B's first exchange goes through a [k_hi][z][kx_lo] tile.
#pragma once
#include "qf_fft_impl.cuh"

namespace qf {

template <int N>
struct F2G {
  static_assert(N == 128 || N == 256, "the two-pass step is built for N = 128 and 256");
  static constexpr int L = N / 16;                     // y_lo values: outer DFT length
  static constexpr int TL = N / 16;                    // threads per line or z column
  static constexpr int RAD1 = plan_radix(N, 1);        // radix of the second stage
  static constexpr int PITCH = N == 256 ? 280 : 136;   // >= N + N/16, 8 mod 16
  static constexpr int TW = plan_tw_size(N);           // per-stage twiddles
  static constexpr int TW1 = plan_tw_off(N, 1);        // second-stage block: wN^{k r}
  static constexpr int TWB = (TW * 8 + 15) / 16 * 16;  // twiddle bytes in shared memory
  // pass B: one (kx_hi, k_lo) block of [y_lo L][z N][kx_lo 2]
  static constexpr int B_ELEMS = 2 * L * N;
  static constexpr int B_THREADS = B_ELEMS / 16;       // 512 / 128
  static constexpr int B_BLOCKS = N / 2 * 16;          // 2048 / 1024
  static constexpr int B_PER_SM = 1024 / B_THREADS;    // resident blocks per SM (64 registers)
  static constexpr int PAIRS = 16 / L;                 // (z, kx_lo) pairs per thread, outer role
  static constexpr int KPW = 16 / TL;                  // k_hi values per warp, z role
  static constexpr int B_TILE = B_ELEMS > 2 * L * PITCH ? B_ELEMS : 2 * L * PITCH;
  static constexpr size_t SMEM_B = TWB + N * 4 + (size_t)B_TILE * 8 + 32 * kNumSums * 8;
  static constexpr long long SKLO = B_ELEMS;           // S stride of k_lo
  // pass A / C: one y_lo of two z-planes
  static constexpr int LINES = 32;
  static constexpr int AC_THREADS = LINES * TL;        // 512 / 256
  static constexpr int AC_BLOCKS = L * N / 2;          // 2048 / 512
  static constexpr int AC_PER_SM = 1024 / AC_THREADS;
  static constexpr size_t SMEM_AC = TWB + (size_t)LINES * PITCH * 8 + 32 * kNumSums * 8;
};

// Register i after the last Stockham stage holds position g + TL f2_pos(i).
template <int N>
__host__ __device__ constexpr int f2_pos(int i) {
  return i / F2G<N>::RAD1 + (i % F2G<N>::RAD1) * (16 / F2G<N>::TL);
}
// f2_pos against the Stockham output index of the second stage (Ns = 16: the butterfly
// j = g + b TL < 16 writes j + 16 r)
template <int N>
constexpr bool f2_pos_consistent() {
  constexpr int RAD1 = F2G<N>::RAD1, TL = F2G<N>::TL;
  if (plan_stages(N) != 2 || plan_radix(N, 0) != 16 || plan_ns(N, 1) != 16 || RAD1 != F2G<N>::L) return false;
  for (int i = 0; i < 16; ++i) {
    const int b = i / RAD1, r = i % RAD1;
    if (b * TL + (TL - 1) >= 16 || b * TL + 16 * r != TL * f2_pos<N>(i)) return false;
  }
  return true;
}
static_assert(f2_pos_consistent<128>() && f2_pos_consistent<256>(), "two-pass register order");

// last-stage register order -> first-stage order (renaming only once unrolled)
template <int N>
__device__ __forceinline__ void f2_to_first_order(cpx<float> (&v)[16]) {
  if constexpr (F2G<N>::RAD1 != 16) {
    cpx<float> t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[f2_pos<N>(i)] = v[i];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = t[i];
  }
}

// wN^{y_lo k_lo} (forward) from the second-stage twiddle block, entries [k][r - 1] =
// wN^{k r} for k < 16, r < L
template <int N>
__device__ __forceinline__ cpx<float> f2_tw(const cpx<float>* tw_s, int ylo, int klo) {
  constexpr int L = F2G<N>::L, TW1 = F2G<N>::TW1;
  if constexpr (L == 16) return klo == 0 ? mk<float>(1.f, 0.f) : tw_s[TW1 + ylo * 15 + klo - 1];
  else return ylo == 0 ? mk<float>(1.f, 0.f) : tw_s[TW1 + klo * (L - 1) + ylo - 1];
}

template <int N>
__device__ __forceinline__ int f2_tile(int line, int e) { return line * F2G<N>::PITCH + e + (e >> 4); }
// B exchange buffer position: one pad element per 16 (the column pitch is 8 mod 16
// between the two kx_lo buffers of a half-warp), so both Stockham access patterns are
// conflict-free
__device__ __forceinline__ int f2_bpad(int p) { return p + (p >> 4); }

// Blocks are dispatched roughly in index order, per_sm per SM at a time, so block
// b + per_sm x (SM count) runs about one wave after block b: passes A and B pull that
// block's inputs into L2 while they work, and the next wave finds them there instead of
// waiting on HBM.
__device__ __forceinline__ int f2_next_wave_block(int per_sm) {
  unsigned nsm;
  asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
  return (int)blockIdx.x + per_sm * (int)nsm;
}
__device__ __forceinline__ void f2_prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// Programmatic dependent launch: a pass launched with programmatic stream serialization
// may start while the kernel before it in the stream is still running.  Every pass
// issues only L2 prefetch hints before this point and reads nothing else, then waits for
// the previous kernel to complete with its writes visible, and lets the next pass launch
// once all of its own blocks are running.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void f2_grid_dependency() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Offset of line `line` of pass-A/C block blk in a natural-order field: the block holds
// y_lo = blk mod L of the z-planes 2 (blk / L) and 2 (blk / L) + 1; line = 2 y_hi + dz.
template <int N>
__device__ __forceinline__ long long f2_row(int blk, int line) {
  constexpr int L = F2G<N>::L;
  const int z = 2 * (blk / L) + (line & 1), y = blk % L + L * (line >> 1);
  return ((long long)z * N + y) * N;
}

// x transform of this thread's 16 elements of its line (first-stage order in, last-stage
// order out), through the line tile for the stage exchange.  A line belongs to TL lanes of
// one warp and its tile row to those lanes alone (callers separate block-wide tile use
// with __syncthreads), so the exchange needs only warp synchronisation.
template <int N, bool INV>
__device__ __forceinline__ void f2_x_transform(cpx<float> (&v)[16], int line, int g, cpx<float>* tile,
                                               const cpx<float>* tw_s) {
  constexpr int RAD1 = F2G<N>::RAD1;
  stage_compute<float, N, 0, INV>(v, g, tw_s);
  __syncwarp();  // the line's earlier reads of its tile row are done
#pragma unroll
  for (int r = 0; r < 16; ++r) tile[f2_tile<N>(line, 16 * g + r)] = v[r];
  __syncwarp();
#pragma unroll
  for (int b = 0; b < 16 / RAD1; ++b)
#pragma unroll
    for (int r = 0; r < RAD1; ++r) v[b * RAD1 + r] = tile[f2_tile<N>(line, e_in<N, 1>(g, b, r))];
  stage_compute<float, N, 1, INV>(v, g, tw_s);
}

// Thread roles in a pass-A/C block (one y_lo, z-planes z0 and z0 + 1).
template <int N>
struct F2Roles {
  int z0, ylo;            // the block's first z-plane and its y_lo
  int line, g;            // x role: line 2 y_hi + s, element group g
  int kx, s;              // cross role: column kx of the lines of z-plane z0 + s
  long long row;          // natural offset of line `line`
  long long sbase;        // S offset of (kx_hi, k_lo = 0, y_lo, z0 + s, kx_lo)
  __device__ __forceinline__ F2Roles(int blk) {
    constexpr int L = F2G<N>::L, TL = F2G<N>::TL;
    z0 = 2 * (blk / L);
    ylo = blk % L;
    const int tid = threadIdx.x;
    line = tid / TL;
    g = tid % TL;
    row = f2_row<N>(blk, line);
    const int kxlo = tid & 1;
    s = (tid >> 1) & 1;
    const int kxhi = tid >> 2;
    kx = 2 * kxhi + kxlo;
    sbase = ((long long)kxhi * 16 * L + ylo) * (2 * N) + 2 * (z0 + s) + kxlo;
  }
};

// Cross stage forward: line tile (x-transformed) -> 16-point DFTs over y_hi, twiddle,
// store into S.
template <int N>
__device__ __forceinline__ void f2_cross_fwd(const F2Roles<N>& q, const cpx<float>* tile, const cpx<float>* tw_s,
                                             cpx<float>* S) {
  cpx<float> u[16];
#pragma unroll
  for (int yh = 0; yh < 16; ++yh) u[yh] = tile[f2_tile<N>(2 * yh + q.s, q.kx)];
  dft16<float, false>(u);
#pragma unroll
  for (int k = 0; k < 16; ++k) S[q.sbase + k * F2G<N>::SKLO] = cmul<float>(u[k], f2_tw<N>(tw_s, q.ylo, k));
}

// x-transformed line values (last-stage order) -> the line tile
template <int N>
__device__ __forceinline__ void f2_store_lines(const F2Roles<N>& q, const cpx<float> (&v)[16], cpx<float>* tile) {
#pragma unroll
  for (int i = 0; i < 16; ++i) tile[f2_tile<N>(q.line, q.g + F2G<N>::TL * f2_pos<N>(i))] = v[i];
}

// Pass A: field `src` (natural order) -> S.  With SUMS (energy of a field that is not
// stepped): also <src|src> and <src|V src> of its sites into partial row blockIdx.x; the
// kinetic part comes from pass B in k-space.
template <int N, bool SUMS = false>
__global__ void __launch_bounds__(F2G<N>::AC_THREADS, F2G<N>::AC_PER_SM)
    fft2_a_kernel(const __grid_constant__ FftGroup<float> gr) {
  using G = F2G<N>;
  const FftPassArgs<float>& a = gr.a[blockIdx.y];
  extern __shared__ __align__(16) unsigned char f2_smem[];
  cpx<float>* tw_s = reinterpret_cast<cpx<float>*>(f2_smem);
  cpx<float>* tile = reinterpret_cast<cpx<float>*>(f2_smem + G::TWB);
  const F2Roles<N> q(blockIdx.x);
  f2_grid_dependency();
  const cpx<float>* __restrict__ src = a.src ? a.src : a.psi;
  cpx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = src[q.row + q.g + G::TL * r];
  CheckSums<float> cs;
  if constexpr (SUMS) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const long long site = q.row + q.g + G::TL * r;
      const cpx<float> vi = a.v_real ? mk<float>(reinterpret_cast<const float*>(a.v)[site], 0.f)
                                     : reinterpret_cast<const cpx<float>*>(a.v)[site];
      cs.add(v[r], mk<float>(0.f, 0.f), vi);
    }
  }
  {
    const int nb = f2_next_wave_block(G::AC_PER_SM);
    if (nb < (int)gridDim.x && threadIdx.x < G::LINES) f2_prefetch_l2(src + f2_row<N>(nb, threadIdx.x), N * 8);
  }
  for (int i = threadIdx.x; i < G::TW; i += G::AC_THREADS) tw_s[i] = a.twiddle[i];
  __syncthreads();
  f2_x_transform<N, false>(v, q.line, q.g, tile, tw_s);
  __syncwarp();
  f2_store_lines<N>(q, v, tile);
  __syncthreads();
  f2_cross_fwd<N>(q, tile, tw_s, a.data);
  if constexpr (SUMS) {
    double acc[kNumSums];
    cs.to(acc);
    block_sum_store<kNumSums>(acc, reinterpret_cast<double*>(tile + G::LINES * G::PITCH),
                              a.partials + (long long)blockIdx.x * kPartialStride);
  }
}

// Pass B: S in place, one (kx_hi, k_lo) block of 2 L N contiguous elements [y_lo][z][kx_lo].
//   outer y DFTs: thread pairs (z, kx_lo) p = tid + B_THREADS q, q < 16 / L, read their L
//     y_lo values straight from global memory (a warp reads 256 contiguous bytes per y_lo)
//     -> natural k_hi;
//   exchange 1 through the [k_hi][z][kx_lo] tile to the z role: warp w holds k_hi =
//     w KPW + lane / (2 TL), lanes (z1, kx_lo) = ((lane / 2) mod TL, lane mod 2) holding
//     z = z1 + TL m;
//   z forward, T(k), z inverse: Stockham stages with warp-local exchanges through padded
//     per-column buffers (which reuse the tile);
//   exchange 2 back to the pairs, inverse outer y DFTs, written straight to global memory.
// Four shared-memory round trips per element.  With SUMS (energy of a field that is not
// stepped): after the z forward transform, <v|H_K v> = sum_k T(k)/N^3 |v^(k)|^2
// (Parseval) into partial row row0 + blockIdx.x, and nothing is written back.
template <int N, bool SUMS = false>
__global__ void __launch_bounds__(F2G<N>::B_THREADS, F2G<N>::B_PER_SM)
    fft2_b_kernel(const __grid_constant__ FftGroup<float> gr, int row0 = 0) {
  using G = F2G<N>;
  constexpr int L = G::L, TL = G::TL, RAD1 = G::RAD1, BT = G::B_THREADS;
  const FftPassArgs<float>& a = gr.a[blockIdx.y];
  extern __shared__ __align__(16) unsigned char f2_smem[];
  cpx<float>* tw_s = reinterpret_cast<cpx<float>*>(f2_smem);
  float* sym_s = reinterpret_cast<float*>(f2_smem + G::TWB);
  cpx<float>* tile = reinterpret_cast<cpx<float>*>(reinterpret_cast<unsigned char*>(sym_s) + N * 4);
  const int blk = blockIdx.x, kxhi = blk >> 4, klo = blk & 15;
  const int tid = threadIdx.x;
  cpx<float>* base = a.data + (long long)blk * G::B_ELEMS;
  {
    const int nb = f2_next_wave_block(G::B_PER_SM);
    if (nb < (int)gridDim.x && tid < 4)
      f2_prefetch_l2(a.data + (long long)nb * G::B_ELEMS + tid * (G::B_ELEMS / 4), G::B_ELEMS / 4 * 8);
  }
  f2_grid_dependency();
  cpx<float> u[16];
#pragma unroll
  for (int q = 0; q < G::PAIRS; ++q)
#pragma unroll
    for (int y = 0; y < L; ++y) u[q * L + y] = base[y * 2 * N + tid + BT * q];
  for (int i = tid; i < G::TW; i += BT) tw_s[i] = a.twiddle[i];
  for (int i = tid; i < N; i += BT) sym_s[i] = a.symbol[i];
#pragma unroll
  for (int q = 0; q < G::PAIRS; ++q) dft<float, L, false>(&u[q * L]);
#pragma unroll
  for (int q = 0; q < G::PAIRS; ++q)
#pragma unroll
    for (int k = 0; k < L; ++k) tile[k * 2 * N + tid + BT * q] = u[q * L + k];
  __syncthreads();
  // z role
  const int w = tid >> 5, lane = tid & 31, kxl = lane & 1, z1 = (lane >> 1) % TL;
  const int khi = w * G::KPW + (lane >> 1) / TL;
  cpx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = tile[khi * 2 * N + 2 * (z1 + TL * r) + kxl];
  __syncthreads();  // the tile becomes the per-column exchange buffers
  cpx<float>* wb = tile + (2 * khi + kxl) * G::PITCH;
  stage_compute<float, N, 0, false>(v, z1, tw_s);
#pragma unroll
  for (int r = 0; r < 16; ++r) wb[f2_bpad(16 * z1 + r)] = v[r];
  __syncwarp();
#pragma unroll
  for (int b = 0; b < 16 / RAD1; ++b)
#pragma unroll
    for (int r = 0; r < RAD1; ++r) v[b * RAD1 + r] = wb[f2_bpad(e_in<N, 1>(z1, b, r))];
  stage_compute<float, N, 1, false>(v, z1, tw_s);
  // kz = z1 + TL f2_pos(i); T(kx, ky, kz)/N^3 with ky = k_lo + 16 k_hi
  {
    const int kx = 2 * kxhi + kxl, ky = klo + 16 * khi;
    const float sxy = sym_s[kx] + sym_s[ky];
    if constexpr (SUMS) {
      CheckSums<float> cs;
#pragma unroll
      for (int i = 0; i < 16; ++i)
        cs.add(v[i],
               cscale<float>(v[i], kin_mult<float>(a.kinetic, sxy, sym_s[z1 + TL * f2_pos<N>(i)], a.tcoef, a.am2)),
               mk<float>(0.f, 0.f));
      double acc[kNumSums];
      cs.to(acc);
      acc[0] = acc[3] = acc[4] = 0.0;  // norm and potential terms come from pass A
      block_sum_store<kNumSums>(acc, reinterpret_cast<double*>(tile + G::B_TILE),
                                a.partials + (long long)(row0 + blockIdx.x) * kPartialStride);
      return;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i)
      v[i] = cscale<float>(v[i], kin_mult<float>(a.kinetic, sxy, sym_s[z1 + TL * f2_pos<N>(i)], a.tcoef, a.am2));
  }
  f2_to_first_order<N>(v);
  stage_compute<float, N, 0, true>(v, z1, tw_s);
  __syncwarp();  // (the buffer's own lanes are its only readers)
#pragma unroll
  for (int r = 0; r < 16; ++r) wb[f2_bpad(16 * z1 + r)] = v[r];
  __syncwarp();
#pragma unroll
  for (int b = 0; b < 16 / RAD1; ++b)
#pragma unroll
    for (int r = 0; r < RAD1; ++r) v[b * RAD1 + r] = wb[f2_bpad(e_in<N, 1>(z1, b, r))];
  stage_compute<float, N, 1, true>(v, z1, tw_s);
  __syncthreads();  // every warp is done with its buffers
#pragma unroll
  for (int i = 0; i < 16; ++i) tile[khi * 2 * N + 2 * (z1 + TL * f2_pos<N>(i)) + kxl] = v[i];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < G::PAIRS; ++q)
#pragma unroll
    for (int k = 0; k < L; ++k) u[q * L + k] = tile[k * 2 * N + tid + BT * q];
#pragma unroll
  for (int q = 0; q < G::PAIRS; ++q) dft<float, L, true>(&u[q * L]);
#pragma unroll
  for (int q = 0; q < G::PAIRS; ++q)
#pragma unroll
    for (int y = 0; y < L; ++y) base[y * 2 * N + tid + BT * q] = u[q * L + y];
}

// Pass C: S -> inverse inner y DFTs, x inverse -> H_K psi; update / sums; with NEXT, pass A
// on psi_{t+1} into S.  OP: OP_FINAL (write), OP_FINAL_SUMS (write + sums), OP_SUMS.
// Everything of pass C after the scratch values u (this thread's 16 k_lo values of its
// cross-role column) are in registers: block `item`.
template <int N, int OP, bool VREAL, bool NEXT>
__device__ __forceinline__ void f2_c_body(const FftPassArgs<float>& a, const F2Roles<N>& q, cpx<float> (&u)[16],
                                          cpx<float>* tile, const cpx<float>* tw_s, double* red_s, int item) {
  constexpr bool WRITE = (OP == OP_FINAL || OP == OP_FINAL_SUMS);
  constexpr bool SUMS = (OP == OP_FINAL_SUMS || OP == OP_SUMS);
  constexpr int TL = F2G<N>::TL;
#pragma unroll
  for (int k = 0; k < 16; ++k) u[k] = cmulc<float>(u[k], f2_tw<N>(tw_s, q.ylo, k));
  dft16<float, true>(u);
#pragma unroll
  for (int yh = 0; yh < 16; ++yh) tile[f2_tile<N>(2 * yh + q.s, q.kx)] = u[yh];
  __syncthreads();
  cpx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = tile[f2_tile<N>(q.line, q.g + TL * r)];
  f2_x_transform<N, true>(v, q.line, q.g, tile, tw_s);
  // v[i] = H_K psi at x = g + TL f2_pos(i) of row `row` (1/N^3 inside T); psi and V are
  // read site by site (registers are the limit)
  CheckSums<float> cs;
  const float sc = WRITE ? float(*a.scale) : 1.f;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const long long site = q.row + q.g + TL * f2_pos<N>(i);
    const cpx<float> pv = a.psi[site];
    cpx<float> vi;
    if constexpr (VREAL) vi = mk<float>(reinterpret_cast<const float*>(a.v)[site], 0.f);
    else vi = reinterpret_cast<const cpx<float>*>(a.v)[site];
    if constexpr (SUMS) cs.add(pv, v[i], vi);
    if constexpr (WRITE) {
      // d = 1 + dtau V/2; coef_B = 1/d; coef_A = (2 - d)/d
      if constexpr (VREAL) {
        const float d = 1.f + a.half_dtau * vi.x;
        const cpx<float> num = cscale<float>(pv, 2.f - d) - cscale<float>(v[i], a.dtau);
        v[i] = cscale<float>(num, __fdividef(sc, d));  // psi_{t+1}
      } else {
        const cpx<float> d = mk<float>(1.f + a.half_dtau * vi.x, a.half_dtau * vi.y);
        const cpx<float> num = cmul<float>(mk<float>(2.f - d.x, -d.y), pv) - cscale<float>(v[i], a.dtau);
        const float inv = __fdividef(sc, d.x * d.x + d.y * d.y);
        v[i] = cscale<float>(cmulc<float>(num, d), inv);  // psi_{t+1}
      }
      a.psi[site] = v[i];
    }
  }
  if constexpr (SUMS) {
    double acc[kNumSums];
    cs.to(acc);
    block_sum_store<kNumSums>(acc, red_s, a.partials + ((long long)item) * kPartialStride);
  }
  if constexpr (WRITE && NEXT) {
    f2_to_first_order<N>(v);
    f2_x_transform<N, false>(v, q.line, q.g, tile, tw_s);
    __syncwarp();
    f2_store_lines<N>(q, v, tile);
    __syncthreads();
    f2_cross_fwd<N>(q, tile, tw_s, a.data);
  }
}

// L2 prefetch of psi and V of the output rows of pass-C block `item` (threads < 2 LINES).
template <int N, bool VREAL>
__device__ __forceinline__ void f2_prefetch_psi_v(const FftPassArgs<float>& a, int item) {
  constexpr int LINES = F2G<N>::LINES;
  if (threadIdx.x < 2 * LINES) {
    const long long row = f2_row<N>(item, threadIdx.x % LINES);
    if (threadIdx.x < LINES) f2_prefetch_l2(a.psi + row, N * 8);
    else if (VREAL) f2_prefetch_l2(reinterpret_cast<const float*>(a.v) + row, N * 4);
    else f2_prefetch_l2(reinterpret_cast<const cpx<float>*>(a.v) + row, N * 8);
  }
}

template <int N, int OP, bool VREAL, bool NEXT>
__global__ void __launch_bounds__(F2G<N>::AC_THREADS, F2G<N>::AC_PER_SM)
    fft2_c_kernel(const __grid_constant__ FftGroup<float> gr) {
  using G = F2G<N>;
  const FftPassArgs<float>& a = gr.a[blockIdx.y];
  extern __shared__ __align__(16) unsigned char f2_smem[];
  cpx<float>* tw_s = reinterpret_cast<cpx<float>*>(f2_smem);
  cpx<float>* tile = reinterpret_cast<cpx<float>*>(f2_smem + G::TWB);
  double* red_s = reinterpret_cast<double*>(tile + G::LINES * G::PITCH);
  const F2Roles<N> q(blockIdx.x);
  // psi and V of the output rows are needed only after the transforms: start pulling them
  // into L2 now, one bulk prefetch per row.  (Measured slower at N = 256: prefetching the
  // next wave's rows or scratch sectors here as well, this pass already moving 36 B per
  // site; and a persistent form with one block per SM that stages the next item's sectors
  // with cp.async while computing, 16 warps per SM being too few for the transforms.)
  f2_prefetch_psi_v<N, VREAL>(a, blockIdx.x);
  f2_grid_dependency();
  for (int i = threadIdx.x; i < G::TW; i += G::AC_THREADS) tw_s[i] = a.twiddle[i];
  cpx<float> u[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) u[k] = a.data[q.sbase + k * G::SKLO];
  __syncthreads();
  f2_c_body<N, OP, VREAL, NEXT>(a, q, u, tile, tw_s, red_s, blockIdx.x);
}

// Launch of one pass over a group (blockIdx.y = member); instantiated per N in
// qf_fft2.cu (N = 256) and qf_fft2_n128.cu (N = 128).
template <int N>
cudaError_t launch_fft2_pass_n(int pass, const FftGroup<float>& g, cudaStream_t st);

}  // namespace qf
