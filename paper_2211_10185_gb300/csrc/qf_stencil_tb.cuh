// Temporally blocked FDTD steps: two imaginary-time steps with the kinetic term of Eq.
// HK0 per pass over HBM (complex FP32 fields), sm_103a.
//
// Two consecutive steps read psi_t and V and write psi_{t+2}; the intermediate psi_{t+1}
// lives only in shared memory.  A block owns a 32 x 32 column tile of the output and
// marches through a chunk of z (chunk sizes differ by at most one plane, so the number of
// chunks can be chosen to fill whole waves of resident blocks).  Three levels are in flight at once:
//   level 0  psi_t on the tile plus a halo of 2 (36 x 36), streamed plane by plane with
//            cp.async.bulk.tensor into a ring of six buffers (each with an mbarrier);
//   level 1  psi_{t+1} on the tile plus a halo of 1 (34 x 34), computed one plane behind
//            level 0 into a ring of four buffers;
//   level 2  psi_{t+2} on the tile, computed two planes behind level 1 and stored.
// One block barrier per plane separates the levels: level 1 of plane p needs level-0
// planes p-1..p+1, level 2 of plane p needs level-1 planes p-1..p+1, and the ring slots
// written in an iteration are never the ones read in it.
//
// Sites with an index 0 (the Dirichlet planes) and sites outside the lattice are zero at
// every level; the input field must already be zero on the Dirichlet planes (true after
// any FDTD step).  Each site is computed with the same rounded operations as the
// single-step kernel, so two single steps and one blocked pass give the same bits.
//
// Every wait is bounded as in the single-step kernel: on time-out the block records a
// flag, drains its own copies with a bounded wait and returns.
//
// A group launch (stencil_tb_group_kernel) steps several lattices of any sizes at once:
// a one-dimensional grid whose blocks are numbered member by member from a block table,
// each block running the same body on its member's tile and z-chunk.
#pragma once
#include "qf_stencil_tma.cuh"

namespace qf {

constexpr int TB_X = 32, TB_Y = 32, TB_ROWS = 4;
constexpr int TB_THREADS = TB_X * (TB_Y / TB_ROWS);  // 256
constexpr int TB_W0 = TB_X + 4, TB_H0 = TB_Y + 4;    // level-0 box: halo 2
constexpr int TB_W1 = TB_X + 2, TB_H1 = TB_Y + 2;    // level-1 region: halo 1
constexpr int TB_D0 = 6, TB_D1 = 4;                  // ring depths
constexpr int TB_L0_WORDS = TB_W0 * TB_H0;           // 1296 complex = 10368 B (81 x 128 B)
constexpr int TB_L1_SITES = TB_W1 * TB_H1;           // 1156
constexpr int TB_L1_STRIDE = (TB_L1_SITES + 15) / 16 * 16;
constexpr int TB_L1_PER_THREAD = (TB_L1_SITES + TB_THREADS - 1) / TB_THREADS;  // 5
constexpr unsigned TB_L0_BYTES = TB_L0_WORDS * 8u;

struct alignas(64) StencilTbArgs {
  CUtensorMap map;        // input field psi_t, box TB_W0 x TB_H0 x 1 of 8-byte elements
  cpx<float>* out;        // psi_{t+2}
  const void* v;          // V: float (v_real) or complex float
  int v_real;
  float half_dtau;        // dtau / 2
  float kd;               // dtau / (2 m a^2)
  const double* scale;    // renormalisation applied in the first of the two steps
  int n;
  int nzb;                // z-chunks per column tile: chunk b holds planes [b n/nzb, (b+1) n/nzb)
  int* err;               // set to 1 when a bounded wait ran out
};

constexpr size_t stencil_tb_smem() { return (size_t)(TB_D0 * TB_L0_WORDS + TB_D1 * TB_L1_STRIDE) * 8; }

__device__ __forceinline__ void tb_plane(const CUtensorMap* map, unsigned long long* bar, void* dst, int x0, int y0,
                                         int z) {
  mbar_expect_tx(bar, TB_L0_BYTES);
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x0 - 2), "r"(y0 - 2), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// V at offset `off` of plane p (the plane's base address computed once per plane)
template <bool VREAL>
__device__ __forceinline__ cpx<float> tb_v(const StencilTbArgs& g, long long plane_off, int off) {
  if constexpr (VREAL) return mk<float>((reinterpret_cast<const float*>(g.v) + plane_off)[off], 0.f);
  else return (reinterpret_cast<const cpx<float>*>(g.v) + plane_off)[off];
}

// Members of a group launch: blocks of member i are start[i] .. start[i+1] - 1 (the
// launcher fills start), each member (n/32)^2 nzb blocks.  All members have the same kind
// of potential (v_real).
struct StencilTbGroup {
  StencilTbArgs m[kGroupMax];
  int start[kGroupMax + 1];
  int count;
};

__host__ __device__ inline int stencil_tb_member_blocks(int n, int nzb) {
  return ((n + TB_X - 1) / TB_X) * ((n + TB_Y - 1) / TB_Y) * nzb;
}

// The two steps for column tile (bx, by) and z-chunk bz of the lattice in g.  VREAL: the
// potential is real (g.v holds floats).  g must live in kernel parameter space (its
// tensor map is read by the copies).
template <bool VREAL>
__device__ __forceinline__ void stencil_tb_body(const StencilTbArgs& g, int bx, int by, int bz) {
  extern __shared__ __align__(128) unsigned long long tb_dyn[];
  cpx<float>* l0 = reinterpret_cast<cpx<float>*>(tb_dyn);
  cpx<float>* l1 = l0 + TB_D0 * TB_L0_WORDS;
  __shared__ alignas(8) unsigned long long bars[TB_D0];
  const int n = g.n;
  const long long plane_sites = (long long)n * n;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int x0 = bx * TB_X, y0 = by * TB_Y;
  const int z0 = (int)((long long)bz * n / g.nzb), z1 = (int)((long long)(bz + 1) * n / g.nzb);
  const int pbase = z0 - 2, last0 = z1 + 1;  // level-0 planes z0-2 .. z1+1
  const float hd = g.half_dtau, kd = g.kd;
  const float sc1 = (float)*g.scale;

  // level-1 sites of this thread: flat index i = tid + 256 q over the 34 x 34 region
  int o0[TB_L1_PER_THREAD], o1[TB_L1_PER_THREAD], gs[TB_L1_PER_THREAD];
  bool in1[TB_L1_PER_THREAD], has1[TB_L1_PER_THREAD];
#pragma unroll
  for (int q = 0; q < TB_L1_PER_THREAD; ++q) {
    const int i = tid + TB_THREADS * q;
    const int ly = i / TB_W1, lx = i - ly * TB_W1;
    const int x = x0 - 1 + lx, y = y0 - 1 + ly;
    has1[q] = i < TB_L1_SITES;
    in1[q] = has1[q] && x >= 1 && x < n && y >= 1 && y < n;
    o0[q] = (ly + 1) * TB_W0 + lx + 1;
    o1[q] = ly * TB_W1 + lx;
    gs[q] = in1[q] ? y * n + x : 0;
  }
  // output sites: column x0 + tx, rows y0 + 4 ty .. y0 + 4 ty + 3
  const int ox = x0 + tx, oy = y0 + TB_ROWS * ty;
  bool in2[TB_ROWS], st2[TB_ROWS];
#pragma unroll
  for (int k = 0; k < TB_ROWS; ++k) {
    st2[k] = ox < n && oy + k < n;
    in2[k] = st2[k] && ox >= 1 && oy + k >= 1;
  }
  const int o2 = oy * n + ox;  // in-plane offset of this thread's first output row
  auto load_v1 = [&](int p, cpx<float>(&v)[TB_L1_PER_THREAD]) {
    const bool zin = p >= 1 && p < n;
    const long long po = zin ? p * plane_sites : 0;
#pragma unroll
    for (int q = 0; q < TB_L1_PER_THREAD; ++q)
      v[q] = (zin && in1[q]) ? tb_v<VREAL>(g, po, gs[q]) : mk<float>(0.f, 0.f);
  };
  auto load_v2 = [&](int p, cpx<float>(&v)[TB_ROWS]) {
    const bool zin = p >= 1 && p < n;
    const long long po = zin ? p * plane_sites : 0;
#pragma unroll
    for (int k = 0; k < TB_ROWS; ++k)
      v[k] = (zin && in2[k]) ? tb_v<VREAL>(g, po, o2 + k * n) : mk<float>(0.f, 0.f);
  };

  if (tid == 0) {
    for (int b = 0; b < TB_D0; ++b) mbar_init(&bars[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  int issued = pbase - 1;
  if (tid == 0)
    for (int p = pbase; p <= last0 && p < pbase + TB_D0; ++p) {
      tb_plane(&g.map, &bars[p - pbase], l0 + (p - pbase) * TB_L0_WORDS, x0, y0, p);
      issued = p;
    }
  cpx<float> v1n[TB_L1_PER_THREAD], v2n[TB_ROWS];
  load_v1(z0 - 1, v1n);
  load_v2(z0 - 2, v2n);
  int waited = pbase - 1;
  bool ok = true;
  for (int j = z0; j <= z1 + 2; ++j) {
    cpx<float> v1c[TB_L1_PER_THREAD], v2c[TB_ROWS];
#pragma unroll
    for (int q = 0; q < TB_L1_PER_THREAD; ++q) v1c[q] = v1n[q];
#pragma unroll
    for (int k = 0; k < TB_ROWS; ++k) v2c[k] = v2n[k];
    if (j <= z1) load_v1(j, v1n);       // level-1 plane of the next iteration
    if (j - 2 >= z0) load_v2(j - 2, v2n);  // level-2 plane of the next iteration
    // level-0 planes up to j must have landed: thread 0 polls (bounded), the block learns
    // the outcome at the barrier, then every thread observes the completed phases itself
    const int need = min(j, last0);
    bool mine = true;
    if (tid == 0)
      while (waited < need && mine) {
        const int u = waited + 1 - pbase;
        mine = mbar_wait_bounded(&bars[u % TB_D0], (unsigned)((u / TB_D0) & 1));
        if (mine) ++waited;
      }
    ok = __syncthreads_and(mine) != 0;
    if (!ok) break;
    if (tid != 0)
      for (; waited < need; ++waited) {
        const int u = waited + 1 - pbase;
        mbar_try_wait(&bars[u % TB_D0], (unsigned)((u / TB_D0) & 1));  // completed: returns at once
      }
    // the slot of level-0 plane j-3 was last read in the previous iteration
    if (tid == 0 && issued < last0 && issued + 1 <= j + 3) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      const int p = issued + 1;
      tb_plane(&g.map, &bars[(p - pbase) % TB_D0], l0 + ((p - pbase) % TB_D0) * TB_L0_WORDS, x0, y0, p);
      issued = p;
    }
    // level 1: psi_{t+1} on plane j-1 (halo 1)
    if (j - 1 <= z1) {
      const int p = j - 1;
      const bool zin = p >= 1 && p < n;
      const cpx<float>* am = l0 + ((p - 1 - pbase) % TB_D0) * TB_L0_WORDS;
      const cpx<float>* ac = l0 + ((p - pbase) % TB_D0) * TB_L0_WORDS;
      const cpx<float>* ap = l0 + ((p + 1 - pbase) % TB_D0) * TB_L0_WORDS;
      cpx<float>* w = l1 + ((p - (z0 - 1)) % TB_D1) * TB_L1_STRIDE;
      // branch-free: every position is computed (halo and wall positions read zeros or
      // finite values) and the Dirichlet/outside ones are replaced by 0; only the last
      // round of the flat index is partial
#pragma unroll
      for (int q = 0; q < TB_L1_PER_THREAD; ++q) {
        if (q == TB_L1_PER_THREAD - 1 && !has1[q]) break;
        const int o = o0[q];
        const cpx<float> c = ac[o];
        const cpx<float> lap =
            lap_of<float>(c, six_sum<float>(ac[o - 1], ac[o + 1], ac[o - TB_W0], ac[o + TB_W0], am[o], ap[o]));
        const cpx<float> u = fdtd_update<float>(c, lap, v1c[q], VREAL, hd, kd, sc1);
        const bool live = zin && in1[q];
        w[o1[q]] = mk<float>(live ? u.x : 0.f, live ? u.y : 0.f);
      }
    }
    // level 2: psi_{t+2} on plane j-3 (the tile), stored
    if (j - 3 >= z0) {
      const int p = j - 3;
      const bool zin = p >= 1 && p < n;
      const cpx<float>* bm = l1 + ((p - 1 - (z0 - 1)) % TB_D1) * TB_L1_STRIDE;
      const cpx<float>* bc = l1 + ((p - (z0 - 1)) % TB_D1) * TB_L1_STRIDE;
      const cpx<float>* bp = l1 + ((p + 1 - (z0 - 1)) % TB_D1) * TB_L1_STRIDE;
      // column of the centre plane: local rows 4 ty .. 4 ty + 5 (level-1 coordinates)
      const int base = (TB_ROWS * ty) * TB_W1 + tx + 1;
      cpx<float> col[TB_ROWS + 2];
#pragma unroll
      for (int k = 0; k < TB_ROWS + 2; ++k) col[k] = bc[base + k * TB_W1];
      cpx<float>* dst = g.out + (p * (long long)n + oy) * n + ox;
#pragma unroll
      for (int k = 0; k < TB_ROWS; ++k) {
        const int o = base + (k + 1) * TB_W1;
        const cpx<float> c = col[k + 1];
        const cpx<float> lap = lap_of<float>(c, six_sum<float>(bc[o - 1], bc[o + 1], col[k], col[k + 2], bm[o], bp[o]));
        const cpx<float> u = fdtd_update<float>(c, lap, v2c[k], VREAL, hd, kd, 1.0f);
        const bool live = zin && in2[k];
        if (st2[k]) dst[(long long)k * n] = mk<float>(live ? u.x : 0.f, live ? u.y : 0.f);
      }
    }
  }
  if (!ok && tid == 0) {
    atomicExch(g.err, 1);
    // copies already issued may still land in this block's shared memory
    for (int p = waited + 1; p <= issued; ++p) {
      const int u = p - pbase;
      mbar_wait_bounded(&bars[u % TB_D0], (unsigned)((u / TB_D0) & 1));
    }
  }
}

template <bool VREAL>
__global__ void __launch_bounds__(TB_THREADS, 2) stencil_tb_kernel(const __grid_constant__ StencilTbArgs g) {
  stencil_tb_body<VREAL>(g, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <bool VREAL>
__global__ void __launch_bounds__(TB_THREADS, 2) stencil_tb_group_kernel(const __grid_constant__ StencilTbGroup gr) {
  // member of this block: the last i with start[i] <= block
  int member = 0;
  {
    int hi = gr.count - 1;
    while (member < hi) {
      const int mid = (member + hi + 1) >> 1;
      if (gr.start[mid] <= (int)blockIdx.x) member = mid;
      else hi = mid - 1;
    }
  }
  const StencilTbArgs& g = gr.m[member];
  const int nbx = (g.n + TB_X - 1) / TB_X, nby = (g.n + TB_Y - 1) / TB_Y;
  const int local = (int)blockIdx.x - gr.start[member];
  stencil_tb_body<VREAL>(g, local % nbx, (local / nbx) % nby, local / (nbx * nby));
}

}  // namespace qf
