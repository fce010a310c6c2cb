// Fused 3D FFT kinetic step (Eqs. HK1-HK3) with the imaginary-time update, sm_103a.
//
// One step is five passes over the lattice, each a batch of 1D transforms of length N
// held in registers and shared memory:
//   1. x forward (reads psi, writes tmp)          2. y forward (tmp in place)
//   3. z forward -> x T(k) -> z inverse (tmp)      4. y inverse (tmp in place)
//   5. x inverse -> H_K psi in registers -> psi' = s (coef_A psi - coef_B dtau H_K psi),
//      FP64 norm/energy partial sums on check steps (psi in place).
// The 1D transforms use the self-sorting Stockham formulation of Govindaraju et al.,
// "High performance discrete Fourier transforms on graphics processors" (SC08): at a
// stage of radix R after sub-transforms of size Ns, butterfly j reads x[j + r N/R],
// multiplies by exp(-+2 pi i r (j mod Ns)/(Ns R)), does an R-point DFT and writes
// y[(j/Ns) Ns R + (j mod Ns) + r Ns], so the output is in natural order.  The first
// stage reads global memory and the last writes it directly (both coalesced);
// intermediate stages exchange through shared memory.
#pragma once
#include "qf_common.cuh"

namespace qf {

// ------------------------------------------------------------------------------------
// Radix plans.  EPT = elements per thread = lcm of the radices.  Plan 0 is the default of
// each size; sizes with has_alt_plan also have plan 1, a radix-16 first stage with 16
// elements per thread (half the threads per line), which the autotuner times against
// plan 0 (tile variants 2 and 3 below).
// ------------------------------------------------------------------------------------
constexpr bool has_alt_plan(int n) { return n == 32 || n == 64 || n == 512; }
constexpr int alt_plan_stages(int n) { return n == 32 ? 2 : n == 64 ? 2 : n == 512 ? 3 : 0; }
constexpr int alt_plan_radix(int n, int s) {
  return n == 32 ? (s == 0 ? 16 : 2) : n == 64 ? (s == 0 ? 16 : 4) : n == 512 ? (s == 0 ? 16 : s == 1 ? 8 : 4) : 0;
}
constexpr int plan_stages0(int n) {
  return n == 8 ? 1 : n == 16 ? 1 : n == 12 ? 2 : n == 24 ? 2 : n == 32 ? 2 : n == 48 ? 3
       : n == 64 ? 2 : n == 96 ? 3 : n == 128 ? 2 : n == 192 ? 3 : n == 256 ? 2 : n == 384 ? 4
       : n == 512 ? 3 : 0;
}
constexpr int plan_radix0(int n, int s) {
  return n == 8 ? 8
       : n == 16 ? 16
       : n == 12 ? (s == 0 ? 4 : 3)
       : n == 24 ? (s == 0 ? 8 : 3)
       : n == 32 ? (s == 0 ? 8 : 4)
       : n == 48 ? (s == 2 ? 3 : 4)
       : n == 64 ? 8
       : n == 96 ? (s == 0 ? 8 : s == 1 ? 4 : 3)
       : n == 128 ? (s == 0 ? 16 : 8)
       : n == 192 ? (s == 2 ? 3 : 8)
       : n == 256 ? 16
       : n == 384 ? (s == 0 ? 8 : s == 3 ? 3 : 4)
       : n == 512 ? 8 : 0;
}
constexpr int plan_ept0(int n) {
  return n == 8 ? 8 : n == 16 ? 16 : n == 12 ? 12 : n == 24 ? 24 : n == 32 ? 8 : n == 48 ? 12
       : n == 64 ? 8 : n == 96 ? 24 : n == 128 ? 16 : n == 192 ? 24 : n == 256 ? 16
       : n == 384 ? 24 : n == 512 ? 8 : 0;
}
constexpr bool use_alt(int n, int p) { return p == 1 && has_alt_plan(n); }
constexpr int plan_stages(int n, int p = 0) { return use_alt(n, p) ? alt_plan_stages(n) : plan_stages0(n); }
constexpr int plan_radix(int n, int s, int p = 0) { return use_alt(n, p) ? alt_plan_radix(n, s) : plan_radix0(n, s); }
constexpr int plan_ept(int n, int p = 0) { return use_alt(n, p) ? 16 : plan_ept0(n); }
// product of the radices before stage s
constexpr int plan_ns(int n, int s, int p = 0) {
  return s == 0 ? 1 : plan_ns(n, s - 1, p) * plan_radix(n, s - 1, p);
}
// offset of stage s in the per-stage twiddle table: entries [k][r-1], k < Ns, 1 <= r < R
constexpr int plan_tw_off(int n, int s, int p = 0) {
  return s == 0 ? 0 : plan_tw_off(n, s - 1, p) + plan_ns(n, s - 1, p) * (plan_radix(n, s - 1, p) - 1);
}
constexpr int plan_tw_size(int n, int p = 0) { return plan_tw_off(n, plan_stages(n, p), p); }

constexpr int largest_divisor_le(int n, int cap) {
  int best = 1;
  for (int d = 1; d <= n && d <= cap; ++d)
    if (n % d == 0) best = d;
  return best;
}

// Tile geometry of the four-pass kernels.  Bit 0 of V: 0 = about 4096 (FP32) / 2048
// (FP64) elements per tile, y/z tiles up to 16 (8) contiguous columns wide; 1 = half the
// tile and half the width (more, smaller blocks per SM).  Bit 1: the radix plan (PLAN).
// The autotuner picks V per N.
template <typename R, int N, int V = 0>
struct Geom {
  static constexpr int PLAN = V >> 1;
  static constexpr int EPT = plan_ept(N, PLAN);
  static constexpr int S = plan_stages(N, PLAN);
  static constexpr int TARGET = (sizeof(R) == 4 ? 4096 : 2048) >> (V & 1);  // elements per tile
  // x pass: LC whole lines per block
  static constexpr int LC = largest_divisor_le(N * N, TARGET / N > 0 ? TARGET / N : 1);
  static constexpr int TL = N / EPT;                       // threads per line
  static constexpr int THREADS_X = LC * TL;
  static constexpr int PAD_SHIFT = sizeof(R) == 4 ? 4 : 3;  // one pad element per 128 B
  static constexpr int PL = N + (N >> PAD_SHIFT) + 1;       // padded line length
  // y/z passes: C = L contiguous columns x P outer slices
  static constexpr int L = largest_divisor_le(N, (sizeof(R) == 4 ? 16 : 8) >> (V & 1));
  static constexpr int P = largest_divisor_le(N, TARGET / (L * N) > 0 ? TARGET / (L * N) : 1);
  static constexpr int C = L * P;
  static constexpr int THREADS_S = C * N / EPT;
  static constexpr int TW = plan_tw_size(N, PLAN);
  static_assert(S > 0 && EPT > 0, "unsupported N");
};

// ------------------------------------------------------------------------------------
// Small DFTs (forward: exp(-2 pi i rk/R); INV flips the sign of the exponent)
// ------------------------------------------------------------------------------------
template <typename R, bool INV>
__device__ __forceinline__ cpx<R> mul_negi(cpx<R> a) {  // a * exp(-+ i pi/2)
  return INV ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x);
}
// a * exp(-+ i theta) given c = cos(theta), s = sin(theta)
template <typename R, bool INV>
__device__ __forceinline__ cpx<R> rot(cpx<R> a, R c, R s) {
  return INV ? mk<R>(a.x * c - a.y * s, a.y * c + a.x * s) : mk<R>(a.x * c + a.y * s, a.y * c - a.x * s);
}

template <typename R, bool INV>
__device__ __forceinline__ void dft2(cpx<R>& a, cpx<R>& b) {
  cpx<R> t = a - b;
  a = a + b;
  b = t;
}

template <typename R, bool INV>
__device__ __forceinline__ void dft4(cpx<R>& x0, cpx<R>& x1, cpx<R>& x2, cpx<R>& x3) {
  cpx<R> a0 = x0 + x2, a1 = x0 - x2, a2 = x1 + x3, a3 = mul_negi<R, INV>(x1 - x3);
  x0 = a0 + a2;
  x2 = a0 - a2;
  x1 = a1 + a3;
  x3 = a1 - a3;
}

template <typename R, bool INV>
__device__ __forceinline__ void dft3(cpx<R>& x0, cpx<R>& x1, cpx<R>& x2) {
  const R h = R(0.86602540378443864676);  // sin(2 pi / 3)
  cpx<R> s = x1 + x2, d = x1 - x2;
  cpx<R> t = mk<R>(x0.x - R(0.5) * s.x, x0.y - R(0.5) * s.y);
  x0 = x0 + s;
  // forward: y1 = t - i h d, y2 = t + i h d
  cpx<R> ihd = mk<R>(-h * d.y, h * d.x);  // i h d
  if (INV) {
    x1 = t + ihd;
    x2 = t - ihd;
  } else {
    x1 = t - ihd;
    x2 = t + ihd;
  }
}

template <typename R, bool INV>
__device__ __forceinline__ void dft8(cpx<R>* x) {
  const R r2 = R(0.70710678118654752440);
  dft4<R, INV>(x[0], x[2], x[4], x[6]);
  dft4<R, INV>(x[1], x[3], x[5], x[7]);
  // odd part times exp(-+ 2 pi i k/8), k = 1, 2, 3
  x[3] = rot<R, INV>(x[3], r2, r2);
  x[5] = mul_negi<R, INV>(x[5]);
  x[7] = rot<R, INV>(x[7], -r2, r2);
  cpx<R> y[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    y[k] = x[2 * k] + x[2 * k + 1];
    y[k + 4] = x[2 * k] - x[2 * k + 1];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = y[k];
}

template <typename R, bool INV>
__device__ __forceinline__ void dft16(cpx<R>* x) {
  const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173);  // pi/8
  const R r2 = R(0.70710678118654752440);
  // n = 4 n1 + n2: length-4 DFTs over n1 for each n2 -> A[n2][k1] stored at x[4 n1 + n2]
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<R, INV>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
  // after dft4, x[4 k1 + n2] holds A[n2][k1]; twiddle by exp(-+ 2 pi i n2 k1 / 16)
  x[4 * 1 + 1] = rot<R, INV>(x[5], c1, s1);     // n2=1,k1=1: 1
  x[4 * 2 + 1] = rot<R, INV>(x[9], r2, r2);     // n2=1,k1=2: 2
  x[4 * 3 + 1] = rot<R, INV>(x[13], s1, c1);    // n2=1,k1=3: 3
  x[4 * 1 + 2] = rot<R, INV>(x[6], r2, r2);     // n2=2,k1=1: 2
  x[4 * 2 + 2] = mul_negi<R, INV>(x[10]);       // n2=2,k1=2: 4
  x[4 * 3 + 2] = rot<R, INV>(x[14], -r2, r2);   // n2=2,k1=3: 6
  x[4 * 1 + 3] = rot<R, INV>(x[7], s1, c1);     // n2=3,k1=1: 3
  x[4 * 2 + 3] = rot<R, INV>(x[11], -r2, r2);   // n2=3,k1=2: 6
  x[4 * 3 + 3] = rot<R, INV>(x[15], -c1, -s1);  // n2=3,k1=3: 9
  // length-4 DFTs over n2 for each k1: y[k1 + 4 k2]
  cpx<R> y[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cpx<R> a = x[4 * k1], b = x[4 * k1 + 1], c = x[4 * k1 + 2], d = x[4 * k1 + 3];
    dft4<R, INV>(a, b, c, d);
    y[k1] = a;
    y[k1 + 4] = b;
    y[k1 + 8] = c;
    y[k1 + 12] = d;
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = y[k];
}

template <typename R, int RAD, bool INV>
__device__ __forceinline__ void dft(cpx<R>* x) {
  if constexpr (RAD == 2) {
    dft2<R, INV>(x[0], x[1]);
  } else if constexpr (RAD == 3) {
    dft3<R, INV>(x[0], x[1], x[2]);
  } else if constexpr (RAD == 4) {
    dft4<R, INV>(x[0], x[1], x[2], x[3]);
  } else if constexpr (RAD == 8) {
    dft8<R, INV>(x);
  } else if constexpr (RAD == 16) {
    dft16<R, INV>(x);
  }
}

// ------------------------------------------------------------------------------------
// One Stockham stage on the registers of one thread: EPT/RAD butterflies, butterfly b
// of thread group g has index j = g + b * TL (TL = N/EPT threads per line).
// ------------------------------------------------------------------------------------
template <typename R, int N, int ST, bool INV, int PL = 0>
__device__ __forceinline__ void stage_compute(cpx<R> (&v)[plan_ept(N, PL)], int g, const cpx<R>* tw_s) {
  constexpr int EPT = plan_ept(N, PL), RAD = plan_radix(N, ST, PL), NS = plan_ns(N, ST, PL), TL = N / EPT;
  constexpr int OFF = plan_tw_off(N, ST, PL);
#pragma unroll
  for (int b = 0; b < EPT / RAD; ++b) {
    if constexpr (NS > 1) {
      const int j = g + b * TL;
      const int k = j % NS;
      const cpx<R>* t = tw_s + OFF + k * (RAD - 1);
      if constexpr (sizeof(R) == 4 && RAD >= 8) {
        // complex FP32, radix 8 / 16: w^r formed by multiplying up from w = t[0], restarting
        // from the table at r = 8 (at most six products deep, a few ulp), so a butterfly
        // reads 1-2 twiddles from shared memory instead of RAD - 1
        const cpx<R> w1 = t[0];
        cpx<R> w = w1;
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          if (r == 8) w = t[7];
          else if (r > 1) w = cmul<R>(w, w1);
          v[b * RAD + r] = INV ? cmulc<R>(v[b * RAD + r], w) : cmul<R>(v[b * RAD + r], w);
        }
      } else {
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          cpx<R> w = t[r - 1];
          v[b * RAD + r] = INV ? cmulc<R>(v[b * RAD + r], w) : cmul<R>(v[b * RAD + r], w);
        }
      }
    }
    dft<R, RAD, INV>(&v[b * RAD]);
  }
}

// element index read by (b, r) at stage ST
template <int N, int ST, int PL = 0>
__device__ __forceinline__ int e_in(int g, int b, int r) {
  constexpr int EPT = plan_ept(N, PL), RAD = plan_radix(N, ST, PL), TL = N / EPT;
  return g + b * TL + r * (N / RAD);
}
// element index written by (b, r) at stage ST
template <int N, int ST, int PL = 0>
__device__ __forceinline__ int e_out(int g, int b, int r) {
  constexpr int EPT = plan_ept(N, PL), RAD = plan_radix(N, ST, PL), NS = plan_ns(N, ST, PL), TL = N / EPT;
  const int j = g + b * TL;
  return (j / NS) * NS * RAD + (j % NS) + r * NS;
}

// ------------------------------------------------------------------------------------
// Shared-memory accessors for the two tile layouts
// ------------------------------------------------------------------------------------
template <typename R, int N, bool STRIDED, int V = 0>
struct Tile {
  using G = Geom<R, N, V>;
  cpx<R>* s;
  int col;  // STRIDED: column; contiguous: line
  __device__ __forceinline__ int idx(int e) const {
    if constexpr (STRIDED) return e * G::C + col;
    else return col * G::PL + e + (e >> G::PAD_SHIFT);
  }
  __device__ __forceinline__ cpx<R> ld(int e) const { return s[idx(e)]; }
  __device__ __forceinline__ void st(int e, cpx<R> v) const { s[idx(e)] = v; }
};

// Runs stages [FIRST, LAST] of one transform direction.  Stage FIRST reads either global
// memory (gsrc: element e of this thread's line at gsrc[e * gstride]) or shared memory;
// stage LAST leaves its outputs in v (natural-order element e_out<N, LAST>).
template <typename R, int N, bool STRIDED, bool INV, int ST, int LAST, int V = 0>
__device__ __forceinline__ void run_stages(cpx<R> (&v)[plan_ept(N, V >> 1)], int g, const Tile<R, N, STRIDED, V>& t,
                                           const cpx<R>* tw_s) {
  constexpr int PL = V >> 1;
  constexpr int RAD = plan_radix(N, ST, PL);
  constexpr int EPT = plan_ept(N, PL);
  stage_compute<R, N, ST, INV, PL>(v, g, tw_s);
  if constexpr (ST < LAST) {
    __syncthreads();  // all reads of this stage's inputs are done
#pragma unroll
    for (int b = 0; b < EPT / RAD; ++b)
#pragma unroll
      for (int r = 0; r < RAD; ++r) t.st(e_out<N, ST, PL>(g, b, r), v[b * RAD + r]);
    __syncthreads();
    constexpr int RN = plan_radix(N, ST + 1, PL);
#pragma unroll
    for (int b = 0; b < EPT / RN; ++b)
#pragma unroll
      for (int r = 0; r < RN; ++r) v[b * RN + r] = t.ld(e_in<N, ST + 1, PL>(g, b, r));
    run_stages<R, N, STRIDED, INV, ST + 1, LAST, V>(v, g, t, tw_s);
  }
}

// Kinetic multiplier T(k)/N^3 for momenta indices (jx, jy, jz) (Eqs. HK1-HK3).
template <typename R>
__device__ __forceinline__ R kin_mult(int kinetic, R sxy, R sz, R tcoef, R am2) {
  R s = sxy + sz;
  if (kinetic == KIN_FFT_REL) {
    // sqrt(u) = u / sqrt(u) for u > 0: FP32 through the hardware reciprocal square root
    // (a few ulp, no branch; u = 0 only if (am)^2 underflows), FP64 correctly rounded
    const R u = s + am2;
    if constexpr (sizeof(R) == 4) return (u > 0.f ? u * rsqrtf(u) : 0.f) * tcoef;
    else return sqrt(u) * tcoef;
  }
  return s * tcoef;
}

// ------------------------------------------------------------------------------------
// Pass kernels
// ------------------------------------------------------------------------------------
// OP_FINAL* are the last x pass: update only, update + check sums, sums only (measure).
enum PassOp : int { OP_FWD = 0, OP_INV = 1, OP_MID = 2, OP_FINAL = 3, OP_FINAL_SUMS = 4, OP_SUMS = 5 };
constexpr bool is_final(int op) { return op >= OP_FINAL; }

template <typename R, int N, int V = 0>
__device__ __forceinline__ void load_twiddles(cpx<R>* tw_s, const cpx<R>* tw) {
  for (int i = threadIdx.x; i < Geom<R, N, V>::TW; i += blockDim.x) tw_s[i] = tw[i];
}

// x pass: LC contiguous lines per block.  OP_FWD: src -> data.  OP_FINAL: data (H_K psi
// in x-transformed space) -> inverse x -> update of psi.  The final pass loads psi and V
// of its output sites at the start, so those reads overlap the inverse transform.
template <typename R, int N, int OP, bool VREAL, bool NEXT = false, int V = 0>
__device__ __forceinline__ void fft_x_body(const FftPassArgs<R>& a, const int bid) {
  using G = Geom<R, N, V>;
  constexpr int PL = G::PLAN;
  constexpr int EPT = G::EPT, S = G::S, R0 = plan_radix(N, 0, PL), RL = plan_radix(N, S - 1, PL);
  constexpr bool FIN = is_final(OP);
  constexpr bool INV = FIN || OP == OP_INV;
  constexpr bool WRITE = (OP == OP_FINAL || OP == OP_FINAL_SUMS);
  constexpr bool SUMS = (OP == OP_FINAL_SUMS || OP == OP_SUMS);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* tw_s = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* data_s = tw_s + G::TW;
  double* red_s = reinterpret_cast<double*>(data_s + G::LC * G::PL);

  const int line = threadIdx.x / G::TL, g = threadIdx.x % G::TL;
  const long long gline = (long long)bid * G::LC + line;
  const long long base = gline * N;
  load_twiddles<R, N, V>(tw_s, a.twiddle);

  const cpx<R>* __restrict__ in = (OP == OP_FWD && a.src) ? a.src : a.data;
  cpx<R> v[EPT];
#pragma unroll
  for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
    for (int r = 0; r < R0; ++r) v[b * R0 + r] = in[base + e_in<N, 0, PL>(g, b, r)];

  // final pass: psi and V at the sites this thread will write (natural order)
  cpx<R> pv[FIN ? EPT : 1];
  cpx<R> vv[FIN && !VREAL ? EPT : 1];
  R vr_[FIN && VREAL ? EPT : 1];
  if constexpr (FIN) {
    const cpx<R>* __restrict__ psi_in = a.psi;
#pragma unroll
    for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) pv[b * RL + r] = psi_in[base + e_out<N, S - 1, PL>(g, b, r)];
    if constexpr (VREAL) {
      const R* __restrict__ vr = reinterpret_cast<const R*>(a.v);
#pragma unroll
      for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
        for (int r = 0; r < RL; ++r) vr_[b * RL + r] = vr[base + e_out<N, S - 1, PL>(g, b, r)];
    } else {
      const cpx<R>* __restrict__ vc = reinterpret_cast<const cpx<R>*>(a.v);
#pragma unroll
      for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
        for (int r = 0; r < RL; ++r) vv[b * RL + r] = vc[base + e_out<N, S - 1, PL>(g, b, r)];
    }
  }
  __syncthreads();  // twiddles visible

  Tile<R, N, false, V> t{data_s, line};
  run_stages<R, N, false, INV, 0, S - 1, V>(v, g, t, tw_s);

  if constexpr (OP == OP_FWD || OP == OP_INV) {
#pragma unroll
    for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
      for (int r = 0; r < RL; ++r) a.data[base + e_out<N, S - 1, PL>(g, b, r)] = v[b * RL + r];
  } else {
    // v = H_K psi at the sites of this line (the 1/N^3 is inside T).
    auto vat = [&](int i) { return VREAL ? mk<R>(vr_[VREAL ? i : 0], R(0)) : vv[VREAL ? 0 : i]; };
    if constexpr (SUMS) {
      CheckSums<R> cs;
#pragma unroll
      for (int i = 0; i < EPT; ++i) cs.add(pv[i], v[i], vat(i));
      double acc[kNumSums];
      cs.to(acc);
      block_sum_store<kNumSums>(acc, red_s, a.partials + (long long)bid * kPartialStride);
    }
    if constexpr (WRITE) {
      const R sc = R(*a.scale);
#pragma unroll
      for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int i = b * RL + r;
          // d = 1 + dtau V/2; coef_B = 1/d; coef_A = (2 - d)/d (FP32: the fast hardware
          // division, a few ulp; FP64: correctly rounded)
          const cpx<R> vi = vat(i);
          if constexpr (VREAL) {
            const R d = R(1) + a.half_dtau * vi.x;
            const cpx<R> num = cscale<R>(pv[i], R(2) - d) - cscale<R>(v[i], a.dtau);
            if constexpr (sizeof(R) == 4) v[i] = cscale<R>(num, __fdividef(sc, d));
            else v[i] = cscale<R>(num, sc / d);
          } else {
            const cpx<R> d = mk<R>(R(1) + a.half_dtau * vi.x, a.half_dtau * vi.y);
            const cpx<R> num = cmul<R>(mk<R>(R(2) - d.x, -d.y), pv[i]) - cscale<R>(v[i], a.dtau);
            R inv;
            if constexpr (sizeof(R) == 4) inv = __fdividef(sc, d.x * d.x + d.y * d.y);
            else inv = sc / (d.x * d.x + d.y * d.y);
            v[i] = cscale<R>(cmulc<R>(num, d), inv);
          }  // v[i] = psi_{t+1}
          a.psi[base + e_out<N, S - 1, PL>(g, b, r)] = v[i];
        }
      if constexpr (NEXT) {
        // forward x transform of psi_{t+1} for the next step (its first pass)
        if constexpr (R0 != RL) {
          __syncthreads();
#pragma unroll
          for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
            for (int r = 0; r < RL; ++r) t.st(e_out<N, S - 1, PL>(g, b, r), v[b * RL + r]);
          __syncthreads();
#pragma unroll
          for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
            for (int r = 0; r < R0; ++r) v[b * R0 + r] = t.ld(e_in<N, 0, PL>(g, b, r));
        }
        // (equal first and last radix: the thread already holds the first stage's inputs)
        run_stages<R, N, false, false, 0, S - 1, V>(v, g, t, tw_s);
#pragma unroll
        for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
          for (int r = 0; r < RL; ++r) a.data[base + e_out<N, S - 1, PL>(g, b, r)] = v[b * RL + r];
      }
    }
  }
}

// y / z passes: C = L x P columns per block.  AXIS 1: points stride N, outer = z (stride
// N^2).  AXIS 2: points stride N^2, outer = y (stride N).
template <typename R, int N, int AXIS, int OP, int V = 0>
__device__ __forceinline__ void fft_s_body(const FftPassArgs<R>& a, const int bid) {
  using G = Geom<R, N, V>;
  constexpr int PL = G::PLAN;
  constexpr int EPT = G::EPT, S = G::S, R0 = plan_radix(N, 0, PL), RL = plan_radix(N, S - 1, PL);
  constexpr long long PSTRIDE = AXIS == 1 ? N : (long long)N * N;
  constexpr long long OSTRIDE = AXIS == 1 ? (long long)N * N : N;
  constexpr bool INV = (OP == OP_INV);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* tw_s = reinterpret_cast<cpx<R>*>(smem_raw);
  R* sym_s = reinterpret_cast<R*>(tw_s + G::TW);
  cpx<R>* data_s = reinterpret_cast<cpx<R>*>(sym_s + ((N * sizeof(R) + 15) / 16) * 16 / sizeof(R));

  const int c = threadIdx.x % G::C, g = threadIdx.x / G::C;
  const int l = c % G::L, p = c / G::L;
  constexpr int XB = N / G::L;
  const int xb = bid % XB, ob = bid / XB;
  const int x = xb * G::L + l, o = ob * G::P + p;
  const long long base = (long long)o * OSTRIDE + x;
  load_twiddles<R, N, V>(tw_s, a.twiddle);
  if (OP == OP_MID)
    for (int i = threadIdx.x; i < N; i += blockDim.x) sym_s[i] = a.symbol[i];

  cpx<R> v[EPT];
#pragma unroll
  for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
    for (int r = 0; r < R0; ++r) v[b * R0 + r] = a.data[base + e_in<N, 0, PL>(g, b, r) * PSTRIDE];
  __syncthreads();

  Tile<R, N, true, V> t{data_s, c};
  if constexpr (OP == OP_MID) {
    run_stages<R, N, true, false, 0, S - 1, V>(v, g, t, tw_s);
    // forward z transform done: natural-order kz; multiply by T and start the inverse
    const R sxy = sym_s[x] + sym_s[o];  // kx = x, ky = o (after the x and y passes)
    if constexpr (R0 == RL) {
      // the last forward stage leaves this thread exactly the elements the first inverse
      // stage reads (j + r N/R for both), so T is applied in registers
#pragma unroll
      for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int kz = e_out<N, S - 1, PL>(g, b, r);
          v[b * RL + r] = cscale<R>(v[b * RL + r], kin_mult<R>(a.kinetic, sxy, sym_s[kz], a.tcoef, a.am2));
        }
    } else {
      __syncthreads();
#pragma unroll
      for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
        for (int r = 0; r < RL; ++r) t.st(e_out<N, S - 1, PL>(g, b, r), v[b * RL + r]);
      __syncthreads();
#pragma unroll
      for (int b = 0; b < EPT / R0; ++b)
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int kz = e_in<N, 0, PL>(g, b, r);
          const R tm = kin_mult<R>(a.kinetic, sxy, sym_s[kz], a.tcoef, a.am2);
          v[b * R0 + r] = cscale<R>(t.ld(kz), tm);
        }
    }
    run_stages<R, N, true, true, 0, S - 1, V>(v, g, t, tw_s);
  } else {
    run_stages<R, N, true, INV, 0, S - 1, V>(v, g, t, tw_s);
  }
#pragma unroll
  for (int b = 0; b < EPT / RL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) a.data[base + e_out<N, S - 1, PL>(g, b, r) * PSTRIDE] = v[b * RL + r];
}

// Entry points: one lattice (arguments by value), or a group of up to kGroupMax lattices
// of the same N advanced by one launch (blockIdx.y selects the lattice; the arguments of
// all members travel in the kernel's parameter space).  Every lattice runs exactly the
// blocks it would run alone.
//
// The x passes that read the inverse-y output walk the lines from the last to the first:
// the y pass wrote its last z-planes most recently, so they are still in L2 when the
// reversed pass starts, and the next step's y pass (first to last) starts where this one
// ended.
template <int OP>
__device__ __forceinline__ int x_block(int b) {
  return (OP == OP_FWD) ? b : (int)gridDim.x - 1 - b;
}
template <typename R, int N, int OP, bool VREAL, bool NEXT = false>
__global__ void __launch_bounds__(Geom<R, N>::THREADS_X) fft_x_kernel(FftPassArgs<R> a) {
  fft_x_body<R, N, OP, VREAL, NEXT>(a, x_block<OP>(blockIdx.x));
}
template <typename R, int N, int AXIS, int OP>
__global__ void __launch_bounds__(Geom<R, N>::THREADS_S) fft_s_kernel(FftPassArgs<R> a) {
  fft_s_body<R, N, AXIS, OP>(a, blockIdx.x);
}
template <typename R, int N, int OP, bool VREAL, bool NEXT = false, int V = 0>
__global__ void __launch_bounds__(Geom<R, N, V>::THREADS_X) fft_x_group_kernel(const __grid_constant__ FftGroup<R> g) {
  fft_x_body<R, N, OP, VREAL, NEXT, V>(g.a[blockIdx.y], x_block<OP>(blockIdx.x));
}
template <typename R, int N, int AXIS, int OP, int V = 0>
__global__ void __launch_bounds__(Geom<R, N, V>::THREADS_S) fft_s_group_kernel(const __grid_constant__ FftGroup<R> g) {
  fft_s_body<R, N, AXIS, OP, V>(g.a[blockIdx.y], blockIdx.x);
}

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
template <typename R, int N, int V = 0>
static size_t smem_x() {
  using G = Geom<R, N, V>;
  return G::TW * sizeof(cpx<R>) + G::LC * G::PL * sizeof(cpx<R>) + 32 * kNumSums * sizeof(double);
}
template <typename R, int N, int V = 0>
static size_t smem_s() {
  using G = Geom<R, N, V>;
  return G::TW * sizeof(cpx<R>) + ((N * sizeof(R) + 15) / 16) * 16 + (size_t)G::C * N * sizeof(cpx<R>);
}

// Variant of the final x pass for (real V, writes psi', check sums, emits the next x transform).
template <typename R, int N, bool GROUP, bool VREAL, int V = 0>
static auto final_kernel(bool write, bool sums, bool next) {
  if constexpr (GROUP) {
    if (!write) return fft_x_group_kernel<R, N, OP_SUMS, VREAL, false, V>;
    if (sums) return next ? fft_x_group_kernel<R, N, OP_FINAL_SUMS, VREAL, true, V>
                          : fft_x_group_kernel<R, N, OP_FINAL_SUMS, VREAL, false, V>;
    return next ? fft_x_group_kernel<R, N, OP_FINAL, VREAL, true, V>
                : fft_x_group_kernel<R, N, OP_FINAL, VREAL, false, V>;
  } else {
    if (!write) return fft_x_kernel<R, N, OP_SUMS, VREAL, false>;
    if (sums) return next ? fft_x_kernel<R, N, OP_FINAL_SUMS, VREAL, true> : fft_x_kernel<R, N, OP_FINAL_SUMS, VREAL, false>;
    return next ? fft_x_kernel<R, N, OP_FINAL, VREAL, true> : fft_x_kernel<R, N, OP_FINAL, VREAL, false>;
  }
}

// Raises the dynamic shared-memory limit of every x-pass variant (the largest tiles need
// more than the default 48 KB).
template <typename R, int N, bool GROUP, int V = 0>
static void set_x_attrs(size_t sx) {
  for (int vr = 0; vr < 2; ++vr)
    for (int w = 0; w < 2; ++w)
      for (int su = 0; su < 2; ++su)
        for (int nx = 0; nx < 2; ++nx) {
          const void* f = vr ? (const void*)final_kernel<R, N, GROUP, true, V>(w, su, nx)
                             : (const void*)final_kernel<R, N, GROUP, false, V>(w, su, nx);
          cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sx);
        }
  if constexpr (GROUP)
    cudaFuncSetAttribute((const void*)fft_x_group_kernel<R, N, OP_FWD, false, false, V>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sx);
  else
    cudaFuncSetAttribute((const void*)fft_x_kernel<R, N, OP_FWD, false, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sx);
}

template <typename R, int N>
static cudaError_t pass_n(int pass, FftPassArgs<R> a, cpx<R>* tmp, cudaStream_t st, int* nfinal) {
  using G = Geom<R, N>;
  const int gx = N * N / G::LC, gs = (N / G::L) * (N / G::P);
  const size_t sx = smem_x<R, N>(), ss = smem_s<R, N>();
  static bool attr_done = false;
  if (!attr_done) {
    set_x_attrs<R, N, false>(sx);
    cudaFuncSetAttribute(fft_s_kernel<R, N, 1, OP_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(fft_s_kernel<R, N, 2, OP_MID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(fft_s_kernel<R, N, 1, OP_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(fft_s_kernel<R, N, 2, OP_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(fft_s_kernel<R, N, 2, OP_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(fft_x_kernel<R, N, OP_INV, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sx);
    attr_done = true;
  }
  if (nfinal) *nfinal = gx;
  FftPassArgs<R> p = a;
  p.data = tmp;
  p.src = (pass == 0) ? a.psi : nullptr;
  const bool write = p.write_psi != 0, sums = p.reduce != 0, next = write && p.emit_next != 0;
  switch (pass) {
    case 0: fft_x_kernel<R, N, OP_FWD, false><<<gx, G::THREADS_X, sx, st>>>(p); break;
    case 1: fft_s_kernel<R, N, 1, OP_FWD><<<gs, G::THREADS_S, ss, st>>>(p); break;
    case 2: fft_s_kernel<R, N, 2, OP_MID><<<gs, G::THREADS_S, ss, st>>>(p); break;
    case 3: fft_s_kernel<R, N, 1, OP_INV><<<gs, G::THREADS_S, ss, st>>>(p); break;
    case 5: fft_s_kernel<R, N, 2, OP_FWD><<<gs, G::THREADS_S, ss, st>>>(p); break;
    case 6: fft_s_kernel<R, N, 2, OP_INV><<<gs, G::THREADS_S, ss, st>>>(p); break;
    case 7: fft_x_kernel<R, N, OP_INV, false><<<gx, G::THREADS_X, sx, st>>>(p); break;
    case 4:
      if (p.v_real) final_kernel<R, N, false, true>(write, sums, next)<<<gx, G::THREADS_X, sx, st>>>(p);
      else final_kernel<R, N, false, false>(write, sums, next)<<<gx, G::THREADS_X, sx, st>>>(p);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// One pass for a group of lattices of size N: g.a[i] holds lattice i's arguments as
// launch_fft_pass would build them (data = its scratch field, src = psi on pass 0).  The
// final pass variant follows member 0 (members of a group agree on it).
template <typename R, int N, int V = 0>
static cudaError_t group_pass_n(int pass, const FftGroup<R>& g, cudaStream_t st) {
  using G = Geom<R, N, V>;
  const size_t sx = smem_x<R, N, V>(), ss = smem_s<R, N, V>();
  static bool attr_done = false;
  if (!attr_done) {
    set_x_attrs<R, N, true, V>(sx);
    cudaFuncSetAttribute(fft_s_group_kernel<R, N, 1, OP_FWD, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(fft_s_group_kernel<R, N, 2, OP_MID, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(fft_s_group_kernel<R, N, 1, OP_INV, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(fft_s_group_kernel<R, N, 2, OP_FWD, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(fft_s_group_kernel<R, N, 2, OP_INV, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(fft_x_group_kernel<R, N, OP_INV, false, false, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sx);
    attr_done = true;
  }
  const dim3 gx(N * N / G::LC, g.count), gs((N / G::L) * (N / G::P), g.count);
  const bool vreal = g.a[0].v_real != 0, sums = g.a[0].reduce != 0, write = g.a[0].write_psi != 0;
  const bool next = write && g.a[0].emit_next != 0;
  switch (pass) {
    case 0: fft_x_group_kernel<R, N, OP_FWD, false, false, V><<<gx, G::THREADS_X, sx, st>>>(g); break;
    case 1: fft_s_group_kernel<R, N, 1, OP_FWD, V><<<gs, G::THREADS_S, ss, st>>>(g); break;
    case 2: fft_s_group_kernel<R, N, 2, OP_MID, V><<<gs, G::THREADS_S, ss, st>>>(g); break;
    case 3: fft_s_group_kernel<R, N, 1, OP_INV, V><<<gs, G::THREADS_S, ss, st>>>(g); break;
    case 5: fft_s_group_kernel<R, N, 2, OP_FWD, V><<<gs, G::THREADS_S, ss, st>>>(g); break;
    case 6: fft_s_group_kernel<R, N, 2, OP_INV, V><<<gs, G::THREADS_S, ss, st>>>(g); break;
    case 7: fft_x_group_kernel<R, N, OP_INV, false, false, V><<<gx, G::THREADS_X, sx, st>>>(g); break;
    case 4:
      if (vreal) final_kernel<R, N, true, true, V>(write, sums, next)<<<gx, G::THREADS_X, sx, st>>>(g);
      else final_kernel<R, N, true, false, V>(write, sums, next)<<<gx, G::THREADS_X, sx, st>>>(g);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Tile variant of the complex-FP32 four-pass kernels in use for size n (0-3: bit 0 the
// tile geometry, bit 1 the radix plan; chosen by the autotuner in the C ABI, qf_fft_f32.cu
// holds the table) and the launchers of variants 1 and 2-3, compiled in translation units
// of their own (qf_fft_group_t1.cu, qf_fft_group_p1.cu).  Variants 2 and 3 read the
// second twiddle table, stored right after the first.
int fft_tile_variant(int n);
cudaError_t launch_fft_group_pass_t1(int n, int pass, const FftGroup<float>& g, cudaStream_t st);
cudaError_t launch_fft_group_pass_p1(int n, int variant, int pass, const FftGroup<float>& g, cudaStream_t st);

// Partial-sum rows of the reducing x pass for size n with tile variant V.
template <typename R, int V>
int fft_final_blocks_v(int n) {
  switch (n) {
#define QF_CASE(NN) \
  case NN:          \
    return NN * NN / Geom<R, NN, V>::LC;
    QF_CASE(8) QF_CASE(12) QF_CASE(16) QF_CASE(24) QF_CASE(32) QF_CASE(48) QF_CASE(64) QF_CASE(96)
    QF_CASE(128) QF_CASE(192) QF_CASE(256) QF_CASE(384) QF_CASE(512)
#undef QF_CASE
    default:
      return 0;
  }
}

// alt_plan: whether the members' twiddle regions hold the second plan's table (the
// lattices' do; the allocation-free entry point's holds the first only).
template <typename R>
cudaError_t launch_fft_group_pass(int n, int pass, const FftGroup<R>& g, cudaStream_t st, bool alt_plan) {
  if constexpr (sizeof(R) == 4) {
    int v = fft_tile_variant(n);
    if (!alt_plan) v &= 1;
    if (v >= 2) return launch_fft_group_pass_p1(n, v, pass, g, st);
    if (v == 1) return launch_fft_group_pass_t1(n, pass, g, st);
  }
  switch (n) {
#define QF_CASE(NN) \
  case NN:          \
    return group_pass_n<R, NN>(pass, g, st);
    QF_CASE(8) QF_CASE(12) QF_CASE(16) QF_CASE(24) QF_CASE(32) QF_CASE(48) QF_CASE(64) QF_CASE(96)
    QF_CASE(128) QF_CASE(192) QF_CASE(256) QF_CASE(384) QF_CASE(512)
#undef QF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

// Partial-sum rows of the reducing x pass for size n as launched now (complex FP32: the
// tile variant in use).
template <typename R>
int fft_final_blocks(int n) {
  if constexpr (sizeof(R) == 4) {
    if (fft_tile_variant(n) & 1) return fft_final_blocks_v<R, 1>(n);  // (the plan bit does not change it)
  }
  return fft_final_blocks_v<R, 0>(n);
}

// The most partial rows any variant's reducing pass writes (workspace sizing).
template <typename R>
int fft_final_blocks_max(int n) {
  const int a = fft_final_blocks_v<R, 0>(n);
  if constexpr (sizeof(R) == 4) {
    const int b = fft_final_blocks_v<R, 1>(n);
    return a > b ? a : b;
  }
  return a;
}

// Complex-FP32 lattices always run the grouped kernels (a lone lattice is a group of one),
// so a lattice executes the same machine code alone and inside a batch.
template <typename R, int N>
static cudaError_t single_pass_n(int pass, FftPassArgs<R> a, cpx<R>* tmp, cudaStream_t st, int* nfinal,
                                 bool alt_plan) {
  if constexpr (sizeof(R) == 4) {
    if (nfinal) *nfinal = fft_final_blocks<R>(N);
    FftGroup<R> g;
    g.count = 1;
    g.a[0] = a;
    g.a[0].data = tmp;
    g.a[0].src = (pass == 0) ? a.psi : nullptr;
    return launch_fft_group_pass<R>(N, pass, g, st, alt_plan);
  } else {
    return pass_n<R, N>(pass, a, tmp, st, nfinal);
  }
}

template <typename R>
cudaError_t launch_fft_pass(int n, int pass, FftPassArgs<R> args, cpx<R>* tmp, cudaStream_t st, int* nfinal,
                            bool alt_plan) {
  switch (n) {
#define QF_CASE(NN) \
  case NN:          \
    return single_pass_n<R, NN>(pass, args, tmp, st, nfinal, alt_plan);
    QF_CASE(8) QF_CASE(12) QF_CASE(16) QF_CASE(24) QF_CASE(32) QF_CASE(48) QF_CASE(64) QF_CASE(96)
    QF_CASE(128) QF_CASE(192) QF_CASE(256) QF_CASE(384) QF_CASE(512)
#undef QF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace qf
