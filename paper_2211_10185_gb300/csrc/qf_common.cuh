// Internal definitions shared by the kernels and the C ABI of libqfdtd (sm_103a).
//
// Field layout: complex N^3 array, site (ix, iy, iz) at (iz*N + iy)*N + ix (x fastest),
// coordinate x_i = (i - N/2) a.  Complex values are interleaved (re, im) pairs of the
// lattice precision R (float for the c64 path, double for the c128 path).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qf {

template <typename R>
struct __align__(2 * sizeof(R)) cpx {
  R x, y;
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) {
  cpx<R> c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R>
__device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename R>
__device__ __forceinline__ cpx<R> cmulc(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename R>
__device__ __forceinline__ cpx<R> cscale(cpx<R> a, R s) { return mk<R>(a.x * s, a.y * s); }

// Kinetic-term identifiers (Eqs. HK0-HK3).
enum Kinetic : int { KIN_FDTD = 0, KIN_FFT_NAIVE = 1, KIN_FFT_SYMANZIK = 2, KIN_FFT_REL = 3 };

// Number of FP64 partial sums a reducing kernel writes per block.
constexpr int kNumSums = 5;  // <psi|psi>, Re/Im <psi|H_K psi>, Re/Im <psi|V psi>
constexpr int kPartialStride = 8;

// Device-resident scalars of one lattice (lives in the caller's workspace).
// Output scale of a step: [0] = 1 (no scaling); [1] = 2^(k+j) / sqrt(norm of the last
// check), the step after a check; [2] = 2^k, the other steps.  The powers of two (exact
// in floating point) keep a field that decays by about lambda per step near unit size
// between checks (k ~ -log2 lambda, j centres the interval's residual growth; both chosen
// by the finishing kernel of each check); the host tracks the accumulated power of two
// and removes it from every field it hands out.
struct DevScalars {
  double scale[4];     // see above; [3] unused
  double sums[8];      // last finished reduction (kNumSums used)
  double energy[6];    // e_re, e_im, norm of the last finished reduction; k, j of the scale
  double gs_coef[8];   // Gram-Schmidt coefficients <v_i|w> (complex, up to 3) + spare
  double gs_scale[2];  // 1/||w|| of the current Gram-Schmidt vector
  double parity_scale[2];
  int err[2];          // [0]: a bounded device wait ran out (QF_ETIMEOUT)
  double spare[1];
};

// Arguments of one pass of the FFT kinetic step.
template <typename R>
struct FftPassArgs {
  cpx<R>* data;           // field transformed in place (pass input and output)
  const cpx<R>* src;      // first pass only: read from here instead of data
  const cpx<R>* twiddle;  // exp(-2 pi i m / N), m in [0, N)
  const R* symbol;        // per-axis kinetic symbol S[j] (k_j^2 or 4 sin^2(k_j/2))
  int kinetic;            // KIN_FFT_*
  R tcoef;                // HK1/HK2: 1/(2 a^2 m N^3); HK3: 1/(a N^3)
  R am2;                  // (a m)^2 for HK3
  // final pass (inverse x + update) only:
  cpx<R>* psi;            // psi_t in, psi_{t+1} out (same sites)
  const void* v;          // potential: cpx<R> (complex) or R (real)
  int v_real;
  R half_dtau;            // dtau / 2
  R dtau;
  const double* scale;    // output scale (device scalar)
  double* partials;       // per-block FP64 sums when reducing
  int write_psi;          // 0: measure only (no write)
  int reduce;             // accumulate the kNumSums sums
  int emit_next;          // final pass that writes psi': also write its forward x transform
                          // into data, so the next step can skip its first pass
};

// Up to kGroupMax lattices of one size advanced by a single launch per pass.
constexpr int kGroupMax = 48;
template <typename R>
struct FftGroup {
  int count;
  FftPassArgs<R> a[kGroupMax];
};

// FDTD stencil step arguments (Eq. HK0 with Dirichlet planes).
template <typename R>
struct StencilArgs {
  const cpx<R>* in;
  cpx<R>* out;            // may be null when only measuring
  const void* v;
  int v_real;
  R kcoef;                // 1/(2 m a^2)
  R half_dtau;
  R dtau;
  R kd;                   // dtau * kcoef
  const double* scale;
  double* partials;
  int write_psi;
  int reduce;
};

// ---- block-level FP64 reduction of kNumSums values (deterministic order) ----------
template <int NV>
__device__ __forceinline__ void warp_sum(double (&s)[NV]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int i = 0; i < NV; ++i) s[i] += __shfl_down_sync(0xffffffffu, s[i], off);
  }
}

// Sums s over the block; thread 0 writes the result to out[0..NV).  scratch must hold
// 32*NV doubles.  Every thread of the block must call it.
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&s)[NV], double* scratch, double* out) {
  warp_sum<NV>(s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  __syncthreads();  // scratch may alias memory used just before
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) scratch[warp * NV + i] = s[i];
  }
  __syncthreads();
  if (warp == 0) {
    double t[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) t[i] = (lane < nwarps) ? scratch[lane * NV + i] : 0.0;
    warp_sum<NV>(t);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) out[i] = t[i];
    }
  }
}

// ---- per-thread sum accumulators ---------------------------------------------------
// Acc<double>: plain FP64.  Acc<float>: an unevaluated sum hi + lo of two floats
// ("double-float") updated with error-free transformations -- the product a*b = p + e
// with e = fma(a, b, -p) (Dekker) and the sum s = x + y with its exact error (Knuth's
// two-sum) -- so a thread's partial sum keeps ~48 significant bits while running on
// the FP32 pipes (FP64 throughput on this part is a small fraction of FP32).  Partial
// sums leave the thread as FP64 and every later stage of a reduction is FP64.
template <typename R>
struct Acc;
template <>
struct Acc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
  // a b + c d
  __device__ __forceinline__ void add_dot2(double a, double b, double c, double d) {
    v = fma(a, b, v);
    v = fma(c, d, v);
  }
  __device__ __forceinline__ double value() const { return v; }
};
template <>
struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float z = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(x, z));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    add(p);
    lo = __fadd_rn(lo, e);
  }
  // a b + c d formed in FP32 (within 2^-24 of its terms), then added exactly
  __device__ __forceinline__ void add_dot2(float a, float b, float c, float d) {
    add(__fmaf_rn(a, b, __fmul_rn(c, d)));
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

// The five sums of a check: <psi|psi>, Re/Im <psi|H_K psi>, Re/Im <psi|V psi>.  Kernels
// that hold only some of the parts at a site pass zeros for the others.
template <typename R>
struct CheckSums {
  Acc<R> n, kr, ki, vr, vi;
  __device__ __forceinline__ void add(cpx<R> p, cpx<R> h, cpx<R> v) {
    n.add_prod(p.x, p.x);
    n.add_prod(p.y, p.y);
    kr.add_prod(p.x, h.x);
    kr.add_prod(p.y, h.y);
    ki.add_prod(p.x, h.y);
    ki.add_prod(-p.y, h.x);
    const R w = p.x * p.x + p.y * p.y;
    vr.add_prod(w, v.x);
    vi.add_prod(w, v.y);
  }
  __device__ __forceinline__ void to(double (&s)[kNumSums]) const {
    s[0] = n.value();
    s[1] = kr.value();
    s[2] = ki.value();
    s[3] = vr.value();
    s[4] = vi.value();
  }
};

// Complex FP32 fields: the site's values |psi|^2, Re/Im conj(psi) H_K psi and
// Re/Im |psi|^2 V are formed in FP32 (a fused multiply-add pair each, within a few 2^-24
// of the site's terms, below the FP32 field's own rounding) and accumulated across
// sites in compensated (FP64-equivalent) sums: five additions per site instead of eight
// exact products.
template <>
struct CheckSums<float> {
  Acc<float> n, kr, ki, vr, vi;
  __device__ __forceinline__ void add(cpx<float> p, cpx<float> h, cpx<float> v) {
    const float w = __fmaf_rn(p.x, p.x, __fmul_rn(p.y, p.y));
    n.add(w);
    kr.add(__fmaf_rn(p.x, h.x, __fmul_rn(p.y, h.y)));
    ki.add(__fmaf_rn(p.x, h.y, __fmul_rn(-p.y, h.x)));
    vr.add(__fmul_rn(w, v.x));
    vi.add(__fmul_rn(w, v.y));
  }
  __device__ __forceinline__ void to(double (&s)[kNumSums]) const {
    s[0] = n.value();
    s[1] = kr.value();
    s[2] = ki.value();
    s[3] = vr.value();
    s[4] = vi.value();
  }
};

// ---- launchers (return cudaError_t of the launch) ------------------------------------
// FFT kinetic step psi_{t+1} = s (coef_A psi_t - coef_B dtau H_K psi_t) is five passes
// (0: x forward psi -> tmp, 1: y forward, 2: z forward x T(k) z inverse, 3: y inverse,
// 4: x inverse + update/sums); tmp is scratch.  nblocks_final: grid of the reducing pass.
constexpr int kFftPasses = 5;
// extra passes for plain transforms: forward = 0, 1, 5 (psi -> data); inverse, in place
// on data and unnormalised = 6 (z), 3 (y), 7 (x)
constexpr int kFftPassZForward = 5, kFftPassZInverse = 6, kFftPassXInverse = 7;
// alt_plan false: the twiddle region holds the first radix plan's table only, so the
// autotuner's plan choice is not used (the tile choice still is).
template <typename R>
cudaError_t launch_fft_pass(int n, int pass, FftPassArgs<R> args, cpx<R>* tmp, cudaStream_t st,
                            int* nblocks_final, bool alt_plan = true);
// One pass for a group of lattices of size n sharing real/complex V and check status
// (c64 only); each member's arguments are as launch_fft_pass would use them.
template <typename R>
cudaError_t launch_fft_group_pass(int n, int pass, const FftGroup<R>& g, cudaStream_t st, bool alt_plan = true);
// Number of blocks the reducing (final) pass of the FFT step uses for lattice size n.
template <typename R>
int fft_final_blocks(int n);

// The most partial rows any tile variant's reducing pass writes (workspace sizing).
template <typename R>
int fft_final_blocks_max(int n);
// Tile variant of the complex-FP32 four-pass kernels for size n: the choice (-1 while
// the autotuner has not run), the variant in use, and the setter (false for bad n/v).
int fft_tile_choice(int n);
int fft_tile_variant(int n);
bool set_fft_tile_choice(int n, int v);

// Whether the FFT path has kernels for this n.
bool fft_supported(int n);

template <typename R>
int stencil_blocks(int n, int zc = 0);

// Finishing reduction: sums nblocks partial rows in index order into sc->sums, then the
// energy; with set_scale also the step scales sc->scale[1..2] and their exponents k, j in
// sc->energy[3..4].  interval > 0: steps since the field last had about unit norm, from
// which the per-step decay is measured; interval 0: estimated from the energy and dtau.
cudaError_t launch_finish(const double* partials, int nblocks, DevScalars* sc, int set_scale,
                          cudaStream_t st, int interval = -1, double dtau = 0.0);

// Gram-Schmidt and field helpers (FP64 accumulation).
template <typename R>
cudaError_t launch_dots(const cpx<R>* const* basis, int nb, const cpx<R>* w, long long n_sites,
                        double* partials, int nblocks, cudaStream_t st);
cudaError_t launch_finish_dots(const double* partials, int nblocks, int nb, double* coef_out,
                               cudaStream_t st);
// w = src - sum_j c_j v_j (c from coef in device memory) and, of the stored w, the sums
// <v_j|w> and <w|w> into per-block partials (same layout as launch_dots).
template <typename R>
cudaError_t launch_axpy_dots(cpx<R>* w, const cpx<R>* src, const cpx<R>* const* basis, int nb,
                             const double* coef, long long n_sites, double* partials, int nblocks,
                             cudaStream_t st);
template <typename R>
cudaError_t launch_scale_copy(cpx<R>* dst, const cpx<R>* src, const double* s, long long n_sites,
                              cudaStream_t st);
template <typename R>
cudaError_t launch_parity(cpx<R>* dst, const cpx<R>* src, int n, int which, int axis,
                          double* partials, int nblocks, cudaStream_t st);
template <typename R>
cudaError_t launch_from_f64(cpx<R>* dst, const double* src, long long n_elems_complex, cudaStream_t st);
template <typename R>
cudaError_t launch_to_f64(double* dst, const cpx<R>* src, double factor, long long n_complex,
                          cudaStream_t st);
template <typename R>
cudaError_t launch_real_from_f64(R* dst, const double* src, long long n, cudaStream_t st);
template <typename R>
cudaError_t launch_pack_f64(cpx<R>* dst, const double* re, const double* im, long long n, cudaStream_t st);
int field_blocks();
// Radial momentum histogram of a transformed field (shells b = round(|n|)); see
// qf_fields.cu.  part: per-block integer histograms (blocks x nb); out: prob[nb].
template <typename R>
cudaError_t launch_momentum_hist(const cpx<R>* hat, int n, int nb, const double* norm, unsigned long long* part,
                                 int blocks, cudaStream_t st);
cudaError_t launch_momentum_finish(const unsigned long long* part, int blocks, int nb, double* prob, cudaStream_t st);
// Spectral zero-padding of an nc^3 transform into an (2 nc)^3 one (see qf_fields.cu).
template <typename R>
cudaError_t launch_pad_spectrum(const cpx<R>* coarse, int nc, cpx<R>* fine, double scale, cudaStream_t st);
// Twiddle table of radix plan p (0, or 1 for the sizes that have a second plan).
int fft_twiddle_count(int n, int p = 0);
void fft_twiddles(int n, double* re_im, int p = 0);
bool fft_has_alt_plan(int n);

}  // namespace qf
