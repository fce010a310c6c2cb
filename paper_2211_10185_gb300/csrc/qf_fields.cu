// Whole-field helpers: finishing reductions, Gram-Schmidt inner products and axpy
// (Sec. 1, excited states from snapshots), parity projectors (Sec. 3) and precision
// conversion at the host boundary.  All sums are FP64 and run in a fixed order, so
// repeated runs give bitwise-identical results.
#include <math.h>

#include "qf_common.cuh"

namespace qf {

constexpr int kFieldThreads = 256;
constexpr int kFieldUnroll = 4;  // independent sites per thread and round of the field loops
int field_blocks() { return 152 * 4; }  // 4 blocks per SM of the 152-SM GB300

// ------------------------------------------------------------------------------------
// Finishing reduction of per-block partial sums
// ------------------------------------------------------------------------------------
constexpr int kFinishThreads = 256;  // one block (1024 threads measured slower: 17 vs 14 us)

__global__ void __launch_bounds__(kFinishThreads) finish_kernel(const double* __restrict__ partials, int nblocks,
                                                     DevScalars* sc, int set_scale, int interval,
                                                     double dtau) {
  __shared__ double red_s[32 * kNumSums];
  __shared__ double tot[kNumSums];
  double s[kNumSums] = {0, 0, 0, 0, 0};
#pragma unroll 4
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int i = 0; i < kNumSums; ++i) s[i] += partials[(long long)b * kPartialStride + i];
  block_sum_store<kNumSums>(s, red_s, tot);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double nrm = tot[0];
    for (int i = 0; i < kNumSums; ++i) sc->sums[i] = tot[i];
    // E = (<psi|H_K psi> + <psi|V psi>) / <psi|psi>
    sc->energy[0] = (tot[1] + tot[3]) / nrm;
    sc->energy[1] = (tot[2] + tot[4]) / nrm;
    sc->energy[2] = nrm;
    if (set_scale) {
      // The field started the interval at about 2^j (unit norm times the centring power
      // of its renormalising step) and grew by lambda 2^k per step, lambda the step's
      // decay: log2 lambda ~ (log2(norm)/2 - j)/interval - k.  The next k cancels lambda
      // to within 2^(+-1/2) per step, and the next j starts the field at 2^(-r c/2) for the
      // residual r, so it ends the next interval of the same length near 2^(+r c/2).
      int k = (int)sc->energy[3], j = (int)sc->energy[4];
      if (interval > 0 && nrm > 0 && isfinite(nrm)) {
        const double lam = (0.5 * log2(nrm) - j) / interval - k;
        const double kn = fmin(fmax(rint(-lam), -30.0), 30.0);
        const double jn = fmin(fmax(-rint(0.5 * (lam + kn) * (interval - 1)), -60.0), 60.0);
        k = (int)kn;
        j = (int)jn;
      } else if (interval == 0 && dtau > 0 && nrm > 0) {
        // no decay measured yet: a state of energy E shrinks by about
        // (1 - dtau E/2) / (1 + dtau E/2) per step
        const double e = sc->energy[0];
        const double q = fabs((1.0 - 0.5 * dtau * e) / (1.0 + 0.5 * dtau * e));
        if (q > 0 && isfinite(q)) {
          k = (int)fmin(fmax(rint(-log2(q)), -30.0), 30.0);
          j = 0;
        }
      }
      sc->scale[1] = nrm > 0 ? ldexp(1.0, k + j) / sqrt(nrm) : ldexp(1.0, k + j);
      sc->scale[2] = ldexp(1.0, k);
      sc->energy[3] = (double)k;
      sc->energy[4] = (double)j;
    }
  }
}

cudaError_t launch_finish(const double* partials, int nblocks, DevScalars* sc, int set_scale, cudaStream_t st,
                          int interval, double dtau) {
  finish_kernel<<<1, kFinishThreads, 0, st>>>(partials, nblocks, sc, set_scale, interval, dtau);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Inner products <v_j|w> (j < nb <= 2) and <w|w>
// ------------------------------------------------------------------------------------
template <typename R>
struct Basis2 {
  const cpx<R>* v[2];
};

template <typename R, int NB>
__global__ void __launch_bounds__(kFieldThreads) dots_kernel(Basis2<R> basis, const cpx<R>* __restrict__ w,
                                                             long long n_sites, double* partials) {
  __shared__ double red_s[32 * kNumSums];
  Acc<R> acc[kNumSums];
  auto site = [&](const cpx<R>& x, const cpx<R>* u) {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      acc[2 * j].add_dot2(u[j].x, x.x, u[j].y, x.y);       // Re conj(u) w
      acc[2 * j + 1].add_dot2(u[j].x, x.y, -u[j].y, x.x);  // Im conj(u) w
    }
    acc[4].add_dot2(x.x, x.x, x.y, x.y);
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // kFieldUnroll sites per round with all their loads issued first (the same site order
  // as one site per round)
  for (; i + (kFieldUnroll - 1) * stride < n_sites; i += kFieldUnroll * stride) {
    cpx<R> x[kFieldUnroll], u[kFieldUnroll][NB > 0 ? NB : 1];
#pragma unroll
    for (int k = 0; k < kFieldUnroll; ++k) {
      x[k] = w[i + k * stride];
#pragma unroll
      for (int j = 0; j < NB; ++j) u[k][j] = basis.v[j][i + k * stride];
    }
#pragma unroll
    for (int k = 0; k < kFieldUnroll; ++k) site(x[k], u[k]);
  }
  for (; i < n_sites; i += stride) {
    cpx<R> u[NB > 0 ? NB : 1];
#pragma unroll
    for (int j = 0; j < NB; ++j) u[j] = basis.v[j][i];
    site(w[i], u);
  }
  double s[kNumSums];
#pragma unroll
  for (int i = 0; i < kNumSums; ++i) s[i] = acc[i].value();
  block_sum_store<kNumSums>(s, red_s, partials + (long long)blockIdx.x * kPartialStride);
}

template <typename R>
cudaError_t launch_dots(const cpx<R>* const* basis, int nb, const cpx<R>* w, long long n_sites, double* partials,
                        int nblocks, cudaStream_t st) {
  Basis2<R> b{{nb > 0 ? basis[0] : nullptr, nb > 1 ? basis[1] : nullptr}};
  if (nb == 0) dots_kernel<R, 0><<<nblocks, kFieldThreads, 0, st>>>(b, w, n_sites, partials);
  else if (nb == 1) dots_kernel<R, 1><<<nblocks, kFieldThreads, 0, st>>>(b, w, n_sites, partials);
  else dots_kernel<R, 2><<<nblocks, kFieldThreads, 0, st>>>(b, w, n_sites, partials);
  return cudaGetLastError();
}

// coef_out: [Re c0, Im c0, Re c1, Im c1, |w|^2, 1/|w|]
__global__ void __launch_bounds__(kFinishThreads) finish_dots_kernel(const double* __restrict__ partials, int nblocks,
                                                          double* coef_out) {
  __shared__ double red_s[32 * kNumSums];
  __shared__ double tot[kNumSums];
  double s[kNumSums] = {0, 0, 0, 0, 0};
#pragma unroll 4
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int i = 0; i < kNumSums; ++i) s[i] += partials[(long long)b * kPartialStride + i];
  block_sum_store<kNumSums>(s, red_s, tot);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < kNumSums; ++i) coef_out[i] = tot[i];
    coef_out[5] = tot[4] > 0 ? 1.0 / sqrt(tot[4]) : 0.0;
  }
}

cudaError_t launch_finish_dots(const double* partials, int nblocks, int nb, double* coef_out, cudaStream_t st) {
  (void)nb;
  finish_dots_kernel<<<1, kFinishThreads, 0, st>>>(partials, nblocks, coef_out);
  return cudaGetLastError();
}

// w = src - sum_j c_j v_j with c_j from device memory, then the sums <v_j|w> and <w|w> of
// the stored (rounded) w.  FP64 fields: the update is FP64.  FP32 fields: each FP64
// coefficient is split as c = c_hi + c_lo (two floats) and applied with fused
// multiply-adds, so the coefficient enters with ~48 bits; what rounding leaves along v_j
// is removed by the re-orthogonalisation pass that follows.
template <typename R>
__device__ __forceinline__ cpx<R> sub_cmul(cpx<R> w, double cr, double ci, cpx<R> u);
template <>
__device__ __forceinline__ cpx<double> sub_cmul<double>(cpx<double> w, double cr, double ci, cpx<double> u) {
  return mk<double>(w.x - (cr * u.x - ci * u.y), w.y - (cr * u.y + ci * u.x));
}
template <>
__device__ __forceinline__ cpx<float> sub_cmul<float>(cpx<float> w, double cr, double ci, cpx<float> u) {
  const float rh = float(cr), rl = float(cr - double(rh));
  const float ih = float(ci), il = float(ci - double(ih));
  float x = w.x, y = w.y;
  x = __fmaf_rn(-rh, u.x, x);
  x = __fmaf_rn(ih, u.y, x);
  x = __fmaf_rn(-rl, u.x, x);
  x = __fmaf_rn(il, u.y, x);
  y = __fmaf_rn(-rh, u.y, y);
  y = __fmaf_rn(-ih, u.x, y);
  y = __fmaf_rn(-rl, u.y, y);
  y = __fmaf_rn(-il, u.x, y);
  return mk<float>(x, y);
}

template <typename R, int NB>
__global__ void __launch_bounds__(kFieldThreads) axpy_dots_kernel(cpx<R>* w, const cpx<R>* src, Basis2<R> basis,
                                                                  const double* __restrict__ coef, long long n_sites,
                                                                  double* partials) {
  __shared__ double red_s[32 * kNumSums];
  double cr[2] = {0, 0}, ci[2] = {0, 0};
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    cr[j] = coef[2 * j];
    ci[j] = coef[2 * j + 1];
  }
  Acc<R> acc[kNumSums];
  // w may be src (in place): each site is read, then written, by the same thread
  auto site = [&](long long i, cpx<R> x, const cpx<R>* u) {
#pragma unroll
    for (int j = 0; j < NB; ++j) x = sub_cmul<R>(x, cr[j], ci[j], u[j]);
    w[i] = x;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      acc[2 * j].add_dot2(u[j].x, x.x, u[j].y, x.y);
      acc[2 * j + 1].add_dot2(u[j].x, x.y, -u[j].y, x.x);
    }
    acc[4].add_dot2(x.x, x.x, x.y, x.y);
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kFieldUnroll - 1) * stride < n_sites; i += kFieldUnroll * stride) {
    cpx<R> x[kFieldUnroll], u[kFieldUnroll][NB > 0 ? NB : 1];
#pragma unroll
    for (int k = 0; k < kFieldUnroll; ++k) {
      x[k] = src[i + k * stride];
#pragma unroll
      for (int j = 0; j < NB; ++j) u[k][j] = basis.v[j][i + k * stride];
    }
#pragma unroll
    for (int k = 0; k < kFieldUnroll; ++k) site(i + k * stride, x[k], u[k]);
  }
  for (; i < n_sites; i += stride) {
    cpx<R> u[NB > 0 ? NB : 1];
#pragma unroll
    for (int j = 0; j < NB; ++j) u[j] = basis.v[j][i];
    site(i, src[i], u);
  }
  double s[kNumSums];
#pragma unroll
  for (int i = 0; i < kNumSums; ++i) s[i] = acc[i].value();
  block_sum_store<kNumSums>(s, red_s, partials + (long long)blockIdx.x * kPartialStride);
}

template <typename R>
cudaError_t launch_axpy_dots(cpx<R>* w, const cpx<R>* src, const cpx<R>* const* basis, int nb, const double* coef,
                             long long n_sites, double* partials, int nblocks, cudaStream_t st) {
  Basis2<R> b{{nb > 0 ? basis[0] : nullptr, nb > 1 ? basis[1] : nullptr}};
  if (nb == 0) axpy_dots_kernel<R, 0><<<nblocks, kFieldThreads, 0, st>>>(w, src, b, coef, n_sites, partials);
  else if (nb == 1) axpy_dots_kernel<R, 1><<<nblocks, kFieldThreads, 0, st>>>(w, src, b, coef, n_sites, partials);
  else axpy_dots_kernel<R, 2><<<nblocks, kFieldThreads, 0, st>>>(w, src, b, coef, n_sites, partials);
  return cudaGetLastError();
}

// dst = src * s (s a device FP64 scalar).  FP64 fields multiply in FP64; FP32 fields by
// the scale rounded to FP32 (a uniform relative change of at most 2^-24: these scales
// are normalisations).
template <typename R>
__global__ void __launch_bounds__(kFieldThreads) scale_copy_kernel(cpx<R>* dst, const cpx<R>* src,
                                                                   const double* __restrict__ s, long long n) {
  const R f = R(*s);
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kFieldUnroll - 1) * stride < n; i += kFieldUnroll * stride) {
    cpx<R> x[kFieldUnroll];
#pragma unroll
    for (int k = 0; k < kFieldUnroll; ++k) x[k] = src[i + k * stride];
#pragma unroll
    for (int k = 0; k < kFieldUnroll; ++k) dst[i + k * stride] = mk<R>(x[k].x * f, x[k].y * f);
  }
  for (; i < n; i += stride) {
    const cpx<R> x = src[i];
    dst[i] = mk<R>(x.x * f, x.y * f);
  }
}

template <typename R>
cudaError_t launch_scale_copy(cpx<R>* dst, const cpx<R>* src, const double* s, long long n, cudaStream_t st) {
  scale_copy_kernel<R><<<field_blocks(), kFieldThreads, 0, st>>>(dst, src, s, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Parity projectors (Sec. 3).  Mirror of index i on an axis: (N - i) mod N, the site at
// coordinate -x_i.  P+- = (psi(r) +- psi(-r))/2;  P-_{p_k} = ((psi(r) + psi(r with the
// other two axes flipped)) - (psi(r with axis k flipped) + psi(-r)))/4.  The grouping
// makes mirror-image outputs bitwise equal (or exactly negated).
// ------------------------------------------------------------------------------------
template <typename R, bool IDX32>
__global__ void __launch_bounds__(kFieldThreads) parity_kernel(cpx<R>* __restrict__ dst, const cpx<R>* __restrict__ src,
                                                               int n, int which, int axis, double* partials) {
  __shared__ double red_s[32 * kNumSums];
  Acc<R> nrm;
  const long long total = (long long)n * n * n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    int ix, iy, iz;
    if constexpr (IDX32) {  // (32-bit divisions: several times cheaper than 64-bit ones)
      const unsigned u = (unsigned)i, t = u / (unsigned)n;
      ix = (int)(u - t * (unsigned)n);
      iy = (int)(t % (unsigned)n);
      iz = (int)(t / (unsigned)n);
    } else {
      ix = (int)(i % n);
      iy = (int)((i / n) % n);
      iz = (int)(i / ((long long)n * n));
    }
    const int mx = ix == 0 ? 0 : n - ix, my = iy == 0 ? 0 : n - iy, mz = iz == 0 ? 0 : n - iz;
    auto at = [&](int x, int y, int z) { return src[((long long)z * n + y) * n + x]; };
    const cpx<R> p = src[i];
    cpx<R> o;
    if (which == 0 || which == 1) {
      const cpx<R> q = at(mx, my, mz);
      o = which == 0 ? p + q : p - q;
      o = cscale<R>(o, R(0.5));
    } else if (which == 2) {
      // axis k in {1, 2, 3} = x, y, z; the other two axes flip together
      const int fx = axis == 1 ? ix : mx, fy = axis == 2 ? iy : my, fz = axis == 3 ? iz : mz;  // others flipped
      const int gx = axis == 1 ? mx : ix, gy = axis == 2 ? my : iy, gz = axis == 3 ? mz : iz;  // axis k flipped
      o = (p + at(fx, fy, fz)) - (at(gx, gy, gz) + at(mx, my, mz));
      o = cscale<R>(o, R(0.25));
    } else {
      // d-wave projectors: e = (1 + R_k)/2 psi at the four mirror images over the two other
      // axes (i, j), then (1 - R_i)(1 - R_j)/4 (which 3) or (1 + R_i)(1 + R_j)/4 followed by
      // the antisymmetrisation over exchanging i and j (which 4).  c[0..2] = (x, y, z).
      const int ka = axis - 1, ia = ka == 0 ? 1 : 0, ja = ka == 2 ? 1 : 2;
      auto mir = [&](int c) { return c == 0 ? 0 : n - c; };
      auto ev = [&](const int* c) {
        int d[3] = {c[0], c[1], c[2]};
        const cpx<R> a0 = at(d[0], d[1], d[2]);
        d[ka] = mir(d[ka]);
        return cscale<R>(a0 + at(d[0], d[1], d[2]), R(0.5));
      };
      auto quad = [&](const int* c, bool odd) {
        int cij[3] = {c[0], c[1], c[2]}, ci[3] = {c[0], c[1], c[2]}, cj[3] = {c[0], c[1], c[2]};
        cij[ia] = mir(c[ia]);
        cij[ja] = mir(c[ja]);
        ci[ia] = mir(c[ia]);
        cj[ja] = mir(c[ja]);
        const cpx<R> s1 = ev(c) + ev(cij), s2 = ev(ci) + ev(cj);
        return cscale<R>(odd ? s1 - s2 : s1 + s2, R(0.25));
      };
      const int c0[3] = {ix, iy, iz};
      if (which == 3) {
        o = quad(c0, true);
      } else {
        int cs[3] = {ix, iy, iz};
        cs[ia] = c0[ja];
        cs[ja] = c0[ia];
        o = cscale<R>(quad(c0, false) - quad(cs, false), R(0.5));
      }
    }
    dst[i] = o;
    nrm.add_dot2(o.x, o.x, o.y, o.y);
  }
  double s[kNumSums] = {0, 0, 0, 0, nrm.value()};  // slot 4 = squared norm (as the dots)
  block_sum_store<kNumSums>(s, red_s, partials + (long long)blockIdx.x * kPartialStride);
}

template <typename R>
cudaError_t launch_parity(cpx<R>* dst, const cpx<R>* src, int n, int which, int axis, double* partials, int nblocks,
                          cudaStream_t st) {
  if ((long long)n * n * n < (1LL << 31))
    parity_kernel<R, true><<<nblocks, kFieldThreads, 0, st>>>(dst, src, n, which, axis, partials);
  else
    parity_kernel<R, false><<<nblocks, kFieldThreads, 0, st>>>(dst, src, n, which, axis, partials);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Precision conversion at the host boundary
// ------------------------------------------------------------------------------------
// src may be device memory (the staging area) or page-locked host memory read over the
// host link, where 16-byte loads (when src is 16-byte aligned) move twice the data per
// request
template <typename R>
__global__ void from_f64_kernel(cpx<R>* dst, const double* __restrict__ src, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  if ((reinterpret_cast<unsigned long long>(src) & 15) == 0) {
    const double2* __restrict__ s2 = reinterpret_cast<const double2*>(src);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const double2 w = s2[i];
      dst[i] = mk<R>(R(w.x), R(w.y));
    }
  } else {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
      dst[i] = mk<R>(R(src[2 * i]), R(src[2 * i + 1]));
  }
}
template <typename R>
cudaError_t launch_from_f64(cpx<R>* dst, const double* src, long long n, cudaStream_t st) {
  from_f64_kernel<R><<<field_blocks(), kFieldThreads, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

template <typename R>
__global__ void to_f64_kernel(double* dst, const cpx<R>* __restrict__ src, double f, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const cpx<R> x = src[i];
    dst[2 * i] = double(x.x) * f;
    dst[2 * i + 1] = double(x.y) * f;
  }
}
template <typename R>
cudaError_t launch_to_f64(double* dst, const cpx<R>* src, double f, long long n, cudaStream_t st) {
  to_f64_kernel<R><<<field_blocks(), kFieldThreads, 0, st>>>(dst, src, f, n);
  return cudaGetLastError();
}

template <typename R>
__global__ void real_from_f64_kernel(R* dst, const double* __restrict__ src, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = R(src[i]);
}
template <typename R>
cudaError_t launch_real_from_f64(R* dst, const double* src, long long n, cudaStream_t st) {
  real_from_f64_kernel<R><<<field_blocks(), kFieldThreads, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

// complex potential from separate real / imaginary FP64 arrays
template <typename R>
__global__ void pack_f64_kernel(cpx<R>* dst, const double* __restrict__ re, const double* __restrict__ im,
                                long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = mk<R>(R(re[i]), R(im[i]));
}
template <typename R>
cudaError_t launch_pack_f64(cpx<R>* dst, const double* re, const double* im, long long n, cudaStream_t st) {
  pack_f64_kernel<R><<<field_blocks(), kFieldThreads, 0, st>>>(dst, re, im, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Momentum-space distribution (Sec. 3, Fig. 2 right): radial histogram of |Psi(k)|^2 over
// shells b = round(|n|) of the integer lattice momentum n_l in (-N/2, N/2].  Each
// contribution is scaled so the whole transform sums to 2^60 (Parseval: N^3 <psi|psi>)
// and added as a 64-bit integer, so the histogram does not depend on the order of the
// atomic additions.
// ------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kFieldThreads) momentum_hist_kernel(const cpx<R>* __restrict__ hat, int n, int nb,
                                                                      const double* __restrict__ norm,
                                                                      unsigned long long* part) {
  extern __shared__ unsigned long long hist_s[];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist_s[b] = 0ull;
  __syncthreads();
  const double total = *norm * (double)n * (double)n * (double)n;
  const double scale = total > 0 ? 1152921504606846976.0 / total : 0.0;  // 2^60 / total
  const long long sites = (long long)n * n * n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += stride) {
    const int jx = (int)(i % n), jy = (int)((i / n) % n), jz = (int)(i / ((long long)n * n));
    const int mx = jx <= n / 2 ? jx : jx - n, my = jy <= n / 2 ? jy : jy - n, mz = jz <= n / 2 ? jz : jz - n;
    const int b = (int)(sqrt((double)(mx * mx + my * my + mz * mz)) + 0.5);
    const cpx<R> h = hat[i];
    const double w = (double(h.x) * double(h.x) + double(h.y) * double(h.y)) * scale;
    atomicAdd(&hist_s[b], __double2ull_rn(w));
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) part[(long long)blockIdx.x * nb + b] = hist_s[b];
}

template <typename R>
cudaError_t launch_momentum_hist(const cpx<R>* hat, int n, int nb, const double* norm, unsigned long long* part,
                                 int blocks, cudaStream_t st) {
  momentum_hist_kernel<R><<<blocks, kFieldThreads, nb * sizeof(unsigned long long), st>>>(hat, n, nb, norm, part);
  return cudaGetLastError();
}

// prob[b] = sum over blocks of part[.][b] / sum over all shells (integer sums: exact)
__global__ void momentum_finish_kernel(const unsigned long long* __restrict__ part, int blocks, int nb, double* prob) {
  __shared__ unsigned long long tot_s;
  if (threadIdx.x == 0) tot_s = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    unsigned long long s = 0;
    for (int k = 0; k < blocks; ++k) s += part[(long long)k * nb + b];
    prob[b] = (double)s;
    atomicAdd(&tot_s, s);
  }
  __syncthreads();
  const double tot = (double)tot_s;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) prob[b] = tot > 0 ? prob[b] / tot : 0.0;
}

cudaError_t launch_momentum_finish(const unsigned long long* part, int blocks, int nb, double* prob, cudaStream_t st) {
  momentum_finish_kernel<<<1, 256, 0, st>>>(part, blocks, nb, prob);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Spectral prolongation nc -> nf = 2 nc on the same box: fine mode m_l in (-nf/2, nf/2]
// takes the coarse mode m_l (mod nc) with weight 1 if |m_l| < nc/2, with weight 1/2 if
// |m_l| = nc/2 (the coarse Nyquist coefficient split between +-nc/2), else 0, times
// `scale` (the inverse transform that follows is unnormalised).
// ------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kFieldThreads) pad_spectrum_kernel(const cpx<R>* __restrict__ coarse, int nc,
                                                                     cpx<R>* __restrict__ fine, double scale) {
  const int nf = 2 * nc, h = nc / 2;
  const long long total = (long long)nf * nf * nf;
  const long long stride = (long long)gridDim.x * blockDim.x;
  auto map = [&](int f, double* w) {
    const int m = f <= nf / 2 ? f : f - nf;
    const int am = m < 0 ? -m : m;
    *w = am < h ? 1.0 : (am == h ? 0.5 : 0.0);
    return (m % nc + nc) % nc;
  };
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int fx = (int)(i % nf), fy = (int)((i / nf) % nf), fz = (int)(i / ((long long)nf * nf));
    double wx, wy, wz;
    const int cx = map(fx, &wx), cy = map(fy, &wy), cz = map(fz, &wz);
    const double w = wx * wy * wz * scale;
    cpx<R> o = mk<R>(R(0), R(0));
    if (w != 0.0) {
      const cpx<R> c = coarse[((long long)cz * nc + cy) * nc + cx];
      o = mk<R>(R(double(c.x) * w), R(double(c.y) * w));
    }
    fine[i] = o;
  }
}

template <typename R>
cudaError_t launch_pad_spectrum(const cpx<R>* coarse, int nc, cpx<R>* fine, double scale, cudaStream_t st) {
  pad_spectrum_kernel<R><<<field_blocks(), kFieldThreads, 0, st>>>(coarse, nc, fine, scale);
  return cudaGetLastError();
}

#define QF_INST(R)                                                                                          \
  template cudaError_t launch_dots<R>(const cpx<R>* const*, int, const cpx<R>*, long long, double*, int,   \
                                      cudaStream_t);                                                        \
  template cudaError_t launch_axpy_dots<R>(cpx<R>*, const cpx<R>*, const cpx<R>* const*, int, const double*,  \
                                           long long, double*, int, cudaStream_t);                          \
  template cudaError_t launch_scale_copy<R>(cpx<R>*, const cpx<R>*, const double*, long long, cudaStream_t); \
  template cudaError_t launch_parity<R>(cpx<R>*, const cpx<R>*, int, int, int, double*, int, cudaStream_t); \
  template cudaError_t launch_from_f64<R>(cpx<R>*, const double*, long long, cudaStream_t);                 \
  template cudaError_t launch_to_f64<R>(double*, const cpx<R>*, double, long long, cudaStream_t);    \
  template cudaError_t launch_real_from_f64<R>(R*, const double*, long long, cudaStream_t);                 \
  template cudaError_t launch_pack_f64<R>(cpx<R>*, const double*, const double*, long long, cudaStream_t); \
  template cudaError_t launch_momentum_hist<R>(const cpx<R>*, int, int, const double*, unsigned long long*, int,  \
                                               cudaStream_t);                                                       \
  template cudaError_t launch_pad_spectrum<R>(const cpx<R>*, int, cpx<R>*, double, cudaStream_t);
QF_INST(float)
QF_INST(double)
#undef QF_INST

}  // namespace qf
