// Host helpers of the fused FFT kinetic step: plan sizes and twiddle tables (kernels in
// qf_fft_impl.cuh; the complex-FP32 entry points are instantiated in qf_fft_group.cu).
#include <math.h>

#include <atomic>

#include "qf_fft_impl.cuh"

namespace qf {

template int fft_final_blocks<float>(int);
template int fft_final_blocks_max<float>(int);

bool fft_supported(int n) { return plan_stages(n) > 0; }

// Tile variant of the complex-FP32 four-pass kernels per FFT size: -1 until chosen
// (variant 0 runs meanwhile), else 0 or 1 (tile geometry), or 2 or 3 (the same with the
// second radix plan, for the sizes that have one).  Process-wide.
static int plan_index(int n) {
  switch (n) {
    case 8: return 0;
    case 12: return 1;
    case 16: return 2;
    case 24: return 3;
    case 32: return 4;
    case 48: return 5;
    case 64: return 6;
    case 96: return 7;
    case 128: return 8;
    case 192: return 9;
    case 256: return 10;
    case 384: return 11;
    case 512: return 12;
    default: return -1;
  }
}
static std::atomic<int> g_tile_variant[13] = {{-1}, {-1}, {-1}, {-1}, {-1}, {-1}, {-1},
                                              {-1}, {-1}, {-1}, {-1}, {-1}, {-1}};

int fft_tile_choice(int n) {
  const int i = plan_index(n);
  return i < 0 ? 0 : g_tile_variant[i].load(std::memory_order_relaxed);
}
int fft_tile_variant(int n) {
  const int v = fft_tile_choice(n);
  return v < 0 ? 0 : v;
}
bool fft_has_alt_plan(int n) { return has_alt_plan(n); }

bool set_fft_tile_choice(int n, int v) {
  const int i = plan_index(n);
  if (i < 0 || v < -1 || v > 3 || (v >= 2 && !has_alt_plan(n))) return false;
  g_tile_variant[i].store(v, std::memory_order_relaxed);
  return true;
}

// Host-side twiddle table in the per-stage layout the kernels read.
int fft_twiddle_count(int n, int p) {
  if (p == 1 && !has_alt_plan(n)) return 0;
  switch (n) {
#define QF_CASE(NN) \
  case NN:          \
    return p == 1 ? plan_tw_size(NN, 1) : plan_tw_size(NN);
    QF_CASE(8) QF_CASE(12) QF_CASE(16) QF_CASE(24) QF_CASE(32) QF_CASE(48) QF_CASE(64) QF_CASE(96)
    QF_CASE(128) QF_CASE(192) QF_CASE(256) QF_CASE(384) QF_CASE(512)
#undef QF_CASE
    default:
      return 0;
  }
}

// Fills tw[off(s) + k (R_s - 1) + r - 1] = exp(-2 pi i r k / (Ns R_s)) in double.
void fft_twiddles(int n, double* re_im, int p) {
  const double two_pi = 6.283185307179586476925286766559;
  int ns = 1, off = 0;
  for (int s = 0; s < plan_stages(n, p); ++s) {
    const int rad = plan_radix(n, s, p);
    for (int k = 0; k < ns; ++k)
      for (int r = 1; r < rad; ++r) {
        const long long num = (long long)r * k;
        const long long den = (long long)ns * rad;
        const double ang = -two_pi * (double)num / (double)den;
        const int idx = off + k * (rad - 1) + (r - 1);
        re_im[2 * idx] = cos(ang);
        re_im[2 * idx + 1] = sin(ang);
      }
    off += ns * (rad - 1);
    ns *= rad;
  }
}

}  // namespace qf
