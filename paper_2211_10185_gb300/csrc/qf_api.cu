// C ABI of libqfdtd (declared in include/qfdtd.h): lattice handles over a caller-owned
// device workspace, the step loop with its checks and snapshots, Gram-Schmidt excited
// states and parity projection.  Every arithmetic step on fields runs in the kernels of
// qf_fft_impl.cuh (four-pass FFT step), qf_fft2.cuh (two-pass step, N = 128 and 256),
// qf_stencil_tma.cuh / qf_stencil_tb.cuh (FDTD steps) and qf_fields.cu; this file only
// sequences them.
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>
#include <string>
#include <algorithm>
#include <vector>

#include "../../include/qfdtd.h"
#include "qf_common.cuh"
#include "qf_stencil_tb.cuh"

namespace qf {
bool encode_stencil_map(CUtensorMap* map, void* field, int n, bool c64);
bool encode_tb_map(CUtensorMap* map, void* field, int n);
bool fft2_supported(int n);
int fft2_final_blocks(int n);
int fft2_measure_blocks(int n);
cudaError_t launch_fft2_group_pass(int n, int pass, const FftGroup<float>& g, cudaStream_t st);
cudaError_t launch_stencil_tb(const StencilTbArgs& g, cudaStream_t st);
cudaError_t launch_stencil_tb_group(const StencilTbGroup& g, cudaStream_t st);
cudaError_t launch_bounded_wait_probe(int* err, cudaStream_t st);
template <typename R>
cudaError_t launch_stencil_tma(const StencilTmaGroup<R>& g, cudaStream_t st);
template <typename R>
cudaError_t launch_pack_f64(cpx<R>* dst, const double* re, const double* im, long long n, cudaStream_t st);
}  // namespace qf

using namespace qf;

static const char* kVersion = "qfdtd-gb300 0.1 (sm_103a)";
static const size_t kAlign = 256;
static const size_t kStageBytes = size_t(32) << 20;  // host<->device staging, FP64 pairs

static size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Kernel kinds for the per-kernel timing of qf_profile.
enum KernelKind {
  K_FFT_X_FWD = 0, K_FFT_Y_FWD, K_FFT_Z_MID, K_FFT_Y_INV, K_FFT_X_INV_UPDATE, K_STENCIL, K_FINISH, K_GS_DOTS,
  K_GS_AXPY, K_SCALE_COPY, K_PARITY, K_CONVERT, K_FFT_X_INV_SUMS, K_STENCIL_SUMS, K_STENCIL_2STEP, K_FFT2_XY_FWD,
  K_FFT2_YZ_MID, K_FFT2_XY_INV_UPDATE, K_FFT2_XY_INV_SUMS, K_FFT2_XY_FWD_SUMS, K_FFT2_YZ_SUMS, K_NUM_KINDS
};
static const char* kKindNames[K_NUM_KINDS] = {"fft_x_fwd", "fft_y_fwd", "fft_z_mid_T", "fft_y_inv",
                                               "fft_x_inv_update", "stencil_step", "finish_sums", "gs_dots",
                                               "gs_axpy", "scale_copy", "parity", "convert", "fft_x_inv_sums",
                                               "stencil_sums", "stencil_2step", "fft2_xy_fwd", "fft2_yz_mid_T",
                                               "fft2_xy_inv_update", "fft2_xy_inv_sums", "fft2_xy_fwd_sums",
                                               "fft2_yz_sums"};
static const int kEventPool = 4096;

struct Layout {
  size_t field = 0, f[2] = {0, 0}, v = 0, snaps = 0, states = 0, plateau = 0, tw = 0, sym = 0, partials = 0,
         scalars = 0, stage = 0, stage_bytes = 0, total = 0;
  int max_blocks = 0;
};

static bool valid_n(int n) { return n >= 8 && n <= 1024 && n % 2 == 0; }

static Layout make_layout(const qf_lattice_desc& d) {
  Layout L;
  const size_t sites = (size_t)d.n * d.n * d.n;
  const size_t elem = d.prec == QF_PREC_C64 ? 8 : 16;
  L.field = align_up(sites * elem);
  size_t off = 0;
  L.f[0] = off;
  off += L.field;
  L.f[1] = off;
  off += L.field;
  L.v = off;
  off += L.field;  // complex V (a real V uses the first half)
  L.snaps = off;
  off += L.field * d.n_snap;
  L.states = off;
  off += L.field * 3;
  L.plateau = off;
  off += L.field * d.plateau_slots;
  L.tw = off;
  off += align_up(4 * elem * (size_t)(d.n + 64));  // the tables of up to two radix plans
  L.sym = off;
  off += align_up(elem * (size_t)d.n);
  // partial sums: the largest grid of any reducing kernel
  int mb = field_blocks();
  if (fft_supported(d.n)) {
    int fb = d.prec == QF_PREC_C64 ? fft_final_blocks_max<float>(d.n) : fft_final_blocks_max<double>(d.n);
    if (fb > mb) mb = fb;
  }
  if (d.prec == QF_PREC_C64 && fft2_supported(d.n) && fft2_measure_blocks(d.n) > mb) mb = fft2_measure_blocks(d.n);
  int sb = d.prec == QF_PREC_C64 ? stencil_blocks<float>(d.n) : stencil_blocks<double>(d.n);
  if (sb > mb) mb = sb;
  L.max_blocks = mb;
  L.partials = off;
  off += align_up((size_t)mb * kPartialStride * sizeof(double));
  L.scalars = off;
  off += align_up(sizeof(DevScalars));
  L.stage_bytes = sites * 16 < kStageBytes ? sites * 16 : kStageBytes;
  L.stage = off;
  off += align_up(L.stage_bytes);
  L.total = off;
  return L;
}

struct qf_lattice {
  qf_lattice_desc d;
  Layout L;
  char* ws = nullptr;
  cudaStream_t st = nullptr;
  long long sites = 0;
  int live = 0;  // index of the live psi buffer (the other is scratch / next)
  int kinetic = -1;
  double mass = 0, dtau = 0;
  bool have_v = false, v_real = false, have_psi = false;
  int64_t step = 0;
  double tau = 0;
  bool pending_scale = false;
  // Power-of-two scale of the stored fields (DevScalars::scale): the live field holds
  // 2^K psi, snapshot slot j holds 2^snapK[j] psi; kcur is the exponent each step applies,
  // K_check the live field's exponent at the last check, renorm_step the step whose output
  // was last renormalised (-1: none since the field was set).
  int kcur = 0, jcur = 0;  // exponents of the steps and of the renormalising step's centring
  long long K = 0, K_check = 0, snapK[3] = {0, 0, 0};
  int64_t renorm_step = -1;
  bool have_prev = false;
  double prev_re = 0, prev_im = 0;
  double prev_de = INFINITY;  // |E| difference at the previous check (extrapolated rule)
  bool have_last = false;
  qf_energy last{};
  int snap_count = 0, snap_head = -1;  // snap_head: slot of the latest snapshot
  bool have_states[3] = {false, false, false};
  // plateau of E_i(tau) (qf_track_excited): records so far, the previous record, and per
  // state the chosen record with its energy and |E_i(tau_j) - E_i(tau_{j-1})|
  int exc_records = 0, exc_n = 0;
  qf_energy exc_prev[3] = {};
  bool plat_have[3] = {false, false, false};
  qf_energy plat[3] = {};
  int plat_rec[3] = {0, 0, 0};
  bool have_plateau_state[3] = {false, false, false};
  // the scratch field holds the forward x transform of the live psi (written by the
  // previous step's final pass), so the next FFT step starts at its second pass
  bool xfwd_valid = false;
  // CUDA graphs of the check_every-1 steps that follow a check (see run_chunk_graph)
  struct Graph {
    int check_every, live, tblock, kzero;
    cudaGraphExec_t exec;
    int flips;         // FDTD buffer swaps done by the replay
    int64_t launches;  // kernels in the graph
  };
  std::vector<Graph> graphs;
  bool use_graphs = true;
  // tensor maps of the two field buffers for the TMA-staged stencil (one-site halo) and
  // for the two-step stencil (two-site halo, complex FP32)
  CUtensorMap fmap[2];
  bool fmap_ok = false;
  CUtensorMap tbmap[2];
  bool tbmap_ok = false;
  // FDTD steps fused per pass (1 or 2) and whether the live field is known to be zero on
  // the Dirichlet planes (it is after any FDTD step), which the two-step kernel needs
  int tblock = 2;
  bool clean = false;
  // N = 128 and 256 complex-FP32 FFT steps in two passes over HBM (qf_fft2.cuh) instead of four;
  // the scratch field then holds the four-step layout, so switching drops xfwd_valid
  bool two_pass = true;
  std::string err;
  // launch accounting and optional CUDA-event timing per kernel kind
  int64_t launches = 0;
  bool prof = false;
  std::vector<cudaEvent_t> ev_free;
  struct Pend {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pend> pend;
  int64_t prof_count[K_NUM_KINDS] = {};
  double prof_ms[K_NUM_KINDS] = {};

  void* field(int i) const { return ws + L.f[i]; }
  void* psi() const { return field(live); }
  void* tmp() const { return field(1 - live); }
  void* snap(int j) const { return ws + L.snaps + L.field * j; }
  void* state(int i) const { return ws + L.states + L.field * i; }
  void* plateau_state(int i) const { return ws + L.plateau + L.field * i; }
  void reset_plateau() {
    exc_records = 0;
    exc_n = 0;
    for (int i = 0; i < 3; ++i) plat_have[i] = have_plateau_state[i] = false;
  }
  double* partials() const { return reinterpret_cast<double*>(ws + L.partials); }
  DevScalars* sc() const { return reinterpret_cast<DevScalars*>(ws + L.scalars); }
  double* stage() const { return reinterpret_cast<double*>(ws + L.stage); }
  bool c64() const { return d.prec == QF_PREC_C64; }
};

// The FFT step of this lattice runs the two-pass kernels.
static bool uses_fft2(const qf_lattice* lat) {
  return lat->two_pass && lat->c64() && lat->kinetic != QF_KIN_FDTD && fft2_supported(lat->d.n);
}

static void drop_graphs(qf_lattice* lat) {
  for (auto& g : lat->graphs) cudaGraphExecDestroy(g.exec);
  lat->graphs.clear();
}

static qf_status fail(qf_lattice* lat, qf_status s, const std::string& msg) {
  if (lat) lat->err = msg;
  return s;
}
static qf_status cuda_fail(qf_lattice* lat, cudaError_t e, const char* where) {
  return fail(lat, QF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define QF_CUDA(lat, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(lat, e_, #call); \
  } while (0)

// Reads back the timings of finished launches (the stream must be synchronised).
static void prof_harvest(qf_lattice* lat) {
  for (auto& p : lat->pend) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      lat->prof_count[p.kind] += 1;
      lat->prof_ms[p.kind] += ms;
    }
    lat->ev_free.push_back(p.a);
    lat->ev_free.push_back(p.b);
  }
  lat->pend.clear();
}

// Runs one kernel launch f(); counts it and, when profiling, brackets it with events.
template <typename F>
static cudaError_t launch(qf_lattice* lat, int kind, F&& f) {
  lat->launches += 1;
  if (!lat->prof) return f();
  if (lat->ev_free.size() < 2) {
    cudaError_t e = cudaStreamSynchronize(lat->st);
    if (e != cudaSuccess) return e;
    prof_harvest(lat);
  }
  cudaEvent_t a = lat->ev_free.back();
  lat->ev_free.pop_back();
  cudaEvent_t b = lat->ev_free.back();
  lat->ev_free.pop_back();
  cudaEventRecord(a, lat->st);
  cudaError_t e = f();
  cudaEventRecord(b, lat->st);
  lat->pend.push_back({kind, a, b});
  return e;
}

static bool desc_ok(const qf_lattice_desc* d) {
  return d && valid_n(d->n) && d->a > 0 && isfinite(d->a) && (d->prec == QF_PREC_C64 || d->prec == QF_PREC_C128) &&
         d->n_snap >= 1 && d->n_snap <= 3 && d->plateau_slots >= 0 && d->plateau_slots <= 3;
}

extern "C" qf_status qf_workspace_bytes(const qf_lattice_desc* desc, size_t* bytes) {
  if (!desc_ok(desc) || !bytes) return QF_EINVAL;
  *bytes = make_layout(*desc).total;
  return QF_OK;
}

extern "C" qf_status qf_create_lattice(const qf_lattice_desc* desc, void* dev_ws, size_t ws_bytes, void* stream,
                                       qf_lattice** out) {
  if (!out) return QF_EINVAL;
  *out = nullptr;
  if (!desc_ok(desc) || !dev_ws) return QF_EINVAL;
  if (reinterpret_cast<uintptr_t>(dev_ws) % kAlign) return QF_EINVAL;
  Layout L = make_layout(*desc);
  if (ws_bytes < L.total) return QF_ENOMEM;
  qf_lattice* lat = new (std::nothrow) qf_lattice();
  if (!lat) return QF_ENOMEM;
  lat->d = *desc;
  lat->L = L;
  lat->ws = static_cast<char*>(dev_ws);
  lat->st = static_cast<cudaStream_t>(stream);
  lat->sites = (long long)desc->n * desc->n * desc->n;
  cudaError_t e = cudaMemsetAsync(lat->ws, 0, L.total, lat->st);
  if (e == cudaSuccess) {
    DevScalars init{};
    init.scale[0] = 1.0;
    init.scale[1] = 1.0;
    init.scale[2] = 1.0;
    e = cudaMemcpyAsync(lat->sc(), &init, sizeof(init), cudaMemcpyHostToDevice, lat->st);
  }
  if (e == cudaSuccess && fft_supported(desc->n)) {
    // per-stage twiddle table exp(-2 pi i r k/(Ns R)) in the lattice precision; complex-FP32
    // lattices of sizes with a second radix plan hold its table right after the first
    const int cnt0 = fft_twiddle_count(desc->n);
    const int cnt1 = desc->prec == QF_PREC_C64 ? fft_twiddle_count(desc->n, 1) : 0;
    const int cnt = cnt0 + cnt1;
    double* tw = new double[2 * (size_t)cnt + 2];
    fft_twiddles(desc->n, tw);
    if (cnt1 > 0) fft_twiddles(desc->n, tw + 2 * (size_t)cnt0, 1);
    if (desc->prec == QF_PREC_C64) {
      float* f = new float[2 * (size_t)cnt + 2];
      for (int i = 0; i < 2 * cnt; ++i) f[i] = (float)tw[i];
      e = cudaMemcpyAsync(lat->ws + L.tw, f, sizeof(float) * 2 * cnt, cudaMemcpyHostToDevice, lat->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
      delete[] f;
    } else {
      e = cudaMemcpyAsync(lat->ws + L.tw, tw, sizeof(double) * 2 * cnt, cudaMemcpyHostToDevice, lat->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
    }
    delete[] tw;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
  if (e != cudaSuccess) {
    delete lat;
    return QF_ECUDA;
  }
  lat->fmap_ok = encode_stencil_map(&lat->fmap[0], lat->field(0), desc->n, desc->prec == QF_PREC_C64) &&
                 encode_stencil_map(&lat->fmap[1], lat->field(1), desc->n, desc->prec == QF_PREC_C64);
  lat->tbmap_ok = desc->prec == QF_PREC_C64 && encode_tb_map(&lat->tbmap[0], lat->field(0), desc->n) &&
                  encode_tb_map(&lat->tbmap[1], lat->field(1), desc->n);
  *out = lat;
  return QF_OK;
}

extern "C" qf_status qf_destroy_lattice(qf_lattice* lat) {
  if (!lat) return QF_OK;
  cudaStreamSynchronize(lat->st);
  prof_harvest(lat);
  for (cudaEvent_t e : lat->ev_free) cudaEventDestroy(e);
  drop_graphs(lat);
  delete lat;
  return QF_OK;
}

// Uploads n doubles (host) to the staging area in chunks and runs fn(stage, first, count)
// after each chunk.
template <typename F>
static qf_status staged_upload(qf_lattice* lat, const double* host, long long n, long long per_item, F fn) {
  // page-locked host memory is read by the conversion kernel itself over the host link,
  // in one launch (no staging copies, one synchronisation)
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, host) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
      attr.devicePointer != nullptr) {
    QF_CUDA(lat, launch(lat, K_CONVERT, [&] { return fn(reinterpret_cast<double*>(attr.devicePointer), 0, n); }));
    QF_CUDA(lat, cudaStreamSynchronize(lat->st));
    return QF_OK;
  }
  cudaGetLastError();  // (a pageable pointer is not an error)
  const long long chunk = (long long)(lat->L.stage_bytes / sizeof(double)) / per_item;
  for (long long first = 0; first < n; first += chunk) {
    const long long cnt = (n - first < chunk) ? n - first : chunk;
    QF_CUDA(lat, cudaMemcpyAsync(lat->stage(), host + first * per_item, cnt * per_item * sizeof(double),
                                 cudaMemcpyHostToDevice, lat->st));
    QF_CUDA(lat, launch(lat, K_CONVERT, [&] { return fn(lat->stage(), first, cnt); }));
    // the staging area is reused by the next chunk
    QF_CUDA(lat, cudaStreamSynchronize(lat->st));
  }
  return QF_OK;
}

extern "C" qf_status qf_set_potential(qf_lattice* lat, const double* v_re, const double* v_im) {
  if (!lat || !v_re) return fail(lat, QF_EINVAL, "null potential");
  const long long n = lat->sites;
  char* vbase = lat->ws + lat->L.v;
  qf_status s;
  if (!v_im) {
    s = staged_upload(lat, v_re, n, 1, [&](double* stg, long long first, long long cnt) {
      return lat->c64() ? launch_real_from_f64<float>(reinterpret_cast<float*>(vbase) + first, stg, cnt, lat->st)
                        : launch_real_from_f64<double>(reinterpret_cast<double*>(vbase) + first, stg, cnt, lat->st);
    });
  } else {
    // real and imaginary halves of one chunk share the staging area
    const long long chunk = (long long)(lat->L.stage_bytes / sizeof(double)) / 2;
    s = QF_OK;
    for (long long first = 0; first < n && s == QF_OK; first += chunk) {
      const long long cnt = (n - first < chunk) ? n - first : chunk;
      double* re = lat->stage();
      double* im = lat->stage() + chunk;
      QF_CUDA(lat, cudaMemcpyAsync(re, v_re + first, cnt * sizeof(double), cudaMemcpyHostToDevice, lat->st));
      QF_CUDA(lat, cudaMemcpyAsync(im, v_im + first, cnt * sizeof(double), cudaMemcpyHostToDevice, lat->st));
      cudaError_t e = launch(lat, K_CONVERT, [&] {
        return lat->c64()
                   ? launch_pack_f64<float>(reinterpret_cast<cpx<float>*>(vbase) + first, re, im, cnt, lat->st)
                   : launch_pack_f64<double>(reinterpret_cast<cpx<double>*>(vbase) + first, re, im, cnt, lat->st);
      });
      QF_CUDA(lat, e);
      QF_CUDA(lat, cudaStreamSynchronize(lat->st));
    }
  }
  if (s != QF_OK) return s;
  lat->have_v = true;
  lat->v_real = (v_im == nullptr);
  drop_graphs(lat);
  lat->reset_plateau();
  return QF_OK;
}

static double default_dtau(int kin, double a, double m) {
  double tmax;
  if (kin == QF_KIN_FDTD || kin == QF_KIN_FFT_SYMANZIK) tmax = 6.0 / (m * a * a);
  else if (kin == QF_KIN_FFT_NAIVE) tmax = 3.0 * M_PI * M_PI / (2.0 * m * a * a);
  else tmax = sqrt(12.0 + (a * m) * (a * m)) / a;
  return 0.75 / tmax;
}

extern "C" qf_status qf_set_kinetic(qf_lattice* lat, int kinetic, double mass, double dtau) {
  if (!lat) return QF_EINVAL;
  if (kinetic < QF_KIN_FDTD || kinetic > QF_KIN_FFT_REL) return fail(lat, QF_EINVAL, "unknown kinetic term");
  if (!(mass > 0) || !isfinite(mass) || !isfinite(dtau)) return fail(lat, QF_EINVAL, "mass must be > 0");
  if (kinetic != QF_KIN_FDTD && !fft_supported(lat->d.n))
    return fail(lat, QF_EINVAL, "no FFT plan for this N (use 8,12,16,24,32,48,64,96,128,192,256,384,512)");
  const double a = lat->d.a;
  drop_graphs(lat);
  lat->reset_plateau();
  lat->clean = false;
  lat->kinetic = kinetic;
  lat->mass = mass;
  lat->dtau = dtau > 0 ? dtau : default_dtau(kinetic, a, mass);
  if (kinetic != QF_KIN_FDTD) {
    // per-axis symbol S[j]: k_j^2 (HK1) or 4 sin^2(k_j/2) (HK2, HK3), k_j in (-pi, pi]
    const int n = lat->d.n;
    double* s = new double[n];
    for (int j = 0; j < n; ++j) {
      const double k = 2.0 * M_PI * (double)(j <= n / 2 ? j : j - n) / (double)n;
      s[j] = kinetic == QF_KIN_FFT_NAIVE ? k * k : 4.0 * sin(0.5 * k) * sin(0.5 * k);
    }
    cudaError_t e;
    if (lat->c64()) {
      float* f = new float[n];
      for (int j = 0; j < n; ++j) f[j] = (float)s[j];
      e = cudaMemcpyAsync(lat->ws + lat->L.sym, f, sizeof(float) * n, cudaMemcpyHostToDevice, lat->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
      delete[] f;
    } else {
      e = cudaMemcpyAsync(lat->ws + lat->L.sym, s, sizeof(double) * n, cudaMemcpyHostToDevice, lat->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
    }
    delete[] s;
    if (e != cudaSuccess) return cuda_fail(lat, e, "symbol upload");
  }
  return QF_OK;
}

extern "C" qf_status qf_set_wavefunction(qf_lattice* lat, const double* re_im) {
  if (!lat || !re_im) return fail(lat, QF_EINVAL, "null wavefunction");
  void* dst = lat->psi();
  qf_status s = staged_upload(lat, re_im, lat->sites, 2, [&](double* stg, long long first, long long cnt) {
    return lat->c64() ? launch_from_f64<float>(reinterpret_cast<cpx<float>*>(dst) + first, stg, cnt, lat->st)
                      : launch_from_f64<double>(reinterpret_cast<cpx<double>*>(dst) + first, stg, cnt, lat->st);
  });
  if (s != QF_OK) return s;
  lat->have_psi = true;
  lat->pending_scale = false;
  lat->xfwd_valid = false;
  lat->clean = false;
  lat->reset_plateau();
  lat->K = 0;
  lat->renorm_step = -1;
  return QF_OK;
}

static void* slot_ptr(qf_lattice* lat, int slot) {
  if (slot == -1) return lat->psi();
  if (slot >= 0 && slot < 3) return lat->have_states[slot] ? lat->state(slot) : nullptr;
  if (slot >= 200 && slot < 200 + lat->d.plateau_slots)
    return lat->have_plateau_state[slot - 200] ? lat->plateau_state(slot - 200) : nullptr;
  if (slot >= 100 && slot < 100 + lat->d.n_snap) {
    const int j = slot - 100;
    if (j >= lat->snap_count) return nullptr;
    const int idx = ((lat->snap_head - j) % lat->d.n_snap + lat->d.n_snap) % lat->d.n_snap;
    return lat->snap(idx);
  }
  return nullptr;
}

// Power of two the stored field of a slot carries (the live field and snapshots; the
// normalised states carry none).
static long long slot_exp2(const qf_lattice* lat, int slot) {
  if (slot == -1) return lat->K;
  if (slot >= 100 && slot < 100 + lat->d.n_snap) {
    const int j = slot - 100;
    const int idx = ((lat->snap_head - j) % lat->d.n_snap + lat->d.n_snap) % lat->d.n_snap;
    return lat->snapK[idx];
  }
  return 0;
}

extern "C" qf_status qf_get_wavefunction(qf_lattice* lat, int slot, double* re_im) {
  if (!lat || !re_im) return fail(lat, QF_EINVAL, "null output");
  void* src = slot_ptr(lat, slot);
  if (!src) return fail(lat, QF_ESTATE, "slot holds no field");
  const double f = ldexp(1.0, (int)-slot_exp2(lat, slot));
  const long long chunk = (long long)(lat->L.stage_bytes / sizeof(double)) / 2;
  for (long long first = 0; first < lat->sites; first += chunk) {
    const long long cnt = (lat->sites - first < chunk) ? lat->sites - first : chunk;
    cudaError_t e = launch(lat, K_CONVERT, [&] {
      return lat->c64() ? launch_to_f64<float>(lat->stage(), reinterpret_cast<cpx<float>*>(src) + first, f,
                                               cnt, lat->st)
                        : launch_to_f64<double>(lat->stage(), reinterpret_cast<cpx<double>*>(src) + first, f,
                                                cnt, lat->st);
    });
    QF_CUDA(lat, e);
    QF_CUDA(lat, cudaMemcpyAsync(re_im + 2 * first, lat->stage(), cnt * 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                 lat->st));
    QF_CUDA(lat, cudaStreamSynchronize(lat->st));
  }
  return QF_OK;
}

extern "C" qf_status qf_field_pointer(qf_lattice* lat, int slot, void** dev_ptr) {
  if (!lat || !dev_ptr) return QF_EINVAL;
  void* p = slot_ptr(lat, slot);
  if (!p) return fail(lat, QF_ESTATE, "slot holds no field");
  *dev_ptr = p;
  return QF_OK;
}

// Arguments of the FFT passes / the stencil for one lattice (kernels in qf_fft_impl.cuh and
// qf_stencil.cu); `in` is the field the kinetic term acts on.
template <typename R>
static FftPassArgs<R> fft_args(qf_lattice* lat, void* in, bool write, bool reduce, const double* scale) {
  const int n = lat->d.n;
  const double a = lat->d.a, m = lat->mass, dt = lat->dtau;
  const double n3 = (double)n * n * n;
  FftPassArgs<R> p{};
  p.twiddle = reinterpret_cast<const cpx<R>*>(lat->ws + lat->L.tw);
  p.symbol = reinterpret_cast<const R*>(lat->ws + lat->L.sym);
  p.kinetic = lat->kinetic;
  p.tcoef = (R)(lat->kinetic == QF_KIN_FFT_REL ? 1.0 / (a * n3) : 1.0 / (2.0 * a * a * m * n3));
  p.am2 = (R)((a * m) * (a * m));
  p.psi = reinterpret_cast<cpx<R>*>(in);
  p.v = lat->ws + lat->L.v;
  p.v_real = lat->v_real;
  p.half_dtau = (R)(0.5 * dt);
  p.dtau = (R)dt;
  p.scale = scale;
  p.partials = lat->partials();
  p.write_psi = write ? 1 : 0;
  p.reduce = reduce ? 1 : 0;
  p.data = reinterpret_cast<cpx<R>*>(lat->tmp());
  return p;
}

template <typename R>
static StencilArgs<R> stencil_args(qf_lattice* lat, void* in, void* out, bool write, bool reduce,
                                   const double* scale) {
  const double a = lat->d.a, m = lat->mass, dt = lat->dtau;
  return StencilArgs<R>{reinterpret_cast<const cpx<R>*>(in), reinterpret_cast<cpx<R>*>(out), lat->ws + lat->L.v,
                        lat->v_real, (R)(1.0 / (2.0 * m * a * a)), (R)(0.5 * dt), (R)dt,
                        (R)(dt / (2.0 * m * a * a)), scale, lat->partials(),
                        write ? 1 : 0, reduce ? 1 : 0};
}

// Appends lattice `lat` (input field `in`) to a TMA stencil group; the tensor map of a
// field buffer is cached, others (state slots) are encoded on the spot.
template <typename R>
static bool stencil_group_member(qf_lattice* lat, void* in, void* out, bool write, bool reduce, const double* scale,
                                 StencilTmaGroup<R>& g, bool first = true, int zc = kStencilZChunks[2]) {
  if (first) {
    g.count = 0;
    g.err = &lat->sc()->err[0];
  }
  const int i = g.count;
  if (i >= kGroupMax) return false;
  g.nm[i] = lat->d.n;
  g.zcm[i] = zc;
  if (in == lat->field(0) && lat->fmap_ok) g.map[i] = lat->fmap[0];
  else if (in == lat->field(1) && lat->fmap_ok) g.map[i] = lat->fmap[1];
  else if (!encode_stencil_map(&g.map[i], in, lat->d.n, lat->c64())) return false;
  g.a[i] = stencil_args<R>(lat, in, out, write, reduce, scale);
  g.count = i + 1;
  return true;
}

// ---- autotuner: z-chunk of the TMA stencil, per (N, precision), process-wide ----------
static std::mutex g_tune_mu;
static std::vector<std::pair<long long, int>> g_tuned_zc;  // key (n * 2 + c64) -> zc

template <typename R>
static int tuned_zchunk(qf_lattice* lat) {
  const long long key = (long long)lat->d.n * 2 + (lat->c64() ? 1 : 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& kv : g_tuned_zc)
      if (kv.first == key) return kv.second;
  }
  // time one step (psi -> scratch, no sums) for each candidate; the scratch field is
  // overwritten by the real step afterwards
  int best = kStencilZChunks[2];
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return best;
  for (int zc : kStencilZChunks) {
    StencilTmaGroup<R> g;
    if (!stencil_group_member<R>(lat, lat->psi(), lat->tmp(), true, false, &lat->sc()->scale[0], g, true, zc)) break;
    float ms = 0, tot = 0;
    bool ok = launch_stencil_tma<R>(g, lat->st) == cudaSuccess;  // warm-up
    for (int rep = 0; rep < 3 && ok; ++rep) {
      ok = cudaEventRecord(e0, lat->st) == cudaSuccess && launch_stencil_tma<R>(g, lat->st) == cudaSuccess &&
           cudaEventRecord(e1, lat->st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      tot += ms;
    }
    lat->launches += 4;
    if (ok && tot < best_ms) {
      best_ms = tot;
      best = zc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned_zc.push_back({key, best});
  return best;
}

// ---- autotuner: tile geometry and radix plan of the complex-FP32 four-pass FFT, per N ---
// On the first four-pass FFT step of a size, every variant (two tile geometries, times two
// radix plans where the size has a second one) times the five passes of a step (the
// reducing pass measuring only: psi is untouched, the scratch field is overwritten) and
// the fastest is kept for the process.  Never runs while the stream is being captured.
static void tune_fft_tiles(qf_lattice* lat) {
  const int n = lat->d.n;
  if (!lat->c64() || lat->kinetic == QF_KIN_FDTD || uses_fft2(lat) || fft_tile_choice(n) >= 0) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(lat->st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (fft_tile_choice(n) >= 0) return;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return;
  }
  FftPassArgs<float> p = fft_args<float>(lat, lat->psi(), false, true, &lat->sc()->scale[0]);
  p.emit_next = 0;
  float best_ms = 1e30f;
  int best = 0;
  const int nvar = fft_has_alt_plan(n) ? 4 : 2;
  for (int v = 0; v < nvar; ++v) {
    set_fft_tile_choice(n, v);
    auto step = [&] {
      cudaError_t e = cudaSuccess;
      for (int ps = 0; ps < kFftPasses && e == cudaSuccess; ++ps)
        e = launch_fft_pass<float>(n, ps, p, p.data, lat->st, nullptr);
      return e;
    };
    bool ok = step() == cudaSuccess;  // warm-up
    float ms = 0, tot = 0;
    for (int rep = 0; rep < 3 && ok; ++rep) {
      ok = cudaEventRecord(e0, lat->st) == cudaSuccess && step() == cudaSuccess &&
           cudaEventRecord(e1, lat->st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      tot += ms;
    }
    lat->launches += 4 * kFftPasses;
    if (ok && tot < best_ms) {
      best_ms = tot;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  set_fft_tile_choice(n, best);
  lat->xfwd_valid = false;  // the scratch field was overwritten
}

// Reads and clears the bounded-wait failure flag of a lattice.
static qf_status check_device_error(qf_lattice* lat) {
  int err = 0;
  QF_CUDA(lat, cudaMemcpyAsync(&err, &lat->sc()->err[0], sizeof(int), cudaMemcpyDeviceToHost, lat->st));
  QF_CUDA(lat, cudaStreamSynchronize(lat->st));
  if (err) {
    QF_CUDA(lat, cudaMemsetAsync(&lat->sc()->err[0], 0, sizeof(int), lat->st));
    return fail(lat, QF_ETIMEOUT, "a bounded device wait ran out (copy engine did not complete)");
  }
  return QF_OK;
}

// ---- two FDTD steps per pass (complex FP32) ----------------------------------------------
static void tb_args(qf_lattice* lat, const double* scale, int nzb, StencilTbArgs& g) {
  const double a = lat->d.a, m = lat->mass, dt = lat->dtau;
  g.map = lat->tbmap[lat->live];
  g.out = reinterpret_cast<cpx<float>*>(lat->tmp());
  g.v = lat->ws + lat->L.v;
  g.v_real = lat->v_real ? 1 : 0;
  // the same single-precision constants as the single-step kernel
  g.half_dtau = (float)(0.5 * dt);
  g.kd = (float)(dt / (2.0 * m * a * a));
  g.scale = scale;
  g.n = lat->d.n;
  g.nzb = nzb;
  g.err = &lat->sc()->err[0];
}

static std::vector<std::pair<long long, int>> g_tuned_tb;  // key n -> z-chunks per tile

// Number of z-chunks per column tile of the two-step kernel, per N, timed on first use
// (psi -> scratch; the scratch field is overwritten by the real pass afterwards) among
// chunks of about 64, 32 and 16 planes and the counts that make the grid about 1-4 full
// waves of two resident blocks per SM.  Must not run during a capture.
static int tuned_tb_zchunk(qf_lattice* lat) {
  const int n = lat->d.n;
  const long long key = n;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& kv : g_tuned_tb)
      if (kv.first == key) return kv.second;
  }
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = ((n + TB_X - 1) / TB_X) * ((n + TB_Y - 1) / TB_Y);
  std::vector<int> cand = {(n + 63) / 64, (n + 31) / 32, (n + 15) / 16};
  for (int w = 1; w <= 4; ++w) {
    cand.push_back(w * 2 * sms / tiles);
    cand.push_back((w * 2 * sms + tiles - 1) / tiles);
  }
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  int best = (n + 31) / 32;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return best;
  for (int nzb : cand) {
    if (nzb < 1 || nzb > n) continue;
    StencilTbArgs g;
    tb_args(lat, &lat->sc()->scale[0], nzb, g);
    float ms = 0, tot = 0;
    bool ok = launch_stencil_tb(g, lat->st) == cudaSuccess;  // warm-up
    for (int rep = 0; rep < 3 && ok; ++rep) {
      ok = cudaEventRecord(e0, lat->st) == cudaSuccess && launch_stencil_tb(g, lat->st) == cudaSuccess &&
           cudaEventRecord(e1, lat->st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      tot += ms;
    }
    lat->launches += 4;
    if (ok && tot < best_ms) {
      best_ms = tot;
      best = nzb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned_tb.push_back({key, best});
  return best;
}

// Whether steps t and t+1 may run as one two-step pass: complex FP32 FDTD with blocking
// on and a clean live field, no check at t or t+1 and no snapshot after step t.
static bool fuse_pair(const qf_lattice* lat, int64_t t, int check_every, int snap_every) {
  if (lat->kinetic != QF_KIN_FDTD || !lat->c64() || lat->tblock < 2 || !lat->clean || !lat->tbmap_ok) return false;
  if (lat->kcur != 0) return false;  // the second step of a pair applies no scale
  if (check_every > 0 && (t % check_every == 0 || (t + 1) % check_every == 0)) return false;
  if (snap_every > 0 && (t + 1) % snap_every == 0) return false;
  return true;
}

// psi_{t+2} into the scratch field; `scale` renormalises the first of the two steps.
static cudaError_t fdtd_pair(qf_lattice* lat, const double* scale, int nzb) {
  StencilTbArgs g;
  tb_args(lat, scale, nzb, g);
  return launch(lat, K_STENCIL_2STEP, [&] { return launch_stencil_tb(g, lat->st); });
}

// One kinetic application on `in` (psi' written to `out` when write), with FP64 sums
// when reduce; returns the number of partial rows written through nblocks.
static cudaError_t kinetic_pass(qf_lattice* lat, void* in, void* out, bool write, bool reduce, const double* scale,
                                int* nblocks) {
  const int n = lat->d.n;
  if (lat->kinetic == QF_KIN_FDTD) {
    const int zc = lat->c64() ? tuned_zchunk<float>(lat) : tuned_zchunk<double>(lat);
    if (nblocks) *nblocks = stencil_blocks<float>(n, zc);
    if (lat->c64()) {
      StencilTmaGroup<float> g;
      if (!stencil_group_member(lat, in, out, write, reduce, scale, g, true, zc)) return cudaErrorInvalidValue;
      return launch(lat, write ? K_STENCIL : K_STENCIL_SUMS, [&] { return launch_stencil_tma<float>(g, lat->st); });
    }
    StencilTmaGroup<double> g;
    if (!stencil_group_member(lat, in, out, write, reduce, scale, g, true, zc)) return cudaErrorInvalidValue;
    return launch(lat, write ? K_STENCIL : K_STENCIL_SUMS, [&] { return launch_stencil_tma<double>(g, lat->st); });
  }
  // FFT terms: in place on `in` (out must equal in when writing); the scratch field is tmp.
  // A step on the live psi emits the next step's first pass and may skip its own.
  tune_fft_tiles(lat);  // first four-pass step of this size in the process (overwrites tmp)
  const bool live = write && in == lat->psi();
  const int first = (live && lat->xfwd_valid) ? 1 : 0;
  lat->xfwd_valid = false;
  if (uses_fft2(lat) && !write) {
    // energy of a field that is not stepped: <v|v> and <v|V v> in pass A, <v|H_K v> in
    // k-space (Parseval) in the forward half of pass B; no inverse transforms
    FftGroup<float> g;
    g.count = 1;
    g.a[0] = fft_args<float>(lat, in, false, true, scale);
    g.a[0].src = reinterpret_cast<const cpx<float>*>(in);
    if (nblocks) *nblocks = fft2_measure_blocks(n);
    cudaError_t e = launch(lat, K_FFT2_XY_FWD_SUMS, [&] { return launch_fft2_group_pass(n, 3, g, lat->st); });
    if (e != cudaSuccess) return e;
    g.a[0].src = nullptr;
    return launch(lat, K_FFT2_YZ_SUMS, [&] { return launch_fft2_group_pass(n, 4, g, lat->st); });
  }
  if (uses_fft2(lat)) {
    // two-pass step: A (natural -> scratch; skipped when the previous step emitted it),
    // B, C; every launch a group of one
    FftGroup<float> g;
    g.count = 1;
    g.a[0] = fft_args<float>(lat, in, write, reduce, scale);
    g.a[0].emit_next = live ? 1 : 0;
    if (nblocks) *nblocks = fft2_final_blocks(n);
    for (int ps = first; ps < 3; ++ps) {
      g.a[0].src = ps == 0 ? reinterpret_cast<const cpx<float>*>(in) : nullptr;
      const int kind = ps == 0 ? K_FFT2_XY_FWD : ps == 1 ? K_FFT2_YZ_MID : write ? K_FFT2_XY_INV_UPDATE
                                                                                  : K_FFT2_XY_INV_SUMS;
      cudaError_t e = launch(lat, kind, [&] { return launch_fft2_group_pass(n, ps, g, lat->st); });
      if (e != cudaSuccess) return e;
    }
    lat->xfwd_valid = live;
    return cudaSuccess;
  }
  if (lat->c64()) {
    FftPassArgs<float> p = fft_args<float>(lat, in, write, reduce, scale);
    p.emit_next = live ? 1 : 0;
    cpx<float>* tmp = p.data;
    for (int ps = first; ps < kFftPasses; ++ps) {
      const int kind = (ps == kFftPasses - 1 && !write) ? K_FFT_X_INV_SUMS : K_FFT_X_FWD + ps;
      cudaError_t e = launch(lat, kind, [&] { return launch_fft_pass<float>(n, ps, p, tmp, lat->st, nblocks); });
      if (e != cudaSuccess) return e;
    }
    lat->xfwd_valid = live;
    return cudaSuccess;
  }
  FftPassArgs<double> p = fft_args<double>(lat, in, write, reduce, scale);
  p.emit_next = live ? 1 : 0;
  cpx<double>* tmp = p.data;
  for (int ps = first; ps < kFftPasses; ++ps) {
    const int kind = (ps == kFftPasses - 1 && !write) ? K_FFT_X_INV_SUMS : K_FFT_X_FWD + ps;
    cudaError_t e = launch(lat, kind, [&] { return launch_fft_pass<double>(n, ps, p, tmp, lat->st, nblocks); });
    if (e != cudaSuccess) return e;
  }
  lat->xfwd_valid = live;
  return cudaSuccess;
}

// Copies the live field into the next ring slot when the step count is a multiple of
// snap_every.
static cudaError_t take_snapshot(qf_lattice* lat, int snap_every, cudaStream_t st) {
  if (snap_every > 0 && lat->step % snap_every == 0) {
    lat->snap_head = (lat->snap_head + 1) % lat->d.n_snap;
    lat->snapK[lat->snap_head] = lat->K;
    cudaError_t e = cudaMemcpyAsync(lat->snap(lat->snap_head), lat->psi(), (size_t)lat->sites * (lat->c64() ? 8 : 16),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    if (lat->snap_count < lat->d.n_snap) lat->snap_count++;
  }
  return cudaSuccess;
}

// Bookkeeping after the kinetic pass of step t has been issued on `st` (shared by
// qf_step_n and qf_batch_step so both advance a lattice identically): finishing sums and
// the pending renormalisation on a check step, buffer swap (FDTD), counters, snapshot.
static cudaError_t after_step(qf_lattice* lat, bool check, int nb, int snap_every, cudaStream_t st) {
  const long long k_in = lat->K;  // exponent of the step's input (the field a check measures)
  if (lat->pending_scale) {
    // this step's output was renormalised by 2^(k+j) / sqrt(norm at K_check)
    lat->K += lat->kcur + lat->jcur - lat->K_check;
    lat->renorm_step = lat->step;
  } else {
    lat->K += lat->kcur;
  }
  lat->pending_scale = false;
  if (check) {
    const int interval = lat->renorm_step >= 0 ? (int)std::min<int64_t>(lat->step - lat->renorm_step, 1 << 30) : 0;
    cudaError_t e =
        launch(lat, K_FINISH, [&] { return launch_finish(lat->partials(), nb, lat->sc(), 1, st, interval, lat->dtau); });
    if (e != cudaSuccess) return e;
    lat->pending_scale = true;
    lat->K_check = k_in;
  }
  if (lat->kinetic == QF_KIN_FDTD) {
    lat->live = 1 - lat->live;
    lat->clean = true;
  }
  lat->step += 1;
  lat->tau += lat->dtau;
  return take_snapshot(lat, snap_every, st);
}

// Bookkeeping after a two-step pass (steps t and t+1): one buffer swap, two steps.
static cudaError_t after_pair(qf_lattice* lat, int snap_every, cudaStream_t st) {
  if (lat->pending_scale) {
    lat->K += lat->jcur - lat->K_check;  // (kcur is 0 whenever steps are paired)
    lat->renorm_step = lat->step;
  }
  lat->pending_scale = false;
  lat->live = 1 - lat->live;
  lat->clean = true;
  for (int i = 0; i < 2; ++i) {
    lat->step += 1;
    lat->tau += lat->dtau;
  }
  return take_snapshot(lat, snap_every, st);
}

// Whether a check with energy difference d = |E_t - E_prev| (previous check's d_prev)
// meets tol under the rule: QF_STOP_DIFFERENCE: d < tol.  QF_STOP_EXTRAPOLATED: the check
// energies approach their limit geometrically, so while d shrinks (rho = d/d_prev < 1)
// the distance left is about d rho/(1 - rho); converged when max(d, d rho/(1 - rho)) < tol,
// never while d >= d_prev (an exact repeat, d = 0, counts as converged).
static bool check_converged(int rule, double d, double d_prev, double tol) {
  if (!(d < INFINITY)) return false;
  if (rule != QF_STOP_EXTRAPOLATED) return d < tol;
  if (d == 0.0) return true;
  if (!(d_prev < INFINITY) || !(d < d_prev)) return false;
  const double rho = d / d_prev;
  return std::max(d, d * rho / (1.0 - rho)) < tol;
}

// Records the energy of the check at step t; returns whether it converged under `rule`
// with tol = tol_abs + tol_rel |E_t|.
static bool record_check(qf_lattice* lat, const double* e3, int64_t t, double tau_t, double tol_abs,
                         double tol_rel, int rule = QF_STOP_DIFFERENCE) {
  qf_energy r{};
  r.e_re = e3[0];
  r.e_im = e3[1];
  r.norm = ldexp(e3[2], (int)(-2 * lat->K_check));  // the measured field held 2^K_check psi
  lat->kcur = (int)e3[3];
  lat->jcur = (int)e3[4];
  r.de = lat->have_prev ? hypot(e3[0] - lat->prev_re, e3[1] - lat->prev_im) : INFINITY;
  r.step = t;
  r.tau = tau_t;
  lat->last = r;
  lat->have_last = true;
  const bool conv = check_converged(rule, r.de, lat->prev_de, tol_abs + tol_rel * hypot(e3[0], e3[1]));
  lat->have_prev = true;
  lat->prev_re = e3[0];
  lat->prev_im = e3[1];
  lat->prev_de = r.de;
  return conv;
}

static qf_status read_energy(qf_lattice* lat, double* e3) {
  QF_CUDA(lat, cudaMemcpyAsync(e3, lat->sc()->energy, 5 * sizeof(double), cudaMemcpyDeviceToHost, lat->st));
  QF_CUDA(lat, cudaStreamSynchronize(lat->st));
  if (lat->prof) prof_harvest(lat);
  return QF_OK;
}

// The check_every - 1 steps after a check step issue the same launches every time (same
// buffers; the first uses the pending renormalisation; FFT steps start at their second
// pass; FDTD steps pair up as in the uncaptured loop), so they are captured once into a
// CUDA graph per (check_every, FDTD buffer parity, blocking) and replayed.  Snapshot
// copies and host bookkeeping stay outside the graph.  *flips receives the number of
// FDTD buffer swaps the replay did.
static cudaError_t run_chunk_graph(qf_lattice* lat, int check_every, int* flips) {
  const int k = check_every - 1;
  const qf_lattice::Graph* hit = nullptr;
  for (auto& g : lat->graphs)
    if (g.check_every == check_every && g.live == lat->live && g.tblock == lat->tblock &&
        g.kzero == (lat->kcur == 0))
      hit = &g;
  if (!hit) {
    // capture the k steps without touching the handle's state
    const int live0 = lat->live;
    const bool xv0 = lat->xfwd_valid, ps0 = lat->pending_scale, clean0 = lat->clean;
    const int64_t launches0 = lat->launches;
    const bool pairs = lat->kinetic == QF_KIN_FDTD && lat->c64() && lat->tblock >= 2 && lat->tbmap_ok;
    const int tzc = pairs ? tuned_tb_zchunk(lat) : 0;  // timed outside the capture
    tune_fft_tiles(lat);
    if (lat->kinetic == QF_KIN_FDTD) {
      if (lat->c64()) tuned_zchunk<float>(lat);
      else tuned_zchunk<double>(lat);
    }
    int nflip = 0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(lat->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    int64_t t = lat->step;
    for (int s = 0; s < k && e == cudaSuccess;) {
      const double* scale = lat->pending_scale ? &lat->sc()->scale[1] : &lat->sc()->scale[2];
      if (pairs && s + 2 <= k && fuse_pair(lat, t, check_every, check_every)) {
        e = fdtd_pair(lat, scale, tzc);
        s += 2;
        t += 2;
      } else {
        void* in = lat->psi();
        void* out = lat->kinetic == QF_KIN_FDTD ? lat->tmp() : in;
        e = kinetic_pass(lat, in, out, true, false, scale, nullptr);
        s += 1;
        t += 1;
      }
      lat->pending_scale = false;
      if (lat->kinetic == QF_KIN_FDTD) {
        lat->live = 1 - lat->live;
        lat->clean = true;
        ++nflip;
      }
    }
    cudaError_t e2 = cudaStreamEndCapture(lat->st, &graph);
    if (e2 != cudaSuccess && graph) {
      cudaGraphDestroy(graph);
      graph = nullptr;
    }
    const int64_t nlaunch = lat->launches - launches0;
    lat->live = live0;
    lat->xfwd_valid = xv0;
    lat->pending_scale = ps0;
    lat->clean = clean0;
    lat->launches = launches0;
    if (e == cudaSuccess) e = e2;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    lat->graphs.push_back({check_every, live0, lat->tblock, lat->kcur == 0 ? 1 : 0, exec, nflip, nlaunch});
    hit = &lat->graphs.back();
  }
  cudaError_t e = cudaGraphLaunch(hit->exec, lat->st);
  if (e != cudaSuccess) return e;
  lat->launches += hit->launches;
  *flips = hit->flips;
  return cudaSuccess;
}

extern "C" qf_status qf_step_n(qf_lattice* lat, int64_t max_steps, double tol_abs, int check_every, int snap_every,
                               int64_t* steps_done) {
  if (steps_done) *steps_done = 0;
  if (!lat) return QF_EINVAL;
  if (max_steps < 0 || check_every < 0 || snap_every < 0 || !(tol_abs >= 0))
    return fail(lat, QF_EINVAL, "negative step counts or tolerance");
  if (!lat->have_v || lat->kinetic < 0 || !lat->have_psi)
    return fail(lat, QF_ESTATE, "set the potential, kinetic term and wavefunction first");
  const bool fdtd = lat->kinetic == QF_KIN_FDTD;
  int64_t done = 0;
  qf_status status = QF_ENOTCONV;
  while (done < max_steps) {
    const int64_t t = lat->step;
    const double tau_t = lat->tau;
    const bool check = check_every > 0 && t % check_every == 0;
    const double* scale = lat->pending_scale ? &lat->sc()->scale[1] : &lat->sc()->scale[2];
    if (done + 2 <= max_steps && fuse_pair(lat, t, check_every, snap_every)) {
      const int tzc = tuned_tb_zchunk(lat);
      QF_CUDA(lat, fdtd_pair(lat, scale, tzc));
      QF_CUDA(lat, after_pair(lat, snap_every, lat->st));
      done += 2;
      continue;
    }
    int nb = 0;
    void* in = lat->psi();
    void* out = fdtd ? lat->tmp() : in;
    QF_CUDA(lat, kinetic_pass(lat, in, out, true, check, scale, &nb));
    QF_CUDA(lat, after_step(lat, check, nb, snap_every, lat->st));
    ++done;
    if (check) {
      double e3[5];
      qf_status s = read_energy(lat, e3);
      if (s != QF_OK) return s;
      if (record_check(lat, e3, t, tau_t, tol_abs, 0.0)) {
        status = QF_OK;
        break;
      }
      // the rest of the check interval as one graph replay when it fits entirely
      const int k = check_every - 1;
      const bool snaps_at_end = snap_every == 0 || snap_every == check_every;
      const bool fft_ready = fdtd || lat->xfwd_valid;
      // (the legacy default stream cannot be captured; a failed capture falls back to
      // ordinary launches for the rest of the handle's life)
      const bool capturable = lat->st != nullptr && lat->st != cudaStreamLegacy && lat->st != cudaStreamPerThread;
      if (lat->use_graphs && capturable && !lat->prof && k >= 2 && done + k <= max_steps && snaps_at_end &&
          fft_ready && lat->pending_scale) {
        int flips = 0;
        if (run_chunk_graph(lat, check_every, &flips) != cudaSuccess) {
          cudaGetLastError();
          lat->use_graphs = false;
          drop_graphs(lat);
          continue;
        }
        for (int s = 0; s < k; ++s) lat->tau += lat->dtau;
        // the first replayed step renormalises (2^(kcur+jcur) / sqrt(norm at K_check)),
        // the others scale by 2^kcur
        lat->K += (long long)k * lat->kcur + lat->jcur - lat->K_check;
        lat->renorm_step = lat->step;
        if (fdtd) {
          lat->live ^= flips & 1;
          lat->clean = true;
        }
        lat->step += k;
        lat->pending_scale = false;
        done += k;
        QF_CUDA(lat, take_snapshot(lat, snap_every, lat->st));
      }
    }
  }
  if (steps_done) *steps_done = done;
  // surface asynchronous launch failures and bounded-wait timeouts before reporting
  QF_CUDA(lat, cudaStreamSynchronize(lat->st));
  if (lat->kinetic == QF_KIN_FDTD) {
    qf_status s = check_device_error(lat);
    if (s != QF_OK) return s;
  }
  return status;
}

extern "C" qf_status qf_energies(qf_lattice* lat, qf_energy* out) {
  if (!lat || !out) return QF_EINVAL;
  if (!lat->have_last) return fail(lat, QF_ESTATE, "no check has run yet");
  *out = lat->last;
  return QF_OK;
}

// <v|H|v>/<v|v> of a field into out (FP64 sums; the field is not modified).
static qf_status measure(qf_lattice* lat, void* f, qf_energy* out) {
  int nb = 0;
  if (lat->kinetic == QF_KIN_FDTD && f != lat->field(0) && f != lat->field(1) && !lat->fmap_ok)
    return fail(lat, QF_ECUDA, "tensor map encoding unavailable");
  // FFT terms transform through tmp and read f; FDTD reads f only
  QF_CUDA(lat, kinetic_pass(lat, f, f, false, true, &lat->sc()->scale[0], &nb));
  QF_CUDA(lat, launch(lat, K_FINISH, [&] { return launch_finish(lat->partials(), nb, lat->sc(), 0, lat->st); }));
  double e3[5];
  qf_status s = read_energy(lat, e3);
  if (s != QF_OK) return s;
  out->e_re = e3[0];
  out->e_im = e3[1];
  out->norm = e3[2];
  out->de = 0;
  out->step = lat->step;
  out->tau = lat->tau;
  return QF_OK;
}

template <typename R>
static qf_status gram_schmidt(qf_lattice* lat, int n_states) {
  double* coef = lat->sc()->gs_coef;  // [Re c0, Im c0, Re c1, Im c1, |w|^2, 1/|w|]
  double* part = lat->partials();
  const int nblk = field_blocks();
  const long long ns = lat->sites;
  for (int i = 0; i < n_states; ++i) {
    const int idx = ((lat->snap_head - i) % lat->d.n_snap + lat->d.n_snap) % lat->d.n_snap;
    const cpx<R>* src = reinterpret_cast<const cpx<R>*>(lat->snap(idx));  // i-th latest snapshot
    cpx<R>* w = reinterpret_cast<cpx<R>*>(lat->state(i));
    const cpx<R>* basis[2] = {reinterpret_cast<const cpx<R>*>(lat->state(0)),
                              reinterpret_cast<const cpx<R>*>(lat->state(1))};
    const int nb = i;
    // coefficients <v_j|S_i> (classical Gram-Schmidt: all from the same vector)
    QF_CUDA(lat, launch(lat, K_GS_DOTS, [&] { return launch_dots<R>(basis, nb, src, ns, part, nblk, lat->st); }));
    QF_CUDA(lat, launch(lat, K_FINISH, [&] { return launch_finish_dots(part, nblk, nb, coef, lat->st); }));
    if (nb > 0) {
      // w = S_i - sum c_j v_j, with <v_j|w> of the result: the re-orthogonalisation pass
      QF_CUDA(lat, launch(lat, K_GS_AXPY,
                          [&] { return launch_axpy_dots<R>(w, src, basis, nb, coef, ns, part, nblk, lat->st); }));
      QF_CUDA(lat, launch(lat, K_FINISH, [&] { return launch_finish_dots(part, nblk, nb, coef, lat->st); }));
      QF_CUDA(lat, launch(lat, K_GS_AXPY,
                          [&] { return launch_axpy_dots<R>(w, w, basis, nb, coef, ns, part, nblk, lat->st); }));
      QF_CUDA(lat, launch(lat, K_FINISH, [&] { return launch_finish_dots(part, nblk, nb, coef, lat->st); }));
      src = w;
    }
    // v_i = w / ||w||  (coef[5] = 1/||w|| of the last pass)
    QF_CUDA(lat, launch(lat, K_SCALE_COPY, [&] { return launch_scale_copy<R>(w, src, coef + 5, ns, lat->st); }));
    lat->have_states[i] = true;
  }
  return QF_OK;
}

extern "C" qf_status qf_project_excited(qf_lattice* lat, int n_states, qf_energy* out) {
  if (!lat || !out) return QF_EINVAL;
  if (n_states < 1 || n_states > 3 || n_states > lat->d.n_snap) return fail(lat, QF_EINVAL, "n_states out of range");
  if (lat->snap_count < n_states) return fail(lat, QF_ESTATE, "not enough snapshots");
  if (!lat->have_v || lat->kinetic < 0) return fail(lat, QF_ESTATE, "set the potential and kinetic term first");
  qf_status s = lat->c64() ? gram_schmidt<float>(lat, n_states) : gram_schmidt<double>(lat, n_states);
  if (s != QF_OK) return s;
  for (int i = 0; i < n_states; ++i) {
    s = measure(lat, lat->state(i), &out[i]);
    if (s != QF_OK) return s;
  }
  return QF_OK;
}

extern "C" qf_status qf_track_excited(qf_lattice* lat, int n_states, qf_energy* out) {
  if (!lat || !out) return QF_EINVAL;
  if (lat->exc_records > 0 && n_states != lat->exc_n)
    return fail(lat, QF_EINVAL, "n_states differs from the one of this history");
  qf_status s = qf_project_excited(lat, n_states, out);
  if (s != QF_OK) return s;
  const int j = lat->exc_records;
  if (j >= 1) {
    for (int i = 0; i < n_states; ++i) {
      const double d = hypot(out[i].e_re - lat->exc_prev[i].e_re, out[i].e_im - lat->exc_prev[i].e_im);
      if (lat->plat_have[i] && !(d < lat->plat[i].de)) continue;
      lat->plat_have[i] = true;
      lat->plat[i] = out[i];
      lat->plat[i].de = d;
      lat->plat_rec[i] = j;
      if (i < lat->d.plateau_slots) {
        QF_CUDA(lat, cudaMemcpyAsync(lat->plateau_state(i), lat->state(i), (size_t)lat->sites * (lat->c64() ? 8 : 16),
                                     cudaMemcpyDeviceToDevice, lat->st));
        lat->have_plateau_state[i] = true;
      }
    }
  }
  for (int i = 0; i < n_states; ++i) lat->exc_prev[i] = out[i];
  lat->exc_n = n_states;
  lat->exc_records = j + 1;
  QF_CUDA(lat, cudaStreamSynchronize(lat->st));
  return QF_OK;
}

extern "C" qf_status qf_excited_plateau(qf_lattice* lat, int n_states, qf_energy* out, int* record) {
  if (!lat || !out) return QF_EINVAL;
  if (lat->exc_records < 2) return fail(lat, QF_ESTATE, "fewer than two records of E_i(tau)");
  if (n_states < 1 || n_states > lat->exc_n) return fail(lat, QF_EINVAL, "n_states exceeds the history's");
  for (int i = 0; i < n_states; ++i) {
    out[i] = lat->plat[i];
    if (record) record[i] = lat->plat_rec[i];
  }
  return QF_OK;
}

template <typename R>
static qf_status parity_t(qf_lattice* lat, int which, int axis, void* target) {
  const int nblk = field_blocks();
  lat->xfwd_valid = false;  // the scratch field is overwritten
  cpx<R>* tmp = reinterpret_cast<cpx<R>*>(lat->tmp());
  QF_CUDA(lat, launch(lat, K_PARITY, [&] { return launch_parity<R>(tmp, reinterpret_cast<const cpx<R>*>(target), lat->d.n, which, axis, lat->partials(),
                                nblk, lat->st); }));
  double* coef = lat->sc()->gs_coef;
  QF_CUDA(lat, launch(lat, K_FINISH, [&] { return launch_finish_dots(lat->partials(), nblk, 0, coef, lat->st); }));
  QF_CUDA(lat, launch(lat, K_SCALE_COPY, [&] { return launch_scale_copy<R>(reinterpret_cast<cpx<R>*>(target), tmp, coef + 5, lat->sites, lat->st); }));
  QF_CUDA(lat, cudaStreamSynchronize(lat->st));
  return QF_OK;
}

extern "C" qf_status qf_parity_project(qf_lattice* lat, int which, int axis, int target) {
  if (!lat) return QF_EINVAL;
  if (which < QF_P_PLUS || which > QF_P_D2_K) return fail(lat, QF_EINVAL, "unknown projector");
  if (which >= QF_P_MINUS_PK && (axis < 1 || axis > 3)) return fail(lat, QF_EINVAL, "axis must be 1..3");
  if (!(target >= -1 && target <= 2) && !(target >= 200 && target < 200 + lat->d.plateau_slots))
    return fail(lat, QF_EINVAL, "target must be -1..2 or a plateau slot 200 + i");
  void* f = slot_ptr(lat, target);
  if (!f || (target == -1 && !lat->have_psi)) return fail(lat, QF_ESTATE, "target holds no field");
  qf_status s = lat->c64() ? parity_t<float>(lat, which, axis, f) : parity_t<double>(lat, which, axis, f);
  if (s != QF_OK) return s;
  if (target == -1) {
    lat->pending_scale = false;
    lat->K = 0;  // renormalised to unit norm
    lat->renorm_step = lat->step;
  }
  return QF_OK;
}

// Radial momentum distribution of a field (no workspace beyond the scratch field and
// the staging area): norm, plain forward 3D transform into the scratch field, integer
// shell histogram.
template <typename R>
static qf_status momentum_t(qf_lattice* lat, void* field, int nb, double* prob_host) {
  const int n = lat->d.n;
  const long long ns = lat->sites;
  double* coef = lat->sc()->gs_coef;
  const int nblk = field_blocks();
  const cpx<R>* f = reinterpret_cast<const cpx<R>*>(field);
  QF_CUDA(lat, launch(lat, K_GS_DOTS, [&] { return launch_dots<R>(nullptr, 0, f, ns, lat->partials(), nblk, lat->st); }));
  QF_CUDA(lat, launch(lat, K_FINISH, [&] { return launch_finish_dots(lat->partials(), nblk, 0, coef, lat->st); }));
  FftPassArgs<R> p = fft_args<R>(lat, field, false, false, &lat->sc()->scale[0]);
  cpx<R>* tmp = p.data;
  lat->xfwd_valid = false;
  for (int ps : {0, 1, kFftPassZForward})
    QF_CUDA(lat, launch(lat, K_FFT_X_FWD + (ps == kFftPassZForward ? 2 : ps),
                        [&] { return launch_fft_pass<R>(n, ps, p, tmp, lat->st, nullptr); }));
  const long long want = (ns + 255) / 256;
  const int blocks = (int)(want < nblk ? want : nblk);
  unsigned long long* part = reinterpret_cast<unsigned long long*>(lat->stage());
  double* prob = reinterpret_cast<double*>(part + (size_t)blocks * nb);
  if ((size_t)blocks * nb * 8 + (size_t)nb * 8 > lat->L.stage_bytes) return fail(lat, QF_ENOMEM, "staging area too small");
  QF_CUDA(lat, launch(lat, K_CONVERT, [&] { return launch_momentum_hist<R>(tmp, n, nb, coef + 4, part, blocks, lat->st); }));
  QF_CUDA(lat, launch(lat, K_FINISH, [&] { return launch_momentum_finish(part, blocks, nb, prob, lat->st); }));
  QF_CUDA(lat, cudaMemcpyAsync(prob_host, prob, nb * sizeof(double), cudaMemcpyDeviceToHost, lat->st));
  QF_CUDA(lat, cudaStreamSynchronize(lat->st));
  return QF_OK;
}

extern "C" qf_status qf_momentum_distribution(qf_lattice* lat, int slot, double* p, double* prob, double* y,
                                              int max_bins, int* nbins) {
  if (!lat || !nbins) return QF_EINVAL;
  const int n = lat->d.n;
  const int half = n / 2;
  const int nb = (int)std::floor(std::sqrt(3.0 * half * half) + 0.5) + 1;
  *nbins = nb;
  if (!fft_supported(n)) return fail(lat, QF_EINVAL, "no FFT plan for this N");
  if (max_bins < nb || !prob) return fail(lat, QF_EINVAL, "output arrays need *nbins entries");
  void* f = slot_ptr(lat, slot);
  if (!f || (slot == -1 && !lat->have_psi)) return fail(lat, QF_ESTATE, "slot holds no field");
  qf_status s = lat->c64() ? momentum_t<float>(lat, f, nb, prob) : momentum_t<double>(lat, f, nb, prob);
  if (s != QF_OK) return s;
  const double dp = 2.0 * M_PI / (n * lat->d.a);
  for (int b = 0; b < nb; ++b) {
    if (p) p[b] = b * dp;
    if (y) y[b] = std::sqrt(prob[b] / dp);
  }
  return QF_OK;
}

// Warm start: spectral prolongation of a coarse field onto a lattice of twice the size.
template <typename R>
static qf_status prolong_t(qf_lattice* c, void* cfield, qf_lattice* f) {
  const int nc = c->d.n, nf = f->d.n;
  FftPassArgs<R> pc = fft_args<R>(c, cfield, false, false, &c->sc()->scale[0]);
  c->xfwd_valid = false;
  for (int ps : {0, 1, kFftPassZForward})
    QF_CUDA(c, launch(c, K_FFT_X_FWD, [&] { return launch_fft_pass<R>(nc, ps, pc, pc.data, c->st, nullptr); }));
  QF_CUDA(c, cudaStreamSynchronize(c->st));
  FftPassArgs<R> pf = fft_args<R>(f, f->psi(), false, false, &f->sc()->scale[0]);
  const double scale = 1.0 / ((double)nc * nc * nc);
  QF_CUDA(f, launch(f, K_CONVERT, [&] { return launch_pad_spectrum<R>(pc.data, nc, pf.data, scale, f->st); }));
  f->xfwd_valid = false;
  f->clean = false;
  for (int ps : {kFftPassZInverse, 3, kFftPassXInverse})
    QF_CUDA(f, launch(f, K_FFT_Y_INV, [&] { return launch_fft_pass<R>(nf, ps, pf, pf.data, f->st, nullptr); }));
  QF_CUDA(f, cudaMemcpyAsync(f->psi(), pf.data, (size_t)f->sites * sizeof(cpx<R>), cudaMemcpyDeviceToDevice, f->st));
  QF_CUDA(f, cudaStreamSynchronize(f->st));
  return QF_OK;
}

extern "C" qf_status qf_prolong(qf_lattice* coarse, int coarse_slot, qf_lattice* fine) {
  if (!coarse || !fine) return QF_EINVAL;
  if (fine->d.n != 2 * coarse->d.n || fine->d.prec != coarse->d.prec ||
      std::fabs(fine->d.a * 2.0 - coarse->d.a) > 1e-12 * coarse->d.a)
    return fail(fine, QF_EINVAL, "fine lattice must have 2N sites, spacing a/2 and the same precision");
  if (!fft_supported(coarse->d.n) || !fft_supported(fine->d.n))
    return fail(fine, QF_EINVAL, "both sizes need FFT plans");
  void* cf = slot_ptr(coarse, coarse_slot);
  if (!cf || (coarse_slot == -1 && !coarse->have_psi)) return fail(fine, QF_ESTATE, "coarse slot holds no field");
  qf_status s = coarse->c64() ? prolong_t<float>(coarse, cf, fine) : prolong_t<double>(coarse, cf, fine);
  if (s != QF_OK) return s;
  fine->have_psi = true;
  fine->pending_scale = false;
  fine->K = slot_exp2(coarse, coarse_slot);  // the interpolant of the stored coarse field
  fine->renorm_step = -1;
  return QF_OK;
}

extern "C" qf_status qf_get_info(qf_lattice* lat, qf_info* out) {
  if (!lat || !out) return QF_EINVAL;
  out->dtau = lat->dtau;
  out->step = lat->step;
  out->tau = lat->tau;
  out->kinetic = lat->kinetic;
  out->n_snapshots = lat->snap_count;
  out->workspace_bytes = lat->L.total;
  out->launches = lat->launches;
  out->temporal_block = lat->tblock;
  out->fft_passes = lat->kinetic == QF_KIN_FDTD ? 0 : uses_fft2(lat) ? 2 : 4;
  out->field_exp2 = lat->K;
  return QF_OK;
}

extern "C" qf_status qf_profile(qf_lattice* lat, int enable) {
  if (!lat) return QF_EINVAL;
  if (enable && lat->ev_free.empty() && lat->pend.empty()) {
    for (int i = 0; i < kEventPool; ++i) {
      cudaEvent_t e;
      QF_CUDA(lat, cudaEventCreate(&e));
      lat->ev_free.push_back(e);
    }
  }
  if (!enable) {
    QF_CUDA(lat, cudaStreamSynchronize(lat->st));
    prof_harvest(lat);
  }
  lat->prof = enable != 0;
  return QF_OK;
}

extern "C" qf_status qf_profile_read(qf_lattice* lat, qf_kernel_stat* out, int max, int* count, int reset) {
  if (!lat || (max > 0 && !out)) return QF_EINVAL;
  QF_CUDA(lat, cudaStreamSynchronize(lat->st));
  prof_harvest(lat);
  int c = 0;
  for (int k = 0; k < K_NUM_KINDS; ++k) {
    if (lat->prof_count[k] == 0) continue;
    if (c < max) {
      memset(out[c].name, 0, sizeof(out[c].name));
      strncpy(out[c].name, kKindNames[k], sizeof(out[c].name) - 1);
      out[c].launches = lat->prof_count[k];
      out[c].total_ms = lat->prof_ms[k];
    }
    ++c;
  }
  if (count) *count = c;
  if (reset)
    for (int k = 0; k < K_NUM_KINDS; ++k) {
      lat->prof_count[k] = 0;
      lat->prof_ms[k] = 0;
    }
  return QF_OK;
}

extern "C" const char* qf_last_error(const qf_lattice* lat) {
  if (!lat) return "null handle";
  return lat->err.c_str();
}

extern "C" const char* qf_version(void) { return kVersion; }

extern "C" qf_status qf_use_graphs(qf_lattice* lat, int enable) {
  if (!lat) return QF_EINVAL;
  lat->use_graphs = enable != 0;
  if (!lat->use_graphs) drop_graphs(lat);
  return QF_OK;
}

extern "C" qf_status qf_use_two_pass_fft(qf_lattice* lat, int enable) {
  if (!lat) return QF_EINVAL;
  if (lat->two_pass != (enable != 0)) {
    lat->two_pass = enable != 0;
    lat->xfwd_valid = false;  // the scratch layouts of the two step forms differ
    drop_graphs(lat);
  }
  return QF_OK;
}

extern "C" qf_status qf_set_fft_tiles(int n, int variant) {
  if (!fft_supported(n) || variant < -1 || variant > 3) return QF_EINVAL;
  return set_fft_tile_choice(n, variant) ? QF_OK : QF_EINVAL;
}

extern "C" qf_status qf_get_fft_tiles(int n, int* variant) {
  if (!fft_supported(n) || !variant) return QF_EINVAL;
  *variant = fft_tile_choice(n);
  return QF_OK;
}

extern "C" qf_status qf_set_temporal_blocking(qf_lattice* lat, int k) {
  if (!lat) return QF_EINVAL;
  if (k != 1 && k != 2) return fail(lat, QF_EINVAL, "temporal blocking factor must be 1 or 2");
  lat->tblock = k;
  return QF_OK;
}

extern "C" qf_status qf_selftest_bounded_wait(qf_lattice* lat) {
  if (!lat) return QF_EINVAL;
  int* flag = &lat->sc()->err[1];
  QF_CUDA(lat, cudaMemsetAsync(flag, 0, sizeof(int), lat->st));
  QF_CUDA(lat, launch_bounded_wait_probe(flag, lat->st));
  int err = 0;
  QF_CUDA(lat, cudaMemcpyAsync(&err, flag, sizeof(int), cudaMemcpyDeviceToHost, lat->st));
  QF_CUDA(lat, cudaStreamSynchronize(lat->st));
  return err ? QF_ETIMEOUT : QF_OK;
}

// ------------------------------------------------------------------------------------
// Batches: many resident lattices advanced together.  Each step, FP32 lattices with the
// same N (and, for FFT terms, the same real/complex V and check status) form groups, and
// each pass of a group is one launch over all its members; FP64 lattices run their own
// launches.  A member computes exactly what qf_step_n computes for it alone.
// ------------------------------------------------------------------------------------
struct qf_batch {
  struct Member {
    qf_lattice* lat;
    int64_t max_steps, steps_done;
    double tol_abs, tol_rel;
    int status;  // QF_BATCH_RUNNING, QF_OK (converged), QF_ENOTCONV (step cap reached)
    bool mid_pair;  // advanced two steps by the previous batch step's launch: sits this one out
  };
  cudaStream_t st = nullptr;
  std::vector<Member> m;
  std::string err;
  int64_t launches = 0;
  int rule = QF_STOP_DIFFERENCE;
  // CUDA graphs of check-free intervals (batch_chunk_graph), dropped when members change
  struct BGraph {
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec;
    int64_t launches;
  };
  std::vector<BGraph> graphs;
  bool use_graphs = true;
  int64_t graph_captures = 0, graph_replays = 0;
  void drop_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }
};

static qf_status bfail(qf_batch* b, qf_status s, const std::string& msg) {
  if (b) b->err = msg;
  return s;
}
#define QF_BCUDA(b, call)                                                                     \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return bfail(b, QF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" qf_status qf_batch_create(void* cuda_stream, qf_batch** out) {
  if (!out) return QF_EINVAL;
  qf_batch* b = new (std::nothrow) qf_batch();
  if (!b) return QF_ENOMEM;
  b->st = static_cast<cudaStream_t>(cuda_stream);
  *out = b;
  return QF_OK;
}

extern "C" qf_status qf_batch_destroy(qf_batch* b) {
  if (!b) return QF_OK;
  cudaStreamSynchronize(b->st);
  b->drop_graphs();
  delete b;
  return QF_OK;
}

extern "C" qf_status qf_batch_add(qf_batch* b, qf_lattice* lat, int64_t max_steps, double tol_abs, double tol_rel) {
  if (!b || !lat) return QF_EINVAL;
  if (max_steps < 0 || !(tol_abs >= 0) || !(tol_rel >= 0)) return bfail(b, QF_EINVAL, "bad step cap or tolerance");
  if (!lat->have_v || lat->kinetic < 0 || !lat->have_psi)
    return bfail(b, QF_ESTATE, "set the potential, kinetic term and wavefunction first");
  for (auto& x : b->m)
    if (x.lat == lat) return bfail(b, QF_EINVAL, "lattice already in the batch");
  // work of the lattice's own stream must be visible to the batch stream
  QF_BCUDA(b, cudaStreamSynchronize(lat->st));
  b->m.push_back({lat, max_steps, 0, tol_abs, tol_rel, QF_BATCH_RUNNING, false});
  b->drop_graphs();
  return QF_OK;
}

extern "C" qf_status qf_batch_remove(qf_batch* b, qf_lattice* lat) {
  if (!b || !lat) return QF_EINVAL;
  for (size_t i = 0; i < b->m.size(); ++i)
    if (b->m[i].lat == lat) {
      QF_BCUDA(b, cudaStreamSynchronize(b->st));
      b->m.erase(b->m.begin() + i);
      b->drop_graphs();
      return QF_OK;
    }
  return bfail(b, QF_EINVAL, "lattice not in the batch");
}

extern "C" qf_status qf_batch_members(qf_batch* b, int* count, int* status, int64_t* steps_done, int max) {
  if (!b) return QF_EINVAL;
  if (count) *count = (int)b->m.size();
  for (int i = 0; i < (int)b->m.size() && i < max; ++i) {
    if (status) status[i] = b->m[i].status;
    if (steps_done) steps_done[i] = b->m[i].steps_done;
  }
  return QF_OK;
}

// Whether a batch member's FDTD steps may run two per launch (the conditions of fuse_pair
// that do not depend on the step's place in the check and snapshot schedule).
static bool pairable(const qf_lattice* L) {
  return L->kinetic == QF_KIN_FDTD && L->c64() && L->tblock >= 2 && L->clean && L->tbmap_ok && L->kcur == 0;
}

// Issues the launches of one batch step for the running members `run` (check flags chk);
// nblk receives each member's partial rows.  pm (optional, per member of run) selects the
// FDTD members' form: 0 one step, 1 two steps in one pass (psi_{t+2} into the scratch
// field; the caller skips the member in the next batch step), 2 nothing (the second step
// of a pair issued in the previous batch step).  Host state is touched only where later
// launches depend on it (xfwd_valid of FFT members).
static qf_status batch_issue_step(qf_batch* b, const std::vector<int>& run, const std::vector<char>& chk,
                                  std::vector<int>& nblk, cudaStream_t st, const std::vector<char>* pm = nullptr) {
  const int R = (int)run.size();
  // group FP32 members by (N, kinetic family, real V, check); FP64 members run alone
  std::vector<char> done(R, 0);
  for (int k = 0; k < R; ++k) {
    if (done[k]) continue;
    qf_lattice* L = b->m[run[k]].lat;
    const double* sk = L->pending_scale ? &L->sc()->scale[1] : &L->sc()->scale[2];
    const bool fdtd = L->kinetic == QF_KIN_FDTD;
    if (!L->c64()) {
      void* in = L->psi();
      const int64_t l0 = L->launches;
      QF_BCUDA(b, kinetic_pass(L, in, fdtd ? L->tmp() : in, true, chk[k], sk, &nblk[k]));
      b->launches += L->launches - l0;
      done[k] = 1;
      continue;
    }
    std::vector<int> g;
    for (int q = k; q < R; ++q) {
      if (done[q]) continue;
      qf_lattice* M = b->m[run[q]].lat;
      // complex-FP32 FDTD members of any size share a launch (the stencil kernel takes
      // each member's N from its block table); FFT members need the same plan (N)
      if (!M->c64() || (M->kinetic == QF_KIN_FDTD) != fdtd || (!fdtd && M->d.n != L->d.n)) continue;
      if (!fdtd && (M->v_real != L->v_real || chk[q] != chk[k] || uses_fft2(M) != uses_fft2(L))) continue;
      g.push_back(q);
      done[q] = 1;
    }
    const int n = L->d.n;
    for (size_t off = 0; off < g.size(); off += kGroupMax) {
      const int cnt = (int)std::min<size_t>(kGroupMax, g.size() - off);
      if (fdtd) {
        // single steps in one launch, pairs in one launch per kind of potential
        StencilTmaGroup<float> sg;
        StencilTbGroup tg[2];
        sg.count = 0;
        tg[0].count = tg[1].count = 0;
        for (int j = 0; j < cnt; ++j) {
          const int q = g[off + j];
          qf_lattice* M = b->m[run[q]].lat;
          const int mode = pm ? (*pm)[q] : 0;
          const double* sq = M->pending_scale ? &M->sc()->scale[1] : &M->sc()->scale[2];
          if (mode == 2) continue;
          if (mode == 1) {
            StencilTbGroup& t = tg[M->v_real ? 1 : 0];
            tb_args(M, sq, tuned_tb_zchunk(M), t.m[t.count++]);
            continue;
          }
          const int zc = tuned_zchunk<float>(M);
          if (!stencil_group_member<float>(M, M->psi(), M->tmp(), true, chk[q], sq, sg, sg.count == 0, zc))
            return bfail(b, QF_ECUDA, "tensor map encoding failed");
          // one error flag per launch: the first member's
          nblk[q] = stencil_blocks<float>(M->d.n, zc);
        }
        if (sg.count > 0) {
          QF_BCUDA(b, launch_stencil_tma<float>(sg, st));
          b->launches += 1;
        }
        for (auto& t : tg)
          if (t.count > 0) {
            QF_BCUDA(b, launch_stencil_tb_group(t, st));
            b->launches += 1;
          }
      } else {
        const bool two = uses_fft2(L);
        tune_fft_tiles(L);  // (runs once per size; never inside a capture)
        FftGroup<float> fg, f0;
        fg.count = cnt;
        f0.count = 0;
        for (int j = 0; j < cnt; ++j) {
          const int q = g[off + j];
          qf_lattice* M = b->m[run[q]].lat;
          const double* sq = M->pending_scale ? &M->sc()->scale[1] : &M->sc()->scale[2];
          fg.a[j] = fft_args<float>(M, M->psi(), true, chk[q], sq);
          fg.a[j].emit_next = 1;
          nblk[q] = two ? fft2_final_blocks(n) : fft_final_blocks<float>(n);
          if (!M->xfwd_valid) {
            f0.a[f0.count] = fg.a[j];
            f0.a[f0.count].src = fg.a[j].psi;
            f0.count++;
          }
          M->xfwd_valid = true;
        }
        if (f0.count > 0) {
          QF_BCUDA(b, two ? launch_fft2_group_pass(n, 0, f0, st) : launch_fft_group_pass<float>(n, 0, f0, st));
          b->launches += 1;
        }
        for (int j = 0; j < cnt; ++j) fg.a[j].src = nullptr;
        for (int ps = 1; ps < (two ? 3 : kFftPasses); ++ps) {
          QF_BCUDA(b, two ? launch_fft2_group_pass(n, ps, fg, st) : launch_fft_group_pass<float>(n, ps, fg, st));
          b->launches += 1;
        }
      }
    }
  }
  return QF_OK;
}

// The check_every - 1 steps after a check that every running member took together
// issue the same launches each time the batch holds the same members in the same buffer
// state, so they are captured once into a CUDA graph (keyed by members, FDTD buffer
// parity, first-pass state and FDTD pairing) and replayed; the host bookkeeping of those
// steps follows the replay.  FDTD members that qualify (pairable) take the interval's
// steps two per launch from its first step on, the last one alone when the count is odd,
// as a lone lattice does.  Returns QF_OK with *used = false when the interval does not
// qualify.
static qf_status batch_chunk_graph(qf_batch* b, const std::vector<int>& run, int64_t steps_left, int check_every,
                                   int snap_every, cudaStream_t st, bool* used) {
  *used = false;
  const int k = check_every - 1;
  if (!b->use_graphs || k < 2 || steps_left < k) return QF_OK;
  if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) return QF_OK;
  if (!(snap_every == 0 || snap_every == check_every)) return QF_OK;
  std::vector<uintptr_t> key;
  key.push_back((uintptr_t)k);
  for (int i : run) {
    const auto& mb = b->m[i];
    qf_lattice* L = mb.lat;
    if (!L->pending_scale || L->prof || L->step % check_every != 1 || mb.steps_done + k > mb.max_steps)
      return QF_OK;
    key.push_back(reinterpret_cast<uintptr_t>(L));
    key.push_back((uintptr_t)((L->live & 1) | (L->xfwd_valid ? 2 : 0) | (uses_fft2(L) ? 4 : 0) |
                              (pairable(L) ? 8 : 0)));
  }
  std::vector<char> pair(run.size(), 0);
  for (size_t q = 0; q < run.size(); ++q) {
    qf_lattice* L = b->m[run[q]].lat;
    pair[q] = pairable(L) ? 1 : 0;
    if (pair[q]) tuned_tb_zchunk(L);  // timed outside the capture
  }
  const qf_batch::BGraph* hit = nullptr;
  for (auto& g : b->graphs)
    if (g.key == key) hit = &g;
  if (!hit) {
    // capture the k steps, then put back the host state the capture advanced
    struct Saved {
      int live;
      bool clean, xfwd, pending;
      int64_t launches;
    };
    std::vector<Saved> saved;
    for (int i : run) {
      qf_lattice* L = b->m[i].lat;
      saved.push_back({L->live, L->clean, L->xfwd_valid, L->pending_scale, L->launches});
    }
    const int64_t l0 = b->launches;
    std::vector<char> nochk(run.size(), 0), pm(run.size(), 0);
    std::vector<int> nblk(run.size(), 0);
    cudaGraph_t graph = nullptr;
    QF_BCUDA(b, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    qf_status s = QF_OK;
    for (int j = 0; j < k && s == QF_OK; ++j) {
      for (size_t q = 0; q < run.size(); ++q) pm[q] = !pair[q] ? 0 : (j & 1) ? 2 : (j + 1 < k) ? 1 : 0;
      s = batch_issue_step(b, run, nochk, nblk, st, &pm);
      for (size_t q = 0; q < run.size(); ++q) {
        qf_lattice* L = b->m[run[q]].lat;
        if (pm[q] == 2) continue;
        L->pending_scale = false;
        if (L->kinetic == QF_KIN_FDTD) L->live = 1 - L->live;
      }
    }
    const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
    const int64_t nl = b->launches - l0;
    b->launches = l0;
    for (size_t q = 0; q < run.size(); ++q) {
      qf_lattice* L = b->m[run[q]].lat;
      L->live = saved[q].live;
      L->clean = saved[q].clean;
      L->xfwd_valid = saved[q].xfwd;
      L->pending_scale = saved[q].pending;
      L->launches = saved[q].launches;
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = e2;
    if (s == QF_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (s != QF_OK || e != cudaSuccess) {
      // (a failed capture leaves the batch on ordinary launches)
      cudaGetLastError();
      b->use_graphs = false;
      return QF_OK;
    }
    if (b->graphs.size() >= 8) {
      cudaGraphExecDestroy(b->graphs.front().exec);
      b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back({key, exec, nl});
    b->graph_captures += 1;
    hit = &b->graphs.back();
  }
  QF_BCUDA(b, cudaGraphLaunch(hit->exec, st));
  b->launches += hit->launches;
  b->graph_replays += 1;
  // host bookkeeping of the k steps: the first renormalises, the others scale by 2^kcur
  for (size_t q = 0; q < run.size(); ++q) {
    auto& mb = b->m[run[q]];
    qf_lattice* L = mb.lat;
    L->K += (long long)k * L->kcur + L->jcur - L->K_check;
    L->renorm_step = L->step;
    L->pending_scale = false;
    if (L->kinetic == QF_KIN_FDTD) {
      const int swaps = pair[q] ? k / 2 + (k & 1) : k;  // one buffer swap per launch
      L->live ^= (swaps & 1);
      L->clean = true;
    }
    for (int j = 0; j < k; ++j) {
      L->step += 1;
      L->tau += L->dtau;
    }
    mb.steps_done += k;
    QF_BCUDA(b, take_snapshot(L, snap_every, st));
  }
  *used = true;
  return QF_OK;
}

extern "C" qf_status qf_batch_step(qf_batch* b, int64_t steps, int check_every, int snap_every, int* n_running) {
  if (!b) return QF_EINVAL;
  if (steps < 0 || check_every < 0 || snap_every < 0) return bfail(b, QF_EINVAL, "negative step counts");
  cudaStream_t st = b->st;
  // during the call every member issues its work on the batch stream
  struct StreamSwap {
    qf_batch* b;
    std::vector<cudaStream_t> saved;
    explicit StreamSwap(qf_batch* bb) : b(bb) {
      for (auto& x : b->m) {
        saved.push_back(x.lat->st);
        x.lat->st = b->st;
      }
    }
    ~StreamSwap() {
      for (size_t i = 0; i < saved.size(); ++i) b->m[i].lat->st = saved[i];
    }
  } swap_guard(b);
  std::vector<int> run;
  std::vector<char> chk;
  std::vector<int> nblk;
  std::vector<double> tau_t;
  std::vector<int64_t> t_of;
  std::vector<double> e3;
  std::vector<char> pm;
  for (int64_t s = 0; s < steps; ++s) {
    run.clear();
    bool any = false;
    for (int i = 0; i < (int)b->m.size(); ++i)
      if (b->m[i].status == QF_BATCH_RUNNING) {
        if (b->m[i].mid_pair) {
          b->m[i].mid_pair = false;  // this step was the second of its pair
          any = true;
        } else if (b->m[i].steps_done >= b->m[i].max_steps) {
          b->m[i].status = QF_ENOTCONV;
        } else {
          run.push_back(i);
        }
      }
    if (run.empty()) {
      if (any) continue;
      break;
    }
    if (check_every > 0 && !any) {  // (not while a member is between the steps of a pair)
      bool used = false;
      qf_status gs = batch_chunk_graph(b, run, steps - s, check_every, snap_every, st, &used);
      if (gs != QF_OK) return gs;
      if (used) {
        s += check_every - 2;  // (the loop adds the last one)
        continue;
      }
    }
    const int R = (int)run.size();
    chk.assign(R, 0);
    nblk.assign(R, 0);
    tau_t.assign(R, 0);
    t_of.assign(R, 0);
    pm.assign(R, 0);
    for (int k = 0; k < R; ++k) {
      const auto& mb = b->m[run[k]];
      qf_lattice* L = mb.lat;
      t_of[k] = L->step;
      tau_t[k] = L->tau;
      chk[k] = check_every > 0 && L->step % check_every == 0;
      // two FDTD steps in one launch where a lone lattice would pair them too
      if (s + 2 <= steps && mb.steps_done + 2 <= mb.max_steps && fuse_pair(L, L->step, check_every, snap_every))
        pm[k] = 1;
    }
    qf_status is = batch_issue_step(b, run, chk, nblk, st, &pm);
    if (is != QF_OK) return is;
    // per-member bookkeeping, identical to qf_step_n
    bool any_check = false;
    for (int k = 0; k < R; ++k) {
      auto& mb = b->m[run[k]];
      qf_lattice* L = mb.lat;
      if (pm[k]) {
        QF_BCUDA(b, after_pair(L, snap_every, st));
        mb.steps_done += 2;
        mb.mid_pair = true;
        continue;
      }
      QF_BCUDA(b, after_step(L, chk[k], nblk[k], snap_every, st));
      if (chk[k]) b->launches += 1;
      mb.steps_done += 1;
      any_check = any_check || chk[k];
    }
    if (any_check) {
      e3.assign(5 * R, 0.0);
      for (int k = 0; k < R; ++k)
        if (chk[k])
          QF_BCUDA(b, cudaMemcpyAsync(&e3[5 * k], b->m[run[k]].lat->sc()->energy, 5 * sizeof(double),
                                      cudaMemcpyDeviceToHost, st));
      QF_BCUDA(b, cudaStreamSynchronize(st));
      for (int k = 0; k < R; ++k) {
        if (!chk[k]) continue;
        auto& mb = b->m[run[k]];
        if (record_check(mb.lat, &e3[5 * k], t_of[k], tau_t[k], mb.tol_abs, mb.tol_rel, b->rule)) mb.status = QF_OK;
      }
    }
  }
  QF_BCUDA(b, cudaStreamSynchronize(st));
  for (auto& x : b->m)
    if (x.lat->kinetic == QF_KIN_FDTD) {
      qf_status es = check_device_error(x.lat);
      if (es != QF_OK) return bfail(b, es, x.lat->err);
    }
  int nr = 0;
  for (auto& x : b->m) {
    if (x.status == QF_BATCH_RUNNING && x.steps_done >= x.max_steps) x.status = QF_ENOTCONV;
    nr += x.status == QF_BATCH_RUNNING;
  }
  if (n_running) *n_running = nr;
  return QF_OK;
}

extern "C" qf_status qf_batch_use_graphs(qf_batch* b, int enable) {
  if (!b) return QF_EINVAL;
  b->use_graphs = enable != 0;
  if (!b->use_graphs) b->drop_graphs();
  return QF_OK;
}

extern "C" qf_status qf_batch_graph_info(qf_batch* b, int64_t* captures, int64_t* replays) {
  if (!b) return QF_EINVAL;
  if (captures) *captures = b->graph_captures;
  if (replays) *replays = b->graph_replays;
  return QF_OK;
}

extern "C" qf_status qf_batch_set_stopping(qf_batch* b, int rule) {
  if (!b) return QF_EINVAL;
  if (rule != QF_STOP_DIFFERENCE && rule != QF_STOP_EXTRAPOLATED) return bfail(b, QF_EINVAL, "unknown stopping rule");
  b->rule = rule;
  return QF_OK;
}

extern "C" qf_status qf_batch_info(qf_batch* b, int64_t* launches) {
  if (!b) return QF_EINVAL;
  if (launches) *launches = b->launches;
  return QF_OK;
}

extern "C" const char* qf_batch_last_error(const qf_batch* b) { return b ? b->err.c_str() : "null batch"; }
