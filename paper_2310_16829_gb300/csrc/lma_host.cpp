// Host side of the LMA library: the C-ABI of include/lma.h, argument
// validation, the FP64 coefficient builder (step a2) and the orchestration of
// the device steps (a1, a3-a7).
//
// Floating-point decisions that select pixels (aperture, detector annulus,
// bandlimit) are taken in FP64 with the same operation order as the
// definitions they implement; build with -ffp-contract=off so that no FMA
// contraction changes them between x86-64 and aarch64 hosts.
#include "../../include/lma.h"
#include "lma_device.h"

#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

using cd = std::complex<double>;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kW = lma_dev::kW;
constexpr int kMaxL = 64;
// probe strip width of the synthesis walk: 32 probe columns keep the exit waves that the
// CTAs in flight read (about (32 + 6) x 11 translates at 4-pixel spacing) well inside L2
constexpr int kSynthStrip = 32;

}  // namespace

enum { K_POT = 0, K_SLICE, K_SYNTH, K_FIN, K_COUNT };

struct lma_ctx {
  int device = -1;
  bool host_only = true;
  std::string err;
  // measurement
  bool prof = false;
  lma_kernel_stat stat[K_COUNT] = {};
  struct Pending {
    cudaEvent_t a, b;
    int kind;
  };
  std::vector<Pending> pend;
  std::vector<cudaEvent_t> pool;
  bool capturing = false;
  // device copies of slice item lists, keyed by contents, least recently used last out.
  // Lists up to kListSlot bytes live in slots of one slab allocated at first use; longer
  // ones get their own buffers, reused on eviction when large enough (cudaMalloc and
  // cudaFree can wait for the whole device, which must not happen on an edit's path)
  struct List {
    std::vector<int32_t> items;
    uint64_t hash = 0;
    void* p = nullptr;
    size_t bytes = 0;
    bool owned = false;   // own buffer (else a slab slot)
    bool used = false;    // holds a list
  };
  std::vector<List> lists;
  void* list_slab = nullptr;
  int64_t alloc_base = 0;                                   // device allocations at profile reset
  std::vector<std::pair<void*, uint64_t>> capture_lists;   // lists read by the capture in progress
  int* d_counter = nullptr;                                 // [0] work counter of dynamic slice launches,
                                                            // [1] status word of the tensor-core slice kernel
  bool tc_launched = false;                                 // a slice launch with a status word since the last check
  void* gen_scratch = nullptr;                              // per-CTA waves of the W = 256 slice kernel
  size_t gen_scratch_bytes = 0;
  // grouped synthesis: probe waves of a chunk of probe rows, and the detection pass's tables
  // (tidx = i, which also serves as the list of region indices, alpha = 1, shift = 0)
  void* psi = nullptr;
  size_t psi_bytes = 0;
  void* psi_tab = nullptr;
  int64_t psi_tab_n = 0;
  int synth_mode = -1;                                      // LMA_SYNTH_*
  int64_t psi_max = int64_t(2) << 30;                       // largest probe-wave buffer (bytes)
  void* stage = nullptr;                                    // pinned staging buffer (kStageBytes)
  // slice launch modes: forced (>= 0), or the timed choice per launch shape
  int forced_mode = -1;
  bool autotune = false;
  // real-space propagation (lma_image_realspace): the K1 x K2 kernel of the call in progress
  int rs_k1 = 0, rs_k2 = 0;
  const float2* rs_q = nullptr;
  struct Tune {
    std::vector<int64_t> key;
    lma_tuning rec;
  };
  std::vector<Tune> tune;
  struct SynthTune {
    std::vector<int64_t> key;
    lma_synth_tuning rec;
  };
  std::vector<SynthTune> synth_tune;
  // captured image sequences (lma_image_many with LMA_IMAGE_GRAPH)
  struct Graph {
    std::vector<uintptr_t> key;
    std::vector<std::pair<void*, uint64_t>> lists;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<Graph> graphs;
};

namespace {

lma_status fail(lma_ctx* ctx, lma_status code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

#define CUDA_TRY(ctx, call)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? LMA_ERR_OOM : LMA_ERR_CUDA,       \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);      \
    }                                                                                        \
  } while (0)

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int mod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// signed frequency index m' in FFT order
int signed_index(int m, int n) { return m < (n + 1) / 2 ? m : m - n; }

// minimum-image offset in [-n/2, n/2)
int min_image(int d, int n) { return mod(d + n / 2, n) - n / 2; }

// -------------------------------------------------------------------------------------------
// host FFT (radix-2, in place), used only for the FP64 probe of the coefficient step
// -------------------------------------------------------------------------------------------
void fft1(cd* a, int n, int stride, bool inverse) {
  std::vector<cd> tmp(n);
  for (int i = 0; i < n; ++i) tmp[i] = a[static_cast<size_t>(i) * stride];
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(tmp[i], tmp[j]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    const double ang = (inverse ? 2.0 : -2.0) * kPi / len;
    for (int i = 0; i < n; i += len) {
      for (int k = 0; k < len / 2; ++k) {
        const cd w(std::cos(ang * k), std::sin(ang * k));
        const cd u = tmp[i + k];
        const cd v = tmp[i + k + len / 2] * w;
        tmp[i + k] = u + v;
        tmp[i + k + len / 2] = u - v;
      }
    }
  }
  for (int i = 0; i < n; ++i) a[static_cast<size_t>(i) * stride] = tmp[i];
}

void fft2(std::vector<cd>& a, int ny, int nx, bool inverse) {
  for (int y = 0; y < ny; ++y) fft1(&a[static_cast<size_t>(y) * nx], nx, 1, inverse);
  for (int x = 0; x < nx; ++x) fft1(&a[x], ny, nx, inverse);
}

// -------------------------------------------------------------------------------------------
// complex Householder least squares: min ||A x - b||, A is m x n column-major
// -------------------------------------------------------------------------------------------
bool lstsq_householder(std::vector<cd>& A, int m, int n, std::vector<cd>& b, std::vector<cd>& x) {
  std::vector<cd> diag(n);
  for (int k = 0; k < n; ++k) {
    cd* a = &A[static_cast<size_t>(k) * m];
    double norm2 = 0.0;
    for (int i = k; i < m; ++i) norm2 += std::norm(a[i]);
    const double nrm = std::sqrt(norm2);
    if (nrm == 0.0) return false;
    const double ak = std::abs(a[k]);
    const cd phase = ak > 0.0 ? a[k] / ak : cd(1.0, 0.0);
    const cd alpha = -phase * nrm;
    a[k] -= alpha;   // v = x - alpha e1, stored in the column
    double vv = 0.0;
    for (int i = k; i < m; ++i) vv += std::norm(a[i]);
    for (int j = k + 1; j < n; ++j) {
      cd* c = &A[static_cast<size_t>(j) * m];
      cd s(0.0, 0.0);
      for (int i = k; i < m; ++i) s += std::conj(a[i]) * c[i];
      s *= 2.0 / vv;
      for (int i = k; i < m; ++i) c[i] -= s * a[i];
    }
    cd s(0.0, 0.0);
    for (int i = k; i < m; ++i) s += std::conj(a[i]) * b[i];
    s *= 2.0 / vv;
    for (int i = k; i < m; ++i) b[i] -= s * a[i];
    diag[k] = alpha;
  }
  x.assign(n, cd(0.0, 0.0));
  for (int k = n - 1; k >= 0; --k) {
    cd s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[static_cast<size_t>(j) * m + k] * x[j];
    x[k] = s / diag[k];
  }
  return true;
}

// bandlimit threshold: the largest s with 4 s <= frac^2 n^2 (FP64 right-hand side)
int bandlimit_r2(double frac, int n) {
  const double lim = frac * frac * static_cast<double>(n) * static_cast<double>(n);
  long s = static_cast<long>(std::floor(lim / 4.0));
  while (4.0 * static_cast<double>(s + 1) <= lim) ++s;
  while (s >= 0 && 4.0 * static_cast<double>(s) > lim) --s;
  return static_cast<int>(s);
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

// device and pinned-host allocations made by the library (all contexts)
std::atomic<int64_t> g_allocations{0};

cudaError_t counted_malloc(void** p, size_t bytes) {
  g_allocations.fetch_add(1, std::memory_order_relaxed);
  return cudaMalloc(p, bytes);
}

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return cudaSuccess;
  b.release();
  cudaError_t e = counted_malloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}

struct Rect {
  int x0, y0, w, h;   // periodic pixel rectangle
};

// Host <-> device copies through the context's pinned staging buffer. A pageable copy
// is staged by the driver through a buffer shared by the whole process, so one
// thread's pageable read-back of a long stream holds up every other thread's
// pageable uploads (an edit waited for a full image). Each chunk is synchronized on
// the stream before the buffer is reused, and the buffer is free when a call returns.
constexpr size_t kStageBytes = size_t(8) << 20;

struct HostPart {
  void* dst;
  const void* src;
  size_t bytes;
};

cudaError_t ensure_stage(lma_ctx* ctx) {
  if (ctx->stage) return cudaSuccess;
  g_allocations.fetch_add(1, std::memory_order_relaxed);
  return cudaMallocHost(&ctx->stage, kStageBytes);
}

// several host -> device copies, packed into the staging buffer
cudaError_t upload_parts(lma_ctx* ctx, std::initializer_list<HostPart> parts, cudaStream_t st) {
  cudaError_t e = ensure_stage(ctx);
  if (e != cudaSuccess) return e;
  char* stage = static_cast<char*>(ctx->stage);
  size_t used = 0;
  for (const HostPart& p : parts) {
    for (size_t off = 0; off < p.bytes;) {
      if (used == kStageBytes) {
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        used = 0;
      }
      const size_t n = std::min(kStageBytes - used, p.bytes - off);
      std::memcpy(stage + used, static_cast<const char*>(p.src) + off, n);
      e = cudaMemcpyAsync(static_cast<char*>(p.dst) + off, stage + used, n, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return e;
      used += n;
      off += n;
    }
  }
  return cudaStreamSynchronize(st);
}

cudaError_t upload(lma_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  return upload_parts(ctx, {HostPart{dst, src, bytes}}, st);
}

// device -> host through the staging buffer; returns when dst holds the data
cudaError_t download(lma_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  cudaError_t e = ensure_stage(ctx);
  if (e != cudaSuccess) return e;
  for (size_t off = 0; off < bytes; off += kStageBytes) {
    const size_t n = std::min(kStageBytes, bytes - off);
    if ((e = cudaMemcpyAsync(ctx->stage, static_cast<const char*>(src) + off, n, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    std::memcpy(static_cast<char*>(dst) + off, ctx->stage, n);
  }
  return cudaSuccess;
}

cudaEvent_t pool_event(lma_ctx* ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// count a launch and, when timing is on, bracket it with events on its stream
template <class F>
cudaError_t counted(lma_ctx* ctx, int kind, int64_t units, cudaStream_t st, F&& launch) {
  if (ctx->capturing) return launch();
  ctx->stat[kind].launches++;
  ctx->stat[kind].units += units;
  if (!ctx->prof) return launch();
  cudaEvent_t a = pool_event(ctx), b = pool_event(ctx);
  if (!a || !b) return launch();
  cudaEventRecord(a, st);
  cudaError_t e = launch();
  cudaEventRecord(b, st);
  ctx->pend.push_back({a, b, kind});
  return e;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// specimen
// ---------------------------------------------------------------------------------------------
struct PhononSet {
  std::vector<double> x, y;
  std::vector<int16_t> sp;
  std::vector<int32_t> slc;
  std::vector<int32_t> slice_start;   // [n_slices + 1] over the slice-sorted arrays
  DevBuf dx, dy, dsp, dss;
  bool dirty = true;
};

struct lma_specimen {
  lma_ctx* ctx = nullptr;
  lma_grid g{};
  std::vector<double> peak, frac, width;
  double r_cut = 0.0;
  std::vector<PhononSet> ph;
  DevBuf d_peak;
  DevBuf d_t;                          // transmission stacks, one slot per configuration in flight
  int t_slots = 0;                     // slots allocated in d_t
  std::vector<int> t_phonon;           // configuration held by each slot (-1: none)
  std::vector<std::vector<Rect>> t_stale;   // per slot: pixel rectangles to rebuild
  int64_t epoch = 0;          // bumps on every edit
};

// ---------------------------------------------------------------------------------------------
// basis
// ---------------------------------------------------------------------------------------------
struct CoefSet {
  std::vector<cd> alpha;
  std::vector<int> odx, ody;   // offsets of the L nearest translates (pixels)
  double err_l2 = 0.0, err_sup = 0.0;
};

struct RegionTables {
  lma_region r{};
  int64_t n_probes = 0;
  DevBuf tidx, alpha, shift;
  std::vector<int32_t> h_tidx;   // host copy of the translate indices
  std::vector<uint8_t> needed;   // translates the region reads
  int shift_abs = 0;             // largest |component| of the placements
};

struct lma_basis {
  lma_ctx* ctx = nullptr;
  const lma_specimen* spec = nullptr;
  lma_probe probe{};
  lma_basis_desc desc{};
  double gauss_sigma = 0.0;
  int trig_n = 0;              // degree n of the trigonometric input waves
  int W = 128;                 // propagation window W = detection window D (pixels)
  float tc_in = 1.f, tc_out = 1.f;   // input-wave factor of the tensor-core DFT passes and its inverse
  int nx = 0, ny = 0;
  int Sx = 0, Sy = 0, ox = 0, oy = 0, nax = 0, nay = 0;
  int64_t nT = 0;
  std::vector<cd> psi0;        // full-grid probe centred at pixel 0 (lazy)
  std::vector<cd> uW;          // W x W input wave
  std::vector<float> ex, ey;   // interleaved complex
  int r2max = 0;
  std::map<std::pair<int, int>, CoefSet> sets;
  // device
  DevBuf d_uW, d_ex, d_ey, d_U, d_Uscale, d_acc, d_det;
  DevBuf d_lab;                  // 3D STEM ring labels: [n_labels + 1] CSR starts, then pixels
  std::vector<double> lab_key;   // (width, n_rings) of d_lab
  DevBuf d_pat, d_pat_acc;       // 4D STEM: FP32 pattern slots, FP64 running sum
  // memory-bounded partition (Sec. 4.2.4): the last plan and its device tables
  struct Part {
    std::vector<int32_t> probes;       // region indices b * npx + a
    std::vector<int32_t> items, outs;  // new translates (even window origins first), their store entries
    int n_even = 0;
    size_t o_probes = 0, o_tidx = 0, o_alpha = 0, o_shift = 0, o_items = 0, o_outs = 0;   // in d_plan
  };
  lma_region plan_r{};
  lma_partition_desc plan_d{};
  bool plan_valid = false, plan_dev = false;
  std::vector<Part> parts;
  int64_t plan_runs = 0, plan_peak = 0;
  std::vector<int32_t> plan_tab;     // host copy of d_plan
  DevBuf d_plan, d_Up, d_Upscale;
  // partial coherence: coefficient tables of the probe variants of the last call
  std::vector<double> var_key;
  DevBuf d_var;                  // [n_var][n_probes][L] complex64 coefficients, then [n_var] weights
  DevBuf d_rsq;                  // real-space propagation kernel [K2][K1] complex64
  std::vector<int> rsq_key;
  bool dev_tables = false;
  int B = 0;                     // exit-wave store slots (configurations in flight)
  std::vector<int> U_phonon;     // configuration held by each slot (-1: none)
  int64_t U_epoch = -1;
  std::vector<uint8_t> valid;    // [slot][translate]
  RegionTables reg;
  bool reg_valid = false;
  std::vector<double> det_key;
};

namespace {

bool device_ready(lma_ctx* ctx) {
  if (!ctx || ctx->host_only) return false;
  return cudaSetDevice(ctx->device) == cudaSuccess;
}

// full-grid probe psi_0 of probe parameters pr (eq. probe_wave_function at p = 0), unit norm
void probe_at_origin(const lma_basis* b, const lma_probe& pr, std::vector<cd>& out) {
  const lma_grid& g = b->spec->g;
  const int nx = g.nx, ny = g.ny;
  const double dx = g.lx / nx, dy = g.ly / ny, lam = g.lambda;
  std::vector<cd> spec(static_cast<size_t>(nx) * ny);
  for (int iy = 0; iy < ny; ++iy) {
    const double ky = signed_index(iy, ny) / (ny * dy);
    for (int ix = 0; ix < nx; ++ix) {
      const double kx = signed_index(ix, nx) / (nx * dx);
      const double k2 = ky * ky + kx * kx;
      const bool ap = lam * std::sqrt(k2) < pr.alpha_max;
      if (!ap) continue;
      const double chi = 0.5 * kPi * pr.cs * lam * lam * lam * k2 * k2 - kPi * pr.defocus * lam * k2;
      spec[static_cast<size_t>(iy) * nx + ix] = std::exp(cd(0.0, -chi));
    }
  }
  fft2(spec, ny, nx, true);
  double n2 = 0.0;
  for (const cd& c : spec) n2 += std::norm(c);
  const double s = 1.0 / std::sqrt(n2);
  for (cd& c : spec) c *= s;
  out.swap(spec);
}

void build_probe(lma_basis* b) {
  if (b->psi0.empty()) probe_at_origin(b, b->probe, b->psi0);
}

// the input wave on its window (Sec. 4.2.3)
void build_input_wave(lma_basis* b) {
  const lma_grid& g = b->spec->g;
  const double dx = g.lx / g.nx, dy = g.ly / g.ny;
  b->uW.assign(static_cast<size_t>(b->W) * b->W, cd(0.0, 0.0));
  if (b->desc.kind == LMA_BASIS_GAUSS) {
    const double s = b->gauss_sigma;
    for (int y = 0; y < b->W; ++y) {
      const double ry = (y - b->W / 2) * dy;
      for (int x = 0; x < b->W; ++x) {
        const double rx = (x - b->W / 2) * dx;
        b->uW[static_cast<size_t>(y) * b->W + x] = cd(std::exp(-(ry * ry + rx * rx) / (2.0 * s * s)), 0.0);
      }
    }
  } else if (b->desc.kind == LMA_BASIS_TRIG || b->desc.kind == LMA_BASIS_TRIG_RADIAL) {
    // phi_n(t) = 1 + 2 sum_{k=1..n} cos(k t) cos(k pi / (2n + 2))
    const int n = b->trig_n;
    auto phi = [n](double t) {
      double v = 1.0;
      for (int k = 1; k <= n; ++k) v += 2.0 * std::cos(k * t) * std::cos(k * kPi / (2 * n + 2));
      return v;
    };
    if (b->desc.kind == LMA_BASIS_TRIG) {
      std::vector<double> py(b->W), px(b->W);
      for (int i = 0; i < b->W; ++i) {
        py[i] = phi(2.0 * kPi * (i - b->W / 2) / g.ny);
        px[i] = phi(2.0 * kPi * (i - b->W / 2) / g.nx);
      }
      for (int y = 0; y < b->W; ++y)
        for (int x = 0; x < b->W; ++x) b->uW[static_cast<size_t>(y) * b->W + x] = cd(py[y] * px[x], 0.0);
    } else {
      for (int y = 0; y < b->W; ++y) {
        const double ry = (y - b->W / 2) * dy;
        for (int x = 0; x < b->W; ++x) {
          const double rx = (x - b->W / 2) * dx;
          b->uW[static_cast<size_t>(y) * b->W + x] = cd(phi(2.0 * kPi * std::sqrt(ry * ry + rx * rx) / g.lx), 0.0);
        }
      }
    }
  } else {
    build_probe(b);
    for (int y = 0; y < b->W; ++y)
      for (int x = 0; x < b->W; ++x)
        b->uW[static_cast<size_t>(y) * b->W + x] =
            b->psi0[static_cast<size_t>(mod(y - b->W / 2, g.ny)) * g.nx + mod(x - b->W / 2, g.nx)];
  }
}

// the L nearest translates of probe p (Sec. 4.2.1 option (iii)); ties by (d^2, dy, dx)
// offsets of the L input waves nearest to pixel (px, py) (the basis's L when L <= 0)
void nearest(const lma_basis* b, int px, int py, std::vector<int>& odx, std::vector<int>& ody, int L = 0) {
  struct Cand {
    long d2;
    int dy, dx;
  };
  std::vector<Cand> c;
  c.reserve(static_cast<size_t>(b->nT));
  for (int ib = 0; ib < b->nay; ++ib) {
    const int ty = mod(b->oy + ib * b->Sy, b->ny);
    const int ddy = min_image(ty - py, b->ny);
    for (int ia = 0; ia < b->nax; ++ia) {
      const int tx = mod(b->ox + ia * b->Sx, b->nx);
      const int ddx = min_image(tx - px, b->nx);
      c.push_back({static_cast<long>(ddx) * ddx + static_cast<long>(ddy) * ddy, ddy, ddx});
    }
  }
  if (L <= 0) L = b->desc.L;
  std::partial_sort(c.begin(), c.begin() + L, c.end(), [](const Cand& u, const Cand& v) {
    if (u.d2 != v.d2) return u.d2 < v.d2;
    if (u.dy != v.dy) return u.dy < v.dy;
    return u.dx < v.dx;
  });
  odx.resize(L);
  ody.resize(L);
  for (int j = 0; j < L; ++j) {
    odx[j] = c[j].dx;
    ody[j] = c[j].dy;
  }
}

// Closed-form coefficients of the tensor trigonometric input waves (Sec. 2, Sec. 4.2.3: no
// least squares). With P the DFT of the probe centred at pixel 0, w_k = cos(k pi / (2n + 2))
// and m_x x m_y input waves of I_f (m >= 2n + 1 per axis), the input wave at offset d from
// the probe gets
//   a(d) = sum_{|k_x|,|k_y|<=n} P(k) / (N_x N_y w_kx w_ky m_x m_y) e^{2 pi i (k_x d_x / N_x + k_y d_y / N_y)};
// over all input waves this represents the probe's part in T_n x T_n exactly (m = 2n + 1:
// the M^-1 of Sec. 2 from its definition M = diag(w) W; m > 2n + 1: the minimum-norm
// representation, the lattice sum of e^{2 pi i (k' - k) X / N} vanishing for k' != k).
void trig_closed_alpha(const lma_basis* b, const std::vector<cd>& psi0, const CoefSet& cs, std::vector<cd>& x) {
  const int nx = b->nx, ny = b->ny, n = b->trig_n, K = 2 * n + 1;
  std::vector<cd> P = psi0;
  fft2(P, ny, nx, false);
  std::vector<double> w(K);
  for (int i = 0; i < K; ++i) w[i] = std::cos((i - n) * kPi / (2 * n + 2));
  const double norm = static_cast<double>(nx) * ny * static_cast<double>(b->nax) * b->nay;
  std::vector<cd> G(static_cast<size_t>(K) * K);
  for (int iy = 0; iy < K; ++iy)
    for (int ix = 0; ix < K; ++ix)
      G[static_cast<size_t>(iy) * K + ix] =
          P[static_cast<size_t>(mod(iy - n, ny)) * nx + mod(ix - n, nx)] / (norm * w[ix] * w[iy]);
  const int L = static_cast<int>(cs.odx.size());
  x.assign(L, cd(0.0, 0.0));
  std::vector<cd> ex(K), ey(K);
  for (int j = 0; j < L; ++j) {
    for (int i = 0; i < K; ++i) {
      ex[i] = std::polar(1.0, 2.0 * kPi * (i - n) * cs.odx[j] / nx);
      ey[i] = std::polar(1.0, 2.0 * kPi * (i - n) * cs.ody[j] / ny);
    }
    cd acc(0.0, 0.0);
    for (int iy = 0; iy < K; ++iy) {
      cd row(0.0, 0.0);
      for (int ix = 0; ix < K; ++ix) row += G[static_cast<size_t>(iy) * K + ix] * ex[ix];
      acc += row * ey[iy];
    }
    x[j] = acc;
  }
}

// least-squares coefficients of one probe class (eqs. lma_approximation_exit1_0 / exit2_0),
// in coordinates relative to the probe (probe at pixel 0, translate j at its offset)
// least squares of probe psi0 on the input waves at cs.odx / cs.ody (their count is L)
lma_status solve_set_for(lma_basis* b, const std::vector<cd>& psi0, CoefSet& cs) {
  const int nx = b->nx, ny = b->ny, L = static_cast<int>(cs.odx.size());
  // bounding box of the union of windows [o - W/2, o + W/2)
  int ylo = 1 << 30, yhi = -(1 << 30), xlo = 1 << 30, xhi = -(1 << 30);
  for (int j = 0; j < L; ++j) {
    ylo = std::min(ylo, cs.ody[j] - b->W / 2);
    yhi = std::max(yhi, cs.ody[j] + b->W / 2);
    xlo = std::min(xlo, cs.odx[j] - b->W / 2);
    xhi = std::max(xhi, cs.odx[j] + b->W / 2);
  }
  if (yhi - ylo >= ny) {
    ylo = 0;
    yhi = ny;
  }
  if (xhi - xlo >= nx) {
    xlo = 0;
    xhi = nx;
  }
  std::vector<size_t> rows;
  std::vector<int> wy, wx;   // window-local coordinates per (row, j) computed on the fly
  for (int yy = ylo; yy < yhi; ++yy)
    for (int xx = xlo; xx < xhi; ++xx) {
      bool any = false;
      for (int j = 0; j < L && !any; ++j)
        any = mod(yy - (cs.ody[j] - b->W / 2), ny) < b->W && mod(xx - (cs.odx[j] - b->W / 2), nx) < b->W;
      if (any) rows.push_back(static_cast<size_t>(mod(yy, ny)) * nx + mod(xx, nx));
    }
  const int m = static_cast<int>(rows.size());
  std::vector<cd> A(static_cast<size_t>(m) * L, cd(0.0, 0.0)), rhs(m);
  std::vector<uint8_t> in_rows(static_cast<size_t>(nx) * ny, 0);
  for (int i = 0; i < m; ++i) {
    const int gy = static_cast<int>(rows[i] / nx), gx = static_cast<int>(rows[i] % nx);
    in_rows[rows[i]] = 1;
    rhs[i] = psi0[rows[i]];
    for (int j = 0; j < L; ++j) {
      const int ly = mod(gy - (cs.ody[j] - b->W / 2), ny), lx = mod(gx - (cs.odx[j] - b->W / 2), nx);
      if (ly < b->W && lx < b->W) A[static_cast<size_t>(j) * m + i] = b->uW[static_cast<size_t>(ly) * b->W + lx];
    }
  }
  std::vector<cd> A0 = A, rhs0 = rhs, x;
  if (b->desc.coef_mode == LMA_COEF_TRIG_CLOSED) {
    trig_closed_alpha(b, psi0, cs, x);
  } else if (!lstsq_householder(A, m, L, rhs, x)) {
    return fail(b->ctx, LMA_ERR_INVALID, "least squares: input waves are linearly dependent");
  }
  cs.alpha = x;
  // errors over the full grid (outside the windows the approximation is zero)
  double r2 = 0.0, rmax = 0.0, n2 = 0.0, pmax = 0.0;
  for (int i = 0; i < m; ++i) {
    cd acc(0.0, 0.0);
    for (int j = 0; j < L; ++j) acc += A0[static_cast<size_t>(j) * m + i] * x[j];
    const double e = std::abs(rhs0[i] - acc);
    r2 += e * e;
    rmax = std::max(rmax, e);
  }
  for (size_t k = 0; k < psi0.size(); ++k) {
    const double a = std::abs(psi0[k]);
    n2 += a * a;
    pmax = std::max(pmax, a);
    if (!in_rows[k]) {
      r2 += a * a;
      rmax = std::max(rmax, a);
    }
  }
  cs.err_l2 = std::sqrt(r2 / n2);
  cs.err_sup = rmax / pmax;
  return LMA_OK;
}

lma_status solve_set(lma_basis* b, CoefSet& cs) {
  build_probe(b);
  return solve_set_for(b, b->psi0, cs);
}

std::pair<int, int> class_key(const lma_basis* b, int px, int py) {
  return {mod(px - b->ox, b->Sx), mod(py - b->oy, b->Sy)};
}

lma_status coef_set(lma_basis* b, int px, int py, const CoefSet** out) {
  const auto key = class_key(b, px, py);
  auto it = b->sets.find(key);
  if (it == b->sets.end()) {
    CoefSet cs;
    nearest(b, px, py, cs.odx, cs.ody);
    lma_status st = solve_set(b, cs);
    if (st != LMA_OK) return st;
    it = b->sets.emplace(key, std::move(cs)).first;
  }
  *out = &it->second;
  return LMA_OK;
}

int64_t translate_index(const lma_basis* b, int tx, int ty) {
  const int ia = mod(tx - b->ox, b->nx) / b->Sx, ib = mod(ty - b->oy, b->ny) / b->Sy;
  return static_cast<int64_t>(ib) * b->nax + ia;
}

lma_status validate_region(lma_ctx* ctx, const lma_basis* b, const lma_region* r) {
  if (!r || r->npx <= 0 || r->npy <= 0 || r->spacing_px[0] <= 0 || r->spacing_px[1] <= 0)
    return fail(ctx, LMA_ERR_INVALID, "region: empty or non-positive spacing");
  if (static_cast<int64_t>(r->npx) * r->npy > (1ll << 26))
    return fail(ctx, LMA_ERR_INVALID, "region: too many probes");
  (void)b;
  return LMA_OK;
}

// device tables of a basis (input wave, propagator factors)
// input wave and propagator factors on the device (no exit-wave store)
// windows the device kernels implement (geometry and coefficients take every supported W)
lma_status device_window(const lma_basis* b) {
  if (b->W == kW) return LMA_OK;
  if (b->desc.precision != LMA_PREC_C64)
    return fail(b->ctx, LMA_ERR_UNSUPPORTED, "window %d: the device path is complex64 only (W = %d has the "
                "FP16 store and the tensor-core form)", b->W, kW);
  return LMA_OK;
}

lma_status ensure_basis_tables(lma_basis* b, cudaStream_t st) {
  lma_ctx* ctx = b->ctx;
  lma_status sw = device_window(b);
  if (sw != LMA_OK) return sw;
  if (b->d_uW.p && b->d_ex.p && b->d_ey.p) return LMA_OK;
  std::vector<float> uw(2 * static_cast<size_t>(b->W) * b->W);
  for (size_t k = 0; k < b->uW.size(); ++k) {
    uw[2 * k] = static_cast<float>(b->uW[k].real());
    uw[2 * k + 1] = static_cast<float>(b->uW[k].imag());
  }
  CUDA_TRY(ctx, ensure(b->d_uW, uw.size() * sizeof(float)));
  CUDA_TRY(ctx, ensure(b->d_ex, b->ex.size() * sizeof(float)));
  CUDA_TRY(ctx, ensure(b->d_ey, b->ey.size() * sizeof(float)));
  CUDA_TRY(ctx, upload_parts(ctx, {HostPart{b->d_uW.p, uw.data(), uw.size() * sizeof(float)},
                                    HostPart{b->d_ex.p, b->ex.data(), b->ex.size() * sizeof(float)},
                                    HostPart{b->d_ey.p, b->ey.data(), b->ey.size() * sizeof(float)}},
                             st));
  return LMA_OK;
}

// tables plus the exit-wave store of B configurations
lma_status ensure_basis_device(lma_basis* b, cudaStream_t st) {
  lma_ctx* ctx = b->ctx;
  if (b->dev_tables) return LMA_OK;
  lma_status s0 = ensure_basis_tables(b, st);
  if (s0 != LMA_OK) return s0;
  // phonon batch: configurations whose exit waves (and transmissions) are held at once
  const bool half = b->desc.precision == LMA_PREC_FP16_STORE;
  const int nph = static_cast<int>(b->spec->ph.size());
  const lma_grid& g = b->spec->g;
  const size_t u_cfg = static_cast<size_t>(b->nT) * b->W * b->W * (half ? 4 : sizeof(float2));
  const size_t t_cfg = static_cast<size_t>(g.n_slices) * (g.nx + kW) * (g.ny + kW) * sizeof(float2);
  int B = b->desc.phonon_batch;
  if (B <= 0) {
    size_t fr = 0, tot = 0;
    CUDA_TRY(ctx, cudaMemGetInfo(&fr, &tot));
    B = static_cast<int>(std::min<size_t>(static_cast<size_t>(nph), (fr * 2 / 5) / (u_cfg + t_cfg)));
  }
  B = std::max(1, std::min(B, nph));
  CUDA_TRY(ctx, ensure(b->d_U, u_cfg * B));
  if (half) CUDA_TRY(ctx, ensure(b->d_Uscale, static_cast<size_t>(b->nT) * B * sizeof(float)));
  b->B = B;
  b->valid.assign(static_cast<size_t>(b->nT) * B, 0);
  b->U_phonon.assign(B, -1);
  b->dev_tables = true;
  return LMA_OK;
}

// x = hi + lo with hi = fp32(x), lo = fp32(x - hi)
float2 split_f32(double x) {
  const float hi = static_cast<float>(x);
  return make_float2(hi, static_cast<float>(x - static_cast<double>(hi)));
}

// upload the atoms of a configuration (slice-sorted) if they changed
lma_status ensure_atoms_device(lma_specimen* sp, int phi, cudaStream_t st) {
  lma_ctx* ctx = sp->ctx;
  PhononSet& p = sp->ph[phi];
  if (!p.dirty && p.dx.p) return LMA_OK;
  const size_t n = std::max<size_t>(1, p.x.size());
  // positions as exact pairs hi + lo of FP32 values (the same 8 bytes as the FP64 value; the
  // potential kernel works with them in FP32 instructions only)
  std::vector<float2> xs(p.x.size()), ys(p.y.size());
  for (size_t i = 0; i < p.x.size(); ++i) {
    xs[i] = split_f32(p.x[i]);
    ys[i] = split_f32(p.y[i]);
  }
  CUDA_TRY(ctx, ensure(p.dx, n * sizeof(float2)));
  CUDA_TRY(ctx, ensure(p.dy, n * sizeof(float2)));
  CUDA_TRY(ctx, ensure(p.dsp, n * sizeof(int16_t)));
  CUDA_TRY(ctx, ensure(p.dss, p.slice_start.size() * sizeof(int32_t)));
  CUDA_TRY(ctx, upload_parts(ctx, {HostPart{p.dx.p, xs.data(), xs.size() * sizeof(float2)},
                                    HostPart{p.dy.p, ys.data(), ys.size() * sizeof(float2)},
                                    HostPart{p.dsp.p, p.sp.data(), p.sp.size() * sizeof(int16_t)},
                                    HostPart{p.dss.p, p.slice_start.data(), p.slice_start.size() * sizeof(int32_t)}},
                             st));
  p.dirty = false;
  return LMA_OK;
}

// x mod l in [0, l)
double wrap_period(double x, double l) {
  double w = x - l * std::floor(x / l);
  if (w >= l) w -= l;
  if (w < 0.0) w += l;
  return w;
}

size_t t_slot_elems(const lma_grid& g) {
  return static_cast<size_t>(g.n_slices) * (g.nx + kW) * (g.ny + kW);
}

lma_status launch_t(lma_specimen* sp, int slot, int phi, const Rect& r, cudaStream_t st) {
  lma_ctx* ctx = sp->ctx;
  const lma_grid& g = sp->g;
  PhononSet& p = sp->ph[phi];
  lma_dev::PotArgs a{};
  a.ax = static_cast<const float2*>(p.dx.p);
  a.ay = static_cast<const float2*>(p.dy.p);
  a.asp = static_cast<const int16_t*>(p.dsp.p);
  a.slice_start = static_cast<const int32_t*>(p.dss.p);
  a.peak = static_cast<const float*>(sp->d_peak.p);
  a.n_species = static_cast<int>(sp->peak.size());
  a.n_terms = static_cast<int>(sp->frac.size());
  for (int q = 0; q < a.n_terms; ++q) {
    a.frac[q] = static_cast<float>(sp->frac[q]);
    a.inv2w2[q] = static_cast<float>(1.0 / (2.0 * sp->width[q] * sp->width[q]));
  }
  a.rc2 = static_cast<float>(sp->r_cut * sp->r_cut);
  a.nx = g.nx;
  a.ny = g.ny;
  a.n_slices = g.n_slices;
  const double dx = g.lx / g.nx, dy = g.ly / g.ny;
  const float2 dx2 = split_f32(dx), dy2 = split_f32(dy);
  a.dx_hi = dx2.x;
  a.dx_lo = dx2.y;
  a.dy_hi = dy2.x;
  a.dy_lo = dy2.y;
  const float2 lx2 = split_f32(g.lx), ly2 = split_f32(g.ly), c75x = split_f32(7.5 * dx), c75y = split_f32(7.5 * dy);
  a.lx_hi = lx2.x;
  a.lx_lo = lx2.y;
  a.ly_hi = ly2.x;
  a.ly_lo = ly2.y;
  a.c75x_hi = c75x.x;
  a.c75x_lo = c75x.y;
  a.c75y_hi = c75y.x;
  a.c75y_lo = c75y.y;
  // a margin far above the FP32 rounding of the offsets keeps the test a superset of the exact one
  a.limx = static_cast<float>(sp->r_cut + 8.0 * dx) + 1e-4f;
  a.limy = static_cast<float>(sp->r_cut + 8.0 * dy) + 1e-4f;
  a.sigma = static_cast<float>(g.sigma);
  // Tiles sit on the absolute 16-pixel grid whatever the rectangle, so a
  // pixel is always computed by the same tile origin: a partial rebuild is
  // bitwise equal to a full one (atoms are taken relative to the tile origin).
  const int x0 = r.x0 - r.x0 % 16, y0 = r.y0 - r.y0 % 16;
  a.rx0 = x0;
  a.ry0 = y0;
  a.rw = std::min(g.nx, ((r.x0 - x0 + r.w + 15) / 16) * 16);
  a.rh = std::min(g.ny, ((r.y0 - y0 + r.h + 15) / 16) * 16);
  a.t = static_cast<float2*>(sp->d_t.p) + slot * t_slot_elems(g);
  const int64_t units = static_cast<int64_t>(r.w) * r.h * g.n_slices;
  CUDA_TRY(ctx, counted(ctx, K_POT, units, st, [&] { return lma_dev::launch_potential(a, st); }));
  return LMA_OK;
}

// at least n transmission slots (growing the buffer forgets every slot's contents)
lma_status reserve_t_slots(lma_specimen* sp, int n) {
  lma_ctx* ctx = sp->ctx;
  if (n <= sp->t_slots) return LMA_OK;
  CUDA_TRY(ctx, ensure(sp->d_t, t_slot_elems(sp->g) * n * sizeof(float2)));
  sp->t_slots = n;
  sp->t_phonon.assign(n, -1);
  sp->t_stale.assign(n, {});
  return LMA_OK;
}

// make transmission slot `slot` hold configuration phi with no stale pixels
lma_status ensure_t(lma_specimen* sp, int slot, int phi, bool force, cudaStream_t st) {
  lma_ctx* ctx = sp->ctx;
  const lma_grid& g = sp->g;
  lma_status s = reserve_t_slots(sp, slot + 1);
  if (s != LMA_OK) return s;
  if (!sp->d_peak.p) {
    std::vector<float> pk(sp->peak.begin(), sp->peak.end());
    CUDA_TRY(ctx, ensure(sp->d_peak, pk.size() * sizeof(float)));
    CUDA_TRY(ctx, upload(ctx, sp->d_peak.p, pk.data(), pk.size() * sizeof(float), st));
  }
  s = ensure_atoms_device(sp, phi, st);
  if (s != LMA_OK) return s;
  if (force || sp->t_phonon[slot] != phi) {
    s = launch_t(sp, slot, phi, Rect{0, 0, g.nx, g.ny}, st);
    if (s != LMA_OK) return s;
    sp->t_phonon[slot] = phi;
    sp->t_stale[slot].clear();
    return LMA_OK;
  }
  for (const Rect& r : sp->t_stale[slot]) {
    s = launch_t(sp, slot, phi, r, st);
    if (s != LMA_OK) return s;
  }
  sp->t_stale[slot].clear();
  return LMA_OK;
}

// window x origin parity of list item (slot * nT + translate): (ox + a Sx - W/2) mod nx
bool origin_even(const lma_basis* b, int32_t item) {
  const int64_t i = item % b->nT;
  return ((b->ox + (i % b->nax) * b->Sx) & 1) == 0;
}

uint64_t hash_items(const std::vector<int32_t>& v) {
  uint64_t h = 1469598103934665603ull;   // FNV-1a over the items
  for (int32_t x : v) {
    h ^= static_cast<uint32_t>(x);
    h *= 1099511628211ull;
  }
  return h;
}

// device copy of an item list from the context's content-keyed cache; repeated
// batches and captured graphs never copy from host memory
constexpr size_t kListSlot = size_t(64) << 10;
constexpr int kListSlots = 16, kListOwned = 8;

lma_status upload_list(lma_ctx* ctx, const std::vector<int32_t>& list, cudaStream_t st, const int32_t** out) {
  const uint64_t h = hash_items(list);
  for (size_t k = 0; k < ctx->lists.size(); ++k) {
    lma_ctx::List& e = ctx->lists[k];
    if (e.used && e.hash == h && e.items == list) {
      if (ctx->capturing) ctx->capture_lists.emplace_back(e.p, h);
      *out = static_cast<const int32_t*>(e.p);
      if (!ctx->capturing) std::rotate(ctx->lists.begin() + k, ctx->lists.begin() + k + 1, ctx->lists.end());
      return LMA_OK;
    }
  }
  if (ctx->capturing) return fail(ctx, LMA_ERR_CUDA, "slice list not resident during graph capture");
  const size_t bytes = list.size() * sizeof(int32_t);
  if (!ctx->list_slab) {
    CUDA_TRY(ctx, counted_malloc(&ctx->list_slab, kListSlot * kListSlots));
    for (int k = 0; k < kListSlots; ++k) {
      lma_ctx::List e;
      e.p = static_cast<char*>(ctx->list_slab) + k * kListSlot;
      e.bytes = kListSlot;
      ctx->lists.insert(ctx->lists.begin(), std::move(e));
    }
  }
  // victim: the least recently used entry of the right kind (slab slot or own buffer)
  const bool small = bytes <= kListSlot;
  int n_owned = 0;
  for (const auto& e : ctx->lists) n_owned += e.owned ? 1 : 0;
  // (a long list gets a new buffer until kListOwned exist)
  auto victim = ctx->lists.end();
  if (small || n_owned >= kListOwned)
    for (auto it = ctx->lists.begin(); it != ctx->lists.end(); ++it)
      if (it->owned != small) {
        victim = it;
        break;
      }
  lma_ctx::List e;
  if (victim != ctx->lists.end()) {
    e = std::move(*victim);
    ctx->lists.erase(victim);
  }
  if (!small && e.bytes < bytes) {   // a new or too small own buffer
    if (e.p) CUDA_TRY(ctx, cudaFree(e.p));
    size_t cap = kListSlot * 2;
    while (cap < bytes) cap <<= 1;
    e.p = nullptr;
    e.bytes = 0;
    CUDA_TRY(ctx, counted_malloc(&e.p, cap));
    e.bytes = cap;
    e.owned = true;
  }
  CUDA_TRY(ctx, upload(ctx, e.p, list.data(), bytes, st));
  e.items = list;
  e.hash = h;
  e.used = true;
  *out = static_cast<const int32_t*>(e.p);
  ctx->lists.push_back(std::move(e));
  return LMA_OK;
}

// the work counter and the status word of the slice launches, zeroed once
lma_status ensure_counter(lma_ctx* ctx) {
  if (ctx->d_counter) return LMA_OK;
  CUDA_TRY(ctx, counted_malloc(reinterpret_cast<void**>(&ctx->d_counter), 2 * sizeof(int)));
  CUDA_TRY(ctx, cudaMemset(ctx->d_counter, 0, 2 * sizeof(int)));
  return LMA_OK;
}

// After a synchronizing read: did a slice launch with bounded waits (tensor-core or W = 256)
// give up one? (The status word is read only when such a launch ran since the last check.)
lma_status check_slice_status(lma_ctx* ctx) {
  if (!ctx->tc_launched || !ctx->d_counter) return LMA_OK;
  int st = 0;
  CUDA_TRY(ctx, cudaMemcpy(&st, ctx->d_counter + 1, sizeof(int), cudaMemcpyDeviceToHost));
  ctx->tc_launched = false;
  if (st != 0) {
    CUDA_TRY(ctx, cudaMemset(ctx->d_counter + 1, 0, sizeof(int)));
    return fail(ctx, LMA_ERR_TIMEOUT, "a slice launch gave up a bounded wait for its MMAs or bulk copies; results are invalid");
  }
  return LMA_OK;
}

// Probe geometry of a synthesis launch over a whole region (psx = 0: none, the grouped form
// does not apply).
struct SynthGeom {
  int psx = 0, psy = 0;        // probe spacing (pixels)
  int shift_abs = 0;           // largest |component| of the region's placements
};

SynthGeom region_geom(const lma_basis* b) {
  SynthGeom g;
  g.psx = b->reg.r.spacing_px[0];
  g.psy = b->reg.r.spacing_px[1];
  g.shift_abs = b->reg.shift_abs;
  return g;
}

// The two group shapes timed for L input waves per probe: up to 4 probes and 512
// (probe, wave) entries per group; 0 when no group of two probes fits.
int group_shapes(int L, int shapes[2][2]) {
  const int gmax = std::min(lma_dev::kGroupDenseProbes, lma_dev::kGroupMaxEntries / std::max(1, L));
  static const int cand[2][2][2] = {{{2, 2}, {4, 1}}, {{2, 1}, {1, 2}}};
  const int k = gmax >= 4 ? 0 : gmax >= 2 ? 1 : -1;
  if (k < 0) return 0;
  std::memcpy(shapes, cand[k], sizeof(cand[k]));
  return 2;
}

// Issue the synthesis of one launch shape in the tuned form, else the default: the gather with
// the default strip and grid, or the grouped form where it is forced and the launch admits it. With
// autotuning on and a shape not seen before, every variant runs once (each assigns the same
// readings) and is timed with events on the stream; the fastest is kept.
lma_status synth_launch(lma_ctx* ctx, lma_dev::SynthArgs& a, bool half, int mode, int64_t units, const SynthGeom& geo,
                        cudaStream_t st) {
  const bool listed = a.probe_list != nullptr;
  std::vector<int64_t> key{half ? 1 : 0, mode, listed ? 1 : 0, listed ? a.n_list : a.n_probes, a.npx, a.npy, a.n_cfg,
                           a.L, a.W, a.cyclic, geo.psx, geo.psy};
  // ---- the grouped form's admission: a whole region, non-periodic windows, placements that
  // fit the sort key, and a wave buffer (allocated here, outside a capture)
  int shapes[2][2] = {};
  bool admit[2] = {false, false};
  const int nsh = (!listed && !a.cyclic && geo.psx > 0 && geo.psy > 0 && a.n_translates < (1 << 30))
                      ? group_shapes(a.L, shapes) : 0;
  const int64_t row_bytes = static_cast<int64_t>(a.npx) * kW * kW * sizeof(float2);
  for (int i = 0; i < nsh; ++i) {
    const int gx = shapes[i][0], gy = shapes[i][1];
    admit[i] = (std::max(gx, gy) - 1) * std::max(geo.psx, geo.psy) + geo.shift_abs < lma_dev::kGroupPosBias &&
               gy * row_bytes <= ctx->psi_max;
  }
  auto psi_ready = [&](int gy) -> bool {
    const int64_t rows = std::min<int64_t>(a.npy, (ctx->psi_max / (gy * row_bytes)) * gy);
    const size_t need = static_cast<size_t>(rows * row_bytes);
    const int64_t n_tab = static_cast<int64_t>(a.npx) * a.npy;
    if (ctx->psi_bytes >= need && ctx->psi_tab_n >= n_tab) return true;
    if (ctx->capturing) return false;
    if (ctx->psi_bytes < need) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess || need > fr / 2) return false;
      if (ctx->psi) cudaFree(ctx->psi);
      ctx->psi = nullptr;
      ctx->psi_bytes = 0;
      if (counted_malloc(&ctx->psi, need) != cudaSuccess) return false;
      ctx->psi_bytes = need;
    }
    if (ctx->psi_tab_n < n_tab) {
      if (ctx->psi_tab) cudaFree(ctx->psi_tab);
      ctx->psi_tab = nullptr;
      ctx->psi_tab_n = 0;
      if (counted_malloc(&ctx->psi_tab, static_cast<size_t>(n_tab) * 20) != cudaSuccess) return false;
      char* t = static_cast<char*>(ctx->psi_tab);
      if (lma_dev::launch_identity_tables(static_cast<int>(n_tab), reinterpret_cast<int32_t*>(t + 16 * n_tab),
                                          reinterpret_cast<float2*>(t), reinterpret_cast<int2*>(t + 8 * n_tab),
                                          st) != cudaSuccess)
        return false;
      ctx->psi_tab_n = n_tab;
    }
    return true;
  };
  auto gather = [&](int strip, int grid) -> cudaError_t {
    a.strip = strip;
    return counted(ctx, K_SYNTH, units, st, [&] { return lma_dev::launch_synth(a, half, mode, grid, st); });
  };
  // grouped form: per configuration and chunk of group rows, the group launch writes the
  // chunk's probe waves and the detection pass (L = 1, identity tables, the chunk's probes
  // as a list of region indices) reads them out into the configuration's slot
  auto grouped = [&](int gx, int gy) -> cudaError_t {
    lma_dev::GroupArgs g{};
    g.gx = gx;
    g.gy = gy;
    g.psx = geo.psx;
    g.psy = geo.psy;
    g.ngx = (a.npx + gx - 1) / gx;
    const int ngy = (a.npy + gy - 1) / gy;
    const int cg = std::max<int>(1, static_cast<int>(ctx->psi_max / (gy * row_bytes)));
    g.gstrip = std::max(1, kSynthStrip / gx);
    g.psi = static_cast<float2*>(ctx->psi);
    const int64_t n_tab = ctx->psi_tab_n;
    const char* t = static_cast<const char*>(ctx->psi_tab);
    const int32_t* iota = reinterpret_cast<const int32_t*>(t + 16 * n_tab);
    const int64_t pat_size = static_cast<int64_t>(2 * a.pat_a + 1) * (2 * a.pat_b + 1);
    for (int c = 0; c < a.n_cfg; ++c) {
      for (int gr0 = 0; gr0 < ngy; gr0 += cg) {
        g.gb_base = gr0;
        g.ngy = std::min(cg, ngy - gr0);
        g.cfg = c;
        const int p0 = gr0 * gy * a.npx;
        const int p1 = std::min(a.npy, (gr0 + g.ngy) * gy) * a.npx;
        cudaError_t e = counted(ctx, K_SYNTH, 0, st, [&] { return lma_dev::launch_synth_group(a, g, half, lma_dev::kSynthGridAuto, st); });
        if (e != cudaSuccess) return e;
        lma_dev::SynthArgs d = a;
        d.U = static_cast<const float2*>(ctx->psi);
        d.Uh = nullptr;
        d.Uscale = nullptr;
        d.tidx = iota;
        d.alpha = reinterpret_cast<const float2*>(t);
        d.shift = reinterpret_cast<const int2*>(t + 8 * n_tab);
        d.L = 1;
        d.probe_list = iota + p0;
        d.n_list = p1 - p0;
        d.n_cfg = 1;
        d.cfg_base = a.cfg_base + c;
        d.n_translates = p1 - p0;
        d.u_slot = 0;
        d.W = kW;
        d.cyclic = 0;
        d.strip = kSynthStrip;
        if (a.pat) d.pat = a.pat + static_cast<int64_t>(c) * a.n_probes * pat_size;
        e = counted(ctx, K_SYNTH, static_cast<int64_t>(p1 - p0), st,
                    [&] { return lma_dev::launch_synth(d, false, mode, lma_dev::kSynthGridAuto, st); });
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  };
  const lma_ctx::SynthTune* tuned = nullptr;
  for (const auto& tt : ctx->synth_tune)
    if (tt.key == key) tuned = &tt;
  // untuned: the gather, unless the grouped form is forced (the gather is the faster of the
  // two on the benchmark: 3.7 ms per configuration against 4.5 + 0.9 ms)
  const bool want_group = ctx->synth_mode == LMA_SYNTH_GROUPED;
  if (tuned || !ctx->autotune || ctx->capturing) {
    if (ctx->synth_mode == LMA_SYNTH_AUTO && tuned) {
      const lma_synth_tuning& r = tuned->rec;
      if (r.grouped && psi_ready(r.group_y)) CUDA_TRY(ctx, grouped(r.group_x, r.group_y));
      else CUDA_TRY(ctx, gather(r.strip, r.persistent ? lma_dev::kSynthGridPersistent : lma_dev::kSynthGridPerItem));
    } else if (want_group && admit[0] && psi_ready(shapes[0][1])) {
      CUDA_TRY(ctx, grouped(shapes[0][0], shapes[0][1]));
    } else {
      CUDA_TRY(ctx, gather(kSynthStrip, lma_dev::kSynthGridAuto));
    }
    return LMA_OK;
  }
  static const int kStrips[3] = {16, 32, 64};
  lma_ctx::SynthTune tn;
  tn.key = key;
  tn.rec = lma_synth_tuning{};
  tn.rec.readout = mode == lma_dev::kReadAnnuli ? 0 : (mode == lma_dev::kReadLabels ? 1 : 2);
  tn.rec.half = half ? 1 : 0;
  tn.rec.n_items = static_cast<int64_t>(listed ? a.n_list : a.n_probes) * a.n_cfg;
  tn.rec.L = a.L;
  tn.rec.window = a.W;
  std::memcpy(tn.rec.group_shape, shapes, sizeof(shapes));
  cudaEvent_t ev[9];
  for (auto& e : ev) CUDA_TRY(ctx, cudaEventCreate(&e));
  cudaError_t err = cudaEventRecord(ev[0], st);
  int nv = 0;
  int var[8];
  for (int si = 0; si < 3 && err == cudaSuccess; ++si) {
    if (listed && si != 1) continue;   // a list is walked in order: the strip does not apply
    for (int g = 0; g < 2 && err == cudaSuccess; ++g) {
      err = gather(kStrips[si], g ? lma_dev::kSynthGridPersistent : lma_dev::kSynthGridPerItem);
      if (err == cudaSuccess) err = cudaEventRecord(ev[nv + 1], st);
      var[nv++] = 2 * si + g;
    }
  }
  for (int i = 0; i < nsh && err == cudaSuccess; ++i) {
    if (!admit[i] || !psi_ready(shapes[i][1])) continue;
    err = grouped(shapes[i][0], shapes[i][1]);
    if (err == cudaSuccess) err = cudaEventRecord(ev[nv + 1], st);
    var[nv++] = 6 + i;
  }
  if (err == cudaSuccess) err = cudaEventSynchronize(ev[nv]);
  int best = -1;
  for (int i = 0; i < nv && err == cudaSuccess; ++i) {
    float ms = 0.f;
    err = cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
    tn.rec.ms[var[i]] = ms;
    if (best < 0 || tn.rec.ms[var[i]] < tn.rec.ms[best]) best = var[i];
  }
  for (auto& e : ev) cudaEventDestroy(e);
  CUDA_TRY(ctx, err);
  if (best >= 6) {
    tn.rec.grouped = 1;
    tn.rec.group_x = shapes[best - 6][0];
    tn.rec.group_y = shapes[best - 6][1];
    tn.rec.strip = kSynthStrip;
    tn.rec.persistent = half ? 0 : 1;
  } else {
    tn.rec.strip = kStrips[best / 2];
    tn.rec.persistent = best % 2;
  }
  ctx->synth_tune.push_back(tn);
  return LMA_OK;
}

lma_dev::SliceJob make_job(const lma_basis* b, const lma_specimen* sp) {
  const lma_grid& g = sp->g;
  lma_dev::SliceJob J{};
  J.t = static_cast<const float2*>(sp->d_t.p);
  J.nx = g.nx;
  J.ny = g.ny;
  J.n_slices = g.n_slices;
  J.t_slot = t_slot_elems(g);
  J.uW = static_cast<const float2*>(b->d_uW.p);
  J.n_translates = static_cast<int>(b->nT);
  J.u_slot = static_cast<size_t>(b->nT) * b->W * b->W;
  J.lat_ox = b->ox;
  J.lat_oy = b->oy;
  J.lat_sx = b->Sx;
  J.lat_sy = b->Sy;
  J.lat_nax = b->nax;
  const bool half = b->desc.precision == LMA_PREC_FP16_STORE;
  J.U = half ? nullptr : static_cast<float2*>(b->d_U.p);
  J.Uh = half ? b->d_U.p : nullptr;
  J.Uscale = half ? static_cast<float*>(b->d_Uscale.p) : nullptr;
  J.ex = static_cast<const float2*>(b->d_ex.p);
  J.ey = static_cast<const float2*>(b->d_ey.p);
  J.r2max = b->r2max;
  J.tc_in = b->tc_in;
  J.tc_out = b->tc_out;
  J.W = b->W;
  return J;
}

// Issue one slice launch, in the forced, tuned or default mode. With autotuning on
// and a shape not seen before, every mode runs once (each writes the same exit
// waves) and is timed with events on the stream; the fastest is kept.
lma_status slice_launch(lma_ctx* ctx, const lma_dev::SliceLaunch& L0, bool even, int prec, int64_t units,
                        cudaStream_t st) {
  const bool half = prec == LMA_PREC_FP16_STORE;
  lma_dev::SliceLaunch L = L0;
  L.status = ctx->d_counter + 1;
  if (L.job[0].W != kW) {
    // W = 64 / 256 windows: k_slice_64 / k_slice_256 (complex64; the basis checks allow nothing else)
    const size_t need = lma_dev::slice_gen_scratch_bytes(L.job[0].W);
    if (need > ctx->gen_scratch_bytes) {
      if (ctx->capturing) return fail(ctx, LMA_ERR_CUDA, "slice scratch missing during graph capture");
      if (ctx->gen_scratch) cudaFree(ctx->gen_scratch);
      ctx->gen_scratch = nullptr;
      ctx->gen_scratch_bytes = 0;
      CUDA_TRY(ctx, counted_malloc(&ctx->gen_scratch, need));
      ctx->gen_scratch_bytes = need;
    }
    float2* scratch = static_cast<float2*>(ctx->gen_scratch);
    ctx->tc_launched = true;   // the status word is checked at the next synchronizing read
    CUDA_TRY(ctx, counted(ctx, K_SLICE, units, st, [&] { return lma_dev::launch_slice_gen(L, L.job[0].W, scratch, st); }));
    return LMA_OK;
  }
  if (prec == LMA_PREC_MIXED && ctx->rs_k1 == 0) {
    // tensor-core DFT passes: one persistent launch shape (no mode to tune)
    ctx->tc_launched = true;
    CUDA_TRY(ctx, counted(ctx, K_SLICE, units, st, [&] { return lma_dev::launch_slice_tc(L, even, st); }));
    return LMA_OK;
  }
  std::vector<int64_t> key{half ? 1 : 0, even ? 1 : 0, L.n_jobs, L.n_list};
  for (int j = 0; j < L.n_jobs; ++j) {
    key.push_back(L.job[j].nx);
    key.push_back(L.job[j].ny);
    key.push_back(L.job[j].n_slices);
    key.push_back(L.start[j + 1] - L.start[j]);
  }
  int mode = L.n_jobs > 1 ? lma_dev::kSliceDynamic : lma_dev::kSliceOnePerItem;
  bool tuned = false;
  for (const auto& t : ctx->tune)
    if (t.key == key) {
      mode = t.rec.mode;
      tuned = true;
    }
  if (ctx->forced_mode >= 0) mode = ctx->forced_mode;
  if (ctx->rs_k1 > 0) {
    CUDA_TRY(ctx, counted(ctx, K_SLICE, units, st,
                          [&] { return lma_dev::launch_slice_rs(L, ctx->rs_q, ctx->rs_k1, ctx->rs_k2, st); }));
    return LMA_OK;
  }
  auto launch = [&](int m) {
    return counted(ctx, K_SLICE, units, st, [&] { return lma_dev::launch_slice(L, even, half, m, st); });
  };
  if (tuned || ctx->forced_mode >= 0 || !ctx->autotune || ctx->capturing) {
    CUDA_TRY(ctx, launch(mode));
    return LMA_OK;
  }
  lma_ctx::Tune t;
  t.key = key;
  t.rec.n_jobs = L.n_jobs;
  t.rec.half = half ? 1 : 0;
  t.rec.even = even ? 1 : 0;
  t.rec.n_items = L.n_list;
  t.rec.translate_slices = units;
  cudaEvent_t ev[lma_dev::kSliceModes + 1];
  for (auto& e : ev) CUDA_TRY(ctx, cudaEventCreate(&e));
  cudaError_t err = cudaEventRecord(ev[0], st);
  for (int m = 0; m < lma_dev::kSliceModes && err == cudaSuccess; ++m) {
    err = launch(m);
    if (err == cudaSuccess) err = cudaEventRecord(ev[m + 1], st);
  }
  if (err == cudaSuccess) err = cudaEventSynchronize(ev[lma_dev::kSliceModes]);
  int best = 0;
  for (int m = 0; m < lma_dev::kSliceModes && err == cudaSuccess; ++m) {
    float ms = 0.f;
    err = cudaEventElapsedTime(&ms, ev[m], ev[m + 1]);
    t.rec.ms[m] = ms;
    if (t.rec.ms[m] < t.rec.ms[best]) best = m;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  CUDA_TRY(ctx, err);
  t.rec.mode = best;
  ctx->tune.push_back(t);
  return LMA_OK;
}

// The exit waves of several jobs (basis, specimen, items slot * nT + translate) in as
// few slice launches as the jobs allow: one per store precision and window-origin
// parity (and per kMaxJobs jobs). Marks the items current.
struct JobWork {
  lma_basis* b;
  lma_specimen* sp;
  std::vector<int32_t> items;
};

lma_status propagate_jobs(lma_ctx* ctx, std::vector<JobWork>& work, cudaStream_t st) {
  if (!ctx->d_counter) {
    if (ctx->capturing) return fail(ctx, LMA_ERR_CUDA, "work counter missing during graph capture");
    lma_status s0 = ensure_counter(ctx);
    if (s0 != LMA_OK) return s0;
  }
  for (int gk = 0; gk < 9; ++gk) {
    // one group per store precision and window
    const int prec = gk / 3, wsize = 64 << (gk % 3);
    std::vector<JobWork*> group;
    for (JobWork& w : work)
      if (!w.items.empty() && w.b->desc.precision == prec && w.b->W == wsize) group.push_back(&w);
    for (size_t c0 = 0; c0 < group.size(); c0 += lma_dev::kMaxJobs) {
      const int nj = static_cast<int>(std::min<size_t>(lma_dev::kMaxJobs, group.size() - c0));
      for (int part = 0; part < 2; ++part) {
        const bool even = part == 0;
        lma_dev::SliceLaunch L{};
        std::vector<int32_t> list;
        int64_t units = 0;
        L.n_jobs = nj;
        for (int j = 0; j < nj; ++j) {
          const JobWork& w = *group[c0 + j];
          L.job[j] = make_job(w.b, w.sp);
          L.start[j] = static_cast<int>(list.size());
          for (int32_t i : w.items)
            if (origin_even(w.b, i) == even) list.push_back(i);
          units += static_cast<int64_t>(list.size() - L.start[j]) * w.sp->g.n_slices;
        }
        L.start[nj] = static_cast<int>(list.size());
        if (list.empty()) continue;
        if (list.size() > static_cast<size_t>(INT32_MAX)) return fail(ctx, LMA_ERR_UNSUPPORTED, "slice list too long");
        lma_status s = upload_list(ctx, list, st, &L.list);
        if (s != LMA_OK) return s;
        L.n_list = static_cast<int>(list.size());
        L.counter = ctx->d_counter;
        if ((s = slice_launch(ctx, L, even, prec, units, st)) != LMA_OK) return s;
      }
    }
  }
  for (JobWork& w : work)
    for (int32_t i : w.items) w.b->valid[i] = 1;
  return LMA_OK;
}

// Make configurations [phi0, phi0 + nb) of one basis ready to propagate on the needed
// translates: transmissions current in their slots; the translates whose exit waves
// are not current are returned as items. Slots [0, nb), or slot phi when every
// configuration has its own slot (then stored waves are reused across calls).
lma_status prepare_batch(lma_basis* b, lma_specimen* sp, int phi0, int nb, const std::vector<uint8_t>& needed,
                         bool recompute, cudaStream_t st, std::vector<int32_t>* items) {
  const int nph = static_cast<int>(sp->ph.size());
  const bool own = b->B >= nph;
  if (b->U_epoch != sp->epoch) {
    // atoms replaced, or edited through another basis: nothing stored is current
    std::fill(b->valid.begin(), b->valid.end(), 0);
    std::fill(b->U_phonon.begin(), b->U_phonon.end(), -1);
    b->U_epoch = sp->epoch;
  }
  lma_status s = reserve_t_slots(sp, b->B);
  if (s != LMA_OK) return s;
  for (int j = 0; j < nb; ++j) {
    const int phi = phi0 + j;
    const int slot = own ? phi : j;
    uint8_t* v = b->valid.data() + static_cast<size_t>(slot) * b->nT;
    if (recompute || b->U_phonon[slot] != phi) {
      std::fill(v, v + b->nT, 0);
      b->U_phonon[slot] = phi;
    }
    const size_t before = items->size();
    for (int64_t i = 0; i < b->nT; ++i)
      if (needed[i] && !v[i]) items->push_back(static_cast<int32_t>(slot * b->nT + i));
    if (items->size() > before && (s = ensure_t(sp, slot, phi, recompute, st)) != LMA_OK) return s;
  }
  return LMA_OK;
}

lma_status ensure_batch(lma_basis* b, lma_specimen* sp, int phi0, int nb, const std::vector<uint8_t>& needed,
                        bool recompute, cudaStream_t st) {
  std::vector<JobWork> work(1);
  work[0].b = b;
  work[0].sp = sp;
  lma_status s = prepare_batch(b, sp, phi0, nb, needed, recompute, st, &work[0].items);
  if (s != LMA_OK) return s;
  return propagate_jobs(b->ctx, work, st);
}

// Probe tables of a region on the host: for probe p = b * npx + a and j < L, the translate
// index of its j-th input wave, its coefficient (complex64) and its window placement.
// A probe's table entries in ascending translate index (translate, index into the coefficient
// set): the order in which both synthesis forms sum them. Every table of per-probe coefficients
// (the region's, the coherence variants') follows it.
void entry_order(const lma_basis* b, int px, int py, const CoefSet& cs, std::vector<std::pair<int32_t, int>>& order) {
  const int L = b->desc.L;
  order.resize(L);
  for (int j = 0; j < L; ++j)
    order[j] = {static_cast<int32_t>(translate_index(b, px + cs.odx[j], py + cs.ody[j])), j};
  std::sort(order.begin(), order.end());
}

lma_status region_tables_host(lma_basis* b, const lma_region* r, std::vector<int32_t>& tidx,
                              std::vector<float>& al, std::vector<int32_t>& sh) {
  const int L = b->desc.L;
  const int64_t np = static_cast<int64_t>(r->npx) * r->npy;
  tidx.assign(static_cast<size_t>(np) * L, 0);
  al.assign(2 * static_cast<size_t>(np) * L, 0.f);
  sh.assign(2 * static_cast<size_t>(np) * L, 0);
  const int half = (b->desc.det_window - b->desc.window) / 2;
  for (int pb = 0; pb < r->npy; ++pb) {
    for (int pa = 0; pa < r->npx; ++pa) {
      const int px = mod(r->px0 + pa * r->spacing_px[0], b->nx);
      const int py = mod(r->py0 + pb * r->spacing_px[1], b->ny);
      const CoefSet* cs = nullptr;
      lma_status s = coef_set(b, px, py, &cs);
      if (s != LMA_OK) return s;
      const size_t base = (static_cast<size_t>(pb) * r->npx + pa) * L;
      std::vector<std::pair<int32_t, int>> order;
      entry_order(b, px, py, *cs, order);
      for (int i = 0; i < L; ++i) {
        const int j = order[i].second;
        tidx[base + i] = order[i].first;
        al[2 * (base + i)] = static_cast<float>(cs->alpha[j].real());
        al[2 * (base + i) + 1] = static_cast<float>(cs->alpha[j].imag());
        sh[2 * (base + i)] = cs->odx[j] + half;
        sh[2 * (base + i) + 1] = cs->ody[j] + half;
      }
    }
  }
  return LMA_OK;
}

lma_status build_region(lma_basis* b, const lma_region* r, cudaStream_t st) {
  lma_ctx* ctx = b->ctx;
  if (b->reg_valid && std::memcmp(&b->reg.r, r, sizeof(lma_region)) == 0) return LMA_OK;
  const int64_t np = static_cast<int64_t>(r->npx) * r->npy;
  std::vector<int32_t> tidx, sh;
  std::vector<float> al;
  lma_status s0 = region_tables_host(b, r, tidx, al, sh);
  if (s0 != LMA_OK) return s0;
  RegionTables& R = b->reg;
  R.needed.assign(static_cast<size_t>(b->nT), 0);
  for (int32_t i : tidx) R.needed[i] = 1;
  CUDA_TRY(ctx, ensure(R.tidx, tidx.size() * sizeof(int32_t)));
  CUDA_TRY(ctx, ensure(R.alpha, al.size() * sizeof(float)));
  CUDA_TRY(ctx, ensure(R.shift, sh.size() * sizeof(int32_t)));
  CUDA_TRY(ctx, upload_parts(ctx, {HostPart{R.tidx.p, tidx.data(), tidx.size() * sizeof(int32_t)},
                                    HostPart{R.alpha.p, al.data(), al.size() * sizeof(float)},
                                    HostPart{R.shift.p, sh.data(), sh.size() * sizeof(int32_t)}},
                             st));
  R.r = *r;
  R.n_probes = np;
  R.shift_abs = 0;
  for (int32_t v : sh) R.shift_abs = std::max(R.shift_abs, v < 0 ? -v : v);
  R.h_tidx.swap(tidx);
  b->reg_valid = true;
  return LMA_OK;
}

// Detector bits in the C layout of the synthesis kernel: word T = kx + 128 k1y, bit j <-> ky =
// k1y + 4 j; bit set where r1 <= lambda |k| < r2 inside the bandlimit (decided in FP64).
void detector_bits_host(const lma_basis* b, const lma_detector* det, int n_det, std::vector<uint32_t>& bits) {
  const lma_grid& g = b->spec->g;
  const int D = b->desc.det_window;
  const double dx = g.lx / g.nx, dy = g.ly / g.ny, lam = g.lambda, frac = g.bandlimit_frac;
  bits.assign(static_cast<size_t>(n_det) * lma_dev::kThreads, 0u);
  for (int d = 0; d < n_det; ++d) {
    for (int iy = 0; iy < D; ++iy) {
      const int my = signed_index(iy, D);
      const double ky = my / (D * dy);
      for (int ix = 0; ix < D; ++ix) {
        const int mx = signed_index(ix, D);
        const double kx = mx / (D * dx);
        const double ang = lam * std::sqrt(ky * ky + kx * kx);
        const bool band = static_cast<double>(4 * (my * my + mx * mx)) <= frac * frac * D * D;
        if (ang >= det[d].r1 && ang < det[d].r2 && band) {
          const int k1y = iy & 3, j = iy >> 2;
          bits[static_cast<size_t>(d) * lma_dev::kThreads + ix + 128 * k1y] |= 1u << j;
        }
      }
    }
  }
}

lma_status build_detectors(lma_basis* b, const lma_detector* det, int n_det, cudaStream_t st) {
  lma_ctx* ctx = b->ctx;
  std::vector<double> key;
  for (int d = 0; d < n_det; ++d) {
    key.push_back(det[d].r1);
    key.push_back(det[d].r2);
  }
  if (b->d_det.p && key == b->det_key) return LMA_OK;
  std::vector<uint32_t> bits;
  detector_bits_host(b, det, n_det, bits);
  CUDA_TRY(ctx, ensure(b->d_det, bits.size() * sizeof(uint32_t)));
  CUDA_TRY(ctx, upload(ctx, b->d_det.p, bits.data(), bits.size() * sizeof(uint32_t), st));
  b->det_key = key;
  return LMA_OK;
}

// 3D STEM ring labels on the D x D detection window: ring a holds the pixels with
// a * width <= lambda |k| < (a + 1) * width inside the bandlimit, decided in FP64 with the
// operation order of the 2D detector. Device table: [n_rings + 1] CSR starts, then the
// pixel indices iy * D + ix of each ring in ascending order.
lma_status build_labels(lma_basis* b, double width, int n_rings, cudaStream_t st) {
  lma_ctx* ctx = b->ctx;
  const std::vector<double> key{width, static_cast<double>(n_rings)};
  if (b->d_lab.p && key == b->lab_key) return LMA_OK;
  const lma_grid& g = b->spec->g;
  const int D = b->desc.det_window;
  const double dx = g.lx / g.nx, dy = g.ly / g.ny, lam = g.lambda, frac = g.bandlimit_frac;
  std::vector<std::vector<int32_t>> ring(n_rings);
  for (int iy = 0; iy < D; ++iy) {
    const int my = signed_index(iy, D);
    const double ky = my / (D * dy);
    for (int ix = 0; ix < D; ++ix) {
      const int mx = signed_index(ix, D);
      const double kx = mx / (D * dx);
      const double ang = lam * std::sqrt(ky * ky + kx * kx);
      const bool band = static_cast<double>(4 * (my * my + mx * mx)) <= frac * frac * D * D;
      if (!band) continue;
      for (int a = 0; a < n_rings; ++a)
        if (ang >= a * width && ang < (a + 1) * width) {
          ring[a].push_back(iy * D + ix);
          break;
        }
    }
  }
  std::vector<int32_t> table(static_cast<size_t>(n_rings) + 1, 0);
  for (int a = 0; a < n_rings; ++a) table[a + 1] = table[a] + static_cast<int32_t>(ring[a].size());
  for (int a = 0; a < n_rings; ++a) table.insert(table.end(), ring[a].begin(), ring[a].end());
  CUDA_TRY(ctx, ensure(b->d_lab, table.size() * sizeof(int32_t)));
  CUDA_TRY(ctx, upload(ctx, b->d_lab.p, table.data(), table.size() * sizeof(int32_t), st));
  b->lab_key = key;
  return LMA_OK;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// device -> host result copy: straight into pinned memory, else through the staging buffer
cudaError_t read_back(lma_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeHost) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
    return e != cudaSuccess ? e : cudaStreamSynchronize(st);
  }
  cudaGetLastError();
  return download(ctx, dst, src, bytes, st);
}

}  // namespace

namespace {

// Device work of the images of several (basis, specimen) pairs (steps a1, a3-a6).
// Configurations go in passes: pass r takes each pair's r-th phonon batch; the
// slice work of all pairs in a pass is one launch (per precision and origin
// parity), then each pair's batch is synthesized into its accumulator slots.
// After the last pass each pair's average goes to its dev_out (or, when that is
// null, to the accumulator's last slot). Needs build_region / build_detectors done.
struct ImageJob {
  lma_basis* b;
  lma_specimen* sp;
  void* dev_out;   // double (annuli, labels) or float (pattern); null: into the basis
};

// what the synthesis kernel reads out of each probe's diffraction plane
struct Readout {
  int mode = lma_dev::kReadAnnuli;
  int n_out = 0;                 // annuli or labels per probe
  int pat_a = 0, pat_b = 0;      // pattern half-widths (4D STEM)
  int64_t pat_size() const { return static_cast<int64_t>(2 * pat_a + 1) * (2 * pat_b + 1); }
};

// results of images_work left in the basis when a job has no device output
const double* basis_result(const lma_basis* b, const lma_specimen* sp, int n_out) {
  return static_cast<const double*>(b->d_acc.p) + sp->ph.size() * static_cast<size_t>(b->reg.n_probes * n_out);
}

lma_status images_work(lma_ctx* ctx, const std::vector<ImageJob>& jobs, const Readout& ro, bool recompute,
                       cudaStream_t st) {
  const bool pattern = ro.mode == lma_dev::kReadPattern;
  int passes = 0;
  for (const ImageJob& J : jobs) {
    const int nph = static_cast<int>(J.sp->ph.size());
    const int64_t np = J.b->reg.n_probes;
    if (pattern) {
      const size_t n = static_cast<size_t>(np) * ro.pat_size();
      CUDA_TRY(ctx, ensure(J.b->d_pat, n * J.b->B * sizeof(float)));
      CUDA_TRY(ctx, ensure(J.b->d_pat_acc, n * sizeof(double)));
    } else {
      // one slot per configuration plus one for the average
      CUDA_TRY(ctx, ensure(J.b->d_acc, static_cast<size_t>(np * ro.n_out) * (nph + 1) * sizeof(double)));
    }
    passes = std::max(passes, (nph + J.b->B - 1) / J.b->B);
  }
  lma_status s;
  for (int r = 0; r < passes; ++r) {
    std::vector<JobWork> work;
    std::vector<std::pair<int, int>> batch;   // (phi0, nb) per job in this pass
    for (const ImageJob& J : jobs) {
      const int nph = static_cast<int>(J.sp->ph.size());
      const int phi0 = r * J.b->B;
      const int nb = phi0 < nph ? std::min(J.b->B, nph - phi0) : 0;
      batch.emplace_back(phi0, nb);
      work.push_back(JobWork{J.b, J.sp, {}});
      if (nb > 0 &&
          (s = prepare_batch(J.b, J.sp, phi0, nb, J.b->reg.needed, recompute, st, &work.back().items)) != LMA_OK)
        return s;
    }
    if ((s = propagate_jobs(ctx, work, st)) != LMA_OK) return s;
    for (size_t k = 0; k < jobs.size(); ++k) {
      const int nb = batch[k].second;
      if (nb == 0) continue;
      lma_basis* b = jobs[k].b;
      const bool half = b->desc.precision == LMA_PREC_FP16_STORE;
      const int64_t np = b->reg.n_probes;
      lma_dev::SynthArgs a{};
      a.U = half ? nullptr : static_cast<const float2*>(b->d_U.p);
      a.Uh = half ? b->d_U.p : nullptr;
      a.Uscale = half ? static_cast<const float*>(b->d_Uscale.p) : nullptr;
      a.tidx = static_cast<const int32_t*>(b->reg.tidx.p);
      a.alpha = static_cast<const float2*>(b->reg.alpha.p);
      a.shift = static_cast<const int2*>(b->reg.shift.p);
      a.L = b->desc.L;
      a.n_probes = static_cast<int>(np);
      a.npx = b->reg.r.npx;
      a.npy = b->reg.r.npy;
      a.strip = kSynthStrip;
      a.n_cfg = nb;
      a.cfg_base = batch[k].first;
      a.n_translates = static_cast<int>(b->nT);
      a.u_slot = static_cast<size_t>(b->nT) * b->W * b->W;
      a.cyclic = (b->W == kW && b->nx == kW && b->ny == kW) ? 1 : 0;
      a.W = b->W;
      a.det_bits = static_cast<const uint32_t*>(b->d_det.p);
      a.n_det = ro.n_out;
      a.acc = static_cast<double*>(b->d_acc.p);
      a.band_r2 = b->r2max;
      if (ro.mode == lma_dev::kReadLabels) {
        a.lab_start = static_cast<const int32_t*>(b->d_lab.p);
        a.lab_pix = a.lab_start + ro.n_out + 1;
      }
      if (pattern) {
        a.pat = static_cast<float*>(b->d_pat.p);
        a.pat_a = ro.pat_a;
        a.pat_b = ro.pat_b;
      }
      { const lma_status ss_ = synth_launch(ctx, a, half, ro.mode, np * nb, region_geom(b), st); if (ss_ != LMA_OK) return ss_; }
      if (pattern) {
        const int64_t n = np * ro.pat_size();
        CUDA_TRY(ctx, counted(ctx, K_FIN, n, st, [&] {
          return lma_dev::launch_pattern_accumulate(static_cast<const float*>(b->d_pat.p), n, nb,
                                                    batch[k].first == 0, static_cast<double*>(b->d_pat_acc.p), st);
        }));
      }
    }
  }
  for (const ImageJob& J : jobs) {
    const int nph = static_cast<int>(J.sp->ph.size());
    if (pattern) {
      const int64_t n = J.b->reg.n_probes * ro.pat_size();
      float* fin = J.dev_out ? static_cast<float*>(J.dev_out) : static_cast<float*>(J.b->d_pat.p);
      CUDA_TRY(ctx, counted(ctx, K_FIN, n, st, [&] {
        return lma_dev::launch_pattern_finalize(static_cast<const double*>(J.b->d_pat_acc.p), n, 1.0 / nph, fin, st);
      }));
      continue;
    }
    const int64_t nout = J.b->reg.n_probes * ro.n_out;
    const double* acc = static_cast<const double*>(J.b->d_acc.p);
    double* fin = J.dev_out ? static_cast<double*>(J.dev_out) : const_cast<double*>(basis_result(J.b, J.sp, ro.n_out));
    CUDA_TRY(ctx, counted(ctx, K_FIN, nout, st,
                          [&] { return lma_dev::launch_finalize(acc, nout, nph, 1.0 / nph, fin, st); }));
  }
  return LMA_OK;
}

lma_status image_work(lma_basis* b, lma_specimen* sp, int n_det, bool recompute, double* dev_out,
                      cudaStream_t st) {
  Readout ro;
  ro.n_out = n_det;
  return images_work(b->ctx, {ImageJob{b, sp, dev_out}}, ro, recompute, st);
}

// slice launches of one API call time their modes (LMA_IMAGE_AUTOTUNE)
struct AutotuneScope {
  lma_ctx* c;
  AutotuneScope(lma_ctx* c_, bool on) : c(c_) { c->autotune = on; }
  ~AutotuneScope() { c->autotune = false; }
};

// validate and slice-sort the atom lists of every configuration into sp->ph
lma_status load_atoms(lma_ctx* ctx, lma_specimen* sp, const lma_atoms* phonons, int n_phonons) {
  const lma_grid& g = sp->g;
  const int n_species = static_cast<int>(sp->peak.size());
  std::vector<PhononSet> ph(n_phonons);
  for (int f = 0; f < n_phonons; ++f) {
    const lma_atoms& A = phonons[f];
    if (A.n_atoms < 0 || (A.n_atoms > 0 && (!A.x || !A.y || !A.slice || !A.species)))
      return fail(ctx, LMA_ERR_INVALID, "atoms %d: null arrays", f);
    if (A.n_atoms > (1ll << 31) - 1) return fail(ctx, LMA_ERR_INVALID, "atoms %d: too many atoms", f);
    std::vector<int64_t> order(static_cast<size_t>(A.n_atoms));
    for (int64_t k = 0; k < A.n_atoms; ++k) {
      order[k] = k;
      if (A.slice[k] < 0 || A.slice[k] >= g.n_slices || A.species[k] < 0 || A.species[k] >= n_species ||
          !std::isfinite(A.x[k]) || !std::isfinite(A.y[k]))
        return fail(ctx, LMA_ERR_INVALID,
                    "atoms %d: atom %lld has slice/species out of range or a non-finite position", f,
                    static_cast<long long>(k));
    }
    std::stable_sort(order.begin(), order.end(), [&](int64_t u, int64_t v) { return A.slice[u] < A.slice[v]; });
    PhononSet& P = ph[f];
    P.x.resize(order.size());
    P.y.resize(order.size());
    P.sp.resize(order.size());
    P.slc.resize(order.size());
    // positions are kept in [0, l): the potential kernel then finds every minimum image
    // with one comparison per axis
    for (size_t k = 0; k < order.size(); ++k) {
      P.x[k] = wrap_period(A.x[order[k]], g.lx);
      P.y[k] = wrap_period(A.y[order[k]], g.ly);
      P.sp[k] = A.species[order[k]];
      P.slc[k] = A.slice[order[k]];
    }
    P.slice_start.assign(g.n_slices + 1, 0);
    for (int32_t s : P.slc) P.slice_start[s + 1]++;
    for (int s = 0; s < g.n_slices; ++s) P.slice_start[s + 1] += P.slice_start[s];
  }
  if (sp->ph.empty()) {
    sp->ph.swap(ph);
    return LMA_OK;
  }
  // keep the device buffers, replace the host lists
  for (int f = 0; f < n_phonons; ++f) {
    PhononSet& P = sp->ph[f];
    P.x.swap(ph[f].x);
    P.y.swap(ph[f].y);
    P.sp.swap(ph[f].sp);
    P.slc.swap(ph[f].slc);
    P.slice_start.swap(ph[f].slice_start);
    P.dirty = true;
  }
  return LMA_OK;
}

}  // namespace

// =============================================================================================
// C-ABI
// =============================================================================================
extern "C" {

lma_status lma_create(int32_t device, lma_ctx** out) {
  if (!out) return LMA_ERR_INVALID;
  lma_ctx* c = new (std::nothrow) lma_ctx();
  if (!c) return LMA_ERR_OOM;
  c->device = device;
  c->host_only = device < 0;
  if (!c->host_only) {
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = lma_dev::init_device_constants();
    if (e != cudaSuccess) {
      delete c;
      return LMA_ERR_CUDA;
    }
  }
  *out = c;
  return LMA_OK;
}

void lma_destroy(lma_ctx* ctx) {
  if (!ctx) return;
  for (auto& g : ctx->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  for (auto& l : ctx->lists)
    if (l.owned && l.p) cudaFree(l.p);
  if (ctx->list_slab) cudaFree(ctx->list_slab);
  if (ctx->d_counter) cudaFree(ctx->d_counter);
  if (ctx->gen_scratch) cudaFree(ctx->gen_scratch);
  if (ctx->psi) cudaFree(ctx->psi);
  if (ctx->psi_tab) cudaFree(ctx->psi_tab);
  if (ctx->stage) cudaFreeHost(ctx->stage);
  delete ctx;
}

const char* lma_last_error(const lma_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

lma_status lma_create_specimen(lma_ctx* ctx, const lma_grid* grid, const lma_potential* pot,
                               const lma_atoms* phonons, int32_t n_phonons, lma_specimen** out) {
  if (!ctx || !grid || !pot || !out || (n_phonons > 0 && !phonons))
    return fail(ctx, LMA_ERR_INVALID, "null argument");
  const lma_grid& g = *grid;
  if (g.nx <= 0 || g.ny <= 0 || !(g.lx > 0) || !(g.ly > 0) || !(g.slice_dz > 0) || g.n_slices <= 0 ||
      !(g.lambda > 0) || !(g.sigma >= 0) || !(g.bandlimit_frac > 0) || g.bandlimit_frac > 1.0)
    return fail(ctx, LMA_ERR_INVALID, "grid: non-positive size, thickness, wavelength or bandlimit");
  if (g.nx % 16 || g.ny % 16) return fail(ctx, LMA_ERR_UNSUPPORTED, "grid sizes must be multiples of 16");
  if (n_phonons <= 0) return fail(ctx, LMA_ERR_INVALID, "need at least one configuration");
  if (pot->n_species <= 0 || !pot->peak || pot->n_terms < 1 || pot->n_terms > lma_dev::kMaxTerms ||
      !pot->term_frac || !pot->term_width)
    return fail(ctx, LMA_ERR_INVALID, "potential: bad species or term count");
  if (!(pot->r_cut > 0) || pot->r_cut >= 0.5 * std::min(g.lx, g.ly))
    return fail(ctx, LMA_ERR_INVALID, "potential: r_cut must be in (0, min(lx, ly)/2)");
  for (int q = 0; q < pot->n_terms; ++q)
    if (!(pot->term_width[q] > 0)) return fail(ctx, LMA_ERR_INVALID, "potential: width <= 0");
  lma_specimen* sp = new (std::nothrow) lma_specimen();
  if (!sp) return fail(ctx, LMA_ERR_OOM, "host allocation");
  sp->ctx = ctx;
  sp->g = g;
  sp->peak.assign(pot->peak, pot->peak + pot->n_species);
  sp->frac.assign(pot->term_frac, pot->term_frac + pot->n_terms);
  sp->width.assign(pot->term_width, pot->term_width + pot->n_terms);
  sp->r_cut = pot->r_cut;
  lma_status st = load_atoms(ctx, sp, phonons, n_phonons);
  if (st != LMA_OK) {
    delete sp;
    return st;
  }
  *out = sp;
  return LMA_OK;
}

lma_status lma_specimen_set_atoms(lma_ctx* ctx, lma_specimen* sp, const lma_atoms* phonons, int32_t n_phonons) {
  if (!ctx || !sp || !phonons) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (n_phonons != static_cast<int>(sp->ph.size()))
    return fail(ctx, LMA_ERR_INVALID, "configuration count differs from the specimen's");
  lma_status st = load_atoms(ctx, sp, phonons, n_phonons);
  if (st != LMA_OK) return st;
  std::fill(sp->t_phonon.begin(), sp->t_phonon.end(), -1);
  for (auto& v : sp->t_stale) v.clear();
  sp->epoch++;
  return LMA_OK;
}

lma_status lma_free_specimen(lma_specimen* sp) {
  if (!sp) return LMA_ERR_INVALID;
  for (PhononSet& p : sp->ph) {
    p.dx.release();
    p.dy.release();
    p.dsp.release();
    p.dss.release();
  }
  sp->d_peak.release();
  sp->d_t.release();
  delete sp;
  return LMA_OK;
}

lma_status lma_transmission(lma_ctx* ctx, lma_specimen* sp, int32_t phonon, float* out, void* stream) {
  if (!ctx || !sp || !out) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (phonon < 0 || phonon >= static_cast<int>(sp->ph.size()))
    return fail(ctx, LMA_ERR_INVALID, "phonon index out of range");
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lma_status s = ensure_t(sp, 0, phonon, false, st);
  if (s != LMA_OK) return s;
  const lma_grid& g = sp->g;
  const bool dev = is_device_pointer(out);
  const size_t pitch = static_cast<size_t>(g.nx + kW) * sizeof(float2);
  const size_t slice = pitch * (g.ny + kW);
  for (int s2 = 0; s2 < g.n_slices; ++s2) {
    CUDA_TRY(ctx, cudaMemcpy2DAsync(reinterpret_cast<char*>(out) + static_cast<size_t>(s2) * g.nx * g.ny * sizeof(float2),
                                    static_cast<size_t>(g.nx) * sizeof(float2),
                                    static_cast<const char*>(sp->d_t.p) + s2 * slice, pitch,
                                    static_cast<size_t>(g.nx) * sizeof(float2), g.ny,
                                    dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  if (!dev) {
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return check_slice_status(ctx);
  }
  return LMA_OK;
}

lma_status lma_create_basis(lma_ctx* ctx, const lma_specimen* spec, const lma_probe* probe,
                            const lma_basis_desc* desc, lma_basis** out) {
  if (!ctx || !spec || !probe || !desc || !out) return fail(ctx, LMA_ERR_INVALID, "null argument");
  const lma_grid& g = spec->g;
  const lma_basis_desc& d = *desc;
  if (d.window != 64 && d.window != 128 && d.window != 256)
    return fail(ctx, LMA_ERR_UNSUPPORTED, "window must be 64, 128 or 256 pixels");
  if (d.det_window != kW) return fail(ctx, LMA_ERR_UNSUPPORTED, "det_window (the detection window D) must be %d", kW);
  if (g.nx < std::max(d.window, kW) || g.ny < std::max(d.window, kW))
    return fail(ctx, LMA_ERR_UNSUPPORTED, "grid smaller than the window or than the detection window");
  if (!is_pow2(g.nx) || !is_pow2(g.ny)) return fail(ctx, LMA_ERR_UNSUPPORTED, "grid sizes must be powers of two");
  if (d.kind != LMA_BASIS_GAUSS && d.kind != LMA_BASIS_PROBE && d.kind != LMA_BASIS_TRIG &&
      d.kind != LMA_BASIS_TRIG_RADIAL)
    return fail(ctx, LMA_ERR_INVALID, "unknown input wave kind");
  if (d.trig_degree < 0 || d.trig_degree > 4096) return fail(ctx, LMA_ERR_INVALID, "trig_degree must be in [0, 4096]");
  if (d.coef_mode != LMA_COEF_LSQ && d.coef_mode != LMA_COEF_TRIG_CLOSED)
    return fail(ctx, LMA_ERR_INVALID, "coef_mode must be LMA_COEF_LSQ or LMA_COEF_TRIG_CLOSED");
  if (d.coef_mode == LMA_COEF_TRIG_CLOSED && d.kind != LMA_BASIS_TRIG)
    return fail(ctx, LMA_ERR_INVALID, "closed-form coefficients need the tensor trigonometric input waves (LMA_BASIS_TRIG)");
  if (d.precision != LMA_PREC_C64 && d.precision != LMA_PREC_FP16_STORE && d.precision != LMA_PREC_MIXED)
    return fail(ctx, LMA_ERR_INVALID, "precision must be LMA_PREC_C64, LMA_PREC_FP16_STORE or LMA_PREC_MIXED");
  if (!(probe->alpha_max > 0)) return fail(ctx, LMA_ERR_INVALID, "alpha_max must be positive");
  const int sx = d.in_spacing_px[0], sy = d.in_spacing_px[1];
  if (sx <= 0 || sy <= 0 || g.nx % sx || g.ny % sy)
    return fail(ctx, LMA_ERR_INVALID, "input lattice spacing must divide the grid");
  if (d.in_offset_px[0] < 0 || d.in_offset_px[0] >= sx || d.in_offset_px[1] < 0 || d.in_offset_px[1] >= sy)
    return fail(ctx, LMA_ERR_INVALID, "input lattice offset must lie in [0, spacing)");
  if (d.f <= 0 || (g.nx / sx) % d.f || (g.ny / sy) % d.f)
    return fail(ctx, LMA_ERR_INVALID, "f must divide the number of input waves per axis");
  const int64_t nT = static_cast<int64_t>(g.nx / sx / d.f) * (g.ny / sy / d.f);
  if (d.L <= 0 || d.L > kMaxL || d.L > nT)
    return fail(ctx, LMA_ERR_INVALID, "L must be in [1, min(|I_f|, %d)]", kMaxL);
  if (nT > (1ll << 31) - 1) return fail(ctx, LMA_ERR_INVALID, "too many input waves");
  const int trig_n = d.trig_degree > 0 ? d.trig_degree : static_cast<int>(std::lround(probe->alpha_max * g.lx / g.lambda));
  if (d.coef_mode == LMA_COEF_TRIG_CLOSED &&
      (g.nx / (sx * d.f) < 2 * trig_n + 1 || g.ny / (sy * d.f) < 2 * trig_n + 1))
    return fail(ctx, LMA_ERR_INVALID,
                "closed-form coefficients need at least 2n + 1 = %d input waves per axis (I_f has %d x %d)",
                2 * trig_n + 1, g.nx / (sx * d.f), g.ny / (sy * d.f));
  lma_basis* b = new (std::nothrow) lma_basis();
  if (!b) return fail(ctx, LMA_ERR_OOM, "host allocation");
  b->ctx = ctx;
  b->spec = spec;
  b->probe = *probe;
  b->desc = d;
  b->gauss_sigma = d.gauss_sigma > 0 ? d.gauss_sigma : g.lambda / (2.0 * probe->alpha_max);
  b->nx = g.nx;
  b->ny = g.ny;
  b->Sx = sx * d.f;
  b->Sy = sy * d.f;
  b->ox = d.in_offset_px[0];
  b->oy = d.in_offset_px[1];
  b->nax = g.nx / b->Sx;
  b->nay = g.ny / b->Sy;
  b->nT = nT;
  b->trig_n = trig_n;
  b->W = d.window;
  build_input_wave(b);
  {
    // tensor-core DFT passes: a power of two bringing the input wave's norm into (2^10, 2^11],
    // times the 2^7 that each transmission takes back (the propagator carries 2^-7, not 1/W^2)
    double n2 = 0.0;
    for (const cd& z : b->uW) n2 += std::norm(z);
    const int e = n2 > 0.0 ? static_cast<int>(std::ceil(0.5 * std::log2(n2))) : 0;
    b->tc_in = std::ldexp(1.0f, 11 - e + 7);
    b->tc_out = std::ldexp(1.0f, -(11 - e + 7));
  }
  // propagator factors on the W-grid: exp(-i pi lambda eps k^2); 1/W^2 folded into e_x
  const double dx = g.lx / g.nx, dy = g.ly / g.ny;
  b->ex.resize(2 * b->W);
  b->ey.resize(2 * b->W);
  for (int m = 0; m < b->W; ++m) {
    const double kx = signed_index(m, b->W) / (b->W * dx);
    const double ky = signed_index(m, b->W) / (b->W * dy);
    const double px = -kPi * g.lambda * g.slice_dz * kx * kx;
    const double py = -kPi * g.lambda * g.slice_dz * ky * ky;
    const double sc = 1.0 / (static_cast<double>(b->W) * b->W);
    b->ex[2 * m] = static_cast<float>(std::cos(px) * sc);
    b->ex[2 * m + 1] = static_cast<float>(std::sin(px) * sc);
    b->ey[2 * m] = static_cast<float>(std::cos(py));
    b->ey[2 * m + 1] = static_cast<float>(std::sin(py));
  }
  b->r2max = bandlimit_r2(g.bandlimit_frac, b->W);
  *out = b;
  return LMA_OK;
}

lma_status lma_free_basis(lma_basis* b) {
  if (!b) return LMA_ERR_INVALID;
  b->d_uW.release();
  b->d_ex.release();
  b->d_ey.release();
  b->d_U.release();
  b->d_Uscale.release();
  b->d_acc.release();
  b->d_det.release();
  b->d_lab.release();
  b->d_pat.release();
  b->d_pat_acc.release();
  b->d_plan.release();
  b->d_var.release();
  b->d_rsq.release();
  b->d_Up.release();
  b->d_Upscale.release();
  b->reg.tidx.release();
  b->reg.alpha.release();
  b->reg.shift.release();
  delete b;
  return LMA_OK;
}

lma_status lma_basis_get_info(const lma_basis* b, lma_basis_info* out) {
  if (!b || !out) return LMA_ERR_INVALID;
  out->n_translates = b->nT;
  out->nax = b->nax;
  out->nay = b->nay;
  out->n_sets = static_cast<int32_t>(b->sets.size());
  out->L = b->desc.L;
  out->window = b->desc.window;
  out->det_window = b->desc.det_window;
  out->gauss_sigma = b->gauss_sigma;
  out->exit_wave_bytes = b->nT * static_cast<int64_t>(b->W) * b->W *
                         (b->desc.precision == LMA_PREC_FP16_STORE ? 4 : static_cast<int64_t>(sizeof(float2)));
  out->phonon_batch = b->B;
  return LMA_OK;
}

lma_status lma_basis_coefficients(lma_ctx* ctx, lma_basis* b, int32_t px, int32_t py, double* alpha,
                                  int32_t* offsets, int64_t* translates, double* err) {
  if (!ctx || !b) return fail(ctx, LMA_ERR_INVALID, "null argument");
  const int x = mod(px, b->nx), y = mod(py, b->ny);
  const CoefSet* cs = nullptr;
  lma_status s = coef_set(b, x, y, &cs);
  if (s != LMA_OK) return s;
  for (int j = 0; j < b->desc.L; ++j) {
    if (alpha) {
      alpha[2 * j] = cs->alpha[j].real();
      alpha[2 * j + 1] = cs->alpha[j].imag();
    }
    if (offsets) {
      offsets[2 * j] = cs->odx[j];
      offsets[2 * j + 1] = cs->ody[j];
    }
    if (translates) translates[j] = translate_index(b, x + cs->odx[j], y + cs->ody[j]);
  }
  if (err) {
    err[0] = cs->err_l2;
    err[1] = cs->err_sup;
  }
  return LMA_OK;
}

lma_status lma_propagate_basis(lma_ctx* ctx, lma_specimen* sp, lma_basis* b, int32_t phonon, void* stream) {
  if (!ctx || !sp || !b) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (b->spec != sp) return fail(ctx, LMA_ERR_INVALID, "basis belongs to another specimen");
  if (phonon < 0 || phonon >= static_cast<int>(sp->ph.size()))
    return fail(ctx, LMA_ERR_INVALID, "phonon index out of range");
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lma_status s = ensure_basis_device(b, st);
  if (s != LMA_OK) return s;
  std::vector<uint8_t> all(static_cast<size_t>(b->nT), 1);
  return ensure_batch(b, sp, phonon, 1, all, true, st);
}

lma_status lma_exit_wave(lma_ctx* ctx, lma_basis* b, int64_t translate, float* out, void* stream) {
  if (!ctx || !b || !out) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (translate < 0 || translate >= b->nT) return fail(ctx, LMA_ERR_INVALID, "translate out of range");
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  if (!b->dev_tables || b->U_epoch != b->spec->epoch || !b->valid[translate])
    return fail(ctx, LMA_ERR_INVALID, "exit wave not current");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool dev = is_device_pointer(out);
  if (b->desc.precision == LMA_PREC_FP16_STORE) {
    const size_t hbytes = static_cast<size_t>(b->W) * b->W * sizeof(__half2);
    const char* src = static_cast<const char*>(b->d_U.p) + translate * hbytes;
    float scale = 1.f;
    CUDA_TRY(ctx, cudaMemcpyAsync(&scale, static_cast<const float*>(b->d_Uscale.p) + translate, sizeof(float),
                                  cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (dev) {
      CUDA_TRY(ctx, lma_dev::launch_expand_half(src, scale, reinterpret_cast<float2*>(out), st));
      return LMA_OK;
    }
    std::vector<__half2> h(static_cast<size_t>(b->W) * b->W);
    CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), src, hbytes, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    for (size_t k = 0; k < h.size(); ++k) {
      const float2 u = __half22float2(h[k]);
      out[2 * k] = u.x * scale;
      out[2 * k + 1] = u.y * scale;
    }
    return LMA_OK;
  }
  const size_t bytes = static_cast<size_t>(b->W) * b->W * sizeof(float2);
  CUDA_TRY(ctx, cudaMemcpyAsync(out, static_cast<const char*>(b->d_U.p) + translate * bytes, bytes,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (!dev) {
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return check_slice_status(ctx);
  }
  return LMA_OK;
}

lma_status lma_image(lma_ctx* ctx, lma_specimen* sp, lma_basis* b, const lma_detector* det, int32_t n_det,
                     const lma_region* region, uint32_t flags, double* out, void* stream) {
  if (!ctx || !sp || !b || !out) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (b->spec != sp) return fail(ctx, LMA_ERR_INVALID, "basis belongs to another specimen");
  if (n_det <= 0 || n_det > lma_dev::kMaxDet || !det) return fail(ctx, LMA_ERR_INVALID, "need 1..%d detectors", lma_dev::kMaxDet);
  for (int d = 0; d < n_det; ++d)
    if (!(det[d].r1 >= 0) || !(det[d].r2 > det[d].r1)) return fail(ctx, LMA_ERR_INVALID, "detector %d: need 0 <= r1 < r2", d);
  lma_status s = validate_region(ctx, b, region);
  if (s != LMA_OK) return s;
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = ensure_basis_device(b, st)) != LMA_OK) return s;
  if ((s = build_region(b, region, st)) != LMA_OK) return s;
  if ((s = build_detectors(b, det, n_det, st)) != LMA_OK) return s;
  const bool dev_out = is_device_pointer(out);
  AutotuneScope tuning(ctx, (flags & LMA_IMAGE_AUTOTUNE) != 0);
  if ((s = image_work(b, sp, n_det, (flags & LMA_IMAGE_RECOMPUTE) != 0, dev_out ? out : nullptr, st)) != LMA_OK)
    return s;
  if (!dev_out) {
    const int64_t nout = b->reg.n_probes * n_det;
    const double* fin = static_cast<const double*>(b->d_acc.p) + static_cast<size_t>(sp->ph.size()) * nout;
    CUDA_TRY(ctx, read_back(ctx, out, fin, static_cast<size_t>(nout) * sizeof(double), st));
    { const lma_status cs_ = check_slice_status(ctx); if (cs_ != LMA_OK) return cs_; }
  }
  CUDA_TRY(ctx, cudaGetLastError());
  return LMA_OK;
}

// ---------------------------------------------------------------------------------------------
// memory-bounded partition (Sec. 4.2.4)
// ---------------------------------------------------------------------------------------------
namespace {

// union sizes by stamping translates with the id of the set they were counted for
struct Stamps {
  std::vector<int32_t> mark;
  explicit Stamps(int64_t n) : mark(static_cast<size_t>(n), -1) {}
  // translates of probe q not yet stamped with id
  int fresh(const int32_t* t, int L, int32_t id) const {
    int k = 0;
    for (int j = 0; j < L; ++j) k += mark[t[j]] != id ? 1 : 0;
    return k;
  }
  int add(const int32_t* t, int L, int32_t id) {
    int k = 0;
    for (int j = 0; j < L; ++j)
      if (mark[t[j]] != id) {
        mark[t[j]] = id;
        ++k;
      }
    return k;
  }
};

using Parts = std::vector<std::vector<int32_t>>;

Parts plan_rows(const std::vector<int32_t>& sets, int L, int npx, int npy, int64_t M, int64_t nT) {
  Parts parts;
  Stamps st(nT);
  int32_t id = 0;
  int64_t size = 0;
  std::vector<int32_t> cur;
  for (int q = 0; q < npx * npy; ++q) {
    const int32_t* t = &sets[static_cast<size_t>(q) * L];
    if (!cur.empty() && size + st.fresh(t, L, id) > M) {
      parts.push_back(cur);
      cur.clear();
      ++id;
      size = 0;
    }
    cur.push_back(q);
    size += st.add(t, L, id);
  }
  if (!cur.empty()) parts.push_back(cur);
  return parts;
}

Parts tiles(int npx, int npy, int w, int h, bool column_major) {
  Parts out;
  std::vector<std::pair<int, int>> org;
  if (column_major) {
    for (int x0 = 0; x0 < npx; x0 += w)
      for (int y0 = 0; y0 < npy; y0 += h) org.emplace_back(x0, y0);
  } else {
    for (int y0 = 0; y0 < npy; y0 += h)
      for (int x0 = 0; x0 < npx; x0 += w) org.emplace_back(x0, y0);
  }
  for (auto [x0, y0] : org) {
    std::vector<int32_t> t;
    for (int b = y0; b < std::min(y0 + h, npy); ++b)
      for (int a = x0; a < std::min(x0 + w, npx); ++a) t.push_back(b * npx + a);
    out.push_back(t);
  }
  return out;
}

Parts plan_rectangles(const std::vector<int32_t>& sets, int L, int npx, int npy, int64_t M, int64_t nT,
                      bool column_major, int per_x, int per_y) {
  Stamps st(nT);
  int32_t gen = 0;
  auto fits = [&](int w, int h) {
    for (int ay = 0; ay < per_y; ++ay)
      for (int ax = 0; ax < per_x; ++ax) {
        ++gen;
        int64_t size = 0;
        for (int b = ay; b < std::min(ay + h, npy); ++b)
          for (int a = ax; a < std::min(ax + w, npx); ++a)
            size += st.add(&sets[static_cast<size_t>(b * npx + a) * L], L, gen);
        if (size > M) return false;
      }
    return true;
  };
  int64_t best_area = -1;
  int best_sq = 0, best_w = 1, best_h = 1;
  for (int w = 1; w <= npx; ++w) {
    if (!fits(w, 1)) break;
    int h = 1;
    while (h < npy && fits(w, h + 1)) ++h;
    const int64_t area = static_cast<int64_t>(w) * h;
    const int sq = -std::abs(w - h);
    // key (area, -|w - h|, w), strictly greater replaces
    if (area > best_area || (area == best_area && (sq > best_sq || (sq == best_sq && w > best_w)))) {
      best_area = area;
      best_sq = sq;
      best_w = w;
      best_h = h;
    }
  }
  return tiles(npx, npy, best_w, best_h, column_major);
}

Parts plan_greedy(const std::vector<int32_t>& sets, int L, int npx, int npy, int64_t M, int64_t nT, int start) {
  const int n = npx * npy;
  std::vector<uint8_t> assigned(n, 0);
  Parts parts;
  std::vector<int32_t> cur;
  Stamps st(nT);
  int32_t id = 0;
  int64_t size = 0, done = 0;
  int nxt = start, scan = 0;
  while (true) {
    const int q = nxt;
    const int32_t* t = &sets[static_cast<size_t>(q) * L];
    if (!cur.empty() && size + st.fresh(t, L, id) > M) {
      parts.push_back(cur);
      cur.clear();
      ++id;
      size = 0;
    }
    cur.push_back(q);
    size += st.add(t, L, id);
    assigned[q] = 1;
    if (++done == n) break;
    const int a = q % npx, b = q / npx;
    int64_t best = -1;
    int bb_best = 0, aa_best = 0;
    for (int bb = b - 1; bb <= b + 1; ++bb)
      for (int aa = a - 1; aa <= a + 1; ++aa) {
        if (aa < 0 || aa >= npx || bb < 0 || bb >= npy || assigned[bb * npx + aa]) continue;
        const int64_t c = size + st.fresh(&sets[static_cast<size_t>(bb * npx + aa) * L], L, id);
        // (cost, b, a) ascending; candidates arrive in (b, a) order, so ties keep the first
        if (best < 0 || c < best) {
          best = c;
          bb_best = bb;
          aa_best = aa;
        }
      }
    if (best >= 0) {
      nxt = bb_best * npx + aa_best;
    } else {
      while (assigned[scan]) ++scan;
      nxt = scan;
    }
  }
  parts.push_back(cur);
  return parts;
}

// T_{P_1..P_l} and max |I(P_j)|
void plan_cost(const std::vector<int32_t>& sets, int L, const Parts& parts, int64_t nT, int64_t* runs, int64_t* peak) {
  Stamps st(nT);
  int64_t T = 0, pk = 0;
  for (size_t j = 0; j < parts.size(); ++j) {
    int64_t size = 0, shared = 0;
    // translates stamped with j - 1 belong to the previous part's union
    for (int32_t q : parts[j]) {
      const int32_t* t = &sets[static_cast<size_t>(q) * L];
      for (int k = 0; k < L; ++k) {
        if (st.mark[t[k]] == static_cast<int32_t>(j)) continue;
        if (j > 0 && st.mark[t[k]] == static_cast<int32_t>(j) - 1) ++shared;
        st.mark[t[k]] = static_cast<int32_t>(j);
        ++size;
      }
    }
    T += size - shared;
    pk = std::max(pk, size);
  }
  *runs = T;
  *peak = pk;
}

int gcd_int(int a, int b) {
  while (b) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace

static lma_status validate_partition(lma_ctx* ctx, const lma_basis* b, const lma_region* r,
                                     const lma_partition_desc* d) {
  if (!d) return fail(ctx, LMA_ERR_INVALID, "null partition descriptor");
  if (d->strategy < LMA_PART_ROWS || d->strategy > LMA_PART_GREEDY)
    return fail(ctx, LMA_ERR_INVALID, "unknown partition strategy %d", d->strategy);
  if (d->max_resident < b->desc.L) return fail(ctx, LMA_ERR_INVALID, "max_resident must be at least L");
  if (d->strategy == LMA_PART_GREEDY &&
      (d->start < 0 || static_cast<int64_t>(d->start) >= static_cast<int64_t>(r->npx) * r->npy))
    return fail(ctx, LMA_ERR_INVALID, "greedy start outside the region");
  return LMA_OK;
}

// the partition of a region (cached in the basis with its cost)
static lma_status make_plan(lma_basis* b, const lma_region* r, const lma_partition_desc* d) {
  if (b->plan_valid && std::memcmp(&b->plan_r, r, sizeof(lma_region)) == 0 &&
      std::memcmp(&b->plan_d, d, sizeof(lma_partition_desc)) == 0)
    return LMA_OK;
  std::vector<int32_t> tidx, sh;
  std::vector<float> al;
  lma_status s = region_tables_host(b, r, tidx, al, sh);
  if (s != LMA_OK) return s;
  const int L = b->desc.L;
  Parts parts;
  if (d->strategy == LMA_PART_ROWS) {
    parts = plan_rows(tidx, L, r->npx, r->npy, d->max_resident, b->nT);
  } else if (d->strategy == LMA_PART_GREEDY) {
    parts = plan_greedy(tidx, L, r->npx, r->npy, d->max_resident, b->nT, d->start);
  } else {
    // the probe/lattice geometry repeats every S / gcd(S, s) probes per axis
    const int per_x = b->Sx / gcd_int(b->Sx, r->spacing_px[0]);
    const int per_y = b->Sy / gcd_int(b->Sy, r->spacing_px[1]);
    parts = plan_rectangles(tidx, L, r->npx, r->npy, d->max_resident, b->nT,
                            d->strategy == LMA_PART_RECTANGLES_COLUMN_MAJOR, per_x, per_y);
  }
  plan_cost(tidx, L, parts, b->nT, &b->plan_runs, &b->plan_peak);
  // store entries: each part keeps the previous part's waves it shares, new waves take
  // the entries freed by the previous part (lowest first). The device tables of every part
  // go into one buffer (32-bit words): probes, store entries of the probes' translates,
  // coefficients (float pairs), placements (int pairs), new items and their entries.
  std::vector<int32_t> entry_of(static_cast<size_t>(b->nT), -1);
  std::vector<int32_t> free_entries;
  for (int64_t e = d->max_resident - 1; e >= 0; --e) free_entries.push_back(static_cast<int32_t>(e));
  std::vector<int32_t> prev, tab;
  auto align4 = [&]() {
    while (tab.size() % 4) tab.push_back(0);
  };
  Stamps st(b->nT);
  b->parts.clear();
  for (size_t j = 0; j < parts.size(); ++j) {
    const int32_t id = static_cast<int32_t>(j);
    std::vector<int32_t> uni;
    for (int32_t q : parts[j])
      for (int k = 0; k < L; ++k) {
        const int32_t t = tidx[static_cast<size_t>(q) * L + k];
        if (st.mark[t] != id) {
          st.mark[t] = id;
          uni.push_back(t);
        }
      }
    for (int32_t t : prev)
      if (st.mark[t] != id) {
        free_entries.push_back(entry_of[t]);
        entry_of[t] = -1;
      }
    std::sort(free_entries.begin(), free_entries.end(), std::greater<int32_t>());
    std::sort(uni.begin(), uni.end());
    lma_basis::Part P;
    P.probes = parts[j];
    std::vector<int32_t> fresh;
    for (int32_t t : uni)
      if (entry_of[t] < 0) {
        entry_of[t] = free_entries.back();
        free_entries.pop_back();
        fresh.push_back(t);
      }
    for (int pass = 0; pass < 2; ++pass)
      for (int32_t t : fresh)
        if (origin_even(b, t) == (pass == 0)) {
          P.items.push_back(t);
          P.outs.push_back(entry_of[t]);
          if (pass == 0) ++P.n_even;
        }
    align4();
    P.o_probes = tab.size();
    tab.insert(tab.end(), P.probes.begin(), P.probes.end());
    align4();
    P.o_tidx = tab.size();
    for (int32_t q : P.probes)
      for (int k = 0; k < L; ++k) tab.push_back(entry_of[tidx[static_cast<size_t>(q) * L + k]]);
    align4();
    P.o_alpha = tab.size();
    for (int32_t q : P.probes)
      for (int k = 0; k < 2 * L; ++k) {
        int32_t w;
        std::memcpy(&w, &al[static_cast<size_t>(q) * 2 * L + k], sizeof(w));
        tab.push_back(w);
      }
    align4();
    P.o_shift = tab.size();
    for (int32_t q : P.probes)
      for (int k = 0; k < 2 * L; ++k) tab.push_back(sh[static_cast<size_t>(q) * 2 * L + k]);
    align4();
    P.o_items = tab.size();
    tab.insert(tab.end(), P.items.begin(), P.items.end());
    align4();
    P.o_outs = tab.size();
    tab.insert(tab.end(), P.outs.begin(), P.outs.end());
    b->parts.push_back(std::move(P));
    prev.swap(uni);
  }
  b->plan_tab.swap(tab);
  b->plan_r = *r;
  b->plan_d = *d;
  b->plan_valid = true;
  b->plan_dev = false;
  return LMA_OK;
}

// q discretized to K1 x K2 pixels: the inverse DFT (FP64) of the window propagator
// exp(-i pi lambda eps |k|^2) times the bandlimit, at offsets -(K/2) .. K/2
// q of Sec. 3.2 discretized to K1 x K2 pixels, in FP64: the inverse DFT of the window's
// propagator (bandlimit included) at offsets -(K/2) .. K - 1 - K/2, [K2][K1]
static void realspace_kernel_fp64(const lma_basis* b, int K1, int K2, std::vector<cd>& q) {
  const lma_grid& g = b->spec->g;
  const double dx = g.lx / g.nx, dy = g.ly / g.ny;
  std::vector<cd> root(b->W);
  for (int m = 0; m < b->W; ++m) root[m] = std::exp(cd(0.0, 2.0 * kPi * m / b->W));
  std::vector<cd> P(static_cast<size_t>(b->W) * b->W, cd(0.0, 0.0));
  for (int iy = 0; iy < b->W; ++iy) {
    const int my = signed_index(iy, b->W);
    const double ky = my / (b->W * dy);
    for (int ix = 0; ix < b->W; ++ix) {
      const int mx = signed_index(ix, b->W);
      if (my * my + mx * mx > b->r2max) continue;
      const double kx = mx / (b->W * dx);
      P[static_cast<size_t>(iy) * b->W + ix] = std::exp(cd(0.0, -kPi * g.lambda * g.slice_dz * (ky * ky + kx * kx)));
    }
  }
  q.assign(static_cast<size_t>(K1) * K2, cd(0.0, 0.0));
  for (int a = 0; a < K2; ++a) {
    const int oy = a - K2 / 2;
    for (int c = 0; c < K1; ++c) {
      const int ox = c - K1 / 2;
      cd sum(0.0, 0.0);
      for (int iy = 0; iy < b->W; ++iy)
        for (int ix = 0; ix < b->W; ++ix)
          sum += P[static_cast<size_t>(iy) * b->W + ix] * root[mod(iy * oy + ix * ox, b->W)];
      q[static_cast<size_t>(a) * K1 + c] = sum / (static_cast<double>(b->W) * b->W);
    }
  }
}

// the same kernel rounded once to complex64 for the device
static void realspace_kernel_host(const lma_basis* b, int K1, int K2, std::vector<float>& q) {
  std::vector<cd> qd;
  realspace_kernel_fp64(b, K1, K2, qd);
  q.assign(2 * qd.size(), 0.f);
  for (size_t k = 0; k < qd.size(); ++k) {
    q[2 * k] = static_cast<float>(qd[k].real());
    q[2 * k + 1] = static_cast<float>(qd[k].imag());
  }
}

lma_status lma_selftest_wait(lma_ctx* ctx, int32_t which, void* stream) {
  if (!ctx) return LMA_ERR_INVALID;
  if (which != 0 && which != 1) return fail(ctx, LMA_ERR_INVALID, "lma_selftest_wait: which must be 0 or 1");
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  const lma_status s0 = ensure_counter(ctx);
  if (s0 != LMA_OK) return s0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CUDA_TRY(ctx, lma_dev::launch_selftest_wait(which, ctx->d_counter + 1, st));
  ctx->tc_launched = true;
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return check_slice_status(ctx);
}

lma_status lma_realspace_gain(lma_ctx* ctx, const lma_basis* b, int32_t K1, int32_t K2, double* gain_all,
                              double* gain_band) {
  if (!ctx || !b || !gain_all || !gain_band) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (K1 < 1 || K2 < 1 || K1 > b->W || K2 > b->W || (K1 & 1) == 0 || (K2 & 1) == 0)
    return fail(ctx, LMA_ERR_INVALID, "K1 and K2 must be odd in 1..W");
  std::vector<cd> q;
  realspace_kernel_fp64(b, K1, K2, q);
  const int W = b->W;
  std::vector<cd> root(W);
  for (int m = 0; m < W; ++m) root[m] = std::exp(cd(0.0, -2.0 * kPi * m / W));
  double ga = 0.0, gb = 0.0;
  for (int iy = 0; iy < W; ++iy) {
    const int my = signed_index(iy, W);
    for (int ix = 0; ix < W; ++ix) {
      const int mx = signed_index(ix, W);
      cd Q(0.0, 0.0);
      for (int a = 0; a < K2; ++a)
        for (int c = 0; c < K1; ++c)
          Q += q[static_cast<size_t>(a) * K1 + c] * root[mod(iy * (a - K2 / 2) + ix * (c - K1 / 2), W)];
      const double m = std::abs(Q);
      ga = std::max(ga, m);
      if (my * my + mx * mx <= b->r2max) gb = std::max(gb, m);
    }
  }
  *gain_all = ga;
  *gain_band = gb;
  return LMA_OK;
}

lma_status lma_image_realspace(lma_ctx* ctx, lma_specimen* sp, lma_basis* b, int32_t K1, int32_t K2,
                               const lma_detector* det, int32_t n_det, const lma_region* region, uint32_t flags,
                               double* out, void* stream) {
  if (!ctx || !sp || !b || !out || !region) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (b->spec != sp) return fail(ctx, LMA_ERR_INVALID, "basis belongs to another specimen");
  if (K1 < 3 || K1 > 25 || (K1 & 1) == 0) return fail(ctx, LMA_ERR_INVALID, "K1 must be odd in 3..25");
  if (K2 < 1 || K2 > 25 || (K2 & 1) == 0) return fail(ctx, LMA_ERR_INVALID, "K2 must be odd in 1..25");
  if (b->desc.precision != LMA_PREC_C64)
    return fail(ctx, LMA_ERR_UNSUPPORTED, "real-space propagation writes the complex64 store only");
  if (b->W != kW) return fail(ctx, LMA_ERR_UNSUPPORTED, "real-space propagation runs on W = %d windows", kW);
  if (n_det <= 0 || n_det > lma_dev::kMaxDet || !det)
    return fail(ctx, LMA_ERR_INVALID, "need 1..%d detectors", lma_dev::kMaxDet);
  for (int d = 0; d < n_det; ++d)
    if (!(det[d].r1 >= 0) || !(det[d].r2 > det[d].r1)) return fail(ctx, LMA_ERR_INVALID, "detector %d: need 0 <= r1 < r2", d);
  lma_status s = validate_region(ctx, b, region);
  if (s != LMA_OK) return s;
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = ensure_basis_device(b, st)) != LMA_OK) return s;
  if ((s = build_region(b, region, st)) != LMA_OK) return s;
  if ((s = build_detectors(b, det, n_det, st)) != LMA_OK) return s;
  const std::vector<int> key{K1, K2};
  if (!b->d_rsq.p || key != b->rsq_key) {
    std::vector<float> q;
    realspace_kernel_host(b, K1, K2, q);
    CUDA_TRY(ctx, ensure(b->d_rsq, q.size() * sizeof(float)));
    CUDA_TRY(ctx, upload(ctx, b->d_rsq.p, q.data(), q.size() * sizeof(float), st));
    b->rsq_key = key;
  }
  const bool dev_out = is_device_pointer(out);
  struct RealSpace {
    lma_ctx* c;
    RealSpace(lma_ctx* c_, int k1, int k2, const void* q) : c(c_) {
      c->rs_k1 = k1;
      c->rs_k2 = k2;
      c->rs_q = static_cast<const float2*>(q);
    }
    ~RealSpace() {
      c->rs_k1 = 0;
      c->rs_k2 = 0;
      c->rs_q = nullptr;
    }
  } scope(ctx, K1, K2, b->d_rsq.p);
  s = image_work(b, sp, n_det, true, dev_out ? out : nullptr, st);
  // the store now holds real-space waves: the Fourier path must not reuse them
  std::fill(b->valid.begin(), b->valid.end(), 0);
  std::fill(b->U_phonon.begin(), b->U_phonon.end(), -1);
  if (s != LMA_OK) return s;
  (void)flags;
  if (!dev_out) {
    const int64_t nout = b->reg.n_probes * n_det;
    CUDA_TRY(ctx, read_back(ctx, out, basis_result(b, sp, n_det), static_cast<size_t>(nout) * sizeof(double), st));
    { const lma_status cs_ = check_slice_status(ctx); if (cs_ != LMA_OK) return cs_; }
  }
  CUDA_TRY(ctx, cudaGetLastError());
  return LMA_OK;
}

lma_status lma_select_L(lma_ctx* ctx, const lma_specimen* spec, const lma_probe* probe, const lma_basis_desc* desc,
                        const lma_region* region, int32_t L_max, double eps_sup, int32_t* L_out, double* err_out) {
  if (!ctx || !spec || !probe || !desc || !region || !L_out) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (L_max < 1 || L_max > kMaxL) return fail(ctx, LMA_ERR_INVALID, "L_max must be in [1, %d]", kMaxL);
  if (!(eps_sup > 0)) return fail(ctx, LMA_ERR_INVALID, "eps_sup must be positive");
  lma_basis_desc d = *desc;
  d.L = L_max;
  lma_basis* b = nullptr;
  lma_status s = lma_create_basis(ctx, spec, probe, &d, &b);
  if (s != LMA_OK) return s;
  struct Free {
    lma_basis* b;
    ~Free() { lma_free_basis(b); }
  } guard{b};
  if ((s = validate_region(ctx, b, region)) != LMA_OK) return s;
  // one representative probe per coefficient class of the region
  std::map<std::pair<int, int>, std::pair<int, int>> reps;
  for (int pb = 0; pb < region->npy; ++pb)
    for (int pa = 0; pa < region->npx; ++pa) {
      const int px = mod(region->px0 + pa * region->spacing_px[0], b->nx);
      const int py = mod(region->py0 + pb * region->spacing_px[1], b->ny);
      reps.emplace(class_key(b, px, py), std::make_pair(px, py));
    }
  build_probe(b);
  double err = 0.0;
  for (int L = 1; L <= L_max; ++L) {
    err = 0.0;
    for (const auto& kv : reps) {
      CoefSet cs;
      nearest(b, kv.second.first, kv.second.second, cs.odx, cs.ody, L);
      if ((s = solve_set_for(b, b->psi0, cs)) != LMA_OK) return s;
      err = std::max(err, cs.err_sup);
    }
    if (err <= eps_sup) {
      *L_out = L;
      if (err_out) *err_out = err;
      return LMA_OK;
    }
  }
  *L_out = 0;
  if (err_out) *err_out = err;
  return LMA_OK;
}

lma_status lma_image_coherent(lma_ctx* ctx, lma_specimen* sp, lma_basis* b, const lma_probe* variants,
                              const double* weights, int32_t n_var, const lma_detector* det, int32_t n_det,
                              const lma_region* region, uint32_t flags, double* out, void* stream) {
  if (!ctx || !sp || !b || !variants || !weights || !out || !region) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (b->spec != sp) return fail(ctx, LMA_ERR_INVALID, "basis belongs to another specimen");
  if (n_var < 1 || n_var > LMA_MAX_VARIANTS) return fail(ctx, LMA_ERR_INVALID, "need 1..%d variants", LMA_MAX_VARIANTS);
  double wsum = 0.0;
  for (int v = 0; v < n_var; ++v) {
    if (!(weights[v] >= 0) || !std::isfinite(weights[v])) return fail(ctx, LMA_ERR_INVALID, "weight %d must be >= 0", v);
    if (variants[v].alpha_max != b->probe.alpha_max)
      return fail(ctx, LMA_ERR_INVALID, "variant %d: alpha_max differs from the basis probe", v);
    if (!std::isfinite(variants[v].defocus) || !std::isfinite(variants[v].cs))
      return fail(ctx, LMA_ERR_INVALID, "variant %d: non-finite aberration", v);
    wsum += weights[v];
  }
  if (!(wsum > 0)) return fail(ctx, LMA_ERR_INVALID, "weights sum to zero");
  if (n_det <= 0 || n_det > lma_dev::kMaxDet || !det)
    return fail(ctx, LMA_ERR_INVALID, "need 1..%d detectors", lma_dev::kMaxDet);
  for (int d = 0; d < n_det; ++d)
    if (!(det[d].r1 >= 0) || !(det[d].r2 > det[d].r1)) return fail(ctx, LMA_ERR_INVALID, "detector %d: need 0 <= r1 < r2", d);
  lma_status s = validate_region(ctx, b, region);
  if (s != LMA_OK) return s;
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = ensure_basis_device(b, st)) != LMA_OK) return s;
  if ((s = build_region(b, region, st)) != LMA_OK) return s;
  if ((s = build_detectors(b, det, n_det, st)) != LMA_OK) return s;
  const int L = b->desc.L;
  const int64_t np = b->reg.n_probes;
  // coefficient tables of the variants (kept for the next call with the same variants)
  std::vector<double> key{static_cast<double>(n_var)};
  for (int32_t v : {region->px0, region->py0, region->npx, region->npy, region->spacing_px[0], region->spacing_px[1]})
    key.push_back(v);
  for (int v = 0; v < n_var; ++v) {
    key.push_back(variants[v].defocus);
    key.push_back(variants[v].cs);
    key.push_back(weights[v]);
  }
  const size_t tab_floats = static_cast<size_t>(n_var) * np * L * 2;
  if (!b->d_var.p || key != b->var_key) {
    std::vector<float> tab(tab_floats + 2 * static_cast<size_t>(n_var), 0.f);
    std::vector<std::pair<int32_t, int>> order;
    for (int v = 0; v < n_var; ++v) {
      std::vector<cd> psi0;
      probe_at_origin(b, variants[v], psi0);
      std::map<std::pair<int, int>, CoefSet> sets;
      for (int pb = 0; pb < region->npy; ++pb)
        for (int pa = 0; pa < region->npx; ++pa) {
          const int px = mod(region->px0 + pa * region->spacing_px[0], b->nx);
          const int py = mod(region->py0 + pb * region->spacing_px[1], b->ny);
          const auto k = class_key(b, px, py);
          auto it = sets.find(k);
          if (it == sets.end()) {
            CoefSet cs;
            nearest(b, px, py, cs.odx, cs.ody);
            if ((s = solve_set_for(b, psi0, cs)) != LMA_OK) return s;
            it = sets.emplace(k, std::move(cs)).first;
          }
          // the entry order of the region tables (nearest() is deterministic)
          const size_t base = ((static_cast<size_t>(v) * np) + static_cast<size_t>(pb) * region->npx + pa) * L;
          entry_order(b, px, py, it->second, order);
          for (int i = 0; i < L; ++i) {
            const int j = order[i].second;
            tab[2 * (base + i)] = static_cast<float>(it->second.alpha[j].real());
            tab[2 * (base + i) + 1] = static_cast<float>(it->second.alpha[j].imag());
          }
        }
    }
    // weights w_v / (sum w * configurations) as doubles after the coefficients
    std::vector<double> wv(n_var);
    for (int v = 0; v < n_var; ++v) wv[v] = weights[v] / wsum / static_cast<double>(sp->ph.size());
    const size_t bytes = tab_floats * sizeof(float) + n_var * sizeof(double);
    CUDA_TRY(ctx, ensure(b->d_var, bytes));
    CUDA_TRY(ctx, upload_parts(ctx, {HostPart{b->d_var.p, tab.data(), tab_floats * sizeof(float)},
                                      HostPart{static_cast<char*>(b->d_var.p) + tab_floats * sizeof(float), wv.data(),
                                               n_var * sizeof(double)}},
                               st));
    b->var_key = key;
  }
  const int nph = static_cast<int>(sp->ph.size());
  const int64_t nout = np * n_det;
  CUDA_TRY(ctx, ensure(b->d_acc, static_cast<size_t>(nout) * (static_cast<size_t>(n_var) * nph + 1) * sizeof(double)));
  const bool half = b->desc.precision == LMA_PREC_FP16_STORE;
  const bool recompute = (flags & LMA_IMAGE_RECOMPUTE) != 0;
  AutotuneScope tuning(ctx, (flags & LMA_IMAGE_AUTOTUNE) != 0);
  for (int phi0 = 0; phi0 < nph; phi0 += b->B) {
    const int nb = std::min(b->B, nph - phi0);
    if ((s = ensure_batch(b, sp, phi0, nb, b->reg.needed, recompute, st)) != LMA_OK) return s;
    for (int v = 0; v < n_var; ++v) {
      lma_dev::SynthArgs a{};
      a.U = half ? nullptr : static_cast<const float2*>(b->d_U.p);
      a.Uh = half ? b->d_U.p : nullptr;
      a.Uscale = half ? static_cast<const float*>(b->d_Uscale.p) : nullptr;
      a.tidx = static_cast<const int32_t*>(b->reg.tidx.p);
      a.alpha = reinterpret_cast<const float2*>(static_cast<const float*>(b->d_var.p) +
                                                static_cast<size_t>(v) * np * L * 2);
      a.shift = static_cast<const int2*>(b->reg.shift.p);
      a.L = L;
      a.n_probes = static_cast<int>(np);
      a.npx = region->npx;
      a.npy = region->npy;
      a.strip = kSynthStrip;
      a.n_cfg = nb;
      a.cfg_base = phi0;
      a.n_translates = static_cast<int>(b->nT);
      a.u_slot = static_cast<size_t>(b->nT) * b->W * b->W;
      a.cyclic = (b->W == kW && b->nx == kW && b->ny == kW) ? 1 : 0;
      a.W = b->W;
      a.det_bits = static_cast<const uint32_t*>(b->d_det.p);
      a.n_det = n_det;
      a.acc = static_cast<double*>(b->d_acc.p) + static_cast<size_t>(v) * nph * nout;
      a.band_r2 = b->r2max;
      { const lma_status ss_ = synth_launch(ctx, a, half, lma_dev::kReadAnnuli, np * nb, region_geom(b), st); if (ss_ != LMA_OK) return ss_; }
    }
  }
  const double* acc = static_cast<const double*>(b->d_acc.p);
  const double* wdev = reinterpret_cast<const double*>(static_cast<const char*>(b->d_var.p) + tab_floats * sizeof(float));
  const bool dev_out = is_device_pointer(out);
  double* fin = dev_out ? out : static_cast<double*>(b->d_acc.p) + static_cast<size_t>(n_var) * nph * nout;
  CUDA_TRY(ctx, counted(ctx, K_FIN, nout, st,
                        [&] { return lma_dev::launch_finalize_variants(acc, nout, nph, n_var, wdev, fin, st); }));
  if (!dev_out) {
    CUDA_TRY(ctx, read_back(ctx, out, fin, static_cast<size_t>(nout) * sizeof(double), st));
    { const lma_status cs_ = check_slice_status(ctx); if (cs_ != LMA_OK) return cs_; }
  }
  CUDA_TRY(ctx, cudaGetLastError());
  return LMA_OK;
}

lma_status lma_partition(lma_ctx* ctx, lma_basis* b, const lma_region* region, const lma_partition_desc* desc,
                         int32_t* part, int32_t* n_parts, int64_t* runs, int64_t* peak) {
  if (!ctx || !b || !region) return fail(ctx, LMA_ERR_INVALID, "null argument");
  lma_status s = validate_region(ctx, b, region);
  if (s != LMA_OK) return s;
  if ((s = validate_partition(ctx, b, region, desc)) != LMA_OK) return s;
  if ((s = make_plan(b, region, desc)) != LMA_OK) return s;
  if (part)
    for (size_t j = 0; j < b->parts.size(); ++j)
      for (int32_t q : b->parts[j].probes) part[q] = static_cast<int32_t>(j);
  if (n_parts) *n_parts = static_cast<int32_t>(b->parts.size());
  if (runs) *runs = b->plan_runs;
  if (peak) *peak = b->plan_peak;
  return LMA_OK;
}

lma_status lma_image_partitioned(lma_ctx* ctx, lma_specimen* sp, lma_basis* b, const lma_detector* det,
                                 int32_t n_det, const lma_region* region, const lma_partition_desc* desc,
                                 uint32_t flags, double* out, void* stream) {
  if (!ctx || !sp || !b || !out || !region) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (b->spec != sp) return fail(ctx, LMA_ERR_INVALID, "basis belongs to another specimen");
  if (n_det <= 0 || n_det > lma_dev::kMaxDet || !det)
    return fail(ctx, LMA_ERR_INVALID, "need 1..%d detectors", lma_dev::kMaxDet);
  for (int d = 0; d < n_det; ++d)
    if (!(det[d].r1 >= 0) || !(det[d].r2 > det[d].r1)) return fail(ctx, LMA_ERR_INVALID, "detector %d: need 0 <= r1 < r2", d);
  lma_status s = validate_region(ctx, b, region);
  if (s != LMA_OK) return s;
  if ((s = validate_partition(ctx, b, region, desc)) != LMA_OK) return s;
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = ensure_basis_tables(b, st)) != LMA_OK) return s;
  if ((s = build_detectors(b, det, n_det, st)) != LMA_OK) return s;
  if ((s = make_plan(b, region, desc)) != LMA_OK) return s;
  const bool half = b->desc.precision == LMA_PREC_FP16_STORE;
  const int64_t M = std::min<int64_t>(desc->max_resident, b->nT);   // entries in use never exceed |I_f|
  if (!b->plan_dev) {
    CUDA_TRY(ctx, ensure(b->d_plan, std::max<size_t>(4, b->plan_tab.size() * sizeof(int32_t))));
    CUDA_TRY(ctx, upload(ctx, b->d_plan.p, b->plan_tab.data(), b->plan_tab.size() * sizeof(int32_t), st));
    b->plan_dev = true;
  }
  CUDA_TRY(ctx, ensure(b->d_Up, static_cast<size_t>(M) * b->W * b->W * (half ? 4 : sizeof(float2))));
  if (half) CUDA_TRY(ctx, ensure(b->d_Upscale, static_cast<size_t>(M) * sizeof(float)));
  if (!ctx->d_counter && (s = ensure_counter(ctx)) != LMA_OK) return s;
  const int nph = static_cast<int>(sp->ph.size());
  const int64_t np = static_cast<int64_t>(region->npx) * region->npy;
  const int64_t nout = np * n_det;
  CUDA_TRY(ctx, ensure(b->d_acc, static_cast<size_t>(nout) * (nph + 1) * sizeof(double)));
  const int32_t* tab = static_cast<const int32_t*>(b->d_plan.p);
  AutotuneScope tuning(ctx, (flags & LMA_IMAGE_AUTOTUNE) != 0);
  for (int phi = 0; phi < nph; ++phi) {
    // transmission of this configuration in slot 0 (rebuilt: the bounded path keeps nothing)
    if ((s = reserve_t_slots(sp, 1)) != LMA_OK) return s;
    if ((s = ensure_t(sp, 0, phi, true, st)) != LMA_OK) return s;
    for (const lma_basis::Part& P : b->parts) {
      lma_dev::SliceLaunch Lh{};
      Lh.n_jobs = 1;
      Lh.job[0] = make_job(b, sp);
      Lh.job[0].U = half ? nullptr : static_cast<float2*>(b->d_Up.p);
      Lh.job[0].Uh = half ? b->d_Up.p : nullptr;
      Lh.job[0].Uscale = half ? static_cast<float*>(b->d_Upscale.p) : nullptr;
      Lh.job[0].u_slot = static_cast<size_t>(M) * b->W * b->W;
      Lh.counter = ctx->d_counter;
      for (int part = 0; part < 2; ++part) {
        const int off = part == 0 ? 0 : P.n_even;
        const int cnt = part == 0 ? P.n_even : static_cast<int>(P.items.size()) - P.n_even;
        if (cnt == 0) continue;
        Lh.list = tab + P.o_items + off;
        Lh.out_index = tab + P.o_outs + off;
        Lh.n_list = cnt;
        Lh.start[0] = 0;
        Lh.start[1] = cnt;
        if ((s = slice_launch(ctx, Lh, part == 0, b->desc.precision, static_cast<int64_t>(cnt) * sp->g.n_slices, st)) != LMA_OK)
          return s;
      }
      lma_dev::SynthArgs a{};
      a.U = half ? nullptr : static_cast<const float2*>(b->d_Up.p);
      a.Uh = half ? b->d_Up.p : nullptr;
      a.Uscale = half ? static_cast<const float*>(b->d_Upscale.p) : nullptr;
      a.tidx = tab + P.o_tidx;
      a.alpha = reinterpret_cast<const float2*>(tab + P.o_alpha);
      a.shift = reinterpret_cast<const int2*>(tab + P.o_shift);
      a.L = b->desc.L;
      a.n_probes = static_cast<int>(np);
      a.probe_list = tab + P.o_probes;
      a.n_list = static_cast<int>(P.probes.size());
      a.npx = region->npx;
      a.npy = region->npy;
      a.strip = kSynthStrip;
      a.n_cfg = 1;
      a.cfg_base = phi;
      a.n_translates = static_cast<int>(M);
      a.u_slot = static_cast<size_t>(M) * b->W * b->W;
      a.cyclic = (b->W == kW && b->nx == kW && b->ny == kW) ? 1 : 0;
      a.W = b->W;
      a.det_bits = static_cast<const uint32_t*>(b->d_det.p);
      a.n_det = n_det;
      a.acc = static_cast<double*>(b->d_acc.p);
      a.band_r2 = b->r2max;
      { const lma_status ss_ = synth_launch(ctx, a, half, lma_dev::kReadAnnuli, static_cast<int64_t>(P.probes.size()), SynthGeom{}, st); if (ss_ != LMA_OK) return ss_; }
    }
  }
  const double* acc = static_cast<const double*>(b->d_acc.p);
  const bool dev_out = is_device_pointer(out);
  double* fin = dev_out ? out : static_cast<double*>(b->d_acc.p) + static_cast<size_t>(nph) * nout;
  CUDA_TRY(ctx, counted(ctx, K_FIN, nout, st, [&] { return lma_dev::launch_finalize(acc, nout, nph, 1.0 / nph, fin, st); }));
  if (!dev_out) {
    CUDA_TRY(ctx, read_back(ctx, out, fin, static_cast<size_t>(nout) * sizeof(double), st));
    { const lma_status cs_ = check_slice_status(ctx); if (cs_ != LMA_OK) return cs_; }
  }
  CUDA_TRY(ctx, cudaGetLastError());
  return LMA_OK;
}

// common steps of the 3D and 4D images: checks, tables, device work, read-back
static lma_status image_readout(lma_ctx* ctx, lma_specimen* sp, lma_basis* b, const Readout& ro, const lma_region* region,
                         uint32_t flags, void* out, size_t out_bytes, cudaStream_t st) {
  lma_status s = validate_region(ctx, b, region);
  if (s != LMA_OK) return s;
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  if ((s = ensure_basis_device(b, st)) != LMA_OK) return s;
  if ((s = build_region(b, region, st)) != LMA_OK) return s;
  const bool dev_out = is_device_pointer(out);
  AutotuneScope tuning(ctx, (flags & LMA_IMAGE_AUTOTUNE) != 0);
  if ((s = images_work(ctx, {ImageJob{b, sp, dev_out ? out : nullptr}}, ro, (flags & LMA_IMAGE_RECOMPUTE) != 0,
                       st)) != LMA_OK)
    return s;
  if (!dev_out) {
    const void* fin = ro.mode == lma_dev::kReadPattern ? b->d_pat.p : static_cast<const void*>(basis_result(b, sp, ro.n_out));
    CUDA_TRY(ctx, read_back(ctx, out, fin, out_bytes, st));
    { const lma_status cs_ = check_slice_status(ctx); if (cs_ != LMA_OK) return cs_; }
  }
  CUDA_TRY(ctx, cudaGetLastError());
  return LMA_OK;
}

lma_status lma_image_rings(lma_ctx* ctx, lma_specimen* sp, lma_basis* b, double ring_width, int32_t n_rings,
                           const lma_region* region, uint32_t flags, double* out, void* stream) {
  if (!ctx || !sp || !b || !out || !region) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (b->spec != sp) return fail(ctx, LMA_ERR_INVALID, "basis belongs to another specimen");
  if (!(ring_width > 0) || !std::isfinite(ring_width)) return fail(ctx, LMA_ERR_INVALID, "ring width must be positive");
  if (n_rings < 1 || n_rings > LMA_MAX_RINGS) return fail(ctx, LMA_ERR_INVALID, "need 1..%d rings", LMA_MAX_RINGS);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  lma_status s = build_labels(b, ring_width, n_rings, st);
  if (s != LMA_OK) return s;
  Readout ro;
  ro.mode = lma_dev::kReadLabels;
  ro.n_out = n_rings;
  const size_t bytes = static_cast<size_t>(region->npx) * region->npy * n_rings * sizeof(double);
  return image_readout(ctx, sp, b, ro, region, flags, out, bytes, st);
}

lma_status lma_image_4d(lma_ctx* ctx, lma_specimen* sp, lma_basis* b, int32_t half_x, int32_t half_y,
                        const lma_region* region, uint32_t flags, float* out, void* stream) {
  if (!ctx || !sp || !b || !out || !region) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (b->spec != sp) return fail(ctx, LMA_ERR_INVALID, "basis belongs to another specimen");
  const int lim = b->desc.det_window / 2 - 1;
  if (half_x < 0 || half_y < 0 || half_x > lim || half_y > lim)
    return fail(ctx, LMA_ERR_INVALID, "pattern half-widths must lie in 0..%d", lim);
  Readout ro;
  ro.mode = lma_dev::kReadPattern;
  ro.pat_a = half_x;
  ro.pat_b = half_y;
  if (static_cast<int64_t>(region->npx) * region->npy * ro.pat_size() > (int64_t(1) << 34))
    return fail(ctx, LMA_ERR_INVALID, "4D output too large");
  const size_t bytes = static_cast<size_t>(region->npx) * region->npy * ro.pat_size() * sizeof(float);
  return image_readout(ctx, sp, b, ro, region, flags, out, bytes, static_cast<cudaStream_t>(stream));
}

lma_status lma_image_many(lma_ctx* ctx, int32_t n, lma_specimen* const* specs, lma_basis* const* bases,
                          const lma_detector* det, int32_t n_det, const lma_region* regions, uint32_t flags,
                          double* const* outs, void* stream) {
  if (!ctx || n <= 0 || !specs || !bases || !regions || !outs) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (n_det <= 0 || n_det > lma_dev::kMaxDet || !det)
    return fail(ctx, LMA_ERR_INVALID, "need 1..%d detectors", lma_dev::kMaxDet);
  for (int d = 0; d < n_det; ++d)
    if (!(det[d].r1 >= 0) || !(det[d].r2 > det[d].r1)) return fail(ctx, LMA_ERR_INVALID, "detector %d: need 0 <= r1 < r2", d);
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  const bool graph = (flags & LMA_IMAGE_GRAPH) != 0;
  const bool recompute = (flags & LMA_IMAGE_RECOMPUTE) != 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (graph && (!recompute || !stream))
    return fail(ctx, LMA_ERR_INVALID, "LMA_IMAGE_GRAPH needs LMA_IMAGE_RECOMPUTE and a non-default stream");
  lma_status s;
  for (int k = 0; k < n; ++k) {
    if (!specs[k] || !bases[k] || !outs[k]) return fail(ctx, LMA_ERR_INVALID, "null specimen, basis or output %d", k);
    if (bases[k]->spec != specs[k]) return fail(ctx, LMA_ERR_INVALID, "basis %d belongs to another specimen", k);
    if (bases[k]->ctx != ctx) return fail(ctx, LMA_ERR_INVALID, "basis %d belongs to another context", k);
    for (int q = 0; q < k; ++q)
      if (specs[q] == specs[k]) return fail(ctx, LMA_ERR_INVALID, "specimen %d appears twice", k);
    if ((s = validate_region(ctx, bases[k], &regions[k])) != LMA_OK) return s;
    if (graph && !is_device_pointer(outs[k])) return fail(ctx, LMA_ERR_INVALID, "LMA_IMAGE_GRAPH needs device outputs");
  }
  for (int k = 0; k < n; ++k) {
    if ((s = ensure_basis_device(bases[k], st)) != LMA_OK) return s;
    if ((s = build_region(bases[k], &regions[k], st)) != LMA_OK) return s;
    if ((s = build_detectors(bases[k], det, n_det, st)) != LMA_OK) return s;
  }
  std::vector<bool> dev_out(n);
  std::vector<ImageJob> jobs;
  for (int k = 0; k < n; ++k) {
    dev_out[k] = is_device_pointer(outs[k]);
    jobs.push_back(ImageJob{bases[k], specs[k], dev_out[k] ? outs[k] : nullptr});
  }
  AutotuneScope tuning(ctx, (flags & LMA_IMAGE_AUTOTUNE) != 0);
  Readout ro;
  ro.n_out = n_det;
  if (!graph) {
    if ((s = images_work(ctx, jobs, ro, recompute, st)) != LMA_OK) return s;
    for (int k = 0; k < n; ++k)
      if (!dev_out[k]) {
        const int64_t nout = bases[k]->reg.n_probes * n_det;
        const double* fin = static_cast<const double*>(bases[k]->d_acc.p) + specs[k]->ph.size() * nout;
        CUDA_TRY(ctx, read_back(ctx, outs[k], fin, static_cast<size_t>(nout) * sizeof(double), st));
        { const lma_status cs_ = check_slice_status(ctx); if (cs_ != LMA_OK) return cs_; }
      }
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return LMA_OK;
  }
  // host-side preparation that a captured graph cannot do: atoms on the device
  for (int k = 0; k < n; ++k)
    for (int phi = 0; phi < static_cast<int>(specs[k]->ph.size()); ++phi)
      if ((s = ensure_atoms_device(specs[k], phi, st)) != LMA_OK) return s;
  // signature of every buffer and size the captured launches depend on; the item
  // lists they read are checked separately against the context's list cache
  auto signature = [&]() {
    std::vector<uintptr_t> key;
    key.push_back(static_cast<uintptr_t>(n));
    key.push_back(static_cast<uintptr_t>(n_det));
    key.push_back(static_cast<uintptr_t>(ctx->forced_mode + 1));
    key.push_back(reinterpret_cast<uintptr_t>(ctx->d_counter));
    for (int d = 0; d < n_det; ++d) {
      uint64_t r1, r2;
      std::memcpy(&r1, &det[d].r1, 8);
      std::memcpy(&r2, &det[d].r2, 8);
      key.push_back(static_cast<uintptr_t>(r1));
      key.push_back(static_cast<uintptr_t>(r2));
    }
    for (int k = 0; k < n; ++k) {
      const lma_specimen* sp = specs[k];
      const lma_basis* b = bases[k];
      for (uintptr_t v : {reinterpret_cast<uintptr_t>(sp), reinterpret_cast<uintptr_t>(b),
                          reinterpret_cast<uintptr_t>(outs[k]), reinterpret_cast<uintptr_t>(sp->d_t.p),
                          reinterpret_cast<uintptr_t>(sp->d_peak.p), reinterpret_cast<uintptr_t>(b->d_U.p),
                          reinterpret_cast<uintptr_t>(b->d_Uscale.p), reinterpret_cast<uintptr_t>(b->d_acc.p),
                          reinterpret_cast<uintptr_t>(b->d_det.p), reinterpret_cast<uintptr_t>(b->reg.tidx.p),
                          reinterpret_cast<uintptr_t>(b->reg.alpha.p), reinterpret_cast<uintptr_t>(b->reg.shift.p),
                          static_cast<uintptr_t>(b->B)})
        key.push_back(v);
      const lma_region& r = regions[k];
      for (int32_t v : {r.px0, r.py0, r.npx, r.npy, r.spacing_px[0], r.spacing_px[1]})
        key.push_back(static_cast<uintptr_t>(static_cast<uint32_t>(v)));
      for (const PhononSet& p : sp->ph)
        for (const DevBuf* d : {&p.dx, &p.dy, &p.dsp, &p.dss}) key.push_back(reinterpret_cast<uintptr_t>(d->p));
    }
    return key;
  };
  auto lists_resident = [&](const lma_ctx::Graph& g) {
    for (const auto& u : g.lists) {
      bool found = false;
      for (const auto& e : ctx->lists) found = found || (e.p == u.first && e.hash == u.second);
      if (!found) return false;
    }
    return true;
  };
  std::vector<uintptr_t> key = signature();
  for (auto& g : ctx->graphs)
    if (g.key == key && lists_resident(g)) {
      CUDA_TRY(ctx, cudaGraphLaunch(g.exec, st));
      return LMA_OK;
    }
  // first call with these buffers: an ordinary run (allocations, list uploads, tuning,
  // outputs), then the same launches captured for later calls
  if ((s = images_work(ctx, jobs, ro, true, st)) != LMA_OK) return s;
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  key = signature();
  lma_ctx::Graph g;
  g.key = key;
  ctx->capture_lists.clear();
  CUDA_TRY(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  ctx->capturing = true;
  lma_status cs = images_work(ctx, jobs, ro, true, st);
  ctx->capturing = false;
  cudaError_t e = cudaStreamEndCapture(st, &g.graph);
  g.lists.swap(ctx->capture_lists);
  if (cs != LMA_OK) {
    if (g.graph) cudaGraphDestroy(g.graph);
    return cs;
  }
  if (e != cudaSuccess) return fail(ctx, LMA_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&g.exec, g.graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g.graph);
    return fail(ctx, LMA_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  if (ctx->graphs.size() >= 8) {
    cudaGraphExecDestroy(ctx->graphs.front().exec);
    cudaGraphDestroy(ctx->graphs.front().graph);
    ctx->graphs.erase(ctx->graphs.begin());
  }
  ctx->graphs.push_back(g);
  return LMA_OK;   // this call's outputs came from the ordinary run
}

lma_status lma_set_slice_mode(lma_ctx* ctx, int32_t mode) {
  if (!ctx) return LMA_ERR_INVALID;
  if (mode < LMA_SLICE_AUTO || mode >= lma_dev::kSliceModes) return fail(ctx, LMA_ERR_INVALID, "unknown slice mode %d", mode);
  ctx->forced_mode = mode;
  return LMA_OK;
}

lma_status lma_set_synth_mode(lma_ctx* ctx, int32_t mode) {
  if (!ctx) return LMA_ERR_INVALID;
  if (mode < LMA_SYNTH_AUTO || mode > LMA_SYNTH_GROUPED) return fail(ctx, LMA_ERR_INVALID, "unknown synthesis form %d", mode);
  ctx->synth_mode = mode;
  return LMA_OK;
}

lma_status lma_set_synth_buffer_limit(lma_ctx* ctx, int64_t bytes) {
  if (!ctx) return LMA_ERR_INVALID;
  if (bytes < 0) return fail(ctx, LMA_ERR_INVALID, "negative buffer limit");
  ctx->psi_max = bytes == 0 ? (int64_t(2) << 30) : bytes;
  return LMA_OK;
}

lma_status lma_tuning_read(lma_ctx* ctx, lma_tuning* out, int32_t cap, int32_t* n) {
  if (!ctx || !n || cap < 0 || (cap > 0 && !out)) return fail(ctx, LMA_ERR_INVALID, "null argument");
  *n = static_cast<int32_t>(ctx->tune.size());
  for (int32_t i = 0; i < cap && i < *n; ++i) out[i] = ctx->tune[i].rec;
  return LMA_OK;
}

lma_status lma_synth_tuning_read(lma_ctx* ctx, lma_synth_tuning* out, int32_t cap, int32_t* n) {
  if (!ctx || !n || cap < 0 || (cap > 0 && !out)) return fail(ctx, LMA_ERR_INVALID, "null argument");
  *n = static_cast<int32_t>(ctx->synth_tune.size());
  for (int32_t i = 0; i < cap && i < *n; ++i) out[i] = ctx->synth_tune[i].rec;
  return LMA_OK;
}

lma_status lma_edit_column(lma_ctx* ctx, lma_specimen* sp, lma_basis* b, double cx, double cy, double r_site,
                           int32_t op, int16_t new_species, int64_t* n_atoms_changed, int64_t* n_stale) {
  if (!ctx || !sp) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (b && b->spec != sp) return fail(ctx, LMA_ERR_INVALID, "basis belongs to another specimen");
  if (!(r_site > 0)) return fail(ctx, LMA_ERR_INVALID, "r_site must be positive");
  if (op != LMA_EDIT_REMOVE && op != LMA_EDIT_SET_SPECIES) return fail(ctx, LMA_ERR_INVALID, "unknown edit op");
  if (op == LMA_EDIT_SET_SPECIES && (new_species < 0 || new_species >= static_cast<int>(sp->peak.size())))
    return fail(ctx, LMA_ERR_INVALID, "new species out of range");
  const lma_grid& g = sp->g;
  const double dx = g.lx / g.nx, dy = g.ly / g.ny;
  int64_t changed = 0;
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
  for (PhononSet& P : sp->ph) {
    std::vector<uint8_t> hit(P.x.size(), 0);
    for (size_t k = 0; k < P.x.size(); ++k) {
      double ddx = P.x[k] - cx, ddy = P.y[k] - cy;
      ddx -= g.lx * std::nearbyint(ddx / g.lx);
      ddy -= g.ly * std::nearbyint(ddy / g.ly);
      if (ddx * ddx + ddy * ddy < r_site * r_site) {
        hit[k] = 1;
        ++changed;
        // unwrapped position next to the column centre
        xmin = std::min(xmin, cx + ddx);
        xmax = std::max(xmax, cx + ddx);
        ymin = std::min(ymin, cy + ddy);
        ymax = std::max(ymax, cy + ddy);
      }
    }
    if (op == LMA_EDIT_SET_SPECIES) {
      for (size_t k = 0; k < P.x.size(); ++k)
        if (hit[k]) P.sp[k] = new_species;
    } else {
      size_t w = 0;
      for (size_t k = 0; k < P.x.size(); ++k) {
        if (hit[k]) continue;
        P.x[w] = P.x[k];
        P.y[w] = P.y[k];
        P.sp[w] = P.sp[k];
        P.slc[w] = P.slc[k];
        ++w;
      }
      P.x.resize(w);
      P.y.resize(w);
      P.sp.resize(w);
      P.slc.resize(w);
      std::fill(P.slice_start.begin(), P.slice_start.end(), 0);
      for (int32_t s : P.slc) P.slice_start[s + 1]++;
      for (int s = 0; s < g.n_slices; ++s) P.slice_start[s + 1] += P.slice_start[s];
    }
    P.dirty = true;
  }
  int64_t stale = 0;
  if (changed > 0) {
    // pixels within r_cut of a touched atom (with one pixel of margin)
    const int x0 = static_cast<int>(std::floor((xmin - sp->r_cut) / dx)) - 1;
    const int x1 = static_cast<int>(std::ceil((xmax + sp->r_cut) / dx)) + 1;
    const int y0 = static_cast<int>(std::floor((ymin - sp->r_cut) / dy)) - 1;
    const int y1 = static_cast<int>(std::ceil((ymax + sp->r_cut) / dy)) + 1;
    Rect r{mod(x0, g.nx), mod(y0, g.ny), std::min(x1 - x0 + 1, g.nx), std::min(y1 - y0 + 1, g.ny)};
    for (int k = 0; k < sp->t_slots; ++k)
      if (sp->t_phonon[k] >= 0) sp->t_stale[k].push_back(r);
    sp->epoch++;
    if (b && b->dev_tables) {
      // exit waves whose window [pos - W/2, pos + W/2) meets the rectangle (periodic)
      auto meets = [](int a0, int aw, int b0, int bw, int n) {
        if (aw >= n || bw >= n) return true;
        const int d = mod(b0 - a0, n);
        return d < aw || mod(a0 - b0, n) < bw;
      };
      for (int ib = 0; ib < b->nay; ++ib) {
        const int wy0 = mod(b->oy + ib * b->Sy - b->W / 2, g.ny);
        if (!meets(wy0, b->W, r.y0, r.h, g.ny)) continue;
        for (int ia = 0; ia < b->nax; ++ia) {
          const int wx0 = mod(b->ox + ia * b->Sx - kW / 2, g.nx);
          if (!meets(wx0, kW, r.x0, r.w, g.nx)) continue;
          const int64_t i = static_cast<int64_t>(ib) * b->nax + ia;
          for (int k = 0; k < b->B; ++k) {
            uint8_t& v = b->valid[static_cast<size_t>(k) * b->nT + i];
            if (v) {
              v = 0;
              ++stale;
            }
          }
        }
      }
      b->U_epoch = sp->epoch;
    }
  }
  if (n_atoms_changed) *n_atoms_changed = changed;
  if (n_stale) *n_stale = stale;
  return LMA_OK;
}

lma_status lma_readout_noalloc(lma_ctx* ctx, lma_basis* b, const float* exit_waves, const lma_detector* det,
                               int32_t n_det, const lma_region* region, double* out, void* stream) {
  if (!ctx || !b || !exit_waves || !out) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (n_det <= 0 || n_det > lma_dev::kMaxDet || !det)
    return fail(ctx, LMA_ERR_INVALID, "need 1..%d detectors", lma_dev::kMaxDet);
  for (int d = 0; d < n_det; ++d)
    if (!(det[d].r1 >= 0) || !(det[d].r2 > det[d].r1))
      return fail(ctx, LMA_ERR_INVALID, "detector %d: need 0 <= r1 < r2", d);
  lma_status s = validate_region(ctx, b, region);
  if (s != LMA_OK) return s;
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  if ((s = device_window(b)) != LMA_OK) return s;
  if (!is_device_pointer(exit_waves) || !is_device_pointer(out))
    return fail(ctx, LMA_ERR_INVALID, "exit_waves and out must be device memory");
  const int L = b->desc.L;
  const int64_t np = static_cast<int64_t>(region->npx) * region->npy;
  const int64_t nout = np * n_det;
  // scratch layout: accumulator | detector bits | translate indices | coefficients | shifts
  auto up = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
  const size_t o_acc = 0;
  const size_t o_det = up(o_acc + static_cast<size_t>(nout) * sizeof(double));
  const size_t o_tidx = up(o_det + static_cast<size_t>(n_det) * lma_dev::kThreads * sizeof(uint32_t));
  const size_t o_alpha = up(o_tidx + static_cast<size_t>(np) * L * sizeof(int32_t));
  const size_t o_shift = up(o_alpha + static_cast<size_t>(np) * L * 2 * sizeof(float));
  const size_t need = up(o_shift + static_cast<size_t>(np) * L * 2 * sizeof(int32_t));
  if (need > lma_dev::kNoAllocScratchBytes)
    return fail(ctx, LMA_ERR_INVALID,
                "region of %lld probes with L = %d needs %zu bytes of scratch; the no-allocation readout "
                "holds %zu bytes (about %lld probes at L = %d)",
                static_cast<long long>(np), L, need, lma_dev::kNoAllocScratchBytes,
                static_cast<long long>(lma_dev::kNoAllocScratchBytes / (L * 20 + 8 * n_det + 1)), L);
  // host tables and detector bits, built as lma_image builds them (FP64 coefficients rounded once)
  std::vector<int32_t> tidx, sh;
  std::vector<float> al;
  if ((s = region_tables_host(b, region, tidx, al, sh)) != LMA_OK) return s;
  std::vector<uint32_t> bits;
  detector_bits_host(b, det, n_det, bits);
  void* scratch = nullptr;
  CUDA_TRY(ctx, lma_dev::noalloc_scratch(&scratch));
  char* base = static_cast<char*>(scratch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CUDA_TRY(ctx, cudaMemsetAsync(base + o_acc, 0, static_cast<size_t>(nout) * sizeof(double), st));
  CUDA_TRY(ctx, cudaMemcpyAsync(base + o_det, bits.data(), bits.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(base + o_tidx, tidx.data(), tidx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(base + o_alpha, al.data(), al.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(base + o_shift, sh.data(), sh.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  lma_dev::SynthArgs a{};
  a.U = reinterpret_cast<const float2*>(exit_waves);
  a.tidx = reinterpret_cast<const int32_t*>(base + o_tidx);
  a.alpha = reinterpret_cast<const float2*>(base + o_alpha);
  a.shift = reinterpret_cast<const int2*>(base + o_shift);
  a.L = L;
  a.n_probes = static_cast<int>(np);
  a.npx = region->npx;
  a.npy = region->npy;
  a.strip = kSynthStrip;
  a.n_cfg = 1;
  a.cfg_base = 0;
  a.n_translates = static_cast<int>(b->nT);
  a.u_slot = 0;
  a.cyclic = (b->W == kW && b->nx == kW && b->ny == kW) ? 1 : 0;
      a.W = b->W;
  a.det_bits = reinterpret_cast<const uint32_t*>(base + o_det);
  a.n_det = n_det;
  a.acc = reinterpret_cast<double*>(base + o_acc);
  CUDA_TRY(ctx, lma_dev::launch_synth(a, false, lma_dev::kReadAnnuli, lma_dev::kSynthGridAuto, st));
  CUDA_TRY(ctx, lma_dev::launch_finalize(a.acc, nout, 1, 1.0, out, st));
  // the host tables above are pageable: keep them alive until the copies have run
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return LMA_OK;
}

lma_status lma_profile_enable(lma_ctx* ctx, int32_t on) {
  if (!ctx) return LMA_ERR_INVALID;
  for (auto& p : ctx->pend) {
    cudaEventSynchronize(p.b);
    ctx->pool.push_back(p.a);
    ctx->pool.push_back(p.b);
  }
  ctx->pend.clear();
  for (auto& k : ctx->stat) k = lma_kernel_stat{};
  ctx->alloc_base = g_allocations.load(std::memory_order_relaxed);
  ctx->prof = on != 0 && !ctx->host_only;
  return LMA_OK;
}

lma_status lma_profile_read(lma_ctx* ctx, lma_profile* out) {
  if (!ctx || !out) return fail(ctx, LMA_ERR_INVALID, "null argument");
  for (auto& p : ctx->pend) {
    CUDA_TRY(ctx, cudaEventSynchronize(p.b));
    float ms = 0.f;
    CUDA_TRY(ctx, cudaEventElapsedTime(&ms, p.a, p.b));
    ctx->stat[p.kind].total_ms += ms;
    ctx->pool.push_back(p.a);
    ctx->pool.push_back(p.b);
  }
  ctx->pend.clear();
  out->potential = ctx->stat[K_POT];
  out->slice = ctx->stat[K_SLICE];
  out->synth = ctx->stat[K_SYNTH];
  out->finalize = ctx->stat[K_FIN];
  out->allocations = g_allocations.load(std::memory_order_relaxed) - ctx->alloc_base;
  return LMA_OK;
}

lma_status lma_affected_probes(lma_ctx* ctx, lma_basis* b, const lma_region* region, uint8_t* out_mask,
                               int64_t* n_affected) {
  if (!ctx || !b) return fail(ctx, LMA_ERR_INVALID, "null argument");
  lma_status s = validate_region(ctx, b, region);
  if (s != LMA_OK) return s;
  int64_t cnt = 0;
  for (int pb = 0; pb < region->npy; ++pb)
    for (int pa = 0; pa < region->npx; ++pa) {
      const int px = mod(region->px0 + pa * region->spacing_px[0], b->nx);
      const int py = mod(region->py0 + pb * region->spacing_px[1], b->ny);
      const CoefSet* cs = nullptr;
      if ((s = coef_set(b, px, py, &cs)) != LMA_OK) return s;
      bool hit = false;
      for (int j = 0; j < b->desc.L && !hit; ++j) {
        const int64_t i = translate_index(b, px + cs->odx[j], py + cs->ody[j]);
        hit = b->valid.empty() || !b->valid[i];   // first slot (the serving case holds one)
      }
      if (out_mask) out_mask[static_cast<size_t>(pb) * region->npx + pa] = hit ? 1 : 0;
      cnt += hit ? 1 : 0;
    }
  if (n_affected) *n_affected = cnt;
  return LMA_OK;
}

}  // extern "C"
