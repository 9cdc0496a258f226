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

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return cudaSuccess;
  b.release();
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}

struct Rect {
  int x0, y0, w, h;   // periodic pixel rectangle
};

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
  DevBuf d_t;                 // transmission of configuration t_phonon
  int t_phonon = -1;
  std::vector<Rect> t_stale;  // pixel rectangles of d_t to rebuild
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
};

struct lma_basis {
  lma_ctx* ctx = nullptr;
  const lma_specimen* spec = nullptr;
  lma_probe probe{};
  lma_basis_desc desc{};
  double gauss_sigma = 0.0;
  int nx = 0, ny = 0;
  int Sx = 0, Sy = 0, ox = 0, oy = 0, nax = 0, nay = 0;
  int64_t nT = 0;
  std::vector<cd> psi0;        // full-grid probe centred at pixel 0 (lazy)
  std::vector<cd> uW;          // W x W input wave
  std::vector<float> ex, ey;   // interleaved complex
  int r2max = 0;
  std::map<std::pair<int, int>, CoefSet> sets;
  // device
  DevBuf d_uW, d_ex, d_ey, d_U, d_Uscale, d_list, d_acc, d_det;
  bool dev_tables = false;
  int U_phonon = -1;
  int64_t U_epoch = -1;
  std::vector<uint8_t> valid;
  std::vector<int32_t> last_list;
  RegionTables reg;
  bool reg_valid = false;
  std::vector<double> det_key;
};

namespace {

bool device_ready(lma_ctx* ctx) {
  if (!ctx || ctx->host_only) return false;
  return cudaSetDevice(ctx->device) == cudaSuccess;
}

// full-grid probe psi_0 (eq. probe_wave_function at p = 0), unit norm
void build_probe(lma_basis* b) {
  if (!b->psi0.empty()) return;
  const lma_grid& g = b->spec->g;
  const int nx = g.nx, ny = g.ny;
  const double dx = g.lx / nx, dy = g.ly / ny, lam = g.lambda;
  std::vector<cd> spec(static_cast<size_t>(nx) * ny);
  for (int iy = 0; iy < ny; ++iy) {
    const double ky = signed_index(iy, ny) / (ny * dy);
    for (int ix = 0; ix < nx; ++ix) {
      const double kx = signed_index(ix, nx) / (nx * dx);
      const double k2 = ky * ky + kx * kx;
      const bool ap = lam * std::sqrt(k2) < b->probe.alpha_max;
      if (!ap) continue;
      const double chi = 0.5 * kPi * b->probe.cs * lam * lam * lam * k2 * k2 -
                         kPi * b->probe.defocus * lam * k2;
      spec[static_cast<size_t>(iy) * nx + ix] = std::exp(cd(0.0, -chi));
    }
  }
  fft2(spec, ny, nx, true);
  double n2 = 0.0;
  for (const cd& c : spec) n2 += std::norm(c);
  const double s = 1.0 / std::sqrt(n2);
  for (cd& c : spec) c *= s;
  b->psi0.swap(spec);
}

// the input wave on its window (Sec. 4.2.3)
void build_input_wave(lma_basis* b) {
  const lma_grid& g = b->spec->g;
  const double dx = g.lx / g.nx, dy = g.ly / g.ny;
  b->uW.assign(static_cast<size_t>(kW) * kW, cd(0.0, 0.0));
  if (b->desc.kind == LMA_BASIS_GAUSS) {
    const double s = b->gauss_sigma;
    for (int y = 0; y < kW; ++y) {
      const double ry = (y - kW / 2) * dy;
      for (int x = 0; x < kW; ++x) {
        const double rx = (x - kW / 2) * dx;
        b->uW[static_cast<size_t>(y) * kW + x] = cd(std::exp(-(ry * ry + rx * rx) / (2.0 * s * s)), 0.0);
      }
    }
  } else {
    build_probe(b);
    for (int y = 0; y < kW; ++y)
      for (int x = 0; x < kW; ++x)
        b->uW[static_cast<size_t>(y) * kW + x] =
            b->psi0[static_cast<size_t>(mod(y - kW / 2, g.ny)) * g.nx + mod(x - kW / 2, g.nx)];
  }
}

// the L nearest translates of probe p (Sec. 4.2.1 option (iii)); ties by (d^2, dy, dx)
void nearest(const lma_basis* b, int px, int py, std::vector<int>& odx, std::vector<int>& ody) {
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
  const int L = b->desc.L;
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

// least-squares coefficients of one probe class (eqs. lma_approximation_exit1_0 / exit2_0),
// in coordinates relative to the probe (probe at pixel 0, translate j at its offset)
lma_status solve_set(lma_basis* b, CoefSet& cs) {
  build_probe(b);
  const int nx = b->nx, ny = b->ny, L = b->desc.L;
  // bounding box of the union of windows [o - W/2, o + W/2)
  int ylo = 1 << 30, yhi = -(1 << 30), xlo = 1 << 30, xhi = -(1 << 30);
  for (int j = 0; j < L; ++j) {
    ylo = std::min(ylo, cs.ody[j] - kW / 2);
    yhi = std::max(yhi, cs.ody[j] + kW / 2);
    xlo = std::min(xlo, cs.odx[j] - kW / 2);
    xhi = std::max(xhi, cs.odx[j] + kW / 2);
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
        any = mod(yy - (cs.ody[j] - kW / 2), ny) < kW && mod(xx - (cs.odx[j] - kW / 2), nx) < kW;
      if (any) rows.push_back(static_cast<size_t>(mod(yy, ny)) * nx + mod(xx, nx));
    }
  const int m = static_cast<int>(rows.size());
  std::vector<cd> A(static_cast<size_t>(m) * L, cd(0.0, 0.0)), rhs(m);
  std::vector<uint8_t> in_rows(static_cast<size_t>(nx) * ny, 0);
  for (int i = 0; i < m; ++i) {
    const int gy = static_cast<int>(rows[i] / nx), gx = static_cast<int>(rows[i] % nx);
    in_rows[rows[i]] = 1;
    rhs[i] = b->psi0[rows[i]];
    for (int j = 0; j < L; ++j) {
      const int ly = mod(gy - (cs.ody[j] - kW / 2), ny), lx = mod(gx - (cs.odx[j] - kW / 2), nx);
      if (ly < kW && lx < kW) A[static_cast<size_t>(j) * m + i] = b->uW[static_cast<size_t>(ly) * kW + lx];
    }
  }
  std::vector<cd> A0 = A, rhs0 = rhs, x;
  if (!lstsq_householder(A, m, L, rhs, x))
    return fail(b->ctx, LMA_ERR_INVALID, "least squares: input waves are linearly dependent");
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
  for (size_t k = 0; k < b->psi0.size(); ++k) {
    const double a = std::abs(b->psi0[k]);
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
lma_status ensure_basis_device(lma_basis* b, cudaStream_t st) {
  lma_ctx* ctx = b->ctx;
  if (b->dev_tables) return LMA_OK;
  std::vector<float> uw(2 * static_cast<size_t>(kW) * kW);
  for (size_t k = 0; k < b->uW.size(); ++k) {
    uw[2 * k] = static_cast<float>(b->uW[k].real());
    uw[2 * k + 1] = static_cast<float>(b->uW[k].imag());
  }
  CUDA_TRY(ctx, ensure(b->d_uW, uw.size() * sizeof(float)));
  CUDA_TRY(ctx, ensure(b->d_ex, b->ex.size() * sizeof(float)));
  CUDA_TRY(ctx, ensure(b->d_ey, b->ey.size() * sizeof(float)));
  CUDA_TRY(ctx, cudaMemcpyAsync(b->d_uW.p, uw.data(), uw.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(b->d_ex.p, b->ex.data(), b->ex.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(b->d_ey.p, b->ey.data(), b->ey.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  const bool half = b->desc.precision == LMA_PREC_MIXED;
  const size_t ubytes = static_cast<size_t>(b->nT) * kW * kW * (half ? 4 : sizeof(float2));
  CUDA_TRY(ctx, ensure(b->d_U, ubytes));
  if (half) CUDA_TRY(ctx, ensure(b->d_Uscale, static_cast<size_t>(b->nT) * sizeof(float)));
  b->last_list.clear();
  b->valid.assign(static_cast<size_t>(b->nT), 0);
  b->U_phonon = -1;
  b->dev_tables = true;
  return LMA_OK;
}

// upload the atoms of a configuration (slice-sorted) if they changed
lma_status ensure_atoms_device(lma_specimen* sp, int phi, cudaStream_t st) {
  lma_ctx* ctx = sp->ctx;
  PhononSet& p = sp->ph[phi];
  if (!p.dirty && p.dx.p) return LMA_OK;
  const size_t n = std::max<size_t>(1, p.x.size());
  CUDA_TRY(ctx, ensure(p.dx, n * sizeof(double)));
  CUDA_TRY(ctx, ensure(p.dy, n * sizeof(double)));
  CUDA_TRY(ctx, ensure(p.dsp, n * sizeof(int16_t)));
  CUDA_TRY(ctx, ensure(p.dss, p.slice_start.size() * sizeof(int32_t)));
  if (!p.x.empty()) {
    CUDA_TRY(ctx, cudaMemcpyAsync(p.dx.p, p.x.data(), p.x.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_TRY(ctx, cudaMemcpyAsync(p.dy.p, p.y.data(), p.y.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_TRY(ctx, cudaMemcpyAsync(p.dsp.p, p.sp.data(), p.sp.size() * sizeof(int16_t), cudaMemcpyHostToDevice, st));
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(p.dss.p, p.slice_start.data(), p.slice_start.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, st));
  // pageable sources: make sure the host vectors may change after return
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  p.dirty = false;
  return LMA_OK;
}

lma_status launch_t(lma_specimen* sp, int phi, const Rect& r, cudaStream_t st) {
  lma_ctx* ctx = sp->ctx;
  const lma_grid& g = sp->g;
  PhononSet& p = sp->ph[phi];
  lma_dev::PotArgs a{};
  a.ax = static_cast<const double*>(p.dx.p);
  a.ay = static_cast<const double*>(p.dy.p);
  a.asp = static_cast<const int16_t*>(p.dsp.p);
  a.slice_start = static_cast<const int32_t*>(p.dss.p);
  a.peak = static_cast<const float*>(sp->d_peak.p);
  a.n_species = static_cast<int>(sp->peak.size());
  a.n_terms = static_cast<int>(sp->frac.size());
  for (int q = 0; q < a.n_terms; ++q) {
    a.frac[q] = static_cast<float>(sp->frac[q]);
    a.inv2w2[q] = static_cast<float>(1.0 / (2.0 * sp->width[q] * sp->width[q]));
  }
  a.rc = sp->r_cut;
  a.rc2 = static_cast<float>(sp->r_cut * sp->r_cut);
  a.nx = g.nx;
  a.ny = g.ny;
  a.n_slices = g.n_slices;
  a.lx = g.lx;
  a.ly = g.ly;
  a.dx = g.lx / g.nx;
  a.dy = g.ly / g.ny;
  a.dx_hi = static_cast<float>(a.dx);
  a.dx_lo = static_cast<float>(a.dx - static_cast<double>(a.dx_hi));
  a.dy_hi = static_cast<float>(a.dy);
  a.dy_lo = static_cast<float>(a.dy - static_cast<double>(a.dy_hi));
  a.sigma = static_cast<float>(g.sigma);
  // Tiles sit on the absolute 16-pixel grid whatever the rectangle, so a
  // pixel is always computed by the same tile origin: a partial rebuild is
  // bitwise equal to a full one (atoms are taken relative to the tile origin).
  const int x0 = r.x0 - r.x0 % 16, y0 = r.y0 - r.y0 % 16;
  a.rx0 = x0;
  a.ry0 = y0;
  a.rw = std::min(g.nx, ((r.x0 - x0 + r.w + 15) / 16) * 16);
  a.rh = std::min(g.ny, ((r.y0 - y0 + r.h + 15) / 16) * 16);
  a.t = static_cast<float2*>(sp->d_t.p);
  const int64_t units = static_cast<int64_t>(r.w) * r.h * g.n_slices;
  CUDA_TRY(ctx, counted(ctx, K_POT, units, st, [&] { return lma_dev::launch_potential(a, st); }));
  return LMA_OK;
}

// make d_t hold configuration phi with no stale pixels
lma_status ensure_t(lma_specimen* sp, int phi, bool force, cudaStream_t st) {
  lma_ctx* ctx = sp->ctx;
  const lma_grid& g = sp->g;
  // periodic halo of W pixels on the right and bottom of every slice
  const size_t tbytes = static_cast<size_t>(g.n_slices) * (g.nx + kW) * (g.ny + kW) * sizeof(float2);
  CUDA_TRY(ctx, ensure(sp->d_t, tbytes));
  if (!sp->d_peak.p) {
    std::vector<float> pk(sp->peak.begin(), sp->peak.end());
    CUDA_TRY(ctx, ensure(sp->d_peak, pk.size() * sizeof(float)));
    CUDA_TRY(ctx, cudaMemcpy(sp->d_peak.p, pk.data(), pk.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  lma_status s = ensure_atoms_device(sp, phi, st);
  if (s != LMA_OK) return s;
  if (force || sp->t_phonon != phi) {
    s = launch_t(sp, phi, Rect{0, 0, g.nx, g.ny}, st);
    if (s != LMA_OK) return s;
    sp->t_phonon = phi;
    sp->t_stale.clear();
    return LMA_OK;
  }
  for (const Rect& r : sp->t_stale) {
    s = launch_t(sp, phi, r, st);
    if (s != LMA_OK) return s;
  }
  sp->t_stale.clear();
  return LMA_OK;
}

// window x origin parity of translate i: (ox + a Sx - W/2) mod nx, nx and W even
bool origin_even(const lma_basis* b, int32_t i) {
  return ((b->ox + (i % b->nax) * b->Sx) & 1) == 0;
}

lma_status propagate_list(lma_basis* b, lma_specimen* sp, const std::vector<int32_t>& list_in,
                          cudaStream_t st) {
  lma_ctx* ctx = b->ctx;
  if (list_in.empty()) return LMA_OK;
  // even window origins first (16-byte staging), then odd ones
  std::vector<int32_t> list;
  list.reserve(list_in.size());
  for (int32_t i : list_in)
    if (origin_even(b, i)) list.push_back(i);
  const size_t n_even = list.size();
  for (int32_t i : list_in)
    if (!origin_even(b, i)) list.push_back(i);
  if (list != b->last_list) {
    // stream order keeps this copy behind the kernels that read the previous list
    CUDA_TRY(ctx, ensure(b->d_list, list.size() * sizeof(int32_t)));
    CUDA_TRY(ctx, cudaMemcpyAsync(b->d_list.p, list.data(), list.size() * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, st));
    b->last_list = list;
  }
  const lma_grid& g = sp->g;
  lma_dev::SliceArgs a{};
  a.t = static_cast<const float2*>(sp->d_t.p);
  a.nx = g.nx;
  a.ny = g.ny;
  a.n_slices = g.n_slices;
  a.uW = static_cast<const float2*>(b->d_uW.p);
  a.lat_ox = b->ox;
  a.lat_oy = b->oy;
  a.lat_sx = b->Sx;
  a.lat_sy = b->Sy;
  a.lat_nax = b->nax;
  const bool half = b->desc.precision == LMA_PREC_MIXED;
  a.U = half ? nullptr : static_cast<float2*>(b->d_U.p);
  a.Uh = half ? b->d_U.p : nullptr;
  a.Uscale = half ? static_cast<float*>(b->d_Uscale.p) : nullptr;
  a.ex = static_cast<const float2*>(b->d_ex.p);
  a.ey = static_cast<const float2*>(b->d_ey.p);
  a.r2max = b->r2max;
  const int32_t* dl = static_cast<const int32_t*>(b->d_list.p);
  for (int part = 0; part < 2; ++part) {
    const size_t off = part == 0 ? 0 : n_even;
    const size_t cnt = part == 0 ? n_even : list.size() - n_even;
    if (cnt == 0) continue;
    a.list = dl + off;
    a.n_list = static_cast<int>(cnt);
    const int64_t units = static_cast<int64_t>(cnt) * g.n_slices;
    CUDA_TRY(ctx, counted(ctx, K_SLICE, units, st, [&] { return lma_dev::launch_slice(a, part == 0, half, st); }));
  }
  for (int32_t i : list) b->valid[i] = 1;
  return LMA_OK;
}

// make U current for configuration phi on the given translates
lma_status ensure_U(lma_basis* b, lma_specimen* sp, int phi, const std::vector<uint8_t>& needed,
                    bool recompute, cudaStream_t st) {
  if (b->U_phonon != phi || recompute || b->U_epoch != sp->epoch) {
    if (b->U_epoch != sp->epoch && b->U_phonon == phi && !recompute) {
      // edited through another basis: no exact bookkeeping here, recompute all
    }
    std::fill(b->valid.begin(), b->valid.end(), 0);
    b->U_phonon = phi;
    b->U_epoch = sp->epoch;
  }
  std::vector<int32_t> list;
  for (int64_t i = 0; i < b->nT; ++i)
    if (needed[i] && !b->valid[i]) list.push_back(static_cast<int32_t>(i));
  if (list.empty()) return LMA_OK;
  lma_status s = ensure_t(sp, phi, recompute, st);
  if (s != LMA_OK) return s;
  return propagate_list(b, sp, list, st);
}

lma_status build_region(lma_basis* b, const lma_region* r, cudaStream_t st) {
  lma_ctx* ctx = b->ctx;
  if (b->reg_valid && std::memcmp(&b->reg.r, r, sizeof(lma_region)) == 0) return LMA_OK;
  const int L = b->desc.L;
  const int64_t np = static_cast<int64_t>(r->npx) * r->npy;
  std::vector<int32_t> tidx(static_cast<size_t>(np) * L);
  std::vector<float> al(2 * static_cast<size_t>(np) * L);
  std::vector<int32_t> sh(2 * static_cast<size_t>(np) * L);
  const int half = (b->desc.det_window - b->desc.window) / 2;
  for (int pb = 0; pb < r->npy; ++pb) {
    for (int pa = 0; pa < r->npx; ++pa) {
      const int px = mod(r->px0 + pa * r->spacing_px[0], b->nx);
      const int py = mod(r->py0 + pb * r->spacing_px[1], b->ny);
      const CoefSet* cs = nullptr;
      lma_status s = coef_set(b, px, py, &cs);
      if (s != LMA_OK) return s;
      const size_t base = (static_cast<size_t>(pb) * r->npx + pa) * L;
      for (int j = 0; j < L; ++j) {
        tidx[base + j] = static_cast<int32_t>(translate_index(b, px + cs->odx[j], py + cs->ody[j]));
        al[2 * (base + j)] = static_cast<float>(cs->alpha[j].real());
        al[2 * (base + j) + 1] = static_cast<float>(cs->alpha[j].imag());
        sh[2 * (base + j)] = cs->odx[j] + half;
        sh[2 * (base + j) + 1] = cs->ody[j] + half;
      }
    }
  }
  RegionTables& R = b->reg;
  CUDA_TRY(ctx, ensure(R.tidx, tidx.size() * sizeof(int32_t)));
  CUDA_TRY(ctx, ensure(R.alpha, al.size() * sizeof(float)));
  CUDA_TRY(ctx, ensure(R.shift, sh.size() * sizeof(int32_t)));
  CUDA_TRY(ctx, cudaMemcpyAsync(R.tidx.p, tidx.data(), tidx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(R.alpha.p, al.data(), al.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaMemcpyAsync(R.shift.p, sh.data(), sh.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  R.r = *r;
  R.n_probes = np;
  R.h_tidx.swap(tidx);
  b->reg_valid = true;
  return LMA_OK;
}

// detector bits in the C layout of the synthesis kernel: word T = kx + 128 k1y, bit j <-> ky = k1y + 4 j
lma_status build_detectors(lma_basis* b, const lma_detector* det, int n_det, cudaStream_t st) {
  lma_ctx* ctx = b->ctx;
  std::vector<double> key;
  for (int d = 0; d < n_det; ++d) {
    key.push_back(det[d].r1);
    key.push_back(det[d].r2);
  }
  if (b->d_det.p && key == b->det_key) return LMA_OK;
  const lma_grid& g = b->spec->g;
  const int D = b->desc.det_window;
  const double dx = g.lx / g.nx, dy = g.ly / g.ny, lam = g.lambda, frac = g.bandlimit_frac;
  std::vector<uint32_t> bits(static_cast<size_t>(n_det) * lma_dev::kThreads, 0u);
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
  CUDA_TRY(ctx, ensure(b->d_det, bits.size() * sizeof(uint32_t)));
  CUDA_TRY(ctx, cudaMemcpyAsync(b->d_det.p, bits.data(), bits.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  b->det_key = key;
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

}  // namespace

namespace {

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
    for (size_t k = 0; k < order.size(); ++k) {
      P.x[k] = A.x[order[k]];
      P.y[k] = A.y[order[k]];
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

void lma_destroy(lma_ctx* ctx) { delete ctx; }

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
  sp->t_phonon = -1;
  sp->t_stale.clear();
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
  lma_status s = ensure_t(sp, phonon, false, st);
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
  if (!dev) CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return LMA_OK;
}

lma_status lma_create_basis(lma_ctx* ctx, const lma_specimen* spec, const lma_probe* probe,
                            const lma_basis_desc* desc, lma_basis** out) {
  if (!ctx || !spec || !probe || !desc || !out) return fail(ctx, LMA_ERR_INVALID, "null argument");
  const lma_grid& g = spec->g;
  const lma_basis_desc& d = *desc;
  if (d.window != kW || d.det_window != kW)
    return fail(ctx, LMA_ERR_UNSUPPORTED, "window and det_window must be %d", kW);
  if (g.nx < kW || g.ny < kW) return fail(ctx, LMA_ERR_UNSUPPORTED, "grid smaller than the window");
  if (!is_pow2(g.nx) || !is_pow2(g.ny)) return fail(ctx, LMA_ERR_UNSUPPORTED, "grid sizes must be powers of two");
  if (d.kind != LMA_BASIS_GAUSS && d.kind != LMA_BASIS_PROBE)
    return fail(ctx, LMA_ERR_INVALID, "unknown input wave kind");
  if (d.precision != LMA_PREC_C64 && d.precision != LMA_PREC_MIXED)
    return fail(ctx, LMA_ERR_INVALID, "precision must be LMA_PREC_C64 or LMA_PREC_MIXED");
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
  build_input_wave(b);
  // propagator factors on the W-grid: exp(-i pi lambda eps k^2); 1/W^2 folded into e_x
  const double dx = g.lx / g.nx, dy = g.ly / g.ny;
  b->ex.resize(2 * kW);
  b->ey.resize(2 * kW);
  for (int m = 0; m < kW; ++m) {
    const double kx = signed_index(m, kW) / (kW * dx);
    const double ky = signed_index(m, kW) / (kW * dy);
    const double px = -kPi * g.lambda * g.slice_dz * kx * kx;
    const double py = -kPi * g.lambda * g.slice_dz * ky * ky;
    const double sc = 1.0 / (static_cast<double>(kW) * kW);
    b->ex[2 * m] = static_cast<float>(std::cos(px) * sc);
    b->ex[2 * m + 1] = static_cast<float>(std::sin(px) * sc);
    b->ey[2 * m] = static_cast<float>(std::cos(py));
    b->ey[2 * m + 1] = static_cast<float>(std::sin(py));
  }
  b->r2max = bandlimit_r2(g.bandlimit_frac, kW);
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
  b->d_list.release();
  b->d_acc.release();
  b->d_det.release();
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
  out->exit_wave_bytes = b->nT * static_cast<int64_t>(kW) * kW *
                         (b->desc.precision == LMA_PREC_MIXED ? 4 : static_cast<int64_t>(sizeof(float2)));
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
  return ensure_U(b, sp, phonon, all, true, st);
}

lma_status lma_exit_wave(lma_ctx* ctx, lma_basis* b, int64_t translate, float* out, void* stream) {
  if (!ctx || !b || !out) return fail(ctx, LMA_ERR_INVALID, "null argument");
  if (translate < 0 || translate >= b->nT) return fail(ctx, LMA_ERR_INVALID, "translate out of range");
  if (!device_ready(ctx)) return fail(ctx, LMA_ERR_UNSUPPORTED, "no device in this context");
  if (!b->dev_tables || !b->valid[translate]) return fail(ctx, LMA_ERR_INVALID, "exit wave not current");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool dev = is_device_pointer(out);
  if (b->desc.precision == LMA_PREC_MIXED) {
    const size_t hbytes = static_cast<size_t>(kW) * kW * sizeof(__half2);
    const char* src = static_cast<const char*>(b->d_U.p) + translate * hbytes;
    float scale = 1.f;
    CUDA_TRY(ctx, cudaMemcpyAsync(&scale, static_cast<const float*>(b->d_Uscale.p) + translate, sizeof(float),
                                  cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (dev) {
      CUDA_TRY(ctx, lma_dev::launch_expand_half(src, scale, reinterpret_cast<float2*>(out), st));
      return LMA_OK;
    }
    std::vector<__half2> h(static_cast<size_t>(kW) * kW);
    CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), src, hbytes, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    for (size_t k = 0; k < h.size(); ++k) {
      const float2 u = __half22float2(h[k]);
      out[2 * k] = u.x * scale;
      out[2 * k + 1] = u.y * scale;
    }
    return LMA_OK;
  }
  const size_t bytes = static_cast<size_t>(kW) * kW * sizeof(float2);
  CUDA_TRY(ctx, cudaMemcpyAsync(out, static_cast<const char*>(b->d_U.p) + translate * bytes, bytes,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (!dev) CUDA_TRY(ctx, cudaStreamSynchronize(st));
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
  const int64_t np = b->reg.n_probes;
  const int64_t nout = np * n_det;
  CUDA_TRY(ctx, ensure(b->d_acc, static_cast<size_t>(nout) * sizeof(double)));
  CUDA_TRY(ctx, cudaMemsetAsync(b->d_acc.p, 0, static_cast<size_t>(nout) * sizeof(double), st));
  std::vector<uint8_t> needed(static_cast<size_t>(b->nT), 0);
  for (int32_t i : b->reg.h_tidx) needed[i] = 1;
  const bool recompute = (flags & LMA_IMAGE_RECOMPUTE) != 0;
  const int nph = static_cast<int>(sp->ph.size());
  for (int phi = 0; phi < nph; ++phi) {
    if ((s = ensure_U(b, sp, phi, needed, recompute, st)) != LMA_OK) return s;
    lma_dev::SynthArgs a{};
    const bool half = b->desc.precision == LMA_PREC_MIXED;
    a.U = half ? nullptr : static_cast<const float2*>(b->d_U.p);
    a.Uh = half ? b->d_U.p : nullptr;
    a.Uscale = half ? static_cast<const float*>(b->d_Uscale.p) : nullptr;
    a.tidx = static_cast<const int32_t*>(b->reg.tidx.p);
    a.alpha = static_cast<const float2*>(b->reg.alpha.p);
    a.shift = static_cast<const int2*>(b->reg.shift.p);
    a.L = b->desc.L;
    a.n_probes = static_cast<int>(np);
    a.cyclic = (b->nx == kW && b->ny == kW) ? 1 : 0;
    a.det_bits = static_cast<const uint32_t*>(b->d_det.p);
    a.n_det = n_det;
    a.acc = static_cast<double*>(b->d_acc.p);
    CUDA_TRY(ctx, counted(ctx, K_SYNTH, np, st, [&] { return lma_dev::launch_synth(a, half, st); }));
  }
  const double scale = 1.0 / nph;
  const double* acc = static_cast<const double*>(b->d_acc.p);
  if (is_device_pointer(out)) {
    CUDA_TRY(ctx, counted(ctx, K_FIN, nout, st, [&] { return lma_dev::launch_finalize(acc, nout, scale, out, st); }));
  } else {
    double* acc_out = static_cast<double*>(b->d_acc.p);
    CUDA_TRY(ctx, counted(ctx, K_FIN, nout, st, [&] { return lma_dev::launch_finalize(acc, nout, scale, acc_out, st); }));
    CUDA_TRY(ctx, cudaMemcpyAsync(out, b->d_acc.p, static_cast<size_t>(nout) * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
  }
  CUDA_TRY(ctx, cudaGetLastError());
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
    if (sp->t_phonon >= 0) sp->t_stale.push_back(r);
    sp->epoch++;
    if (b && b->dev_tables) {
      // exit waves whose window [pos - W/2, pos + W/2) meets the rectangle (periodic)
      auto meets = [](int a0, int aw, int b0, int bw, int n) {
        if (aw >= n || bw >= n) return true;
        const int d = mod(b0 - a0, n);
        return d < aw || mod(a0 - b0, n) < bw;
      };
      for (int ib = 0; ib < b->nay; ++ib) {
        const int wy0 = mod(b->oy + ib * b->Sy - kW / 2, g.ny);
        if (!meets(wy0, kW, r.y0, r.h, g.ny)) continue;
        for (int ia = 0; ia < b->nax; ++ia) {
          const int wx0 = mod(b->ox + ia * b->Sx - kW / 2, g.nx);
          if (!meets(wx0, kW, r.x0, r.w, g.nx)) continue;
          const int64_t i = static_cast<int64_t>(ib) * b->nax + ia;
          if (b->valid[i]) {
            b->valid[i] = 0;
            ++stale;
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
  // host tables (FP64 coefficients rounded once, as in lma_image)
  std::vector<int32_t> tidx(static_cast<size_t>(np) * L), sh(2 * static_cast<size_t>(np) * L);
  std::vector<float> al(2 * static_cast<size_t>(np) * L);
  const int half = (b->desc.det_window - b->desc.window) / 2;
  for (int pb = 0; pb < region->npy; ++pb)
    for (int pa = 0; pa < region->npx; ++pa) {
      const int px = mod(region->px0 + pa * region->spacing_px[0], b->nx);
      const int py = mod(region->py0 + pb * region->spacing_px[1], b->ny);
      const CoefSet* cs = nullptr;
      if ((s = coef_set(b, px, py, &cs)) != LMA_OK) return s;
      const size_t base = (static_cast<size_t>(pb) * region->npx + pa) * L;
      for (int j = 0; j < L; ++j) {
        tidx[base + j] = static_cast<int32_t>(translate_index(b, px + cs->odx[j], py + cs->ody[j]));
        al[2 * (base + j)] = static_cast<float>(cs->alpha[j].real());
        al[2 * (base + j) + 1] = static_cast<float>(cs->alpha[j].imag());
        sh[2 * (base + j)] = cs->odx[j] + half;
        sh[2 * (base + j) + 1] = cs->ody[j] + half;
      }
    }
  const lma_grid& g = b->spec->g;
  const int D = b->desc.det_window;
  const double dx = g.lx / g.nx, dy = g.ly / g.ny, lam = g.lambda, frac = g.bandlimit_frac;
  std::vector<uint32_t> bits(static_cast<size_t>(n_det) * lma_dev::kThreads, 0u);
  for (int d = 0; d < n_det; ++d)
    for (int iy = 0; iy < D; ++iy) {
      const int my = signed_index(iy, D);
      const double ky = my / (D * dy);
      for (int ix = 0; ix < D; ++ix) {
        const int mx = signed_index(ix, D);
        const double kx = mx / (D * dx);
        const double ang = lam * std::sqrt(ky * ky + kx * kx);
        const bool band = static_cast<double>(4 * (my * my + mx * mx)) <= frac * frac * D * D;
        if (ang >= det[d].r1 && ang < det[d].r2 && band)
          bits[static_cast<size_t>(d) * lma_dev::kThreads + ix + 128 * (iy & 3)] |= 1u << (iy >> 2);
      }
    }
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
  a.cyclic = (b->nx == kW && b->ny == kW) ? 1 : 0;
  a.det_bits = reinterpret_cast<const uint32_t*>(base + o_det);
  a.n_det = n_det;
  a.acc = reinterpret_cast<double*>(base + o_acc);
  CUDA_TRY(ctx, lma_dev::launch_synth(a, false, st));
  CUDA_TRY(ctx, lma_dev::launch_finalize(a.acc, nout, 1.0, out, st));
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
        hit = b->valid.empty() || !b->valid[i];
      }
      if (out_mask) out_mask[static_cast<size_t>(pb) * region->npx + pa] = hit ? 1 : 0;
      cnt += hit ? 1 : 0;
    }
  if (n_affected) *n_affected = cnt;
  return LMA_OK;
}

}  // extern "C"
