// Internal interface between the host library (lma_host.cpp) and the CUDA
// kernels (lma_kernels.cu). Not part of the public C-ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lma_dev {

constexpr int kW = 128;              // propagation window W = detection window D
constexpr int kThreads = 512;        // threads per CTA of the FFT kernels
constexpr int kMaxTerms = 4;
constexpr int kMaxDet = 4;

// Step a1: projected potential and transmission of one configuration.
struct PotArgs {
  const float2* ax;            // atom x (Angstrom) in [0, l_x), sorted by slice, as an exact
                               // pair x = hi + lo of the FP64 value (lo = fp32(x - hi))
  const float2* ay;            // atom y in [0, l_y), the same form
  const int16_t* asp;          // species
  const int32_t* slice_start;  // [n_slices + 1]
  const float* peak;           // [n_species] V*Angstrom
  int n_species;
  int n_terms;
  float frac[kMaxTerms];
  float inv2w2[kMaxTerms];     // 1 / (2 w^2)
  float rc2;                   // r_cut^2
  int nx, ny, n_slices;
  float dx_hi, dx_lo, dy_hi, dy_lo;          // the pixel pitch as hi + lo
  float lx_hi, lx_lo, ly_hi, ly_lo;          // the periods as hi + lo
  float c75x_hi, c75x_lo, c75y_hi, c75y_lo;  // 7.5 dx and 7.5 dy (tile centre to pixel 0) as hi + lo
  float limx, limy;            // r_cut + 8 dx (8 dy) rounded up: an atom farther from the tile
                               // centre on either axis reaches none of its pixels
  float sigma;
  int rx0, ry0, rw, rh;        // pixel rectangle to (re)build, may wrap; full grid = (0,0,nx,ny)
  float2* t;                   // [n_slices][ny][nx]
};

// Step a3: multislice of lattice translates on W x W windows. One job = one
// specimen and basis; a launch covers the items of up to kMaxJobs jobs.
constexpr int kMaxJobs = 8;

struct SliceJob {
  const float2* t;             // [slots][n_slices][ny + W][nx + W] (periodic halo of W pixels)
  int nx, ny, n_slices;
  size_t t_slot;               // elements of one configuration's transmission stack
  const float2* uW;            // [W][W] input wave, centre at (W/2, W/2)
  int n_translates;            // |I_f|
  size_t u_slot;               // elements (waves x W x W) of one configuration's exit-wave store
  int lat_ox, lat_oy, lat_sx, lat_sy, lat_nax;   // I_f: pos(a, b) = (ox + a sx, oy + b sy)
  float2* U;                   // [slots][n_translates][W][W] complex64 store, or
  void* Uh;                    // [slots][n_translates][W][W] FP16 pairs (mixed store) with
  float* Uscale;               // [slots][n_translates] power-of-two factor restoring each wave
  const float2* ex;            // [W] exp(-i pi lambda eps kx^2) / W^2
  const float2* ey;            // [W] exp(-i pi lambda eps ky^2)
  int r2max;                   // bandlimit: m'^2 + n'^2 <= r2max
  float tc_in, tc_out;         // tensor-core DFT (k_slice_tc): power-of-two factor of the input
                               // wave, and its inverse applied to the exit wave
  int W;                       // window of this job (kW, or 64 / 256 for k_slice_64 / k_slice_256); uW, the
                               // store entries and ex, ey have this size
};

// How the CTAs of a slice launch take their items.
enum SliceMode : int {
  kSliceOnePerItem = 0,        // grid = items, the hardware schedules the CTAs
  kSlicePersistent = 1,        // one CTA per SM, item li = blockIdx + k * gridDim
  kSliceDynamic = 2,           // one CTA per SM, items fetched from an atomic counter
  kSliceModes = 3
};

struct SliceLaunch {
  SliceJob job[kMaxJobs];
  int start[kMaxJobs + 1];     // list[start[j] .. start[j + 1]) holds job j's items
  int n_jobs;
  const int32_t* list;         // items slot * n_translates + translate
  const int32_t* out_index;    // null: item i's wave goes to store entry `translate`; else to
                               // entry out_index[i] of its slot (bounded store of a partition)
  int n_list;
  int* counter;                // kSliceDynamic: zeroed before the launch
  int* status;                 // k_slice_tc: set to 1 when a bounded tensor-core wait gives up
};

// Steps a4-a6: synthesis, detector reading, FP64 accumulation over configurations.
struct SynthArgs {
  const float2* U;             // [n_translates][W][W] complex64 store, or
  const void* Uh;              // FP16 pairs (mixed store) with
  const float* Uscale;         // per-wave factors
  const int32_t* tidx;         // [n_probes][L]
  const float2* alpha;         // [n_probes][L]
  const int2* shift;           // [n_probes][L] placement of U in the probe window
  int L;
  int n_probes;                // probes of the region (stride of the accumulator)
  const int32_t* probe_list;   // null: every region probe, walked in strips (tables indexed by p);
  int n_list;                  // else these n_list probes (tables indexed by list position)
  int npx, npy;                // region shape: probe p = b * npx + a
  int strip;                   // probes are visited in vertical strips of this many columns
  int n_cfg;                   // configurations in this launch (store slots 0..n_cfg-1)
  int cfg_base;                // index of slot 0's configuration in the accumulator
  int n_translates;            // |I_f| (stride of the per-wave factors between slots)
  size_t u_slot;               // elements of one slot of the exit-wave store
  int cyclic;                  // windows are the whole periodic grid (then W = D = kW)
  int W;                       // exit-wave window (row length of the store), 64..256; the
                               // probe window D is kW
  const uint32_t* det_bits;    // [n_det][kThreads] detector bits in C layout
  int n_det;                   // annuli: detectors; labels: labels (outputs per probe)
  double* acc;                 // [configuration][n_det][n_probes] readings (assigned)
  // kReadLabels: pixel lists of the labels (3D STEM rings), CSR over pixel ky * W + kx
  const int32_t* lab_start;    // [n_det + 1]
  const int32_t* lab_pix;      // ascending pixel indices of each label
  // kReadPattern: |DFT|^2 / W^2 at |kx| <= pat_a, |ky| <= pat_b (4D STEM), zero outside
  // the band kx^2 + ky^2 <= band_r2, FP32 per configuration slot
  float* pat;                  // [slot][n_probes][2 pat_b + 1][2 pat_a + 1]
  int pat_a, pat_b;
  int band_r2;
};

// Readouts of the synthesis kernel.
enum ReadMode : int {
  kReadAnnuli = 0,             // up to kMaxDet 2D STEM annuli (bit masks)
  kReadLabels = 1,             // disjoint labelled pixel sets (3D STEM rings), deterministic sums
  kReadPattern = 2             // the diffraction pattern on a centred crop (4D STEM)
};

// Scratch of the no-allocation readout: a file-scope device array of this size
// on each device; noalloc_scratch() returns its device address for the current device.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;
cudaError_t noalloc_scratch(void** ptr);

cudaError_t init_device_constants();
size_t slice_smem_bytes();
size_t synth_smem_bytes();
cudaError_t launch_potential(const PotArgs& a, cudaStream_t s);
// even_origins: every translate of the list has an even window x origin (16-byte staging);
// half: write the FP16 store (Uh, Uscale) instead of the complex64 one; mode: SliceMode
// (kSliceDynamic zeroes a.counter on the stream first)
cudaError_t launch_slice(const SliceLaunch& a, bool even_origins, bool half, int mode, cudaStream_t s);
int sm_count();
// step a3 with the 32-point DFT passes as split-FP16 tensor-core products (complex64 store):
// persistent CTAs, one per SM; a.status must be set
cudaError_t launch_slice_tc(const SliceLaunch& a, bool even_origins, cudaStream_t s);
size_t slice_tc_smem_bytes();
// step a3 on W = 64 or W = 256 windows (every job of the launch has that W), complex64 store:
// persistent CTAs (two per SM at W = 64, one at W = 256); W = 256 needs
// slice_gen_scratch_bytes(256) of scratch
cudaError_t launch_slice_gen(const SliceLaunch& a, int W, float2* scratch, cudaStream_t s);
size_t slice_gen_scratch_bytes(int W);
// one warp runs the bounded mbarrier wait of the tensor-core (which = 0) or W = 256 (which = 1)
// slice kernel on a phase that never completes; *status |= 1 when it gives up
cudaError_t launch_selftest_wait(int which, int* status, cudaStream_t s);
// synthesis grid: kSynthGridAuto (persistent for the complex64 store, one CTA per item for the
// FP16 store), one CTA per item, or persistent (one CTA per SM); every grid gives the same bits
constexpr int kSynthGridAuto = 0, kSynthGridPerItem = 1, kSynthGridPersistent = 2;
cudaError_t launch_synth(const SynthArgs& a, bool half, int mode, int grid_mode, cudaStream_t s);

// Step a4 for groups of neighbouring probes (probe_list null, non-periodic placement): each
// CTA takes gx x gy probes of the region, forms the union of their (translate, placement)
// pairs in ascending translate order and writes Psi_p = sum_j alpha_j U_{i_j} of every probe
// of the group into psi, loading each exit-wave element once for all the group's probes that
// use it. Each probe's terms are summed in ascending translate index, as k_synth_detect does
// with tables sorted that way, so a detection pass over psi (launch_synth with the identity
// tables below) gives the same bits as the per-probe gather.
struct GroupArgs {
  int gx, gy;                  // probes per group along x and y: gx gy <= 4, gx gy L <= 512
  int psx, psy;                // probe spacing (pixels): offset between neighbouring probe windows
  int ngx, ngy;                // groups per region row; group rows of this launch
  int gb_base;                 // first group row of this launch
  int gstrip;                  // groups are visited in vertical strips of this many columns
  int cfg;                     // store slot read
  float2* psi;                 // probe waves of the launch's probe rows, [probe - gb_base gy npx][kW][kW]
};
constexpr int kGroupMaxEntries = 512;  // (probe, wave) entries of one group
constexpr int kGroupDenseProbes = 4;   // probes per group of the kernel's accumulators (gx gy <= 4)
constexpr int kGroupPosBias = 2048;   // translate placements in a group's frame lie in [-2048, 2048)
size_t synth_group_smem_bytes();
// grid_mode as for launch_synth (kSynthGridAuto: persistent)
cudaError_t launch_synth_group(const SynthArgs& a, const GroupArgs& g, bool half, int grid_mode, cudaStream_t s);
// tables of the detection pass over psi: tidx[i] = i, alpha[i] = 1, shift[i] = 0, i < n
cudaError_t launch_identity_tables(int n, int32_t* tidx, float2* alpha, int2* shift, cudaStream_t s);
// step a3 with the propagation as a periodic convolution with the K1 x K2 kernel q (device,
// [K2][K1] complex64, offsets -(K/2) .. K/2); K1 in {3, 5, ..., 13}, K2 odd <= 25; complex64 store
cudaError_t launch_slice_rs(const SliceLaunch& a, const float2* q, int K1, int K2, cudaStream_t s);
// out[i] = sum over variants v (in order) of w[v] * sum over n_cfg slots (in order) of
// acc[(v * n_cfg + c) * n + i]; w has n_var entries on the device
cudaError_t launch_finalize_variants(const double* acc, int64_t n, int n_cfg, int n_var, const double* w, double* out,
                                     cudaStream_t s);
// acc[i] (+)= sum over n_cfg slots (in slot order) of slots[c * n + i]; first: assign
cudaError_t launch_pattern_accumulate(const float* slots, int64_t n, int n_cfg, bool first, double* acc,
                                      cudaStream_t s);
// out[i] = scale * acc[i] as float
cudaError_t launch_pattern_finalize(const double* acc, int64_t n, double scale, float* out, cudaStream_t s);
// complex64 copy of one wave of the FP16 store
cudaError_t launch_expand_half(const void* src, float scale, float2* dst, cudaStream_t s);
// out[i] = scale * sum over n_cfg slots (in slot order) of acc[c * n + i]
cudaError_t launch_finalize(const double* acc, int64_t n, int n_cfg, double scale, double* out,
                            cudaStream_t s);

}  // namespace lma_dev
