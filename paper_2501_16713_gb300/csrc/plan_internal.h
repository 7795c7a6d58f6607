// Host-side plan structure and kernel launchers (internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

namespace nrs {

struct TilePlan {
  int t0, t1, t2;       // tile size (grid points per axis)
  int nt0, nt1, nt2;    // tiles per axis (last tile may be ragged)
  long long ntiles;
};

// Sorted points of one gridding problem (one k-space phase, or all displaced
// voxels of all phases for the image-space adjoint).
struct PointSet {
  long long npts = 0;
  TilePlan tp{};                // tiles of this set's spreading/interpolation
  float4* qs = nullptr;         // sorted: (f0, f1, f2, packed base bits)
  int32_t* perm = nullptr;      // sorted index -> value row
  // spreading: per-tile halo lists of (sorted index, value row)
  int2* list = nullptr;
  SpreadItem* items = nullptr;  // heaviest first
  int32_t* bins = nullptr;      // per item: W + T + 1 plane-offset bin starts (relative)
  // 8^3 tiles, W = 4: the list with every item's entries ordered by footprint
  // class (4^3 sub-blocks touched), and kCubeBins class starts per item
  int2* clist = nullptr;
  int32_t* cbins = nullptr;
  int n_items = 0;
  ReduceItem* reduces = nullptr;
  int n_reduces = 0;
  int n_slots = 0;              // partial tiles needed in scratch
  int n_occupied = 0;           // tiles with at least one point in their halo lists
  long long list_len = 0;
  // interpolation: sorted ranges of the points whose first tap lies in a tile
  SpreadItem* iitems = nullptr;
  int n_iitems = 0;
};

}  // namespace nrs

struct nrsense_cg_ws;  // CG workspace (solver.cu)
struct nrsense_fista_ws;  // FISTA workspace (fista.cu)
struct nrsense_motion_ws;  // density compensation / weighted adjoint workspace (motion.cu)
struct nrsense_cnn_s;  // preconditioner network (cnn.cu)

struct nrsense_plan_s {
  nrsense_desc desc{};
  nrs::Geo geo{};
  int P = 0, C = 0, W = 0;
  double beta = 0.0;
  nrs::KernelCoefs kc{};
  double poly_err = 0.0;
  bool identity_warp = false;

  // tables
  float* deapod = nullptr;       // 1/C(m/G) for m in [-N/2, N/2), per axis, offsets 0, n0, n0+n1
  float* disp = nullptr;         // (P, 3, nvox)
  nrsense_c64* smaps = nullptr;  // (C, nvox) coil-major

  // k-space
  std::vector<long long> M, off;
  long long Mtot = 0;
  std::vector<nrs::PointSet> kpts;  // per phase
  nrs::PointSet ipts;               // displaced voxels of all phases
  nrs::HomeSet ihome{};             // the same, sorted by 8^3 home tile (home-tile spread)
  bool home_ok = false;             // ihome built (W = 4, not compensated)
  bool interp_home = false;         // image-space interpolation over super-tiles (autotuned)
  nrsense_c64* home_scratch = nullptr;  // super-tile rims of the home-tile spread
  nrs::TilePlan ktiles{}, itiles{};  // k-space and image-space tiles
  int phase_chunk = 1;              // phases per launch

  // work buffers
  nrsense_c64* b_xhat = nullptr;   // N^3
  nrsense_c64* b_upad = nullptr;   // G^3, zero outside the K_N block
  nrsense_c64* b_ugrid = nullptr;  // G^3
  nrsense_c64* b_m = nullptr;      // P * N^3
  // coil grids of one phase chunk, (phase_chunk * C) x G^3 each
  // coil grids, phase_chunk * C * G^3 values each, complex FP32 or (grid_bf16)
  // complex BF16
  void* b_xpad = nullptr;     // zero outside the centred N^3 blocks
  void* b_xwork = nullptr;    // FFT outputs
  void* b_xspread = nullptr;  // spread target; tiles no phase occupies stay zero
  void* b_xmid = nullptr;     // forward FFT after the 2D step; planes off the data blocks stay zero
  bool grid_bf16 = false;     // desc.precision == NRSENSE_BF16_STORE
  int spread_variant = 1;     // kSpreadRegister or kSpreadShared (autotuned)
  int interp_coils = 8;       // coils per interpolation CTA (autotuned)
  int spread_image_variant = 2;  // image-space spread: kSpreadShared (CTA per tile),
                                 // kSpreadRegisterWarp (CTA per plane pair) or kSpreadHome
                                 // (home tiles, spread_home.cu) (autotuned)
  bool interp_tma = false;    // TMA-staged interpolation (autotuned; needs tma_ok)
  bool tma_ok = false;        // tensor maps of b_xwork built
  long long tma_poll_limit = -1;  // polls of the halo wait before ERR_TIMEOUT (-1: the
                                  // kernel's own limit; NRSENSE_TMA_POLL_LIMIT at plan time)
  CUtensorMap tmap_xwork4{}, tmap_xwork8{}, tmap_xwork2{};  // boxes of 4, 8, 2 coil grids
  bool comp_spread = false;   // desc.precision == NRSENSE_FP32_COMPENSATED
  nrsense_c64* b_y = nullptr;      // Mtot * C
  nrsense_c64* b_tmp = nullptr;    // N^3 (normal operator scratch)
  nrsense_c64* b_scratch = nullptr;  // partial tiles
  long long scratch_elems = 0;
  int32_t* d_status = nullptr;

  cufftHandle fft_n = 0, fft_g = 0;
  bool have_fft_n = false, have_fft_g = false;
  // k-space coil-grid FFTs, pruned to the zero padding: per batch of grids,
  // 2D transforms over the z-plane blocks that can hold data (the centred
  // n0 planes: the top n0/2 planes of grid k and the bottom n0/2 of grid k+1
  // are contiguous; fft_p2 takes n0 planes, fft_p2h n0/2 at the two ends) and
  // a strided 1D transform along z per grid (fft_z).  The forward direction
  // goes 2D (into b_xmid, whose other planes stay zero) then z; the inverse
  // z then 2D in place on the planes the crop reads.
  cufftHandle fft_p2 = 0, fft_p2h = 0, fft_z = 0;
  bool have_gc = false;


  long long device_bytes = 0;
  std::vector<void*> allocations;
  std::vector<size_t> allocation_bytes;  // size of each entry of allocations
  std::vector<char> kunion;              // k-space tiles written by the spread (plan time)
  int spread_max_item = 1024;            // list entries per k-space spreading work item

  // stage profiling (nrsense_profile_start/stop)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_events;  // pairs
  std::vector<int> prof_stage;           // stage of each recorded pair
  long long launches = 0;                // own kernels launched (always counted)
  long long launches_at_start = 0;

  // own pruned coil-grid transforms with the coil fan-out and combination fused
  bool fft_pruned_ok = false;  // supported: sigma 2, power-of-two grids of 32..256, FP32 grids
  bool fft_pruned = false;     // chosen (else cuFFT plus the K5 / K8 kernels)
  // image-space G^3 transforms of T / T^H by the pruned passes (scratch in
  // b_upad, whose zero padding the cuFFT path then has to restore)
  bool image_fft_ok = false;
  bool image_fft_pruned = false;
  bool upad_dirty = false;
  bool pad_dirty = false;      // b_xpad / b_xmid hold the pruned transforms' intermediates
  // k-space tiles written by the spread (the union over phases), as one
  // 32-bit mask over axis-0 tiles per (axis-1, axis-2) tile column; null when
  // axis 0 has more than 32 tiles.  Tiles outside it are zero in the spread
  // target and never read by the interpolation.
  uint32_t* kcolmask = nullptr;
  double kcol_fraction = 1.0;  // tile columns with at least one such tile
  double kuni_fraction = 1.0;  // tiles of the union

  // reduction of the phase sum over ranks that hold the other motion states
  // (nrsense_plan_set_reduce); null: this plan holds every state
  nrsense_reduce_fn reduce_fn = nullptr;
  void* reduce_user = nullptr;
  nrsense_cg_ws* cg = nullptr;  // allocated by the first nrsense_solve_cg
  // bumped whenever a device buffer or launch choice that a captured solver
  // graph bakes in may have changed (tuning, re-tiling, reduction hook,
  // deflation space, solver workspace reallocation): graphs are re-captured
  uint64_t epoch = 0;
  // circulant preconditioner (nrsense_set_circulant, solver.cu)
  float* circ_d = nullptr;          // per frequency (DFT order): 1 / (max(Re hhat, 0) + lambda)
  nrsense_c64* circ_tmp = nullptr;  // image-sized work vector
  cufftHandle fft_circ = 0;
  bool have_fft_circ = false;
  bool circ_on = false;
  // recycled deflation space (nrsense_set_deflation, solver.cu): W, E0 W and
  // E W (k image vectors each, E W for defl_lambda), the k x k FP64 Gram
  // matrices W^H E0 W and W^H W (host), E_c^-1 and the projection
  // coefficients (device, complex FP64), dot-product partial sums
  int defl_k = 0;
  nrsense_c64* defl_w = nullptr;
  nrsense_c64* defl_e0w = nullptr;
  nrsense_c64* defl_ew = nullptr;
  double defl_lambda = -1.0;  // lambda of defl_ew and defl_ecinv (< 0: not formed)
  std::vector<double> defl_g0, defl_gw;  // k x k complex, row-major, (re, im) pairs
  double* defl_ecinv = nullptr;          // k x k complex
  double* defl_coef = nullptr;           // k complex
  double* defl_partial = nullptr;        // 2 k x kDeflBlocks
  nrsense_fista_ws* fista = nullptr;  // allocated by the first FISTA or power-iteration call
  nrsense_motion_ws* motion = nullptr;  // allocated by the first DCF or weighted-adjoint call
};

namespace nrs {
// RAII stage marker: records an event pair around a stage when profiling.
struct StageMark {
  nrsense_plan_s* p;
  cudaStream_t s;
  int pair = -1;
  StageMark(nrsense_plan_s* plan, int stage, cudaStream_t stream) : p(plan), s(stream) {
    if (p->prof_on && p->prof_stage.size() * 2 + 2 <= p->prof_events.size()) {
      pair = int(p->prof_stage.size());
      p->prof_stage.push_back(stage);
      cudaEventRecord(p->prof_events[2 * pair], s);
    }
  }
  ~StageMark() {
    if (pair >= 0) cudaEventRecord(p->prof_events[2 * pair + 1], s);
  }
};
}  // namespace nrs

namespace nrs {

// ---- preconditioner network (cnn.cu) --------------------------------------
long long cnn_nvox(const nrsense_cnn_s* net);
bool cnn_shape_matches(const nrsense_cnn_s* net, int n0, int n1, int n2);
uint64_t cnn_serial(const nrsense_cnn_s* net);  // unique per created network (0: none)
// z = M(r) on stream s, no host synchronisation; sumsq_dev (may be null) is an
// FP64 sum of |r|^2 already on the device.  Returns the kernels launched.
long long cnn_apply_async(nrsense_cnn_s* net, const float2* r, const double* sumsq_dev, float2* z,
                          cudaStream_t s);

// ---- launchers (kernels_*.cu) -------------------------------------------
// image space
int launch_deapod_pad(const Geo& g, const float* deapod, const nrsense_c64* xhat,
                       nrsense_c64* upad, cudaStream_t s);
int launch_crop_deapod(const Geo& g, const float* deapod, const nrsense_c64* ufreq,
                        nrsense_c64* xhat, cudaStream_t s);
int launch_interp_image(const Geo& g, int W, const KernelCoefs& kc, int P,
                         const float* disp, const nrsense_c64* u, nrsense_c64* m,
                         cudaStream_t s);
int launch_axpby(long long n, const nrsense_c64* x, float a, nrsense_c64* y, float b,
                  cudaStream_t s);
int launch_copy_phases(const Geo& g, int P, const nrsense_c64* x, nrsense_c64* m,
                        cudaStream_t s);
int launch_sum_phases(const Geo& g, int P, const nrsense_c64* m, nrsense_c64* x,
                       cudaStream_t s);

// k space
// Coil grids are complex FP32 (bf16 == false) or complex BF16 (bf16 == true).
int launch_coil_fanout_pad(const Geo& g, int C, int nph, const float* deapod,
                           const nrsense_c64* smaps, const nrsense_c64* m, void* xpad, bool bf16,
                           cudaStream_t s);
int launch_image_to_padded(const Geo& g, int C, const float* deapod, const nrsense_c64* v,
                           void* xpad, bool bf16, cudaStream_t s);
// coil_chunk: coils per CTA (8 or 4; W = 4 and C > 4 only, else ignored);
// tmap (may be null): tensor map of `grids` with a box of coil_chunk coils,
// which selects the TMA-staged kernel (W = 4); status receives a timeout.
int launch_interp_kspace(const Geo& g, int W, const KernelCoefs& kc, int C, const TilePlan& tp,
                         const PhaseTable& pt, const void* grids, bool bf16, nrsense_c64* y,
                         int coil_chunk, const CUtensorMap* tmap, int32_t* status,
                         cudaStream_t s, long long poll_limit = -1);
// Tensor map of `slots` consecutive coil grids at base ([slot][G0][G1][G2]
// values) with a halo box of 12 x 11 x 11 values x coil_chunk grids.
// cuTensorMapEncodeTiled through the runtime's driver entry point (null if unavailable)
void* tensor_map_encoder();
bool make_grid_tensor_map(CUtensorMap* m, const void* base, const Geo& g, long long slots,
                          bool bf16, int coil_chunk);
// one-time kernel attributes (large dynamic shared memory); plan time
cudaError_t configure_kernels();
cudaError_t configure_spread_kernels();
int launch_crop_coilsum(const Geo& g, int C, int nph, const float* deapod,
                        const nrsense_c64* smaps, const void* xg, bool bf16, nrsense_c64* w,
                        cudaStream_t s);
int launch_crop_to_coils(const Geo& g, int C, const float* deapod, const void* xg, bool bf16,
                         nrsense_c64* v, cudaStream_t s);

// spreading (both domains)
// Spread the phases of `pt` (values at rows row0[jj] + perm of vals) into
// consecutive grid slots (phase jj at grids + jj * C * G^3); comp selects
// compensated accumulation (W = 4 kernels); variant selects register or
// shared-memory accumulation for the multi-coil W = 4 kernel (register
// accumulation with a CTA per tile, or with a CTA per tile plane).
constexpr int kSpreadRegister = 1, kSpreadShared = 2, kSpreadRegisterWarp = 3, kSpreadMMA = 4,
              kSpreadHome = 5;
// a spread variant value carries, in bits 8-15, the warps per CTA of the
// tensor-core kernel (1, 2 or 4; 0 means 1) and, in bit 16, its geometry
// (0: a warp per tile plane, 1: a warp per 4^3 sub-block)
inline int spread_base(int v) { return v & 0xff; }
inline int spread_mma_wpc(int v) { return ((v >> 8) & 0xff) ? ((v >> 8) & 0xff) : 1; }
inline bool spread_mma_cube(int v) { return ((v >> 16) & 1) != 0; }
inline int spread_mma_variant(int wpc, bool cube = false) {
  return kSpreadMMA | (wpc << 8) | (cube ? 1 << 16 : 0);
}
int launch_spread(const Geo& g, int W, const KernelCoefs& kc, int C, const TilePlan& tp,
                  const PhaseTable& pt, const nrsense_c64* vals, void* grids, bool bf16,
                  bool comp, int variant, nrsense_c64* scratch, int32_t* status, cudaStream_t s);
// coils handled by one spreading CTA
int spread_coil_chunk(int C);
// home-tile image-space spread (spread_home.cu): all points of `hs` (values at
// rows perm of vals) into grid; scratch holds home_scratch_elems(hs) values.
// Returns the kernels launched.
int launch_spread_home(const Geo& g, const KernelCoefs& kc, const HomeSet& hs,
                       const nrsense_c64* vals, nrsense_c64* grid, nrsense_c64* scratch,
                       cudaStream_t s);
long long home_scratch_elems(const HomeSet& hs);
// image-space interpolation over the same super-tiles (spread_home.cu): m rows
// perm of the home set's points, all phases
int launch_interp_home(const Geo& g, const KernelCoefs& kc, const HomeSet& hs,
                       const nrsense_c64* u, nrsense_c64* m, cudaStream_t s);
cudaError_t configure_home_kernels();
// own pruned coil-grid transforms (fft_pruned.cu).  Forward: grid slots
// jj * C + c of phases jj < nph = DFT3(S_c m_jj / C3 zero-padded), through the
// intermediates t1 (slots x N0 x N1 x G2) and t2 (slots x N0 x G1 x G2).
// Inverse: w_jj = C3^-1 sum_c conj(S_c) crop(IDFT3(grid slot jj * C + c)).
// Each returns the number of kernels launched.
bool pruned_fft_supported(const Geo& g, int C, bool bf16);
bool pruned_image_fft_supported(const Geo& g);
int launch_pruned_image_forward(const Geo& g, const float* deapod, const nrsense_c64* xhat,
                                void* t1, void* t2, nrsense_c64* ugrid, cudaStream_t s);
int launch_pruned_image_adjoint(const Geo& g, const float* deapod, const nrsense_c64* ugrid,
                                void* t2, void* t1, nrsense_c64* xhat, cudaStream_t s);
cudaError_t init_pruned_fft();
int launch_pruned_forward(const Geo& g, int C, int nph, const uint32_t* colmask,
                          const float* deapod,
                          const nrsense_c64* smaps, const nrsense_c64* m, void* t1, void* t2,
                          void* grid, cudaStream_t s);
int launch_pruned_inverse(const Geo& g, int C, int nph, const uint32_t* colmask,
                          const float* deapod,
                          const nrsense_c64* smaps, const void* grid, void* t2, void* t1,
                          nrsense_c64* w, cudaStream_t s);
// rebuild the k-space spreading work items of every phase with at most
// max_item list entries per item (plan.cu; the lists of split tiles are
// re-dealt, the sorted points stay) and grow the split-tile scratch if needed
nrsense_status retile_kspace(nrsense_plan_s* p, int max_item, cudaStream_t s);
// free the CG workspace of a plan (solver.cu)
void cg_release(nrsense_plan_s* p);
// free the FISTA workspace of a plan (fista.cu)
void fista_release(nrsense_plan_s* p);
// free the motion-capture workspace of a plan (motion.cu)
void motion_release(nrsense_plan_s* p);
// point table of one phase of the k-space point sets, rows relative to the
// phase's first sample (apply.cu)
PhaseTable kspace_phase_table(const nrsense_plan_s* p, int phase, bool spread);
// tile edge of a point set: 16 for the single-channel W=4 spread (image
// space) on grids of at least 16 + W - 1 points per axis, 8 otherwise
int spread_tile_edge(int W, int C, int gmin);
constexpr int kSpreadTile = 8;
// largest number of list entries one spreading work item processes (heavier
// tiles are split and their partial tiles summed): k space, and the image
// space, whose 16^3 tiles hold a few thousand entries each and whose
// single-channel partial sums cost more than the longer items (measured)
constexpr int kSpreadMaxItem = 1024;
constexpr int kSpreadMaxItemImage = 4096;
// largest number of points one interpolation CTA processes
constexpr int kInterpMaxItem = 1024;

}  // namespace nrs
