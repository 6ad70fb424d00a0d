// Internal structures of the msrc library (host planning + device kernels).
// Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "device_cache.h"
#include "msrc.h"

namespace msrc {

// Thread-local message returned by msrc_last_error (defined with the C ABI).
void set_last_error(const char* msg);

// Signal-side Farrow structure (Sec. II-B, Eq. 5): the tap weight of tap k is a
// degree-kFarrowDeg polynomial in a local variable of the fractional delay,
// piecewise over kFarrowSegs segments of [0, 1). The prefilter produces one
// signal row per (segment, power): z[s][q][m] = sum_k c[s][q][k] x[m - k],
// stored per segment as one float4 per column, {z0, z1, z2, (z3, z4)} with the
// two highest powers scaled by a power of two and rounded to half precision
// (they carry under 1 % of the value), so that one image-sample gathers its 5
// values with one 16-byte load (4 shared-memory wavefronts per warp).
constexpr int kFarrowSegs = 4;
constexpr int kFarrowDeg = 4;
constexpr int kFarrowCoef = kFarrowDeg + 1;
constexpr int kZRows = kFarrowSegs * kFarrowCoef;
static_assert(kFarrowCoef == 5 && kFarrowSegs == 4, "row layout assumes 4 segments x 5 coefficients");
// The gradient kernel needs de/dalpha, whose error grows with the degree of
// the fit's derivative; it reads its own rows of a degree-5 fit on the same
// segments (float4 row for powers 0..3, float2 row for powers 4..5).
constexpr int kGradCoef = 6;
constexpr int kGradRows = kFarrowSegs * kGradCoef;
constexpr int kMaxTaps = 64;
constexpr int kMaxScenesInline = 1;

// Error bits of the device error word.
constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrWindowClamp = 2u;
constexpr uint32_t kErrUpsampleScratch = 4u;
// Band-limited knot upsampling: largest upsampling factor and kernel half-width.
constexpr int kMaxUpsample = 512;
constexpr int kMaxUpHalfwidth = 8;
// Emission-time delays: the source path table holds kDenseOver points per
// sample (linear interpolation between them is exact to h^2 |s''| / 8).
constexpr int kDenseOver = 4;

// Per-scene description as the kernels see it. All offsets are in elements of
// the array they index. Images are stored sorted by (tier, distance at the
// middle of the trajectory); "block" = kBlockImages consecutive images of one
// tier; "tile" = consecutive output samples of one synthesis item.
struct SceneDev {
  double dims[3];
  double beta[6];
  double c, fs, duration;
  double mics[MSRC_MAX_MICS][3];
  double traj[48];
  int32_t traj_kind, n_ctrl;
  // spline source: per segment s the cubic in x = m t / duration - s (m
  // segments), traj_poly[s][coordinate][power], for the FP64 knot positions
  double traj_poly[MSRC_MAX_CTRL - 3][3][4];
  // microphone array motion: microphones at mics[m] + a(t) - a(0)
  double arr_params[48];
  double arr_duration;
  int32_t arr_moving, arr_kind, arr_n_ctrl;
  int32_t K, n_mics, n_tiers, n_images;
  int32_t tier_max_rho[MSRC_MAX_TIERS];
  int32_t tier_step[MSRC_MAX_TIERS];       // knot spacing N_t (samples)
  int32_t tier_count[MSRC_MAX_TIERS];      // images in tier
  int32_t tier_first[MSRC_MAX_TIERS];      // first sorted image of tier
  int32_t tier_intervals[MSRC_MAX_TIERS];  // J_t intervals per image (knots J_t + 1)
  int32_t tier_blocks[MSRC_MAX_TIERS];     // blocks of the tier
  int32_t block_first[MSRC_MAX_TIERS];     // first (scene-local) block of the tier
  int32_t n_blocks;                        // blocks over all tiers
  int32_t n_tiles;                         // output tiles
  int32_t tile;                            // samples per tile
  int32_t tier_block_images[MSRC_MAX_TIERS];  // images per block of the tier
  // band-limited knot upsampling (tier_up[t] > 1): records every
  // tier_step = tier_coarse / tier_up samples at virtual knots interpolated
  // from the knots (every tier_coarse samples) by a kernel of half-width
  // up_q knots; the tier's knot table starts knot_shift knots before t = 0
  int32_t tier_up[MSRC_MAX_TIERS];
  int32_t tier_coarse[MSRC_MAX_TIERS];     // knot spacing (samples); tier_step when linear
  int32_t knot_shift[MSRC_MAX_TIERS];      // up_q for band-limited tiers, else 0
  int32_t up_q;
  int32_t upw_base[MSRC_MAX_TIERS];        // first float of the tier's weight table in upw
  int64_t bl_tau_base[MSRC_MAX_TIERS];     // first double of the tier's knot delays in bl_tau
  int64_t bl_units_first[MSRC_MAX_TIERS];  // prefix over upsampled tiers of mics x images x knots
  int32_t bl_knots[MSRC_MAX_TIERS];        // knots per image in the tier's table (J_c + 1 + 2 up_q)
  // emission-time delays (delay_model 1): the source path sampled every
  // 1 / (kDenseOver fs) s from entry dense_k0 (in those units) on, n_dense
  // entries from dense_base in the dense tables
  int32_t delay_model;
  int64_t dense_base, dense_k0, n_dense;
  // the anchors' double-float operands: hi + lo of L_d, of every microphone
  // coordinate and of fs / c
  float dims_hl[3][2];
  float mics_hl[MSRC_MAX_MICS][3][2];
  float fsc_hl[2];
  int64_t img_base;                        // first entry of this scene in the image table
  int64_t master_base;                     // first entry in the per-image (lattice order) tables
  // time groups: the images are ordered separately for every group of
  // tile_group consecutive output tiles (by tier, then distance at the group's
  // middle), so that the images of a block stay close in delay over the
  // group's tiles; group g's table starts at img_base + g * n_images. Reverse
  // mode with a band-limited tier or emission-time delays uses one group
  // (tile_group >= n_tiles).
  int32_t tile_group;                      // output tiles per time group
  int32_t n_time_groups;                   // time groups of the scene
  int64_t sort_group0;                     // the scene's first group in the sort key
  int64_t gpos_base;                       // its first entry in the group position table
  int64_t knot_base[MSRC_MAX_TIERS];       // first knot position (double3) per tier
  int64_t knot_units_first[MSRC_MAX_TIERS];// prefix over tiers of (J_t + 1)
  int64_t part_base;                       // first partial-sum float
  int64_t n_in, n_out;
  int64_t z_base;                          // first column of the scene's z rows (x kFarrowSegs rows)
  int64_t z_len;                           // columns (samples) per row
  int64_t z_m0;                            // sample index of z column 0
  const float* x;
  float* y;
  // reverse mode (msrc_synthesize_backward)
  const float* dy;                         // [n_mics][n_out]
  float* dx;                               // [n_in] or null
  double* dparams;                         // [48] or null
  double* dbeta;                           // [6] or null
  double* darray;                          // [48] or null: dL/d(array trajectory parameters)
  int64_t dxb_base;                        // first float of the per-(mic, block group) dx rows
  int32_t n_groups;                        // dx block groups over all tiers
  int32_t group_first[MSRC_MAX_TIERS];     // first group of tier t
  int32_t group_blocks[MSRC_MAX_TIERS];    // blocks per group of tier t
  int32_t range_tiles;                     // tiles per dx item (tile range)
  int32_t n_ranges;                        // tile ranges
  int32_t dx_rows;                         // dx rows per (mic, group): one per range parity
  int64_t kslot_first[MSRC_MAX_TIERS];     // first knot-gradient slot of tier t (mic 0)
  int64_t kslot_mic_stride;                // slots per microphone
  int32_t kcap[MSRC_MAX_TIERS];            // knot slots per (block, tile) item of tier t
  int64_t bpart_base;                      // first float of the per-(mic, block) beta partials
  // reverse mode over tiers whose delays are not linear in the knot positions
  // (band-limited upsampling, emission-time delays): one unit per
  // (microphone, image, record knot), [mic][image][knot] from opt_units_first[t]
  int64_t opt_units_first[MSRC_MAX_TIERS];
  int64_t n_opt_units;
  float c_over_fs;                         // metres per sample of delay
  float fsc;                               // fs / c (samples of delay per metre), FP32
  double fs_over_c;                        // fs / c, FP64
};

// Tile configuration of the synthesis launch: CTA threads, 32-sample chunks per
// warp (tile = threads * chunks samples), shared z-window capacity (samples),
// shared record capacity (float2 units: one per image and knot interval, or
// with knot records one per image pair and knot), maximum images per block,
// record format (0 interval records, 1 knot records).
struct TileConfig {
  int threads, chunks, wcap, reccap, block, knots;
};
int tile_config_count();
const TileConfig& tile_config(int cfg);

// Per-kernel "units" of one scene and the prefix tables that map a global
// unit index to its scene (batched launches).
struct LaunchTables {
  const int64_t* enum_prefix;    // images
  const int64_t* knots_prefix;   // trajectory knots
  const int64_t* dx_prefix;      // input samples (reverse mode)
  const int64_t* z_prefix;       // prefilter units
  const int64_t* item_prefix;    // synthesis items
  const int64_t* red_prefix;     // reduction units
  const int64_t* bl_prefix;      // knot delays of upsampled tiers
  const int64_t* dense_prefix;   // source path table entries (emission-time delays)
  const int64_t* img_prefix;     // images (lattice order, once per scene)
  const int64_t* opt_prefix;     // reverse mode: (mic, image, record knot) units of the
                                 // upsampled and emission-time tiers
};
// Image table units of the enumeration and sort: time groups x images. Sort
// key: (scene's time group << kSortGroupShift) | (tier << 24) | distance (24 bits).
constexpr int kSortGroupShift = 26;

struct DevicePtrs {
  uint32_t* err;                 // device error word
  uint32_t* counter;             // work-queue head of the persistent synthesis launch
  uint64_t* keys_in;
  uint64_t* keys_out;
  uint32_t* vals_in;
  uint32_t* vals_out;
  void* sort_temp;
  size_t sort_temp_bytes;
  uint32_t* img_code;            // packed lattice triple and parity
  uint32_t* m_code;              // per image in lattice order: packed code,
  float* m_gain;                 //   gain beta_i / (4 pi) * fs / c,
  float4* m_off;                 //   2 n o L - m (FP32) and parity bits | tier << 4,
  int32_t* m_pos;                //   position in the first time group's sorted table
  double* gpos;                  // per (scene, time group): source position and array
                                 // displacement at the group's middle (6 doubles), sort keys
  float* img_gain;               // beta_i / (4 pi)
  double* knot_pos;              // s(t_j), 3 doubles per knot
  double* arr_pos;               // a(t_j) - a(0), 3 doubles per knot (scenes with a moving array)
  float4* knot_hl;               // s(t_j) as double-float pairs: hi (x, y, z, 0) then lo, per knot
  float4* arr_hl;                // a(t_j) - a(0) the same way (moving array)
  float4* zq;                    // prefiltered rows, [scene rows][segment][column]: forward
                                 // {z0, z1, z2, half2(s z3, s z4)}, reverse mode powers 0..3
  uint32_t* xmax;                // per scene: max |x| (float bits), scale of the half-precision powers
  float2* zg;                    // reverse mode: powers 4..5 of the degree-5 rows (zq holds 0..3)
  float* part;                   // partial sums
  // reverse mode
  float* dxb;                    // dx rows per (scene, mic, block group, range parity)
  int64_t dxb_floats;            // floats of all dx rows (zeroed before the dx launch)
  float* kslot;                  // knot-gradient slots (3 floats each)
  float* bpart;                  // beta partials (8 floats per (scene, mic, block))
  double* gk;                    // dL/ds(t_j) per tier knot (3 doubles, indexed like knot_pos)
  float* kslot_arr;              // moving arrays: knot slots of dL/da(t_j), like kslot
  double* garr;                  // moving arrays: dL/da(t_j) per tier knot, like gk
  double* ppart;                 // trajectory-parameter partials (48 doubles per (scene, knot chunk))
  float4* bwt;                   // per image: dbeta_i/dbeta_w / (4 pi) for walls 0..3 | walls 4..5, gain, 0
  float2* trange;                // reverse mode: delay range (tmin, tmax) of every (mic, block, tile) item
  // reverse mode, upsampled / emission-time tiers, per (mic, image, record knot)
  // unit: the knot delay (samples) of the gradient kernel's records, and the
  // interval's dL/dd sums toward its two knots (A to knot k, B to knot k + 1)
  double* otau;
  float2* ograd;
  float* cgrad;                  // upsampled tiers: dL/dd at the knots, [knot][mic x image] from bl_tau_base[t]
  // band-limited knot upsampling: per (scene, tier) a table of tier_up rows
  // of 2 up_q + 1 floats, row p = the normalised kernel weights of knots
  // j0 - up_q + 1 .. j0 + up_q at the virtual knot p / tier_up past knot j0,
  // then their first moment sum_i w_i (i - up_q + 1)
  const float* upw;
  // and the delay tau = d fs / c of every (microphone, image, knot) of an
  // upsampled tier as a double-float pair, [mic][image][knot] from bl_tau_base[t]
  float2* bl_tau;
  // emission-time delays: the source path every 1 / (kDenseOver fs) s as the
  // FP32 pair hi + lo of each coordinate
  float4* dense_hi;
  float4* dense_lo;
};
constexpr int kParamPartialsPerScene = 128 * 48;

constexpr int kUnitKinds = 10;

struct KernelArgs {
  SceneDev scene0;               // used when n_scenes == 1
  const SceneDev* scenes;        // used when n_scenes > 1
  int32_t n_scenes;
  int64_t totals[kUnitKinds];    // total units per kernel kind (enum, knots, rec, z, item, red, bl, dense,
                                 // img, opt)
  LaunchTables tab;
  DevicePtrs p;
  float farrow[kFarrowSegs][kFarrowCoef][kMaxTaps];  // coefficients c[s][q][k + L/2] of the powers of w
  float farrow_g[kFarrowSegs][kGradCoef][kMaxTaps];  // degree-5 coefficients (gradient kernel)
  int32_t taps;
  float zh_gain;                 // max over segments of sum_k |c_q[k]| (q = 3, 4): z bound per unit |x|
  int64_t n_sort_groups;         // time groups over all scenes (the sort key's leading field)
  int32_t max_time_groups;       // largest time-group count of one scene
  uint32_t test_extra_tx;        // test hook: bytes a window staging expects beyond its copies (0)
  int32_t want_array;            // reverse mode: some scene asks for dL/d(array trajectory)
};
// passed by value as a __grid_constant__ kernel parameter
static_assert(sizeof(KernelArgs) <= 32000, "kernel parameter space");

// Image code: n_d + 64 in 7 bits each, parity bits above.
__host__ __device__ inline uint32_t pack_image(int nx, int ny, int nz, int pbits) {
  return uint32_t(nx + 64) | (uint32_t(ny + 64) << 7) | (uint32_t(nz + 64) << 14) |
         (uint32_t(pbits) << 21);
}
__host__ __device__ inline void unpack_image(uint32_t code, int n[3], int p[3]) {
  n[0] = int(code & 127u) - 64;
  n[1] = int((code >> 7) & 127u) - 64;
  n[2] = int((code >> 14) & 127u) - 64;
  p[0] = int((code >> 21) & 1u);
  p[1] = int((code >> 22) & 1u);
  p[2] = int((code >> 23) & 1u);
}

// Shared-memory scratch (floats) of the band-limited record builder for `cnt`
// images, nk virtual knots and nj knot intervals: the anchor, the chord rows
// and the relative delays.
__host__ __device__ inline int64_t bl_scratch_floats(int cnt, int nk, int nj, int Q) {
  return int64_t(cnt) * (1 + nj * (2 * Q + 2) + nk);
}

// Grid of a persistent kernel on the current device (SMs x resident CTAs of
// `threads` threads and `smem` bytes of dynamic shared memory), with the
// kernel's dynamic shared-memory limit raised to `smem`: set up once per device
// and kernel (one PerDevice per kernel instantiation), thread-safe.
template <typename K>
cudaError_t persistent_grid(PerDevice& cache, K kern, int threads, size_t smem, int* grid) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaError_t ie = cudaSuccess;
  const int st = cache.get(
      dev,
      [&](int* v) {
        ie = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (ie != cudaSuccess) return 1;
        int sms = 0, occ = 0;
        ie = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (ie != cudaSuccess) return 1;
        ie = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
        if (ie != cudaSuccess) return 1;
        *v = sms * (occ > 0 ? occ : 1);
        return 0;
      },
      grid);
  if (st == -1) return cudaErrorInvalidDevice;
  if (st != 0) return ie != cudaSuccess ? ie : cudaErrorUnknown;
  return cudaSuccess;
}

// Launch entry points (defined in the .cu files).
cudaError_t launch_setup(const KernelArgs& a, cudaStream_t s);
// Reverse-mode tile configuration (threads = tile samples, one per thread).
const TileConfig& backward_tile_config();
// Shared-memory floats both reverse-mode kernels give the band-limited record
// builder's scratch.
int64_t backward_bl_scratch_floats();
cudaError_t launch_forward(const KernelArgs& a, int tile_config, cudaStream_t s,
                           cudaEvent_t* ev /* nullable: [after prefilter, after synthesis] */);
size_t sort_temp_bytes(int64_t n_items, int end_bit);
cudaError_t launch_sort(const KernelArgs& a, int64_t n, int end_bit, cudaStream_t s);

}  // namespace msrc
