// Setup kernels of the synthesis path:
//   k_group_pos    source position at the middle of every time group (sort keys)
//   k_images       per image: code, gain and offset from the microphone
//   k_enumerate    image set of every scene (Sec. II-A, Eq. 1; lattice |n|_1 <= K,
//                  8 parities), one copy per time group of the scene, with a sort
//                  key (scene and time group, tier, distance at the group's middle)
//   (radix sort)   images ordered by key
//   k_image_table  per time group: packed image codes and gains beta_i / (4 pi) * fs / c
//   k_traj_knots   source position s(t_j) (and the array displacement a(t_j) - a(0)
//                  when the microphones move) at every knot of every tier, FP64
//                  (Sec. II-C: trajectory sampled at the tier's spatial rate)
#include <cub/device/device_radix_sort.cuh>

#include "msrc_internal.h"
#include "synth_common.cuh"

namespace msrc {
namespace {

__device__ __forceinline__ int locate(const KernelArgs& a, const int64_t* prefix, int64_t gid,
                                      int64_t* local) {
  if (a.n_scenes == 1) { *local = gid; return 0; }
  int s = find_scene(prefix, a.n_scenes, gid);
  *local = gid - prefix[s];
  return s;
}

__device__ __forceinline__ int tier_of(const SceneDev& S, int rho) {
  for (int t = 0; t < S.n_tiers; ++t)
    if (rho <= S.tier_max_rho[t]) return t;
  return S.n_tiers - 1;
}

// Source position and array displacement at the middle of every time group
// (FP64), for the sort keys: thread x of block row y = group x of scene y.
__global__ void k_group_pos(const __grid_constant__ KernelArgs a) {
  const int s = blockIdx.y;
  const int grp = blockIdx.x * blockDim.x + threadIdx.x;
  const SceneDev& S = scene_of(a, s);
  if (grp >= S.n_time_groups) return;
  double tm = 0.5 * S.duration;  // one group: the middle of the trajectory
  if (S.n_time_groups > 1) {
    const int64_t a0 = int64_t(grp) * S.tile_group * S.tile;
    const int64_t a1 = min(int64_t(grp + 1) * S.tile_group * S.tile, S.n_out);
    tm = 0.5 * double(a0 + a1 - 1) / S.fs;
  }
  double sp[3], ad[3];
  source_position(S, tm, sp);
  array_displacement(S, tm, ad);
  double* o = a.p.gpos + 6 * (S.gpos_base + grp);
  for (int d = 0; d < 3; ++d) {
    o[d] = sp[d];
    o[3 + d] = ad[d];
  }
}

// Position of every image in the first time group's sorted table (the row of
// its band-limited knot delays), by lattice index: unit k = group-0 position k.
__global__ void k_group0_pos(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[8]) return;
  int64_t k;
  const int s = locate(a, a.tab.img_prefix, gid, &k);
  const SceneDev& S = scene_of(a, s);
  a.p.m_pos[S.master_base + a.p.vals_out[S.img_base + k]] = int32_t(k);
}

// One unit per image of a scene (lattice order): its packed code, gain
// beta_i / (4 pi) * fs / c (Allen-Berkley product, FP64) and, for the sort
// keys of every time group, its offset 2 n o L - m from the first microphone
// (FP32) with the parity bits and the tier.
__global__ void k_images(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[8]) return;
  int64_t unit;
  const int s = locate(a, a.tab.img_prefix, gid, &unit);
  const SceneDev& S = scene_of(a, s);
  int li = int(unit >> 3);
  const int pb = int(unit & 7);
  const int K = S.K;
  // lattice order: n_x ascending, then n_y, then n_z, over |n|_1 <= K
  int nx = -K;
  for (; nx <= K; ++nx) {
    const int r = K - abs(nx);
    const int cnt = 2 * r * r + 2 * r + 1;
    if (li < cnt) break;
    li -= cnt;
  }
  const int r = K - abs(nx);
  int ny = -r;
  for (; ny <= r; ++ny) {
    const int cnt = 2 * (r - abs(ny)) + 1;
    if (li < cnt) break;
    li -= cnt;
  }
  const int nz = -(r - abs(ny)) + li;
  const int n[3] = {nx, ny, nz};
  const int p[3] = {pb & 1, (pb >> 1) & 1, (pb >> 2) & 1};
  int rho = 0;
  for (int d = 0; d < 3; ++d) rho += abs(2 * n[d] - p[d]);
  const int tier = tier_of(S, rho);
  // beta_i = prod_d beta_{d,0}^{|n_d - p_d|} beta_{d,1}^{|n_d|} (Allen-Berkley)
  double b = 1.0;
  for (int d = 0; d < 3; ++d) {
    const int e0 = abs(n[d] - p[d]), e1 = abs(n[d]);
    for (int q = 0; q < e0; ++q) b *= S.beta[2 * d];
    for (int q = 0; q < e1; ++q) b *= S.beta[2 * d + 1];
  }
  const int64_t m = S.master_base + unit;
  a.p.m_code[m] = pack_image(nx, ny, nz, pb);
  a.p.m_gain[m] = float(b / (4.0 * 3.14159265358979323846) * S.fs_over_c);
  float o[3];
  for (int d = 0; d < 3; ++d) o[d] = float(2.0 * n[d] * S.dims[d] - S.mics[0][d]);
  a.p.m_off[m] = make_float4(o[0], o[1], o[2], __int_as_float(pb | (tier << 4)));
}

// One unit per (scene, time group, image): the sort key (time group, tier,
// distance to the first microphone at the group's middle) and the image's
// index in the scene's lattice order.
__global__ void k_enumerate(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[0]) return;
  int64_t local;
  const int s = locate(a, a.tab.enum_prefix, gid, &local);
  const SceneDev& S = scene_of(a, s);
  const int64_t grp = local / S.n_images;
  const int64_t unit = local - grp * S.n_images;  // the image within the group's copy
  const float4 o = a.p.m_off[S.master_base + unit];
  const int bits = __float_as_int(o.w);
  const int tier = bits >> 4;
  // source position and array displacement at the group's middle; FP32 is
  // enough for an ordering key
  const double* gp = a.p.gpos + 6 * (S.gpos_base + grp);
  const float ov[3] = {o.x, o.y, o.z};
  float acc = 0.0f;
  for (int d = 0; d < 3; ++d) {
    const float sd = float(gp[d]);
    const float v = ((bits >> d) & 1 ? -sd : sd) + ov[d] - float(gp[3 + d]);
    acc = fmaf(v, v, acc);
  }
  // distance in 24 bits (units of 2^-12 m up to 4 km): the key only orders
  // images, and fewer key bits are fewer radix passes
  const float dist = fminf(sqrtf(acc), 4095.99f);
  const uint64_t dq = uint64_t(dist * 4096.0f);
  a.p.keys_in[gid] = (uint64_t(S.sort_group0 + grp) << kSortGroupShift) | (uint64_t(tier) << 24) | dq;
  a.p.vals_in[gid] = uint32_t(unit);
}

// The time groups' image tables in sorted order: code and gain gathered from
// the per-image table.
__global__ void k_image_table(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[0]) return;
  int64_t local;
  const int s = locate(a, a.tab.enum_prefix, gid, &local);
  const SceneDev& S = scene_of(a, s);
  const int64_t m = S.master_base + a.p.vals_out[gid];
  a.p.img_code[gid] = a.p.m_code[m];
  a.p.img_gain[gid] = a.p.m_gain[m];
}

__global__ void k_traj_knots(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[1]) return;
  int64_t local;
  const int s = locate(a, a.tab.knots_prefix, gid, &local);
  const SceneDev& S = scene_of(a, s);
  int t = 0;
  while (t + 1 < S.n_tiers && local >= S.knot_units_first[t + 1]) ++t;
  const int64_t j = local - S.knot_units_first[t];
  // knot j of the table is knot j - knot_shift of the tier (band-limited tiers
  // keep knot_shift knots before t = 0)
  const double time = double((j - S.knot_shift[t]) * S.tier_coarse[t]) / S.fs;
  double sp[3];
  source_position(S, time, sp);
  const int64_t k = S.knot_base[t] + j;
  double* out = a.p.knot_pos + 3 * k;
  out[0] = sp[0];
  out[1] = sp[1];
  out[2] = sp[2];
  float4 hi = make_float4(float(sp[0]), float(sp[1]), float(sp[2]), 0.0f);
  a.p.knot_hl[2 * k] = hi;
  a.p.knot_hl[2 * k + 1] =
      make_float4(float(sp[0] - double(hi.x)), float(sp[1] - double(hi.y)), float(sp[2] - double(hi.z)), 0.0f);
  if (S.arr_moving) {
    double ad[3];
    array_displacement(S, time, ad);
    double* o2 = a.p.arr_pos + 3 * k;
    o2[0] = ad[0];
    o2[1] = ad[1];
    o2[2] = ad[2];
    hi = make_float4(float(ad[0]), float(ad[1]), float(ad[2]), 0.0f);
    a.p.arr_hl[2 * k] = hi;
    a.p.arr_hl[2 * k + 1] =
        make_float4(float(ad[0] - double(hi.x)), float(ad[1] - double(hi.y)), float(ad[2] - double(hi.z)), 0.0f);
  }
}

// Delay tau = d fs / c (double-float) of every (microphone, image, knot) of a
// tier with band-limited knot upsampling (the upsampler's input, Sec. II-C),
// once per knot: every synthesis item whose virtual knots reach a knot reads
// it. One warp per (microphone, image) row, lanes over its knots (coalesced
// stores); the image's constant part 2 n L - m is formed once per lane.
constexpr int kBlTauThreads = 256;
__global__ void k_bl_tau(const __grid_constant__ KernelArgs a) {
  const int64_t wid = (int64_t(blockIdx.x) * kBlTauThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= a.totals[6]) return;
  int64_t local;
  const int s = locate(a, a.tab.bl_prefix, wid, &local);
  const SceneDev& S = scene_of(a, s);
  int t = -1;
  for (int k = 0; k < S.n_tiers; ++k)
    if (S.tier_up[k] > 1 && S.bl_units_first[k] <= local) t = k;
  if (t < 0) return;
  const int64_t row = local - S.bl_units_first[t];
  const int nkt = S.bl_knots[t];
  const int mic = int(row / S.tier_count[t]);
  const int img = int(row - int64_t(mic) * S.tier_count[t]);
  int n[3], p[3];
  unpack_image(a.p.img_code[S.img_base + S.tier_first[t] + img], n, p);
  DF o[3];  // 2 n L - m, double-float
  for (int d = 0; d < 3; ++d) {
    const float tn = float(2 * n[d]);  // exact
    const float pr = __fmul_rn(tn, S.dims_hl[d][0]);
    const DF off = fast_two_sum(pr, fmaf(tn, S.dims_hl[d][1], fmaf(tn, S.dims_hl[d][0], -pr)));
    o[d] = df_add(off, DF{-S.mics_hl[mic][d][0], -S.mics_hl[mic][d][1]});
  }
  const bool moving = S.arr_moving != 0;
  const DF fscd{S.fsc_hl[0], S.fsc_hl[1]};
  float2* out = a.p.bl_tau + S.bl_tau_base[t] + row * nkt;
  for (int j = lane; j < nkt; j += 32) {
    const int64_t k = S.knot_base[t] + j;
    const float4 h = a.p.knot_hl[2 * k], l = a.p.knot_hl[2 * k + 1];
    const float sh[3] = {h.x, h.y, h.z}, sl[3] = {l.x, l.y, l.z};
    float ah[3] = {0.f, 0.f, 0.f}, al[3] = {0.f, 0.f, 0.f};
    if (moving) {
      const float4 ha = a.p.arr_hl[2 * k], la = a.p.arr_hl[2 * k + 1];
      ah[0] = ha.x; ah[1] = ha.y; ah[2] = ha.z;
      al[0] = la.x; al[1] = la.y; al[2] = la.z;
    }
    DF q = {0.0f, 0.0f};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const DF sd = p[d] ? DF{-sh[d], -sl[d]} : DF{sh[d], sl[d]};
      const DF v = df_add(df_add(sd, o[d]), DF{-ah[d], -al[d]});
      q = df_add(q, df_mul(v, v));
    }
    const DF tau = df_mul(df_sqrt(q), fscd);
    out[j] = make_float2(tau.hi, tau.lo);
  }
}

// Source path table of a scene with emission-time delays: s(t) at
// t = (dense_k0 + k) / (kDenseOver fs) as FP32 pairs hi + lo.
__global__ void k_dense_traj(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[7]) return;
  int64_t local;
  const int s = locate(a, a.tab.dense_prefix, gid, &local);
  const SceneDev& S = scene_of(a, s);
  const double t = double(S.dense_k0 + local) / (double(kDenseOver) * S.fs);
  double sp[3];
  source_position(S, t, sp);
  const int64_t e = S.dense_base + local;
  const float hx = float(sp[0]), hy = float(sp[1]), hz = float(sp[2]);
  a.p.dense_hi[e] = make_float4(hx, hy, hz, 0.0f);
  a.p.dense_lo[e] = make_float4(float(sp[0] - hx), float(sp[1] - hy), float(sp[2] - hz), 0.0f);
}

}  // namespace

size_t sort_temp_bytes(int64_t n_items, int end_bit) {
  size_t bytes = 0;
  const cudaError_t e = cub::DeviceRadixSort::SortPairs(
      nullptr, bytes, (const uint64_t*)nullptr, (uint64_t*)nullptr, (const uint32_t*)nullptr,
      (uint32_t*)nullptr, int(n_items), 0, end_bit);
  if (e != cudaSuccess) {
    // no device to query (host-only size estimate): a generous bound
    cudaGetLastError();
    bytes = size_t(n_items) * 16 + (size_t(8) << 20);
  }
  return bytes;
}

cudaError_t launch_sort(const KernelArgs& a, int64_t n, int end_bit, cudaStream_t st) {
  size_t bytes = a.p.sort_temp_bytes;
  return cub::DeviceRadixSort::SortPairs(a.p.sort_temp, bytes, a.p.keys_in, a.p.keys_out,
                                         a.p.vals_in, a.p.vals_out, int(n), 0, end_bit, st);
}

static inline unsigned blocks_for(int64_t n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

cudaError_t launch_setup(const KernelArgs& a, cudaStream_t st) {
  const int T = 256;
  if (a.totals[0] > 0) {
    k_group_pos<<<dim3(unsigned((a.max_time_groups + 63) / 64), unsigned(a.n_scenes)), 64, 0, st>>>(a);
    k_images<<<blocks_for(a.totals[8], T), T, 0, st>>>(a);
    k_enumerate<<<blocks_for(a.totals[0], T), T, 0, st>>>(a);
    int end_bit = kSortGroupShift;
    while ((int64_t(1) << (end_bit - kSortGroupShift)) < a.n_sort_groups) ++end_bit;
    cudaError_t e = launch_sort(a, a.totals[0], end_bit, st);
    if (e != cudaSuccess) return e;
    k_image_table<<<blocks_for(a.totals[0], T), T, 0, st>>>(a);
    if (a.totals[6] > 0) k_group0_pos<<<blocks_for(a.totals[8], T), T, 0, st>>>(a);
  }
  if (a.totals[1] > 0) k_traj_knots<<<blocks_for(a.totals[1], T), T, 0, st>>>(a);
  // k_bl_tau: one warp per unit (a (microphone, image) row of knots)
  if (a.totals[6] > 0) k_bl_tau<<<blocks_for(a.totals[6] * 32, kBlTauThreads), kBlTauThreads, 0, st>>>(a);
  if (a.totals[7] > 0) k_dense_traj<<<blocks_for(a.totals[7], T), T, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace msrc
