// Forward synthesis kernels (Sec. II-B Eq. 3-5, Sec. II-C Eq. 8):
//
//   k_prefilter  signal side of the Farrow structure (Eq. 5): for every
//                segment s and power q of the tap polynomial,
//                z[s][q][m] = sum_k c[s][q][k] x[m - k].
//   k_synth      persistent gather-accumulate over a work queue of
//                (scene, microphone, image block, output tile) items. Per
//                image-sample: interpolate the delay from the knot records,
//                split it into read position m0 and fraction alpha, evaluate
//                e = sum_q v^q z[seg(alpha)][q][m0] by Horner, and accumulate
//                (beta_i / (4 pi d_i(n))) e. The z window of the item is staged
//                in shared memory with cp.async; each item writes one partial
//                row (no atomics).
//   k_reduce     y[mic][n] = sum over image blocks of the partial rows, in a
//                fixed order (bitwise reproducible).
#include <cstdint>

#include "msrc_internal.h"

namespace msrc {
namespace {

__device__ __forceinline__ const SceneDev& scene_of(const KernelArgs& a, int s) {
  return a.n_scenes == 1 ? a.scene0 : a.scenes[s];
}

__device__ __forceinline__ int find_scene(const int64_t* prefix, int n, int64_t idx) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= idx) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ prefilter
constexpr int kPreThreads = 256;

template <int kL>
__global__ void __launch_bounds__(kPreThreads) k_prefilter(const __grid_constant__ KernelArgs a) {
  __shared__ float xs[kPreThreads + kL];
  int s = 0;
  int64_t blk = blockIdx.x;
  if (a.n_scenes > 1) {
    s = find_scene(a.tab.z_prefix, a.n_scenes, blk);
    blk -= a.tab.z_prefix[s];
  }
  const SceneDev& S = scene_of(a, s);
  const int64_t m_first = S.z_m0 + blk * kPreThreads;  // sample index of this CTA's first column
  // x[m - k] for k in [-kL/2, kL/2 - 1] and m in [m_first, m_first + kPreThreads)
  // spans x[m_first - kL/2 + 1 .. m_first + kPreThreads - 1 + kL/2]
  const int64_t x_lo = m_first - kL / 2 + 1;
  for (int i = threadIdx.x; i < kPreThreads + kL; i += kPreThreads) {
    const int64_t m = x_lo + i;
    xs[i] = (m >= 0 && m < S.n_in) ? __ldg(S.x + m) : 0.0f;
  }
  __syncthreads();
  const int64_t col = blk * kPreThreads + threadIdx.x;
  if (col >= S.z_len) return;
  // xs index of x[m - k] is (threadIdx.x - k) + kL/2 - 1
  float acc[kZRows];
#pragma unroll
  for (int r = 0; r < kZRows; ++r) acc[r] = 0.0f;
#pragma unroll
  for (int kk = 0; kk < kL; ++kk) {  // kk = k + kL/2
    const float xv = xs[threadIdx.x - kk + kL - 1];
#pragma unroll
    for (int r = 0; r < kZRows; ++r)
      acc[r] = fmaf(a.farrow[r / kFarrowCoef][r % kFarrowCoef][kk], xv, acc[r]);
  }
  float* z = a.p.z + S.z_base + col;
#pragma unroll
  for (int r = 0; r < kZRows; ++r) z[int64_t(r) * S.z_len] = acc[r];
}

// ------------------------------------------------------------------ synthesis
struct TileShape {
  int threads;   // CTA size
  int chunks;    // 32-sample chunks per warp (tile = threads * chunks)
  int wcap;      // shared-memory window capacity (samples)
  int block;     // images per block
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Delay interpolation and read position of one image-sample.
// rec = {I_j = n_j - D_j, f_j, slope, d_j}; r = n - n_j.
struct Tap {
  int m0;     // read position floor(n - tau)
  int seg;    // Farrow segment of alpha
  float v;    // local polynomial variable in [-1, 1]
  float d;    // interpolated distance
};

__device__ __forceinline__ Tap delay_split(const int4 rec, int r, float rf, float c_over_fs) {
  const float fj = __int_as_float(rec.y);
  const float st = __int_as_float(rec.z);
  const float dj = __int_as_float(rec.w);
  // phi = tau(n) - D_j, |phi| small; n - tau = r + I_j - phi
  const float phi = fmaf(rf, st, fj);
  // ceil(phi) with the round-to-nearest magic constant 1.5 * 2^23
  const float q = phi + 12582912.0f;
  const int kr = __float_as_int(q) - 0x4B400000;
  const float cf = q - 12582912.0f;
  const int up = cf < phi ? 1 : 0;
  const float alpha = (cf - phi) + float(up);  // in [0, 1]
  Tap t;
  t.m0 = r + rec.x - (kr + up);
  const float psi = alpha * float(kFarrowSegs);
  int seg = int(psi);
  seg = seg > kFarrowSegs - 1 ? kFarrowSegs - 1 : seg;
  t.seg = seg;
  t.v = fmaf(psi - float(seg), 2.0f, -1.0f);
  t.d = fmaf(rf, st * c_over_fs, dj);
  return t;
}

template <int kThreads, int kChunks, int kWcap, int kBlock>
__global__ void __launch_bounds__(kThreads) k_synth(const __grid_constant__ KernelArgs a) {
  extern __shared__ __align__(16) float zs[];  // kZRows rows of kWcap floats
  __shared__ int s_item;
  __shared__ float s_red[2][kThreads / 32];
  constexpr int kTile = kThreads * kChunks;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;

  for (;;) {
    if (threadIdx.x == 0) s_item = int(atomicAdd(a.p.counter, 1u));
    __syncthreads();
    const int64_t item = s_item;
    if (item >= a.totals[4]) break;
    int s = 0;
    int64_t li = item;
    if (a.n_scenes > 1) {
      s = find_scene(a.tab.item_prefix, a.n_scenes, item);
      li = item - a.tab.item_prefix[s];
    }
    const SceneDev& S = scene_of(a, s);
    const int tile = int(li % S.n_tiles);
    const int64_t mb = li / S.n_tiles;
    const int mic = int(mb / S.n_blocks);
    const int blk = int(mb - int64_t(mic) * S.n_blocks);
    int t = 0;
    while (t + 1 < S.n_tiers && blk >= S.block_first[t + 1]) ++t;
    const int blk_t = blk - S.block_first[t];
    const int img0 = blk_t * kBlock;                         // first image within the tier
    const int cnt = min(kBlock, S.tier_count[t] - img0);
    const int N = S.tier_step[t];
    const int J = S.tier_intervals[t];
    const int n0 = tile * kTile;
    const int n_end = int(min(int64_t(n0 + kTile), S.n_out)) - 1;
    const int4* rec = a.p.rec + S.rec_base[t] + int64_t(mic) * S.rec_mic_stride + int64_t(img0) * J;
    const float* gain = a.p.img_gain + S.img_base + S.tier_first[t] + img0;

    // --- delay range of the item (linear between knots: extremes at knots)
    const int jf = n0 / N, jl = n_end / N;
    const int nk = jl - jf + 2;
    float tmin = 3.0e38f, tmax = -3.0e38f;
    const int pairs = cnt * nk;
    for (int pidx = threadIdx.x; pidx < pairs; pidx += kThreads) {
      const int ib = pidx / nk;
      const int jj = jf + (pidx - ib * nk);
      const int jr = jj <= jl ? jj : jl;
      const int4 R = __ldg(rec + int64_t(ib) * J + jr);
      float tau = float(jr * N - R.x) + __int_as_float(R.y);
      if (jj > jl) tau = fmaf(float(N), __int_as_float(R.z), tau);
      tmin = fminf(tmin, tau);
      tmax = fmaxf(tmax, tau);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
      tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    }
    if (lane == 0) { s_red[0][warp] = tmin; s_red[1][warp] = tmax; }
    __syncthreads();
    tmin = s_red[0][0];
    tmax = s_red[1][0];
#pragma unroll
    for (int w = 1; w < kThreads / 32; ++w) {
      tmin = fminf(tmin, s_red[0][w]);
      tmax = fmaxf(tmax, s_red[1][w]);
    }
    const int m_lo = (n0 - int(ceilf(tmax)) - 2) & ~3;
    const int m_hi = n_end - int(floorf(tmin)) + 2;
    const int width = ((m_hi - m_lo + 1) + 3) & ~3;
    const bool in_smem = width <= kWcap;

    // --- stage the z window [m_lo, m_lo + width) of all rows
    const float* zg = a.p.z + S.z_base;
    if (in_smem) {
      const int64_t lo_c = max(int64_t(m_lo), S.z_m0);
      const int64_t hi_c = min(int64_t(m_lo) + width, S.z_m0 + S.z_len);
      if ((lo_c != m_lo || hi_c != int64_t(m_lo) + width) && threadIdx.x == 0)
        atomicOr(a.p.err, kErrWindowClamp);
      const int vec = int(hi_c > lo_c ? hi_c - lo_c : int64_t(0)) >> 2;
      const int dst0 = int(lo_c - m_lo);
      for (int i = threadIdx.x; i < kZRows * vec; i += kThreads) {
        const int r = i / vec, c4 = i - r * vec;
        cp_async16(zs + r * kWcap + dst0 + 4 * c4, zg + int64_t(r) * S.z_len + (lo_c - S.z_m0) + 4 * c4);
      }
      cp_async_wait_all();
    }
    __syncthreads();

    // --- gather-accumulate: warp w owns samples n0 + 32 (w kChunks + c) + lane
    int jr[kChunks], rr[kChunks];
    float rf[kChunks], acc[kChunks];
    bool valid[kChunks];
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      const int n = n0 + 32 * (warp * kChunks + c) + lane;
      valid[c] = n <= n_end;
      const int nn = valid[c] ? n : n_end;
      jr[c] = nn / N;
      rr[c] = nn - jr[c] * N;
      rf[c] = float(rr[c]);
      acc[c] = 0.0f;
    }
    const float cfs = S.c_over_fs;
    if (in_smem) {
      const unsigned wmax = unsigned(width - 1);
      for (int ib = 0; ib < cnt; ++ib) {
        const float g = __ldg(gain + ib);
        const int4* ri = rec + int64_t(ib) * J;
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
          const Tap tp = delay_split(__ldg(ri + jr[c]), rr[c], rf[c], cfs);
          const unsigned col = min(unsigned(tp.m0 - m_lo), wmax);
          const float* zp = zs + tp.seg * (kFarrowCoef * kWcap) + col;
          float e = zp[kFarrowDeg * kWcap];
#pragma unroll
          for (int q = kFarrowDeg - 1; q >= 0; --q) e = fmaf(e, tp.v, zp[q * kWcap]);
          acc[c] = fmaf(__fdividef(g, tp.d), e, acc[c]);
        }
      }
    } else {
      // window wider than shared memory: read the L2-resident rows directly
      const uint64_t zmax = uint64_t(S.z_len - 1);
      for (int ib = 0; ib < cnt; ++ib) {
        const float g = __ldg(gain + ib);
        const int4* ri = rec + int64_t(ib) * J;
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
          const Tap tp = delay_split(__ldg(ri + jr[c]), rr[c], rf[c], cfs);
          const uint64_t col = min(uint64_t(int64_t(tp.m0) - S.z_m0), zmax);
          const float* zp = zg + int64_t(tp.seg) * kFarrowCoef * S.z_len + col;
          float e = __ldg(zp + int64_t(kFarrowDeg) * S.z_len);
#pragma unroll
          for (int q = kFarrowDeg - 1; q >= 0; --q) e = fmaf(e, tp.v, __ldg(zp + int64_t(q) * S.z_len));
          acc[c] = fmaf(__fdividef(g, tp.d), e, acc[c]);
        }
      }
    }
    float* out = a.p.part + S.part_base + (int64_t(mic) * S.n_blocks + blk) * S.n_out;
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      const int n = n0 + 32 * (warp * kChunks + c) + lane;
      if (valid[c]) out[n] = acc[c];
    }
    __syncthreads();  // shared window and s_item are reused by the next item
  }
}

// ------------------------------------------------------------------ reduction
__global__ void k_reduce(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[5]) return;
  int s = 0;
  int64_t local = gid;
  if (a.n_scenes > 1) {
    s = find_scene(a.tab.red_prefix, a.n_scenes, gid);
    local = gid - a.tab.red_prefix[s];
  }
  const SceneDev& S = scene_of(a, s);
  const int mic = int(local / S.n_out);
  const int64_t n = local - int64_t(mic) * S.n_out;
  const float* p = a.p.part + S.part_base + int64_t(mic) * S.n_blocks * S.n_out + n;
  float acc = 0.0f;
  for (int b = 0; b < S.n_blocks; ++b) acc += p[int64_t(b) * S.n_out];
  S.y[int64_t(mic) * S.n_out + n] = acc;
}

template <int kThreads, int kChunks, int kWcap, int kBlock>
cudaError_t run_synth(const KernelArgs& a, cudaStream_t st) {
  auto kern = k_synth<kThreads, kChunks, kWcap, kBlock>;
  const size_t smem = size_t(kZRows) * kWcap * sizeof(float);
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    grid = sms * (occ > 0 ? occ : 1);
  }
  const int64_t items = a.totals[4];
  const int g = int(items < grid ? items : grid);
  cudaError_t e = cudaMemsetAsync(a.p.counter, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (g > 0) kern<<<g, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

struct TileConfig {
  int threads, chunks, wcap, block;
};
static const TileConfig kConfigs[] = {
    {256, 3, 1792, 256},
    {256, 2, 1536, 256},
    {256, 4, 2048, 128},
    {512, 2, 3584, 256},
};

int tile_config_count() { return int(sizeof(kConfigs) / sizeof(kConfigs[0])); }
int tile_samples(int cfg) { return kConfigs[cfg].threads * kConfigs[cfg].chunks; }
int tile_block_images(int cfg) { return kConfigs[cfg].block; }

cudaError_t launch_forward(const KernelArgs& a, int cfg, cudaStream_t st, cudaEvent_t* ev) {
  const int T = 256;
  if (a.totals[3] > 0) {
    const unsigned g = unsigned(a.totals[3]);
    if (a.taps <= 16) k_prefilter<16><<<g, kPreThreads, 0, st>>>(a);
    else if (a.taps <= 32) k_prefilter<32><<<g, kPreThreads, 0, st>>>(a);
    else k_prefilter<64><<<g, kPreThreads, 0, st>>>(a);
  }
  if (ev) cudaEventRecord(ev[0], st);
  cudaError_t e = cudaSuccess;
  switch (cfg) {
    case 1: e = run_synth<256, 2, 1536, 256>(a, st); break;
    case 2: e = run_synth<256, 4, 2048, 128>(a, st); break;
    case 3: e = run_synth<512, 2, 3584, 256>(a, st); break;
    default: e = run_synth<256, 3, 1792, 256>(a, st); break;
  }
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], st);
  if (a.totals[5] > 0) k_reduce<<<unsigned((a.totals[5] + T - 1) / T), T, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace msrc
