// Forward synthesis kernels (Sec. II-B Eq. 3-5, Sec. II-C Eq. 8):
//
//   k_prefilter  signal side of the Farrow structure (Eq. 5): for every
//                segment s and power q of the tap polynomial,
//                z[s][q][m] = sum_k c[s][q][k] x[m - k].
//   k_synth      persistent gather-accumulate over a work queue of
//                (scene, microphone, image block, output tile) items.
//                Item prologue: the hierarchical delay knots of the block's
//                images over the tile (Sec. II-C, "Fast Architecture") are
//                evaluated into shared memory: one FP64 anchor distance per
//                image, the other knots by an exact FP32 increment of the
//                squared distance. Then the z window of the item is staged in
//                shared memory with cp.async. Per image-sample: interpolate the
//                delay linearly between knots, split it into read position m0
//                and fraction alpha, evaluate e = sum_q w^q z[seg(alpha)][q][m0]
//                by Horner and accumulate (beta_i / (4 pi d_i(n))) e. Each item
//                writes one partial row (no atomics).
//   k_reduce     y[mic][n] = sum over image blocks of the partial rows, in a
//                fixed order (bitwise reproducible).
#include <cstdint>

#include "msrc_internal.h"
#include "synth_common.cuh"

namespace msrc {
namespace {

// ------------------------------------------------------------------ prefilter
constexpr int kPreThreads = 256;

// kCoef = kFarrowCoef: the synthesis rows (degree 4, zq + zp); kCoef =
// kGradCoef: the gradient kernel's rows (degree 5, zq + zg).
template <int kL, int kCoef>
__global__ void __launch_bounds__(kPreThreads) k_prefilter(const __grid_constant__ KernelArgs a) {
  static_assert(kCoef == kFarrowCoef || kCoef == kGradCoef, "row sets");
  constexpr int kRows = kFarrowSegs * kCoef;
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
  float acc[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) acc[r] = 0.0f;
#pragma unroll
  for (int kk = 0; kk < kL; ++kk) {  // kk = k + kL/2
    const float xv = xs[threadIdx.x - kk + kL - 1];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const float c = kCoef == kFarrowCoef ? a.farrow[r / kCoef][r % kCoef][kk]
                                           : a.farrow_g[r / kCoef][r % kCoef][kk];
      acc[r] = fmaf(c, xv, acc[r]);
    }
  }
  float4* zq = a.p.zq + S.z_base + col;
#pragma unroll
  for (int sg = 0; sg < kFarrowSegs; ++sg) {
    const float* c = acc + sg * kCoef;
    zq[int64_t(sg) * S.z_len] = make_float4(c[0], c[1], c[2], c[3]);
    if constexpr (kCoef == kFarrowCoef) a.p.zp[S.z_base + col + int64_t(sg) * S.z_len] = c[4];
    else a.p.zg[S.z_base + col + int64_t(sg) * S.z_len] = make_float2(c[4], c[kCoef - 1]);
  }
}

// ------------------------------------------------------------------ synthesis


// acc + (beta_i / (4 pi d_i(n))) e_i(n) for one image-sample read from the
// staged window (kStride columns per segment). The gain of the image record is
// beta_i / (4 pi) * fs / c, so the gain at n is gain / tau with tau in samples.
// kChecked: the window is processed in several column passes and only columns
// inside this pass count; otherwise every read position lies inside the window
// by construction and the index is only clamped to the window arrays.
// Unchecked reads index the window by byte offset (split_offset): the offset
// of the power-4 value, 4 times it for the powers 0..3.
template <int kStride, bool kChecked>
__device__ __forceinline__ float image_sample(const float4* zq, const float* zp, const float2 rec, const int4 im,
                                              unsigned I4, int rmj, unsigned rmc4, float rf, unsigned wmax,
                                              float acc) {
  const float Dp = __int_as_float(im.y);
  float w, tau;
  float4 A;
  float B;
  if (kChecked) {
    const DelaySplit ds = split_delay(rec, rmj + im.x, rf, Dp);
    if (unsigned(ds.col) > wmax) return acc;
    const unsigned idx = unsigned(ds.seg * kStride + ds.col);
    A = zq[idx];
    B = zp[idx];
    w = ds.w;
    tau = ds.tau;
  } else {
    const unsigned off = min(split_offset<kStride>(rec, I4, rmc4, rf, Dp, &w, &tau),
                             unsigned(4 * (kFarrowSegs * kStride - 1)));
    A = *reinterpret_cast<const float4*>(reinterpret_cast<const unsigned char*>(zq) + 4u * off);
    B = *reinterpret_cast<const float*>(reinterpret_cast<const unsigned char*>(zp) + off);
  }
  const float e = horner5(A, B, w);
  return fmaf(__fdividef(__int_as_float(im.z), tau), e, acc);
}

// All images of the block for this thread's kChunks samples; rmj[c] =
// r - m_lo + jj N_t of chunk c (its interval jj = jc[c]).
// kOne: every chunk of this lane lies in one knot interval (warp-uniform), so
// one record load per image serves all chunks.
template <int kStride, int kChunks, int kUnroll, bool kChecked, bool kOne>
__device__ __forceinline__ void gather_images(const float4* zq, const float* zp, const float2* rec_s,
                                              const int4* img_s, int cnt, const int* jc, const int* rmj,
                                              const float* rf, unsigned wmax, float* acc) {
  unsigned rmc4[kChunks];
  const float2* row[kChunks];  // records of chunk c: row jc[c] of the interval-major table
#pragma unroll
  for (int c = 0; c < kChunks; ++c) {
    rmc4[c] = fold_rounding(rmj[c]) << 2;
    row[c] = rec_s + jc[c] * cnt;
  }
  int ib = 0;
  for (; ib + kUnroll <= cnt; ib += kUnroll) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int4 im = img_s[ib + u];
      const unsigned I4 = unsigned(im.w);  // 4 im.x
      const float2 r0 = row[0][ib + u];
#pragma unroll
      for (int c = 0; c < kChunks; ++c)
        acc[c] = image_sample<kStride, kChecked>(zq, zp, (kOne || c == 0) ? r0 : row[c][ib + u], im, I4, rmj[c],
                                                 rmc4[c], rf[c], wmax, acc[c]);
    }
  }
  for (; ib < cnt; ++ib) {
    const int4 im = img_s[ib];
    const unsigned I4 = unsigned(im.w);  // 4 im.x
    const float2 r0 = row[0][ib];
#pragma unroll
    for (int c = 0; c < kChunks; ++c)
      acc[c] = image_sample<kStride, kChecked>(zq, zp, (kOne || c == 0) ? r0 : row[c][ib], im, I4, rmj[c],
                                               rmc4[c], rf[c], wmax, acc[c]);
  }
}

template <int kThreads, int kChunks, int kWcap, int kRecCap, int kBlock, int kUnroll>
__global__ void __launch_bounds__(kThreads, (kThreads <= 256 ? 2 : 1)) k_synth(const __grid_constant__ KernelArgs a) {
  extern __shared__ __align__(16) float4 smem4[];
  float4* zq_s = smem4;                                                  // kFarrowSegs x kWcap
  float* zp_s = reinterpret_cast<float*>(smem4 + kFarrowSegs * kWcap);    // kFarrowSegs x kWcap
  float2* rec_s = reinterpret_cast<float2*>(zp_s + kFarrowSegs * kWcap);  // kRecCap interval records
  int4* img_s = reinterpret_cast<int4*>(rec_s + kRecCap);                 // kBlock image records
  static_assert((kRecCap * sizeof(float2)) % 16 == 0 && (kFarrowSegs * kWcap * sizeof(float)) % 16 == 0,
                "every shared array starts on a 16-byte boundary");
  // prologue scratch aliases the z window (used before the window is staged)
  float4* u_s = smem4;
  float4* um_s = u_s + kThreads * kChunks + 4;                           // moving array
  float4* anc_s = um_s + kThreads * kChunks + 4;                         // 3 x kBlock
  float* phi_s = reinterpret_cast<float*>(anc_s + 3 * kBlock);           // kRecCap + kBlock
  // emission-time delays: u_s holds the array increments, then 6 x kBlock anchors, then phi
  float4* an6_s = um_s;
  float* phi_r = reinterpret_cast<float*>(an6_s + 6 * kBlock);
  __shared__ int s_item;
  __shared__ float s_red[2][kThreads / 32];
  __shared__ __align__(8) uint64_t s_mbar;  // completion of the window's bulk copies
  static_assert(kWcap % 4 == 0, "16-byte aligned power-4 row segments");
  static_assert(kBlock <= kThreads, "the record builders give every image at least one thread");
  constexpr int kTile = kThreads * kChunks;
  static_assert(4 * (2 * (kTile + 4) + 3 * kBlock) + kRecCap + kBlock <= 4 * kFarrowSegs * kWcap,
                "prologue scratch");
  static_assert(4 * ((kTile + 4) + 6 * kBlock) + kRecCap + kBlock <= 4 * kFarrowSegs * kWcap,
                "prologue scratch (emission-time delays)");
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) mbar_init(&s_mbar, 1);
  unsigned phase = 0;  // of s_mbar, the same in every thread

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
    const ItemGeom g = item_geometry(S, li, kTile);

    // --- delay knots of the block over the tile (records in shared memory)
    float tmin, tmax;
    int cnt = g.cnt;
    if (S.delay_model == 1) {
      item_records_ret<kThreads>(a, S, g, rec_s, img_s, u_s, an6_s, phi_r, &tmin, &tmax);
    } else if (S.tier_up[g.t] > 1) {
      // band-limited knot upsampling: its scratch takes the z window and power rows
      if (!item_records_bl<kThreads>(a, S, g, rec_s, img_s, reinterpret_cast<float*>(smem4),
                                     int64_t(kFarrowSegs) * kWcap * 5, &tmin, &tmax))
        cnt = 0;
    } else {
      item_records<kThreads>(a, S, g, rec_s, img_s, u_s, um_s, anc_s, phi_s, &tmin, &tmax);
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
    // window start congruent to the z rows' origin mod 4: power-4 row segments
    // then start on 16-byte boundaries on both sides of the bulk copy
    int m_lo = g.n0 - int(ceilf(tmax)) - 2;
    m_lo -= int(((int64_t(m_lo) - S.z_m0) % 4 + 4) % 4);
    const int width = g.n_end - int(floorf(tmin)) + 2 - m_lo + 1;

    // this thread's samples: warp w owns n0 + 32 (w kChunks + c) + lane
    int jc[kChunks], rr[kChunks], rmj[kChunks];
    float rf[kChunks], acc[kChunks];
    bool valid[kChunks];
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      const int n = g.n0 + 32 * (warp * kChunks + c) + lane;
      valid[c] = n <= g.n_end;
      const int nn = valid[c] ? n : g.n_end;
      const int j = nn / g.N;
      rr[c] = nn - j * g.N;
      jc[c] = j - g.jf;
      rf[c] = float(rr[c]);
      acc[c] = 0.0f;
    }
    // every chunk of every lane in one knot interval (e.g. 96-sample intervals
    // aligned with this warp's 96 samples): one record load per image
    bool one = true;
#pragma unroll
    for (int c = 1; c < kChunks; ++c) one = one && (jc[c] == jc[0]);
    one = __all_sync(0xffffffffu, one);
    const float4* zqg = a.p.zq + S.z_base;
    const float* zpg = a.p.zp + S.z_base;

    // --- the window [m_lo, m_lo + width) in passes of at most kWcap columns
    for (int p0 = 0; p0 < width; p0 += kWcap) {
      const int pass_lo = m_lo + p0;
      const int pw = min(kWcap, width - p0);
      // generic-proxy reads and writes of this shared memory (the prologue
      // scratch, or the previous pass) are done before the async copies land
      fence_proxy_async();
      __syncthreads();
      const int64_t lo_c = max(int64_t(pass_lo), S.z_m0);
      const int64_t hi_c = min(int64_t(pass_lo) + pw, S.z_m0 + S.z_len);
      if ((lo_c != pass_lo || hi_c != int64_t(pass_lo) + pw) && threadIdx.x == 0)
        atomicOr(a.p.err, kErrWindowClamp);
      const int cnt_c = int(hi_c > lo_c ? hi_c - lo_c : int64_t(0));
      const int dst0 = int(lo_c - pass_lo);    // a multiple of 4 (see m_lo)
      const int64_t src0 = lo_c - S.z_m0;      // a multiple of 4
      if (cnt_c > 0) {
        if (threadIdx.x == 0) {
          const unsigned bq = unsigned(cnt_c) * 16u;
          const unsigned bp = unsigned((cnt_c + 3) & ~3) * 4u;  // within the padded rows
          mbar_expect_tx(&s_mbar, unsigned(kFarrowSegs) * (bq + bp) + a.test_extra_tx);
          for (int sg = 0; sg < kFarrowSegs; ++sg) {
            bulk_g2s(zq_s + sg * kWcap + dst0, zqg + int64_t(sg) * S.z_len + src0, bq, &s_mbar);
            bulk_g2s(zp_s + sg * kWcap + dst0, zpg + int64_t(sg) * S.z_len + src0, bp, &s_mbar);
          }
        }
        const bool ok = mbar_wait(&s_mbar, phase);
        if (__syncthreads_or(!ok)) {
          // the copies did not complete in time: flag it, give them one more
          // bounded wait, and stop this CTA
          if (threadIdx.x == 0) atomicOr(a.p.err, kErrTimeout);
          mbar_wait(&s_mbar, phase);
          return;
        }
        phase ^= 1u;
      }
#pragma unroll
      for (int c = 0; c < kChunks; ++c) rmj[c] = rr[c] - pass_lo + jc[c] * g.N;
      const unsigned wmax = unsigned(pw - 1);
      if (width <= kWcap) {
        if (one)
          gather_images<kWcap, kChunks, kUnroll, false, true>(zq_s, zp_s, rec_s, img_s, cnt, jc, rmj, rf, wmax, acc);
        else
          gather_images<kWcap, kChunks, kUnroll, false, false>(zq_s, zp_s, rec_s, img_s, cnt, jc, rmj, rf, wmax, acc);
      } else {
        gather_images<kWcap, kChunks, kUnroll, true, false>(zq_s, zp_s, rec_s, img_s, cnt, jc, rmj, rf, wmax, acc);
      }
    }
    float* out = a.p.part + S.part_base + (int64_t(g.mic) * S.n_blocks + g.blk) * S.n_out;
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      const int n = g.n0 + 32 * (warp * kChunks + c) + lane;
      if (valid[c]) out[n] = acc[c];
    }
    __syncthreads();  // shared memory and s_item are reused by the next item
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

template <int kThreads, int kChunks, int kWcap, int kRecCap, int kBlock, int kUnroll>
cudaError_t run_synth(const KernelArgs& a, cudaStream_t st) {
  auto kern = k_synth<kThreads, kChunks, kWcap, kRecCap, kBlock, kUnroll>;
  const size_t smem = size_t(kFarrowSegs) * kWcap * (sizeof(float4) + sizeof(float)) +
                      size_t(kRecCap) * sizeof(float2) + size_t(kBlock) * sizeof(int4);
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

// Tile configurations of the synthesis launch (see TileConfig).
#define MSRC_TILE_CONFIGS(X)             \
  X(0, 512, 3, 2432, 4096, 256, 8)       \
  X(1, 256, 2, 1152, 1664, 256, 4)       \
  X(2, 384, 2, 2048, 3072, 256, 4)       \
  X(3, 1024, 1, 2432, 4096, 256, 2)      \
  X(4, 512, 2, 2432, 4096, 256, 8)       \
  X(5, 512, 1, 2432, 4096, 256, 8)       \
  X(6, 512, 3, 2432, 4096, 256, 4)       \
  X(7, 512, 2, 2432, 4096, 256, 16)      \
  X(8, 512, 3, 1792, 8192, 256, 8)       \
  X(9, 512, 2, 1792, 8192, 256, 8)       \
  X(10, 512, 2, 1536, 10240, 256, 8)

static const TileConfig kConfigs[] = {
#define MSRC_ROW(id, th, ch, wc, rc, bl, un) {th, ch, wc, rc, bl},
    MSRC_TILE_CONFIGS(MSRC_ROW)
#undef MSRC_ROW
};

int tile_config_count() { return int(sizeof(kConfigs) / sizeof(kConfigs[0])); }
const TileConfig& tile_config(int cfg) { return kConfigs[cfg]; }

cudaError_t launch_prefilter(const KernelArgs& a, cudaStream_t st, bool gradient_rows) {
  if (a.totals[3] > 0) {
    const unsigned g = unsigned(a.totals[3]);
    if (gradient_rows) {
      if (a.taps <= 16) k_prefilter<16, kGradCoef><<<g, kPreThreads, 0, st>>>(a);
      else if (a.taps <= 32) k_prefilter<32, kGradCoef><<<g, kPreThreads, 0, st>>>(a);
      else k_prefilter<64, kGradCoef><<<g, kPreThreads, 0, st>>>(a);
    } else {
      if (a.taps <= 16) k_prefilter<16, kFarrowCoef><<<g, kPreThreads, 0, st>>>(a);
      else if (a.taps <= 32) k_prefilter<32, kFarrowCoef><<<g, kPreThreads, 0, st>>>(a);
      else k_prefilter<64, kFarrowCoef><<<g, kPreThreads, 0, st>>>(a);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_forward(const KernelArgs& a, int cfg, cudaStream_t st, cudaEvent_t* ev) {
  const int T = 256;
  cudaError_t pe = launch_prefilter(a, st, false);
  if (pe != cudaSuccess) return pe;
  if (ev) cudaEventRecord(ev[0], st);
  cudaError_t e = cudaSuccess;
  switch (cfg) {
#define MSRC_CASE(id, th, ch, wc, rc, bl, un) \
  case id: e = run_synth<th, ch, wc, rc, bl, un>(a, st); break;
    MSRC_TILE_CONFIGS(MSRC_CASE)
#undef MSRC_CASE
    default: e = cudaErrorInvalidValue; break;
  }
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], st);
  if (a.totals[5] > 0) k_reduce<<<unsigned((a.totals[5] + T - 1) / T), T, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace msrc
