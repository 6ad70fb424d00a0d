// Forward synthesis kernels (Sec. II-B Eq. 3-5, Sec. II-C Eq. 8):
//
//   k_absmax     largest |x| of every scene (the scale of the half-precision
//                powers of the prefiltered rows).
//   k_prefilter  signal side of the Farrow structure (Eq. 5): for every
//                segment s and power q of the tap polynomial,
//                z[s][q][m] = sum_k c[s][q][k] x[m - k], stored per column and
//                segment as one float4 {z0, z1, z2, half2(s z3, s z4)}.
//   k_synth      persistent gather-accumulate over a work queue of
//                (scene, microphone, image block, output tile) items.
//                Item prologue: the hierarchical delay knots of the block's
//                images over the tile (Sec. II-C, "Fast Architecture") are
//                evaluated into shared memory: a double-float anchor distance
//                per image, the other knots by an exact FP32 increment of the
//                squared distance, stored as interval records of image pairs.
//                Then the z window of the item is staged in shared memory by
//                bulk copies (cp.async.bulk) completing on an mbarrier. Per
//                image-sample: interpolate the delay linearly between knots,
//                split it into read position m0 and fraction alpha, evaluate
//                e = sum_q w^q z[seg(alpha)][q][m0] by Horner and accumulate
//                (beta_i / (4 pi d_i(n))) e; the delay arithmetic and the
//                accumulation run on float2 pairs of images (FFMA2). Each item
//                writes one partial row (no atomics).
//   k_reduce     y[mic][n] = sum over image blocks of the partial rows, in a
//                fixed order (bitwise reproducible).
#include <cstdint>

#include <cuda_fp16.h>

#include "msrc_internal.h"
#include "synth_common.cuh"

namespace msrc {
namespace {

// ------------------------------------------------------------------ prefilter
constexpr int kPreThreads = 256;

// Largest |x| of every scene (as float bits, atomicMax over the prefilter's
// column tiles: order-independent, so reproducible); the synthesis rows' power
// 3 and 4 values are scaled by it (zh_scale) before they are stored in half
// precision.
__global__ void __launch_bounds__(kPreThreads) k_absmax(const __grid_constant__ KernelArgs a) {
  __shared__ unsigned red[kPreThreads / 32];
  int s = 0;
  int64_t blk = blockIdx.x;
  if (a.n_scenes > 1) {
    s = find_scene(a.tab.z_prefix, a.n_scenes, blk);
    blk -= a.tab.z_prefix[s];
  }
  const SceneDev& S = scene_of(a, s);
  const int64_t m = S.z_m0 + blk * kPreThreads + threadIdx.x;
  unsigned v = (m >= 0 && m < S.n_in) ? __float_as_uint(fabsf(__ldg(S.x + m))) : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kPreThreads / 32; ++w) v = max(v, red[w]);
    if (v) atomicMax(a.p.xmax + s, v);
  }
}

// kCoef = kFarrowCoef: the synthesis rows (degree 4): per column and segment
// one float4 {z0, z1, z2, (z3, z4) scaled in half precision} (zh_scale);
// kCoef = kGradCoef: the gradient kernel's rows (degree 5, zq + zg, FP32).
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
  if constexpr (kCoef == kFarrowCoef) {
    const float sc = zh_scale(a, s).x;
#pragma unroll
    for (int sg = 0; sg < kFarrowSegs; ++sg) {
      const float* c = acc + sg * kCoef;
      zq[int64_t(sg) * S.z_len] = make_float4(c[0] * sc, c[1] * sc, c[2] * sc, pack_half2(c[3] * sc, c[4] * sc));
    }
  } else {
#pragma unroll
    for (int sg = 0; sg < kFarrowSegs; ++sg) {
      const float* c = acc + sg * kCoef;
      zq[int64_t(sg) * S.z_len] = make_float4(c[0], c[1], c[2], c[3]);
      a.p.zg[S.z_base + col + int64_t(sg) * S.z_len] = make_float2(c[4], c[kCoef - 1]);
    }
  }
}

// ------------------------------------------------------------------ synthesis


// Approximate reciprocal (one MUFU operation, relative error about 2^-23).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// acc + (beta_i / (4 pi d_i(n))) e_i(n) for one chunk sample of an image pair
// (paired layout, see records_from_phi), read from the staged window (kStride
// columns per segment). Y = the pair's Y(n) from its records (see
// gather_pairs), AB its gain terms, I4 its column byte offsets. The rounding of
// the delay, the local variable w, tau / G and the accumulation run as float2
// pairs (one instruction for both images); the window offsets, the loads and
// the Farrow polynomial per image.
// kChecked: the window is processed in several column passes and only columns
// inside this pass count; otherwise every read position lies inside the window
// by construction and the index is only clamped to the window arrays.
// Unchecked reads index the window by byte offset (split_offset's form): the
// offset of the power-4 value, 4 times it for the powers 0..3.
template <int kStride, bool kChecked>
__device__ __forceinline__ float2 pair_sample(const float4* zq, const float2 Y, const float4 AB, const int2 I4,
                                              unsigned rmc4, int rmj, unsigned wmax, float2 acc) {
  const float2 q = __fadd2_rn(Y, make_float2(kRound, kRound));
  const float2 t = __fadd2_rn(q, make_float2(-kRound, -kRound));
  const float2 w = __ffma2_rn(t, make_float2(-1.0f, -1.0f), Y);       // Y - round(Y), exact
  const float2 tg = __ffma2_rn(Y, make_float2(AB.x, AB.y), make_float2(AB.z, AB.w));  // tau / G
  float g0 = rcp_approx(tg.x), g1 = rcp_approx(tg.y);
  const unsigned b0 = __float_as_uint(q.x), b1 = __float_as_uint(q.y);
  unsigned o0, o1;
  if (kChecked) {
    // column of the read position within this pass, then the byte offset of
    // its power-4 value; columns outside the pass contribute nothing
    int c0 = rmj + (I4.x >> 2) + (int(b0 >> 2) - (kRoundBits >> 2));
    int c1 = rmj + (I4.y >> 2) + (int(b1 >> 2) - (kRoundBits >> 2));
    if (unsigned(c0) > wmax) { g0 = 0.0f; c0 = 0; }
    if (unsigned(c1) > wmax) { g1 = 0.0f; c1 = 0; }
    o0 = 4u * ((b0 & 3u) * unsigned(kStride) + unsigned(c0));
    o1 = 4u * ((b1 & 3u) * unsigned(kStride) + unsigned(c1));
  } else {
    constexpr unsigned kCap = unsigned(4 * (kFarrowSegs * kStride - 1));
    o0 = min((b0 & 3u) * unsigned(4 * kStride - 1) + b0 + (unsigned(I4.x) + rmc4), kCap);
    o1 = min((b1 & 3u) * unsigned(4 * kStride - 1) + b1 + (unsigned(I4.y) + rmc4), kCap);
  }
  const unsigned char* zqb = reinterpret_cast<const unsigned char*>(zq);
  const float4 A0 = *reinterpret_cast<const float4*>(zqb + 4u * o0);
  const float4 A1 = *reinterpret_cast<const float4*>(zqb + 4u * o1);
  const float e0 = horner_zh(A0, w.x), e1 = horner_zh(A1, w.y);  // s e (rows scaled by s, gains by 1/s)
  return __ffma2_rn(make_float2(g0, g1), make_float2(e0, e1), acc);
}

// All image pairs of the block for this thread's kChunks samples; rmj[c] =
// r - m_lo + jj N_t of chunk c (its interval jj = jc[c]). acc[c] holds the
// sums over the even and the odd images of the block.
// kKnots = false: interval records, Y = Psi + sigma r from one float4 per pair;
// kKnots = true: knot records, Y = (1 - s) K_jj + s K_jj+1 from two float2 per
// pair (s = r / N_t; half the record storage, one more load and multiply).
// kOne: every chunk of this lane lies in one knot interval (warp-uniform), so
// one record load per pair serves all chunks.
template <int kStride, int kChunks, int kUnroll, bool kChecked, bool kOne, bool kKnots>
__device__ __forceinline__ void gather_pairs(const float4* zq, const float2* rec, const float4* ab_s,
                                             const int2* i4_s, int cntp, const int* jc, const int* rmj,
                                             const float* rf, float invN, unsigned wmax, float2* acc) {
  unsigned rmc4[kChunks];
  float2 wa[kChunks], wb[kChunks];  // interval records: {r, r}; knot records: {1 - s, 1 - s}, {s, s}
  const float2* row[kChunks];      // records of chunk c: row jc[c] of the interval- (knot-) major table
#pragma unroll
  for (int c = 0; c < kChunks; ++c) {
    rmc4[c] = fold_rounding(rmj[c]) << 2;
    if (kKnots) {
      const float sN = rf[c] * invN;
      wa[c] = make_float2(1.0f - sN, 1.0f - sN);
      wb[c] = make_float2(sN, sN);
      row[c] = rec + jc[c] * cntp;
    } else {
      wa[c] = make_float2(rf[c], rf[c]);
      row[c] = reinterpret_cast<const float2*>(reinterpret_cast<const float4*>(rec) + jc[c] * cntp);
    }
  }
  auto pair_y = [&](int c, int q, const float4 R0) {
    if constexpr (kKnots) {
      const float2 K0 = (kOne || c == 0) ? make_float2(R0.x, R0.y) : row[c][q];
      const float2 K1 = (kOne || c == 0) ? make_float2(R0.z, R0.w) : row[c][q + cntp];
      return __ffma2_rn(wb[c], K1, __fmul2_rn(wa[c], K0));
    } else {
      const float4 R = (kOne || c == 0) ? R0 : reinterpret_cast<const float4*>(row[c])[q];
      return __ffma2_rn(wa[c], make_float2(R.z, R.w), make_float2(R.x, R.y));
    }
  };
  auto first = [&](int q) {  // chunk 0's records of pair q (all chunks' with kOne)
    if constexpr (kKnots) {
      const float2 K0 = row[0][q], K1 = row[0][q + cntp];
      return make_float4(K0.x, K0.y, K1.x, K1.y);
    } else {
      return reinterpret_cast<const float4*>(row[0])[q];
    }
  };
  int p = 0;
  for (; p + kUnroll <= cntp; p += kUnroll) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const float4 AB = ab_s[p + u];
      const int2 I4 = i4_s[p + u];
      const float4 R0 = first(p + u);
#pragma unroll
      for (int c = 0; c < kChunks; ++c)
        acc[c] = pair_sample<kStride, kChecked>(zq, pair_y(c, p + u, R0), AB, I4, rmc4[c], rmj[c], wmax, acc[c]);
    }
  }
  for (; p < cntp; ++p) {
    const float4 AB = ab_s[p];
    const int2 I4 = i4_s[p];
    const float4 R0 = first(p);
#pragma unroll
    for (int c = 0; c < kChunks; ++c)
      acc[c] = pair_sample<kStride, kChecked>(zq, pair_y(c, p, R0), AB, I4, rmc4[c], rmj[c], wmax, acc[c]);
  }
}

template <int kThreads, int kChunks, int kWcap, int kRecCap, int kBlock, int kUnroll, bool kKnots>
__global__ void __launch_bounds__(kThreads, (kThreads <= 256 ? 2 : 1)) k_synth(const __grid_constant__ KernelArgs a) {
  static_assert(kBlock <= kThreads, "the record builders give every image of a block its own thread");
  constexpr int kLayout = kKnots ? kRecForwardKnots : kRecForward;
  // relative knot delays of the block (cnt x nk floats): knot records hold twice
  // as many image-knots as interval records hold image-intervals
  constexpr int kPhiCap = (kKnots ? 2 * kRecCap : kRecCap) + kBlock;
  extern __shared__ __align__(16) float4 smem4[];
  float4* zq_s = smem4;                                                  // kFarrowSegs x kWcap
  float2* rec_s = reinterpret_cast<float2*>(zq_s + kFarrowSegs * kWcap);  // kRecCap interval records
  int4* img_s = reinterpret_cast<int4*>(rec_s + kRecCap);                 // kBlock image records
  static_assert((kRecCap * sizeof(float2)) % 16 == 0, "every shared array starts on a 16-byte boundary");
  // prologue scratch aliases the z window (used before the window is staged)
  float4* u_s = smem4;
  float4* um_s = u_s + kThreads * kChunks + 4;                           // moving array
  float4* anc_s = um_s + kThreads * kChunks + 4;                         // 3 x kBlock
  float* phi_s = reinterpret_cast<float*>(anc_s + 3 * kBlock);           // kPhiCap
  // emission-time delays: u_s holds the array increments, then 6 x kBlock anchors, then phi
  float4* an6_s = um_s;
  float* phi_r = reinterpret_cast<float*>(an6_s + 6 * kBlock);
  __shared__ int s_item;
  __shared__ float s_red[2][kThreads / 32];
  __shared__ __align__(8) uint64_t s_mbar;  // completion of the window's bulk copies
  static_assert(kWcap % 4 == 0, "window columns in steps of 4 (the bulk copies' alignment of the rows)");
  static_assert(kBlock <= kThreads, "the record builders give every image at least one thread");
  constexpr int kTile = kThreads * kChunks;
  static_assert(4 * (2 * (kTile + 4) + 3 * kBlock) + kPhiCap <= 4 * kFarrowSegs * kWcap, "prologue scratch");
  static_assert(4 * ((kTile + 4) + 6 * kBlock) + kPhiCap <= 4 * kFarrowSegs * kWcap,
                "prologue scratch (emission-time delays)");
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) mbar_init(&s_mbar, 1);
  unsigned phase = 0;  // of s_mbar, the same in every thread
  // batched calls: the scene of the current item (s_scene) and the scene
  // cursor, kept in shared memory by thread 0 (no registers held over the loop)
  __shared__ int s_scene;
  __shared__ SceneCursor s_cursor;

  if (threadIdx.x == 0) {
    s_cursor = fresh_cursor();
    s_item = int(atomicAdd(a.p.counter, 1u));
    s_scene = (a.n_scenes > 1 && s_item < a.totals[4]) ? scene_at(a.tab.item_prefix, a.n_scenes, s_item, s_cursor) : 0;
  }
  for (;;) {
    __syncthreads();
    const int64_t item = s_item;
    if (item >= a.totals[4]) break;
    // the next item's index is requested now and stored after this item's
    // gather, so that the atomic's round trip overlaps the work
    unsigned next_item = 0;
    if (threadIdx.x == 0) next_item = atomicAdd(a.p.counter, 1u);
    const int s = s_scene;
    const int64_t li = a.n_scenes > 1 ? item - s_cursor.lo : item;
    const SceneDev& S = scene_of(a, s);
    const ItemGeom g = item_geometry(S, li, kTile);

    // --- delay knots of the block over the tile (records in shared memory)
    // the rows are scaled by s (zh_scale), so the image gains are scaled by 1/s
    const float gscale = zh_scale(a, s).y;
    float tmin, tmax;
    int cnt = g.cnt;
    if (S.delay_model == 1) {
      item_records_ret<kThreads, kLayout>(a, S, g, rec_s, img_s, u_s, an6_s, phi_r, &tmin, &tmax, gscale);
    } else if (S.tier_up[g.t] > 1) {
      // band-limited knot upsampling: its scratch takes the z window
      if (!item_records_bl<kThreads, kLayout>(a, S, g, rec_s, img_s, reinterpret_cast<float*>(smem4),
                                           int64_t(kFarrowSegs) * kWcap * 4, &tmin, &tmax, gscale))
        cnt = 0;
    } else {
      item_records<kThreads, kLayout>(a, S, g, rec_s, img_s, u_s, um_s, anc_s, phi_s, &tmin, &tmax, gscale);
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
    // window start congruent to the z rows' origin mod 4 (the rows are padded to
    // a multiple of 4 columns; kept from the layout with a separate power-4 row)
    int m_lo = g.n0 - int(ceilf(tmax)) - 2;
    m_lo -= int(((int64_t(m_lo) - S.z_m0) % 4 + 4) % 4);
    const int width = g.n_end - int(floorf(tmin)) + 2 - m_lo + 1;

    // this thread's samples: warp w owns n0 + 32 (w kChunks + c) + lane
    int jc[kChunks], rr[kChunks], rmj[kChunks];
    float rf[kChunks];
    float2 acc[kChunks];
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
      acc[c] = make_float2(0.0f, 0.0f);
    }
    // every chunk of every lane in one knot interval (e.g. 96-sample intervals
    // aligned with this warp's 96 samples): one record load per image
    bool one = true;
#pragma unroll
    for (int c = 1; c < kChunks; ++c) one = one && (jc[c] == jc[0]);
    one = __all_sync(0xffffffffu, one);
    // paired record layout (see records_from_phi)
    const int cntp = pair_count(cnt);
    const float invN = 1.0f / float(g.N);
    const float4* ab_s = reinterpret_cast<const float4*>(img_s);
    const int2* i4_s = reinterpret_cast<const int2*>(ab_s + cntp);
    const float4* zqg = a.p.zq + S.z_base;

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
          mbar_expect_tx(&s_mbar, unsigned(kFarrowSegs) * bq + a.test_extra_tx);
          for (int sg = 0; sg < kFarrowSegs; ++sg)
            bulk_g2s(zq_s + sg * kWcap + dst0, zqg + int64_t(sg) * S.z_len + src0, bq, &s_mbar);
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
      constexpr int kPairUnroll = kUnroll >= 2 ? kUnroll / 2 : 1;
      if (width <= kWcap) {
        if (one)
          gather_pairs<kWcap, kChunks, kPairUnroll, false, true, kKnots>(zq_s, rec_s, ab_s, i4_s, cntp, jc, rmj, rf,
                                                                         invN, wmax, acc);
        else
          gather_pairs<kWcap, kChunks, kPairUnroll, false, false, kKnots>(zq_s, rec_s, ab_s, i4_s, cntp, jc, rmj,
                                                                          rf, invN, wmax, acc);
      } else {
        gather_pairs<kWcap, kChunks, kPairUnroll, true, false, kKnots>(zq_s, rec_s, ab_s, i4_s, cntp, jc, rmj, rf,
                                                                       invN, wmax, acc);
      }
    }
    float* out = a.p.part + S.part_base + (int64_t(g.mic) * S.n_blocks + g.blk) * S.n_out;
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      const int n = g.n0 + 32 * (warp * kChunks + c) + lane;
      if (valid[c]) out[n] = acc[c].x + acc[c].y;
    }
    __syncthreads();  // shared memory is reused by the next item
    if (threadIdx.x == 0) {
      s_item = int(next_item);
      if (a.n_scenes > 1 && int64_t(next_item) < a.totals[4])
        s_scene = scene_at(a.tab.item_prefix, a.n_scenes, int64_t(next_item), s_cursor);
    }
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

template <int kThreads, int kChunks, int kWcap, int kRecCap, int kBlock, int kUnroll, bool kKnots>
cudaError_t run_synth(const KernelArgs& a, cudaStream_t st) {
  auto kern = k_synth<kThreads, kChunks, kWcap, kRecCap, kBlock, kUnroll, kKnots>;
  const size_t smem = size_t(kFarrowSegs) * kWcap * sizeof(float4) + size_t(kRecCap) * sizeof(float2) +
                      size_t(kBlock) * sizeof(int4);
  static PerDevice setup;  // per device: shared-memory limit set, grid computed
  int grid = 0;
  cudaError_t e = persistent_grid(setup, kern, kThreads, smem, &grid);
  if (e != cudaSuccess) return e;
  const int64_t items = a.totals[4];
  const int g = int(items < grid ? items : grid);
  e = cudaMemsetAsync(a.p.counter, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (g > 0) kern<<<g, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

// Tile configurations of the synthesis launch (see TileConfig).
// Columns: id, threads, chunks, window columns, record capacity (float2),
// images per block, pair unroll x 2, knot records.
#define MSRC_TILE_CONFIGS(X)                \
  X(0, 512, 3, 3040, 4096, 256, 8, 0)       \
  X(1, 256, 2, 1440, 1664, 256, 4, 0)       \
  X(2, 384, 2, 2560, 3072, 256, 4, 0)       \
  X(3, 1024, 1, 3040, 4096, 256, 2, 0)      \
  X(4, 512, 2, 3040, 4096, 256, 8, 0)       \
  X(5, 512, 1, 3040, 4096, 256, 8, 0)       \
  X(6, 512, 3, 3040, 4096, 256, 4, 0)       \
  X(7, 512, 2, 3040, 4096, 256, 16, 0)      \
  X(8, 512, 3, 2240, 8192, 256, 8, 0)       \
  X(9, 512, 2, 2240, 8192, 256, 8, 0)       \
  X(10, 512, 2, 1920, 10240, 256, 8, 0)     \
  X(11, 256, 3, 1440, 2048, 256, 8, 0)      \
  X(12, 256, 3, 1440, 2048, 256, 8, 1)      \
  X(13, 512, 2, 1920, 8448, 256, 8, 1)      \
  X(14, 256, 3, 1200, 4000, 256, 8, 1)

static const TileConfig kConfigs[] = {
#define MSRC_ROW(id, th, ch, wc, rc, bl, un, kn) {th, ch, wc, rc, bl, kn},
    MSRC_TILE_CONFIGS(MSRC_ROW)
#undef MSRC_ROW
};

int tile_config_count() { return int(sizeof(kConfigs) / sizeof(kConfigs[0])); }
const TileConfig& tile_config(int cfg) { return kConfigs[cfg]; }

cudaError_t launch_prefilter(const KernelArgs& a, cudaStream_t st, bool gradient_rows) {
  if (a.totals[3] > 0) {
    const unsigned g = unsigned(a.totals[3]);
    if (!gradient_rows) {  // the scale of the half-precision powers: max |x| per scene
      const cudaError_t e = cudaMemsetAsync(a.p.xmax, 0, sizeof(uint32_t) * size_t(a.n_scenes), st);
      if (e != cudaSuccess) return e;
      k_absmax<<<g, kPreThreads, 0, st>>>(a);
    }
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
#define MSRC_CASE(id, th, ch, wc, rc, bl, un, kn) \
  case id: e = run_synth<th, ch, wc, rc, bl, un, kn != 0>(a, st); break;
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
