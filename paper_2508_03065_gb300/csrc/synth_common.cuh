// Device helpers shared by the synthesis and adjoint kernels: scene lookup,
// work-item geometry, the per-item delay knots (Sec. II-C, "Fast
// Architecture") and the split of an interpolated delay into read position and
// Farrow fraction (Sec. II-B).
#pragma once

#include <cstdint>

#include <cuda_fp16.h>

#include "msrc_internal.h"

namespace msrc {

__device__ __forceinline__ const SceneDev& scene_of(const KernelArgs& a, int s) {
  return a.n_scenes == 1 ? a.scene0 : a.scenes[s];
}

// Largest s with prefix[s] <= idx (prefix has n + 1 entries).
__device__ __forceinline__ int find_scene(const int64_t* prefix, int n, int64_t idx) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= idx) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Scene of the work items of a persistent CTA. Its items come from one
// increasing counter, so the scene index only grows: the cursor keeps the
// current scene's item range and advances by at most a few scenes before it
// falls back to the binary search (one uncached global load per scene change
// instead of a search per item).
struct SceneCursor {  // plain data: it also lives in shared memory
  int s;
  int64_t lo, hi;
};
__device__ __forceinline__ SceneCursor fresh_cursor() {
  SceneCursor c;
  c.s = 0;
  c.lo = 0;
  c.hi = -1;
  return c;
}
__device__ __forceinline__ int scene_at(const int64_t* prefix, int n, int64_t idx, SceneCursor& c) {
  if (idx >= c.lo && idx < c.hi) return c.s;
  int s = -1;
  if (c.hi >= 0 && idx >= c.hi) {
    for (int k = c.s + 1; k < n && k <= c.s + 4; ++k)
      if (idx < prefix[k + 1]) { s = k; break; }
  }
  if (s < 0) s = find_scene(prefix, n, idx);
  c.s = s;
  c.lo = prefix[s];
  c.hi = prefix[s + 1];
  return s;
}

// Point of a trajectory (FP64): line p0 + v t dir/|dir|, circle
// centre + R (cos, sin, 0)(theta0 + v t / R), or clamped uniform cubic B-spline
// by de Boor's algorithm on the knot vector {0,0,0,0, 1/m, ..., (m-1)/m, 1,1,1,1}
// with u = clamp(t / duration, 0, 1).
__device__ inline void trajectory_point(int kind, const double* p, int n_ctrl, double duration, double t,
                                 double out[3]) {
  if (kind == 0) {
    const double inv = 1.0 / sqrt(p[3] * p[3] + p[4] * p[4] + p[5] * p[5]);
    for (int d = 0; d < 3; ++d) out[d] = p[d] + p[6] * t * p[3 + d] * inv;
  } else if (kind == 1) {
    const double ang = p[5] + p[4] * t / p[3];
    double sn, cs;
    sincos(ang, &sn, &cs);
    out[0] = p[0] + p[3] * cs;
    out[1] = p[1] + p[3] * sn;
    out[2] = p[2];
  } else {
    // in units of the knot spacing: um = m u, knot i at clamp(i - 3, 0, m);
    // de Boor's ratios (u - knot_i) / (knot_{i+4-r} - knot_i) then divide by
    // an integer q = 1..3 (a multiplication by 1/q: one FP64 division per point)
    const int m = n_ctrl - 3;  // segments
    const double um = fmin(double(m), fmax(0.0, t * (double(m) / duration)));
    const int span = min(int(um), m - 1);  // segment index
    auto kk = [m](int i) { return min(max(i - 3, 0), m); };
    double dd[4][3];
    for (int j = 0; j < 4; ++j)
      for (int c = 0; c < 3; ++c) dd[j][c] = p[3 * (span + j) + c];
    const int k = span + 3;
    for (int r = 1; r <= 3; ++r)
      for (int j = 3; j >= r; --j) {
        const int i = j + k - 3;
        const int q = kk(i + 4 - r) - kk(i);
        const double rq = q == 1 ? 1.0 : (q == 2 ? 0.5 : (1.0 / 3.0));
        const double al = q > 0 ? (um - double(kk(i))) * rq : 0.0;
        for (int c = 0; c < 3; ++c) dd[j][c] = fma(al, dd[j][c] - dd[j - 1][c], dd[j - 1][c]);
      }
    for (int c = 0; c < 3; ++c) out[c] = dd[3][c];
  }
}

// Source position s(t); a spline by its segment's cubic (Horner).
__device__ inline void source_position(const SceneDev& S, double t, double out[3]) {
  if (S.traj_kind != 2) {
    trajectory_point(S.traj_kind, S.traj, S.n_ctrl, S.duration, t, out);
    return;
  }
  const int m = S.n_ctrl - 3;
  const double um = fmin(double(m), fmax(0.0, t * (double(m) / S.duration)));
  const int sg = min(int(um), m - 1);
  const double x = um - double(sg);
  for (int c = 0; c < 3; ++c) {
    const double* q = S.traj_poly[sg][c];
    out[c] = fma(fma(fma(q[3], x, q[2]), x, q[1]), x, q[0]);
  }
}

// Displacement of the microphone array a(t) - a(0) (zero for a static array).
__device__ inline void array_displacement(const SceneDev& S, double t, double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  if (!S.arr_moving) return;
  double a0[3], at[3];
  trajectory_point(S.arr_kind, S.arr_params, S.arr_n_ctrl, S.arr_duration, 0.0, a0);
  trajectory_point(S.arr_kind, S.arr_params, S.arr_n_ctrl, S.arr_duration, t, at);
  for (int d = 0; d < 3; ++d) out[d] = at[d] - a0[d];
}

// A work item: microphone `mic`, block `blk` (images img0 .. img0+cnt-1 of tier
// t), output samples n0 .. n_end. The knots of tier t touching the tile are
// jf .. jf+nk-1; the item's records cover intervals jf .. jf+nk-2.
struct ItemGeom {
  int mic, blk, t, img0, cnt, N, n0, n_end, jf, nk;
  int64_t img_off;  // the item's time group in the image table (group * n_images)
};

__device__ __forceinline__ ItemGeom item_geometry(const SceneDev& S, int64_t li, int tile) {
  ItemGeom g;
  // item index of one scene < 2^31 (checked when planning): 32-bit division
  const unsigned l32 = unsigned(li);
  const unsigned mb = l32 / unsigned(S.n_tiles);
  const int tl = int(l32 - mb * unsigned(S.n_tiles));
  g.mic = int(mb / unsigned(S.n_blocks));
  g.blk = int(mb - unsigned(g.mic) * unsigned(S.n_blocks));
  int t = 0;
  while (t + 1 < S.n_tiers && g.blk >= S.block_first[t + 1]) ++t;
  g.t = t;
  const int B = S.tier_block_images[t];
  g.img0 = (g.blk - S.block_first[t]) * B;
  g.cnt = min(B, S.tier_count[t] - g.img0);
  g.N = S.tier_step[t];
  g.n0 = tl * tile;
  g.n_end = int(min(int64_t(g.n0 + tile), S.n_out)) - 1;
  g.jf = g.n0 / g.N;
  g.nk = g.n_end / g.N - g.jf + 2;
  g.img_off = int64_t(tl / S.tile_group) * S.n_images;
  return g;
}

// Knot j of an image relative to its anchor knot a: with Delta the
// image-to-microphone vector at the anchor, w = sigma o Delta_a (FP32),
// u = s(t_j) - s(t_a) and q = |Delta_j|^2 - |Delta_a|^2 = 2 w.u + |u|^2 exactly,
// the distance increment is d_j - d_a = q / (d_a + sqrt(d_a^2 + q)); every
// term is small, so FP32 keeps it to ~1e-7 of the increment.
__device__ __forceinline__ void knot_increment(const float4 A, const float4 U, float fsc, float fa,
                                               float* phi, float* d) {
  const float q = fmaf(2.0f, fmaf(A.x, U.x, fmaf(A.y, U.y, A.z * U.z)), U.w);
  const float den = A.w + sqrtf(fmaf(A.w, A.w, q));
  const float dd = q / den;
  *phi = fmaf(dd, fsc, fa);
  *d = A.w + dd;
}

// knot_increment with a moving array: the vector changes by v = sigma o u - u_m,
// so q = |Delta_j|^2 - |Delta_a|^2 = 2 Delta_a.v + |v|^2
//      = (2 w.u + |u|^2) - 2 sum_d sigma_d u_m,d (w_d + u_d) + |u_m|^2,
// w = sigma o Delta_a (A.xyz), sigma in sg.xyz, u in U, u_m in Um.
__device__ __forceinline__ void knot_increment_moving(const float4 A, const float4 sg, const float4 U,
                                                      const float4 Um, float fsc, float fa, float* phi,
                                                      float* d) {
  float q = fmaf(2.0f, fmaf(A.x, U.x, fmaf(A.y, U.y, A.z * U.z)), U.w);
  const float c = fmaf(sg.x * Um.x, A.x + U.x, fmaf(sg.y * Um.y, A.y + U.y, sg.z * Um.z * (A.z + U.z)));
  q = fmaf(-2.0f, c, q) + Um.w;
  const float den = A.w + sqrtf(fmaf(A.w, A.w, q));
  const float dd = q / den;
  *phi = fmaf(dd, fsc, fa);
  *d = A.w + dd;
}

// Bulk copies through the tensor memory accelerator (cp.async.bulk, untiled):
// one thread issues a whole z row segment into shared memory and the copies
// complete on an mbarrier that every thread then waits on (a bounded wait).
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* mb, unsigned count) {
  asm volatile("mbarrier.init.shared.b64 [%0], %1;\n" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mb, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;\n" ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* mb) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mb))
               : "memory");
}
// One poll of the mbarrier phase; the thread may be suspended for at most
// about kSuspendHintNs while the phase is incomplete.
constexpr unsigned kSuspendHintNs = 8192;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mb, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(mb)), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase `parity` of the mbarrier; gives up (false) after about
// kWaitLimitNs of wall time, or after kSpinLimit polls, whichever comes first.
constexpr int kSpinLimit = 1 << 20;
constexpr uint64_t kWaitLimitNs = uint64_t(1) << 30;  // about 1.07 s
__device__ __forceinline__ bool mbar_wait(uint64_t* mb, unsigned parity) {
  if (mbar_try_wait(mb, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int it = 1; it < kSpinLimit; ++it) {
    if (mbar_try_wait(mb, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
  return false;
}

// Double-float arithmetic (a value is hi + lo, |lo| <= ulp(hi) / 2): Knuth's
// two-sum and the FMA two-product give the rounding error of a float sum or
// product exactly, so sums and products of pairs keep about 44 bits. The
// item anchors below use it in place of FP64, which runs at a small fraction
// of the FP32 rate on this GPU.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -p)));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_sqrt(DF x) {  // x > 0
  const float s = __fsqrt_rn(x.hi);
  const float p = __fmul_rn(s, s);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), fmaf(s, s, -p)), x.lo);
  return fast_two_sum(s, __fmul_rn(r, __fdiv_rn(0.5f, s)));
}

__device__ __forceinline__ float df_floor(DF x) {  // floor of hi + lo (|hi| < 2^24)
  float f = floorf(x.hi);
  if (x.hi == f && x.lo < 0.0f) f -= 1.0f;
  return f;
}

// Anchor of one image at a knot, in double-float: source at s (pairs sH + sL),
// microphone at m (pairs mH + mL), Delta = sigma o s + 2 n o L - m,
// d_a = |Delta|, tau = d_a fs / c, D_a = floor(tau):
// A = {sigma o Delta, d_a}, B = {tau - D_a, D_a}, SG = {sigma, 0} (floats).
// tau is good to about 1e-12 relative, far below the FP32 record terms.
__device__ __forceinline__ void anchor_df(const SceneDev& S, uint32_t code, const float4 sH, const float4 sL,
                                          const DF* m, float4* A, float2* B, float4* SG) {
  int n[3], p[3];
  unpack_image(code, n, p);
  const float sh[3] = {sH.x, sH.y, sH.z}, sl[3] = {sL.x, sL.y, sL.z};
  DF D[3];
  DF q = {0.0f, 0.0f};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const DF sd = p[d] ? DF{-sh[d], -sl[d]} : DF{sh[d], sl[d]};
    const float tn = float(2 * n[d]);  // exact
    const float pr = __fmul_rn(tn, S.dims_hl[d][0]);
    const DF off = fast_two_sum(pr, fmaf(tn, S.dims_hl[d][1], fmaf(tn, S.dims_hl[d][0], -pr)));
    D[d] = df_add(df_add(sd, off), DF{-m[d].hi, -m[d].lo});
    q = df_add(q, df_mul(D[d], D[d]));
  }
  const DF da = df_sqrt(q);
  const DF tau = df_mul(da, DF{S.fsc_hl[0], S.fsc_hl[1]});
  float Dfl = floorf(tau.hi);
  if (tau.hi == Dfl && tau.lo < 0.0f) Dfl -= 1.0f;
  const float fa = __fadd_rn(__fsub_rn(tau.hi, Dfl), tau.lo);
  const float s0 = p[0] ? -1.0f : 1.0f, s1 = p[1] ? -1.0f : 1.0f, s2 = p[2] ? -1.0f : 1.0f;
  *A = make_float4(s0 * D[0].hi, s1 * D[1].hi, s2 * D[2].hi, da.hi);
  *B = make_float2(fa, Dfl);
  *SG = make_float4(s0, s1, s2, 0.0f);
}

// Record layouts: one record per image (the reverse-mode dx kernel), or per
// image pair for the forward synthesis and the gradient kernel; the forward
// synthesis also takes per-knot records (kRecForwardKnots, below), half the
// size of interval records, for tiers whose knots are close together.
constexpr int kRecPlain = 0, kRecForward = 1, kRecAdjoint = 2, kRecForwardKnots = 3;

// Paired record layout of the forward synthesis (kRecForward): images 2p and 2p + 1
// of a block share one 16-byte interval record per interval jj,
//   rec[jj * cntp + p] = {Psi_2p, Psi_2p+1, sigma_2p, sigma_2p+1}    (float4),
// and their image records sit in two arrays at img_s,
//   ab[p] = {a_2p, a_2p+1, b_2p, b_2p+1} (float4), i4[p] = {4 I_2p, 4 I_2p+1} (int2),
// with a = -1 / (S G) and b = (D_a - 1/(2S)) / G (G the image's gain), so that
// tau(n) / G = a Y(n) + b and the gain at n is its reciprocal. cntp = ceil(cnt / 2);
// an odd block's last pair carries a copy of its last image with zero gain
// (a = 0, b = +inf), which reads in-bounds columns and adds nothing. Every
// operand of the pair arithmetic is then one aligned 8-byte register pair.
// Per-knot layout (kRecForwardKnots): per knot jj and pair p one float2
//   kn[jj * cntp + p] = {K_2p, K_2p+1},  K = -S phi_jj - 1/2,
// so that Y = (1 - s) K_jj + s K_jj+1 (s = r / N_t) for a sample of interval jj
// (the same Y as Psi + sigma r); image records as for kRecForward.
__device__ __forceinline__ int pair_count(int cnt) { return (cnt + 1) >> 1; }

// Interval records of an item from the relative delays phi at its knots
// (phi_s[ib * nk + jj]); see item_records for the record layout.
template <int kThreads, int kLayout = kRecPlain>
__device__ __forceinline__ void records_from_phi(const ItemGeom& g, const float* phi_s, float2* rec_s) {
  constexpr bool kPaired = kLayout != kRecPlain;
  const float sN = float(kFarrowSegs) / float(g.N);
  const int nk = g.nk;
  const int nrec = nk - 1;
  const int cntp = pair_count(g.cnt);
  if (kLayout == kRecForwardKnots) {  // one float2 per (knot, pair): K = -S phi - 1/2
    const int tpk = kThreads / g.cnt;
    if (threadIdx.x < tpk * g.cnt) {
      const int j0 = threadIdx.x / g.cnt;
      const int ib = threadIdx.x - j0 * g.cnt;
      for (int jj = j0; jj < nk; jj += tpk) {
        const float K = fmaf(-float(kFarrowSegs), phi_s[ib * nk + jj], -0.5f);
        float* f = reinterpret_cast<float*>(rec_s + jj * cntp + (ib >> 1));
        f[ib & 1] = K;
        if ((ib & 1) == 0 && ib == g.cnt - 1) f[1] = K;  // odd block: the zero-gain copy
      }
    }
    return;
  }
  // image-fastest as in item_records: consecutive threads, consecutive records
  const int tpi = kThreads / g.cnt;
  if (threadIdx.x < tpi * g.cnt) {
    const int j0 = threadIdx.x / g.cnt;
    const int ib = threadIdx.x - j0 * g.cnt;
    for (int jj = j0; jj < nrec; jj += tpi) {
      const float phi0 = phi_s[ib * nk + jj], phi1 = phi_s[ib * nk + jj + 1];
      const float psi = fmaf(-float(kFarrowSegs), phi0, -0.5f), sig = (phi0 - phi1) * sN;
      if (kPaired) {
        float* f = reinterpret_cast<float*>(reinterpret_cast<float4*>(rec_s) + jj * cntp + (ib >> 1));
        const int h = ib & 1;
        f[h] = psi;
        f[2 + h] = sig;
        if (h == 0 && ib == g.cnt - 1) {  // odd block: the zero-gain copy
          f[1] = psi;
          f[3] = sig;
        }
      } else {
        rec_s[jj * g.cnt + ib] = make_float2(psi, sig);
      }
    }
  }
}

// Records of the item's images over its intervals, in shared memory.
// With tau = d fs / c, D_a = floor(tau) at the anchor knot jf (double-float) and
// phi_j = tau_j - D_a, the delay between knots j and j + 1 is
// tau(n) = D_a + phi_j + (phi_{j+1} - phi_j) r / N_t (r = n - n_j). Stored:
//   rec_s[jj * cnt + ib] = {Psi_j = -S phi_j - 1/2, sigma_j = -S (phi_{j+1} - phi_j) / N_t}
//                          (float2, interval-major so that consecutive images of one
//                          interval are adjacent; j = jf + jj; S = kFarrowSegs),
//   img_s[ib]            = {I = n_jf - D_a, D_a - 1/(2S) (float), gain (float), 4 I}
// so that Y(n) = Psi_j + sigma_j r = S (n - tau(n) - n_j + I + jj N_t) - 1/2 up to
// the integer read position, and tau(n) = (D_a - 1/(2S)) - Y / S.
// (kPaired: the same values in the paired layout described above.)
// u_s and um_s (nk entries each), anc_s (3 * cnt entries) and phi_s (cnt * nk
// floats, at most the record capacity plus the block size) are scratch. With
// a moving array the knots also carry the array displacement: per knot
// u_m = a(t_j) - a(t_jf) and the image-to-microphone vector changes by
// sigma o u - u_m. Returns this thread's min / max of tau over its knots
// (window bounds of the item). d_s (cnt * nk floats, nullable) receives the
// distance at every knot of every image (the adjoint's unit vectors).
// Image record of a work item: {I = n_jf - D_a (column offset), D_a - 1/8
// (bits), gain (bits), 4 I (the synthesis gather's byte offset of the column)}.
__device__ __forceinline__ int4 image_record(int I, float Dfl, float gain) {
  return make_int4(I, __float_as_int(Dfl - 0.5f / kFarrowSegs), __float_as_int(gain), int(unsigned(I) << 2));
}

// Writes image ib's record (column offset I, anchor delay floor Dfl, gain) in
// layout kLayout: kRecPlain {I, Dp, gain, 4 I} per image (Dp = D_a - 1/(2S));
// kRecForward per pair {a, a', b, b'} (a = -1/(S G), b = Dp / G) and {4 I, 4 I'};
// kRecAdjoint per pair {Dp, Dp', G, G'} and {I, I'}. An odd block's last pair
// carries a copy of its last image with zero gain.
template <int kLayout>
__device__ __forceinline__ void put_image_record(int4* img_s, int ib, int cnt, int I, float Dfl, float gain) {
  if (kLayout == kRecPlain) {
    img_s[ib] = image_record(I, Dfl, gain);
    return;
  }
  float* ab = reinterpret_cast<float*>(reinterpret_cast<float4*>(img_s) + (ib >> 1));
  int* i4 = reinterpret_cast<int*>(reinterpret_cast<int2*>(reinterpret_cast<float4*>(img_s) + pair_count(cnt)) +
                                   (ib >> 1));
  const int h = ib & 1;
  const float Dp = Dfl - 0.5f / kFarrowSegs;
  if (kLayout == kRecForward || kLayout == kRecForwardKnots) {
    const float inf = __int_as_float(0x7f800000);
    const bool live = gain > 0.0f;
    ab[h] = live ? -(1.0f / kFarrowSegs) / gain : 0.0f;
    ab[2 + h] = live ? Dp / gain : inf;
    i4[h] = int(unsigned(I) << 2);
    if (h == 0 && ib == cnt - 1) {  // odd block: the zero-gain copy
      ab[1] = 0.0f;
      ab[3] = inf;
      i4[1] = i4[0];
    }
  } else {
    ab[h] = Dp;
    ab[2 + h] = gain;
    i4[h] = I;
    if (h == 0 && ib == cnt - 1) {
      ab[1] = Dp;
      ab[3] = 0.0f;
      i4[1] = I;
    }
  }
}

// With unit_xy / unit_z (nullable) the unit vectors of the reverse mode are
// written as well, per image pair and knot {x, x', y, y'} and {z, z'}: the
// source's (sigma o Delta) / d, or with unit_array the microphone's -Delta / d
// (an odd block's zero-gain copy gets zeros).
template <int kThreads, int kLayout = kRecPlain>
__device__ void item_records(const KernelArgs& a, const SceneDev& S, const ItemGeom& g, float2* rec_s,
                             int4* img_s, float4* u_s, float4* um_s, float4* anc_s, float* phi_s,
                             float* tmin_out, float* tmax_out, float gscale = 1.0f, float* d_s = nullptr,
                             float4* unit_xy = nullptr, float2* unit_z = nullptr, bool unit_array = false) {
  // knot positions and array displacements as double-float pairs; increments
  // from the anchor knot jf: hi differences of nearby positions are exact
  const int64_t kj = S.knot_base[g.t] + g.jf;
  const float4* khl = a.p.knot_hl + 2 * kj;
  const float4 sH = khl[0], sL = khl[1];
  for (int jj = threadIdx.x; jj < g.nk; jj += kThreads) {
    const float4 h = khl[2 * jj], l = khl[2 * jj + 1];
    const float ux = (h.x - sH.x) + (l.x - sL.x);
    const float uy = (h.y - sH.y) + (l.y - sL.y);
    const float uz = (h.z - sH.z) + (l.z - sL.z);
    u_s[jj] = make_float4(ux, uy, uz, fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
  }
  const bool moving = S.arr_moving != 0;
  const float4* ahl = a.p.arr_hl + 2 * kj;
  const float4 aH = moving ? ahl[0] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 aL = moving ? ahl[1] : make_float4(0.f, 0.f, 0.f, 0.f);
  if (moving) {
    for (int jj = threadIdx.x; jj < g.nk; jj += kThreads) {
      const float4 h = ahl[2 * jj], l = ahl[2 * jj + 1];
      const float mx = (h.x - aH.x) + (l.x - aL.x);
      const float my = (h.y - aH.y) + (l.y - aL.y);
      const float mz = (h.z - aH.z) + (l.z - aL.z);
      um_s[jj] = make_float4(mx, my, mz, fmaf(mx, mx, fmaf(my, my, mz * mz)));
    }
  }
  const uint32_t* codes = a.p.img_code + S.img_base + g.img_off + S.tier_first[g.t] + g.img0;
  const float* gain = a.p.img_gain + S.img_base + g.img_off + S.tier_first[g.t] + g.img0;
  // the microphone at the anchor knot (carried by the array), double-float
  DF mdf[3];
  {
    const float ah[3] = {aH.x, aH.y, aH.z}, al[3] = {aL.x, aL.y, aL.z};
#pragma unroll
    for (int d = 0; d < 3; ++d)
      mdf[d] = df_add(DF{S.mics_hl[g.mic][d][0], S.mics_hl[g.mic][d][1]}, DF{ah[d], al[d]});
  }
  for (int ib = threadIdx.x; ib < g.cnt; ib += kThreads) {
    float4 A, SG;
    float2 B;
    anchor_df(S, codes[ib], sH, sL, mdf, &A, &B, &SG);
    anc_s[2 * ib] = A;
    anc_s[2 * ib + 1] = make_float4(B.x, B.y, 0.0f, 0.0f);
    anc_s[2 * g.cnt + ib] = SG;
    put_image_record<kLayout>(img_s, ib, g.cnt, g.jf * g.N - int(B.y), B.y, __ldg(gain + ib) * gscale);
  }
  __syncthreads();
  // relative delay phi at every knot of every image (once per knot), then the
  // records from consecutive knots
  const float fsc = S.fsc;
  const int nk = g.nk;
  float tmin = 3.0e38f, tmax = -3.0e38f;
  // thread t takes image t mod cnt and every (kThreads / cnt)-th knot from
  // t / cnt: no division per unit, one anchor load per thread
  const int tpi = kThreads / g.cnt;  // >= 1: a block holds at most kThreads images
  if (threadIdx.x < tpi * g.cnt) {
    const int j0 = threadIdx.x / g.cnt;
    const int ib = threadIdx.x - j0 * g.cnt;
    const float4 A = anc_s[2 * ib];
    const float4 A2 = anc_s[2 * ib + 1];
    const float4 SG = anc_s[2 * g.cnt + ib];
    for (int jj = j0; jj < nk; jj += tpi) {
      float phi, d;
      const float4 U = u_s[jj];
      const float4 Um = moving ? um_s[jj] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (moving) knot_increment_moving(A, SG, U, Um, fsc, A2.x, &phi, &d);
      else knot_increment(A, U, fsc, A2.x, &phi, &d);
      phi_s[ib * nk + jj] = phi;
      if (d_s) d_s[ib * nk + jj] = d;
      tmin = fminf(tmin, A2.y + phi);
      tmax = fmaxf(tmax, A2.y + phi);
      if (unit_xy) {
        // sigma o Delta_j = A + u - sigma o u_m; the microphone's -Delta / d
        // is -sigma o (sigma o Delta) / d
        const float inv = __fdividef(1.0f, d);
        const float ix = unit_array ? -SG.x * inv : inv, iy = unit_array ? -SG.y * inv : inv,
                    iz = unit_array ? -SG.z * inv : inv;
        const int h = ib & 1;
        float* fxy = reinterpret_cast<float*>(unit_xy + (ib >> 1) * nk + jj);
        float* fz = reinterpret_cast<float*>(unit_z + (ib >> 1) * nk + jj);
        fxy[h] = fmaf(-SG.x, Um.x, A.x + U.x) * ix;
        fxy[2 + h] = fmaf(-SG.y, Um.y, A.y + U.y) * iy;
        fz[h] = fmaf(-SG.z, Um.z, A.z + U.z) * iz;
        if (h == 0 && ib == g.cnt - 1) {
          fxy[1] = 0.0f;
          fxy[3] = 0.0f;
          fz[1] = 0.0f;
        }
      }
    }
  }
  __syncthreads();
  records_from_phi<kThreads, kLayout>(g, phi_s, rec_s);
  *tmin_out = tmin;
  *tmax_out = tmax;
}

// item_records for a tier with band-limited knot upsampling (Sec. II-C: the
// distance is a band-limited signal sampled at the knots and recovered by an
// upsampler). The item's records sit at virtual knots k = jf .. jf + nk - 1
// (every N = N_c / U samples, N_c the knot spacing); the distance there is
// sum_i w_p[i] d(j0 - Q + 1 + i) with j0 = floor(k / U), p = k - j0 U and the
// normalised weights w_p of the windowed-sinc kernel. With tau_j = d_j fs / c
// at the knots (double-float, computed once per knot by k_bl_tau), Delta =
// tau_{j0+1} - tau_j0 and the deviations from the chord
// e_i = tau_{j0-Q+1+i} - tau_j0 - (i - Q + 1) Delta, and since the weights sum
// to one,
//   tau(k) = tau_j0 + Delta M_p + sum_i w_p[i] e_i,   M_p = sum_i w_p[i] (i - Q + 1),
// so that the FP32 sum only carries the small chord deviations; tau_j0 - D
// and Delta are formed in double-float and rounded once. D = floor(tau) at knot
// floor(jf / U) is the image's anchor. Scratch `scr` (`cap` floats): D (cnt),
// chord rows (cnt x nj x (2Q + 2)), phi (cnt x nk). If the item does not fit,
// the error word gets kErrUpsampleScratch, no record is written and the result
// is false (the caller then treats the block as empty). With dfl_out / phi_out
// (nullable) the anchors D (cnt floats) are also stored at dfl_out and
// *phi_out points at the relative delays phi[ib * nk + jj] in the scratch: the
// delay at virtual knot jf + jj is D + phi.
template <int kThreads, int kLayout = kRecPlain>
__device__ bool item_records_bl(const KernelArgs& a, const SceneDev& S, const ItemGeom& g, float2* rec_s,
                                int4* img_s, float* scr, int64_t cap, float* tmin_out, float* tmax_out,
                                float gscale = 1.0f, float* dfl_out = nullptr, const float** phi_out = nullptr) {
  const int U = S.tier_up[g.t];
  const int Q = S.up_q;
  const int nk = g.nk;
  const int j0_first = g.jf / U;
  const int nj = (g.jf + nk - 1) / U - j0_first + 1;
  float tmin = 3.0e38f, tmax = -3.0e38f;
  if (bl_scratch_floats(g.cnt, nk, nj, Q) > cap) {
    if (threadIdx.x == 0) atomicOr(a.p.err, kErrUpsampleScratch);
    *tmin_out = 0.0f;
    *tmax_out = 0.0f;
    return false;
  }
  float* dfl_s = scr;
  float* e_s = dfl_s + g.cnt;
  const int er = 2 * Q + 2;
  float* phi_s = e_s + g.cnt * nj * er;
  const int nkt = S.bl_knots[g.t];
  // delays of an image: rows[p * nkt + j + Q] is knot j (the table starts at
  // knot -Q), p its position in the tier in the first time group's order
  const float2* rows = a.p.bl_tau + S.bl_tau_base[g.t] + int64_t(g.mic) * S.tier_count[g.t] * nkt + Q;
  const uint32_t* masters = a.p.vals_out + S.img_base + g.img_off + S.tier_first[g.t] + g.img0;
  const float* gain = a.p.img_gain + S.img_base + g.img_off + S.tier_first[g.t] + g.img0;
  // image-fastest thread mapping (one division per thread): image t mod cnt,
  // intervals / knots from t / cnt in steps of kThreads / cnt
  const int tpi = kThreads / g.cnt;
  const bool act = threadIdx.x < tpi * g.cnt;
  const int t0i = threadIdx.x / g.cnt;
  const int tib = threadIdx.x - t0i * g.cnt;
  for (int jr = act ? t0i : nj; jr < nj; jr += tpi) {
    const int ib = tib;
    const int pidx = ib * nj + jr;
    const int p0 = g.img_off == 0 ? g.img0 + ib
                                   : a.p.m_pos[S.master_base + __ldg(masters + ib)] - S.tier_first[g.t];
    const float2* row = rows + int64_t(p0) * nkt;
    const float2 an = row[j0_first];
    const float Dfl = df_floor(DF{an.x, an.y});  // the anchor, knot floor(jf / U)
    if (jr == 0) {
      dfl_s[ib] = Dfl;
      if (dfl_out) dfl_out[ib] = Dfl;
      put_image_record<kLayout>(img_s, ib, g.cnt, g.jf * g.N - int(Dfl), Dfl, __ldg(gain + ib) * gscale);
    }
    const float2* tv = row + (j0_first + jr - Q + 1);  // knots j0 - Q + 1 .. j0 + Q
    const DF t0{tv[Q - 1].x, tv[Q - 1].y};
    const DF dl = df_add(DF{tv[Q].x, tv[Q].y}, DF{-t0.hi, -t0.lo});
    // chord value at knot i: t0 + (i - Q + 1) dl; knots j0 and j0 + 1 lie on
    // the chord (e = 0)
    float* E = e_s + pidx * er;
#pragma unroll
    for (int i = 0; i < 2 * kMaxUpHalfwidth; ++i) {
      if (i < 2 * Q) {
        if (i == Q - 1 || i == Q) {
          E[i] = 0.0f;
        } else {
          const DF ch = df_add(t0, df_mul(dl, DF{float(i - Q + 1), 0.0f}));
          const DF e = df_add(DF{tv[i].x, tv[i].y}, DF{-ch.hi, -ch.lo});
          E[i] = e.hi + e.lo;
        }
      }
    }
    const DF r0 = df_add(t0, DF{-Dfl, 0.0f});
    E[2 * Q] = r0.hi + r0.lo;
    E[2 * Q + 1] = dl.hi + dl.lo;
  }
  __syncthreads();
  const float* W0 = a.p.upw + S.upw_base[g.t];
  if (act) {
    const int ib = tib;
    const float D = dfl_s[ib];
    // virtual knot k = jf + jj = j0 U + pp, advanced by tpi without dividing
    int j0 = (g.jf + t0i) / U;
    int pp = g.jf + t0i - j0 * U;
    for (int jj = t0i; jj < nk; jj += tpi) {
      const float* E = e_s + (ib * nj + (j0 - j0_first)) * er;
      const float* W = W0 + pp * (2 * Q + 1);
      float phi = fmaf(E[2 * Q + 1], __ldg(W + 2 * Q), E[2 * Q]);
      for (int i = 0; i < 2 * Q; ++i) phi = fmaf(__ldg(W + i), E[i], phi);
      phi_s[ib * nk + jj] = phi;
      tmin = fminf(tmin, D + phi);
      tmax = fmaxf(tmax, D + phi);
      pp += tpi;
      while (pp >= U) {
        pp -= U;
        ++j0;
      }
    }
  }
  __syncthreads();
  records_from_phi<kThreads, kLayout>(g, phi_s, rec_s);
  if (phi_out) *phi_out = phi_s;
  *tmin_out = tmin;
  *tmax_out = tmax;
  return true;
}

// item_records for emission-time (retarded) delays (delay_model 1): the
// distance at reception knot j is the path length d_j = c tau_j with
// c tau_j = |r_i(t_j - tau_j) - m(t_j)|; records, delay and gain follow from
// d_j exactly as for reception-time distances.
//   Anchor (knot jf, double-float, per image): the first-order guess
//   tau_0 = d(t) / (c + u . sigma o s'(t)) (reception-time distance, unit
//   vector and source velocity), one Newton step on F(tau) = tau - |Delta(tau)| fs / c
//   (source at the emission time read from the path table's pairs, linear
//   between its points, kDenseOver per sample; slope in FP32) to tau_a, and the
//   residual eps = |Delta(tau_a)| fs / c - tau_a, which the FP32 stage absorbs.
//   Other knots (FP32, per image and knot): delta_j = tau_j - tau_a solves
//   delta = (d_j - d_a) fs / c + eps, d_a = |Delta(tau_a)|; Newton steps from
//   delta = eps + r h + r2 h^2 / 2 (h = jj N; r, r2 the anchor's first and
//   second derivatives of the delay), a second step only when the first moved
//   delta by 1e-2 samples or more.
//   d_j - d_a uses the exact identity of knot_increment with the vector change
//   v = sigma o (s(e_j) - s(e_a)) - (m_j - m_a). The source displacement
//   between the two emission points comes from the FP32 pair tables (hi
//   differences of nearby positions are exact); the second step reads the
//   table again only when its emission point lies in another segment.
// Scratch: um_s (nk, moving array), an6 (6 x cnt float4), phi_s (cnt x nk).
// The delay at knot jf + jj is D + phi_s[ib * nk + jj], D the image's anchor
// (stored at dfl_out when it is not null).
struct RetAnchor {
  float4 A, H, Lw, dA, Sg, E;
};

__device__ __forceinline__ float ret_increment(const RetAnchor& r, const float4 um, const float4* HI,
                                               const float4* LO, int64_t base_idx, int64_t kmax, float fsc,
                                               float c4, float delta) {
  const int64_t Ka = int64_t(__float_as_int(r.Sg.w)) + base_idx;
  int64_t I = -1;
  float dx = 0.0f, dy = 0.0f, dz = 0.0f, bx = 0.0f, by = 0.0f, bz = 0.0f;
  float step = 1.0f;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    // from the quadratic guess one step is usually enough: a step below 1e-2
    // samples leaves an error of order tau'' (1e-2)^2, far below FP32 rounding
    if (it == 1 && fabsf(step) < 1e-2f) break;
    const float gq = fmaf(-float(kDenseOver), delta, r.H.w);
    const float gi = floorf(gq);
    const float fr = gq - gi;
    const int64_t In = min(max(Ka + int64_t(gi), int64_t(0)), kmax);
    if (In != I) {  // the emission point left the table segment read last: read its own
      I = In;
      const float4 h0 = HI[I], h1 = HI[I + 1], l0 = LO[I], l1 = LO[I + 1];
      dx = (h1.x - h0.x) + (l1.x - l0.x);
      dy = (h1.y - h0.y) + (l1.y - l0.y);
      dz = (h1.z - h0.z) + (l1.z - l0.z);
      // displacement of the segment start from the anchor's emission point
      bx = fmaf(-r.H.w, r.dA.x, (h0.x - r.H.x) + (l0.x - r.Lw.x));
      by = fmaf(-r.H.w, r.dA.y, (h0.y - r.H.y) + (l0.y - r.Lw.y));
      bz = fmaf(-r.H.w, r.dA.z, (h0.z - r.H.z) + (l0.z - r.Lw.z));
    }
    const float frc = (In == Ka + int64_t(gi)) ? fr : gq - float(I - Ka);  // clamped: extrapolate
    const float vx = fmaf(r.Sg.x, fmaf(frc, dx, bx), -um.x);
    const float vy = fmaf(r.Sg.y, fmaf(frc, dy, by), -um.y);
    const float vz = fmaf(r.Sg.z, fmaf(frc, dz, bz), -um.z);
    const float q = fmaf(2.0f, fmaf(r.A.x, vx, fmaf(r.A.y, vy, r.A.z * vz)), fmaf(vx, vx, fmaf(vy, vy, vz * vz)));
    const float dd = __fdividef(q, r.A.w + sqrtf(fmaf(r.A.w, r.A.w, q)));
    const float gs = __fdividef((r.A.x + vx) * r.Sg.x * dx + (r.A.y + vy) * r.Sg.y * dy + (r.A.z + vz) * r.Sg.z * dz,
                                r.A.w + dd);
    step = __fdividef(delta - fmaf(dd, fsc, r.E.x), fmaf(gs, c4, 1.0f));
    delta -= step;
  }
  return delta;
}

template <int kThreads, int kLayout = kRecPlain>
__device__ void item_records_ret(const KernelArgs& a, const SceneDev& S, const ItemGeom& g, float2* rec_s,
                                 int4* img_s, float4* um_s, float4* an6, float* phi_s, float* tmin_out,
                                 float* tmax_out, float gscale = 1.0f, float* dfl_out = nullptr) {
  const bool moving = S.arr_moving != 0;
  const int64_t kj = S.knot_base[g.t] + g.jf;
  const float4* ahl = a.p.arr_hl + 2 * kj;
  const float4 aH = moving ? ahl[0] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 aL = moving ? ahl[1] : make_float4(0.f, 0.f, 0.f, 0.f);
  if (moving) {
    for (int jj = threadIdx.x; jj < g.nk; jj += kThreads) {
      const float4 h = ahl[2 * jj], l = ahl[2 * jj + 1];
      um_s[jj] = make_float4((h.x - aH.x) + (l.x - aL.x), (h.y - aH.y) + (l.y - aL.y), (h.z - aH.z) + (l.z - aL.z),
                             0.0f);
    }
  }
  // double-float operands: the source at the anchor's reception time and the
  // microphone there (carried by the array)
  const float4 sH = a.p.knot_hl[2 * kj], sL = a.p.knot_hl[2 * kj + 1];
  DF mdf[3];
  {
    const float ah[3] = {aH.x, aH.y, aH.z}, al[3] = {aL.x, aL.y, aL.z};
#pragma unroll
    for (int d = 0; d < 3; ++d)
      mdf[d] = df_add(DF{S.mics_hl[g.mic][d][0], S.mics_hl[g.mic][d][1]}, DF{ah[d], al[d]});
  }
  const DF fscd{S.fsc_hl[0], S.fsc_hl[1]};
  const uint32_t* codes = a.p.img_code + S.img_base + g.img_off + S.tier_first[g.t] + g.img0;
  const float* gain = a.p.img_gain + S.img_base + g.img_off + S.tier_first[g.t] + g.img0;
  const float4* HI = a.p.dense_hi + S.dense_base;
  const float4* LO = a.p.dense_lo + S.dense_base;
  const int64_t kmax = S.n_dense - 2;  // last table index whose successor exists
  // table coordinate of emission sample n_a - tau is x0 - kDenseOver tau
  const int64_t x0 = int64_t(kDenseOver) * (int64_t(g.jf) * g.N) - S.dense_k0;
  const float c4 = float(kDenseOver) * S.fsc;  // delay change (samples) per metre and table step
  // table index of the reception time itself (the velocity there seeds the anchor)
  const int64_t k_rec = min(max(x0, int64_t(0)), kmax);
  const float4 vr0 = HI[k_rec], vr1 = HI[k_rec + 1];
  for (int ib = threadIdx.x; ib < g.cnt; ib += kThreads) {
    int n[3], p[3];
    unpack_image(codes[ib], n, p);
    float sg[3];
    DF o[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      sg[d] = p[d] ? -1.0f : 1.0f;
      const float tn = float(2 * n[d]);  // exact
      const float pr = __fmul_rn(tn, S.dims_hl[d][0]);
      const DF off = fast_two_sum(pr, fmaf(tn, S.dims_hl[d][1], fmaf(tn, S.dims_hl[d][0], -pr)));
      o[d] = df_add(off, DF{-mdf[d].hi, -mdf[d].lo});  // 2 n L - m
    }
    // first-order guess from the reception-time distance and the source velocity
    DF tau;
    {
      const float shh[3] = {sH.x, sH.y, sH.z}, sll[3] = {sL.x, sL.y, sL.z};
      DF q = {0.0f, 0.0f};
      float dot = 0.0f;
      const float vd[3] = {vr1.x - vr0.x, vr1.y - vr0.y, vr1.z - vr0.z};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const DF D = df_add(DF{sg[d] * shh[d], sg[d] * sll[d]}, o[d]);
        q = df_add(q, df_mul(D, D));
        dot = fmaf(D.hi * sg[d], vd[d], dot);
      }
      const DF d0 = df_sqrt(q);
      const float gsl = dot / d0.hi * c4;
      tau = df_mul(df_mul(d0, fscd), DF{1.0f / (1.0f + gsl), 0.0f});
    }
    // source at the emission time n_a - tau from the path table (linear between
    // its points), and the image-to-microphone vector and distance there
    DF Dv[3], dist;
    int64_t k = 0;
    float f = 0.0f;
    float4 h0, h1, l0, l1;
    auto eval = [&](DF tv) {
      const float ti = df_floor(tv);
      const float tr = __fadd_rn(__fsub_rn(tv.hi, ti), tv.lo);  // tau - ti, in [0, 1) up to rounding
      const float xr = -float(kDenseOver) * tr;
      const float xi = floorf(xr);
      const int64_t kk = x0 - int64_t(kDenseOver) * int64_t(ti) + int64_t(xi);
      k = min(max(kk, int64_t(0)), kmax);
      f = (xr - xi) + float(kk - k);  // the fraction (extrapolated when clamped)
      h0 = HI[k];
      h1 = HI[k + 1];
      l0 = LO[k];
      l1 = LO[k + 1];
      const float h0v[3] = {h0.x, h0.y, h0.z}, l0v[3] = {l0.x, l0.y, l0.z};
      const float dsv[3] = {(h1.x - h0.x) + (l1.x - l0.x), (h1.y - h0.y) + (l1.y - l0.y),
                            (h1.z - h0.z) + (l1.z - l0.z)};
      DF q = {0.0f, 0.0f};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const DF sd = df_add(DF{h0v[d], l0v[d]}, DF{__fmul_rn(f, dsv[d]), 0.0f});
        Dv[d] = df_add(DF{sg[d] * sd.hi, sg[d] * sd.lo}, o[d]);
        q = df_add(q, df_mul(Dv[d], Dv[d]));
      }
      dist = df_sqrt(q);
    };
    eval(tau);
    {
      const float gsl = ((Dv[0].hi * sg[0]) * (h1.x - h0.x) + (Dv[1].hi * sg[1]) * (h1.y - h0.y) +
                         (Dv[2].hi * sg[2]) * (h1.z - h0.z)) / dist.hi * c4;
      const DF res = df_add(tau, df_mul(dist, DF{-fscd.hi, -fscd.lo}));  // tau - d fs / c
      tau = df_add(tau, DF{-res.hi / (1.0f + gsl), 0.0f});
    }
    eval(tau);
    const DF resid = df_add(df_mul(dist, fscd), DF{-tau.hi, -tau.lo});
    const float eps = resid.hi + resid.lo;
    const float Dfl = df_floor(tau);
    const float fa = __fadd_rn(__fsub_rn(tau.hi, Dfl), tau.lo);
    const float dsx = (h1.x - h0.x) + (l1.x - l0.x);
    const float dsy = (h1.y - h0.y) + (l1.y - l0.y);
    const float dsz = (h1.z - h0.z) + (l1.z - l0.z);
    const float Ax = Dv[0].hi, Ay = Dv[1].hi, Az = Dv[2].hi, da = dist.hi;
    const float gsl = (Ax * sg[0] * dsx + Ay * sg[1] * dsy + Az * sg[2] * dsz) / da * c4;
    // curvature of the delay for the guess of the other knots (still microphone):
    // with D(e) = d(e) fs / c, tau'' = D'' / (1 + D')^3, D'' = fs/c ((|v|^2 - (u.v)^2) / d + u.a),
    // v and a the per-sample velocity and acceleration of sigma o s from table differences
    float r2;
    {
      const int64_t k2 = min(k + 2, kmax + 1);
      const float4 h2 = HI[k2], l2 = LO[k2];
      const float ax = ((h2.x - h1.x) + (l2.x - l1.x)) - dsx;
      const float ay = ((h2.y - h1.y) + (l2.y - l1.y)) - dsy;
      const float az = ((h2.z - h1.z) + (l2.z - l1.z)) - dsz;
      const float kd = float(kDenseOver), kd2 = kd * kd;
      const float uv = (Ax * sg[0] * dsx + Ay * sg[1] * dsy + Az * sg[2] * dsz) / da * kd;
      const float ua = (Ax * sg[0] * ax + Ay * sg[1] * ay + Az * sg[2] * az) / da * kd2;
      const float vv = (dsx * dsx + dsy * dsy + dsz * dsz) * kd2;
      const float D2 = S.fsc * ((vv - uv * uv) / da + ua);
      const float o1 = 1.0f + gsl;
      r2 = D2 / (o1 * o1 * o1);
    }
    an6[6 * ib + 0] = make_float4(Ax, Ay, Az, da);
    an6[6 * ib + 1] = make_float4(h0.x, h0.y, h0.z, f);
    an6[6 * ib + 2] = make_float4(l0.x, l0.y, l0.z, fa);
    // table step of the path there; rate of change of the delay per output sample (still microphone)
    an6[6 * ib + 3] = make_float4(dsx, dsy, dsz, gsl / (1.0f + gsl));
    an6[6 * ib + 4] = make_float4(sg[0], sg[1], sg[2], __int_as_float(int(k)));
    an6[6 * ib + 5] = make_float4(eps, Dfl, r2, 0.0f);
    if (dfl_out) dfl_out[ib] = Dfl;
    put_image_record<kLayout>(img_s, ib, g.cnt, g.jf * g.N - int(Dfl), Dfl, __ldg(gain + ib) * gscale);
  }
  __syncthreads();
  const int nk = g.nk;
  const float fsc = S.fsc;
  float tmin = 3.0e38f, tmax = -3.0e38f;
  const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  // (image, knot) units image-fastest, so that a warp's lanes take neighbouring
  // images (nearby emission points, shared cache lines) at one knot; four
  // knots per pass so that their table reads are in flight together
  constexpr int kRetUnits = 4;
  const int tpi = kThreads / g.cnt;  // image-fastest mapping: one division per thread
  if (threadIdx.x < tpi * g.cnt) {
    const int j0 = threadIdx.x / g.cnt;
    const int ib = threadIdx.x - j0 * g.cnt;
    const RetAnchor r{an6[6 * ib], an6[6 * ib + 1], an6[6 * ib + 2], an6[6 * ib + 3], an6[6 * ib + 4],
                      an6[6 * ib + 5]};
    for (int jb = j0; jb < nk; jb += kRetUnits * tpi) {
      float de[kRetUnits];
#pragma unroll
      for (int k = 0; k < kRetUnits; ++k) {
        const int jj = min(jb + k * tpi, nk - 1);
        const float4 um = moving ? um_s[jj] : zero4;
        const float h = float(jj * g.N);
        de[k] = ret_increment(r, um, HI, LO, int64_t(kDenseOver) * jj * g.N, kmax, fsc, c4,
                              fmaf(0.5f * r.E.z * h, h, fmaf(r.dA.w, h, r.E.x)));
      }
#pragma unroll
      for (int k = 0; k < kRetUnits; ++k) {
        const int jj = jb + k * tpi;
        if (jj < nk) {
          const float phi = r.Lw.w + de[k];
          phi_s[ib * nk + jj] = phi;
          tmin = fminf(tmin, r.E.y + phi);
          tmax = fmaxf(tmax, r.E.y + phi);
        }
      }
    }
  }
  __syncthreads();
  records_from_phi<kThreads, kLayout>(g, phi_s, rec_s);
  *tmin_out = tmin;
  *tmax_out = tmax;
}

// Interpolated delay of one image-sample split into the read position m0
// (window column `col`, not clamped), the Farrow segment `seg` of the fraction
// alpha, its local variable w and the delay tau in samples.
// With p = n - tau(n) the read position, Y = S p - 1/2 (relative to an integer
// offset), one rounding R = round(Y) gives m0 = floor(R / S) and seg = R mod S
// (S = 4, shifts and masks), and w = Y - R = S alpha - seg - 1/2 in [-1/2, 1/2]
// is half the v = 2 (S alpha - seg) - 1 of the fit: the device tables hold the
// coefficients of the powers of w (c_q 2^q, an exact rescaling). At a segment
// boundary either neighbour is taken, and alpha = 1 reads as alpha = 0 at
// m0 + 1: the pieces agree there to the fit error (the fractional-delay kernel
// is continuous, h(k; 1) = h(k + 1; 0)).
// rec = {Psi_j, sigma_j}; rmI = r - m_lo + I + jj N_t (r = n - n_j); Dp = img.y.
constexpr float kRound = 12582912.0f;     // 1.5 * 2^23: x + kRound rounds x to an integer
constexpr int kRoundBits = 0x4B400000;    // bit pattern of kRound
static_assert(kFarrowSegs == 4, "the segment split uses R mod 4 and R / 4");
static_assert((kRoundBits & 3) == 0, "kRound bits divisible by the segment count");

struct DelaySplit {
  int col;
  int seg;
  float w;
  float tau;
};

__device__ __forceinline__ DelaySplit split_delay(const float2 rec, int rmI, float rf, float Dp) {
  const float Y = fmaf(rf, rec.y, rec.x);
  const float q = Y + kRound;
  const int b = __float_as_int(q);
  DelaySplit ds;
  ds.col = rmI + ((b >> 2) - (kRoundBits >> 2));
  ds.seg = b & 3;
  ds.w = Y - (q - kRound);
  ds.tau = fmaf(Y, -1.0f / kFarrowSegs, Dp);
  return ds;
}

// The same split for a gather from a window of kStride columns per segment:
// returns seg * kStride + col (mod 2^32) with rmc = r - m_lo + jj N_t -
// kRoundBits / 4 (once per chunk and window pass) and I = img.x.
template <int kStride>
__device__ __forceinline__ unsigned split_index(const float2 rec, int I, unsigned rmc, float rf, float Dp,
                                                float* w, float* tau) {
  const float Y = fmaf(rf, rec.y, rec.x);
  const float q = Y + kRound;
  const unsigned b = unsigned(__float_as_int(q));
  *w = Y - (q - kRound);
  *tau = fmaf(Y, -1.0f / kFarrowSegs, Dp);
  return (b & 3u) * unsigned(kStride) + ((b >> 2) + unsigned(I) + rmc);
}
__device__ __forceinline__ unsigned fold_rounding(int r_minus_mlo_plus_jjN) {
  return unsigned(r_minus_mlo_plus_jjN) - unsigned(kRoundBits >> 2);
}

// The same index times 4 (the byte offset of a 4-byte element), formed from
// the rounded bits b without splitting them: with seg = b & 3,
//   4 (seg kStride + col) = seg (4 kStride - 1) + b + 4 I + 4 rmc   (mod 2^32),
// since b - seg = 4 (b >> 2). I4 = 4 img.x (once per image), rmc4 = 4 rmc.
template <int kStride>
__device__ __forceinline__ unsigned split_offset(const float2 rec, unsigned I4, unsigned rmc4, float rf, float Dp,
                                                 float* w, float* tau) {
  const float Y = fmaf(rf, rec.y, rec.x);
  const float q = Y + kRound;
  const unsigned b = unsigned(__float_as_int(q));
  *w = Y - (q - kRound);
  *tau = fmaf(Y, -1.0f / kFarrowSegs, Dp);
  return (b & 3u) * unsigned(4 * kStride - 1) + b + (I4 + rmc4);
}

// Power-of-two scale of the synthesis rows, chosen for their half-precision
// powers 3 and 4. |z_q| <= (sum_k |c_q[k]|) max|x| for q = 3, 4 (zh_gain = the
// larger sum over the segments), so s = 2^(14 - e) with C max|x| = m 2^e,
// m in [1/2, 1), keeps every scaled value at or below 2^14 (half precision
// holds 65504) and as high in its range as the bound allows (relative
// precision 2^-11 down to 2^-14 of the bound). All five powers are stored
// times s and the image gains times 1/s (exact powers of two): {s, 1/s}. A
// silent or non-finite signal uses s = 1.
__device__ __forceinline__ float2 zh_scale(const KernelArgs& a, int scene) {
  const float mx = __uint_as_float(a.p.xmax[scene]) * a.zh_gain;
  if (!(mx > 0.0f) || !(mx < 3.0e38f)) return make_float2(1.0f, 1.0f);
  int e = 0;
  const float m = frexpf(mx, &e);
  int k = (m == 0.5f ? 15 : 14) - e;
  k = max(-120, min(120, k));
  return make_float2(ldexpf(1.0f, k), ldexpf(1.0f, -k));
}

// The bits of (lo, hi) rounded to half precision, as the 4th lane of a float4
// row (moved, never used as a float).
__device__ __forceinline__ float pack_half2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return __uint_as_float(*reinterpret_cast<const unsigned*>(&h));
}

// Farrow polynomial (degree 4) from a synthesis row A = {s z0, s z1, s z2,
// half2(s z3, s z4)}, Horner in w: s e (the caller's gains carry the 1/s).
__device__ __forceinline__ float horner_zh(const float4 A, float w) {
  const unsigned u = __float_as_uint(A.w);
  const float2 h = __half22float2(*reinterpret_cast<const __half2*>(&u));
  float e = fmaf(h.y, w, h.x);
  e = fmaf(e, w, A.z);
  e = fmaf(e, w, A.y);
  return fmaf(e, w, A.x);
}

// Farrow polynomial (degree 4) from the powers 0..3 (A) and 4 (B), Horner in w.
__device__ __forceinline__ float horner5(const float4 A, const float B, float w) {
  float e = fmaf(B, w, A.w);
  e = fmaf(e, w, A.z);
  e = fmaf(e, w, A.y);
  return fmaf(e, w, A.x);
}

}  // namespace msrc
