// Device helpers shared by the synthesis and adjoint kernels: scene lookup,
// work-item geometry, the per-item delay knots (Sec. II-C, "Fast
// Architecture") and the split of an interpolated delay into read position and
// Farrow fraction (Sec. II-B).
#pragma once

#include <cstdint>

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

// A work item: microphone `mic`, block `blk` (images img0 .. img0+cnt-1 of tier
// t), output samples n0 .. n_end. The knots of tier t touching the tile are
// jf .. jf+nk-1; the item's records cover intervals jf .. jf+nk-2.
struct ItemGeom {
  int mic, blk, t, img0, cnt, N, n0, n_end, jf, nk;
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
  return g;
}

// sqrt(q) for q > 0 in FP64 from an FP32 reciprocal-square-root seed and one
// Newton step: the seed has relative error ~1e-7, the step squares it (~1e-14).
__device__ __forceinline__ double fast_sqrt(double q) {
  const float r = rsqrtf(float(q));
  const double d0 = double(float(q) * r);
  return fma(fma(-d0, d0, q), 0.5 * double(r), d0);
}

// Knot j of an image relative to its anchor knot a: with Delta the FP64
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

// Records of the item's images over its intervals, in shared memory
// (interval-major, so that consecutive images of one interval are adjacent):
//   rec_s[jj * cnt + ib] = {I_j = n_j - D_a, psi_j = -phi_j - 1/2,
//                                -(phi_{j+1} - phi_j) / N_t, D_a - 1/2},  j = jf + jj,
// where tau = d fs / c, D_a = floor(tau) at the anchor knot jf (FP64) and
// phi_j = tau_j - D_a. u_s (nk entries) and anc_s (2 * cnt entries) are
// scratch. Returns this thread's min / max of tau over its knots (window
// bounds of the item).
template <int kThreads>
__device__ void item_records(const KernelArgs& a, const SceneDev& S, const ItemGeom& g, int4* rec_s,
                             float4* u_s, float4* anc_s, float* tmin_out, float* tmax_out) {
  const double* kp = a.p.knot_pos + 3 * (S.knot_base[g.t] + g.jf);
  const double sa0 = kp[0], sa1 = kp[1], sa2 = kp[2];
  for (int jj = threadIdx.x; jj < g.nk; jj += kThreads) {
    const float ux = float(kp[3 * jj] - sa0);
    const float uy = float(kp[3 * jj + 1] - sa1);
    const float uz = float(kp[3 * jj + 2] - sa2);
    u_s[jj] = make_float4(ux, uy, uz, fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
  }
  const double fs_c = S.fs_over_c;
  const uint32_t* codes = a.p.img_code + S.img_base + S.tier_first[g.t] + g.img0;
  const double* mic = S.mics[g.mic];
  for (int ib = threadIdx.x; ib < g.cnt; ib += kThreads) {
    int n[3], p[3];
    unpack_image(codes[ib], n, p);
    const double s0 = 1.0 - 2.0 * p[0], s1 = 1.0 - 2.0 * p[1], s2 = 1.0 - 2.0 * p[2];
    const double D0 = s0 * sa0 + 2.0 * n[0] * S.dims[0] - mic[0];
    const double D1 = s1 * sa1 + 2.0 * n[1] * S.dims[1] - mic[1];
    const double D2 = s2 * sa2 + 2.0 * n[2] * S.dims[2] - mic[2];
    const double da = fast_sqrt(fma(D0, D0, fma(D1, D1, D2 * D2)));
    const double tau = da * fs_c;
    const double Dfl = floor(tau);
    anc_s[2 * ib] = make_float4(float(s0 * D0), float(s1 * D1), float(s2 * D2), float(da));
    anc_s[2 * ib + 1] = make_float4(float(tau - Dfl), __int_as_float(g.jf * g.N - int(Dfl)), float(Dfl), 0.0f);
  }
  __syncthreads();
  const float fsc = S.fsc;
  const float invN = 1.0f / float(g.N);
  const int nrec = g.nk - 1;
  const int total = g.cnt * nrec;
  float tmin = 3.0e38f, tmax = -3.0e38f;
  for (int pidx = threadIdx.x; pidx < total; pidx += kThreads) {
    const int ib = pidx / nrec;
    const int jj = pidx - ib * nrec;
    const float4 A = anc_s[2 * ib];
    const float4 A2 = anc_s[2 * ib + 1];
    float phi0, phi1, d0, d1;
    knot_increment(A, u_s[jj], fsc, A2.x, &phi0, &d0);
    knot_increment(A, u_s[jj + 1], fsc, A2.x, &phi1, &d1);
    rec_s[jj * g.cnt + ib] = make_int4(__float_as_int(A2.y) + jj * g.N, __float_as_int(-phi0 - 0.5f),
                            __float_as_int((phi0 - phi1) * invN), __float_as_int(A2.z - 0.5f));
    tmin = fminf(tmin, A2.z + fminf(phi0, phi1));
    tmax = fmaxf(tmax, A2.z + fmaxf(phi0, phi1));
  }
  *tmin_out = tmin;
  *tmax_out = tmax;
}

// Interpolated delay of one image-sample split into the read position m0
// (window column `col`, not clamped), the Farrow segment `seg` of the fraction
// alpha, its local variable and the delay tau in samples.
// With y = -phi(n) - 1/2, k = round(y) is floor(-phi) except when phi is an
// integer, where it may be one less and alpha = 1 instead of 0: the two
// readings give the same value because the fractional-delay kernel is
// continuous across alpha = 0 / 1 (h(k; 1) = h(k + 1; 0)).
// Segments: a = alpha - 1/2 in [-1/2, 1/2]; seg = round(3 a + 1) in {0, 1, 2}
// (the same rounding constant, one FMA) and the local variable is
// w = 3 a + 1 - seg in [-1/2, 1/2], i.e. half the v = 2 (S alpha - seg) - 1
// of the fit: the device tables hold the coefficients of the powers of w
// (c_q 2^q, an exact rescaling). At a segment boundary either neighbour is
// taken (the segment polynomials agree there to the fit error).
// rec = {I_j, psi_j, -slope_j, D_a - 1/2}; rm = r - m_lo where r = n - n_j.
constexpr float kRound = 12582912.0f;     // 1.5 * 2^23: x + kRound rounds x to an integer
constexpr int kRoundBits = 0x4B400000;    // bit pattern of kRound

struct DelaySplit {
  int col;
  int seg;
  float v;    // w in [-1/2, 1/2]
  float tau;
};

__device__ __forceinline__ DelaySplit split_delay(const int4 rec, int rm, float rf) {
  const float y = fmaf(rf, __int_as_float(rec.z), __int_as_float(rec.y));
  const float q = y + kRound;
  const float a = y - (q - kRound);
  const float q2 = fmaf(a, 3.0f, kRound + 1.0f);
  DelaySplit ds;
  ds.col = rm + rec.x + (__float_as_int(q) - kRoundBits);
  ds.seg = __float_as_int(q2) - kRoundBits;
  ds.v = fmaf(a, 3.0f, (kRound + 1.0f) - q2);  // (kRound + 1) - q2 = 1 - seg exactly
  ds.tau = __int_as_float(rec.w) - y;          // tau(n) = D_a + phi(n)
  return ds;
}

// The same split for a gather from a window of kStride columns per segment:
// idx = seg * kStride + col with the rounding offsets folded into rmc, where
// rmc = rm - kRoundBits * (1 + kStride) (mod 2^32, once per window pass).
template <int kStride>
__device__ __forceinline__ unsigned split_index(const int4 rec, unsigned rmc, float rf, float* w, float* tau) {
  const float y = fmaf(rf, __int_as_float(rec.z), __int_as_float(rec.y));
  const float q = y + kRound;
  const float a = y - (q - kRound);
  const float q2 = fmaf(a, 3.0f, kRound + 1.0f);
  *w = fmaf(a, 3.0f, (kRound + 1.0f) - q2);
  *tau = __int_as_float(rec.w) - y;
  return unsigned(__float_as_int(q2)) * unsigned(kStride) +
         (unsigned(__float_as_int(q)) + unsigned(rec.x) + rmc);
}
__device__ __forceinline__ unsigned fold_rounding(int rm, int stride) {
  return unsigned(rm) - unsigned(kRoundBits) * (1u + unsigned(stride));
}

// Farrow polynomial (degree 5) from the powers 0..3 (A) and 4..5 (B), Horner in w.
__device__ __forceinline__ float horner6(const float4 A, const float2 B, float v) {
  float e = fmaf(B.y, v, B.x);
  e = fmaf(e, v, A.w);
  e = fmaf(e, v, A.z);
  e = fmaf(e, v, A.y);
  return fmaf(e, v, A.x);
}

}  // namespace msrc
