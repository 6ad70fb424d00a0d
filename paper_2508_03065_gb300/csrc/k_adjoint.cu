// Reverse mode of the synthesis (adjoint of Eq. 8 with the Farrow structure of
// Eq. 5 and the hierarchical knots of Sec. II-C).
//
// With e_i(n) = sum_q w^q z[seg][q][m0], g_i(n) = beta_i / (4 pi d_i(n)) and
// y = sum_i g_i e_i, for an upstream gradient dy:
//   dx[m]       = sum_{s,q,k} c[s][q][k] W[s][q][m + k],
//                 W[s][q][m] = sum over image-samples with (seg, m0) = (s, m) of dy g w^q
//   dL/dd_i(n)  = -dy g (fs/c) (S de/dw + e / tau)         (tau = d fs / c, S segments,
//                 w = S alpha - seg - 1/2 the local variable of the Farrow tables)
//   dL/dd_{i,j} = sum_n dL/dd_i(n) * (linear-interpolation weight of knot j)
//   dL/ds(t_j)  = sum_i dL/dd_{i,j} (sigma_i o Delta_{i,j}) / d_{i,j}
//   dL/dbeta_w  = sum_i (dbeta_i/dbeta_w) sum_n dy e / (4 pi d)
// then the trajectory parameters through ds(t_j)/dparams.
//
// k_adj_grad: persistent over (scene, mic, image block, tile) items, shaped
//   like the forward synthesis: per image-sample e and de/dv from the staged z
//   window, the knot gradients (a lane's knots are the same for every image)
//   and the wall gradients accumulate in registers; no barriers in the image
//   loop. Per item: a warp-segmented scan folds the lanes' knot vectors into
//   knot slots; the wall partials are reduced in a fixed order.
// k_adj_dx: persistent over (scene, mic, block group, tile range) items, a
//   group being consecutive image blocks of one tier (about 256 images, at
//   least two blocks), a range spanning more than the largest delay; walks
//   the range's tiles in order, two output samples per thread. dy g w^q of
//   every image of the group is scattered into one shared w window; within
//   one image no two samples share a (segment, column) bin, so images are
//   separated by a barrier and no atomics are used. Each tile's window is
//   correlated once with the Farrow coefficients and added, in tile order, to
//   the dx row of the range's parity (ranges two apart write disjoint
//   columns). The window is the union of the blocks' delay ranges, which the
//   gradient kernel stores per (mic, block, tile) item; wide windows run in
//   several column passes.
// k_dx_final / k_knot_final / k_param_partial + k_param_final / k_beta_final:
// fixed-order sums.
#include <cstdint>

#include "msrc_internal.h"
#include "synth_common.cuh"

namespace msrc {
namespace {

constexpr int kBwThreads = 512;
constexpr int kBwChunks = 2;                    // output samples per thread per tile
constexpr int kBwTile = kBwThreads * kBwChunks;
constexpr int kBwRecCap = 3328;                 // records (image x interval)
constexpr int kBwUnitCap = 3584;                // unit vectors (image x knot)
constexpr int kBwBlock = 256;                   // images per block at most
static_assert(kBwBlock <= kBwThreads, "the record builders give every image of a block its own thread");
constexpr int kGradWcap = 1408;                 // shared z window of the gradient kernel
constexpr int kDxWcap = 1760;                   // shared w window of the dx kernel
constexpr int kSegCap = 33;                     // knot intervals touched by 32 consecutive samples

constexpr size_t kGradSmem = size_t(kFarrowSegs) * kGradWcap * (sizeof(float4) + sizeof(float2)) +
                             size_t(kBwRecCap) * sizeof(float2) + size_t(kBwBlock) * sizeof(int4) +
                             size_t(kBwUnitCap) * sizeof(float4) + size_t(2 * kBwBlock) * sizeof(float4);
constexpr int kDxGroupImages = 256;             // images per dx item (block group), about; >= 2 blocks
constexpr int kDxSlots = kFarrowSegs * kDxWcap + 4;   // w window + a discard slot (+ 16-byte alignment)
static_assert((kDxSlots * sizeof(float)) % 16 == 0 && (kBwRecCap * sizeof(float2)) % 16 == 0,
              "every shared array of the reverse-mode kernels starts on a 16-byte boundary");
static_assert((kFarrowSegs * kGradWcap * sizeof(float2)) % 16 == 0, "gradient window alignment");
constexpr size_t kDxSmem = size_t(kDxSlots) * (sizeof(float4) + sizeof(float)) +
                           size_t(kBwRecCap) * sizeof(float2) + size_t(kBwBlock) * sizeof(int4) +
                           size_t(2 * (kBwTile + 4) + 3 * kBwBlock) * sizeof(float4) +
                           size_t(kBwRecCap + kBwBlock) * sizeof(float);
static_assert(kBwRecCap % 2 == 0, "16-byte alignment of the image records");
// the gradient kernel's z window (powers 0..3 and 4..5) is free while records are built
constexpr int64_t kGradScratchFloats = int64_t(kFarrowSegs) * kGradWcap * 6;
static_assert(kBwBlock <= kBwThreads, "the record builders give every image at least one thread");
static_assert(kGradSmem <= 232448 && kDxSmem <= 232448, "shared memory per CTA");

// dbeta_i / dbeta_w of beta_i = prod_w beta_w^{e_w} (FP64; handles beta_w = 0).
__device__ void beta_weights(const SceneDev& S, uint32_t code, double out[6]) {
  int n[3], p[3];
  unpack_image(code, n, p);
  int e[6];
  for (int d = 0; d < 3; ++d) {
    e[2 * d] = abs(n[d] - p[d]);
    e[2 * d + 1] = abs(n[d]);
  }
  for (int w = 0; w < 6; ++w) {
    if (e[w] == 0) { out[w] = 0.0; continue; }
    double v = double(e[w]);
    for (int r = 0; r < e[w] - 1; ++r) v *= S.beta[w];
    for (int o = 0; o < 6; ++o)
      if (o != w)
        for (int r = 0; r < e[o]; ++r) v *= S.beta[o];
    out[w] = v;
  }
}

// Per image of the sorted table: dbeta_i/dbeta_w / (4 pi) and the gain.
__global__ void k_beta_table(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[0]) return;
  int s = 0;
  int64_t i = gid;
  if (a.n_scenes > 1) {
    s = find_scene(a.tab.enum_prefix, a.n_scenes, gid);
    i = gid - a.tab.enum_prefix[s];
  }
  const SceneDev& S = scene_of(a, s);
  double D[6];
  beta_weights(S, a.p.img_code[S.img_base + i], D);
  const double hb = 1.0 / (4.0 * 3.14159265358979323846);
  float4* o = a.p.bwt + 2 * (S.img_base + i);
  o[0] = make_float4(float(D[0] * hb), float(D[1] * hb), float(D[2] * hb), float(D[3] * hb));
  o[1] = make_float4(float(D[4] * hb), float(D[5] * hb), a.p.img_gain[S.img_base + i], 0.0f);
}

__device__ __forceinline__ int next_item(const KernelArgs& a, int* s_item) {
  if (threadIdx.x == 0) *s_item = int(atomicAdd(a.p.counter, 1u));
  __syncthreads();
  return *s_item;
}

// Item delay range -> window [m_lo, m_lo + width); the block-wide range is
// returned in *tmin_out / *tmax_out when they are not null.
template <int kThreads>
__device__ __forceinline__ void window_of(float tmin, float tmax, const ItemGeom& g, float (*s_red)[kThreads / 32],
                                          int* m_lo, int* width, float* tmin_out = nullptr,
                                          float* tmax_out = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
    tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
  }
  if (lane == 0) { s_red[0][warp] = tmin; s_red[1][warp] = tmax; }
  __syncthreads();
  tmin = s_red[0][0];
  tmax = s_red[1][0];
  for (int w = 1; w < kThreads / 32; ++w) {
    tmin = fminf(tmin, s_red[0][w]);
    tmax = fmaxf(tmax, s_red[1][w]);
  }
  *m_lo = g.n0 - int(ceilf(tmax)) - 2;
  *width = g.n_end - int(floorf(tmin)) + 2 - *m_lo + 1;
  if (tmin_out) *tmin_out = tmin;
  if (tmax_out) *tmax_out = tmax;
}

// Shared-memory scratch of the record builders in both reverse-mode kernels:
// u_s, um_s (kBwTile + 4 float4 each), anc_s (3 kBwBlock float4) and phi_s
// (kBwRecCap + kBwBlock floats), contiguous and in that order. The
// band-limited builder takes the region from u_s on; the emission-time builder
// takes u_s for the microphone path and its anchors (6 float4 per image) from
// um_s on, across um_s and anc_s.
constexpr int64_t kRecScratchFloats = 4 * (2 * (kBwTile + 4) + 3 * kBwBlock) + kBwRecCap + kBwBlock;
static_assert(6 * kBwBlock <= (kBwTile + 4) + 3 * kBwBlock, "emission-time anchors within um_s and anc_s");
static_assert(kBwTile + 1 <= kBwTile + 4, "microphone path of every knot of a tile (N >= 1) within u_s");

__device__ __forceinline__ bool opt_tier(const SceneDev& S, int t) { return S.delay_model == 1 || S.tier_up[t] > 1; }

// Records of one item in layout kLayout, by the builder of the item's tier:
// emission-time delays, band-limited upsampling (scratch from u_s on,
// kRecScratchFloats floats) or linear knots (d_s, nullable, receives the knot
// distances). Returns the item's image count: 0 when the upsampler's scratch
// did not fit (the builder then flags the error word and writes no record).
// For the two option builders, dfl_out (cnt floats, nullable) receives the
// anchors D and *phi_out the relative knot delays phi (cnt x nk): the delay at
// knot jf + jj of image ib is D[ib] + phi[ib * nk + jj].
template <int kLayout>
__device__ int adjoint_records(const KernelArgs& a, const SceneDev& S, const ItemGeom& g, float2* rec_s,
                               int4* img_s, float4* u_s, float4* um_s, float4* anc_s, float* phi_s, float* tmin,
                               float* tmax, float* d_s = nullptr, float* dfl_out = nullptr,
                               const float** phi_out = nullptr, float4* unit_xy = nullptr,
                               float2* unit_z = nullptr, bool unit_array = false) {
  if (S.delay_model == 1) {
    item_records_ret<kBwThreads, kLayout>(a, S, g, rec_s, img_s, u_s, um_s, phi_s, tmin, tmax, 1.0f, dfl_out);
    if (phi_out) *phi_out = phi_s;
    return g.cnt;
  }
  if (S.tier_up[g.t] > 1)
    return item_records_bl<kBwThreads, kLayout>(a, S, g, rec_s, img_s, reinterpret_cast<float*>(u_s),
                                                kRecScratchFloats, tmin, tmax, 1.0f, dfl_out, phi_out)
               ? g.cnt
               : 0;
  item_records<kBwThreads, kLayout>(a, S, g, rec_s, img_s, u_s, um_s, anc_s, phi_s, tmin, tmax, 1.0f, d_s, unit_xy,
                                    unit_z, unit_array);
  return g.cnt;
}

// First (mic, image, record knot) unit of tier t of scene s in the global
// option-unit tables (otau, ograd), laid out [mic][knot][image] (J_t + 1
// knots), so that consecutive images of one knot are adjacent.
__device__ __forceinline__ int64_t opt_row0(const KernelArgs& a, const SceneDev& S, int s, int t) {
  return (a.n_scenes > 1 ? a.tab.opt_prefix[s] : int64_t(0)) + S.opt_units_first[t];
}

// The gradient kernel's image loop for this thread's chunks, over image pairs
// (paired records, see put_image_record). Per image-sample: e and de/dw
// (degree-5 rows), dL/dd_i(n) = -dy g (fs/c) (S de/dw + e / tau), its knot
// weights (1 - s, s) times the unit vectors of the interval's knots, and the
// wall terms dy e (fs/c) / tau times dbeta_i/dbeta_w / (4 pi). The delay, its
// rounding, the gains and the knot weights run as float2 pairs of images.
// kChecked: the window is processed in several passes and read positions
// outside this pass contribute nothing; otherwise every position lies inside
// the window by construction (the index is only clamped to the arrays).
// dyf[c] = dy (fs/c) of the chunk's sample (0 for samples past the output).
__device__ __forceinline__ void horner_d5(const float4 A, const float2 B, float w, float* pe_out, float* pd_out) {
  float pe = B.y, pd = 0.0f;  // e = P(w) and dP/dw together (Horner, degree 5)
  pd = fmaf(pd, w, pe); pe = fmaf(pe, w, B.x);
  pd = fmaf(pd, w, pe); pe = fmaf(pe, w, A.w);
  pd = fmaf(pd, w, pe); pe = fmaf(pe, w, A.z);
  pd = fmaf(pd, w, pe); pe = fmaf(pe, w, A.y);
  pd = fmaf(pd, w, pe); pe = fmaf(pe, w, A.x);
  *pe_out = pe;
  *pd_out = pd;
}

template <bool kChecked>
__device__ __forceinline__ void grad_pairs(const float4* zq_s, const float2* zp_s, const float4* rec4,
                                           const float4* id_s, const int2* ii_s, const float4* uxy_s,
                                           const float2* uz_s, const float4* bwp_s, int cntp, int nk,
                                           const int* jc, const int* rmj, const float* rf, const float* sN,
                                           const float* dyf, unsigned pw, float2 (&V)[kBwChunks][6],
                                           float2 (&bacc)[6]) {
  constexpr unsigned kCap = unsigned(kFarrowSegs * kGradWcap - 1);
  const float4* row[kBwChunks];
  unsigned rmc[kBwChunks];
  float2 rf2[kBwChunks], sN2[kBwChunks], dy2[kBwChunks];
#pragma unroll
  for (int c = 0; c < kBwChunks; ++c) {
    row[c] = rec4 + jc[c] * cntp;
    rmc[c] = fold_rounding(rmj[c]);
    rf2[c] = make_float2(rf[c], rf[c]);
    sN2[c] = make_float2(sN[c], sN[c]);
    dy2[c] = make_float2(dyf[c], dyf[c]);
  }
  for (int p = 0; p < cntp; ++p) {
    const float4 ID = id_s[p];  // {Dp, Dp', G, G'}
    const int2 II = ii_s[p];    // {I, I'}
    const float2 G2n = make_float2(-ID.z, -ID.w);  // minus the gains
    const int ub = p * nk;
    float2 hsum = make_float2(0.0f, 0.0f);  // dy e (fs/c) / tau of the two images, over the chunks
#pragma unroll
    for (int c = 0; c < kBwChunks; ++c) {
      const float4 R = row[c][p];
      const float2 Y = __ffma2_rn(rf2[c], make_float2(R.z, R.w), make_float2(R.x, R.y));
      const float2 q = __fadd2_rn(Y, make_float2(kRound, kRound));
      const float2 t = __fadd2_rn(q, make_float2(-kRound, -kRound));
      const float2 w = __ffma2_rn(t, make_float2(-1.0f, -1.0f), Y);
      const float2 tau = __ffma2_rn(Y, make_float2(-1.0f / kFarrowSegs, -1.0f / kFarrowSegs),
                                    make_float2(ID.x, ID.y));
      const unsigned b0 = __float_as_uint(q.x), b1 = __float_as_uint(q.y);
      float2 dy = dy2[c];
      unsigned i0, i1;
      if (kChecked) {
        const int c0 = rmj[c] + II.x + (int(b0 >> 2) - (kRoundBits >> 2));
        const int c1 = rmj[c] + II.y + (int(b1 >> 2) - (kRoundBits >> 2));
        const bool in0 = unsigned(c0) < pw, in1 = unsigned(c1) < pw;
        dy = make_float2(in0 ? dy.x : 0.0f, in1 ? dy.y : 0.0f);
        i0 = in0 ? (b0 & 3u) * unsigned(kGradWcap) + unsigned(c0) : 0u;
        i1 = in1 ? (b1 & 3u) * unsigned(kGradWcap) + unsigned(c1) : 0u;
      } else {
        i0 = min((b0 & 3u) * unsigned(kGradWcap) + ((b0 >> 2) + unsigned(II.x) + rmc[c]), kCap);
        i1 = min((b1 & 3u) * unsigned(kGradWcap) + ((b1 >> 2) + unsigned(II.y) + rmc[c]), kCap);
      }
      float pe0, pd0, pe1, pd1;
      horner_d5(zq_s[i0], zp_s[i0], w.x, &pe0, &pd0);
      horner_d5(zq_s[i1], zp_s[i1], w.y, &pe1, &pd1);
      const float2 rt = make_float2(__fdividef(1.0f, tau.x), __fdividef(1.0f, tau.y));
      const float2 et = __fmul2_rn(make_float2(pe0, pe1), rt);                       // e / tau
      const float2 gd = __fmul2_rn(__fmul2_rn(dy, G2n), rt);                         // -dy g (fs/c)
      const float2 ad = __fmul2_rn(gd, __ffma2_rn(make_float2(float(kFarrowSegs), float(kFarrowSegs)),
                                                  make_float2(pd0, pd1), et));      // dL/dd_i(n)
      hsum = __ffma2_rn(dy, et, hsum);
      const float2 w1 = __fmul2_rn(ad, sN2[c]);
      const float2 w0 = __ffma2_rn(w1, make_float2(-1.0f, -1.0f), ad);
      const float4 U0 = uxy_s[ub + jc[c]], U1 = uxy_s[ub + jc[c] + 1];
      const float2 Z0 = uz_s[ub + jc[c]], Z1 = uz_s[ub + jc[c] + 1];
      V[c][0] = __ffma2_rn(w0, make_float2(U0.x, U0.y), V[c][0]);
      V[c][1] = __ffma2_rn(w0, make_float2(U0.z, U0.w), V[c][1]);
      V[c][2] = __ffma2_rn(w0, Z0, V[c][2]);
      V[c][3] = __ffma2_rn(w1, make_float2(U1.x, U1.y), V[c][3]);
      V[c][4] = __ffma2_rn(w1, make_float2(U1.z, U1.w), V[c][4]);
      V[c][5] = __ffma2_rn(w1, Z1, V[c][5]);
    }
    // the wall weights depend on the image only: once per pair
    const float4 W0 = bwp_s[3 * p], W1 = bwp_s[3 * p + 1], W2 = bwp_s[3 * p + 2];
    bacc[0] = __ffma2_rn(hsum, make_float2(W0.x, W0.y), bacc[0]);
    bacc[1] = __ffma2_rn(hsum, make_float2(W0.z, W0.w), bacc[1]);
    bacc[2] = __ffma2_rn(hsum, make_float2(W1.x, W1.y), bacc[2]);
    bacc[3] = __ffma2_rn(hsum, make_float2(W1.z, W1.w), bacc[3]);
    bacc[4] = __ffma2_rn(hsum, make_float2(W2.x, W2.y), bacc[4]);
    bacc[5] = __ffma2_rn(hsum, make_float2(W2.z, W2.w), bacc[5]);
  }
}

// ------------------------------------------------------------------ gradients
// kArray = false: the source-trajectory knot gradients, the wall terms and the
// delay ranges (and the option tiers' knot delays). kArray = true: a second
// pass over the linear tiers of the scenes asking for dL/d(array trajectory),
// with the unit vectors of the microphone, dd/dm = -Delta / d, into kslot_arr.
template <bool kArray>
__global__ void __launch_bounds__(kBwThreads, 1) k_adj_grad(const __grid_constant__ KernelArgs a) {
  extern __shared__ __align__(16) float4 sm[];
  float4* zq_s = sm;                                                    // kFarrowSegs x kGradWcap
  float2* zp_s = reinterpret_cast<float2*>(zq_s + kFarrowSegs * kGradWcap);  // powers 4..5
  float2* rec_s = zp_s + kFarrowSegs * kGradWcap;
  int4* img_s = reinterpret_cast<int4*>(rec_s + kBwRecCap);
  float4* unit_s = reinterpret_cast<float4*>(img_s + kBwBlock);        // unit vectors, paired (below)
  float4* bw_s = unit_s + kBwUnitCap;                                   // wall weights, 3 per image pair
  float4* u_s = sm;                                                     // prologue scratch
  float4* um_s = sm + kBwTile + 4;
  float4* anc_s = um_s + kBwTile + 4;
  float* phi_s = reinterpret_cast<float*>(anc_s + 3 * kBwBlock);       // kBwRecCap + kBwBlock
  float* dk_s = phi_s + kBwRecCap + kBwBlock;                           // distances at the knots, as phi_s
  float* seg_s = reinterpret_cast<float*>(sm);                          // knot scan scratch (after the loop)
  static_assert(4 * (2 * (kBwTile + 4) + 3 * kBwBlock) + 2 * (kBwRecCap + kBwBlock) <= 4 * kFarrowSegs * kGradWcap,
                "prologue scratch");
  static_assert(6 * kSegCap * (kBwTile / 32) <= 4 * kFarrowSegs * kGradWcap, "scan scratch");
  static_assert(kGradWcap % 4 == 0, "16-byte aligned row segments");
  __shared__ __align__(8) uint64_t s_mbar;  // completion of the window's bulk copies
  if (threadIdx.x == 0) mbar_init(&s_mbar, 1);
  unsigned phase = 0;
  __shared__ int s_item;
  __shared__ float s_red[2][kBwThreads / 32];
  __shared__ float s_beta[kBwThreads / 32][6];
  SceneCursor cursor = fresh_cursor();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  if (threadIdx.x == 0) s_item = int(atomicAdd(a.p.counter, 1u));
  for (;;) {
    __syncthreads();
    const int64_t item = s_item;
    if (item >= a.totals[4]) break;
    // the next item's index is requested now and published at this item's
    // end, so that the atomic's round trip overlaps the work
    unsigned next_item = 0;
    if (threadIdx.x == 0) next_item = atomicAdd(a.p.counter, 1u);
    int s = 0;
    int64_t li = item;
    if (a.n_scenes > 1) {
      s = scene_at(a.tab.item_prefix, a.n_scenes, item, cursor);
      li = item - a.tab.item_prefix[s];
    }
    const SceneDev& S = scene_of(a, s);
    ItemGeom g = item_geometry(S, li, kBwTile);
    const float fsc = S.fsc;
    // upsampled and emission-time tiers: the knot gradients come from the
    // per-(mic, image, knot) kernels; this item only adds the wall terms and
    // the delay range (zero unit vectors)
    const bool opt = opt_tier(S, g.t);
    if (kArray && (opt || !S.darray || !S.arr_moving)) {
      __syncthreads();  // s_item is read by every thread before the next item replaces it
      if (threadIdx.x == 0) s_item = int(next_item);
      continue;
    }

    float tmin, tmax;
    const float* kphi = nullptr;
    // paired layouts of the image loop: unit vectors per (pair, knot) as
    // {x, x', y, y'} and {z, z'} (written by the linear tiers' record pass;
    // zeros for the option tiers), wall weights per pair as three float4 of
    // (w, w') pairs; an odd block's zero-gain copy gets zeros
    float4* uxy_s = unit_s;
    float2* uz_s = reinterpret_cast<float2*>(uxy_s + pair_count(g.cnt) * g.nk);
    g.cnt = adjoint_records<kRecAdjoint>(a, S, g, rec_s, img_s, u_s, um_s, anc_s, phi_s, &tmin, &tmax, nullptr, dk_s,
                                         &kphi, uxy_s, uz_s, kArray);
    if (!kArray && opt && g.cnt > 0) {
      // the knot delays D + phi of the item's images, each (mic, image, knot)
      // written by exactly one item: the tile holding the knot's sample, the
      // last tile for the knot past the output
      const int nk = g.nk;
      const bool last_tile = g.n_end == S.n_out - 1;
      const int J1 = S.tier_intervals[g.t] + 1;
      const int cnt_t = S.tier_count[g.t];
      double* obase = a.p.otau + opt_row0(a, S, s, g.t) + int64_t(g.mic) * J1 * cnt_t + g.img0;
      for (int i = threadIdx.x; i < g.cnt * nk; i += kBwThreads) {
        const int jj = i / g.cnt, ib = i - jj * g.cnt;
        const int k = g.jf + jj;
        const int64_t kn = int64_t(k) * g.N;
        if ((kn >= g.n0 && kn <= g.n_end) || (last_tile && kn > g.n_end))
          obase[int64_t(k) * cnt_t + ib] = double(dk_s[ib]) + double(kphi[ib * nk + jj]);
      }
    }
    int m_lo, width;
    float rmin, rmax;
    window_of<kBwThreads>(tmin, tmax, g, s_red, &m_lo, &width, &rmin, &rmax);
    {  // window start congruent to the z rows' origin mod 4 (16-byte row segments)
      const int sh = int(((int64_t(m_lo) - S.z_m0) % 4 + 4) % 4);
      m_lo -= sh;
      width += sh;
    }
    // the item's delay range, for the dx kernel's window
    if (!kArray && threadIdx.x == 0) a.p.trange[item] = make_float2(rmin, rmax);
    // the first pass's powers 4..5 start copying now: their rows (zp_s) lie
    // above every prologue scratch array, so only powers 0..3 (zq_s) wait for
    // the scratch to be dead
    const float4* zqg = a.p.zq + S.z_base;
    const float2* zpg = a.p.zg + S.z_base;
    {
      const int64_t lo_c = max(int64_t(m_lo), S.z_m0);
      const int64_t hi_c = min(int64_t(m_lo) + min(kGradWcap, width), S.z_m0 + S.z_len);
      const int cnt_c = int(hi_c > lo_c ? hi_c - lo_c : int64_t(0));
      if (cnt_c > 0) {
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
          const unsigned bq = unsigned(cnt_c) * 16u;
          const unsigned bp = unsigned((cnt_c + 3) & ~3) * 8u;  // within the padded rows
          mbar_expect_tx(&s_mbar, unsigned(kFarrowSegs) * (bq + bp) + a.test_extra_tx);
          const int dst0 = int(lo_c - m_lo);
          const int64_t src0 = lo_c - S.z_m0;
          for (int sg = 0; sg < kFarrowSegs; ++sg)
            bulk_g2s(zp_s + sg * kGradWcap + dst0, zpg + int64_t(sg) * S.z_len + src0, bp, &s_mbar);
        }
      }
    }
    const int cntp = pair_count(g.cnt);
    if (opt) {
      for (int i = threadIdx.x; i < cntp * g.nk; i += kBwThreads) {
        uxy_s[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        uz_s[i] = make_float2(0.f, 0.f);
      }
    }
    // dbeta_i/dbeta_w / (4 pi) of the block's images (in the item's time
    // group's order), paired
    {
      const float4* bwt = a.p.bwt + 2 * (S.img_base + g.img_off + S.tier_first[g.t] + g.img0);
      for (int i = threadIdx.x; i < 2 * cntp; i += kBwThreads) {
        const int ib = 2 * (i >> 1) + (i & 1);  // image of this thread: pair i / 2, member i % 2
        float wv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (ib < g.cnt) {
          const float4 b0 = bwt[2 * ib], b1 = bwt[2 * ib + 1];
          wv[0] = b0.x; wv[1] = b0.y; wv[2] = b0.z; wv[3] = b0.w; wv[4] = b1.x; wv[5] = b1.y;
        }
        float* f = reinterpret_cast<float*>(bw_s + 3 * (ib >> 1));
        const int h = ib & 1;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          f[4 * k + h] = wv[2 * k];
          f[4 * k + 2 + h] = wv[2 * k + 1];
        }
      }
    }

    int jc[kBwChunks], rr[kBwChunks];
    float rf[kBwChunks], sN[kBwChunks], dyf[kBwChunks];
    float2 V[kBwChunks][6];
#pragma unroll
    for (int c = 0; c < kBwChunks; ++c) {
      const int n = g.n0 + 32 * (warp * kBwChunks + c) + lane;
      const bool valid = n <= g.n_end;
      const int nn = valid ? n : g.n_end;
      const int j = nn / g.N;
      rr[c] = nn - j * g.N;
      jc[c] = j - g.jf;
      rf[c] = float(rr[c]);
      sN[c] = rf[c] / float(g.N);
      dyf[c] = valid ? __ldg(S.dy + int64_t(g.mic) * S.n_out + n) * fsc : 0.0f;
#pragma unroll
      for (int k = 0; k < 6; ++k) V[c][k] = make_float2(0.0f, 0.0f);
    }
    float2 bacc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) bacc[k] = make_float2(0.0f, 0.0f);

    for (int p0 = 0; p0 < width; p0 += kGradWcap) {
      const int pass_lo = m_lo + p0;
      const int pw = min(kGradWcap, width - p0);
      // prologue scratch / previous pass done (generic proxy) before the async copies
      fence_proxy_async();
      __syncthreads();
      const int64_t lo_c = max(int64_t(pass_lo), S.z_m0);
      const int64_t hi_c = min(int64_t(pass_lo) + pw, S.z_m0 + S.z_len);
      const int cnt_c = int(hi_c > lo_c ? hi_c - lo_c : int64_t(0));
      if (cnt_c != pw && threadIdx.x == 0) atomicOr(a.p.err, kErrWindowClamp);
      const int dst0 = int(lo_c - pass_lo);  // multiples of 4 (see m_lo)
      const int64_t src0 = lo_c - S.z_m0;
      if (cnt_c > 0) {
        if (threadIdx.x == 0) {
          const unsigned bq = unsigned(cnt_c) * 16u;
          const unsigned bp = unsigned((cnt_c + 3) & ~3) * 8u;  // within the padded rows
          // the first pass's expected bytes and powers 4..5 were issued above
          if (p0 > 0) mbar_expect_tx(&s_mbar, unsigned(kFarrowSegs) * (bq + bp) + a.test_extra_tx);
          for (int sg = 0; sg < kFarrowSegs; ++sg) {
            bulk_g2s(zq_s + sg * kGradWcap + dst0, zqg + int64_t(sg) * S.z_len + src0, bq, &s_mbar);
            if (p0 > 0) bulk_g2s(zp_s + sg * kGradWcap + dst0, zpg + int64_t(sg) * S.z_len + src0, bp, &s_mbar);
          }
        }
        const bool ok = mbar_wait(&s_mbar, phase);
        if (__syncthreads_or(!ok)) {
          if (threadIdx.x == 0) atomicOr(a.p.err, kErrTimeout);
          mbar_wait(&s_mbar, phase);
          return;
        }
        phase ^= 1u;
      }
      int rmj[kBwChunks];
#pragma unroll
      for (int c = 0; c < kBwChunks; ++c) rmj[c] = rr[c] - pass_lo + jc[c] * g.N;
      const float4* rec4 = reinterpret_cast<const float4*>(rec_s);
      const float4* id_s = reinterpret_cast<const float4*>(img_s);
      const int2* ii_s = reinterpret_cast<const int2*>(id_s + cntp);
      if (width <= kGradWcap)
        grad_pairs<false>(zq_s, zp_s, rec4, id_s, ii_s, uxy_s, uz_s, bw_s, cntp, g.nk, jc, rmj, rf, sN, dyf,
                          unsigned(pw), V, bacc);
      else
        grad_pairs<true>(zq_s, zp_s, rec4, id_s, ii_s, uxy_s, uz_s, bw_s, cntp, g.nk, jc, rmj, rf, sN, dyf,
                         unsigned(pw), V, bacc);
    }
    __syncthreads();  // the z window is reused as scan scratch
    // knot slots of the item: per chunk a warp-segmented scan over the lanes'
    // intervals, segment tails stored per (chunk, interval), then per knot a
    // sum over the chunks in sample order
#pragma unroll
    for (int c = 0; c < kBwChunks; ++c) {
      float vals[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) vals[k] = V[c][k].x + V[c][k].y;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int kd = __shfl_up_sync(0xffffffffu, jc[c], d);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float t = __shfl_up_sync(0xffffffffu, vals[k], d);
          if (lane >= d && kd == jc[c]) vals[k] += t;
        }
      }
      const int jn = __shfl_down_sync(0xffffffffu, jc[c], 1);
      const int jw = __shfl_sync(0xffffffffu, jc[c], 0);
      if (lane == 31 || jn != jc[c]) {
        const int chunk = warp * kBwChunks + c;
#pragma unroll
        for (int k = 0; k < 6; ++k) seg_s[(chunk * kSegCap + (jc[c] - jw)) * 6 + k] = vals[k];
      }
    }
    __syncthreads();
    {
      float* slot = (kArray ? a.p.kslot_arr : a.p.kslot) +
                    3 * (S.kslot_first[g.t] + int64_t(g.mic) * S.kslot_mic_stride +
                         (int64_t(g.blk - S.block_first[g.t]) * S.n_tiles + (g.n0 / kBwTile)) * S.kcap[g.t]);
      constexpr int kChunksPerTile = kBwTile / 32;
      for (int jj = threadIdx.x; jj < g.nk; jj += kBwThreads) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
        // chunks holding samples of intervals jj - 1 and jj (in sample order)
        const int c_lo = max(0, ((g.jf + jj - 1) * g.N - g.n0) >> 5);
        const int c_hi = min(kChunksPerTile - 1, ((g.jf + jj + 1) * g.N - 1 - g.n0) >> 5);
        for (int ch = c_lo; ch <= c_hi; ++ch) {
          const int na = g.n0 + 32 * ch;
          if (na > g.n_end) break;
          const int first = na / g.N - g.jf;
          const int last = min(na + 31, g.n_end) / g.N - g.jf;
          if (jj >= first && jj <= last) {  // V0 of interval jj
            const float* v = seg_s + (ch * kSegCap + (jj - first)) * 6;
            sx += v[0]; sy += v[1]; sz += v[2];
          }
          if (jj - 1 >= first && jj - 1 <= last) {  // V1 of interval jj - 1
            const float* v = seg_s + (ch * kSegCap + (jj - 1 - first)) * 6;
            sx += v[3]; sy += v[4]; sz += v[5];
          }
        }
        slot[3 * jj] = sx; slot[3 * jj + 1] = sy; slot[3 * jj + 2] = sz;
      }
    }
    // wall partials of the item (fixed-order block sum)
#pragma unroll
    for (int w = 0; w < 6; ++w) {
      float v = bacc[w].x + bacc[w].y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_beta[warp][w] = v;
    }
    __syncthreads();
    if (!kArray && threadIdx.x < 6) {
      float v = 0.f;
      for (int w = 0; w < kBwThreads / 32; ++w) v += s_beta[w][threadIdx.x];
      a.p.bpart[S.bpart_base + li * 8 + threadIdx.x] = v;
    }
    __syncthreads();  // shared memory is reused by the next item
    if (threadIdx.x == 0) s_item = int(next_item);
  }
}

// The dx kernel's scatter of one block's images into the w window: per
// image-sample, dy g w^q goes to bin (segment, column); samples past the output
// (and, with kChecked, read positions outside this pass) go to a discard slot
// past the window. Within one image no two samples share a bin (the source is
// slower than c/2), so images are separated by a barrier and no atomics are
// needed.
template <bool kChecked>
__device__ __forceinline__ void dx_bins(const float2* const* row, const int4 im, const unsigned* rmc, const int* rmj,
                                        const float* rf, const float* dyv, const bool* valid, unsigned pw,
                                        unsigned* idx, float* val, float* w) {
  constexpr unsigned kDiscard = unsigned(kFarrowSegs * kDxWcap);
  const float gi = __int_as_float(im.z);
  const float Dp = __int_as_float(im.y);
#pragma unroll
  for (int c = 0; c < kBwChunks; ++c) {
    float tau;
    if (kChecked) {
      const DelaySplit ds = split_delay(row[c][0], rmj[c] + im.x, rf[c], Dp);
      idx[c] = (valid[c] && unsigned(ds.col) < pw) ? unsigned(ds.seg * kDxWcap + ds.col) : kDiscard;
      w[c] = ds.w;
      tau = ds.tau;
    } else {
      const unsigned i = split_index<kDxWcap>(row[c][0], im.x, rmc[c], rf[c], Dp, &w[c], &tau);
      idx[c] = valid[c] ? min(i, kDiscard - 1) : kDiscard;
    }
    val[c] = dyv[c] * __fdividef(gi, tau);  // dy g
  }
}

// The dx kernel's scatter of one block's images into the w window: per
// image-sample, dy g w^q goes to bin (segment, column); samples past the output
// (and, with kChecked, read positions outside this pass) go to a discard slot
// past the window. Within one image no two samples share a bin (the source is
// slower than c/2), so images are separated by a barrier and no atomics are
// needed. The bins and values of the next image are computed while this
// image's window reads are in flight (the records are read-only here).
template <bool kChecked>
__device__ __forceinline__ void dx_images(float4* wq_s, float* wp_s, const float2* rec_s, const int4* img_s, int cnt,
                                          const int* jc, const int* rmj, const float* rf, const float* dyv,
                                          const bool* valid, unsigned pw) {
  if (cnt <= 0) return;
  const float2* row[kBwChunks];
  unsigned rmc[kBwChunks];
#pragma unroll
  for (int c = 0; c < kBwChunks; ++c) {
    row[c] = rec_s + jc[c] * cnt;
    rmc[c] = fold_rounding(rmj[c]);
  }
  unsigned idx[kBwChunks];
  float val[kBwChunks], w[kBwChunks];
  dx_bins<kChecked>(row, img_s[0], rmc, rmj, rf, dyv, valid, pw, idx, val, w);
  for (int ib = 0; ib < cnt; ++ib) {
    float4 wa[kBwChunks];
    float wb[kBwChunks];
#pragma unroll
    for (int c = 0; c < kBwChunks; ++c) {
      wa[c] = wq_s[idx[c]];
      wb[c] = wp_s[idx[c]];
    }
    // the last image recomputes its own bins (unused)
    const int nb = min(ib + 1, cnt - 1);
    unsigned nidx[kBwChunks];
    float nval[kBwChunks], nw[kBwChunks];
    const float2* nrow[kBwChunks];
#pragma unroll
    for (int c = 0; c < kBwChunks; ++c) nrow[c] = row[c] + nb;
    dx_bins<kChecked>(nrow, img_s[nb], rmc, rmj, rf, dyv, valid, pw, nidx, nval, nw);
#pragma unroll
    for (int c = 0; c < kBwChunks; ++c) {
      const float p1 = val[c] * w[c], p2 = p1 * w[c], p3 = p2 * w[c], p4 = p3 * w[c];
      wa[c].x += val[c]; wa[c].y += p1; wa[c].z += p2; wa[c].w += p3;
      wb[c] += p4;
    }
    // both chunks of a thread lie in different bins, or both in the discard slot
#pragma unroll
    for (int c = 0; c < kBwChunks; ++c) {
      wq_s[idx[c]] = wa[c];
      wp_s[idx[c]] = wb[c];
    }
    __syncthreads();  // the next image may write the same bins
#pragma unroll
    for (int c = 0; c < kBwChunks; ++c) {
      idx[c] = nidx[c];
      val[c] = nval[c];
      w[c] = nw[c];
    }
  }
}

// ------------------------------------------------------------------ dx
template <int kL>
__global__ void __launch_bounds__(kBwThreads, 1) k_adj_dx(const __grid_constant__ KernelArgs a) {
  extern __shared__ __align__(16) float4 sm[];
  float4* wq_s = sm;                                                       // kFarrowSegs x kDxWcap (powers 0..3)
  float* wp_s = reinterpret_cast<float*>(wq_s + kDxSlots);                 // power 4
  float2* rec_s = reinterpret_cast<float2*>(wp_s + kDxSlots);
  int4* img_s = reinterpret_cast<int4*>(rec_s + kBwRecCap);
  float4* u_s = reinterpret_cast<float4*>(img_s + kBwBlock);              // record scratch
  float4* um_s = u_s + kBwTile + 4;
  float4* anc_s = um_s + kBwTile + 4;                                      // 3 x kBwBlock
  float* phi_s = reinterpret_cast<float*>(anc_s + 3 * kBwBlock);          // kBwRecCap + kBwBlock
  __shared__ int s_item;
  __shared__ float s_red[2][kBwThreads / 32];
  SceneCursor cursor = fresh_cursor();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a gradient kernel that gave up on a wait left some delay ranges unwritten:
  // windows sized from them could be arbitrary, so nothing is scattered (the
  // call reports the timeout; the error word is cleared at the start of a call)
  if (*reinterpret_cast<volatile const uint32_t*>(a.p.err) & kErrTimeout) return;

  for (;;) {
    const int64_t item = next_item(a, &s_item);
    if (item >= a.totals[5]) break;
    int s = 0;
    int64_t li = item;
    if (a.n_scenes > 1) {
      s = scene_at(a.tab.red_prefix, a.n_scenes, item, cursor);
      li = item - a.tab.red_prefix[s];
    }
    const SceneDev& S = scene_of(a, s);
    const int range = int(li % S.n_ranges);
    const int64_t mg = li / S.n_ranges;
    const int mic = int(mg / S.n_groups);
    const int grp = int(mg - int64_t(mic) * S.n_groups);
    int t = 0;
    while (t + 1 < S.n_tiers && grp >= S.group_first[t + 1]) ++t;
    const int b0 = S.block_first[t] + (grp - S.group_first[t]) * S.group_blocks[t];
    const int b1 = min(b0 + S.group_blocks[t], S.block_first[t] + S.tier_blocks[t]);
    const int64_t item0 = int64_t(mic) * S.n_blocks;
    // rows are zeroed before the launch; ranges of one parity write disjoint columns
    float* dxrow = a.p.dxb + S.dxb_base + (mg * S.dx_rows + range % S.dx_rows) * S.n_in;
    const int tile_end = min(S.n_tiles, (range + 1) * S.range_tiles);

    // the gradient kernel stored every (mic, block, tile) item's delay range
    const float2* trange = a.p.trange + (a.n_scenes > 1 ? a.tab.item_prefix[s] : int64_t(0));
    for (int tile = range * S.range_tiles; tile < tile_end; ++tile) {
      // the group's delay range over the tile: union of its blocks' ranges
      float tmin = 3.0e38f, tmax = -3.0e38f;
      for (int b = b0; b < b1; ++b) {
        const float2 r = trange[(item0 + b) * S.n_tiles + tile];
        tmin = fminf(tmin, r.x);
        tmax = fmaxf(tmax, r.y);
      }
      const ItemGeom g0 = item_geometry(S, (item0 + b0) * S.n_tiles + tile, kBwTile);
      int m_lo, width;
      window_of<kBwThreads>(tmin, tmax, g0, s_red, &m_lo, &width);
      // every block of the group has the tier's knot spacing and the same tile
      int jc[kBwChunks], rr[kBwChunks];
      float rf[kBwChunks], dyv[kBwChunks];
      bool valid[kBwChunks];
#pragma unroll
      for (int c = 0; c < kBwChunks; ++c) {
        const int n = g0.n0 + 32 * (warp * kBwChunks + c) + lane;
        valid[c] = n <= g0.n_end;
        const int nn = valid[c] ? n : g0.n_end;
        const int j = nn / g0.N;
        rr[c] = nn - j * g0.N;
        jc[c] = j - g0.jf;
        rf[c] = float(rr[c]);
        dyv[c] = valid[c] ? __ldg(S.dy + int64_t(mic) * S.n_out + n) : 0.0f;
      }
      const bool single = (b1 - b0 == 1);  // a single block keeps its records over the passes
      int cnt_b = 0;                        // images of the block whose records are built
      for (int p0 = 0; p0 < width; p0 += kDxWcap) {
        const int pass_lo = m_lo + p0;
        const int pw = min(kDxWcap, width - p0);
        __syncthreads();  // the previous pass's correlation is done with the window
        for (int i = threadIdx.x; i < kFarrowSegs * kDxWcap; i += kBwThreads) {
          wq_s[i] = make_float4(0.f, 0.f, 0.f, 0.f);
          wp_s[i] = 0.f;
        }
        int rmj[kBwChunks];
#pragma unroll
        for (int c = 0; c < kBwChunks; ++c) rmj[c] = rr[c] - pass_lo + jc[c] * g0.N;
        for (int b = b0; b < b1; ++b) {
          const ItemGeom g = item_geometry(S, (item0 + b) * S.n_tiles + tile, kBwTile);
          if (!single || p0 == 0) {
            float lo, hi;
            __syncthreads();  // the previous block's records are no longer read
            cnt_b = adjoint_records<kRecPlain>(a, S, g, rec_s, img_s, u_s, um_s, anc_s, phi_s, &lo, &hi);
          }
          __syncthreads();  // records and the zeroed window are complete
          if (width <= kDxWcap)
            dx_images<false>(wq_s, wp_s, rec_s, img_s, cnt_b, jc, rmj, rf, dyv, valid, unsigned(pw));
          else
            dx_images<true>(wq_s, wp_s, rec_s, img_s, cnt_b, jc, rmj, rf, dyv, valid, unsigned(pw));
        }
        // dx[m'] += sum_{row, k} c[row][k] w[row][m' + k] for the outputs m' =
        // pass_lo - kL/2 + 1 + q, q in [0, pw + kL - 1); output q reads window
        // columns q + 1 - kL + k. A thread takes the 4 outputs q = 32 g + l + 8 o
        // (g = i / 8, l = i % 8, o = 0..3), so the 8 lanes of a quarter warp read
        // 8 consecutive columns (no bank conflicts) and every column a thread
        // reads serves up to 4 of its outputs.
        const int n_outv = pw + kL - 1;
        for (int i = threadIdx.x; 32 * (i >> 3) + (i & 7) < n_outv; i += kBwThreads) {
          const int q0 = 32 * (i >> 3) + (i & 7);
          float acc4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int tt = 0; tt < kL + 24; ++tt) {
            // column q0 + 1 - kL + tt feeds output q0 + 8 o through tap kk = tt - 8 o
            const int cc = q0 + 1 - kL + tt;
            if (cc < 0 || cc >= pw) continue;
            float wv[kZRows];
#pragma unroll
            for (int sg = 0; sg < kFarrowSegs; ++sg) {
              const float4 w4 = wq_s[sg * kDxWcap + cc];
              float* o = wv + sg * kFarrowCoef;
              o[0] = w4.x; o[1] = w4.y; o[2] = w4.z; o[3] = w4.w; o[4] = wp_s[sg * kDxWcap + cc];
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) {
              const int kk = tt - 8 * o;
              if (kk < 0 || kk >= kL) continue;
#pragma unroll
              for (int row = 0; row < kZRows; ++row)
                acc4[o] = fmaf(a.farrow[row / kFarrowCoef][row % kFarrowCoef][kk], wv[row], acc4[o]);
            }
          }
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            const int q = q0 + 8 * o;
            const int mp = pass_lo - kL / 2 + 1 + q;
            if (q < n_outv && mp >= 0 && mp < S.n_in) dxrow[mp] += acc4[o];
          }
        }
      }
      __syncthreads();  // the correlation is done before the next tile's records
    }
    __syncthreads();
  }
}

// dx[m] = sum over microphones and block groups of the dx rows (fixed order).
__global__ void k_dx_final(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[2]) return;
  int s = 0;
  int64_t m = gid;
  if (a.n_scenes > 1) {
    s = find_scene(a.tab.dx_prefix, a.n_scenes, gid);
    m = gid - a.tab.dx_prefix[s];
  }
  const SceneDev& S = scene_of(a, s);
  if (!S.dx) return;
  const float* p = a.p.dxb + S.dxb_base + m;
  const int rows = S.n_mics * S.n_groups * S.dx_rows;
  float acc = 0.f;
  for (int rr = 0; rr < rows; ++rr) acc += p[int64_t(rr) * S.n_in];
  S.dx[m] = acc;
}

// dL/ds(t_j) per tier knot: sum over microphones, blocks of the tier and the
// (at most two) tiles whose knot range holds j.
// 32 knots per CTA x 8 lanes per knot: lane q sums blocks q, q + 8, ... (in
// order), the 8 lane sums are added in lane order (bitwise reproducible).
constexpr int kKnotsPerCta = 32;
constexpr int kKnotLanes = 8;
// kArray: the array pass's slots into dL/da(t_j) (garr).
template <bool kArray>
__global__ void __launch_bounds__(kKnotsPerCta * kKnotLanes) k_knot_final(const __grid_constant__ KernelArgs a) {
  __shared__ double part[kKnotLanes][kKnotsPerCta][3];
  const int kq = threadIdx.x % kKnotsPerCta, q = threadIdx.x / kKnotsPerCta;
  const int64_t gid = int64_t(blockIdx.x) * kKnotsPerCta + kq;
  double gx = 0.0, gy = 0.0, gz = 0.0;
  int s = 0, t = 0, j = 0;
  const bool live = gid < a.totals[1];
  if (live) {
    int64_t local = gid;
    if (a.n_scenes > 1) {
      s = find_scene(a.tab.knots_prefix, a.n_scenes, gid);
      local = gid - a.tab.knots_prefix[s];
    }
    const SceneDev& S = scene_of(a, s);
    while (t + 1 < S.n_tiers && local >= S.knot_units_first[t + 1]) ++t;
    j = int(local - S.knot_units_first[t]);
    const int N = S.tier_step[t];
    // upsampled and emission-time tiers: zero here (k_opt_bl_knots writes the
    // upsampled tiers' knots; emission-time gradients go to the parameters
    // directly)
    if (S.tier_count[t] > 0 && !opt_tier(S, t) && (!kArray || S.darray)) {
      // samples weighting knot j: intervals j - 1 and j, n in [(j-1) N, (j+1) N)
      const int64_t s_lo = max(int64_t(j - 1) * N, int64_t(0));
      const int64_t s_hi = min(int64_t(j + 1) * N - 1, S.n_out - 1);
      const int tile_lo = int(s_lo / S.tile), tile_hi = int(s_hi / S.tile);
      for (int mic = 0; mic < S.n_mics; ++mic)
        for (int b = q; b < S.tier_blocks[t]; b += kKnotLanes)
          for (int tile = tile_lo; tile <= tile_hi; ++tile) {
            const int n0 = tile * S.tile;
            const int n_end = int(min(int64_t(n0 + S.tile), S.n_out)) - 1;
            const int jf = n0 / N, nk = n_end / N - jf + 2;
            if (j < jf || j >= jf + nk) continue;
            const float* slot = (kArray ? a.p.kslot_arr : a.p.kslot) +
                                3 * (S.kslot_first[t] + int64_t(mic) * S.kslot_mic_stride +
                                     (int64_t(b) * S.n_tiles + tile) * S.kcap[t] + (j - jf));
            gx += slot[0];
            gy += slot[1];
            gz += slot[2];
          }
    }
  }
  part[q][kq][0] = gx;
  part[q][kq][1] = gy;
  part[q][kq][2] = gz;
  __syncthreads();
  if (q == 0 && live) {
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int r = 0; r < kKnotLanes; ++r) {
      sx += part[r][kq][0];
      sy += part[r][kq][1];
      sz += part[r][kq][2];
    }
    const SceneDev& S = scene_of(a, s);
    double* out = (kArray ? a.p.garr : a.p.gk) + 3 * (S.knot_base[t] + j);
    out[0] = sx;
    out[1] = sy;
    out[2] = sz;
  }
}

constexpr int kParamThreads = 256;
constexpr int kParamChunks = 128;  // CTAs per scene of the parameter reduction
static_assert(kParamChunks * 48 == kParamPartialsPerScene, "parameter partials per scene");

// J(t)^T g for the trajectory parameters, J = ds(t)/dparams (3 x 48): its
// non-zero terms form one block of consecutive parameters, v[i] for parameter
// p0 + i (returned p0; jacobian_count terms: line 7, circle 6, spline 12, the
// four control points of t's span). In the scalar T: FP64 for the knots, FP32
// for the emission-time units (images x knots of them).
__device__ __forceinline__ void sin_cos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void sin_cos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ int jacobian_count(int kind) { return kind == 0 ? 7 : (kind == 1 ? 6 : 12); }
__device__ __forceinline__ int jacobian_count(const SceneDev& S) { return jacobian_count(S.traj_kind); }

template <class T>
__device__ int jacobian_terms(int kind, const double* q, int n_ctrl, double duration, T t, const T g[3],
                              T v[12]) {
  if (kind == 0) {  // s = p0 + v t u, u = dir / |dir|
    const T nrm = sqrt(T(q[3]) * T(q[3]) + T(q[4]) * T(q[4]) + T(q[5]) * T(q[5]));
    const T u[3] = {T(q[3]) / nrm, T(q[4]) / nrm, T(q[5]) / nrm};
    const T ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
    const T f = T(q[6]) * t / nrm;
    for (int d = 0; d < 3; ++d) {
      v[d] = g[d];
      v[3 + d] = f * (g[d] - u[d] * ug);
    }
    v[6] = t * ug;
    return 0;
  }
  if (kind == 1) {  // s = c + R (cos th, sin th, 0), th = th0 + v t / R
    const T R = T(q[3]), vel = T(q[4]);
    T sn, cs;
    sin_cos(T(q[5]) + vel * t / R, &sn, &cs);
    const T w = vel * t / R;
    for (int d = 0; d < 3; ++d) v[d] = g[d];
    v[3] = (cs + sn * w) * g[0] + (sn - cs * w) * g[1];
    v[4] = t * (cs * g[1] - sn * g[0]);
    v[5] = R * (cs * g[1] - sn * g[0]);
    return 0;
  }
  // clamped uniform cubic B-spline: s = sum_c N_c(u) P_c
  const int m = n_ctrl - 3;
  const T u = fmin(T(1), fmax(T(0), t / T(duration)));
  const int span = min(int(u * T(m)), m - 1);
  auto knot = [m](int i) { return fmin(T(1), fmax(T(0), T(i - 3) / T(m))); };
  // the four non-zero basis functions on the span (triangular scheme)
  const int K = span + 3;
  T Nb[4], left[4], right[4];
  Nb[0] = T(1);
  for (int jdeg = 1; jdeg <= 3; ++jdeg) {
    left[jdeg] = u - knot(K + 1 - jdeg);
    right[jdeg] = knot(K + jdeg) - u;
    T saved = T(0);
    for (int rr = 0; rr < jdeg; ++rr) {
      const T den = right[rr + 1] + left[jdeg - rr];
      const T tmp = den != T(0) ? Nb[rr] / den : T(0);
      Nb[rr] = saved + right[rr + 1] * tmp;
      saved = left[jdeg - rr] * tmp;
    }
    Nb[jdeg] = saved;
  }
  for (int r = 0; r < 4; ++r)
    for (int d = 0; d < 3; ++d) v[3 * r + d] = Nb[r] * g[d];
  return 3 * span;
}

// The source trajectory's terms.
template <class T>
__device__ __forceinline__ int jacobian_terms(const SceneDev& S, T t, const T g[3], T v[12]) {
  return jacobian_terms<T>(S.traj_kind, S.traj, S.n_ctrl, S.duration, t, g, v);
}

// Adds J(t)^T g to the thread's FP64 parameter column:
// row[p * kParamThreads] += sum_d J[d][p] g[d].
__device__ void add_source_jacobian(const SceneDev& S, double t, const double g[3], double* row) {
  double v[12];
  const int p0 = jacobian_terms<double>(S, t, g, v);
  const int nt = jacobian_count(S);
  for (int i = 0; i < nt; ++i) row[(p0 + i) * kParamThreads] += v[i];
}

// FP32 sums of J(t)^T g over consecutive emission-time units of one trajectory
// (the source's or the array's), added to the FP64 column when the block of
// parameters changes (another spline span), every kJacRun units and at the end.
constexpr int kJacRun = 64;
struct JacAcc {
  int kind, n_ctrl;
  const double* q;
  double duration;
  float v[12];
  int p0 = -1, n = 0;
  __device__ JacAcc(int k, const double* params, int nc, double dur) : kind(k), n_ctrl(nc), q(params), duration(dur) {}
  __device__ void flush(double* row) {
    if (p0 >= 0) {
      const int nt = jacobian_count(kind);
      for (int i = 0; i < nt; ++i) row[(p0 + i) * kParamThreads] += double(v[i]);
    }
    p0 = -1;
    n = 0;
  }
  __device__ void add(float t, const float g[3], double* row) {
    float w[12];
    const int q0 = jacobian_terms<float>(kind, q, n_ctrl, duration, t, g, w);
    if (q0 != p0 || n == kJacRun) {
      flush(row);
      p0 = q0;
#pragma unroll
      for (int i = 0; i < 12; ++i) v[i] = 0.0f;
    }
    ++n;
#pragma unroll
    for (int i = 0; i < 12; ++i) v[i] += w[i];
  }
};

// Unit (mic, image, record knot) of the upsampled / emission-time tiers of a
// scene: tier, microphone, image (sorted position in the tier), knot; units
// are numbered [tier][mic][knot][image].
struct OptUnit {
  int t, mic, img, k;
};
__device__ __forceinline__ OptUnit opt_unit(const SceneDev& S, int64_t local) {
  int t = 0;
  for (int q = 0; q < S.n_tiers; ++q)
    if (opt_tier(S, q) && S.opt_units_first[q] <= local) t = q;
  const int64_t r = local - S.opt_units_first[t];
  const int cnt = S.tier_count[t];
  const int64_t per_mic = (int64_t(S.tier_intervals[t]) + 1) * cnt;
  OptUnit u;
  u.t = t;
  if (r < (int64_t(1) << 31) && per_mic < (int64_t(1) << 31)) {  // 32-bit divisions
    const unsigned r32 = unsigned(r), pm = unsigned(per_mic);
    u.mic = int(r32 / pm);
    const unsigned rem = r32 - unsigned(u.mic) * pm;
    u.k = int(rem / unsigned(cnt));
    u.img = int(rem - unsigned(u.k) * unsigned(cnt));
    return u;
  }
  u.mic = int(r / per_mic);
  const int64_t rem = r - u.mic * per_mic;
  u.k = int(rem / cnt);
  u.img = int(rem - int64_t(u.k) * cnt);
  return u;
}

// Partial dL/dparams of one chunk of a scene's units (flattened): every thread
// sums J^T g over its units (a contiguous range of knots; every stride-th
// emission-time unit) into its own shared column, then the columns are summed
// in thread order. Units: the knots of every tier,
// J(t_j)^T dL/ds(t_j) (t_j = (j - knot_shift) times the knot spacing); with
// emission-time delays instead the (mic, image, knot) units: with
// e = t_j - tau the emission time, u = Delta / d and sigma o u = dd/ds,
//   dd/dparams = (sigma o u)^T J(e) / (1 + (sigma o u) . s'(e) / c)
// (implicit differentiation of c tau = |sigma o s(t_j - tau) + 2 n L - m(t_j)|),
// times dL/dd at the knot; s(e) and s'(e) from the source path table (linear
// between its points), in FP32 after one FP64 difference for the emission time
// (the unit vector to ~1e-6, the table fraction to ~1e-2 of a table step).
__global__ void __launch_bounds__(kParamThreads) k_param_partial(const __grid_constant__ KernelArgs a) {
  const int s = blockIdx.x / kParamChunks, chunk = blockIdx.x % kParamChunks;
  const SceneDev& S = scene_of(a, s);
  extern __shared__ double rows[];  // [48][kParamThreads]
  for (int p = 0; p < 48; ++p) rows[p * kParamThreads + threadIdx.x] = 0.0;
  const int last = S.n_tiers - 1;
  const bool ret = S.delay_model == 1;
  const int64_t total = ret ? S.n_opt_units
                            : S.knot_units_first[last] +
                                  (S.tier_up[last] > 1 ? int64_t(S.bl_knots[last]) : int64_t(S.tier_intervals[last]) + 1);
  const int64_t per_cta = (total + kParamChunks - 1) / kParamChunks;
  const int64_t per_thr = (per_cta + kParamThreads - 1) / kParamThreads;
  const int64_t lo = min(total, chunk * per_cta + threadIdx.x * per_thr);
  const int64_t hi = min(min(total, (chunk + 1) * per_cta), lo + per_thr);
  if (S.dparams && !ret) {
    int t = 0;
    for (int64_t k = lo; k < hi; ++k) {
      while (t + 1 < S.n_tiers && k >= S.knot_units_first[t + 1]) ++t;
      if (S.tier_count[t] == 0) continue;
      const int64_t j = k - S.knot_units_first[t];
      const double* gk = a.p.gk + 3 * (S.knot_base[t] + j);
      const double g[3] = {gk[0], gk[1], gk[2]};
      add_source_jacobian(S, double((j - S.knot_shift[t]) * S.tier_coarse[t]) / S.fs, g, rows + threadIdx.x);
    }
  } else if (S.dparams) {
    // emission-time units: thread q of the scene's kParamChunks x kParamThreads
    // takes units q, q + stride, ... (adjacent lanes, adjacent units: coalesced
    // loads; a thread's successive units lie a few knots apart, so a spline
    // span changes rarely along them)
    const int64_t base = a.n_scenes > 1 ? a.tab.opt_prefix[s] : int64_t(0);
    const float4* HI = a.p.dense_hi + S.dense_base;
    const float4* LO = a.p.dense_lo + S.dense_base;
    const float xs = float(kDenseOver) * float(S.fs);  // path table points per second
    const float rc = float(1.0 / S.c);
    const float rfs = float(1.0 / S.fs);
    const float k0 = float(S.dense_k0);
    const int64_t kmax = S.n_dense - 2;
    JacAcc acc(S.traj_kind, S.traj, S.n_ctrl, S.duration);
    const int64_t stride = int64_t(kParamChunks) * kParamThreads;
    for (int64_t k = int64_t(chunk) * kParamThreads + threadIdx.x; k < total; k += stride) {
      const OptUnit u = opt_unit(S, k);
      const int cnt = S.tier_count[u.t];
      const float gr = a.p.ograd[base + k].x + (u.k > 0 ? a.p.ograd[base + k - cnt].y : 0.0f);
      if (gr == 0.0f) continue;
      // emission time e = (n_j - tau) / fs (samples: n_j - tau, one FP64 difference)
      const float es = float(double(int64_t(u.k) * S.tier_step[u.t]) - a.p.otau[base + k]);
      const float x = fmaf(float(kDenseOver), es, -k0);  // path table coordinate
      const float xi = floorf(x);
      const int64_t i = min(max(int64_t(xi), int64_t(0)), kmax);
      const float f = x - float(i);
      const float4 h0 = HI[i], h1 = HI[i + 1], l0 = LO[i], l1 = LO[i + 1];
      const float ds[3] = {(h1.x - h0.x) + (l1.x - l0.x), (h1.y - h0.y) + (l1.y - l0.y),
                           (h1.z - h0.z) + (l1.z - l0.z)};
      const float sp[3] = {fmaf(f, ds[0], h0.x + l0.x), fmaf(f, ds[1], h0.y + l0.y), fmaf(f, ds[2], h0.z + l0.z)};
      const double* ap = a.p.arr_pos + 3 * (S.knot_base[u.t] + u.k);
      int n[3], p[3];
      unpack_image(a.p.img_code[S.img_base + S.tier_first[u.t] + u.img], n, p);
      float su[3], D[3];
      for (int d = 0; d < 3; ++d) {
        su[d] = p[d] ? -1.0f : 1.0f;
        const float m = float(S.mics[u.mic][d]) + (S.arr_moving ? float(ap[d]) : 0.0f);
        D[d] = fmaf(su[d], sp[d], fmaf(float(2 * n[d]), float(S.dims[d]), -m));
      }
      const float rd = rsqrtf(fmaf(D[0], D[0], fmaf(D[1], D[1], D[2] * D[2])));
      for (int d = 0; d < 3; ++d) su[d] *= D[d] * rd;  // sigma o u
      const float vs = xs * (su[0] * ds[0] + su[1] * ds[1] + su[2] * ds[2]);  // (sigma o u) . s'(e)
      const float fac = gr / fmaf(vs, rc, 1.0f);
      const float g[3] = {fac * su[0], fac * su[1], fac * su[2]};
      acc.add(es * rfs, g, rows + threadIdx.x);
    }
    acc.flush(rows + threadIdx.x);
  }
  __syncthreads();
  if (threadIdx.x < 48) {
    double acc = 0.0;
    for (int r = 0; r < kParamThreads; ++r) acc += rows[threadIdx.x * kParamThreads + r];
    a.p.ppart[(int64_t(s) * kParamChunks + chunk) * 48 + threadIdx.x] = acc;
  }
}

// ------------------------------------------------- upsampled / emission-time tiers
// Their delays are not linear in the knot positions, so their knot gradients
// are formed per (mic, image, record knot) unit. The gradient kernel stores
// the FP32 knot delays of its records (otau); k_opt_grad sums dL/dd_i(n) over
// every knot interval with the two knots' linear weights (ograd); the chain
// rule then runs through the upsampler's weights to the knots and the unit
// vectors there (k_opt_bl_rows, k_opt_bl_knots), or, for emission-time delays,
// through the implicit emission time to the trajectory parameters
// (k_param_partial).

// Unit (row, interval j) of the option tiers: per sample n = j N + r of the
// interval, dL/dd_i(n) = -dy g (fs/c) (S de/dw + e / tau) with e and de/dw from
// the degree-5 rows in global memory and the delay linear between the knot
// delays; stored: A = sum (1 - r/N) dL/dd_i(n) (to knot j) and
// B = sum (r/N) dL/dd_i(n) (to knot j + 1). The read position is formed
// relative to D = floor(tau_j) in FP32. Unit j = J (no interval) stores zeros.
__global__ void __launch_bounds__(256) k_opt_grad(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[9]) return;
  int s = 0;
  int64_t local = gid;
  if (a.n_scenes > 1) {
    s = find_scene(a.tab.opt_prefix, a.n_scenes, gid);
    local = gid - a.tab.opt_prefix[s];
  }
  const SceneDev& S = scene_of(a, s);
  const OptUnit u = opt_unit(S, local);
  const int N = S.tier_step[u.t];
  const int j = u.k;
  const int64_t n0 = int64_t(j) * N;
  float A = 0.0f, B = 0.0f;
  if (j < S.tier_intervals[u.t] && n0 < S.n_out) {
    const double t0 = a.p.otau[gid], t1 = a.p.otau[gid + S.tier_count[u.t]];  // knots j and j + 1
    const double D = floor(t0);
    const float phi0 = float(t0 - D), dphi = float(t1 - t0);
    const float Df = float(D);
    const int64_t base = n0 - int64_t(D) - S.z_m0;  // z column of read position n - D at r = 0
    const float G = a.p.img_gain[S.img_base + S.tier_first[u.t] + u.img];
    const float* dy = S.dy + int64_t(u.mic) * S.n_out + n0;
    const float4* zq = a.p.zq + S.z_base;
    const float2* zg = a.p.zg + S.z_base;
    const float invN = 1.0f / float(N);
    const int nr = int(min(int64_t(N), S.n_out - n0));
    for (int r = 0; r < nr; ++r) {
      const float sr = float(r) * invN;
      const float phi = fmaf(dphi, sr, phi0);
      const float pr = float(r) - phi;  // read position n - tau relative to n0 - D
      const float fl = floorf(pr);
      const float v = float(kFarrowSegs) * (pr - fl);
      const int seg = min(int(v), kFarrowSegs - 1);
      const float w = v - float(seg) - 0.5f;
      const int64_t col = base + int64_t(fl);
      if (col < 0 || col >= S.z_len) continue;  // x is zero there
      float pe, pd;
      horner_d5(zq[int64_t(seg) * S.z_len + col], zg[int64_t(seg) * S.z_len + col], w, &pe, &pd);
      const float tau = Df + phi;
      const float rt = 1.0f / tau;
      const float ad = -dy[r] * S.fsc * G * rt * fmaf(float(kFarrowSegs), pd, pe * rt);
      A = fmaf(1.0f - sr, ad, A);
      B = fmaf(sr, ad, B);
    }
  }
  a.p.ograd[gid] = make_float2(A, B);
}

// dL/dd at every knot of an upsampled tier's table, per (mic, image) row: the
// record knots' dL/dd (A_k + B_{k-1}) through the chord form's derivatives,
// w_p[i] off the chord's two knots, M_p - sum' w_p[i] c_i for knot j0 + 1 and
// 1 - M_p - sum' w_p[i] (1 - c_i) for knot j0 (c_i = i - Q + 1; sum' over i
// other than the chord's knots). One thread per row walks its record knots in
// order with 2Q running knot sums; stored knot-major (cgrad[knot][row]).
__global__ void k_opt_bl_rows(const __grid_constant__ KernelArgs a) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= a.totals[6]) return;
  int s = 0;
  int64_t local = gid;
  if (a.n_scenes > 1) {
    s = find_scene(a.tab.bl_prefix, a.n_scenes, gid);
    local = gid - a.tab.bl_prefix[s];
  }
  const SceneDev& S = scene_of(a, s);
  int t = -1;
  for (int q = 0; q < S.n_tiers; ++q)
    if (S.tier_up[q] > 1 && S.bl_units_first[q] <= local) t = q;
  if (t < 0) return;
  const int64_t row = local - S.bl_units_first[t];
  const int64_t rows = int64_t(S.n_mics) * S.tier_count[t];
  const int U = S.tier_up[t], Q = S.up_q, nkt = S.bl_knots[t];
  const int J1 = S.tier_intervals[t] + 1;
  const int cnt = S.tier_count[t];
  const int mic = int(row / cnt);
  // record knot k of this (mic, image) at gr[k * cnt]
  const float2* gr = a.p.ograd + opt_row0(a, S, s, t) + int64_t(mic) * J1 * cnt + (row - int64_t(mic) * cnt);
  float* cg = a.p.cgrad + S.bl_tau_base[t] + row;  // knot jt at cg[jt * rows]
  constexpr int kW = 2 * kMaxUpHalfwidth;
  float acc[kW];
#pragma unroll
  for (int i = 0; i < kW; ++i) acc[i] = 0.0f;
  cg[0] = 0.0f;  // knot -Q: no record knot reaches it
  int j0 = 0;    // acc[i] holds knot j0 - Q + 1 + i (table index j0 + 1 + i)
  float prevB = 0.0f;
  for (int k = 0; k < J1; ++k) {
    const int jk = k / U;
    for (; j0 < jk; ++j0) {  // knot j0 - Q + 1 is complete
      cg[int64_t(j0 + 1) * rows] = acc[0];
#pragma unroll
      for (int i = 0; i + 1 < kW; ++i) acc[i] = acc[i + 1];
      acc[kW - 1] = 0.0f;
    }
    const float2 ab = gr[int64_t(k) * cnt];
    const float g = ab.x + prevB;
    prevB = ab.y;
    const float* W = a.p.upw + S.upw_base[t] + (k - j0 * U) * (2 * Q + 1);
    float s0 = 0.0f, s1 = 0.0f;
    for (int i = 0; i < 2 * Q; ++i)
      if (i != Q - 1 && i != Q) {
        const float wi = __ldg(W + i);
        s0 += wi;
        s1 = fmaf(wi, float(i - Q + 1), s1);
      }
    const float M = __ldg(W + 2 * Q);
#pragma unroll
    for (int i = 0; i < kW; ++i) {
      if (i < 2 * Q) {
        const float wi = (i == Q) ? M - s1 : (i == Q - 1) ? 1.0f - M - s0 + s1 : __ldg(W + i);
        acc[i] = fmaf(wi, g, acc[i]);
      }
    }
  }
  // the last 2Q knots reached, then zeros to the end of the table
#pragma unroll
  for (int i = 0; i < kW; ++i)
    if (i < 2 * Q && j0 + 1 + i < nkt) cg[int64_t(j0 + 1 + i) * rows] = acc[i];
  for (int jt = j0 + 1 + 2 * Q; jt < nkt; ++jt) cg[int64_t(jt) * rows] = 0.0f;
}

// dL/ds(t_j) at knot j of an upsampled tier (one CTA per knot of the tier's
// table): sum over (mic, image) of dL/dd there times sigma o Delta / d, in a
// fixed order; with a moving array whose gradient is asked for, also
// dL/da(t_j): the same sum with -Delta / d.
constexpr int kBlThreads = 256;
__global__ void __launch_bounds__(kBlThreads) k_opt_bl_knots(const __grid_constant__ KernelArgs a) {
  __shared__ double part[6][kBlThreads];
  const int64_t gid = blockIdx.x;
  if (gid >= a.totals[1]) return;
  int s = 0;
  int64_t local = gid;
  if (a.n_scenes > 1) {
    s = find_scene(a.tab.knots_prefix, a.n_scenes, gid);
    local = gid - a.tab.knots_prefix[s];
  }
  const SceneDev& S = scene_of(a, s);
  int t = 0;
  while (t + 1 < S.n_tiers && local >= S.knot_units_first[t + 1]) ++t;
  if (S.tier_up[t] <= 1 || S.delay_model == 1) return;
  const int jt = int(local - S.knot_units_first[t]);
  const int64_t rows = int64_t(S.n_mics) * S.tier_count[t];
  const float* cg = a.p.cgrad + S.bl_tau_base[t] + int64_t(jt) * rows;
  const double* sp = a.p.knot_pos + 3 * (S.knot_base[t] + jt);
  const double* ap = a.p.arr_pos + 3 * (S.knot_base[t] + jt);
  double gx = 0.0, gy = 0.0, gz = 0.0, hx = 0.0, hy = 0.0, hz = 0.0;
  const bool arr = S.darray && S.arr_moving;
  for (int64_t r = threadIdx.x; r < rows; r += kBlThreads) {
    const float c = cg[r];
    if (c == 0.0f) continue;
    const int mic = int(r / S.tier_count[t]);
    const int img = int(r - int64_t(mic) * S.tier_count[t]);
    int n[3], p[3];
    unpack_image(a.p.img_code[S.img_base + S.tier_first[t] + img], n, p);
    float D[3], sg[3];
    for (int d = 0; d < 3; ++d) {
      sg[d] = p[d] ? -1.0f : 1.0f;
      const double m = S.mics[mic][d] + (S.arr_moving ? ap[d] : 0.0);
      D[d] = float(double(sg[d]) * sp[d] + 2.0 * n[d] * S.dims[d] - m);
    }
    const float f = c * rsqrtf(fmaf(D[0], D[0], fmaf(D[1], D[1], D[2] * D[2])));
    gx += double(f * sg[0] * D[0]);
    gy += double(f * sg[1] * D[1]);
    gz += double(f * sg[2] * D[2]);
    hx -= double(f * D[0]);
    hy -= double(f * D[1]);
    hz -= double(f * D[2]);
  }
  part[0][threadIdx.x] = gx;
  part[1][threadIdx.x] = gy;
  part[2][threadIdx.x] = gz;
  part[3][threadIdx.x] = hx;
  part[4][threadIdx.x] = hy;
  part[5][threadIdx.x] = hz;
  __syncthreads();
  if (threadIdx.x < (arr ? 6 : 3)) {
    double acc = 0.0;
    for (int r = 0; r < kBlThreads; ++r) acc += part[threadIdx.x][r];
    if (threadIdx.x < 3) a.p.gk[3 * (S.knot_base[t] + jt) + threadIdx.x] = acc;
    else a.p.garr[3 * (S.knot_base[t] + jt) + threadIdx.x - 3] = acc;
  }
}

// dL/dparams[p]: sum of the chunk partials in chunk order (one CTA per scene).
__global__ void k_param_final(const __grid_constant__ KernelArgs a) {
  const SceneDev& S = scene_of(a, blockIdx.x);
  if (!S.dparams || threadIdx.x >= 48) return;
  double acc = 0.0;
  for (int c = 0; c < kParamChunks; ++c) acc += a.p.ppart[(int64_t(blockIdx.x) * kParamChunks + c) * 48 + threadIdx.x];
  S.dparams[threadIdx.x] = acc;
}

// Partial dL/d(array trajectory parameters) of one chunk of a scene's units,
// arranged as k_param_partial. The microphones sit at m + a(t) - a(0), so
// dL/dtheta_a = sum_j (J_a(t_j) - J_a(0))^T dL/da(t_j), dL/da summed over the
// microphones. Units: the knots of every tier, dL/da(t_j) from garr; with
// emission-time delays the (mic, knot, image) units, where at the reception
// time t_j the implicit derivative of c tau = |sigma o s(t_j - tau) + 2 n L - m(t_j)|
// gives dd/dm = -u / (1 + (sigma o u) . s'(e) / c), u = Delta / d.
__global__ void __launch_bounds__(kParamThreads) k_arr_param_partial(const __grid_constant__ KernelArgs a) {
  const int s = blockIdx.x / kParamChunks, chunk = blockIdx.x % kParamChunks;
  const SceneDev& S = scene_of(a, s);
  if (!S.darray || !S.arr_moving) return;
  extern __shared__ double rows[];  // [48][kParamThreads]
  for (int p = 0; p < 48; ++p) rows[p * kParamThreads + threadIdx.x] = 0.0;
  double* row = rows + threadIdx.x;
  const int last = S.n_tiers - 1;
  const bool ret = S.delay_model == 1;
  const int64_t total = ret ? S.n_opt_units
                            : S.knot_units_first[last] +
                                  (S.tier_up[last] > 1 ? int64_t(S.bl_knots[last]) : int64_t(S.tier_intervals[last]) + 1);
  double gsum[3] = {0.0, 0.0, 0.0};  // for the -J_a(0) term
  if (!ret) {
    const int64_t per_cta = (total + kParamChunks - 1) / kParamChunks;
    const int64_t per_thr = (per_cta + kParamThreads - 1) / kParamThreads;
    const int64_t lo = min(total, chunk * per_cta + threadIdx.x * per_thr);
    const int64_t hi = min(min(total, (chunk + 1) * per_cta), lo + per_thr);
    int t = 0;
    for (int64_t k = lo; k < hi; ++k) {
      while (t + 1 < S.n_tiers && k >= S.knot_units_first[t + 1]) ++t;
      if (S.tier_count[t] == 0) continue;
      const int64_t j = k - S.knot_units_first[t];
      const double* gk = a.p.garr + 3 * (S.knot_base[t] + j);
      const double g[3] = {gk[0], gk[1], gk[2]};
      double v[12];
      const int p0 = jacobian_terms<double>(S.arr_kind, S.arr_params, S.arr_n_ctrl, S.arr_duration,
                                            double((j - S.knot_shift[t]) * S.tier_coarse[t]) / S.fs, g, v);
      const int nt = jacobian_count(S.arr_kind);
      for (int i = 0; i < nt; ++i) row[(p0 + i) * kParamThreads] += v[i];
      for (int d = 0; d < 3; ++d) gsum[d] += g[d];
    }
  } else {
    const int64_t base = a.n_scenes > 1 ? a.tab.opt_prefix[s] : int64_t(0);
    const float4* HI = a.p.dense_hi + S.dense_base;
    const float4* LO = a.p.dense_lo + S.dense_base;
    const float xs = float(kDenseOver) * float(S.fs);
    const float rc = float(1.0 / S.c);
    const float rfs = float(1.0 / S.fs);
    const float k0 = float(S.dense_k0);
    const int64_t kmax = S.n_dense - 2;
    JacAcc acc(S.arr_kind, S.arr_params, S.arr_n_ctrl, S.arr_duration);
    const int64_t stride = int64_t(kParamChunks) * kParamThreads;
    for (int64_t k = int64_t(chunk) * kParamThreads + threadIdx.x; k < total; k += stride) {
      const OptUnit u = opt_unit(S, k);
      const int cnt = S.tier_count[u.t];
      const float gr = a.p.ograd[base + k].x + (u.k > 0 ? a.p.ograd[base + k - cnt].y : 0.0f);
      if (gr == 0.0f) continue;
      const int64_t kn = int64_t(u.k) * S.tier_step[u.t];
      const float es = float(double(kn) - a.p.otau[base + k]);  // emission time (samples)
      const float x = fmaf(float(kDenseOver), es, -k0);
      const int64_t i = min(max(int64_t(floorf(x)), int64_t(0)), kmax);
      const float f = x - float(i);
      const float4 h0 = HI[i], h1 = HI[i + 1], l0 = LO[i], l1 = LO[i + 1];
      const float ds[3] = {(h1.x - h0.x) + (l1.x - l0.x), (h1.y - h0.y) + (l1.y - l0.y),
                           (h1.z - h0.z) + (l1.z - l0.z)};
      const float sp[3] = {fmaf(f, ds[0], h0.x + l0.x), fmaf(f, ds[1], h0.y + l0.y), fmaf(f, ds[2], h0.z + l0.z)};
      const double* ap = a.p.arr_pos + 3 * (S.knot_base[u.t] + u.k);
      int n[3], p[3];
      unpack_image(a.p.img_code[S.img_base + S.tier_first[u.t] + u.img], n, p);
      float sg[3], D[3];
      for (int d = 0; d < 3; ++d) {
        sg[d] = p[d] ? -1.0f : 1.0f;
        const float m = float(S.mics[u.mic][d]) + float(ap[d]);
        D[d] = fmaf(sg[d], sp[d], fmaf(float(2 * n[d]), float(S.dims[d]), -m));
      }
      const float rd = rsqrtf(fmaf(D[0], D[0], fmaf(D[1], D[1], D[2] * D[2])));
      const float uv[3] = {D[0] * rd, D[1] * rd, D[2] * rd};
      const float vs = xs * (sg[0] * uv[0] * ds[0] + sg[1] * uv[1] * ds[1] + sg[2] * uv[2] * ds[2]);
      const float fac = -gr / fmaf(vs, rc, 1.0f);
      const float g[3] = {fac * uv[0], fac * uv[1], fac * uv[2]};
      acc.add(float(kn) * rfs, g, row);  // the microphone at the reception time
      for (int d = 0; d < 3; ++d) gsum[d] += double(g[d]);
    }
    acc.flush(row);
  }
  {  // - J_a(0)^T sum_j dL/da(t_j)
    const double g0[3] = {-gsum[0], -gsum[1], -gsum[2]};
    double v[12];
    const int p0 = jacobian_terms<double>(S.arr_kind, S.arr_params, S.arr_n_ctrl, S.arr_duration, 0.0, g0, v);
    const int nt = jacobian_count(S.arr_kind);
    for (int i = 0; i < nt; ++i) row[(p0 + i) * kParamThreads] += v[i];
  }
  __syncthreads();
  if (threadIdx.x < 48) {
    double acc = 0.0;
    for (int r = 0; r < kParamThreads; ++r) acc += rows[threadIdx.x * kParamThreads + r];
    a.p.ppart[(int64_t(s) * kParamChunks + chunk) * 48 + threadIdx.x] = acc;
  }
}

// dL/d(array trajectory parameters): the chunk partials in chunk order.
__global__ void k_arr_param_final(const __grid_constant__ KernelArgs a) {
  const SceneDev& S = scene_of(a, blockIdx.x);
  if (!S.darray || !S.arr_moving || threadIdx.x >= 48) return;
  double acc = 0.0;
  for (int c = 0; c < kParamChunks; ++c) acc += a.p.ppart[(int64_t(blockIdx.x) * kParamChunks + c) * 48 + threadIdx.x];
  S.darray[threadIdx.x] = acc;
}

// dL/dbeta_w: sum of the item partials in item order (one CTA per scene).
// 256 threads per scene: thread r sums rows r, r + 256, ... per wall (in
// order), then the thread sums are added in thread order.
constexpr int kBetaThreads = 256;
__global__ void __launch_bounds__(kBetaThreads) k_beta_final(const __grid_constant__ KernelArgs a) {
  __shared__ double part[6][kBetaThreads];
  const SceneDev& S = scene_of(a, blockIdx.x);
  if (!S.dbeta) return;
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int64_t rows = int64_t(S.n_mics) * S.n_blocks * S.n_tiles;
  for (int64_t rr = threadIdx.x; rr < rows; rr += kBetaThreads) {
    const float4 v0 = *reinterpret_cast<const float4*>(a.p.bpart + S.bpart_base + rr * 8);
    const float2 v1 = *reinterpret_cast<const float2*>(a.p.bpart + S.bpart_base + rr * 8 + 4);
    acc[0] += v0.x; acc[1] += v0.y; acc[2] += v0.z; acc[3] += v0.w; acc[4] += v1.x; acc[5] += v1.y;
  }
  for (int w = 0; w < 6; ++w) part[w][threadIdx.x] = acc[w];
  __syncthreads();
  if (threadIdx.x < 6) {
    double sum = 0.0;
    for (int r = 0; r < kBetaThreads; ++r) sum += part[threadIdx.x][r];
    S.dbeta[threadIdx.x] = sum;
  }
}

template <typename K>
cudaError_t persistent_launch(K kern, size_t smem, int64_t items, const KernelArgs& a, cudaStream_t st,
                              PerDevice* setup) {
  int grid = 0;
  cudaError_t pe = persistent_grid(*setup, kern, kBwThreads, smem, &grid);
  if (pe != cudaSuccess) return pe;
  const int g = int(items < grid ? items : grid);
  cudaError_t e = cudaMemsetAsync(a.p.counter, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (g > 0) kern<<<g, kBwThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

static const TileConfig kBwConfig = {kBwThreads, kBwChunks, kGradWcap, kBwRecCap, kBwBlock, 0};
const TileConfig& backward_tile_config() { return kBwConfig; }
size_t backward_unit_cap() { return kBwUnitCap; }
int64_t backward_bl_scratch_floats() { return kGradScratchFloats < kRecScratchFloats ? kGradScratchFloats : kRecScratchFloats; }
int backward_group_images() { return kDxGroupImages; }

cudaError_t launch_prefilter(const KernelArgs& a, cudaStream_t st, bool gradient_rows);

cudaError_t launch_backward_kernels(const KernelArgs& a, cudaStream_t st) {
  cudaError_t e = launch_prefilter(a, st, true);
  if (e != cudaSuccess) return e;
  // per device and kernel: shared-memory limit and persistent grid
  static PerDevice g_grad, g_grad_arr, g_dx16, g_dx32, g_dx64;
  if (a.totals[0] > 0) k_beta_table<<<unsigned((a.totals[0] + 255) / 256), 256, 0, st>>>(a);
  e = persistent_launch(k_adj_grad<false>, kGradSmem, a.totals[4], a, st, &g_grad);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.p.dxb, 0, sizeof(float) * size_t(a.p.dxb_floats), st);
  if (e != cudaSuccess) return e;
  if (a.taps <= 16) e = persistent_launch(k_adj_dx<16>, kDxSmem, a.totals[5], a, st, &g_dx16);
  else if (a.taps <= 32) e = persistent_launch(k_adj_dx<32>, kDxSmem, a.totals[5], a, st, &g_dx32);
  else e = persistent_launch(k_adj_dx<64>, kDxSmem, a.totals[5], a, st, &g_dx64);
  if (e != cudaSuccess) return e;
  const int T = 256;
  if (a.totals[2] > 0) k_dx_final<<<unsigned((a.totals[2] + T - 1) / T), T, 0, st>>>(a);
  if (a.totals[9] > 0) k_opt_grad<<<unsigned((a.totals[9] + 255) / 256), 256, 0, st>>>(a);
  if (a.totals[1] > 0)
    k_knot_final<false><<<unsigned((a.totals[1] + kKnotsPerCta - 1) / kKnotsPerCta), kKnotsPerCta * kKnotLanes, 0,
                          st>>>(a);
  if (a.want_array) {  // the array pass over the linear tiers, then dL/da per knot
    e = persistent_launch(k_adj_grad<true>, kGradSmem, a.totals[4], a, st, &g_grad_arr);
    if (e != cudaSuccess) return e;
    if (a.totals[1] > 0)
      k_knot_final<true><<<unsigned((a.totals[1] + kKnotsPerCta - 1) / kKnotsPerCta), kKnotsPerCta * kKnotLanes, 0,
                           st>>>(a);
  }
  if (a.totals[6] > 0 && a.totals[9] > 0) {
    k_opt_bl_rows<<<unsigned((a.totals[6] + 127) / 128), 128, 0, st>>>(a);
    k_opt_bl_knots<<<unsigned(a.totals[1]), kBlThreads, 0, st>>>(a);
  }
  {
    constexpr size_t smem = 48 * kParamThreads * sizeof(double);
    static PerDevice attr;  // the shared-memory limit, once per device
    int dev = 0, done = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaError_t ae = cudaSuccess;
    const int st_attr = attr.get(
        dev,
        [&](int* v) {
          ae = cudaFuncSetAttribute(k_param_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
          if (ae == cudaSuccess)
            ae = cudaFuncSetAttribute(k_arr_param_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
          *v = 1;
          return ae == cudaSuccess ? 0 : 1;
        },
        &done);
    if (st_attr != 0) return ae != cudaSuccess ? ae : cudaErrorInvalidDevice;
    k_param_partial<<<unsigned(a.n_scenes * kParamChunks), kParamThreads, smem, st>>>(a);
    k_param_final<<<unsigned(a.n_scenes), 64, 0, st>>>(a);
    if (a.want_array) {
      k_arr_param_partial<<<unsigned(a.n_scenes * kParamChunks), kParamThreads, smem, st>>>(a);
      k_arr_param_final<<<unsigned(a.n_scenes), 64, 0, st>>>(a);
    }
  }
  k_beta_final<<<unsigned(a.n_scenes), kBetaThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace msrc
