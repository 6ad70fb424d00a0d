// FP64 CPU oracle for moving-source image-source synthesis.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load
// this file; only the tests, the smoke check and the benchmark's CPU-baseline
// leg do. It shares no code, header, table or helper with the CUDA library.
//
// What it computes (arXiv 2508.03065, "Fast Algorithm for Moving Sound Source"):
//   * image set (Sec. II-A, Eq. 1, Allen-Berkley lattice): every lattice triple n
//     with |n_x|+|n_y|+|n_z| <= K and every parity p in {0,1}^3; image position
//     r_i(t) = (1-2p) o s(t) + 2 n o L_room; reflection factor
//     beta_i = prod_d beta_{d,0}^{|n_d-p_d|} beta_{d,1}^{|n_d|};
//     reflection count rho_i = sum_d |2 n_d - p_d|;
//   * hierarchical spatio-temporal sampling (Sec. II-C, "Fast Architecture"):
//     image i is in tier t (by rho_i); its distance d_i is evaluated exactly at
//     knots n_j = j*N_t and linearly interpolated to every audio sample;
//   * delay tau_i(n) = d_i(n) fs / c and gain A_i(n) = beta_i / (4 pi d_i(n))
//     (Sec. II-A, text after Eq. 2; Sec. II-C, text before Eq. 8); d_i at a
//     knot is the distance at the reception time, or (delay model 1) the
//     emission-time path length c tau with c tau = |r_i(t - tau) - m(t)|;
//   * discrete time-varying fractional delay (Sec. II-B): the ideal delay kernel
//     sin(pi u)/(pi u), truncated to L taps k = -L/2 .. L/2-1 and windowed
//     (Hann or Kaiser) -- or a Farrow polynomial per tap (Eq. 3) whose
//     coefficients come from a least-squares design -- applied at read
//     position t = n - tau_i(n):
//     m0 = floor(t), alpha = t - m0, e_i(n) = sum_k w(alpha+k) sinc(alpha+k) x[m0-k];
//   * superposition over images (Eq. 2 / Eq. 8): y[n] = sum_i A_i(n) e_i(n).
// x[m] is zero outside [0, Ns).
// Where the tap kernel jumps at the wrap alpha = 1 -> 0 (a low-order Farrow
// polynomial), read positions within a small delta of an integer may take
// either side in a lower precision; the *_envelope routines report the
// difference between the two sides, for comparisons beyond it
// (tests/test_oracle_envelope.py pins them).
//
// Every routine is templated on the scalar so that the same code, run in
// std::complex<double>, gives complex-step derivatives of the loss with respect
// to trajectory parameters and wall reflection coefficients, under either delay
// model (the emission-time delay's Newton iteration runs in the same scalar).
// Integer decisions (floor, tier, knot index, spline span) always use the real
// part.
//
// Parity pins: tests/test_oracle_pins.py (closed forms, library special
// cases, brute force, invariants). Readings of the paper where it is silent or
// garbled are listed in the design notes of the repository.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <limits>
#include <type_traits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cplx = std::complex<double>;
constexpr double kPi = 3.14159265358979323846264338327950288;

inline double re(double v) { return v; }
inline double re(const cplx& v) { return v.real(); }

// Read positions within `delta` samples of an integer: t = n - tau lies near
// the wrap alpha = 0 <-> alpha = 1, where a precision other than FP64 may take
// the other side, (m0 - 1, alpha + 1) or (m0 + 1, alpha - 1). Both sides are
// evaluations of the method; they agree up to the tap kernel's jump at the
// wrap (zero for the windowed sinc, not for a low-order Farrow polynomial).
// Returns false away from the wrap, else true with the other side's m0 and
// alpha in *m1, *a1.
bool other_side(double alpha, long m0, double delta, long* m1, double* a1) {
  if (alpha < delta) { *m1 = m0 - 1; *a1 = alpha + 1.0; return true; }
  if (alpha > 1.0 - delta) { *m1 = m0 + 1; *a1 = alpha - 1.0; return true; }
  return false;
}

}  // namespace

extern "C" {

// Scene description shared with oracle/api.py through ctypes.
struct OracleScene {
  double dims[3];         // room size L_x, L_y, L_z (m)
  double beta[6];         // reflection coefficients of walls x=0, x=Lx, y=0, y=Ly, z=0, z=Lz
  double c;               // speed of sound (m/s)
  double fs;              // sample rate (Hz)
  double kaiser_beta;     // Kaiser window shape
  double traj[48];        // trajectory parameters (see source_position)
  double duration;        // trajectory duration T (s), used by the spline
  double mic[3];          // microphone position (m)
  int32_t K;              // image set |n|_1 <= K
  int32_t n_tiers;        // number of sampling tiers (1..4)
  int32_t tier_max_rho[4];// tier t holds images with rho <= tier_max_rho[t] (first match)
  int32_t tier_step[4];   // knot spacing N_t (samples) of tier t
  int32_t taps;           // L (even)
  int32_t window;         // 0 = Hann, 1 = Kaiser, 2 = Farrow polynomial given in `farrow`
  int32_t traj_kind;      // 0 = line, 1 = circle, 2 = clamped cubic B-spline
  int32_t n_ctrl;         // number of spline control points
  int32_t farrow_order;   // window 2: polynomial order M
  const double* farrow;   // window 2: c[(k + L/2) * (M + 1) + q], tap weight sum_q c alpha^q
  int32_t arr_kind;       // microphone motion: -1 static; else a trajectory a(t) (kinds as the
  int32_t arr_n_ctrl;     //   source's) and the microphone sits at mic + a(t) - a(0)
  double arr_traj[48];
  double arr_duration;
  int32_t tier_up[4];     // knot upsampling of tier t: <= 1 linear between knots; U > 1: the
                          //   distance at U virtual knots per interval from a band-limited
                          //   interpolation of the knots, then linear between virtual knots
  int32_t up_halfwidth;   // half-width Q (knots) of that interpolation kernel
  int32_t delay_model;    // 0: the knot distance is |r_i(t) - m(t)| at the reception time t;
                          // 1: it is the emission-time (retarded) path length c tau with
                          //    c tau = |r_i(t - tau) - m(t)|
};

}  // extern "C"

namespace {

struct Image {
  int n[3];
  int p[3];
  int e[6];   // reflections off each wall
  int rho;    // total reflection count
  int tier;
};

// Image enumeration, Sec. II-A (Eq. 1) with the Allen-Berkley lattice.
std::vector<Image> enumerate_images(const OracleScene& S) {
  std::vector<Image> out;
  const int K = S.K;
  for (int nx = -K; nx <= K; ++nx)
    for (int ny = -K; ny <= K; ++ny)
      for (int nz = -K; nz <= K; ++nz) {
        if (std::abs(nx) + std::abs(ny) + std::abs(nz) > K) continue;
        for (int pb = 0; pb < 8; ++pb) {
          Image im;
          im.n[0] = nx; im.n[1] = ny; im.n[2] = nz;
          im.p[0] = pb & 1; im.p[1] = (pb >> 1) & 1; im.p[2] = (pb >> 2) & 1;
          im.rho = 0;
          for (int d = 0; d < 3; ++d) {
            im.e[2 * d] = std::abs(im.n[d] - im.p[d]);  // wall at coordinate 0
            im.e[2 * d + 1] = std::abs(im.n[d]);        // wall at coordinate L_d
            im.rho += std::abs(2 * im.n[d] - im.p[d]);
          }
          im.tier = S.n_tiers - 1;
          for (int t = 0; t < S.n_tiers; ++t)
            if (im.rho <= S.tier_max_rho[t]) { im.tier = t; break; }
          out.push_back(im);
        }
      }
  return out;
}

template <class T>
struct Params {
  T traj[48];
  T beta[6];
  T arr[48];  // microphone-array trajectory (used when arr_kind >= 0)
};

template <class T>
Params<T> params_from(const OracleScene& S) {
  Params<T> P;
  for (int i = 0; i < 48; ++i) P.traj[i] = T(S.traj[i]);
  for (int i = 0; i < 6; ++i) P.beta[i] = T(S.beta[i]);
  for (int i = 0; i < 48; ++i) P.arr[i] = T(S.arr_traj[i]);
  return P;
}

// Cox-de Boor recursion for the clamped uniform cubic B-spline basis.
// Knot vector: four zeros, interior knots k/(n_ctrl-3), four ones. The
// parameter u may be complex (a complex-step emission time): the knot span is
// chosen by its real part and the basis is the span's polynomial in u.
template <class U>
U bspline_basis(int i, int deg, U u, const std::vector<double>& kv) {
  const double ur = re(u);
  if (deg == 0) {
    const int last = static_cast<int>(kv.size()) - 1;
    // the closing interval includes u = 1
    if (ur == kv[last]) return U((kv[i] < ur && kv[i + 1] == ur) ? 1.0 : 0.0);
    return U((kv[i] <= ur && ur < kv[i + 1]) ? 1.0 : 0.0);
  }
  U a = U(0.0), b = U(0.0);
  const double d1 = kv[i + deg] - kv[i];
  const double d2 = kv[i + deg + 1] - kv[i + 1];
  if (d1 > 0) a = (u - kv[i]) / d1 * bspline_basis(i, deg - 1, u, kv);
  if (d2 > 0) b = (kv[i + deg + 1] - u) / d2 * bspline_basis(i + 1, deg - 1, u, kv);
  return a + b;
}

std::vector<double> clamped_knots(int n_ctrl) {
  const int segs = n_ctrl - 3;
  std::vector<double> kv;
  for (int i = 0; i < 4; ++i) kv.push_back(0.0);
  for (int i = 1; i < segs; ++i) kv.push_back(static_cast<double>(i) / segs);
  for (int i = 0; i < 4; ++i) kv.push_back(1.0);
  return kv;
}

// Point of a trajectory of one of the source's kinds at time t, with real or
// complex parameters p and a real or complex time t (the emission time of a
// complex-step delay). Parameter layout:
//   line:   p0[3], direction[3] (normalised here), speed v      -> p0 + v t dir
//   circle: centre[3], radius R, speed v, start angle theta0    -> centre + R(cos, sin, 0)(theta0 + v t / R)
//   spline: control points P_0..P_{n_ctrl-1} (3 each); u = clamp(t / T, 0, 1)
template <class T, class TT>
void trajectory_point_t(int kind, const T* p, int n_ctrl, double duration, TT t, T out[3]) {
  if (kind == 0) {
    T nrm = std::sqrt(p[3] * p[3] + p[4] * p[4] + p[5] * p[5]);
    for (int d = 0; d < 3; ++d) out[d] = p[d] + p[6] * t * p[3 + d] / nrm;
  } else if (kind == 1) {
    T R = p[3];
    T ang = p[5] + p[4] * t / R;
    out[0] = p[0] + R * std::cos(ang);
    out[1] = p[1] + R * std::sin(ang);
    out[2] = p[2];
  } else {
    // u = clamp(t / T, 0, 1), by the real part (a clamped u is constant)
    TT u = t / duration;
    if (re(u) < 0.0) u = TT(0.0);
    if (re(u) > 1.0) u = TT(1.0);
    const std::vector<double> kv = clamped_knots(n_ctrl);
    for (int d = 0; d < 3; ++d) out[d] = T(0.0);
    for (int c = 0; c < n_ctrl; ++c) {
      const TT B = bspline_basis(c, 3, u, kv);
      for (int d = 0; d < 3; ++d) out[d] += B * p[3 * c + d];
    }
  }
}

// Source position s(t), Sec. II-C ("sample a segment of the band-limited
// trajectory p(n)"), with the trajectory parameters of P.
template <class T, class TT>
void source_position(const OracleScene& S, const Params<T>& P, TT t, T out[3]) {
  trajectory_point_t(S.traj_kind, P.traj, S.n_ctrl, S.duration, t, out);
}

// Point of a trajectory with real parameters (the array motion and the
// exported helpers).
void trajectory_point(int kind, const double* p, int n_ctrl, double duration, double t, double out[3]) {
  trajectory_point_t(kind, p, n_ctrl, duration, t, out);
}

// Microphone position at time t: static, or carried by the array motion a(t)
// as mic + a(t) - a(0), with the array trajectory parameters of P.
template <class T>
void mic_position(const OracleScene& S, const Params<T>& P, double t, T out[3]) {
  for (int d = 0; d < 3; ++d) out[d] = T(S.mic[d]);
  if (S.arr_kind < 0) return;
  T a0[3], at[3];
  trajectory_point_t(S.arr_kind, P.arr, S.arr_n_ctrl, S.arr_duration, 0.0, a0);
  trajectory_point_t(S.arr_kind, P.arr, S.arr_n_ctrl, S.arr_duration, t, at);
  for (int d = 0; d < 3; ++d) out[d] += at[d] - a0[d];
}

// Euclidean distance from image i to the microphone at time t (Sec. II-A).
template <class T>
T image_distance(const OracleScene& S, const Params<T>& P, const Image& im, double t) {
  T s[3];
  source_position(S, P, t, s);
  T m[3];
  mic_position(S, P, t, m);
  T acc = T(0.0);
  for (int d = 0; d < 3; ++d) {
    const double sigma = 1.0 - 2.0 * im.p[d];
    T r = sigma * s[d] + 2.0 * im.n[d] * S.dims[d];
    T diff = r - m[d];
    acc += diff * diff;
  }
  return std::sqrt(acc);
}

// Emission-time (retarded) delay at reception time t (s): the tau > 0 with
// c tau = |r_i(t - tau) - m(t)|, i.e. the sound that reaches the microphone at
// t left the moving image at t - tau (the Green's function of Sec. II-A
// integrated along the image's path; Sec. II-A's delta(t - t' - R/c) read with
// R measured from the emission point). Newton's method from the reception-time
// distance, with the path's rate of change by a central difference (which only
// sets the rate of convergence), until the step's real part is below 1e-15 s,
// then three more steps. The function t_e -> t_e + |r_i(t_e) - m| / c is
// increasing below the speed of sound, so the root is unique. In complex
// arithmetic (a complex-step parameter) the iteration converges to the complex
// root, whose imaginary part is h times the implicit derivative of tau; the
// extra steps let that part settle (each step multiplies its error by about
// the difference between the slope and its central-difference estimate).
template <class T>
T retarded_delay(const OracleScene& S, const Params<T>& P, const Image& im, double t) {
  T m[3];
  mic_position(S, P, t, m);
  auto dist = [&](T te) {
    T s[3];
    source_position(S, P, te, s);
    T acc = T(0.0);
    for (int d = 0; d < 3; ++d) {
      const T r = (1.0 - 2.0 * im.p[d]) * s[d] + 2.0 * im.n[d] * S.dims[d] - m[d];
      acc += r * r;
    }
    return std::sqrt(acc);
  };
  T tau = dist(T(t)) / S.c;
  const double h = 1e-6;
  int settled = 0;
  for (int it = 0; it < 100 && settled < 4; ++it) {
    const T te = t - tau;
    const T F = S.c * tau - dist(te);
    const T dF = S.c + (dist(te + h) - dist(te - h)) / (2.0 * h);
    const T step = F / dF;
    tau -= step;
    if (std::fabs(re(step)) < 1e-15) ++settled;
  }
  return tau;
}

// Distance that sets an image's delay and gain at knot time t: the distance at
// the reception time, or the emission-time path length (delay_model 1).
template <class T>
T knot_distance(const OracleScene& S, const Params<T>& P, const Image& im, double t) {
  if (S.delay_model != 1) return image_distance(S, P, im, t);
  return S.c * retarded_delay(S, P, im, t);
}

template <class T>
T image_beta(const Params<T>& P, const Image& im) {
  T b = T(1.0);
  for (int w = 0; w < 6; ++w)
    for (int r = 0; r < im.e[w]; ++r) b *= P.beta[w];
  return b;
}

// Window over u in [-L/2, L/2].
template <class T>
T window_value(const OracleScene& S, T u) {
  const double L = S.taps;
  if (S.window == 0) return 0.5 * (1.0 + std::cos(2.0 * kPi * u / L));
  // Kaiser: I0(beta sqrt(z)) / I0(beta), z = 1 - (2u/L)^2, with
  // I0(beta sqrt(z)) = sum_j (beta^2 z / 4)^j / (j!)^2 (power series).
  const double b = S.kaiser_beta;
  T z = 1.0 - (2.0 * u / L) * (2.0 * u / L);
  T term = T(1.0), sum = T(1.0);
  double term0 = 1.0, sum0 = 1.0;
  for (int j = 1; j < 80; ++j) {
    term *= (b * b * z / 4.0) / (double(j) * double(j));
    sum += term;
    term0 *= (b * b / 4.0) / (double(j) * double(j));
    sum0 += term0;
  }
  return sum / sum0;
}

// Ideal fractional-delay kernel sin(pi u)/(pi u) (Sec. II-B).
template <class T>
T sinc_value(T u) {
  if (std::abs(u) == 0.0) return T(1.0);
  return std::sin(kPi * u) / (kPi * u);
}

// Tap weight for tap k at fractional read position alpha: the windowed ideal
// kernel, or (window 2) the Farrow polynomial of Eq. 3, h(k; alpha) =
// sum_q c_q(k) alpha^q, with coefficients designed outside (oracle/gls.py).
template <class T>
T tap_weight(const OracleScene& S, int k, T alpha) {
  if (S.window == 2) {
    const int P = S.farrow_order + 1;
    const double* c = S.farrow + (k + S.taps / 2) * P;
    T h = T(c[P - 1]);
    for (int q = P - 2; q >= 0; --q) h = h * alpha + c[q];
    return h;
  }
  T u = alpha + double(k);
  return window_value(S, u) * sinc_value(u);
}

inline double xval(const double* x, long Ns, long m) { return (m >= 0 && m < Ns) ? x[m] : 0.0; }

// Delay tau_i(n) (in samples), gain A_i(n) and distance d_i(n) at output sample
// n: knots of image i's tier at n_j = j N_t, exact distances there, linear
// interpolation of the distance in between (Sec. II-C, "Fast Architecture").
//
// Band-limited knot upsampling (tiers with U > 1, Sec. II-C: the distance is a
// band-limited signal sampled at the knots, recovered by an upsampler): the
// distance at virtual knot k (sample k N/U) is sum_j w_j d_j over the knots j
// with |k/U - j| < Q, w_j = h(k/U - j) / sum_i h(k/U - i), h(u) = sinc(u) times
// a Kaiser window over [-Q, Q] (shape 8, I0 by its power series); between
// virtual knots it is linear. At a knot (k multiple of U) the weights reduce to
// that knot alone.
double bessel_i0_series(double x) {
  double sum = 1.0, term = 1.0;
  for (int j = 1; j < 80; ++j) {
    term *= (x * x / 4.0) / (double(j) * double(j));
    sum += term;
  }
  return sum;
}

template <class T>
T upsampled_distance(const OracleScene& S, const Params<T>& P, const Image& im, long N, int U, long k) {
  const int Q = S.up_halfwidth > 0 ? S.up_halfwidth : 4;
  const double kBeta = 8.0;
  const long j0 = (k >= 0) ? k / U : -((-k + U - 1) / U);  // floor(k / U)
  const double x = double(k) / U;
  double w[64];
  double wsum = 0.0;
  for (int i = 0; i < 2 * Q; ++i) {
    const double u = x - double(j0 - Q + 1 + i);
    const double sincv = (u == 0.0) ? 1.0 : std::sin(kPi * u) / (kPi * u);
    const double z = std::max(0.0, 1.0 - (u / Q) * (u / Q));
    w[i] = sincv * bessel_i0_series(kBeta * std::sqrt(z)) / bessel_i0_series(kBeta);
    wsum += w[i];
  }
  T acc = T(0.0);
  for (int i = 0; i < 2 * Q; ++i)
    acc += (w[i] / wsum) * knot_distance(S, P, im, double((j0 - Q + 1 + i) * N) / S.fs);
  return acc;
}

template <class T>
void delay_gain(const OracleScene& S, const Params<T>& P, const Image& im, long n,
                T* tau, T* gain, T* dist) {
  const long Nc = S.tier_step[im.tier];
  const int U = S.tier_up[im.tier] > 1 ? S.tier_up[im.tier] : 1;
  const long N = Nc / U;  // spacing of the interpolated points
  const long j = n / N;
  const long nj = j * N;
  const double s = double(n - nj) / double(N);
  T dj = (U == 1) ? knot_distance(S, P, im, double(nj) / S.fs) : upsampled_distance(S, P, im, Nc, U, j);
  T d = dj;
  if (s != 0.0) {
    T dj1 = (U == 1) ? knot_distance(S, P, im, double(nj + N) / S.fs) : upsampled_distance(S, P, im, Nc, U, j + 1);
    d = dj + s * (dj1 - dj);
  }
  *dist = d;
  *tau = d * S.fs / S.c;
  *gain = image_beta(P, im) / (4.0 * kPi * d);
}

// Contribution A_i(n) e_i(n) of one image to output sample n (Eq. 8).
template <class T>
T image_sample(const OracleScene& S, const Params<T>& P, const Image& im,
               const double* x, long Ns, long n) {
  T tau, g, d;
  delay_gain(S, P, im, n, &tau, &g, &d);
  T t = double(n) - tau;
  const long m0 = static_cast<long>(std::floor(re(t)));
  T alpha = t - double(m0);
  const int half = S.taps / 2;
  T e = T(0.0);
  for (int k = -half; k <= half - 1; ++k) e += tap_weight(S, k, alpha) * xval(x, Ns, m0 - k);
  return g * e;
}

template <class T>
T output_sample(const OracleScene& S, const Params<T>& P, const std::vector<Image>& imgs,
                const double* x, long Ns, long n) {
  T acc = T(0.0);
  for (const Image& im : imgs) acc += image_sample(S, P, im, x, Ns, n);
  return acc;
}

std::vector<Image> select_images(const OracleScene& S, const int32_t* list, long n_list) {
  std::vector<Image> all = enumerate_images(S);
  if (!list) return all;
  std::vector<Image> sel;
  sel.reserve(n_list);
  for (long i = 0; i < n_list; ++i) sel.push_back(all[list[i]]);
  return sel;
}

}  // namespace

extern "C" {

long oracle_image_count(int32_t K) {
  long cnt = 0;
  for (int nx = -K; nx <= K; ++nx)
    for (int ny = -K; ny <= K; ++ny)
      for (int nz = -K; nz <= K; ++nz)
        if (std::abs(nx) + std::abs(ny) + std::abs(nz) <= K) cnt += 8;
  return cnt;
}

// Image table in enumeration order: n[3], p[3], e[6], rho, tier per image,
// beta_i in FP64.
void oracle_enumerate(const OracleScene* S, int32_t* n_out, int32_t* p_out, int32_t* e_out,
                      int32_t* rho_out, int32_t* tier_out, double* beta_out) {
  std::vector<Image> imgs = enumerate_images(*S);
  Params<double> P = params_from<double>(*S);
  for (size_t i = 0; i < imgs.size(); ++i) {
    for (int d = 0; d < 3; ++d) { n_out[3 * i + d] = imgs[i].n[d]; p_out[3 * i + d] = imgs[i].p[d]; }
    for (int w = 0; w < 6; ++w) e_out[6 * i + w] = imgs[i].e[w];
    rho_out[i] = imgs[i].rho;
    tier_out[i] = imgs[i].tier;
    beta_out[i] = image_beta(P, imgs[i]);
  }
}

void oracle_source_position(const OracleScene* S, const double* t, long n_t, double* out) {
  Params<double> P = params_from<double>(*S);
  for (long i = 0; i < n_t; ++i) source_position(*S, P, t[i], out + 3 * i);
}

// Exact distance of image `idx` (enumeration order) at times t[].
// Delay (s) of image idx at knot times t under the scene's delay model.
void oracle_knot_delay(const OracleScene* S, long idx, const double* t, long n_t, double* out) {
  const std::vector<Image> imgs = enumerate_images(*S);
  Params<double> P = params_from<double>(*S);
  for (long i = 0; i < n_t; ++i) out[i] = knot_distance(*S, P, imgs[idx], t[i]) / S->c;
}

// Complex-step derivative of the knot delay (s) of image idx at times t[]
// with respect to one parameter (ids as in oracle_loss_grad_cs):
// out[i] = Im(delay(theta + i h e_q)) / h.
void oracle_knot_delay_cs(const OracleScene* S, long idx, const double* t, long n_t, int32_t param_id, double h,
                          double* out) {
  const std::vector<Image> imgs = enumerate_images(*S);
  Params<cplx> P = params_from<cplx>(*S);
  if (param_id < 48) P.traj[param_id] += cplx(0.0, h);
  else if (param_id < 54) P.beta[param_id - 48] += cplx(0.0, h);
  else P.arr[param_id - 54] += cplx(0.0, h);
  for (long i = 0; i < n_t; ++i) out[i] = (knot_distance(*S, P, imgs[idx], t[i]) / S->c).imag() / h;
}

void oracle_image_distance(const OracleScene* S, long idx, const double* t, long n_t, double* out) {
  std::vector<Image> imgs = enumerate_images(*S);
  Params<double> P = params_from<double>(*S);
  for (long i = 0; i < n_t; ++i) out[i] = image_distance(*S, P, imgs[idx], t[i]);
}

// Interpolated delay (samples), gain and distance of image `idx` at samples n[].
void oracle_delay_gain(const OracleScene* S, long idx, const int64_t* n, long n_n,
                       double* tau, double* gain, double* dist) {
  std::vector<Image> imgs = enumerate_images(*S);
  Params<double> P = params_from<double>(*S);
  for (long i = 0; i < n_n; ++i) delay_gain(*S, P, imgs[idx], n[i], tau + i, gain + i, dist + i);
}

void oracle_tap_weights(const OracleScene* S, const double* alpha, long n_alpha, double* out) {
  const int half = S->taps / 2;
  for (long a = 0; a < n_alpha; ++a)
    for (int k = -half; k <= half - 1; ++k)
      out[a * S->taps + (k + half)] = tap_weight(*S, k, alpha[a]);
}

void oracle_window(const OracleScene* S, const double* u, long n_u, double* out) {
  for (long i = 0; i < n_u; ++i) out[i] = window_value(*S, u[i]);
}

// y[idx[q]] for the listed output samples, over the listed images (enumeration
// indices, in the given order; null = all images in enumeration order).
void oracle_y_at(const OracleScene* S, const double* x, long Ns, const int64_t* idx, long n_idx,
                 const int32_t* img_list, long n_img, double* y) {
  std::vector<Image> imgs = select_images(*S, img_list, n_img);
  Params<double> P = params_from<double>(*S);
#pragma omp parallel for schedule(dynamic, 4)
  for (long q = 0; q < n_idx; ++q) y[q] = output_sample(*S, P, imgs, x, Ns, idx[q]);
}

// Full output y[0 .. n_out).
void oracle_synthesize(const OracleScene* S, const double* x, long Ns, long n_out, double* y) {
  std::vector<Image> imgs = enumerate_images(*S);
  Params<double> P = params_from<double>(*S);
#pragma omp parallel for schedule(dynamic, 16)
  for (long n = 0; n < n_out; ++n) y[n] = output_sample(*S, P, imgs, x, Ns, n);
}

// Adjoint with respect to the source signal: dx = A^T dy, with A the linear map
// x -> y defined above, written as the plain transpose sum
// dx[m0_i(n) - k] += dy[n] A_i(n) w(alpha_i(n)+k) sinc(alpha_i(n)+k).
void oracle_adjoint_x(const OracleScene* S, const double* dy, long n_out, long Ns, double* dx) {
  std::vector<Image> imgs = enumerate_images(*S);
  Params<double> P = params_from<double>(*S);
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  std::vector<std::vector<double>> part(nthr, std::vector<double>(Ns, 0.0));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    std::vector<double>& acc = part[tid];
#pragma omp for schedule(dynamic, 16)
    for (long n = 0; n < n_out; ++n) {
      if (dy[n] == 0.0) continue;
      for (const Image& im : imgs) {
        double tau, g, d;
        delay_gain(*S, P, im, n, &tau, &g, &d);
        const double t = double(n) - tau;
        const long m0 = static_cast<long>(std::floor(t));
        const double alpha = t - double(m0);
        const int half = S->taps / 2;
        for (int k = -half; k <= half - 1; ++k) {
          const long m = m0 - k;
          if (m >= 0 && m < Ns) acc[m] += dy[n] * g * tap_weight(*S, k, alpha);
        }
      }
    }
  }
  for (long m = 0; m < Ns; ++m) {
    double s = 0.0;
    for (int t = 0; t < nthr; ++t) s += part[t][m];
    dx[m] = s;
  }
}

// y as oracle_synthesize, and env[n] = sum over the image-samples of output n
// whose read position lies within `delta` of an integer of |A_i(n)| times the
// difference between the two sides' tap sums (see other_side): the spread of
// valid results where the read position's side is a matter of precision.
void oracle_synthesize_envelope(const OracleScene* S, const double* x, long Ns, long n_out, double delta,
                                double* y, double* env) {
  std::vector<Image> imgs = enumerate_images(*S);
  Params<double> P = params_from<double>(*S);
  const int half = S->taps / 2;
#pragma omp parallel for schedule(dynamic, 16)
  for (long n = 0; n < n_out; ++n) {
    double acc = 0.0, spread = 0.0;
    for (const Image& im : imgs) {
      double tau, g, d;
      delay_gain(*S, P, im, n, &tau, &g, &d);
      const double t = double(n) - tau;
      const long m0 = static_cast<long>(std::floor(t));
      const double alpha = t - double(m0);
      double e = 0.0;
      for (int k = -half; k <= half - 1; ++k) e += tap_weight(*S, k, alpha) * xval(x, Ns, m0 - k);
      acc += g * e;
      long m1;
      double a1;
      if (other_side(alpha, m0, delta, &m1, &a1)) {
        double e1 = 0.0;
        for (int k = -half; k <= half - 1; ++k) e1 += tap_weight(*S, k, a1) * xval(x, Ns, m1 - k);
        spread += std::fabs(g * (e1 - e));
      }
    }
    y[n] = acc;
    env[n] = spread;
  }
}

// dx as oracle_adjoint_x, and env[m] = sum over the image-samples (n, i) near
// the wrap (see other_side) of |dy[n] A_i(n)| times the difference between the
// two sides' weights of x[m].
void oracle_adjoint_x_envelope(const OracleScene* S, const double* dy, long n_out, long Ns, double delta,
                               double* dx, double* env) {
  std::vector<Image> imgs = enumerate_images(*S);
  Params<double> P = params_from<double>(*S);
  const int half = S->taps / 2;
  for (long m = 0; m < Ns; ++m) { dx[m] = 0.0; env[m] = 0.0; }
  std::vector<double> w0(S->taps + 1), w1(S->taps + 1);
  for (long n = 0; n < n_out; ++n) {
    if (dy[n] == 0.0) continue;
    for (const Image& im : imgs) {
      double tau, g, d;
      delay_gain(*S, P, im, n, &tau, &g, &d);
      const double t = double(n) - tau;
      const long m0 = static_cast<long>(std::floor(t));
      const double alpha = t - double(m0);
      for (int k = -half; k <= half - 1; ++k) {
        const long m = m0 - k;
        if (m >= 0 && m < Ns) dx[m] += dy[n] * g * tap_weight(*S, k, alpha);
      }
      long m1;
      double a1;
      if (!other_side(alpha, m0, delta, &m1, &a1)) continue;
      // weights of x[m] on either side, over the union of the two tap ranges
      const long lo = std::min(m0, m1) - (half - 1), hi = std::max(m0, m1) + half;
      for (long m = lo; m <= hi; ++m) {
        const long k0 = m0 - m, k1 = m1 - m;
        const double h0 = (k0 >= -half && k0 <= half - 1) ? tap_weight(*S, int(k0), alpha) : 0.0;
        const double h1 = (k1 >= -half && k1 <= half - 1) ? tap_weight(*S, int(k1), a1) : 0.0;
        if (m >= 0 && m < Ns) env[m] += std::fabs(dy[n] * g * (h1 - h0));
      }
    }
  }
}

// Loss 0.5 * sum_n (y[n] - target[n])^2 over n in [0, n_out).
double oracle_loss(const OracleScene* S, const double* x, long Ns, long n_out, const double* target) {
  std::vector<double> y(n_out);
  oracle_synthesize(S, x, Ns, n_out, y.data());
  double L = 0.0;
  for (long n = 0; n < n_out; ++n) L += 0.5 * (y[n] - target[n]) * (y[n] - target[n]);
  return L;
}

// Complex-step derivatives of the loss: for each requested parameter q,
// param_ids[q] < 48 selects traj[param_ids[q]], 48..53 selects beta[param_ids[q]-48],
// 54..101 selects the array trajectory's arr_traj[param_ids[q]-54];
// grad[q] = Im(L(theta + i h e_q)) / h.
void oracle_loss_grad_cs(const OracleScene* S, const double* x, long Ns, long n_out,
                         const double* target, const int32_t* param_ids, long n_params,
                         double h, double* grad) {
  std::vector<Image> imgs = enumerate_images(*S);
  for (long q = 0; q < n_params; ++q) {
    Params<cplx> P = params_from<cplx>(*S);
    const int id = param_ids[q];
    if (id < 48) P.traj[id] += cplx(0.0, h);
    else if (id < 54) P.beta[id - 48] += cplx(0.0, h);
    else P.arr[id - 54] += cplx(0.0, h);
    double im_sum = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : im_sum)
    for (long n = 0; n < n_out; ++n) {
      cplx y = output_sample(*S, P, imgs, x, Ns, n);
      cplx r = y - target[n];
      im_sum += (0.5 * r * r).imag();
    }
    grad[q] = im_sum / h;
  }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
