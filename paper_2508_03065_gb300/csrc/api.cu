// Host side of the msrc C ABI: validation, Farrow coefficient fit, workspace
// planning and launch sequencing. See include/msrc.h for the contract.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "msrc_internal.h"

namespace msrc {
cudaError_t launch_backward_kernels(const KernelArgs& a, cudaStream_t st);
size_t backward_unit_cap();
int backward_group_images();
}  // namespace msrc

using namespace msrc;

namespace {
thread_local std::string g_last_error;
}

namespace msrc {
// Sets the thread-local message returned by msrc_last_error (used by entry
// points defined in other translation units).
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
}  // namespace msrc

struct msrc_room {
  msrc_room_desc d;
  int32_t tier_step[MSRC_MAX_TIERS];
  int64_t n_images;
  int64_t tier_count[MSRC_MAX_TIERS];
  int kL;  // tap template length (16, 32 or 64)
  double gls[kMaxTaps * (kFarrowDeg + 1)];              // window 2: c[k + L/2][q] of the design
  float farrow[kFarrowSegs][kFarrowCoef][kMaxTaps];    // synthesis and dx (degree 4)
  float farrow_g[kFarrowSegs][kGradCoef][kMaxTaps];    // gradient kernel (degree 5)
  double fit_error;                                    // of the synthesis table
  double fit_error_g;
  bool has_traj;
  msrc_traj_desc traj;
  double mics[MSRC_MAX_MICS][3];
  int32_t n_mics;
  bool arr_moving;          // microphones carried by `arr`: m + a(t) - a(0)
  msrc_traj_desc arr;
  double validated_from;   // trajectory checked on [validated_from, validated_until]
  double validated_until;  // (empty while validated_until < validated_from)
  double max_speed;        // largest speed seen on that range (m/s, 1 ms steps)
  int32_t tier_up[MSRC_MAX_TIERS];  // band-limited knot upsampling factor (1 = linear)
  int32_t up_q;                     // its kernel half-width (knots)
};

namespace {

// Tile configuration of calls that name none (MSRC_TILE_DEFAULT): the process
// default set by msrc_set_tile_config; initially MSRC_TILE_AUTO.
std::atomic<int> g_tile_config{MSRC_TILE_AUTO};
uint32_t g_test_extra_tx = 0;  // msrc_test_stall_window_copies

// MSRC_TILE_AUTO: the configuration measured fastest for the call's knot
// layout. Knot spacings of at most 24 samples (1 kHz knots at 16 kHz) need
// many records per image: tile configuration 14 (768-sample tiles, two CTAs
// per SM, knot records: 162 images per block at 16-sample spacing) holds
// enough images per block. Sparser knots run in configuration 11 (the same
// tiles with interval records, which save a load and a multiply per image
// pair and sample). The spacing that counts is that of the tiers holding most
// of the call's images.
int auto_config(const msrc_room_t* rooms, int n) {
  int64_t dense = 0, sparse = 0;
  for (int r = 0; r < n; ++r) {
    const msrc_room* R = rooms ? rooms[r] : nullptr;
    if (!R) continue;
    for (int t = 0; t < R->d.n_tiers; ++t) {
      const int N = R->tier_step[t] / std::max(1, R->tier_up[t]);
      (N <= 24 ? dense : sparse) += R->tier_count[t] * int64_t(R->n_mics);
    }
  }
  return dense > sparse ? 14 : 11;
}

// The configuration a call runs in: its own, the process default, or the
// automatic choice for these rooms.
int call_config(int32_t tile_config, const msrc_room_t* rooms, int n) {
  const int c = tile_config == MSRC_TILE_DEFAULT ? g_tile_config.load() : tile_config;
  return c == MSRC_TILE_AUTO ? auto_config(rooms, n) : c;
}

// Optional per-phase timing with CUDA events recorded on the launching stream.
// Phases: 0 setup (images, sort, knots, records), 1 prefilter, 2 synthesis, 3 reduction.
constexpr int kPhases = 4;
constexpr int kProfSets = 256;
struct Profiler {
  bool on = false;
  cudaEvent_t ev[kProfSets][kPhases + 1];
  int next = 0, pending = 0;
} g_prof;

msrc_status fail(msrc_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

msrc_status cuda_fail(cudaError_t e, const char* what) {
  return fail(MSRC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr double kPiD = 3.14159265358979323846;

// ---------------------------------------------------------------- windowed sinc
double bessel_i0(double x) {
  // I0(x) = sum_j ((x/2)^j / j!)^2
  double sum = 1.0, term = 1.0;
  for (int j = 1; j < 200; ++j) {
    term *= (x * 0.5) / j;
    const double t2 = term * term;
    sum += t2;
    if (t2 < 1e-18 * sum) break;
  }
  return sum;
}

double window_fn(const msrc_room_desc& d, double u) {
  const double L = d.taps;
  if (d.window == 0) return 0.5 * (1.0 + std::cos(2.0 * kPiD * u / L));
  const double r = 2.0 * u / L;
  const double z = std::max(0.0, 1.0 - r * r);
  return bessel_i0(d.kaiser_beta * std::sqrt(z)) / bessel_i0(d.kaiser_beta);
}

double kernel_fn(const msrc_room_desc& d, double u) {
  const double s = (u == 0.0) ? 1.0 : std::sin(kPiD * u) / (kPiD * u);
  return window_fn(d, u) * s;
}

// ---------------------------------------------------------------- least-squares Farrow design
// Gauss-Legendre nodes and weights on [0, 1] (Newton on the three-term
// recurrence of the Legendre polynomials).
void gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPiD * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Solves A X = B in place (A n x n, B n x m, row-major) by Gaussian
// elimination with partial pivoting; false when A is singular.
bool solve_dense(int n, int m, std::vector<double>& A, std::vector<double>& B) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[r * n + col]) > std::fabs(A[piv * n + col])) piv = r;
    if (A[piv * n + col] == 0.0) return false;
    if (piv != col) {
      for (int c = 0; c < n; ++c) std::swap(A[col * n + c], A[piv * n + c]);
      for (int c = 0; c < m; ++c) std::swap(B[col * m + c], B[piv * m + c]);
    }
    for (int r = col + 1; r < n; ++r) {
      const double f = A[r * n + col] / A[col * n + col];
      if (f == 0.0) continue;
      for (int c = col; c < n; ++c) A[r * n + c] -= f * A[col * n + c];
      for (int c = 0; c < m; ++c) B[r * m + c] -= f * B[col * m + c];
    }
  }
  for (int r = n - 1; r >= 0; --r)
    for (int c = 0; c < m; ++c) {
      double acc = B[r * m + c];
      for (int k = r + 1; k < n; ++k) acc -= A[r * n + k] * B[k * m + c];
      B[r * m + c] = acc / A[r * n + r];
    }
  return true;
}

// Least-squares Farrow design (Sec. II-B, Eq. 3-4, the complex-domain fit of
// the frequency response): c[k + L/2][q], q <= M, minimising the integral over
// alpha in [0, 1] and w in [0, pi] of V(w) |sum_k h(k; alpha) e^{-jwk} - e^{jw alpha}|^2
// (V = 1 up to wp, kStopWeight above). Normal equations: the Gram matrix
// factors as A (x) T with A[q][q'] = 1/(q + q' + 1) (the alpha integral) and
// T[k][k'] = integral of V(w) cos(w (k - k')) dw, the right-hand side is
// b[k][q] = integral over alpha of alpha^q * integral of V(w) cos(w (alpha + k)) dw,
// so C = T^{-1} B A^{-1}.
constexpr double kStopWeight = 1e-3;
bool gls_design(int L, int M, double passband, double* c /* L x (M + 1) */) {
  const double wp = passband * kPiD, lam = kStopWeight;
  const int P = M + 1;
  // integral of V(w) cos(w u) dw over [0, pi]
  auto vcos = [&](double u) {
    if (u == 0.0) return (1.0 - lam) * wp + lam * kPiD;
    return ((1.0 - lam) * std::sin(wp * u) + lam * std::sin(kPiD * u)) / u;
  };
  std::vector<double> T(size_t(L) * L), B(size_t(L) * P, 0.0), A(size_t(P) * P);
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) {
      const int m = i - j;
      T[size_t(i) * L + j] = m == 0 ? vcos(0.0) : (1.0 - lam) * std::sin(wp * m) / m;  // sin(pi m) = 0
    }
  constexpr int kNodes = 64;
  double xa[kNodes], wa[kNodes];
  gauss_legendre01(kNodes, xa, wa);
  for (int i = 0; i < L; ++i) {
    const int k = i - L / 2;
    for (int g = 0; g < kNodes; ++g) {
      const double v = wa[g] * vcos(xa[g] + k);
      double pw = 1.0;
      for (int q = 0; q < P; ++q) { B[size_t(i) * P + q] += v * pw; pw *= xa[g]; }
    }
  }
  if (!solve_dense(L, P, T, B)) return false;  // B <- T^{-1} B
  for (int q = 0; q < P; ++q)
    for (int r = 0; r < P; ++r) A[size_t(q) * P + r] = 1.0 / (q + r + 1.0);
  // C = B A^{-1}: solve A C^T = B^T (A symmetric)
  std::vector<double> Bt(size_t(P) * L);
  for (int i = 0; i < L; ++i)
    for (int q = 0; q < P; ++q) Bt[size_t(q) * L + i] = B[size_t(i) * P + q];
  if (!solve_dense(P, L, A, Bt)) return false;
  for (int i = 0; i < L; ++i)
    for (int q = 0; q < P; ++q) c[size_t(i) * P + q] = Bt[size_t(q) * L + i];
  return true;
}

// Tap weight h(k; alpha) of the room's fractional-delay filter: the windowed
// ideal kernel (Hann, Kaiser) or the least-squares Farrow polynomial.
double tap_fn(const msrc_room& R, int k, double alpha) {
  if (R.d.window == 2) {
    const int P = R.d.farrow_order + 1;
    const double* c = R.gls + size_t(k + R.d.taps / 2) * P;
    double h = c[P - 1];
    for (int q = P - 2; q >= 0; --q) h = h * alpha + c[q];
    return h;
  }
  return kernel_fn(R.d, alpha + k);
}

// Farrow coefficients (Sec. II-B, Eq. 3-4): for tap k and segment s of the
// fractional delay alpha in [s/S, (s+1)/S), h(k; alpha) ~ sum_q c[s][q][k] v^q
// with v = 2 (alpha S - s) - 1, q < P. Interpolation at the Chebyshev nodes of
// v (near-minimax); returns the error against the exact windowed sinc measured
// on a dense grid with the float coefficients the device uses. out is
// [kFarrowSegs][P][kMaxTaps].
double fit_farrow(const msrc_room& R, int P, float* out) {
  const int L = R.d.taps;
  const int kL = R.kL;
  std::memset(out, 0, sizeof(float) * kFarrowSegs * P * kMaxTaps);
  auto C = [&](int s, int q, int kk) -> float& { return out[(s * P + q) * kMaxTaps + kk]; };
  double worst = 0.0;
  for (int s = 0; s < kFarrowSegs; ++s)
    for (int k = -L / 2; k <= L / 2 - 1; ++k) {
      double V[kGradCoef][kGradCoef + 1];
      for (int i = 0; i < P; ++i) {
        const double v = std::cos(kPiD * (i + 0.5) / P);
        const double alpha = (s + 0.5 * (v + 1.0)) / kFarrowSegs;
        double pw = 1.0;
        for (int q = 0; q < P; ++q) { V[i][q] = pw; pw *= v; }
        V[i][P] = tap_fn(R, k, alpha);
      }
      // Gaussian elimination with partial pivoting
      for (int col = 0; col < P; ++col) {
        int piv = col;
        for (int r = col + 1; r < P; ++r)
          if (std::fabs(V[r][col]) > std::fabs(V[piv][col])) piv = r;
        if (piv != col)
          for (int c = 0; c <= P; ++c) std::swap(V[col][c], V[piv][c]);
        for (int r = col + 1; r < P; ++r) {
          const double f = V[r][col] / V[col][col];
          for (int c = col; c <= P; ++c) V[r][c] -= f * V[col][c];
        }
      }
      double coef[kGradCoef];
      for (int r = P - 1; r >= 0; --r) {
        double acc = V[r][P];
        for (int c = r + 1; c < P; ++c) acc -= V[r][c] * coef[c];
        coef[r] = acc / V[r][r];
      }
      for (int q = 0; q < P; ++q) C(s, q, k + kL / 2) = float(coef[q]);
      for (int g = 0; g <= 400; ++g) {
        const double v = -1.0 + 2.0 * g / 400.0;
        const double alpha = (s + 0.5 * (v + 1.0)) / kFarrowSegs;
        double e = 0.0;
        for (int q = P - 1; q >= 0; --q) e = e * v + double(C(s, q, k + kL / 2));
        worst = std::max(worst, std::fabs(e - tap_fn(R, k, alpha)));
      }
    }
  return worst;
}

// ---------------------------------------------------------------- geometry
int64_t count_images(int K) {
  return 8LL * (2 * K + 1) * (2LL * K * K + 2 * K + 3) / 3;
}

int tier_of(const msrc_room_desc& d, int rho) {
  for (int t = 0; t < d.n_tiers; ++t)
    if (rho <= d.tier_max_rho[t]) return t;
  return d.n_tiers - 1;
}

void count_tiers(msrc_room& R) {
  for (int t = 0; t < MSRC_MAX_TIERS; ++t) R.tier_count[t] = 0;
  const int K = R.d.max_order;
  for (int nx = -K; nx <= K; ++nx)
    for (int ny = -K; ny <= K; ++ny)
      for (int nz = -K; nz <= K; ++nz) {
        if (std::abs(nx) + std::abs(ny) + std::abs(nz) > K) continue;
        for (int pb = 0; pb < 8; ++pb) {
          const int n[3] = {nx, ny, nz};
          int rho = 0;
          for (int d = 0; d < 3; ++d) rho += std::abs(2 * n[d] - ((pb >> d) & 1));
          R.tier_count[tier_of(R.d, rho)]++;
        }
      }
  R.n_images = count_images(K);
}

void host_source(const msrc_traj_desc& T, double t, double out[3]) {
  const double* p = T.params;
  if (T.kind == 0) {
    const double nrm = std::sqrt(p[3] * p[3] + p[4] * p[4] + p[5] * p[5]);
    for (int d = 0; d < 3; ++d) out[d] = p[d] + p[6] * t * p[3 + d] / nrm;
  } else if (T.kind == 1) {
    const double a = p[5] + p[4] * t / p[3];
    out[0] = p[0] + p[3] * std::cos(a);
    out[1] = p[1] + p[3] * std::sin(a);
    out[2] = p[2];
  } else {
    // uniform clamped cubic B-spline via de Boor
    const int m = T.n_ctrl - 3;
    double u = std::min(1.0, std::max(0.0, t / T.duration_s));
    const int span = std::min(int(u * m), m - 1);
    auto knot = [m](int i) { return std::min(1.0, std::max(0.0, double(i - 3) / m)); };
    double dd[4][3];
    for (int j = 0; j < 4; ++j)
      for (int c = 0; c < 3; ++c) dd[j][c] = p[3 * (span + j) + c];
    const int k = span + 3;
    for (int r = 1; r <= 3; ++r)
      for (int j = 3; j >= r; --j) {
        const int i = j + k - 3;
        const double den = knot(i + 4 - r) - knot(i);
        const double al = den > 0 ? (u - knot(i)) / den : 0.0;
        for (int c = 0; c < 3; ++c) dd[j][c] = (1 - al) * dd[j - 1][c] + al * dd[j][c];
      }
    for (int c = 0; c < 3; ++c) out[c] = dd[3][c];
  }
}

// Power-basis cubics of the spline's segments: segment s is interpolated at
// x = 0, 1/3, 2/3, 1 (host_source, de Boor) and the cubic through the four
// points solved for (the segment is a cubic, so this is exact up to rounding:
// about 1e-14 relative).
void spline_segments(const msrc_traj_desc& T, double poly[MSRC_MAX_CTRL - 3][3][4]) {
  const int m = T.n_ctrl - 3;
  for (int sg = 0; sg < m; ++sg) {
    double v[4][3];
    for (int k = 0; k < 4; ++k) host_source(T, (sg + k / 3.0) / m * T.duration_s, v[k]);
    for (int c = 0; c < 3; ++c) {
      // Newton divided differences on the nodes 0, h, 2h, 3h (h = 1/3)
      const double h = 1.0 / 3.0;
      const double f0 = v[0][c], f1 = v[1][c], f2 = v[2][c], f3 = v[3][c];
      const double d1 = (f1 - f0) / h, d2 = (f2 - f1) / h, d3 = (f3 - f2) / h;
      const double e1 = (d2 - d1) / (2 * h), e2 = (d3 - d2) / (2 * h);
      const double g = (e2 - e1) / (3 * h);
      // p(x) = f0 + d1 x + e1 x (x - h) + g x (x - h)(x - 2h), in powers of x
      poly[sg][c][0] = f0;
      poly[sg][c][1] = d1 - e1 * h + g * 2 * h * h;
      poly[sg][c][2] = e1 - 3 * g * h;
      poly[sg][c][3] = g;
    }
  }
}

// Checks the source path and the microphones on a 1 ms grid over
// [t_begin, t_end] (t_begin <= 0 <= t_end; band-limited knot upsampling
// evaluates the path's extension before 0 and past its end): the source
// strictly inside the room, every microphone (carried by the array motion when
// there is one) strictly inside and at least 0.1 m from the source, and the
// source speed plus the array speed (a bound on the rate of change of every
// image distance) below c. Records that largest rate.
msrc_status validate_traj_range(msrc_room& R, double t_begin, double t_end) {
  const bool have = R.validated_until >= R.validated_from;
  if (have && t_begin >= R.validated_from && t_end <= R.validated_until) return MSRC_OK;
  const double dt = 1e-3;
  const long steps = long(std::ceil((t_end - t_begin) / dt));
  double prev[3], aprev[3] = {0.0, 0.0, 0.0}, a0[3] = {0.0, 0.0, 0.0};
  double vmax = 0.0;
  host_source(R.traj, t_begin, prev);
  if (R.arr_moving) {
    host_source(R.arr, 0.0, a0);
    host_source(R.arr, t_begin, aprev);
  }
  for (long i = 0; i <= steps; ++i) {
    const double t = std::min(t_begin + i * dt, t_end);
    double s[3], a[3] = {0.0, 0.0, 0.0};
    host_source(R.traj, t, s);
    if (R.arr_moving) host_source(R.arr, t, a);
    for (int d = 0; d < 3; ++d)
      if (!(s[d] > 0.0 && s[d] < R.d.dims[d]))
        return fail(MSRC_ERR_INVALID_ARG, "trajectory leaves the room at t=%.4f s", t);
    for (int m = 0; m < R.n_mics; ++m) {
      double q = 0;
      for (int d = 0; d < 3; ++d) {
        const double md = R.mics[m][d] + (R.arr_moving ? a[d] - a0[d] : 0.0);
        if (!(md > 0.0 && md < R.d.dims[d]))
          return fail(MSRC_ERR_INVALID_ARG, "microphone %d leaves the room at t=%.4f s", m, t);
        q += (s[d] - md) * (s[d] - md);
      }
      if (std::sqrt(q) < 0.1)
        return fail(MSRC_ERR_INVALID_ARG, "trajectory within 0.1 m of microphone %d at t=%.4f s", m, t);
    }
    if (i > 0) {
      double q = 0, qa = 0;
      for (int d = 0; d < 3; ++d) {
        q += (s[d] - prev[d]) * (s[d] - prev[d]);
        qa += (a[d] - aprev[d]) * (a[d] - aprev[d]);
      }
      const double v = (std::sqrt(q) + std::sqrt(qa)) / dt;
      if (v >= R.d.c)
        return fail(MSRC_ERR_INVALID_ARG, "source plus array speed reaches c near t=%.4f s", t);
      vmax = std::max(vmax, v);
    }
    std::memcpy(prev, s, sizeof(prev));
    std::memcpy(aprev, a, sizeof(aprev));
  }
  // both ranges contain [0, duration], so their union is an interval
  R.validated_from = have ? std::min(R.validated_from, t_begin) : t_begin;
  R.validated_until = have ? std::max(R.validated_until, t_end) : t_end;
  R.max_speed = have ? std::max(R.max_speed, vmax) : vmax;
  return MSRC_OK;
}

// Band-limited knot upsampler (Sec. II-C): kernel h(u) = sinc(u) times a Kaiser
// window of shape 8 over |u| < Q (bessel_i0 above). Row p of a factor-U
// table holds the weights of knots j0 - Q + 1 .. j0 + Q at the point p / U past
// knot j0, normalised to sum 1, then their first moment sum_i w_i (i - Q + 1).
// Returns the largest sum_i |w_i| over the rows (the factor by which an
// interpolated distance can exceed the largest knot distance).
double upsampler_rows(int U, int Q, std::vector<float>& out) {
  const double kShape = 8.0;
  const double i0b = bessel_i0(kShape);
  double l1max = 0.0;
  std::vector<double> w(2 * Q);
  for (int p = 0; p < U; ++p) {
    const double x = double(p) / U;
    double sum = 0.0;
    for (int i = 0; i < 2 * Q; ++i) {
      const double u = x - double(i - Q + 1);
      const double sinc = (u == 0.0) ? 1.0 : std::sin(kPiD * u) / (kPiD * u);
      const double r = u / Q;
      w[i] = sinc * bessel_i0(kShape * std::sqrt(std::max(0.0, 1.0 - r * r))) / i0b;
      sum += w[i];
    }
    double l1 = 0.0, moment = 0.0;
    for (int i = 0; i < 2 * Q; ++i) {
      w[i] /= sum;
      l1 += std::fabs(w[i]);
      moment += w[i] * double(i - Q + 1);
      out.push_back(float(w[i]));
    }
    out.push_back(float(moment));
    l1max = std::max(l1max, l1);
  }
  return l1max;
}

// ---------------------------------------------------------------- planning
inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Plan {
  std::vector<SceneDev> scenes;
  std::vector<int64_t> prefix[kUnitKinds];
  int64_t totals[kUnitKinds] = {};
  int end_bit = kSortGroupShift;
  // byte offsets in the workspace
  size_t off_desc = 0, off_keys_in = 0, off_keys_out = 0, off_vals_in = 0, off_vals_out = 0;
  size_t off_sort = 0, sort_bytes = 0, off_code = 0, off_gain = 0, off_knots = 0;
  size_t off_mcode = 0, off_mgain = 0, off_moff = 0, off_mpos = 0;
  size_t off_z = 0, off_zp = 0, off_part = 0, fwd_bytes = 0, desc_bytes = 0, off_arr = 0, off_xmax = 0;
  // reverse mode
  bool backward = false;
  int cfg = 0;                      // forward tile configuration
  int64_t dxb_floats = 0;
  size_t off_dxb = 0, off_kslot = 0, off_bpart = 0, off_gk = 0, off_ppart = 0, off_bwt = 0, off_trange = 0;
  size_t off_otau = 0, off_ograd = 0, off_cgrad = 0, off_kslot_arr = 0, off_garr = 0;
  int kL = 32;
  int taps = 32;
  // band-limited knot upsampling: weight tables (uploaded to off_upw)
  std::vector<float> upw;
  std::vector<int> upw_key;       // U * 64 + Q of each table
  std::vector<int> upw_at;        // its first float
  std::vector<double> upw_l1;     // its largest absolute row sum
  size_t off_upw = 0, off_bl_tau = 0, off_dense_hi = 0, off_dense_lo = 0, off_knot_hl = 0,
         off_arr_hl = 0;
  // time groups of the forward image order: source position and array
  // displacement at every group's middle (6 doubles each, written by the setup
  // kernels at off_gpos)
  size_t off_gpos = 0;
  int64_t n_sort_groups = 0;
  int max_groups = 1;
};

// Output samples per time group of the forward image order (rounded to whole
// tiles): short enough that a block's images stay close in delay over the
// group, long enough that the extra copies of the image table stay cheap.
constexpr int64_t kTimeGroupSamples = 12288;

// Workspace layout and per-scene descriptors of one call. Forward mode uses
// the selected synthesis tile configuration; reverse mode its own (one sample
// per thread) and adds the gradient buffers.
msrc_status make_plan(const msrc_room_t* rooms, int n, const int64_t* n_in, const int64_t* n_out,
                      Plan& P, bool backward = false, int cfg = 0) {
  if (!rooms || n <= 0 || !n_in || !n_out)
    return fail(MSRC_ERR_INVALID_ARG, "null rooms/lengths or n_rooms <= 0");
  P.backward = backward;
  if (cfg < 0 || cfg >= tile_config_count()) return fail(MSRC_ERR_INVALID_ARG, "tile configuration %d out of range", cfg);
  P.cfg = cfg;
  const TileConfig& tc = backward ? backward_tile_config() : tile_config(cfg);
  const int T = tc.threads * tc.chunks;
  P.scenes.resize(n);
  for (auto& v : P.prefix) v.assign(n + 1, 0);
  int64_t img_acc = 0, knot_acc = 0, z_acc = 0, part_acc = 0, group_acc = 0, master_acc = 0;
  int64_t dxb_acc = 0, kslot_acc = 0, bpart_acc = 0, bl_acc = 0, dense_acc = 0;
  bool any_moving = false;
  for (int s = 0; s < n; ++s) {
    msrc_room* R = rooms[s];
    if (!R) return fail(MSRC_ERR_INVALID_ARG, "room %d is null", s);
    if (!R->has_traj) return fail(MSRC_ERR_STATE, "room %d has no trajectory", s);
    if (n_in[s] <= 0 || n_out[s] <= 0 || n_in[s] > (int64_t(1) << 24) || n_out[s] > (int64_t(1) << 24))
      return fail(MSRC_ERR_INVALID_ARG, "room %d: lengths must be in [1, 2^24]", s);
    if (s > 0) {
      const msrc_room* R0 = rooms[0];
      if (R->d.taps != R0->d.taps || R->d.window != R0->d.window ||
          (R->d.window == 1 && R->d.kaiser_beta != R0->d.kaiser_beta) ||
          (R->d.window == 2 && (R->d.farrow_order != R0->d.farrow_order || R->d.passband != R0->d.passband)))
        return fail(MSRC_ERR_UNSUPPORTED, "rooms in one call must share taps and window");
    }
    SceneDev& S = P.scenes[s];
    std::memset(&S, 0, sizeof(S));
    for (int d = 0; d < 3; ++d) S.dims[d] = R->d.dims[d];
    for (int w = 0; w < 6; ++w) S.beta[w] = R->d.beta[w];
    S.c = R->d.c;
    S.fs = R->d.fs;
    S.duration = R->traj.duration_s;
    for (int m = 0; m < R->n_mics; ++m)
      for (int d = 0; d < 3; ++d) S.mics[m][d] = R->mics[m][d];
    std::memcpy(S.traj, R->traj.params, sizeof(S.traj));
    S.traj_kind = R->traj.kind;
    if (R->traj.kind == 2) spline_segments(R->traj, S.traj_poly);
    S.n_ctrl = R->traj.n_ctrl;
    if (R->arr_moving) {
      S.arr_moving = 1;
      std::memcpy(S.arr_params, R->arr.params, sizeof(S.arr_params));
      S.arr_kind = R->arr.kind;
      S.arr_n_ctrl = R->arr.n_ctrl;
      S.arr_duration = R->arr.duration_s;
      any_moving = true;
    }
    S.K = R->d.max_order;
    S.n_mics = R->n_mics;
    S.n_tiers = R->d.n_tiers;
    S.n_images = int32_t(R->n_images);
    S.n_in = n_in[s];
    S.n_out = n_out[s];
    S.tile = T;
    S.n_tiles = int32_t((n_out[s] + T - 1) / T);
    S.c_over_fs = float(R->d.c / R->d.fs);
    S.fs_over_c = R->d.fs / R->d.c;
    S.fsc = float(S.fs_over_c);
    // double-float pairs v = hi + lo (hi the nearest float, lo the rest)
    auto split = [](double v, float* hl) {
      hl[0] = float(v);
      hl[1] = float(v - double(hl[0]));
    };
    for (int d = 0; d < 3; ++d) split(R->d.dims[d], S.dims_hl[d]);
    for (int m = 0; m < R->n_mics; ++m)
      for (int d = 0; d < 3; ++d) split(R->mics[m][d], S.mics_hl[m][d]);
    split(S.fs_over_c, S.fsc_hl);
    int first = 0, blk = 0;
    int64_t kfirst = 0, bl_units = 0;
    // trajectory range the knots reach, and the bound on an interpolated
    // distance relative to the largest knot distance
    double t_lo = 0.0, t_hi = R->traj.duration_s, l1 = 1.0;
    const int Q = R->up_q;
    S.up_q = Q;
    for (int t = 0; t < S.n_tiers; ++t) {
      const int Nc = R->tier_step[t];
      const int U = R->tier_up[t];
      const bool bl = U > 1;
      const int N = Nc / U;  // record spacing: knots, or virtual knots when upsampled
      S.tier_max_rho[t] = R->d.tier_max_rho[t];
      S.tier_step[t] = N;
      S.tier_coarse[t] = Nc;
      S.tier_up[t] = U;
      S.knot_shift[t] = bl ? Q : 0;
      S.tier_count[t] = int32_t(R->tier_count[t]);
      S.tier_first[t] = first;
      first += S.tier_count[t];
      const int J = int((n_out[s] - 1) / N + 1);
      S.tier_intervals[t] = J;
      // images per block: the item's records (one per image and knot interval
      // touching the tile) must fit the shared record capacity
      // (the forward synthesis and the gradient kernel store them for image
      // pairs: an even count)
      const int rec_per_image = (T - 1) / N + 2;
      // interval records: one float2 per image and interval (a pair takes two
      // images' worth); knot records: one float2 per image pair and knot
      if ((tc.knots ? rec_per_image : 2 * rec_per_image) > tc.reccap)
        return fail(MSRC_ERR_UNSUPPORTED, "tile configuration too small for knot spacing %d", N);
      int B = std::max(1, std::min(tc.block, (tc.knots ? 2 * tc.reccap : tc.reccap) / rec_per_image));
      if (backward) B = std::max(1, std::min(B, int(backward_unit_cap()) / (rec_per_image + 1)));
      if (B > 1) B &= ~1;
      int64_t n_knots = J + 1;
      if (bl) {
        // the upsampler's scratch shares the shared z window (4 floats per column and segment)
        const int nk = rec_per_image + 1;
        const int nj = (nk - 1) / U + 2;
        const int64_t per = bl_scratch_floats(1, nk, nj, Q);
        const int64_t cap = backward ? backward_bl_scratch_floats() : int64_t(kFarrowSegs) * tc.wcap * 4;
        if (per > cap)
          return fail(MSRC_ERR_UNSUPPORTED, "tile configuration too small for the upsampling of tier %d", t);
        B = std::min<int64_t>(B, cap / per);
        if (B > 1) B &= ~1;
        const int key = U * 64 + Q;
        size_t k = 0;
        while (k < P.upw_key.size() && P.upw_key[k] != key) ++k;
        if (k == P.upw_key.size()) {
          P.upw_key.push_back(key);
          P.upw_at.push_back(int(P.upw.size()));
          P.upw_l1.push_back(upsampler_rows(U, Q, P.upw));
        }
        S.upw_base[t] = P.upw_at[k];
        l1 = std::max(l1, P.upw_l1[k]);
        // knots -Q .. J_c + Q, J_c the knot intervals covering the output
        const int64_t Jc = (n_out[s] - 1) / Nc + 1;
        n_knots = Jc + 1 + 2 * Q;
        // k_bl_tau units: (microphone, image) rows of n_knots delays
        S.bl_knots[t] = int32_t(n_knots);
        S.bl_units_first[t] = bl_units;
        S.bl_tau_base[t] = bl_acc;
        bl_units += int64_t(R->n_mics) * R->tier_count[t];
        bl_acc += int64_t(R->n_mics) * R->tier_count[t] * n_knots;
        t_lo = std::min(t_lo, -double(Q) * Nc / R->d.fs);
        t_hi = std::max(t_hi, double(Jc + Q) * Nc / R->d.fs);
      } else {
        t_hi = std::max(t_hi, double(J) * N / R->d.fs);
      }
      S.tier_block_images[t] = B;
      S.tier_blocks[t] = (S.tier_count[t] + B - 1) / B;
      S.block_first[t] = blk;
      blk += S.tier_blocks[t];
      S.knot_base[t] = knot_acc + kfirst;
      S.knot_units_first[t] = kfirst;
      kfirst += n_knots;
    }
    S.n_blocks = blk;
    S.img_base = img_acc;
    S.master_base = master_acc;
    // time groups: one per kTimeGroupSamples of output. Reverse mode keeps one
    // (ordered at the middle of the trajectory) when a tier is band-limited or
    // the delays are emission-time: the per-(mic, image, knot) tables of those
    // tiers are indexed by the first group's image order.
    {
      bool opt_tiers = R->d.delay_model == 1;
      for (int t = 0; t < S.n_tiers; ++t) opt_tiers = opt_tiers || S.tier_up[t] > 1;
      const int tg = int(std::max<int64_t>(1, kTimeGroupSamples / T));
      const bool grouped = !(backward && opt_tiers) && S.n_tiles > tg;
      S.tile_group = grouped ? tg : S.n_tiles;
      S.n_time_groups = grouped ? (S.n_tiles + tg - 1) / tg : 1;
      S.sort_group0 = group_acc;
      S.gpos_base = group_acc;
      group_acc += S.n_time_groups;
      P.max_groups = std::max(P.max_groups, S.n_time_groups);
    }
    if (backward) {
      int groups = 0;
      for (int t = 0; t < S.n_tiers; ++t) {
        // dx items take groups of blocks of one tier (about the same number
        // of images each), so one Farrow correlation serves the whole group;
        // at least two blocks, so that tiers with full 256-image blocks share
        // it between 512 images (the 10 s array scene: 3.08 -> 2.83 s, and
        // half the dx rows)
        S.group_blocks[t] = std::max(2, backward_group_images() / S.tier_block_images[t]);
        S.group_first[t] = groups;
        groups += (S.tier_blocks[t] + S.group_blocks[t] - 1) / S.group_blocks[t];
      }
      S.n_groups = groups;
      int64_t kslot = 0;
      for (int t = 0; t < S.n_tiers; ++t) {
        S.kcap[t] = (T - 1) / S.tier_step[t] + 3;
        S.kslot_first[t] = kslot_acc + kslot;
        kslot += int64_t(S.tier_blocks[t]) * S.n_tiles * S.kcap[t];
      }
      S.kslot_mic_stride = kslot;
      // dx items split the tiles into ranges; a range writes dx columns within
      // [first sample - tau_max - L, last sample + L], so ranges two apart
      // never share a column once a range spans tau_max + 2L samples: ranges
      // of equal parity share one dx row per (mic, group)
      {
        double mL = 0, dg = 0;
        for (int d = 0; d < 3; ++d) { mL = std::max(mL, R->d.dims[d]); dg += R->d.dims[d] * R->d.dims[d]; }
        const double dm = 2.0 * S.K * mL + 2.0 * std::sqrt(dg) + 1.0;
        const int64_t tb = int64_t(std::ceil(dm * R->d.fs / R->d.c)) + 2;
        S.range_tiles = int32_t(std::max<int64_t>(1, (tb + 2 * R->d.taps + 16 + T - 1) / T));
        S.n_ranges = (S.n_tiles + S.range_tiles - 1) / S.range_tiles;
        S.dx_rows = S.n_ranges > 1 ? 2 : 1;
      }
      S.dxb_base = dxb_acc;
      S.bpart_base = bpart_acc;
      kslot_acc += int64_t(S.n_mics) * kslot;
      dxb_acc += int64_t(S.n_mics) * S.n_groups * S.dx_rows * S.n_in;
      bpart_acc += int64_t(S.n_mics) * S.n_blocks * S.n_tiles * 8;
    }
    // z rows cover every read position: n - tau with tau in [0, tau_bound]
    // (an upsampled distance is at most l1 times the largest knot distance)
    double maxL = 0, diag = 0;
    for (int d = 0; d < 3; ++d) { maxL = std::max(maxL, R->d.dims[d]); diag += R->d.dims[d] * R->d.dims[d]; }
    const double dmax = (2.0 * S.K * maxL + 2.0 * std::sqrt(diag) + 1.0) * l1;
    const int64_t tau_bound = int64_t(std::ceil(dmax * R->d.fs / R->d.c)) + 2;
    const int64_t zlo = -tau_bound - 16;
    const int64_t zhi = std::max(n_out[s], n_in[s] + R->d.taps) + 16;
    S.z_m0 = zlo;
    S.z_len = (zhi - zlo + 3) & ~int64_t(3);  // rows start on 16-byte boundaries (bulk copies)
    S.z_base = z_acc;
    S.part_base = part_acc;
    // emission-time delays: the source path table spans the emission times of
    // every knot, [first knot - tau_bound, last knot] with a margin, in steps
    // of 1 / (kDenseOver fs)
    S.delay_model = R->d.delay_model;
    int64_t u_dense = 0;
    if (S.delay_model == 1) {
      for (int t = 0; t < S.n_tiers; ++t)
        if (S.tier_up[t] > 1)
          return fail(MSRC_ERR_UNSUPPORTED,
                      "room %d: emission-time delays need linear knot interpolation (tier %d is upsampled)", s, t);
      const int64_t last = int64_t(std::ceil(t_hi * R->d.fs)) + 4;
      S.dense_k0 = int64_t(kDenseOver) * (-tau_bound - 4);
      S.n_dense = int64_t(kDenseOver) * last - S.dense_k0 + 1;
      S.dense_base = dense_acc;
      dense_acc += S.n_dense;
      u_dense = S.n_dense;
      t_lo = std::min(t_lo, double(S.dense_k0) / (kDenseOver * R->d.fs));
      t_hi = std::max(t_hi, double(last) / R->d.fs);
    }
    // trajectory evaluated at every knot (and every emission time)
    msrc_status vs = validate_traj_range(*R, t_lo, t_hi);
    if (vs != MSRC_OK) return vs;
    // reverse mode scatters one image's samples into shared (segment, column)
    // bins without atomics: below c/2 the read position advances by more than
    // 1/2 sample per output sample, so no two samples of an image share a bin
    if (backward && !(R->max_speed < 0.5 * R->d.c))
      return fail(MSRC_ERR_UNSUPPORTED, "room %d: reverse mode needs source speed below c/2", s);

    const int64_t u_enum = int64_t(S.n_time_groups) * S.n_images;
    const int64_t u_knots = kfirst;
    const int64_t u_rec = backward ? S.n_in : 0;  // reverse mode: dx samples
    const int64_t u_z = (S.z_len + 255) / 256;
    // work items: (microphone, image block, tile); reverse mode adds the dx
    // items (microphone, image block) in the reduction slot
    const int64_t u_item = int64_t(S.n_mics) * S.n_blocks * S.n_tiles;
    const int64_t u_red = backward ? int64_t(S.n_mics) * S.n_groups * S.n_ranges : int64_t(S.n_mics) * S.n_out;
    const int64_t u_bl = bl_units;  // (mic, image) rows of FP64 knot delays of upsampled tiers
    // reverse mode: (mic, image, record knot) units of the tiers whose delays
    // are not linear in the knot positions (upsampled, emission-time)
    int64_t u_opt = 0;
    for (int t = 0; t < S.n_tiers; ++t) {
      S.opt_units_first[t] = u_opt;
      if (backward && (S.delay_model == 1 || S.tier_up[t] > 1))
        u_opt += int64_t(S.n_mics) * S.tier_count[t] * (int64_t(S.tier_intervals[t]) + 1);
    }
    S.n_opt_units = u_opt;
    if (int64_t(S.n_mics) * S.n_blocks * S.n_tiles >= (int64_t(1) << 31))
      return fail(MSRC_ERR_UNSUPPORTED, "room %d: more than 2^31 work items", s);
    const int64_t u[kUnitKinds] = {u_enum, u_knots, u_rec, u_z, u_item, u_red, u_bl, u_dense, S.n_images, u_opt};
    for (int k = 0; k < kUnitKinds; ++k) {
      P.prefix[k][s + 1] = P.prefix[k][s] + u[k];
      P.totals[k] += u[k];
    }
    img_acc += u_enum;
    master_acc += S.n_images;
    knot_acc += kfirst;
    z_acc += int64_t(kFarrowSegs) * S.z_len;
    part_acc += int64_t(S.n_mics) * S.n_blocks * S.n_out;
  }
  P.taps = rooms[0]->d.taps;
  P.kL = rooms[0]->kL;
  P.n_sort_groups = group_acc;
  P.end_bit = kSortGroupShift;
  while ((int64_t(1) << (P.end_bit - kSortGroupShift)) < group_acc) ++P.end_bit;
  if (P.end_bit > 64) return fail(MSRC_ERR_UNSUPPORTED, "too many time groups in one call");
  // workspace layout
  size_t off = 256;  // error word + work counter
  P.desc_bytes = (n > 1) ? n * sizeof(SceneDev) + kUnitKinds * (n + 1) * sizeof(int64_t) : 0;
  P.off_desc = off; off = align256(off + P.desc_bytes);
  const size_t I = size_t(img_acc);
  P.off_keys_in = off; off = align256(off + 8 * I);
  P.off_keys_out = off; off = align256(off + 8 * I);
  P.off_vals_in = off; off = align256(off + 4 * I);
  P.off_vals_out = off; off = align256(off + 4 * I);
  P.sort_bytes = sort_temp_bytes(int64_t(I), P.end_bit);
  P.off_sort = off; off = align256(off + P.sort_bytes);
  P.off_code = off; off = align256(off + 4 * I);
  P.off_mcode = off; off = align256(off + 4 * size_t(master_acc));
  P.off_mgain = off; off = align256(off + 4 * size_t(master_acc));
  P.off_moff = off; off = align256(off + 16 * size_t(master_acc));
  P.off_mpos = off; off = align256(off + 4 * size_t(master_acc));
  P.off_gain = off; off = align256(off + 4 * I);
  P.off_knots = off; off = align256(off + 24 * size_t(knot_acc));
  P.off_arr = off; off = align256(off + (any_moving ? 24 * size_t(knot_acc) : 0));
  P.off_knot_hl = off; off = align256(off + 32 * size_t(knot_acc));
  P.off_arr_hl = off; off = align256(off + (any_moving ? 32 * size_t(knot_acc) : 0));
  P.off_upw = off; off = align256(off + 4 * P.upw.size());
  P.off_gpos = off; off = align256(off + 48 * size_t(group_acc));
  P.off_bl_tau = off; off = align256(off + 8 * size_t(bl_acc));
  P.off_dense_hi = off; off = align256(off + 16 * size_t(dense_acc));
  P.off_dense_lo = off; off = align256(off + 16 * size_t(dense_acc));
  P.off_z = off; off = align256(off + 16 * size_t(z_acc));
  // reverse mode: powers 4..5 of the degree-5 rows the gradient kernel reads
  // (zq holds its powers 0..3; the forward rows are whole in zq)
  // (+64 B: a bulk copy of a row's last columns may read up to 12 B past it)
  P.off_zp = off; off = align256(off + (backward ? 8 * size_t(z_acc) + 64 : 0));
  P.off_xmax = off; off = align256(off + 4 * size_t(n));
  if (!backward) {
    P.off_part = off; off = align256(off + 4 * size_t(part_acc));
  } else {
    P.off_dxb = off; off = align256(off + 4 * size_t(dxb_acc));
    P.dxb_floats = dxb_acc;
    P.off_kslot = off; off = align256(off + 12 * size_t(kslot_acc));
    P.off_bpart = off; off = align256(off + 4 * size_t(bpart_acc));
    P.off_gk = off; off = align256(off + 24 * size_t(knot_acc));
    // moving arrays: the second knot-slot set and knot gradients of dL/da
    P.off_kslot_arr = off; off = align256(off + (any_moving ? 12 * size_t(kslot_acc) : 0));
    P.off_garr = off; off = align256(off + (any_moving ? 24 * size_t(knot_acc) : 0));
    P.off_ppart = off; off = align256(off + 8 * size_t(n) * kParamPartialsPerScene);
    P.off_bwt = off; off = align256(off + 32 * I);
    P.off_trange = off; off = align256(off + 8 * size_t(P.totals[4]));
    P.off_otau = off; off = align256(off + 8 * size_t(P.totals[9]));
    P.off_ograd = off; off = align256(off + 8 * size_t(P.totals[9]));
    P.off_cgrad = off; off = align256(off + 4 * size_t(bl_acc));
  }
  P.fwd_bytes = off;
  if (I > (size_t(1) << 31)) return fail(MSRC_ERR_UNSUPPORTED, "more than 2^31 images in one call");
  return MSRC_OK;
}

void fill_args(const Plan& P, const msrc_room_t* rooms, char* ws, KernelArgs& a) {
  std::memset(&a, 0, sizeof(a));
  a.n_scenes = int32_t(P.scenes.size());
  if (a.n_scenes == 1) a.scene0 = P.scenes[0];
  for (int k = 0; k < kUnitKinds; ++k) a.totals[k] = P.totals[k];
  a.test_extra_tx = g_test_extra_tx;
  a.p.err = reinterpret_cast<uint32_t*>(ws);
  a.p.counter = reinterpret_cast<uint32_t*>(ws + 4);
  a.p.keys_in = reinterpret_cast<uint64_t*>(ws + P.off_keys_in);
  a.p.keys_out = reinterpret_cast<uint64_t*>(ws + P.off_keys_out);
  a.p.vals_in = reinterpret_cast<uint32_t*>(ws + P.off_vals_in);
  a.p.vals_out = reinterpret_cast<uint32_t*>(ws + P.off_vals_out);
  a.p.sort_temp = ws + P.off_sort;
  a.p.sort_temp_bytes = P.sort_bytes;
  a.p.img_code = reinterpret_cast<uint32_t*>(ws + P.off_code);
  a.p.img_gain = reinterpret_cast<float*>(ws + P.off_gain);
  a.p.m_code = reinterpret_cast<uint32_t*>(ws + P.off_mcode);
  a.p.m_gain = reinterpret_cast<float*>(ws + P.off_mgain);
  a.p.m_off = reinterpret_cast<float4*>(ws + P.off_moff);
  a.p.m_pos = reinterpret_cast<int32_t*>(ws + P.off_mpos);
  a.p.knot_pos = reinterpret_cast<double*>(ws + P.off_knots);
  a.p.arr_pos = reinterpret_cast<double*>(ws + P.off_arr);
  a.p.knot_hl = reinterpret_cast<float4*>(ws + P.off_knot_hl);
  a.p.arr_hl = reinterpret_cast<float4*>(ws + P.off_arr_hl);
  a.p.upw = reinterpret_cast<const float*>(ws + P.off_upw);
  a.p.gpos = reinterpret_cast<double*>(ws + P.off_gpos);
  a.n_sort_groups = P.n_sort_groups;
  a.max_time_groups = P.max_groups;
  a.p.bl_tau = reinterpret_cast<float2*>(ws + P.off_bl_tau);
  a.p.dense_hi = reinterpret_cast<float4*>(ws + P.off_dense_hi);
  a.p.dense_lo = reinterpret_cast<float4*>(ws + P.off_dense_lo);
  a.p.zq = reinterpret_cast<float4*>(ws + P.off_z);
  a.p.xmax = reinterpret_cast<uint32_t*>(ws + P.off_xmax);
  a.p.zg = P.backward ? reinterpret_cast<float2*>(ws + P.off_zp) : nullptr;
  a.p.part = reinterpret_cast<float*>(ws + P.off_part);
  if (P.backward) {
    a.p.dxb = reinterpret_cast<float*>(ws + P.off_dxb);
    a.p.dxb_floats = P.dxb_floats;
    a.p.kslot = reinterpret_cast<float*>(ws + P.off_kslot);
    a.p.bpart = reinterpret_cast<float*>(ws + P.off_bpart);
    a.p.gk = reinterpret_cast<double*>(ws + P.off_gk);
    a.p.kslot_arr = reinterpret_cast<float*>(ws + P.off_kslot_arr);
    a.p.garr = reinterpret_cast<double*>(ws + P.off_garr);
    a.p.ppart = reinterpret_cast<double*>(ws + P.off_ppart);
    a.p.bwt = reinterpret_cast<float4*>(ws + P.off_bwt);
    a.p.trange = reinterpret_cast<float2*>(ws + P.off_trange);
    a.p.otau = reinterpret_cast<double*>(ws + P.off_otau);
    a.p.ograd = reinterpret_cast<float2*>(ws + P.off_ograd);
    a.p.cgrad = reinterpret_cast<float*>(ws + P.off_cgrad);
  }
  // device tables: coefficients of the powers of w = v / 2 (c_q 2^q, exact)
  for (int sg = 0; sg < kFarrowSegs; ++sg)
    for (int q = 0; q < kFarrowCoef; ++q)
      for (int k = 0; k < kMaxTaps; ++k) a.farrow[sg][q][k] = std::ldexp(rooms[0]->farrow[sg][q][k], q);
  for (int sg = 0; sg < kFarrowSegs; ++sg)
    for (int q = 0; q < kGradCoef; ++q)
      for (int k = 0; k < kMaxTaps; ++k) a.farrow_g[sg][q][k] = std::ldexp(rooms[0]->farrow_g[sg][q][k], q);
  // bound of |z_3|, |z_4| per unit max |x| (the half-precision scale)
  double zg = 0.0;
  for (int sg = 0; sg < kFarrowSegs; ++sg)
    for (int q = 3; q <= 4; ++q) {
      double l1 = 0.0;
      for (int k = 0; k < kMaxTaps; ++k) l1 += std::fabs(double(a.farrow[sg][q][k]));
      zg = std::max(zg, l1);
    }
  a.zh_gain = float(zg * (1.0 + 1e-6));
  a.taps = P.kL;
  if (a.n_scenes > 1) {
    char* d = ws + P.off_desc;
    a.scenes = reinterpret_cast<const SceneDev*>(d);
    const int64_t* pre = reinterpret_cast<const int64_t*>(d + P.scenes.size() * sizeof(SceneDev));
    const int n1 = a.n_scenes + 1;
    a.tab.enum_prefix = pre;
    a.tab.knots_prefix = pre + n1;
    a.tab.dx_prefix = pre + 2 * n1;
    a.tab.z_prefix = pre + 3 * n1;
    a.tab.item_prefix = pre + 4 * n1;
    a.tab.red_prefix = pre + 5 * n1;
    a.tab.bl_prefix = pre + 6 * n1;
    a.tab.dense_prefix = pre + 7 * n1;
    a.tab.img_prefix = pre + 8 * n1;
    a.tab.opt_prefix = pre + 9 * n1;
  }
}

msrc_status check_ws(const Plan& P, void* ws, size_t bytes) {
  if (!ws) return fail(MSRC_ERR_WORKSPACE, "workspace is null");
  if (reinterpret_cast<uintptr_t>(ws) & 255)
    return fail(MSRC_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < P.fwd_bytes)
    return fail(MSRC_ERR_WORKSPACE, "workspace too small: %zu < %zu bytes", bytes, P.fwd_bytes);
  return MSRC_OK;
}

// Uploads the upsampler weight tables, and the scene descriptors and prefix
// tables of a batched call (pageable sources: each copy returns once its data
// is staged).
msrc_status upload_tables(const Plan& P, char* ws, cudaStream_t st, std::vector<char>& blob) {
  if (!P.upw.empty()) {
    const cudaError_t e =
        cudaMemcpyAsync(ws + P.off_upw, P.upw.data(), 4 * P.upw.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "upsampler table upload");
  }
  if (P.scenes.size() <= 1) return MSRC_OK;
  blob.resize(P.desc_bytes);
  std::memcpy(blob.data(), P.scenes.data(), P.scenes.size() * sizeof(SceneDev));
  int64_t* pre = reinterpret_cast<int64_t*>(blob.data() + P.scenes.size() * sizeof(SceneDev));
  const size_t n1 = P.scenes.size() + 1;
  for (int k = 0; k < kUnitKinds; ++k) std::memcpy(pre + k * n1, P.prefix[k].data(), n1 * sizeof(int64_t));
  cudaError_t e = cudaMemcpyAsync(ws + P.off_desc, blob.data(), P.desc_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "descriptor upload");
  return MSRC_OK;
}

msrc_status run_forward(const msrc_room_t* rooms, int32_t n, const float* const* x_dev,
                        const int64_t* n_in, float* const* y_dev, const int64_t* n_out,
                        void* ws, size_t ws_bytes, cudaStream_t st, int cfg) {
  if (!x_dev || !y_dev) return fail(MSRC_ERR_INVALID_ARG, "null signal pointer array");
  Plan P;
  msrc_status s = make_plan(rooms, n, n_in, n_out, P, false, cfg);
  if (s != MSRC_OK) return s;
  s = check_ws(P, ws, ws_bytes);
  if (s != MSRC_OK) return s;
  for (int r = 0; r < n; ++r) {
    if (!x_dev[r] || !y_dev[r]) return fail(MSRC_ERR_INVALID_ARG, "room %d: null x or y", r);
    if ((reinterpret_cast<uintptr_t>(x_dev[r]) | reinterpret_cast<uintptr_t>(y_dev[r])) & 15)
      return fail(MSRC_ERR_INVALID_ARG, "room %d: x and y must be 16-byte aligned", r);
    P.scenes[r].x = x_dev[r];
    P.scenes[r].y = y_dev[r];
  }
  char* w = static_cast<char*>(ws);
  KernelArgs* a = new (std::nothrow) KernelArgs;
  if (!a) return fail(MSRC_ERR_INVALID_ARG, "out of host memory");
  fill_args(P, rooms, w, *a);
  std::vector<char> blob;
  cudaError_t e = cudaMemsetAsync(w, 0, 256, st);
  if (e != cudaSuccess) { delete a; return cuda_fail(e, "workspace header clear"); }
  s = upload_tables(P, w, st, blob);
  if (s != MSRC_OK) { delete a; return s; }
  cudaEvent_t* ev = nullptr;
  if (g_prof.on) {
    ev = g_prof.ev[g_prof.next];
    g_prof.next = (g_prof.next + 1) % kProfSets;
    g_prof.pending = std::min(g_prof.pending + 1, kProfSets);
    cudaEventRecord(ev[0], st);
  }
  e = launch_setup(*a, st);
  if (ev) cudaEventRecord(ev[1], st);
  if (e == cudaSuccess) e = launch_forward(*a, P.cfg, st, ev ? ev + 2 : nullptr);
  if (ev) cudaEventRecord(ev[4], st);
  delete a;
  if (e != cudaSuccess) return cuda_fail(e, "synthesis launch");
  return MSRC_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

msrc_status msrc_create_room(const msrc_room_desc* desc, msrc_room_t* out) {
  if (!desc || !out) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const msrc_room_desc& d = *desc;
  for (int k = 0; k < 3; ++k)
    if (!(d.dims[k] > 0.0) || !std::isfinite(d.dims[k]))
      return fail(MSRC_ERR_INVALID_ARG, "room dimension %d must be positive and finite", k);
  for (int w = 0; w < 6; ++w)
    if (!(d.beta[w] >= 0.0 && d.beta[w] <= 1.0))
      return fail(MSRC_ERR_INVALID_ARG, "reflection coefficient %d must be in [0, 1]", w);
  if (!(d.c > 0.0) || !std::isfinite(d.c)) return fail(MSRC_ERR_INVALID_ARG, "c must be positive");
  if (!(d.fs > 0.0) || !std::isfinite(d.fs)) return fail(MSRC_ERR_INVALID_ARG, "fs must be positive");
  if (d.max_order < 0 || d.max_order > MSRC_MAX_ORDER)
    return fail(MSRC_ERR_INVALID_ARG, "max_order must be in [0, %d]", MSRC_MAX_ORDER);
  if (d.n_tiers < 1 || d.n_tiers > MSRC_MAX_TIERS)
    return fail(MSRC_ERR_INVALID_ARG, "n_tiers must be in [1, %d]", MSRC_MAX_TIERS);
  if (d.taps < 8 || d.taps > kMaxTaps || (d.taps & 1))
    return fail(MSRC_ERR_INVALID_ARG, "taps must be even and in [8, %d]", kMaxTaps);
  if (d.window < 0 || d.window > 2) return fail(MSRC_ERR_INVALID_ARG, "window must be 0, 1 or 2");
  if (d.window == 1 && !(d.kaiser_beta >= 0.0 && d.kaiser_beta <= 20.0))
    return fail(MSRC_ERR_INVALID_ARG, "kaiser_beta must be in [0, 20]");
  if (d.window == 2 && (d.farrow_order < 1 || d.farrow_order > kFarrowDeg))
    return fail(MSRC_ERR_INVALID_ARG, "farrow_order must be in [1, %d]", kFarrowDeg);
  if (d.window == 2 && !(d.passband >= 0.05 && d.passband <= 0.98))
    return fail(MSRC_ERR_INVALID_ARG, "passband must be in [0.05, 0.98]");
  if (d.delay_model < 0 || d.delay_model > 1) return fail(MSRC_ERR_INVALID_ARG, "delay_model must be 0 or 1");
  if (d.upsample_halfwidth < 0 || d.upsample_halfwidth > kMaxUpHalfwidth)
    return fail(MSRC_ERR_INVALID_ARG, "upsample_halfwidth must be in [0, %d]", kMaxUpHalfwidth);
  msrc_room* R = new (std::nothrow) msrc_room;
  if (!R) return fail(MSRC_ERR_INVALID_ARG, "out of host memory");
  std::memset(R, 0, sizeof(*R));
  R->d = d;
  R->up_q = d.upsample_halfwidth > 0 ? d.upsample_halfwidth : 4;
  for (int t = 0; t < d.n_tiers; ++t) {
    const double rate = d.tier_rate_hz[t];
    if (!(rate > 0.0) || rate > d.fs) { delete R; return fail(MSRC_ERR_INVALID_ARG, "tier %d rate must be in (0, fs]", t); }
    const double ratio = d.fs / rate;
    const double rr = std::round(ratio);
    if (std::fabs(ratio - rr) > 1e-9 * ratio || rr < 1 || rr > (1 << 20)) {
      delete R;
      return fail(MSRC_ERR_INVALID_ARG, "tier %d: fs / rate must be an integer (got %.6f)", t, ratio);
    }
    R->tier_step[t] = int32_t(rr);
    const int32_t U = d.tier_upsample[t];
    if (U < 0 || U > kMaxUpsample || (U > 1 && R->tier_step[t] % U != 0)) {
      delete R;
      return fail(MSRC_ERR_INVALID_ARG, "tier %d: tier_upsample must be in [0, %d] and divide fs / rate",
                  t, kMaxUpsample);
    }
    R->tier_up[t] = U > 1 ? U : 1;
    if (t > 0 && d.tier_max_rho[t] < d.tier_max_rho[t - 1] && t < d.n_tiers - 1) {
      delete R;
      return fail(MSRC_ERR_INVALID_ARG, "tier_max_rho must be non-decreasing");
    }
  }
  R->kL = d.taps <= 16 ? 16 : (d.taps <= 32 ? 32 : 64);
  if (d.window == 2 && !gls_design(d.taps, d.farrow_order, d.passband, R->gls)) {
    delete R;
    return fail(MSRC_ERR_UNSUPPORTED, "least-squares Farrow design failed (singular normal equations)");
  }
  count_tiers(*R);
  R->fit_error = fit_farrow(*R, kFarrowCoef, &R->farrow[0][0][0]);
  R->fit_error_g = fit_farrow(*R, kGradCoef, &R->farrow_g[0][0][0]);
  // worst error of one tap weight; the output error is several times smaller
  // (errors of different taps and images do not align): 4e-6 keeps it well
  // inside the 1e-5 relative budget for every window the description admits
  if (R->fit_error > 4e-6) {
    const double err = R->fit_error;
    delete R;
    return fail(MSRC_ERR_UNSUPPORTED, "Farrow fit error %.3g exceeds 4e-6 for this window", err);
  }
  *out = R;
  return MSRC_OK;
}

msrc_status msrc_destroy_room(msrc_room_t room) {
  delete room;
  return MSRC_OK;
}

namespace {
msrc_status check_traj_params(const msrc_traj_desc* traj) {
  if (!(traj->duration_s > 0.0) || !std::isfinite(traj->duration_s))
    return fail(MSRC_ERR_INVALID_ARG, "duration must be positive");
  for (int i = 0; i < 48; ++i)
    if (!std::isfinite(traj->params[i])) return fail(MSRC_ERR_INVALID_ARG, "non-finite trajectory parameter");
  if (traj->kind == 0) {
    const double* p = traj->params;
    if (!(p[3] * p[3] + p[4] * p[4] + p[5] * p[5] > 0.0))
      return fail(MSRC_ERR_INVALID_ARG, "line direction must be non-zero");
  } else if (traj->kind == 1) {
    if (!(traj->params[3] > 0.0)) return fail(MSRC_ERR_INVALID_ARG, "circle radius must be positive");
  } else if (traj->kind == 2) {
    if (traj->n_ctrl < 4 || traj->n_ctrl > MSRC_MAX_CTRL)
      return fail(MSRC_ERR_INVALID_ARG, "spline needs 4..%d control points", MSRC_MAX_CTRL);
  } else {
    return fail(MSRC_ERR_INVALID_ARG, "unknown trajectory kind %d", traj->kind);
  }
  return MSRC_OK;
}
}  // namespace

msrc_status msrc_set_trajectory(msrc_room_t room, const msrc_traj_desc* traj, const double* mics,
                                int32_t n_mics) {
  if (!room || !traj || !mics) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  if (n_mics < 1 || n_mics > MSRC_MAX_MICS)
    return fail(MSRC_ERR_INVALID_ARG, "n_mics must be in [1, %d]", MSRC_MAX_MICS);
  const msrc_status ps = check_traj_params(traj);
  if (ps != MSRC_OK) return ps;
  for (int m = 0; m < n_mics; ++m)
    for (int d = 0; d < 3; ++d) {
      const double v = mics[3 * m + d];
      if (!(v > 0.0 && v < room->d.dims[d]))
        return fail(MSRC_ERR_INVALID_ARG, "microphone %d is not strictly inside the room", m);
    }
  msrc_room saved = *room;
  room->traj = *traj;
  room->n_mics = n_mics;
  for (int m = 0; m < n_mics; ++m)
    for (int d = 0; d < 3; ++d) room->mics[m][d] = mics[3 * m + d];
  room->validated_from = 0.0;
  room->validated_until = -1.0;
  room->max_speed = 0.0;
  room->has_traj = true;
  msrc_status s = validate_traj_range(*room, 0.0, traj->duration_s);
  if (s != MSRC_OK) {
    *room = saved;
    return s;
  }
  return MSRC_OK;
}

msrc_status msrc_trajectory_positions(msrc_room_t room, const double* times, int64_t n_times, double* out) {
  if (!room || (n_times > 0 && (!times || !out)) || n_times < 0) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  if (!room->has_traj) return fail(MSRC_ERR_STATE, "room has no trajectory");
  for (int64_t i = 0; i < n_times; ++i) host_source(room->traj, times[i], out + 3 * i);
  return MSRC_OK;
}

msrc_status msrc_suggest_knot_rates(msrc_room_t room, double tol_samples, int32_t max_step, double* rates_hz) {
  if (!room || !rates_hz) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  if (!(tol_samples > 0.0) || max_step < 1) return fail(MSRC_ERR_INVALID_ARG, "need tol_samples > 0 and max_step >= 1");
  if (!room->has_traj) return fail(MSRC_ERR_STATE, "room has no trajectory");
  const msrc_room& R = *room;
  const double T = R.traj.duration_s, fs = R.d.fs, c = R.d.c;
  // motion bounds between coarse grid points from second differences on a 1 ms grid
  constexpr int kGrid = 256;
  const double hs = 1e-3;
  const long fine = std::max(2L, long(std::ceil(T / hs)));
  std::vector<double> vmax(kGrid, 0.0), amax(kGrid, 0.0);
  auto pos = [&](double t, double out[3]) {
    host_source(R.traj, t, out);
    if (R.arr_moving) {
      double a0[3], at[3];
      host_source(R.arr, 0.0, a0);
      host_source(R.arr, t, at);
      for (int d = 0; d < 3; ++d) out[d + 3] = at[d] - a0[d];
    } else {
      out[3] = out[4] = out[5] = 0.0;
    }
  };
  double vall = 0.0;
  for (long i = 0; i <= fine; ++i) {
    // interior points only: the clamped spline's end kinks are knots (t = 0) or past the bound
    const double t = std::min(std::max(i * T / fine, 0.5 * hs), T - 0.5 * hs);
    const double e = std::min(0.25 * hs, 0.5 * std::min(t, T - t));
    double p0[6], pm[6], pp[6];
    pos(t, p0);
    pos(t - e, pm);
    pos(t + e, pp);
    double vs = 0, vm = 0, as = 0, am = 0;
    for (int d = 0; d < 3; ++d) {
      vs += std::pow((pp[d] - pm[d]) / (2 * e), 2);
      vm += std::pow((pp[d + 3] - pm[d + 3]) / (2 * e), 2);
      as += std::pow((pp[d] - 2 * p0[d] + pm[d]) / (e * e), 2);
      am += std::pow((pp[d + 3] - 2 * p0[d + 3] + pm[d + 3]) / (e * e), 2);
    }
    const double v = std::sqrt(vs) + std::sqrt(vm), a = std::sqrt(as) + std::sqrt(am);
    const int g = std::min(kGrid - 1, int(double(i) / fine * kGrid));
    vmax[g] = std::max(vmax[g], v);
    amax[g] = std::max(amax[g], a);
    vall = std::max(vall, v);
  }
  // smallest image distance of each tier at the coarse grid points
  std::vector<double> dmin(size_t(R.d.n_tiers) * (kGrid + 1), 1e300);
  std::vector<double> src(3 * (kGrid + 1)), mic(3 * (kGrid + 1));
  for (int gi = 0; gi <= kGrid; ++gi) {
    double q[6];
    pos(T * gi / kGrid, q);
    for (int d = 0; d < 3; ++d) src[3 * gi + d] = q[d];
    for (int d = 0; d < 3; ++d) mic[3 * gi + d] = q[d + 3];
  }
  const int K = R.d.max_order;
  for (int nx = -K; nx <= K; ++nx)
    for (int ny = -K; ny <= K; ++ny)
      for (int nz = -K; nz <= K; ++nz) {
        if (std::abs(nx) + std::abs(ny) + std::abs(nz) > K) continue;
        const int n[3] = {nx, ny, nz};
        for (int pb = 0; pb < 8; ++pb) {
          int rho = 0;
          double sg[3], off[3];
          for (int d = 0; d < 3; ++d) {
            const int p = (pb >> d) & 1;
            rho += std::abs(2 * n[d] - p);
            sg[d] = 1.0 - 2.0 * p;
            off[d] = 2.0 * n[d] * R.d.dims[d];
          }
          double* dm = dmin.data() + size_t(tier_of(R.d, rho)) * (kGrid + 1);
          for (int m = 0; m < R.n_mics; ++m)
            for (int gi = 0; gi <= kGrid; ++gi) {
              double acc = 0.0;
              for (int d = 0; d < 3; ++d) {
                const double v = sg[d] * src[3 * gi + d] + off[d] - (R.mics[m][d] + mic[3 * gi + d]);
                acc += v * v;
              }
              dm[gi] = std::min(dm[gi], std::sqrt(acc));
            }
        }
      }
  for (int t = 0; t < R.d.n_tiers; ++t) {
    const double* dm = dmin.data() + size_t(t) * (kGrid + 1);
    double D2 = 0.0;
    for (int g = 0; g < kGrid; ++g) {
      if (dm[g] > 1e299) continue;  // empty tier
      const double dlo = std::max(0.05, std::min(dm[g], dm[g + 1]) - 0.5 * vall * T / kGrid);
      D2 = std::max(D2, vmax[g] * vmax[g] / dlo + amax[g]);
    }
    D2 *= 1.25;
    double Nb = double(max_step);
    if (D2 > 0.0) Nb = std::min(Nb, std::floor(std::sqrt(8.0 * tol_samples * c * fs / D2)));
    long N = std::max(1L, long(Nb));
    // a clamped spline stops at its end: with N dividing the path's length in
    // samples that end is a knot, so no interval straddles its kink
    long len = 0;
    if (R.traj.kind == 2) len = std::llround(T * fs);
    if (R.arr_moving && R.arr.kind == 2) {
      const long la = std::llround(R.arr.duration_s * fs);
      len = len ? std::gcd(len, la) : la;
    }
    if (len > 0)
      while (N > 1 && len % N != 0) --N;
    rates_hz[t] = fs / double(N);
  }
  return MSRC_OK;
}

msrc_status msrc_suggest_bandlimited_rates(msrc_room_t room, double tol_samples, double* rates_hz) {
  if (!room || !rates_hz) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  if (!(tol_samples > 0.0)) return fail(MSRC_ERR_INVALID_ARG, "need tol_samples > 0");
  if (!room->has_traj) return fail(MSRC_ERR_STATE, "room has no trajectory");
  const msrc_room& R = *room;
  const double T = R.traj.duration_s, fs = R.d.fs, fs_c = R.d.fs / R.d.c;
  const int Q = R.up_q;
  // microphone 0 (carried by the array) and the source at time t
  auto geometry = [&](double t, double s[3], double m[3]) {
    host_source(R.traj, t, s);
    double a0[3] = {0, 0, 0}, at[3] = {0, 0, 0};
    if (R.arr_moving) {
      host_source(R.arr, 0.0, a0);
      host_source(R.arr, t, at);
    }
    for (int d = 0; d < 3; ++d) m[d] = R.mics[0][d] + at[d] - a0[d];
  };
  struct Img { double dist; int n[3], p[3]; };
  auto distance = [&](const Img& c, double t) {
    double s[3], m[3];
    geometry(t, s, m);
    double acc = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double v = (1.0 - 2.0 * c.p[d]) * s[d] + 2.0 * c.n[d] * R.d.dims[d] - m[d];
      acc += v * v;
    }
    return std::sqrt(acc);
  };
  // the tier's four nearest images at mid-duration
  std::vector<std::vector<Img>> near(R.d.n_tiers);
  const int K = R.d.max_order;
  for (int nx = -K; nx <= K; ++nx)
    for (int ny = -K; ny <= K; ++ny)
      for (int nz = -K; nz <= K; ++nz) {
        if (std::abs(nx) + std::abs(ny) + std::abs(nz) > K) continue;
        for (int pb = 0; pb < 8; ++pb) {
          Img c{0.0, {nx, ny, nz}, {pb & 1, (pb >> 1) & 1, (pb >> 2) & 1}};
          int rho = 0;
          for (int d = 0; d < 3; ++d) rho += std::abs(2 * c.n[d] - c.p[d]);
          c.dist = distance(c, 0.5 * T);
          auto& v = near[tier_of(R.d, rho)];
          v.push_back(c);
          std::sort(v.begin(), v.end(), [](const Img& x, const Img& y) { return x.dist < y.dist; });
          if (v.size() > 4) v.pop_back();
        }
      }
  // the kernel's weights at 16 points per knot interval
  constexpr int kPts = 16;
  std::vector<float> wt;
  upsampler_rows(kPts, Q, wt);
  for (int t = 0; t < R.d.n_tiers; ++t) {
    double chosen = fs;
    std::vector<double> dk;
    for (double rate = std::max(0.5, 1.0 / T);; rate *= 1.25) {
      const double Nc = std::max(1.0, std::floor(fs / rate));
      const double h = Nc / fs;  // knot spacing (s)
      const int J = int(std::ceil(T / h));
      double worst = 0.0;
      for (const Img& c : near[t]) {
        dk.resize(J + 1 + 2 * Q);
        for (int j = -Q; j <= J + Q; ++j) dk[j + Q] = distance(c, j * h);
        for (int j = 0; j < J; ++j)
          for (int p = 0; p < kPts; ++p) {
            const float* w = &wt[p * (2 * Q + 1)];
            double acc = 0.0;
            for (int i = 0; i < 2 * Q; ++i) acc += double(w[i]) * dk[j - Q + 1 + i + Q];
            const double tt = (j + double(p) / kPts) * h;
            if (tt > T) break;
            worst = std::max(worst, std::fabs(acc - distance(c, tt)));
          }
      }
      if (worst * fs_c <= tol_samples || Nc <= 1.0) {
        chosen = fs / Nc;
        break;
      }
    }
    rates_hz[t] = chosen;
  }
  return MSRC_OK;
}

msrc_status msrc_set_array_trajectory(msrc_room_t room, const msrc_traj_desc* traj) {
  if (!room) return fail(MSRC_ERR_INVALID_ARG, "null room");
  msrc_room saved = *room;
  if (!traj) {
    room->arr_moving = false;
  } else {
    const msrc_status ps = check_traj_params(traj);
    if (ps != MSRC_OK) return ps;
    room->arr_moving = true;
    room->arr = *traj;
  }
  room->validated_from = 0.0;
  room->validated_until = -1.0;
  room->max_speed = 0.0;
  if (room->has_traj) {
    msrc_status s = validate_traj_range(*room, 0.0, room->traj.duration_s);
    if (s != MSRC_OK) {
      *room = saved;
      return s;
    }
  }
  return MSRC_OK;
}

msrc_status msrc_set_reflection(msrc_room_t room, const double* beta) {
  if (!room || !beta) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  for (int w = 0; w < 6; ++w)
    if (!(beta[w] >= 0.0 && beta[w] <= 1.0))
      return fail(MSRC_ERR_INVALID_ARG, "reflection coefficient %d must be in [0, 1]", w);
  for (int w = 0; w < 6; ++w) room->d.beta[w] = beta[w];
  return MSRC_OK;
}

msrc_status msrc_workspace_size(const msrc_room_t* rooms, int32_t n_rooms, const int64_t* n_in,
                                const int64_t* n_out, size_t* fwd_bytes, size_t* bwd_bytes) {
  return msrc_workspace_size_cfg(rooms, n_rooms, n_in, n_out, MSRC_TILE_DEFAULT, fwd_bytes, bwd_bytes);
}

msrc_status msrc_workspace_size_cfg(const msrc_room_t* rooms, int32_t n_rooms, const int64_t* n_in,
                                    const int64_t* n_out, int32_t tile_config, size_t* fwd_bytes,
                                    size_t* bwd_bytes) {
  Plan P;
  msrc_status s = make_plan(rooms, n_rooms, n_in, n_out, P, false, call_config(tile_config, rooms, n_rooms));
  if (s != MSRC_OK) return s;
  if (fwd_bytes) *fwd_bytes = P.fwd_bytes;
  if (bwd_bytes) {
    Plan B;
    s = make_plan(rooms, n_rooms, n_in, n_out, B, true);
    if (s != MSRC_OK) return s;
    *bwd_bytes = B.fwd_bytes;
  }
  return MSRC_OK;
}

msrc_status msrc_synthesize(const msrc_room_t* rooms, int32_t n_rooms, const float* const* x_dev,
                            const int64_t* n_in, float* const* y_dev, const int64_t* n_out,
                            void* ws, size_t ws_bytes, void* stream) {
  return run_forward(rooms, n_rooms, x_dev, n_in, y_dev, n_out, ws, ws_bytes,
                     static_cast<cudaStream_t>(stream), call_config(MSRC_TILE_DEFAULT, rooms, n_rooms));
}

msrc_status msrc_synthesize_cfg(const msrc_room_t* rooms, int32_t n_rooms, const float* const* x_dev,
                                const int64_t* n_in, float* const* y_dev, const int64_t* n_out,
                                int32_t tile_config, void* ws, size_t ws_bytes, void* stream) {
  return run_forward(rooms, n_rooms, x_dev, n_in, y_dev, n_out, ws, ws_bytes,
                     static_cast<cudaStream_t>(stream), call_config(tile_config, rooms, n_rooms));
}

msrc_status msrc_host_io_bytes(const msrc_room_t* rooms, int32_t n_rooms, const int64_t* n_in,
                               const int64_t* n_out, size_t* bytes) {
  if (!rooms || !n_in || !n_out || !bytes || n_rooms <= 0) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  size_t b = 0;
  for (int r = 0; r < n_rooms; ++r) {
    if (!rooms[r]) return fail(MSRC_ERR_INVALID_ARG, "room %d is null", r);
    b += align256(4 * size_t(n_in[r])) + align256(4 * size_t(n_out[r]) * size_t(rooms[r]->n_mics));
  }
  *bytes = b;
  return MSRC_OK;
}

msrc_status msrc_synthesize_host(const msrc_room_t* rooms, int32_t n_rooms, const float* const* x_host,
                                 const int64_t* n_in, float* const* y_host, const int64_t* n_out,
                                 void* ws, size_t ws_bytes, void* stream) {
  if (!x_host || !y_host) return fail(MSRC_ERR_INVALID_ARG, "null host signal array");
  const int cfg = call_config(MSRC_TILE_DEFAULT, rooms, n_rooms);
  Plan P;
  msrc_status s = make_plan(rooms, n_rooms, n_in, n_out, P, false, cfg);
  if (s != MSRC_OK) return s;
  size_t io = 0;
  s = msrc_host_io_bytes(rooms, n_rooms, n_in, n_out, &io);
  if (s != MSRC_OK) return s;
  if (ws_bytes < P.fwd_bytes + io)
    return fail(MSRC_ERR_WORKSPACE, "workspace too small for host I/O: %zu < %zu", ws_bytes, P.fwd_bytes + io);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws) + P.fwd_bytes;
  std::vector<const float*> xd(n_rooms);
  std::vector<float*> yd(n_rooms);
  size_t off = 0;
  for (int r = 0; r < n_rooms; ++r) {
    if (!x_host[r] || !y_host[r]) return fail(MSRC_ERR_INVALID_ARG, "room %d: null host buffer", r);
    float* xdev = reinterpret_cast<float*>(base + off);
    off += align256(4 * size_t(n_in[r]));
    float* ydev = reinterpret_cast<float*>(base + off);
    off += align256(4 * size_t(n_out[r]) * size_t(rooms[r]->n_mics));
    cudaError_t e = cudaMemcpyAsync(xdev, x_host[r], 4 * size_t(n_in[r]), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    xd[r] = xdev;
    yd[r] = ydev;
  }
  s = run_forward(rooms, n_rooms, xd.data(), n_in, yd.data(), n_out, ws, P.fwd_bytes, st, cfg);
  if (s != MSRC_OK) return s;
  for (int r = 0; r < n_rooms; ++r) {
    cudaError_t e = cudaMemcpyAsync(y_host[r], yd[r], 4 * size_t(n_out[r]) * size_t(rooms[r]->n_mics),
                                    cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
  }
  return MSRC_OK;
}

msrc_status msrc_synthesize_backward(const msrc_room_t* rooms, int32_t n_rooms, const float* const* x_dev,
                                     const int64_t* n_in, const float* const* dy_dev, const int64_t* n_out,
                                     float* const* dx_dev, double* const* dparams_dev,
                                     double* const* dbeta_dev, void* ws, size_t ws_bytes, void* stream) {
  return msrc_synthesize_backward_ex(rooms, n_rooms, x_dev, n_in, dy_dev, n_out, dx_dev, dparams_dev, dbeta_dev,
                                     nullptr, ws, ws_bytes, stream);
}

msrc_status msrc_synthesize_backward_ex(const msrc_room_t* rooms, int32_t n_rooms, const float* const* x_dev,
                                        const int64_t* n_in, const float* const* dy_dev, const int64_t* n_out,
                                        float* const* dx_dev, double* const* dparams_dev,
                                        double* const* dbeta_dev, double* const* darray_dev, void* ws,
                                        size_t ws_bytes, void* stream) {
  if (!x_dev || !dy_dev) return fail(MSRC_ERR_INVALID_ARG, "null signal pointer array");
  Plan P;
  msrc_status s = make_plan(rooms, n_rooms, n_in, n_out, P, true);
  if (s != MSRC_OK) return s;
  s = check_ws(P, ws, ws_bytes);
  if (s != MSRC_OK) return s;
  for (int r = 0; r < n_rooms; ++r) {
    if (!x_dev[r] || !dy_dev[r]) return fail(MSRC_ERR_INVALID_ARG, "room %d: null x or dy", r);
    P.scenes[r].x = x_dev[r];
    P.scenes[r].dy = dy_dev[r];
    P.scenes[r].dx = dx_dev ? dx_dev[r] : nullptr;
    P.scenes[r].dparams = dparams_dev ? dparams_dev[r] : nullptr;
    P.scenes[r].dbeta = dbeta_dev ? dbeta_dev[r] : nullptr;
    // dL/d(array trajectory): computed for rooms with a moving array, zero otherwise
    P.scenes[r].darray = (darray_dev && P.scenes[r].arr_moving) ? darray_dev[r] : nullptr;
  }
  char* w = static_cast<char*>(ws);
  KernelArgs* a = new (std::nothrow) KernelArgs;
  if (!a) return fail(MSRC_ERR_INVALID_ARG, "out of host memory");
  fill_args(P, rooms, w, *a);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<char> blob;
  cudaError_t e = cudaMemsetAsync(w, 0, 256, st);
  if (e != cudaSuccess) { delete a; return cuda_fail(e, "workspace header clear"); }
  for (int r = 0; r < n_rooms; ++r) {
    if (P.scenes[r].darray) a->want_array = 1;
    if (darray_dev && darray_dev[r] && !P.scenes[r].darray) {  // a still array: zero gradient
      e = cudaMemsetAsync(darray_dev[r], 0, 48 * sizeof(double), st);
      if (e != cudaSuccess) { delete a; return cuda_fail(e, "array gradient clear"); }
    }
  }
  s = upload_tables(P, w, st, blob);
  if (s != MSRC_OK) { delete a; return s; }
  e = launch_setup(*a, st);
  if (e == cudaSuccess) e = launch_backward_kernels(*a, st);
  delete a;
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  return MSRC_OK;
}

}  // extern "C"

struct msrc_batch {
  Plan P;
  KernelArgs* a = nullptr;
  int cfg = 0;
  char* ws = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {
cudaError_t enqueue_forward(const KernelArgs& a, char* ws, int cfg, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ws, 0, 256, st);
  if (e == cudaSuccess) e = launch_setup(a, st);
  if (e == cudaSuccess) e = launch_forward(a, cfg, st, nullptr);
  return e;
}
}  // namespace

extern "C" {

msrc_status msrc_batch_create(const msrc_room_t* rooms, int32_t n, const float* const* x_dev,
                              const int64_t* n_in, float* const* y_dev, const int64_t* n_out, void* ws,
                              size_t ws_bytes, void* stream, msrc_batch_t* out) {
  return msrc_batch_create_cfg(rooms, n, x_dev, n_in, y_dev, n_out, MSRC_TILE_DEFAULT, ws, ws_bytes, stream, out);
}

msrc_status msrc_batch_create_cfg(const msrc_room_t* rooms, int32_t n, const float* const* x_dev,
                                  const int64_t* n_in, float* const* y_dev, const int64_t* n_out,
                                  int32_t tile_config, void* ws, size_t ws_bytes, void* stream,
                                  msrc_batch_t* out) {
  if (!out || !x_dev || !y_dev) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  msrc_batch* b = new (std::nothrow) msrc_batch;
  if (!b) return fail(MSRC_ERR_INVALID_ARG, "out of host memory");
  msrc_status s = make_plan(rooms, n, n_in, n_out, b->P, false, call_config(tile_config, rooms, n));
  if (s == MSRC_OK) s = check_ws(b->P, ws, ws_bytes);
  if (s != MSRC_OK) { delete b; return s; }
  for (int r = 0; r < n; ++r) {
    if (!x_dev[r] || !y_dev[r]) { delete b; return fail(MSRC_ERR_INVALID_ARG, "room %d: null x or y", r); }
    b->P.scenes[r].x = x_dev[r];
    b->P.scenes[r].y = y_dev[r];
  }
  b->a = new (std::nothrow) KernelArgs;
  if (!b->a) { delete b; return fail(MSRC_ERR_INVALID_ARG, "out of host memory"); }
  b->ws = static_cast<char*>(ws);
  b->cfg = b->P.cfg;
  fill_args(b->P, rooms, b->ws, *b->a);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<char> blob;
  s = upload_tables(b->P, b->ws, st, blob);
  if (s == MSRC_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "descriptor upload");
  }
  if (s != MSRC_OK) { delete b->a; delete b; return s; }
  *out = b;
  return MSRC_OK;
}

msrc_status msrc_batch_run(msrc_batch_t b, int32_t use_graph, void* stream) {
  if (!b) return fail(MSRC_ERR_INVALID_ARG, "null batch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!use_graph) {
    cudaError_t e = enqueue_forward(*b->a, b->ws, b->cfg, st);
    return e == cudaSuccess ? MSRC_OK : cuda_fail(e, "batch launch");
  }
  if (!b->exec) {
    if (st == nullptr) return fail(MSRC_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    // warm-up outside the capture: first launches set kernel attributes
    cudaError_t e = enqueue_forward(*b->a, b->ws, b->cfg, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture begin");
    cudaError_t le = enqueue_forward(*b->a, b->ws, b->cfg, st);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(le != cudaSuccess ? le : e, "graph capture");
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); b->exec = nullptr; return cuda_fail(e, "graph instantiate"); }
    b->graph = g;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, st);
  return e == cudaSuccess ? MSRC_OK : cuda_fail(e, "graph launch");
}

msrc_status msrc_batch_destroy(msrc_batch_t b) {
  if (!b) return MSRC_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b->a;
  delete b;
  return MSRC_OK;
}

msrc_status msrc_autotune(const msrc_room_t* rooms, int32_t n, const float* const* x_dev, const int64_t* n_in,
                          float* const* y_dev, const int64_t* n_out, void* ws, size_t ws_bytes, void* stream,
                          int32_t reps, double* ms, int32_t* best) {
  if (!ms || !best || reps < 1) return fail(MSRC_ERR_INVALID_ARG, "null output or reps < 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(MSRC_ERR_CUDA, "event creation");
  int pick = -1;
  double best_ms = 0.0;
  msrc_status result = MSRC_OK;
  for (int c = 0; c < tile_config_count(); ++c) {
    ms[c] = -1.0;
    Plan P;
    if (make_plan(rooms, n, n_in, n_out, P, false, c) != MSRC_OK || P.fwd_bytes > ws_bytes) continue;
    msrc_status s = msrc_synthesize_cfg(rooms, n, x_dev, n_in, y_dev, n_out, c, ws, ws_bytes, stream);
    if (s != MSRC_OK) { result = s; break; }
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && s == MSRC_OK; ++r)
      s = msrc_synthesize_cfg(rooms, n, x_dev, n_in, y_dev, n_out, c, ws, ws_bytes, stream);
    cudaEventRecord(e1, st);
    if (s != MSRC_OK) { result = s; break; }
    if (cudaEventSynchronize(e1) != cudaSuccess) { result = fail(MSRC_ERR_CUDA, "event synchronize"); break; }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    ms[c] = double(t) / reps;
    if (pick < 0 || ms[c] < best_ms) { pick = c; best_ms = ms[c]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best = pick;
  if (result != MSRC_OK) return result;
  if (pick < 0) return fail(MSRC_ERR_WORKSPACE, "no tile configuration fits the workspace");
  return MSRC_OK;
}

msrc_status msrc_workspace_errors(void* ws, void* stream, uint32_t* flags) {
  if (!ws || !flags) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, ws, sizeof(v), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "error word read");
  *flags = v;
  return (v & kErrTimeout) ? MSRC_ERR_TIMEOUT : MSRC_OK;
}

msrc_status msrc_room_image_count(msrc_room_t room, int64_t* count, int64_t* per_tier) {
  if (!room || !count) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  *count = room->n_images;
  if (per_tier)
    for (int t = 0; t < MSRC_MAX_TIERS; ++t) per_tier[t] = t < room->d.n_tiers ? room->tier_count[t] : 0;
  return MSRC_OK;
}

msrc_status msrc_room_fit_error(msrc_room_t room, double* err) {
  if (!room || !err) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  *err = room->fit_error;
  return MSRC_OK;
}

msrc_status msrc_room_farrow_table(msrc_room_t room, int32_t which, float* out, int32_t* n_powers) {
  if (!room || !out || !n_powers) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  if (which != 0 && which != 1) return fail(MSRC_ERR_INVALID_ARG, "which must be 0 (synthesis) or 1 (gradient)");
  const int P = which == 0 ? kFarrowCoef : kGradCoef;
  const int L = room->d.taps, kL = room->kL;
  // the values the kernels receive: coefficients of the powers of w = v / 2
  // (c_q 2^q, an exact rescaling of the fit in v)
  for (int sg = 0; sg < kFarrowSegs; ++sg)
    for (int q = 0; q < P; ++q)
      for (int k = -L / 2; k < L / 2; ++k) {
        const float c = which == 0 ? room->farrow[sg][q][k + kL / 2] : room->farrow_g[sg][q][k + kL / 2];
        out[(size_t(sg) * P + q) * L + (k + L / 2)] = std::ldexp(c, q);
      }
  *n_powers = P;
  return MSRC_OK;
}

msrc_status msrc_profile_enable(int32_t on) {
  if (on && !g_prof.on) {
    for (int i = 0; i < kProfSets; ++i)
      for (int k = 0; k <= kPhases; ++k) {
        cudaError_t e = cudaEventCreate(&g_prof.ev[i][k]);
        if (e != cudaSuccess) return cuda_fail(e, "event creation");
      }
    g_prof.on = true;
    g_prof.next = g_prof.pending = 0;
  } else if (!on && g_prof.on) {
    for (int i = 0; i < kProfSets; ++i)
      for (int k = 0; k <= kPhases; ++k) cudaEventDestroy(g_prof.ev[i][k]);
    g_prof.on = false;
  }
  return MSRC_OK;
}

msrc_status msrc_profile_read(double* ms, int32_t* n_calls) {
  if (!ms || !n_calls) return fail(MSRC_ERR_INVALID_ARG, "null argument");
  for (int k = 0; k < kPhases; ++k) ms[k] = 0.0;
  *n_calls = 0;
  if (!g_prof.on) return fail(MSRC_ERR_STATE, "profiling is not enabled");
  const int n = g_prof.pending;
  for (int c = 0; c < n; ++c) {
    const int i = (g_prof.next - n + c + kProfSets) % kProfSets;
    cudaError_t e = cudaEventSynchronize(g_prof.ev[i][kPhases]);
    if (e != cudaSuccess) return cuda_fail(e, "event synchronize");
    for (int k = 0; k < kPhases; ++k) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, g_prof.ev[i][k], g_prof.ev[i][k + 1]);
      if (e != cudaSuccess) return cuda_fail(e, "event elapsed time");
      ms[k] += t;
    }
  }
  *n_calls = n;
  g_prof.pending = 0;
  return MSRC_OK;
}

msrc_status msrc_test_stall_window_copies(uint32_t bytes) {
  if (bytes % 16) return fail(MSRC_ERR_INVALID_ARG, "bytes must be a multiple of 16");
  g_test_extra_tx = bytes;
  return MSRC_OK;
}

msrc_status msrc_set_tile_config(int32_t id) {
  if (id != MSRC_TILE_AUTO && (id < 0 || id >= tile_config_count()))
    return fail(MSRC_ERR_INVALID_ARG, "tile config %d out of range", id);
  g_tile_config.store(id);
  return MSRC_OK;
}

int32_t msrc_tile_configs(void) { return tile_config_count(); }

const char* msrc_status_string(msrc_status s) {
  switch (s) {
    case MSRC_OK: return "ok";
    case MSRC_ERR_INVALID_ARG: return "invalid argument";
    case MSRC_ERR_UNSUPPORTED: return "unsupported";
    case MSRC_ERR_WORKSPACE: return "workspace too small or misaligned";
    case MSRC_ERR_CUDA: return "CUDA error";
    case MSRC_ERR_TIMEOUT: return "device wait timed out";
    case MSRC_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

const char* msrc_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
