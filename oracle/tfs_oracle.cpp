// FP64 CPU oracle for the time-frequency semi-coherent detection statistic of
// arXiv:2510.19047 ("Global time-frequency search for stellar-mass binary black
// holes in LISA").
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the CUDA
// library is checked against. Only the tests, the package smoke check and the
// CPU-baseline leg of bench.py may load it; the product path never does. It shares
// no code, header or constant table with the CUDA sources.
//
// Inputs and outputs are FP64. The per-template evaluation is written once as
// templates over the scalar type R: R = long double (x87 extended precision, 64-bit
// mantissa) gives the statistic, R = Dual (FP64 forward-mode derivative in the 8
// template parameters) gives its exact gradient, with the window position (ceil) and
// the Fresnel branch held fixed, i.e. the almost-everywhere derivative. The value
// path uses extended precision because the printed tranche transform takes sines of
// arguments up to ~1e7 rad (pi v^2 / 2 and pi fdot zeta^2, which cancel) and a
// two-year phase reaches ~1e7 rad: in FP64 those carry ~1e-9 rad of rounding, in
// extended precision ~1e-12.
//
// Paper passages followed (section / equation of the paper):
//   inner products ............ Eqs. inner-cont, inner-complex-cont, inner-all-cont
//   phase-maximised overlap ... Eq. overlap, Eq. overlap-n
//   semi-coherent statistic ... Eq. Upsilon, Eq. Upsilon-seg
//   tranche decomposition ..... Eq. inner-tf, Eq. inner-segment-tf, Eq. inner-tranche-tf
//   quadratic phase per tranche "Time-frequency waveform representation" (Taylor
//                               expansion about the tranche start t_nm)
//   tranche Fourier transform . Eq. fresnel-ft, Eq. kernel-function
//   Fresnel integrals ......... asymptotic form for |z| > 6 and rational form for
//                               |z| <= 6 (same section), odd symmetry
//   21-bin window ............. N_F = 21 bins about ceil(f_nm / delta f)
//   per-tranche response ...... Eq. tdi2 (one complex factor per tranche)
//   gaps ...................... "Search extension to data with gaps": a tranche that
//                               overlaps a gap is left out of Eq. inner-tf
//   compactness diagnostic .... Appendix A: fdot * dT <= 10 delta f
//
// Readings where the paper is silent (each is listed in the design notes):
//   * chirp model: Newtonian (pn_order 0) or 1PN TaylorT3 (pn_order 1) in
//     (M_c, eta, f_0); f_0 and phi_0 are the GW frequency and phase at solar-system
//     barycentre time t' = 0; the amplitude is A = f(t')^(2/3) (its scale cancels).
//   * response (response 1): long-wavelength A/E channels of a rigid LISA
//     constellation on a circular 1 AU orbit; t' = t + n.r(t)/c; f_nm and fdot_nm
//     include the Doppler factors dt'/dt and d2t'/dt2. response 0: T = 1, t' = t.
//     response 2: the TDI-1.5 A/E transfer of the same rigidly rotating constellation
//     with 2.5e9 m arms, evaluated at (t_nm, f_nm) (tdi_transfer below).
//   * the window centre printed as ceil(f / f_nm) delta f is read as
//     k_c = ceil(f_nm / delta f); bins k_c-10 .. k_c+10.
//   * a tranche is active iff its mask is set, t'_nm < t_c, fdot_nm > 0 and the
//     window lies inside bins [1, N_bins-1].
//   * the constant phase of each segment is maximised away (Eq. overlap-n), so the
//     phase of tranche m is taken relative to the start of its segment; this is
//     exactly the same statistic, and keeps the FP64 phase accurate to ~1e-16 of the
//     phase advanced inside one segment instead of inside the whole track.
//   * a segment with <y|y>_n = 0 (no active tranche) adds nothing; N_eff counts the
//     segments that do contribute.
//   * multi-harmonic templates (Sec. "Outlook": {A, f, fdot, phi} per harmonic, then
//     the Fresnel expressions per harmonic): harmonic h has phase nu_h Phi(t'),
//     frequency nu_h f_nm, derivative nu_h fdot_nm and amplitude c_h A (complex c_h),
//     with the dominant mode's polarisation content (the TDI-1.5 transfer taken at the
//     harmonic's frequency). The tranche's template is the sum of the harmonics'
//     21-bin windows, so a bin inside two windows carries both and <y|y> keeps the
//     cross terms. A harmonic whose window leaves [1, N_bins-1] adds nothing; the
//     tranche needs t'_nm < t_c and fdot_nm > 0 as before. The phases are absolute
//     (phi_0 included): the harmonics' relative phases change along the track, so they
//     do not cancel per segment.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

constexpr double PI = 3.14159265358979323846;
constexpr double GMSUN_S = 4.925490947e-6;  // G M_sun / c^3 [s]
constexpr double AU_S = 499.004784;         // 1 AU / c [s]
constexpr double YEAR_S = 31557600.0;       // Julian year [s]
constexpr double OMEGA_ORB = 2.0 * PI / YEAR_S;
constexpr double ARM_S = 2.5e9 / 299792458.0;  // constellation arm length L / c [s]
constexpr int NF = 21;                      // N_F, bins per tranche
constexpr int NF_HALF = 10;
constexpr int NPAR = 8;  // (M_c, eta, f_0, phi_0, lambda, beta, psi, iota)

// ----------------------------------------------------------------------------
// Forward-mode dual numbers: value and derivative along the 8 template parameters.
// ----------------------------------------------------------------------------
struct Dual {
  double v;
  double d[NPAR];
  Dual() : v(0) { std::memset(d, 0, sizeof d); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof d); }
};
static inline Dual chain(const Dual& a, double val, double dval) {
  Dual r(val);
  for (int i = 0; i < NPAR; ++i) r.d[i] = dval * a.d[i];
  return r;
}
static inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v);
  for (int i = 0; i < NPAR; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
static inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v);
  for (int i = 0; i < NPAR; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
static inline Dual operator-(const Dual& a) {
  Dual r(-a.v);
  for (int i = 0; i < NPAR; ++i) r.d[i] = -a.d[i];
  return r;
}
static inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v);
  for (int i = 0; i < NPAR; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
static inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  for (int i = 0; i < NPAR; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
static inline Dual operator+(const Dual& a, double b) { Dual r = a; r.v += b; return r; }
static inline Dual operator+(double b, const Dual& a) { return a + b; }
static inline Dual operator-(const Dual& a, double b) { Dual r = a; r.v -= b; return r; }
static inline Dual operator-(double b, const Dual& a) { return (-a) + b; }
static inline Dual operator*(const Dual& a, double b) {
  Dual r(a.v * b);
  for (int i = 0; i < NPAR; ++i) r.d[i] = a.d[i] * b;
  return r;
}
static inline Dual operator*(double b, const Dual& a) { return a * b; }
static inline Dual operator/(const Dual& a, double b) { return a * (1.0 / b); }
static inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
static inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
static inline Dual& operator-=(Dual& a, const Dual& b) { a = a - b; return a; }
static inline Dual& operator*=(Dual& a, const Dual& b) { a = a * b; return a; }

static inline double val(double x) { return x; }
static inline double val(long double x) { return (double)x; }
static inline double val(const Dual& x) { return x.v; }
static inline long double lval(double x) { return x; }
static inline long double lval(long double x) { return x; }
static inline long double lval(const Dual& x) { return x.v; }

static inline double sin_(double x) { return std::sin(x); }
static inline double cos_(double x) { return std::cos(x); }
static inline double sqrt_(double x) { return std::sqrt(x); }
static inline double log_(double x) { return std::log(x); }
static inline double exp_(double x) { return std::exp(x); }
static inline double expm1_(double x) { return std::expm1(x); }
static inline double log1p_(double x) { return std::log1p(x); }
static inline double pow_(double x, double p) { return std::pow(x, p); }
static inline long double sin_(long double x) { return std::sin(x); }
static inline long double cos_(long double x) { return std::cos(x); }
static inline long double sqrt_(long double x) { return std::sqrt(x); }
static inline long double log_(long double x) { return std::log(x); }
static inline long double exp_(long double x) { return std::exp(x); }
static inline long double expm1_(long double x) { return std::expm1(x); }
static inline long double log1p_(long double x) { return std::log1p(x); }
static inline long double pow_(long double x, double p) { return std::pow(x, (long double)p); }
static inline Dual sin_(const Dual& x) { return chain(x, std::sin(x.v), std::cos(x.v)); }
static inline Dual cos_(const Dual& x) { return chain(x, std::cos(x.v), -std::sin(x.v)); }
static inline Dual sqrt_(const Dual& x) {
  double s = std::sqrt(x.v);
  return chain(x, s, 0.5 / s);
}
static inline Dual log_(const Dual& x) { return chain(x, std::log(x.v), 1.0 / x.v); }
static inline Dual exp_(const Dual& x) {
  double e = std::exp(x.v);
  return chain(x, e, e);
}
static inline Dual expm1_(const Dual& x) { return chain(x, std::expm1(x.v), std::exp(x.v)); }
static inline Dual log1p_(const Dual& x) { return chain(x, std::log1p(x.v), 1.0 / (1.0 + x.v)); }
static inline Dual pow_(const Dual& x, double p) {
  double y = std::pow(x.v, p);
  return chain(x, y, p * std::pow(x.v, p - 1.0));
}

template <class R>
struct Cx {
  R re, im;
};
template <class R>
static inline Cx<R> cadd(const Cx<R>& a, const Cx<R>& b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
static inline Cx<R> cmul(const Cx<R>& a, const Cx<R>& b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// ----------------------------------------------------------------------------
// Fresnel integrals C(z) = int_0^z cos(pi x^2/2) dx, S(z) = int_0^z sin(pi x^2/2) dx.
// ----------------------------------------------------------------------------

// The paper's forms: for |z| > 6 the leading asymptotic term, for |z| <= 6 the
// rational auxiliary functions f(z), g(z) with the printed coefficients; odd in z.
template <class R>
static void fresnel_paper(const R& z, R& C, R& S) {
  const bool neg = val(z) < 0.0;
  const R a = neg ? -z : z;
  const R x = (PI / 2.0) * a * a;
  const R sx = sin_(x), cx = cos_(x);
  if (val(a) > 6.0) {
    C = 0.5 + sx / (PI * a);
    S = 0.5 - cx / (PI * a);
  } else {
    const R f = (1.0 + 0.926 * a) / (2.0 + 1.792 * a + 3.104 * a * a);
    const R g = 1.0 / (2.0 + 4.142 * a + 3.492 * a * a + 6.670 * a * a * a);
    C = 0.5 + f * sx - g * cx;
    S = 0.5 - f * cx - g * sx;
  }
  if (neg) {
    C = -C;
    S = -S;
  }
}

// Exact Fresnel integrals (used only by the pins that test the closed-form tranche
// transform independently of the paper's approximations): composite 10-point
// Gauss-Legendre quadrature of the defining integrals for |z| <= 8, and for |z| > 8
// the asymptotic expansion obtained by repeated integration by parts of
// int_z^inf exp(i pi t^2/2) dt, summed until its terms fall below 1e-18.
struct GaussLegendre10 {
  double x[10], w[10];
  GaussLegendre10() {
    const int n = 10;
    for (int i = 0; i < n; ++i) {
      double t = std::cos(PI * (i + 0.75) / (n + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        double dp = n * (t * p1 - p0) / (t * t - 1.0);
        double dt = p1 / dp;
        t -= dt;
        if (std::fabs(dt) < 1e-16) break;
      }
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (t * p1 - p0) / (t * t - 1.0);
      x[i] = t;
      w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
  }
};
static const GaussLegendre10& gl10() {
  static GaussLegendre10 g;
  return g;
}

static void fresnel_exact_value(double z, double& C, double& S) {
  const bool neg = z < 0.0;
  const double a = std::fabs(z);
  if (a <= 8.0) {
    const GaussLegendre10& g = gl10();
    const int panels = (int)std::ceil(a / 0.02) + 1;
    const double h = a / panels;
    double c = 0.0, s = 0.0;
    for (int p = 0; p < panels; ++p) {
      const double lo = p * h, mid = lo + 0.5 * h;
      for (int i = 0; i < 10; ++i) {
        const double t = mid + 0.5 * h * g.x[i];
        const double ph = 0.5 * PI * t * t;
        c += 0.5 * h * g.w[i] * std::cos(ph);
        s += 0.5 * h * g.w[i] * std::sin(ph);
      }
    }
    C = c;
    S = s;
  } else {
    // C + iS = (1+i)/2 - (g + i f) exp(i pi a^2 / 2)
    // f = (1/(pi a)) sum_k (-1)^k (4k-1)!! / (pi a^2)^(2k)
    // g = (1/(pi^2 a^3)) sum_k (-1)^k (4k+1)!! / (pi a^2)^(2k)
    const double q = 1.0 / (PI * a * a);
    double tf = 1.0, tg = 1.0, sf = 1.0, sg = 1.0;
    for (int k = 1; k < 40; ++k) {
      tf *= -(4.0 * k - 3.0) * (4.0 * k - 1.0) * q * q;
      tg *= -(4.0 * k - 1.0) * (4.0 * k + 1.0) * q * q;
      sf += tf;
      sg += tg;
      if (std::fabs(tf) < 1e-18 && std::fabs(tg) < 1e-18) break;
    }
    const double f = sf / (PI * a), g = sg / (PI * PI * a * a * a);
    const double ph = 0.5 * PI * a * a;
    const double cph = std::cos(ph), sph = std::sin(ph);
    C = 0.5 - (g * cph - f * sph);
    S = 0.5 - (g * sph + f * cph);
  }
  if (neg) {
    C = -C;
    S = -S;
  }
}
static inline void fresnel_exact(double z, double& C, double& S) { fresnel_exact_value(z, C, S); }
static inline void fresnel_exact(long double z, long double& C, long double& S) {
  double c, s;
  fresnel_exact_value((double)z, c, s);
  C = c;
  S = s;
}
static inline void fresnel_exact(const Dual& z, Dual& C, Dual& S) {
  double c, s;
  fresnel_exact_value(z.v, c, s);
  const double ph = 0.5 * PI * z.v * z.v;
  C = chain(z, c, std::cos(ph));
  S = chain(z, s, std::sin(ph));
}

template <class R>
static inline void fresnel(int mode, const R& z, R& C, R& S) {
  if (mode == 1)
    fresnel_exact(z, C, S);
  else
    fresnel_paper(z, C, S);
}

// ----------------------------------------------------------------------------
// Source model: chirp constants, polarisation tensors, Doppler coefficients.
// ----------------------------------------------------------------------------
template <class R>
struct Source {
  R tc;        // coalescence time (SSB) [s]
  R F0, C2;    // f(t') = F0 (y^3 + C2 y^5), y = (1 - t'/t_c)^(-1/8)
  R P5, P3;    // Phi(t') = phi0 + P5 (1 - u^(5/8)) + P3 (1 - u^(3/8)), u = 1 - t'/t_c
  R phi0;
  R ep[3][3], ex[3][3];  // e+ = p p - q q, ex = p q + q p
  R Ap, Ax;              // (1 + cos^2 iota)/2, cos iota
  R dop_c, dop_s;        // (R/c) cos(beta) cos(lambda), (R/c) cos(beta) sin(lambda)
  R nhat[3];             // direction to the source (cos b cos l, cos b sin l, sin b)
};

// Chirp constants are evaluated at the precision of R with the exact rational
// exponents and coefficients (-3/5, -8/3, -5/3, 743/2688, ...) and pi and G M_sun/c^3
// to extended precision: their double roundings would bias t_c and P5 by ~1e-16
// relative, which a two-year phase of ~1e7 rad turns into ~1e-9 rad.
constexpr long double PI_L = 3.141592653589793238462643383279502884L;
constexpr long double GMSUN_S_L = 4.925490947e-6L;
static inline double powq(double x, long double p) { return std::pow(x, (double)p); }
static inline long double powq(long double x, long double p) { return std::pow(x, p); }
static inline Dual powq(const Dual& x, long double p) { return pow_(x, (double)p); }

// 1PN TaylorT3 coefficients (GW phase = 2 x orbital phase; Theta = eta (t_c - t)/(5M)):
//   f   = Theta^(-3/8) / (8 pi M) [1 + (743/2688 + 11 eta/32) Theta^(-1/4)]
//   Phi = phi_c - (2/eta) Theta^(5/8) [1 + (3715/8064 + 55 eta/96) Theta^(-1/4)]
template <class R>
static Source<R> make_source(const R th[NPAR], int pn_order) {
  Source<R> s;
  const R Mc = th[0] * R(GMSUN_S_L);
  const R eta = th[1];
  const R f0 = th[2];
  s.phi0 = th[3];
  if (pn_order == 0) {
    // Newtonian chirp: tau0 = (5/256) (pi f0)^(-8/3) Mc^(-5/3),
    // f = f0 (1 - t/tau0)^(-3/8), Phi = phi0 + (16 pi/5) f0 tau0 [1 - (1 - t/tau0)^(5/8)].
    const R tau0 = (5.0 / 256.0) * powq(R(PI_L) * f0, -8.0L / 3.0L) * powq(Mc, -5.0L / 3.0L);
    s.tc = tau0;
    s.F0 = f0;
    s.C2 = R(0.0);
    s.P5 = R(16.0L * PI_L / 5.0L) * f0 * tau0;
    s.P3 = R(0.0);
  } else {
    const R M = Mc * powq(eta, -3.0L / 5.0L);
    const R cf = R(743.0L / 2688.0L) + (11.0 / 32.0) * eta;
    const R cp = R(3715.0L / 8064.0L) + R(55.0L / 96.0L) * eta;
    const R y = R(8.0L * PI_L) * M * f0;  // x^3 + cf x^5 = y, x = Theta^(-1/8)
    // Newton iterations on the value, then two on R so that derivatives follow the
    // implicit function theorem exactly.
    double xv = std::cbrt(val(y));
    for (int it = 0; it < 60; ++it) {
      const double g = xv * xv * xv + val(cf) * std::pow(xv, 5) - val(y);
      const double gp = 3.0 * xv * xv + 5.0 * val(cf) * std::pow(xv, 4);
      const double dx = g / gp;
      xv -= dx;
      if (std::fabs(dx) < 1e-17 * xv) break;
    }
    R x(xv);
    for (int it = 0; it < 2; ++it) {
      const R g = x * x * x + cf * x * x * x * x * x - y;
      const R gp = 3.0 * x * x + 5.0 * cf * x * x * x * x;
      x = x - g / gp;
    }
    const R Theta0 = pow_(x, -8.0);
    s.tc = 5.0 * M * Theta0 / eta;
    s.F0 = x * x * x / (R(8.0L * PI_L) * M);
    s.C2 = cf * x * x;
    s.P5 = (2.0 / eta) * pow_(Theta0, 0.625);
    s.P3 = (2.0 / eta) * cp * pow_(Theta0, 0.375);
  }
  // Polarisation: source direction n = (cos b cos l, cos b sin l, sin b), wave vector
  // k = -n; reference basis p0 = (sin l, -cos l, 0), q0 = n x p0, rotated by psi.
  const R lam = th[4], bet = th[5], psi = th[6], iota = th[7];
  const R cl = cos_(lam), sl = sin_(lam), cb = cos_(bet), sb = sin_(bet);
  const R cps = cos_(psi), sps = sin_(psi);
  const R p0[3] = {sl, -cl, R(0.0)};
  const R q0[3] = {sb * cl, sb * sl, -cb};
  R p[3], q[3];
  for (int i = 0; i < 3; ++i) {
    p[i] = cps * p0[i] + sps * q0[i];
    q[i] = -sps * p0[i] + cps * q0[i];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      s.ep[i][j] = p[i] * p[j] - q[i] * q[j];
      s.ex[i][j] = p[i] * q[j] + q[i] * p[j];
    }
  const R ci = cos_(iota);
  s.Ap = 0.5 * (1.0 + ci * ci);
  s.Ax = ci;
  s.dop_c = AU_S * cb * cl;
  s.dop_s = AU_S * cb * sl;
  s.nhat[0] = cb * cl;
  s.nhat[1] = cb * sl;
  s.nhat[2] = sb;
  return s;
}

// Long-wavelength detector tensors of the A and E channels at detector time t.
// Guiding centre at r = (cos a, sin a, 0) AU, a = 2 pi t / yr. The constellation
// plane has normal n_c = -r/2 + (sqrt3/2) z (60 degrees to the ecliptic) and the
// three spacecraft sit at angles sigma_i = -a + 2 pi i/3 in that plane
// (cartwheel). Michelson X = (l01 l01 - l02 l02)/2 and cyclic; A = (Z - X)/sqrt2,
// E = (X - 2Y + Z)/sqrt6.
static void detector_tensors(double t, double DA[3][3], double DE[3][3]) {
  const double a = 2.0 * PI * t / YEAR_S;
  const double ca = std::cos(a), sa = std::sin(a);
  const double rhat[3] = {ca, sa, 0.0};
  const double e1[3] = {0.5 * std::sqrt(3.0) * rhat[0], 0.5 * std::sqrt(3.0) * rhat[1], 0.5};
  const double e2[3] = {-sa, ca, 0.0};
  double pos[3][3];
  for (int i = 0; i < 3; ++i) {
    const double sg = -a + 2.0 * PI * i / 3.0;
    for (int k = 0; k < 3; ++k) pos[i][k] = std::cos(sg) * e1[k] + std::sin(sg) * e2[k];
  }
  auto arm = [&](int i, int j, double l[3]) {
    double n2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      l[k] = pos[j][k] - pos[i][k];
      n2 += l[k] * l[k];
    }
    const double n = std::sqrt(n2);
    for (int k = 0; k < 3; ++k) l[k] /= n;
  };
  double D[3][3][3];  // X, Y, Z
  for (int c = 0; c < 3; ++c) {
    double l1[3], l2[3];
    arm(c, (c + 1) % 3, l1);
    arm(c, (c + 2) % 3, l2);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) D[c][i][j] = 0.5 * (l1[i] * l1[j] - l2[i] * l2[j]);
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      DA[i][j] = (D[2][i][j] - D[0][i][j]) / std::sqrt(2.0);
      DE[i][j] = (D[0][i][j] - 2.0 * D[1][i][j] + D[2][i][j]) / std::sqrt(6.0);
    }
}

// Per-tranche transfer factor T_alpha = F+ A+ - i Fx Ax (Eq. tdi2 in the
// long-wavelength limit) at detector time t.
template <class R>
static void response(const Source<R>& s, double t, int n_chan, Cx<R> T[2]) {
  double DA[3][3], DE[3][3];
  detector_tensors(t, DA, DE);
  for (int c = 0; c < n_chan; ++c) {
    const double(*D)[3] = c == 0 ? DA : DE;
    R Fp(0.0), Fx(0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        Fp += D[i][j] * s.ep[i][j];
        Fx += D[i][j] * s.ex[i][j];
      }
    T[c].re = Fp * s.Ap;
    T[c].im = -(Fx * s.Ax);
  }
}

// Spacecraft positions relative to the guiding centre [light-seconds] at detector time
// t: the vertices of the same rotating triangle as detector_tensors, side ARM_S.
static void spacecraft_offsets(double t, double p[3][3]) {
  const double a = 2.0 * PI * t / YEAR_S;
  const double ca = std::cos(a), sa = std::sin(a);
  const double e1[3] = {0.5 * std::sqrt(3.0) * ca, 0.5 * std::sqrt(3.0) * sa, 0.5};
  const double e2[3] = {-sa, ca, 0.0};
  const double rad = ARM_S / std::sqrt(3.0);
  for (int i = 0; i < 3; ++i) {
    const double sg = -a + 2.0 * PI * i / 3.0;
    for (int k = 0; k < 3; ++k) p[i][k] = rad * (std::cos(sg) * e1[k] + std::sin(sg) * e2[k]);
  }
}

// TDI-1.5 transfer factors of the A and E channels at detector time t and GW frequency
// f (Eq. tdi2 with the full response; the paper builds its TDI variables from
// single-link observables of a rigidly rotating, constant-arm constellation). For the
// complex polarisation tensor P = A+ e+ - i Ax ex and propagation direction k = -n:
//   single link s -> r, unit vector n_sr = (p_r - p_s)/L:
//     G_sr = i pi f L sinc(pi f L (1 - k.n_sr)) exp(-i pi f (L + k.(p_s + p_r))) n_sr.P.n_sr
//   (the plane-wave fractional frequency shift [H(t - k.p_r) - H(t - L - k.p_s)] /
//   (2 (1 - k.n_sr)) of a locally monochromatic wave, with the barycentre delay of the
//   guiding centre left in the template phase); with z = exp(-2 pi i f L),
//     X = (1 - z^2) [(G_10 + z G_01) - (G_20 + z G_02)]   (G_sr for link s -> r)
//   and Y, Z cyclic; A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6. In the long-wavelength
//   limit X -> -16 pi^2 f^2 L^2 D_X : P.
template <class R>
static void tdi_transfer(const Source<R>& s, double t, const R& f, int n_chan, Cx<R> T[2]) {
  double p[3][3];
  spacecraft_offsets(t, p);
  const double L = ARM_S;
  R kp[3];  // k . p_i
  for (int i = 0; i < 3; ++i) kp[i] = -(s.nhat[0] * p[i][0] + s.nhat[1] * p[i][1] + s.nhat[2] * p[i][2]);
  // n.P.n for the arm (i, j) (the same for both directions)
  auto nPn = [&](int i, int j) {
    double n[3];
    for (int k = 0; k < 3; ++k) n[k] = (p[j][k] - p[i][k]) / L;
    R ep(0.0), ex(0.0);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        ep += n[a] * n[b] * s.ep[a][b];
        ex += n[a] * n[b] * s.ex[a][b];
      }
    return Cx<R>{s.Ap * ep, -(s.Ax * ex)};
  };
  const Cx<R> q01 = nPn(0, 1), q02 = nPn(0, 2), q12 = nPn(1, 2);
  auto link = [&](int sd, int rc, const Cx<R>& q) {
    const R kn = (kp[rc] - kp[sd]) / L;        // k . n_sr
    const R x = PI * f * L * (1.0 - kn);
    const R sinc = std::fabs(lval(x)) < 1e-6 ? R(1.0) - x * x / 6.0 : sin_(x) / x;
    const R ph = -PI * f * (L + kp[sd] + kp[rc]);
    const R amp = PI * f * L * sinc;            // times i
    const Cx<R> e = {cos_(ph), sin_(ph)};
    const Cx<R> iq = {-amp * q.im, amp * q.re};  // i amp q
    return cmul(e, iq);
  };
  const Cx<R> G01 = link(0, 1, q01), G10 = link(1, 0, q01);
  const Cx<R> G02 = link(0, 2, q02), G20 = link(2, 0, q02);
  const Cx<R> G12 = link(1, 2, q12), G21 = link(2, 1, q12);
  const R w = -2.0 * PI * f * L;
  const Cx<R> z = {cos_(w), sin_(w)};
  const Cx<R> z2 = cmul(z, z);
  const Cx<R> one_mz2 = {1.0 - z2.re, -z2.im};
  auto rt = [&](const Cx<R>& a, const Cx<R>& b) { return cadd(a, cmul(z, b)); };
  auto sub = [](const Cx<R>& a, const Cx<R>& b) { return Cx<R>{a.re - b.re, a.im - b.im}; };
  const Cx<R> X = cmul(one_mz2, sub(rt(G10, G01), rt(G20, G02)));
  const Cx<R> Y = cmul(one_mz2, sub(rt(G21, G12), rt(G01, G10)));
  const Cx<R> Z = cmul(one_mz2, sub(rt(G02, G20), rt(G12, G21)));
  const double r2 = 1.0 / std::sqrt(2.0), r6 = 1.0 / std::sqrt(6.0);
  T[0] = {(Z.re - X.re) * r2, (Z.im - X.im) * r2};
  if (n_chan > 1) T[1] = {(X.re - 2.0 * Y.re + Z.re) * r6, (X.im - 2.0 * Y.im + Z.im) * r6};
}

// Doppler delay n.r(t)/c and its first two time derivatives.
template <class R>
static void doppler(const Source<R>& s, double t, int resp, R& d0, R& d1, R& d2) {
  if (resp == 0) {
    d0 = R(0.0);
    d1 = R(0.0);
    d2 = R(0.0);
    return;
  }
  const double a = 2.0 * PI * t / YEAR_S;
  const double ca = std::cos(a), sa = std::sin(a);
  d0 = s.dop_c * ca + s.dop_s * sa;
  d1 = OMEGA_ORB * (s.dop_s * ca - s.dop_c * sa);
  d2 = -(OMEGA_ORB * OMEGA_ORB) * d0;
}

// Frequency track, its derivative, amplitude and the phase advanced since an
// anchor, at detector time t (retarded SSB time t' = t + n.r/c).
template <class R>
struct TrackPoint {
  bool alive;  // t' < t_c
  R f, fdot, amp, dphi;
};
template <class R>
static TrackPoint<R> track_point(const Source<R>& s, int resp, double t, double t_anchor) {
  TrackPoint<R> tp;
  R d0, d1, d2, a0, a1, a2;
  doppler(s, t, resp, d0, d1, d2);
  doppler(s, t_anchor, resp, a0, a1, a2);
  const R tp_m = t + d0;         // t'
  const R tp_a = t_anchor + a0;  // t' at anchor
  tp.alive = val(tp_m) < val(s.tc) && val(tp_a) < val(s.tc);
  if (!tp.alive) return tp;
  const R u = 1.0 - tp_m / s.tc;
  const R y = pow_(u, -0.125);
  const R y2 = y * y, y3 = y2 * y;
  const R fsrc = s.F0 * (y3 + s.C2 * y3 * y2);
  const R y11 = y3 * y3 * y3 * y2;
  const R fdsrc = s.F0 * y11 * (3.0 + 5.0 * s.C2 * y2) / (8.0 * s.tc);
  const R dtp = 1.0 + d1;  // dt'/dt
  tp.f = fsrc * dtp;
  tp.fdot = fdsrc * dtp * dtp + fsrc * d2;
  tp.amp = pow_(fsrc, 2.0 / 3.0);
  // Phi(t'_m) - Phi(t'_a) = P5 (u_a^(5/8) - u^(5/8)) + P3 (u_a^(3/8) - u^(3/8)),
  // evaluated as u_a^p * (-expm1(p log1p(rho))), rho = -(t'_m - t'_a)/(t_c - t'_a).
  const R delta = (t - t_anchor) + (d0 - a0);
  const R ua = 1.0 - tp_a / s.tc;
  const R rho = -delta / (s.tc - tp_a);
  const R l1p = log1p_(rho);
  tp.dphi = s.P5 * pow_(ua, 0.625) * (-expm1_(0.625 * l1p)) +
            s.P3 * pow_(ua, 0.375) * (-expm1_(0.375 * l1p));
  return tp;
}

// Eq. fresnel-ft: the Fourier transform over one tranche of A e^{i phi(t)} with
// phi quadratic about the tranche start, at f = k delta f, written out as printed.
template <class R>
static Cx<R> tranche_ft_bin(const R& amp, const R& phi, const R& fm, const R& fdot, double dT,
                            double fk, int fmode) {
  const R zeta = (fm - fk) / fdot;
  const R s2 = sqrt_(2.0 * fdot);
  const R v1 = s2 * zeta;
  const R v2 = s2 * (dT + zeta);
  R C1, S1, C2, S2;
  fresnel(fmode, v1, C1, S1);
  fresnel(fmode, v2, C2, S2);
  const R ph = phi - PI * fdot * zeta * zeta;
  const R pre = amp / s2;
  const Cx<R> e = {pre * cos_(ph), pre * sin_(ph)};
  const Cx<R> F = {C2 - C1, S2 - S1};
  return cmul(e, F);
}

struct Grid {
  int n_chan, n_tranche, n_bins;
  double dT, t0, df;
  const double *d_re, *d_im, *w;  // [chan][tranche][bin]
  const uint8_t* mask;            // [tranche] (nullptr = all kept)
};

struct Diag {
  int n_active, n_noncompact;
};

// Upsilon_{N_seg} (Eq. Upsilon-seg) for one template. Returns N_eff.
template <class R>
static int statistic_one(const Grid& g, const R th[NPAR], int pn_order, int resp, int fmode,
                         int n_seg, R& out, Diag* diag, double* seg_zr = nullptr,
                         double* seg_zi = nullptr, double* seg_n = nullptr,
                         R* seg_full = nullptr, std::vector<R>* tr_vals = nullptr,
                         std::vector<int>* tr_seg = nullptr) {
  const Source<R> src = make_source(th, pn_order);
  const int seg_len = g.n_tranche / n_seg;
  R ups(0.0);
  int neff = 0, nact = 0, nnc = 0;
  for (int n = 0; n < n_seg; ++n) {
    const double t_anchor = g.t0 + (double)n * seg_len * g.dT;
    Cx<R> Z = {R(0.0), R(0.0)};
    R N(0.0);
    for (int m = n * seg_len; m < (n + 1) * seg_len; ++m) {
      if (g.mask && !g.mask[m]) continue;
      const double tm = g.t0 + (double)m * g.dT;
      const TrackPoint<R> tp = track_point(src, resp, tm, t_anchor);
      if (!tp.alive) continue;
      if (!(val(tp.fdot) > 0.0)) continue;
      const long kc = (long)std::ceil(lval(tp.f) / (long double)g.df);
      if (kc - NF_HALF < 1 || kc + NF_HALF > g.n_bins - 1) continue;
      ++nact;
      if (val(tp.fdot) * g.dT > 10.0 * g.df) ++nnc;
      Cx<R> T[2];
      if (resp == 0) {
        T[0] = {R(1.0), R(0.0)};
        T[1] = {R(1.0), R(0.0)};
      } else if (resp == 2) {
        tdi_transfer(src, tm, tp.f, g.n_chan, T);
      } else {
        response(src, tm, g.n_chan, T);
      }
      Cx<R> zc[2] = {{R(0.0), R(0.0)}, {R(0.0), R(0.0)}};
      R nc[2] = {R(0.0), R(0.0)};
      for (int j = 0; j < NF; ++j) {
        const long k = kc - NF_HALF + j;
        const Cx<R> h = tranche_ft_bin(tp.amp, tp.dphi, tp.f, tp.fdot, g.dT, k * g.df, fmode);
        const R hh = h.re * h.re + h.im * h.im;
        for (int c = 0; c < g.n_chan; ++c) {
          const size_t idx = ((size_t)c * g.n_tranche + m) * g.n_bins + k;
          const double wr = g.w[idx] * g.df;
          const double dr = g.d_re[idx], di = g.d_im[idx];
          // conj(d) h w delta f
          zc[c].re += (dr * h.re + di * h.im) * wr;
          zc[c].im += (dr * h.im - di * h.re) * wr;
          nc[c] += hh * wr;
        }
      }
      Cx<R> zt = {R(0.0), R(0.0)};
      R nt(0.0);
      for (int c = 0; c < g.n_chan; ++c) {
        zt = cadd(zt, cmul(T[c], zc[c]));
        nt += (T[c].re * T[c].re + T[c].im * T[c].im) * nc[c];
      }
      Z = cadd(Z, zt);
      N += nt;
      if (tr_vals) {  // this tranche's share of Z_n and N_n
        tr_vals->push_back(zt.re);
        tr_vals->push_back(zt.im);
        tr_vals->push_back(nt);
        tr_seg->push_back(n);
      }
    }
    if (seg_zr) {
      seg_zr[n] = val(Z.re);
      seg_zi[n] = val(Z.im);
      seg_n[n] = val(N);
    }
    if (seg_full) {
      seg_full[3 * n] = Z.re;
      seg_full[3 * n + 1] = Z.im;
      seg_full[3 * n + 2] = N;
    }
    if (val(N) > 0.0) {
      ups += 4.0 * (Z.re * Z.re + Z.im * Z.im) / N;
      ++neff;
    }
  }
  out = ups;
  if (diag) {
    diag->n_active = nact;
    diag->n_noncompact = nnc;
  }
  return neff;
}

// Harmonic set of a multi-harmonic template: n harmonics (nu_h, c_h).
struct Harmonics {
  int n;
  const double *nu, *c_re, *c_im;
};

// Absolute phase Phi(t') = phi0 + P5 (1 - u^(5/8)) + P3 (1 - u^(3/8)), u = 1 - t'/t_c,
// with 1 - u^p = -expm1(p log1p(-t'/t_c)).
template <class R>
static R phase_abs(const Source<R>& s, const R& tprime) {
  const R l = log1p_(-tprime / s.tc);
  return s.phi0 + s.P5 * (-expm1_(0.625 * l)) + s.P3 * (-expm1_(0.375 * l));
}

// Upsilon_{N_seg} of a multi-harmonic template, Eq. Upsilon-seg with the template of
// each tranche written out bin by bin as the sum of its harmonics' Eq. fresnel-ft
// windows. Returns N_eff.
template <class R>
static int statistic_harm_one(const Grid& g, const R th[NPAR], int pn_order, int resp,
                              int fmode, const Harmonics& H, int n_seg, R& out, Diag* diag,
                              double* seg_zr = nullptr, double* seg_zi = nullptr,
                              double* seg_n = nullptr) {
  const Source<R> src = make_source(th, pn_order);
  const int seg_len = g.n_tranche / n_seg;
  R ups(0.0);
  int neff = 0, nact = 0, nnc = 0;
  for (int n = 0; n < n_seg; ++n) {
    const double t_anchor = g.t0 + (double)n * seg_len * g.dT;
    R a0, a1, a2;
    doppler(src, t_anchor, resp, a0, a1, a2);
    const R tp_anchor = t_anchor + a0;
    // Phi at the anchor; track_point gives the phase advanced from there
    const R phi_anchor = val(tp_anchor) < val(src.tc) ? phase_abs(src, tp_anchor) : R(0.0);
    Cx<R> Z = {R(0.0), R(0.0)};
    R N(0.0);
    for (int m = n * seg_len; m < (n + 1) * seg_len; ++m) {
      if (g.mask && !g.mask[m]) continue;
      const double tm = g.t0 + (double)m * g.dT;
      const TrackPoint<R> tp = track_point(src, resp, tm, t_anchor);
      if (!tp.alive) continue;
      if (!(val(tp.fdot) > 0.0)) continue;
      const R phi = phi_anchor + tp.dphi;
      // the tranche's template per channel, bin -> value (T_alpha included)
      std::map<long, Cx<R>> y[2];
      bool any = false;
      for (int h = 0; h < H.n; ++h) {
        const R fh = H.nu[h] * tp.f, fdh = H.nu[h] * tp.fdot;
        const long kc = (long)std::ceil(lval(fh) / (long double)g.df);
        if (kc - NF_HALF < 1 || kc + NF_HALF > g.n_bins - 1) continue;
        any = true;
        Cx<R> T[2];
        if (resp == 0) {
          T[0] = {R(1.0), R(0.0)};
          T[1] = {R(1.0), R(0.0)};
        } else if (resp == 2) {
          tdi_transfer(src, tm, fh, g.n_chan, T);
        } else {
          response(src, tm, g.n_chan, T);
        }
        const Cx<R> ch = {R(H.c_re[h]), R(H.c_im[h])};
        for (int j = 0; j < NF; ++j) {
          const long k = kc - NF_HALF + j;
          const Cx<R> hk = tranche_ft_bin(tp.amp, H.nu[h] * phi, fh, fdh, g.dT, k * g.df, fmode);
          for (int c = 0; c < g.n_chan; ++c) {
            Cx<R>& v = y[c].emplace(k, Cx<R>{R(0.0), R(0.0)}).first->second;
            v = cadd(v, cmul(cmul(T[c], ch), hk));
          }
        }
      }
      if (!any) continue;
      ++nact;
      if (val(tp.fdot) * g.dT > 10.0 * g.df) ++nnc;
      for (int c = 0; c < g.n_chan; ++c) {
        for (const auto& kv : y[c]) {
          const size_t idx = ((size_t)c * g.n_tranche + m) * g.n_bins + kv.first;
          const double wr = g.w[idx] * g.df;
          const double dr = g.d_re[idx], di = g.d_im[idx];
          const Cx<R>& v = kv.second;
          Z.re += (dr * v.re + di * v.im) * wr;  // conj(d) y w delta f
          Z.im += (dr * v.im - di * v.re) * wr;
          N += (v.re * v.re + v.im * v.im) * wr;
        }
      }
    }
    if (seg_zr) {
      seg_zr[n] = val(Z.re);
      seg_zi[n] = val(Z.im);
      seg_n[n] = val(N);
    }
    if (val(N) > 0.0) {
      ups += 4.0 * (Z.re * Z.re + Z.im * Z.im) / N;
      ++neff;
    }
  }
  out = ups;
  if (diag) {
    diag->n_active = nact;
    diag->n_noncompact = nnc;
  }
  return neff;
}

}  // namespace orc

using namespace orc;

static bool grid_ok(int n_chan, int n_tranche, int n_bins, double dT) {
  return n_chan >= 1 && n_chan <= 2 && n_tranche >= 1 && n_bins >= 2 * NF_HALF + 2 && dT > 0;
}

extern "C" {

// Error codes shared in meaning (not in code) with the CUDA library.
enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_NSEG = -3 };

// Upsilon_{N_seg} for n_tpl templates. theta is SoA [8][n_tpl] in the order
// (M_c [M_sun], eta, f_0 [Hz], phi_0, lambda, beta, psi, iota). Grids are
// [chan][tranche][bin]; w = 1/S. Outputs: out_stat[n_tpl], out_neff[n_tpl] and, if
// non-null, the active and non-compact tranche counts per template.
int oracle_statistic(int n_chan, int n_tranche, int n_bins, double dT, double t0,
                     const double* d_re, const double* d_im, const double* w,
                     const uint8_t* mask, int pn_order, int resp, int fresnel_mode,
                     const double* theta, int64_t n_tpl, int n_seg, double* out_stat,
                     int32_t* out_neff, int32_t* out_nact, int32_t* out_nnc, int n_threads) {
  if (!grid_ok(n_chan, n_tranche, n_bins, dT) || n_tpl < 0 || !theta || !out_stat) return ORC_ERR_ARG;
  if (n_seg < 1 || n_tranche % n_seg != 0) return ORC_ERR_NSEG;
  Grid g{n_chan, n_tranche, n_bins, dT, t0, 1.0 / dT, d_re, d_im, w, mask};
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < n_tpl; ++i) {
    long double th[NPAR];
    for (int p = 0; p < NPAR; ++p) th[p] = theta[p * n_tpl + i];
    long double ups;
    Diag dg;
    const int neff =
        statistic_one<long double>(g, th, pn_order, resp, fresnel_mode, n_seg, ups, &dg);
    out_stat[i] = (double)ups;
    if (out_neff) out_neff[i] = neff;
    if (out_nact) out_nact[i] = dg.n_active;
    if (out_nnc) out_nnc[i] = dg.n_noncompact;
  }
  return ORC_OK;
}

// Upsilon_{N_seg} and its gradient d Upsilon / d theta, out_grad SoA [8][n_tpl].
int oracle_gradient(int n_chan, int n_tranche, int n_bins, double dT, double t0,
                    const double* d_re, const double* d_im, const double* w,
                    const uint8_t* mask, int pn_order, int resp, int fresnel_mode,
                    const double* theta, int64_t n_tpl, int n_seg, double* out_stat,
                    double* out_grad, int n_threads) {
  if (!grid_ok(n_chan, n_tranche, n_bins, dT) || n_tpl < 0 || !theta || !out_stat || !out_grad)
    return ORC_ERR_ARG;
  if (n_seg < 1 || n_tranche % n_seg != 0) return ORC_ERR_NSEG;
  Grid g{n_chan, n_tranche, n_bins, dT, t0, 1.0 / dT, d_re, d_im, w, mask};
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < n_tpl; ++i) {
    Dual th[NPAR];
    for (int p = 0; p < NPAR; ++p) {
      th[p] = Dual(theta[p * n_tpl + i]);
      th[p].d[p] = 1.0;
    }
    Dual ups;
    statistic_one<Dual>(g, th, pn_order, resp, fresnel_mode, n_seg, ups, nullptr);
    out_stat[i] = ups.v;
    for (int p = 0; p < NPAR; ++p) out_grad[p * n_tpl + i] = ups.d[p];
  }
  return ORC_OK;
}

// Term scale of each gradient component: dUpsilon/dtheta_p is the sum over segments of
//   8 Re(conj(Z_n) dZ_n/dtheta_p) / N_n  -  4 |Z_n|^2 (dN_n/dtheta_p) / N_n^2
// (Eq. Upsilon-seg differentiated). tranche_level == 0: out_scale[p][i] is the sum of
// the absolute values of those 2 N_seg terms; tranche_level == 1: Z_n and N_n are split
// into their tranches' shares z_m, n_m (Eq. inner-tranche-tf) and out_scale is the sum
// over every (segment, tranche) of |8 Re(conj(Z_n) dz_m)/N_n - 4 |Z_n|^2 dn_m/N_n^2|.
// A component much smaller than its term scale is a cancelling sum, which arithmetic of
// unit roundoff u that forms those terms resolves only to ~u times the scale.
int oracle_gradient_scale(int n_chan, int n_tranche, int n_bins, double dT, double t0,
                          const double* d_re, const double* d_im, const double* w,
                          const uint8_t* mask, int pn_order, int resp, int fresnel_mode,
                          const double* theta, int64_t n_tpl, int n_seg, double* out_scale,
                          int tranche_level, int n_threads) {
  if (!grid_ok(n_chan, n_tranche, n_bins, dT) || n_tpl < 0 || !theta || !out_scale)
    return ORC_ERR_ARG;
  if (n_seg < 1 || n_tranche % n_seg != 0) return ORC_ERR_NSEG;
  Grid g{n_chan, n_tranche, n_bins, dT, t0, 1.0 / dT, d_re, d_im, w, mask};
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < n_tpl; ++i) {
    Dual th[NPAR];
    for (int p = 0; p < NPAR; ++p) {
      th[p] = Dual(theta[p * n_tpl + i]);
      th[p].d[p] = 1.0;
    }
    Dual ups;
    std::vector<Dual> seg(3 * (size_t)n_seg), trv;
    std::vector<int> trs;
    statistic_one<Dual>(g, th, pn_order, resp, fresnel_mode, n_seg, ups, nullptr, nullptr,
                        nullptr, nullptr, seg.data(), tranche_level ? &trv : nullptr,
                        tranche_level ? &trs : nullptr);
    for (int p = 0; p < NPAR; ++p) {
      double sc = 0.0;
      if (tranche_level) {
        // every (segment, tranche) term 8 Re(conj(Z_n) dz_m)/N_n - 4 |Z_n|^2 dn_m / N_n^2
        for (size_t t = 0; t < trs.size(); ++t) {
          const int n = trs[t];
          const Dual &zr = seg[3 * n], &zi = seg[3 * n + 1], &nn = seg[3 * n + 2];
          if (!(nn.v > 0.0)) continue;
          const Dual &mr = trv[3 * t], &mi = trv[3 * t + 1], &mn = trv[3 * t + 2];
          sc += std::fabs(8.0 * (zr.v * mr.d[p] + zi.v * mi.d[p]) / nn.v -
                          4.0 * (zr.v * zr.v + zi.v * zi.v) * mn.d[p] / (nn.v * nn.v));
        }
      } else {
        for (int n = 0; n < n_seg; ++n) {
          const Dual &zr = seg[3 * n], &zi = seg[3 * n + 1], &nn = seg[3 * n + 2];
          if (!(nn.v > 0.0)) continue;
          sc += std::fabs(8.0 * (zr.v * zr.d[p] + zi.v * zi.d[p]) / nn.v) +
                std::fabs(4.0 * (zr.v * zr.v + zi.v * zi.v) * nn.d[p] / (nn.v * nn.v));
        }
      }
      out_scale[p * n_tpl + i] = sc;
    }
  }
  return ORC_OK;
}

// Per-segment complex overlap Z_n = sum_alpha (d_alpha,n | y_alpha,n) and norm
// N_n = sum_alpha (y_alpha,n | y_alpha,n) of one template (Eqs. overlap-n,
// inner-segment-tf); O_n = 4|Z_n| and <y|y>_n = 4 N_n.
int oracle_segments(int n_chan, int n_tranche, int n_bins, double dT, double t0,
                    const double* d_re, const double* d_im, const double* w,
                    const uint8_t* mask, int pn_order, int resp, int fresnel_mode,
                    const double* th8, int n_seg, double* zr, double* zi, double* nn,
                    double* out_stat) {
  if (!grid_ok(n_chan, n_tranche, n_bins, dT) || !th8 || !zr || !zi || !nn) return ORC_ERR_ARG;
  if (n_seg < 1 || n_tranche % n_seg != 0) return ORC_ERR_NSEG;
  Grid g{n_chan, n_tranche, n_bins, dT, t0, 1.0 / dT, d_re, d_im, w, mask};
  long double th[NPAR];
  for (int p = 0; p < NPAR; ++p) th[p] = th8[p];
  long double ups;
  statistic_one<long double>(g, th, pn_order, resp, fresnel_mode, n_seg, ups, nullptr, zr, zi,
                             nn);
  if (out_stat) *out_stat = (double)ups;
  return ORC_OK;
}

// Upsilon_{N_seg} of multi-harmonic templates: as oracle_statistic, with n_harm
// harmonics (nu[h] > 0, complex amplitude c_re[h] + i c_im[h]) shared by all templates.
int oracle_statistic_harm(int n_chan, int n_tranche, int n_bins, double dT, double t0,
                          const double* d_re, const double* d_im, const double* w,
                          const uint8_t* mask, int pn_order, int resp, int fresnel_mode,
                          int n_harm, const double* nu, const double* c_re, const double* c_im,
                          const double* theta, int64_t n_tpl, int n_seg, double* out_stat,
                          int32_t* out_neff, int32_t* out_nact, int32_t* out_nnc, int n_threads) {
  if (!grid_ok(n_chan, n_tranche, n_bins, dT) || n_tpl < 0 || !theta || !out_stat) return ORC_ERR_ARG;
  if (n_harm < 1 || !nu || !c_re || !c_im) return ORC_ERR_ARG;
  for (int h = 0; h < n_harm; ++h)
    if (!(nu[h] > 0.0)) return ORC_ERR_ARG;
  if (n_seg < 1 || n_tranche % n_seg != 0) return ORC_ERR_NSEG;
  Grid g{n_chan, n_tranche, n_bins, dT, t0, 1.0 / dT, d_re, d_im, w, mask};
  const Harmonics H{n_harm, nu, c_re, c_im};
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < n_tpl; ++i) {
    long double th[NPAR];
    for (int p = 0; p < NPAR; ++p) th[p] = theta[p * n_tpl + i];
    long double ups;
    Diag dg;
    const int neff =
        statistic_harm_one<long double>(g, th, pn_order, resp, fresnel_mode, H, n_seg, ups, &dg);
    out_stat[i] = (double)ups;
    if (out_neff) out_neff[i] = neff;
    if (out_nact) out_nact[i] = dg.n_active;
    if (out_nnc) out_nnc[i] = dg.n_noncompact;
  }
  return ORC_OK;
}

// Per-segment Z_n, N_n of one multi-harmonic template (as oracle_segments).
int oracle_segments_harm(int n_chan, int n_tranche, int n_bins, double dT, double t0,
                         const double* d_re, const double* d_im, const double* w,
                         const uint8_t* mask, int pn_order, int resp, int fresnel_mode,
                         int n_harm, const double* nu, const double* c_re, const double* c_im,
                         const double* th8, int n_seg, double* zr, double* zi, double* nn,
                         double* out_stat) {
  if (!grid_ok(n_chan, n_tranche, n_bins, dT) || !th8 || !zr || !zi || !nn) return ORC_ERR_ARG;
  if (n_harm < 1 || !nu || !c_re || !c_im) return ORC_ERR_ARG;
  if (n_seg < 1 || n_tranche % n_seg != 0) return ORC_ERR_NSEG;
  Grid g{n_chan, n_tranche, n_bins, dT, t0, 1.0 / dT, d_re, d_im, w, mask};
  const Harmonics H{n_harm, nu, c_re, c_im};
  long double th[NPAR];
  for (int p = 0; p < NPAR; ++p) th[p] = th8[p];
  long double ups;
  statistic_harm_one<long double>(g, th, pn_order, resp, fresnel_mode, H, n_seg, ups, nullptr,
                                  zr, zi, nn);
  if (out_stat) *out_stat = (double)ups;
  return ORC_OK;
}

// Fresnel integrals: mode 0 = the paper's forms, mode 1 = exact.
void oracle_fresnel(int mode, const double* z, int64_t n, double* C, double* S) {
  for (int64_t i = 0; i < n; ++i) fresnel<double>(mode, z[i], C[i], S[i]);
}

// Tranche transform h~(k delta f), k = k0 .. k0+nk-1 (Eq. fresnel-ft).
void oracle_tranche_ft(double amp, double phi, double fm, double fdot, double dT, int64_t k0,
                       int64_t nk, int fresnel_mode, double* re, double* im) {
  const double df = 1.0 / dT;
  for (int64_t i = 0; i < nk; ++i) {
    const Cx<long double> h = tranche_ft_bin<long double>(amp, phi, fm, fdot, dT,
                                                          (long double)(k0 + i) * df, fresnel_mode);
    re[i] = (double)h.re;
    im[i] = (double)h.im;
  }
}

// Source constants of one template: out = (t_c, F0, C2, P5, P3).
void oracle_source(const double* th8, int pn_order, double* out5) {
  const Source<double> s = make_source<double>(th8, pn_order);
  out5[0] = s.tc;
  out5[1] = s.F0;
  out5[2] = s.C2;
  out5[3] = s.P5;
  out5[4] = s.P3;
}

// Track at detector times t[n]: f, fdot, amplitude, phase advanced since
// t_anchor, retarded time t'; alive[i] = 0 past coalescence.
void oracle_track(const double* th8, int pn_order, int resp, const double* t, int64_t n,
                  double t_anchor, double* f, double* fdot, double* amp, double* dphi,
                  double* tprime, uint8_t* alive) {
  long double th[NPAR];
  for (int p = 0; p < NPAR; ++p) th[p] = th8[p];
  const Source<long double> s = make_source<long double>(th, pn_order);
  for (int64_t i = 0; i < n; ++i) {
    const TrackPoint<long double> tp = track_point(s, resp, t[i], t_anchor);
    long double d0, d1, d2;
    doppler(s, t[i], resp, d0, d1, d2);
    tprime[i] = (double)(t[i] + d0);
    alive[i] = tp.alive ? 1 : 0;
    f[i] = tp.alive ? (double)tp.f : 0.0;
    fdot[i] = tp.alive ? (double)tp.fdot : 0.0;
    amp[i] = tp.alive ? (double)tp.amp : 0.0;
    dphi[i] = tp.alive ? (double)tp.dphi : 0.0;
  }
}

// Response factors T_alpha at detector times t[n]: T_re/T_im [chan][n].
void oracle_response(const double* th8, const double* t, int64_t n, int n_chan, double* T_re,
                     double* T_im) {
  const Source<double> s = make_source<double>(th8, 0);
  for (int64_t i = 0; i < n; ++i) {
    Cx<double> T[2];
    response(s, t[i], n_chan, T);
    for (int c = 0; c < n_chan; ++c) {
      T_re[c * n + i] = T[c].re;
      T_im[c * n + i] = T[c].im;
    }
  }
}

// TDI-1.5 transfer factors at detector times t[n] and GW frequencies f[n]:
// T_re/T_im [chan][n].
void oracle_response_tdi(const double* th8, const double* t, const double* f, int64_t n,
                         int n_chan, double* T_re, double* T_im) {
  long double th[NPAR];
  for (int p = 0; p < NPAR; ++p) th[p] = th8[p];
  const Source<long double> s = make_source<long double>(th, 0);
  for (int64_t i = 0; i < n; ++i) {
    Cx<long double> T[2];
    tdi_transfer(s, t[i], (long double)f[i], n_chan, T);
    for (int c = 0; c < n_chan; ++c) {
      T_re[c * n + i] = (double)T[c].re;
      T_im[c * n + i] = (double)T[c].im;
    }
  }
}

// Spacecraft offsets from the guiding centre [light-seconds], row-major [3][3].
void oracle_spacecraft_offsets(double t, double* p9) {
  double p[3][3];
  spacecraft_offsets(t, p);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) p9[3 * i + k] = p[i][k];
}

// Detector tensors D_A, D_E (row-major 3x3 each) at detector time t.
void oracle_detector_tensors(double t, double* DA9, double* DE9) {
  double DA[3][3], DE[3][3];
  detector_tensors(t, DA, DE);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      DA9[3 * i + j] = DA[i][j];
      DE9[3 * i + j] = DE[i][j];
    }
}

// Polarisation tensors (row-major 3x3) of one template.
void oracle_polarisation(const double* th8, double* ep9, double* ex9) {
  const Source<double> s = make_source<double>(th8, 0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      ep9[3 * i + j] = s.ep[i][j];
      ex9[3 * i + j] = s.ex[i][j];
    }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
