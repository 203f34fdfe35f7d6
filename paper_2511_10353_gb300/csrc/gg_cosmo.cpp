// FP64 host mathematics of the Sec. 2.1 inputs: transfer functions, the
// sigma_8 normalisation of P(k), linear growth D(a) and f(a), and the tables
// the kernels read (density filter S(m^2), psi gain G(m^2), FFT twiddles).
//
// Readings (the paper takes cosmological parameters and a tabulated P(k) but
// fixes no model): LambdaCDM with curvature, no radiation; Heath (1977)
// growth integral; P(k, 0) = A k^n_s T(k)^2 normalised by the top-hat
// sigma(8 Mpc/h); BBKS (1986) eq. G3 and Eisenstein & Hu (1998) eqs. 26,
// 28-31 transfer functions; v = 100 a E f psi km/s.
#include "gg_cosmo.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace gg {
namespace cosmo {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Gauss-Kronrod (7, 15) abscissae and weights on [-1, 1] (Kronrod 1965;
// the QUADPACK tables of Piessens et al. 1983).
constexpr double kXgk[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
constexpr double kWgk[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
constexpr double kWg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                           0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

template <class F>
void gk15(const F &f, double a, double b, double *val, double *err) {
  const double c = 0.5 * (a + b), h = 0.5 * (b - a);
  const double fc = f(c);
  double rk = fc * kWgk[7], rg = fc * kWg[3];
  for (int j = 0; j < 7; ++j) {
    const double x = h * kXgk[j];
    const double s = f(c - x) + f(c + x);
    rk += kWgk[j] * s;
    if (j & 1) rg += kWg[j / 2] * s;
  }
  *val = rk * h;
  *err = std::fabs((rk - rg) * h);
}

// Globally adaptive bisection until the summed error estimate is below
// max(abs_tol, rel_tol * |total|).
template <class F>
double integrate(const F &f, double a, double b, double rel_tol, double abs_tol) {
  struct Seg { double a, b, v, e; };
  std::vector<Seg> segs;
  double v, e;
  gk15(f, a, b, &v, &e);
  segs.push_back({a, b, v, e});
  for (int it = 0; it < 4000; ++it) {
    double tot = 0, etot = 0;
    size_t worst = 0;
    for (size_t i = 0; i < segs.size(); ++i) {
      tot += segs[i].v;
      etot += segs[i].e;
      if (segs[i].e > segs[worst].e) worst = i;
    }
    if (etot <= std::max(abs_tol, rel_tol * std::fabs(tot))) break;
    const Seg s = segs[worst];
    const double m = 0.5 * (s.a + s.b);
    double v1, e1, v2, e2;
    gk15(f, s.a, m, &v1, &e1);
    gk15(f, m, s.b, &v2, &e2);
    segs[worst] = {s.a, m, v1, e1};
    segs.push_back({m, s.b, v2, e2});
  }
  double tot = 0;
  for (const Seg &s : segs) tot += s.v;
  return tot;
}

double tophat(double x) {
  if (std::fabs(x) < 1e-2) {
    const double x2 = x * x;
    return 1.0 - x2 / 10.0 + x2 * x2 / 280.0 - x2 * x2 * x2 / 15120.0;
  }
  return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

}  // namespace

double Model::E(double a) const {
  return std::sqrt(om / (a * a * a) + ok / (a * a) + ol);
}

double Model::growth_integral(double a) const {
  auto f = [this](double x) {
    if (x <= 0) return 0.0;
    const double xe = x * E(x);
    return 1.0 / (xe * xe * xe);
  };
  return integrate(f, 0.0, a, 1e-13, 0.0);
}

double Model::growth_unnormalised(double a) const { return 2.5 * om * E(a) * growth_integral(a); }

double Model::growth_rate(double a) const {
  const double e2 = E(a) * E(a);
  return -(3.0 * om / (a * a * a) + 2.0 * ok / (a * a)) / (2.0 * e2) +
         5.0 * om / (2.0 * a * a * e2 * growth_unnormalised(a));
}

double Model::transfer(double k) const {
  if (tf == 0) {  // BBKS eq. G3, q = k / (Om h)
    const double q = k / (om * h);
    const double lg = q > 1e-9 ? std::log1p(2.34 * q) / (2.34 * q) : 1.0 - 1.17 * q;
    const double poly = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) +
                        std::pow(6.71 * q, 4);
    return lg * std::pow(poly, -0.25);
  }
  // Eisenstein & Hu 1998, zero-baryon-oscillation form
  const double omh2 = om * h * h, obh2 = ob * h * h, fb = ob / om;
  const double theta = tcmb / 2.7;
  const double s = 44.5 * std::log(9.83 / omh2) / std::sqrt(1.0 + 10.0 * std::pow(obh2, 0.75));
  const double alpha = 1.0 - 0.328 * std::log(431.0 * omh2) * fb +
                       0.38 * std::log(22.3 * omh2) * fb * fb;
  const double ks = 0.43 * k * h * s;
  const double gamma = om * h * (alpha + (1.0 - alpha) / (1.0 + ks * ks * ks * ks));
  const double q = k * theta * theta / gamma;
  const double l0 = std::log(2.0 * 2.71828182845904523536 + 1.8 * q);
  const double c0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
  return l0 / (l0 + c0 * q * q);
}

double Model::shape(double k) const {
  if (tf == 2) {
    if (tab_k.empty() || k < tab_k.front() || k > tab_k.back()) return 0.0;
    size_t i = std::upper_bound(tab_k.begin(), tab_k.end(), k) - tab_k.begin();
    if (i == 0) i = 1;
    if (i >= tab_k.size()) i = tab_k.size() - 1;
    const double x0 = std::log(tab_k[i - 1]), x1 = std::log(tab_k[i]);
    const double y0 = std::log(tab_p[i - 1]), y1 = std::log(tab_p[i]);
    const double t = (std::log(k) - x0) / (x1 - x0);
    return std::exp(y0 + t * (y1 - y0));
  }
  const double t = transfer(k);
  return std::pow(k, ns) * t * t;
}

double Model::variance_shape(double radius) const {
  double lo = std::log(1e-6), hi = std::log(1e3);
  if (tf == 2) {
    lo = std::log(tab_k.front());
    hi = std::log(tab_k.back());
  }
  auto f = [this, radius](double lnk) {
    const double k = std::exp(lnk);
    const double w = tophat(k * radius);
    return k * k * k * shape(k) * w * w;
  };
  const int pieces = 64;
  double rough = 0;
  for (int i = 0; i < pieces; ++i)
    rough += integrate(f, lo + (hi - lo) * i / pieces, lo + (hi - lo) * (i + 1) / pieces, 1e-8, 0.0);
  double tot = 0;
  for (int i = 0; i < pieces; ++i)
    tot += integrate(f, lo + (hi - lo) * i / pieces, lo + (hi - lo) * (i + 1) / pieces, 1e-13,
                     1e-15 * std::fabs(rough));
  return tot / (2.0 * kPi * kPi);
}

void Model::normalise() {
  if (tf == 2 && sigma8 == 0.0) {
    amp = 1.0;
  } else {
    amp = sigma8 * sigma8 / variance_shape(8.0);
  }
}

double Model::power(double k) const { return amp * shape(k); }

double Model::sigma(double radius) const { return std::sqrt(amp * variance_shape(radius)); }

}  // namespace cosmo
}  // namespace gg
