// FP64 cosmology model of the host runtime (see gg_cosmo.cpp).
#pragma once

#include <vector>

namespace gg {
namespace cosmo {

struct Model {
  double om = 0.3, ol = 0.7, ok = 0.0, ob = 0.049, h = 0.7, ns = 1.0, sigma8 = 0.8, tcmb = 2.7255;
  int tf = 0;  // 0 BBKS, 1 EH no-wiggle, 2 table
  std::vector<double> tab_k, tab_p;
  double amp = 1.0;

  double E(double a) const;                    // H(a)/H0
  double growth_integral(double a) const;      // int_0^a da'/(a'E)^3
  double growth_unnormalised(double a) const;  // (5 Om/2) E(a) int_0^a ...
  double growth(double a) const { return growth_unnormalised(a) / growth_unnormalised(1.0); }
  double growth_rate(double a) const;          // dlnD/dlna
  double transfer(double k) const;             // T(k), k in h/Mpc
  double shape(double k) const;                // unnormalised P(k, 0)
  double variance_shape(double radius) const;  // sigma^2(R) of the shape (A = 1)
  void normalise();                            // sets amp from sigma8
  double power(double k) const;                // normalised P(k, 0)
  double sigma(double radius) const;
};

}  // namespace cosmo
}  // namespace gg
