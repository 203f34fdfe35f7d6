"""Cosmology inputs of Eq. 1: P(k), sigma_8 normalisation, growth (oracle).

Sec. 2.1 says the generator needs the cosmological parameters and a
tabulated power spectrum. The paper fixes no transfer function and no growth
model. Readings taken (stated here, not in the paper):

* Flat-or-curved LambdaCDM without radiation:
  E(a)^2 = Om a^-3 + Ok a^-2 + OL,  Ok = 1 - Om - OL (OL < 0 means 1 - Om).
* Linear growth (Heath 1977): D_u(a) = (5 Om / 2) E(a) int_0^a da'/(a' E)^3,
  normalised to D(1) = 1. Growth rate f = dlnD/dlna, in closed form
  f = -(3 Om a^-3 + 2 Ok a^-2) / (2 E^2) + 5 Om / (2 a^2 E^2 D_u).
* P(k, z=0) = A k^n_s T(k)^2, A fixed by sigma(R = 8 Mpc/h) = sigma_8 with
  the real-space top-hat window W(x) = 3 (sin x - x cos x) / x^3.
  P(k, z) = D(z)^2 P(k, 0).
* BBKS transfer function (Bardeen, Bond, Kaiser, Szalay 1986, eq. G3) with
  q = k / (Om h), k in h/Mpc, no baryon correction.
* Eisenstein & Hu 1998 (ApJ 496, 605) "no-wiggle" transfer function,
  eqs. 26, 28-31.
* Peculiar velocity per unit displacement: v = a H f psi = 100 a E f psi
  km/s for psi in Mpc/h (Sec. 2.2 gives x = q - D/(a Ddot) v, i.e. the
  velocity field and the displacement differ by the factor a Ddot / D).

All arithmetic FP64; integrals by scipy.integrate.quad.
"""
import math

import numpy as np
from scipy import integrate

SIGMA_R = 8.0  # Mpc/h, the radius in the definition of sigma_8 (Sec. 2.1 footnote)


class Cosmology:
    """Plain parameter holder plus the FP64 functions of the oracle."""

    def __init__(self, omega_m, h, n_s, sigma_8, tf="bbks", omega_l=-1.0,
                 omega_b=0.049, t_cmb=2.7255, tab_k=None, tab_p=None):
        self.omega_m = float(omega_m)
        self.omega_l = float(1.0 - omega_m if omega_l < 0 else omega_l)
        self.omega_k = 1.0 - self.omega_m - self.omega_l
        self.omega_b = float(omega_b)
        self.h = float(h)
        self.n_s = float(n_s)
        self.sigma_8 = float(sigma_8)
        self.t_cmb = float(t_cmb)
        self.tf = tf
        self.tab_k = None if tab_k is None else np.asarray(tab_k, dtype=np.float64)
        self.tab_p = None if tab_p is None else np.asarray(tab_p, dtype=np.float64)
        self._amp = None

    # ---------------------------------------------------------------- background
    def E(self, a):
        """Dimensionless Hubble rate H(a)/H0."""
        a = np.asarray(a, dtype=np.float64)
        return np.sqrt(self.omega_m / a ** 3 + self.omega_k / a ** 2 + self.omega_l)

    def _growth_integral(self, a):
        f = lambda x: 1.0 / (x * self.E(x)) ** 3 if x > 0 else 0.0
        val, _ = integrate.quad(f, 0.0, a, epsabs=0.0, epsrel=1e-13, limit=500)
        return val

    def growth_unnormalised(self, a):
        """D_u(a) = (5 Om/2) E(a) int_0^a da'/(a'E)^3 (equals a in EdS)."""
        return 2.5 * self.omega_m * float(self.E(a)) * self._growth_integral(a)

    def growth(self, a):
        """D(a) / D(1)."""
        return self.growth_unnormalised(a) / self.growth_unnormalised(1.0)

    def growth_rate(self, a):
        """f = dlnD/dlna from the closed form of the derivative of D_u."""
        e2 = float(self.E(a)) ** 2
        du = self.growth_unnormalised(a)
        return (-(3.0 * self.omega_m / a ** 3 + 2.0 * self.omega_k / a ** 2) / (2.0 * e2)
                + 5.0 * self.omega_m / (2.0 * a * a * e2 * du))

    def velocity_factor(self, a):
        """v [km/s] per unit displacement psi [Mpc/h]: 100 a E(a) f(a)."""
        return 100.0 * a * float(self.E(a)) * self.growth_rate(a)

    # ---------------------------------------------------------- transfer function
    @staticmethod
    def bbks_of_q(q):
        """BBKS eq. G3 as a function of q:
        T = ln(1 + 2.34 q)/(2.34 q) [1 + 3.89 q + (16.1 q)^2 + (5.46 q)^3 + (6.71 q)^4]^(-1/4).
        Pinned by its series at q -> 0 and its asymptote at q -> infinity."""
        q = np.asarray(q, dtype=np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            lg = np.where(q > 1e-9, np.log1p(2.34 * q) / (2.34 * q), 1.0 - 1.17 * q)
        poly = 1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4
        return lg * poly ** -0.25

    def transfer_bbks(self, k):
        """BBKS eq. G3, q = k/(Om h), k in h/Mpc (no baryon correction)."""
        k = np.asarray(k, dtype=np.float64)
        return self.bbks_of_q(k / (self.omega_m * self.h))

    def eh_sound_horizon(self):
        """EH98 eq. 26 approximation of the sound horizon s [Mpc].
        Parity unpinned beyond the check against the measured drag-epoch
        sound horizon (3%): its coefficients are an input definition."""
        om_h2 = self.omega_m * self.h ** 2
        ob_h2 = self.omega_b * self.h ** 2
        return 44.5 * math.log(9.83 / om_h2) / math.sqrt(1.0 + 10.0 * ob_h2 ** 0.75)

    @staticmethod
    def eh_t0_of_q(q):
        """EH98 eqs. 29 (the zero-baryon shape) as a function of q:
        T0 = L0 / (L0 + C0 q^2), L0 = ln(2e + 1.8 q), C0 = 14.2 + 731/(1 + 62.5 q).
        Pinned by its series at q -> 0 and its asymptote at q -> infinity."""
        q = np.asarray(q, dtype=np.float64)
        l0 = np.log(2.0 * math.e + 1.8 * q)
        c0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
        return l0 / (l0 + c0 * q * q)

    def eh_gamma_eff(self, k):
        """EH98 eqs. 30-31: the effective shape Gamma_eff(k) (k in h/Mpc),
        with q = k Theta^2 / Gamma_eff. Pinned only by its limits
        Gamma_eff -> Om h (k -> 0) and Om h alpha (k -> infinity), alpha = 1
        without baryons; alpha's coefficients are an input definition
        (parity unpinned)."""
        k = np.asarray(k, dtype=np.float64)
        om_h2 = self.omega_m * self.h ** 2
        fb = self.omega_b / self.omega_m
        s = self.eh_sound_horizon()
        alpha = 1.0 - 0.328 * math.log(431.0 * om_h2) * fb + 0.38 * math.log(22.3 * om_h2) * fb * fb
        kmpc = k * self.h  # 1/Mpc
        return self.omega_m * self.h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * kmpc * s) ** 4))

    def transfer_eh_nowiggle(self, k):
        """EH98 eqs. 28-31 (zero-baryon-oscillation shape), k in h/Mpc."""
        k = np.asarray(k, dtype=np.float64)
        theta = self.t_cmb / 2.7
        return self.eh_t0_of_q(k * theta * theta / self.eh_gamma_eff(k))

    def _shape(self, k):
        """Unnormalised P(k, 0) shape (the amplitude A is applied separately)."""
        k = np.asarray(k, dtype=np.float64)
        if self.tf == "bbks":
            return k ** self.n_s * self.transfer_bbks(k) ** 2
        if self.tf == "eh_nw":
            return k ** self.n_s * self.transfer_eh_nowiggle(k) ** 2
        if self.tf == "table":
            lk = np.log(self.tab_k)
            lp = np.log(self.tab_p)
            inside = (k >= self.tab_k[0]) & (k <= self.tab_k[-1])
            out = np.zeros_like(k)
            kk = np.where(inside, k, self.tab_k[0])
            out[inside] = np.exp(np.interp(np.log(kk), lk, lp))[inside]
            return out
        raise ValueError(self.tf)

    # ------------------------------------------------------------- normalisation
    @staticmethod
    def tophat(x):
        """Fourier transform of the unit real-space top hat, 3 j_1(x)/x."""
        x = np.asarray(x, dtype=np.float64)
        small = np.abs(x) < 1e-2
        xs = np.where(small, 1.0, x)
        full = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
        x2 = x * x
        series = 1.0 - x2 / 10.0 + x2 * x2 / 280.0 - x2 * x2 * x2 / 15120.0
        return np.where(small, series, full)

    def variance(self, pk, radius, window=None, kmin=1e-6, kmax=1e3, breaks=None):
        """sigma^2(R) = 1/(2 pi^2) int_kmin^kmax k^2 P(k) W(kR)^2 dk.

        ``breaks``: the nodes of a piecewise-smooth P (a tabulated spectrum,
        interpolated linearly in log-log); the integral is then taken in ln k
        between consecutive nodes, where the integrand is smooth (a node
        interval holds a few oscillations of the window at most).

        A general window is integrated in ln k on 63 equal pieces. For the
        top hat (window None) that holds only up to x = kR = 10: beyond it
        W(x)^2 oscillates hundreds of times per piece. There the square is
        expanded with the double-angle identities,
            (sin x - x cos x)^2 = (1 + x^2)/2 + (x^2 - 1)/2 cos 2x - x sin 2x,
        so W^2 = 9/x^6 [...] splits into a smooth part (integrated in ln k)
        and two parts with the weights cos(2Rk) and sin(2Rk), which quad
        integrates with its rule for oscillatory weights (QUADPACK QAWO).
        For x >= 10 no term of the expansion cancels another catastrophically.
        """
        tophat = window is None
        window = self.tophat if window is None else window
        norm = 2.0 * math.pi ** 2

        def integrand(lnk):
            k = math.exp(lnk)
            w = float(window(k * radius))
            return k ** 3 * float(pk(k)) * w * w

        k1 = min(max(10.0 / radius, kmin), kmax) if tophat else kmax
        pieces = []
        if breaks is not None:
            nodes = np.unique(np.clip(np.concatenate([[kmin, kmax], np.asarray(breaks, float)]),
                                      kmin, kmax))
            ln = np.log(nodes)
            pieces = [("lnk", integrand, lo, hi) for lo, hi in zip(ln[:-1], ln[1:])]
            k1 = kmax
        elif k1 > kmin:
            edges = np.linspace(math.log(kmin), math.log(k1), 64)
            pieces += [("lnk", integrand, lo, hi) for lo, hi in zip(edges[:-1], edges[1:])]
        if k1 < kmax:
            r = radius
            smooth = lambda lnk: (math.exp(lnk) ** 3 * float(pk(math.exp(lnk))) * 9.0
                                  * (1.0 + (math.exp(lnk) * r) ** 2) / (2.0 * (math.exp(lnk) * r) ** 6))
            amp_c = lambda k: k * k * float(pk(k)) * 9.0 * ((k * r) ** 2 - 1.0) / (2.0 * (k * r) ** 6)
            amp_s = lambda k: -k * k * float(pk(k)) * 9.0 * (k * r) / (k * r) ** 6
            edges = np.linspace(math.log(k1), math.log(kmax), 16)
            pieces += [("lnk", smooth, lo, hi) for lo, hi in zip(edges[:-1], edges[1:])]
            pieces += [("cos", amp_c, k1, kmax), ("sin", amp_s, k1, kmax)]

        def run(kind, f, lo, hi, epsabs, epsrel):
            if kind == "lnk":
                return integrate.quad(f, lo, hi, epsabs=epsabs, epsrel=epsrel, limit=200)[0]
            return integrate.quad(f, lo, hi, weight=kind, wvar=2.0 * radius, epsabs=epsabs,
                                  epsrel=epsrel, limit=400)[0]

        # first pass fixes the scale; the second asks each piece for 1e-15 of it
        rough = sum(abs(run(*pc, 0.0, 1e-8)) for pc in pieces)
        tol = 1e-15 * rough
        return sum(run(*pc, tol, 1e-13) for pc in pieces) / norm

    def amplitude(self):
        """A such that sigma(8 Mpc/h) = sigma_8 at z = 0."""
        if self._amp is None:
            if self.tf == "table" and self.sigma_8 == 0.0:
                self._amp = 1.0
            else:
                kmin, kmax = (1e-6, 1e3)
                if self.tf == "table":
                    kmin, kmax = float(self.tab_k[0]), float(self.tab_k[-1])
                var = self.variance(self._shape, SIGMA_R, kmin=kmin, kmax=kmax,
                                    breaks=self.tab_k if self.tf == "table" else None)
                self._amp = self.sigma_8 ** 2 / var
        return self._amp

    def power(self, k):
        """Normalised linear P(k) at z = 0 [(Mpc/h)^3], k in h/Mpc."""
        return self.amplitude() * self._shape(k)

