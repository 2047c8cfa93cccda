"""Expansion factor a(t) and da/dt, used by drivers to supply a and adot per step (a = 1 today).

* ``FlatLCDM``: matter and a cosmological constant, closed form
  a = (Om/OL)^{1/3} sinh^{2/3}(3/2 sqrt(OL) H0 t).
* ``LambdaFree``: the Lambda = 0 models of the verification problem (Omega_m = 2 q0): for
  q0 = 1/2 (Einstein-de Sitter) a = (3/2 H0 t)^{2/3}; for q0 < 1/2 (open) the cycloid solution
  of the Friedmann equation a = A (cosh u - 1), H0 t = B (sinh u - u), A = Om / (2 (1 - Om)),
  B = Om / (2 (1 - Om)^{3/2}) (Peebles 1993, Eqs. 13-3 and 13-10, which the paper names).
"""
import math

H100 = 100.0 * 1e5 / 3.0856775814913673e24   # 100 km/s/Mpc in 1/s


class FlatLCDM:
    """Flat matter + Lambda expansion; times in seconds since the big bang."""

    def __init__(self, Omega_m=0.3, Omega_L=0.7, h=0.7, **_):
        self.Om, self.OL = Omega_m, Omega_L
        self.H0 = h * H100

    def a(self, t):
        """Scale factor at time t."""
        return (self.Om / self.OL) ** (1.0 / 3.0) * math.sinh(1.5 * math.sqrt(self.OL) * self.H0 * t) ** (2.0 / 3.0)

    def adot(self, t):
        """da/dt = H0 a sqrt(Om / a^3 + OL)."""
        a = self.a(t)
        return self.H0 * a * math.sqrt(self.Om / a**3 + self.OL)

    def t_of_z(self, z):
        """Time at redshift z."""
        a = 1.0 / (1.0 + z)
        return 2.0 / (3.0 * math.sqrt(self.OL) * self.H0) * math.asinh(math.sqrt(self.OL / self.Om) * a**1.5)


def _sinh_minus_x(u):
    """sinh u - u without cancellation for small u."""
    if u < 1e-2:
        u2 = u * u
        return u * u2 / 6.0 * (1.0 + u2 / 20.0 * (1.0 + u2 / 42.0))
    return math.sinh(u) - u


class LambdaFree:
    """Lambda = 0 expansion with Omega_m = 2 q0 (0 < q0 <= 1/2); times in seconds since the
    big bang."""

    def __init__(self, q0, h, **_):
        self.q0 = q0
        self.Om = 2.0 * q0
        self.H0 = h * H100
        if not 0.0 < self.Om <= 1.0:
            raise ValueError("LambdaFree covers 0 < q0 <= 1/2")
        self.eds = abs(self.Om - 1.0) < 1e-12
        if not self.eds:
            self.A = self.Om / (2.0 * (1.0 - self.Om))
            self.B = self.Om / (2.0 * (1.0 - self.Om) ** 1.5)

    def a(self, t):
        """Scale factor at time t (the cycloid's u by Newton's method when open)."""
        if self.eds:
            return (1.5 * self.H0 * t) ** (2.0 / 3.0)
        y = self.H0 * t / self.B
        # B (sinh u - u) = H0 t is increasing and convex in u: Newton from u^3/6 >= y's root side
        u = (6.0 * y) ** (1.0 / 3.0)
        for _ in range(100):
            f = _sinh_minus_x(u) - y
            step = f / (math.cosh(u) - 1.0)
            u -= step
            if abs(step) <= 1e-15 * u:
                break
        return self.A * (math.cosh(u) - 1.0)

    def adot(self, t):
        """da/dt = H0 a sqrt(Om / a^3 + (1 - Om) / a^2)."""
        a = self.a(t)
        return self.H0 * a * math.sqrt(self.Om / a**3 + (1.0 - self.Om) / a**2)

    def t_of_z(self, z):
        """Time at redshift z."""
        a = 1.0 / (1.0 + z)
        if self.eds:
            return 2.0 / (3.0 * self.H0) * a**1.5
        u = math.acosh(1.0 + a / self.A)
        return self.B * _sinh_minus_x(u) / self.H0


def from_dict(c):
    """The expansion history a workload names: keys q0, h (Lambda-free) or Omega_m, Omega_L, h."""
    return LambdaFree(**c) if "q0" in c else FlatLCDM(**c)
