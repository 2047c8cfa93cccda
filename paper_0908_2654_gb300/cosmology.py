"""Expansion factor a(t) and da/dt for flat LCDM (Friedmann equation with matter and a
cosmological constant, closed form), used by drivers to supply a and adot per step."""
import math

H100 = 100.0 * 1e5 / 3.0856775814913673e24   # 100 km/s/Mpc in 1/s


class FlatLCDM:
    def __init__(self, Omega_m=0.3, Omega_L=0.7, h=0.7, **_):
        self.Om, self.OL = Omega_m, Omega_L
        self.H0 = h * H100

    def a(self, t):
        return (self.Om / self.OL) ** (1.0 / 3.0) * math.sinh(1.5 * math.sqrt(self.OL) * self.H0 * t) ** (2.0 / 3.0)

    def adot(self, t):
        a = self.a(t)
        return self.H0 * a * math.sqrt(self.Om / a**3 + self.OL)

    def t_of_z(self, z):
        a = 1.0 / (1.0 + z)
        return 2.0 / (3.0 * math.sqrt(self.OL) * self.H0) * math.asinh(math.sqrt(self.OL / self.Om) * a**1.5)
