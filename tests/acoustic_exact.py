"""Linear-acoustics solution of the 1D acoustic wave of Sec. 4.3 (Eq. acoustic-1d-ref):
the initial velocity perturbation eps a cos(w x) and density perturbation eps rho cos(2 w x)
split into left- and right-running waves.  Cell averages in closed form."""
import math

import numpy as np

EPS, OMEGA, RHO_INF, P_INF = 1e-5, 6.0 * math.pi, 1.1771, 101325.0
X0, X1 = 0.0, 1.0 / 3.0


def sound_speed(gamma=1.4):
    return math.sqrt(gamma * P_INF / RHO_INF)


def cell_average_density(N, t, gamma=1.4):
    a = sound_speed(gamma)
    h = (X1 - X0) / N
    xl = X0 + h * np.arange(N)
    xr = xl + h

    def avg_cos(k, shift):   # cell average of cos(k (x + shift))
        return (np.sin(k * (xr + shift)) - np.sin(k * (xl + shift))) / (k * h)

    w = OMEGA
    return RHO_INF + 0.5 * EPS * RHO_INF * (avg_cos(2 * w, -a * t) + avg_cos(2 * w, a * t)
                                            + avg_cos(w, -a * t) - avg_cos(w, a * t))


def amplitude():
    return EPS * RHO_INF
