"""Meniscus position of horizontal imbibition in a slit (Section 3.4.1,
Eq. lucas_washburn_ode), solved with the classical fourth-order Runge-Kutta
scheme from l(0) = 0, dl/dt(0) = 0 as in the paper.

Test infrastructure: only tests import this module.

The printed equation is garbled: its viscous term lacks dl/dt, and its
second-order inertia term carries the total mass instead of the density jump.
This module takes the momentum balance of the liquid column l and the vapour
column L - l in a slit of width H, which is what the printed terms abbreviate:

  d/dt{[rho_l l + rho_v (L - l)] dl/dt} = 2 sigma cos(theta) / H
                                          - (12 / H^2) [mu_l l + mu_v (L - l)] dl/dt
i.e.
  [rho_l l + rho_v (L - l)] l'' + (rho_l - rho_v) l'^2
      + (12 / H^2) [mu_l l + mu_v (L - l)] l' = 2 sigma cos(theta) / H.

Its limits are closed forms, which the tests use as pins: Lucas-Washburn
l^2 = sigma H cos(theta) t / (3 mu_l) (no inertia, no vapour viscosity), constant
speed sigma H cos(theta) / (6 mu L) (equal viscosities, no inertia), and
l = t sqrt(2 sigma cos(theta) / (H rho_l)) (no viscosity, no vapour mass).
"""
import math


def rhs(state, sigma, theta, H, L, rho_l, rho_v, mu_l, mu_v):
    l, v = state
    drive = 2.0 * sigma * math.cos(theta) / H
    mass = rho_l * l + rho_v * (L - l)
    visc = 12.0 / (H * H) * (mu_l * l + mu_v * (L - l))
    return v, (drive - (rho_l - rho_v) * v * v - visc * v) / mass


def meniscus(times, sigma, theta, H, L, rho_l, rho_v, mu_l, mu_v, dt):
    """l(t) at the given (ascending) times, RK4 with step dt (the last step before
    each output time is shortened to land on it)."""
    out = []
    t, state = 0.0, (0.0, 0.0)
    args = (sigma, theta, H, L, rho_l, rho_v, mu_l, mu_v)
    for target in times:
        while t < target - 1e-12:
            h = min(dt, target - t)
            k1 = rhs(state, *args)
            k2 = rhs((state[0] + 0.5 * h * k1[0], state[1] + 0.5 * h * k1[1]), *args)
            k3 = rhs((state[0] + 0.5 * h * k2[0], state[1] + 0.5 * h * k2[1]), *args)
            k4 = rhs((state[0] + h * k3[0], state[1] + h * k3[1]), *args)
            state = (state[0] + h / 6.0 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]),
                     state[1] + h / 6.0 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]))
            t += h
        out.append(state[0])
    return out
