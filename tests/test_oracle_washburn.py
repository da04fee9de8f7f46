"""The imbibition ODE of Section 3.4.1 (RK4, oracle/washburn.py) against its
closed-form limits and its own order of convergence."""
import math

from oracle import washburn

SIG, TH, H, L = 0.05, math.radians(19.0), 28.0, 300.0


def test_lucas_washburn_limit():
    # small inertia (velocity relaxation time rho H^2 / (12 mu) = 0.13 << t), no vapour
    # viscosity: l^2 = sigma H cos(theta) t / (3 mu_l)
    mu = 0.5
    ts = [2000.0, 8000.0]
    ls = washburn.meniscus(ts, SIG, TH, H, L, 1e-3, 1e-6, mu, 0.0, dt=0.05)
    for t, l in zip(ts, ls):
        exact = math.sqrt(SIG * H * math.cos(TH) * t / (3 * mu))
        assert abs(l - exact) / exact < 2e-3


def test_equal_viscosity_gives_constant_speed():
    mu = 0.4
    ts = [1000.0, 5000.0]
    ls = washburn.meniscus(ts, SIG, TH, H, L, 1e-3, 1e-3, mu, mu, dt=0.05)
    speed = SIG * H * math.cos(TH) / (6 * mu * L)
    for t, l in zip(ts, ls):
        assert abs(l - speed * t) / (speed * t) < 1e-3


def test_inviscid_limit_moves_at_constant_speed():
    # d/dt(rho_l l l') = 2 sigma cos(theta) / H with l l' = 0 at t = 0:
    # l = t sqrt(2 sigma cos(theta) / (H rho_l)) (a small vapour mass, 0.3 % of the
    # liquid column at t = 50, regularises t = 0)
    rho = 1.0
    ts = [50.0, 200.0]
    ls = washburn.meniscus(ts, SIG, TH, H, L, rho, 1e-5, 0.0, 0.0, dt=0.01)
    v = math.sqrt(2 * SIG * math.cos(TH) / (H * rho))
    for t, l in zip(ts, ls):
        assert abs(l - v * t) / (v * t) < 2e-3


def test_fourth_order_convergence():
    args = (SIG, TH, H, L, 0.35, 0.02, 0.1, 0.007)
    t = [3000.0]
    ref = washburn.meniscus(t, *args, dt=0.25)[0]
    e1 = abs(washburn.meniscus(t, *args, dt=8.0)[0] - ref)
    e2 = abs(washburn.meniscus(t, *args, dt=4.0)[0] - ref)
    assert 10.0 < e1 / e2 < 22.0
