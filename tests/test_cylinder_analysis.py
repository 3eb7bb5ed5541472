"""The cylinder runner's analysis of the force history (host code, no GPU):
the Strouhal number and the lift and drag amplitudes from the spectrum of
C_L and C_D (Eq. 18's coefficients), on synthetic histories whose answers
are known: a pure lift sinusoid with a drag oscillation at twice its
frequency, then the same under strong high-frequency noise of the size the
weakly compressible force carries, on a non-uniform sampling grid."""
import numpy as np
import pytest

from paper_2411_13992_gb300 import cylinder


def test_coefficients_of_eq18():
    cd, cl = cylinder.coefficients(np.array([0.74, -0.2, 0.0]), rho0=1.0, U=1.0, D=1.0)
    assert cd == pytest.approx(1.48) and cl == pytest.approx(-0.4)
    cd, cl = cylinder.coefficients(np.array([3.0, 1.0, 0.0]), rho0=2.0, U=1.5, D=2.0)
    assert cd == pytest.approx(2 * 3.0 / (2.0 * 2.25 * 2.0)) and cl == pytest.approx(2 * 1.0 / (2.0 * 2.25 * 2.0))


def test_strouhal_and_amplitudes_of_a_known_signal():
    t = np.linspace(0.0, 120.0, 7200)
    st, al, ad = 0.178, 0.405, 0.015
    cl = al * np.sin(2 * np.pi * st * t)
    cd = 1.48 + ad * np.sin(4 * np.pi * st * t + 0.3)
    r = cylinder.shedding(t, cl, cd)
    assert r["St"] == pytest.approx(st, rel=0.01)
    assert r["C_L_amplitude"] == pytest.approx(al, rel=0.03)
    assert r["C_D_amplitude"] == pytest.approx(ad, rel=0.05)


def test_strouhal_under_acoustic_noise_on_a_nonuniform_grid():
    rng = np.random.default_rng(3)
    dt = rng.uniform(0.015, 0.02, 6000)
    t = np.cumsum(dt)
    st, al = 0.16, 0.25
    noise = 1.0 * np.sin(2 * np.pi * 5.3 * t) + 0.8 * np.sin(2 * np.pi * 11.0 * t + 1.0) + rng.normal(0, 0.5, len(t))
    cl = 0.05 + al * np.sin(2 * np.pi * st * t) + noise
    r = cylinder.shedding(t, cl, 1.4 + 0.0 * t)
    assert r["St"] == pytest.approx(st, rel=0.03)
    assert r["C_L_amplitude"] == pytest.approx(al, rel=0.3)
