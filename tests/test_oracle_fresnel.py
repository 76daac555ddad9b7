"""Pins for the oracle's reflection coefficients (Sec. II-B.1, Eq. 6-8).

The paper does not print the Fresnel formula; these checks come from the
textbook forms through Snell's law, the Brewster angle, energy conservation,
the PEC limit and the Rayleigh roughness factor written in wavelengths.
"""
import numpy as np
import pytest

import oracle

C0 = 299792458.0
EPS0 = 8.8541878128e-12


def test_normal_incidence_is_n1_minus_n2_over_sum():
    # (n1 - n2)/(n1 + n2) with n1 = 1, n2 = sqrt(eta), complex for a lossy medium
    for er, sig, f in [(5.31, 0.48, 28e9), (6.27, 0.1, 300e9), (3.0, 0.01, 100e9), (2.25, 0.0, 1e9)]:
        te, tm = oracle.fresnel(er, sig, f, 1.0)
        n2 = np.sqrt(er - 1j * sig / (2 * np.pi * f * EPS0))
        ref = (1 - n2) / (1 + n2)
        assert abs(te - ref) < 1e-14
        assert abs(tm + ref) < 1e-14  # TM = -TE at normal incidence in this sign convention


def test_textbook_forms_through_snell_lossless():
    n = np.sqrt(5.31)
    for th in np.radians([0.0, 10.0, 33.0, 60.0, 80.0, 89.0]):
        tt = np.arcsin(np.sin(th) / n)
        rs = (np.cos(th) - n * np.cos(tt)) / (np.cos(th) + n * np.cos(tt))
        rp = (n * np.cos(th) - np.cos(tt)) / (n * np.cos(th) + np.cos(tt))
        te, tm = oracle.fresnel(5.31, 0.0, 28e9, np.cos(th))
        assert abs(te - rs) < 1e-13 and abs(tm - rp) < 1e-13


def test_brewster_zero_tm():
    for er in (2.25, 3.0, 5.31, 6.27):
        thb = np.arctan(np.sqrt(er))
        te, tm = oracle.fresnel(er, 0.0, 10e9, np.cos(thb))
        assert abs(tm) < 1e-14
        assert abs(te) > 0.05


def test_energy_conservation_lossless():
    er = 6.27
    for th in np.radians(np.linspace(0, 89.5, 40)):
        c = np.cos(th)
        k = np.sqrt(er - np.sin(th) ** 2)
        te, tm = oracle.fresnel(er, 0.0, 10e9, c)
        t_te = 2 * c / (c + k)
        t_tm = 2 * np.sqrt(er) * c / (er * c + k)
        assert abs(abs(te) ** 2 + (k / c) * t_te ** 2 - 1) < 1e-12
        assert abs(abs(tm) ** 2 + (k / c) * t_tm ** 2 - 1) < 1e-12


def test_magnitude_at_most_one_lossy():
    rng = np.random.default_rng(0)
    for _ in range(500):
        er = rng.uniform(1.0, 20.0)
        sig = 10 ** rng.uniform(-4, 2)
        f = 10 ** rng.uniform(8, 12)
        c = rng.uniform(1e-6, 1.0)
        te, tm = oracle.fresnel(er, sig, f, c)
        assert abs(te) <= 1 + 1e-14 and abs(tm) <= 1 + 1e-14


def test_pec_limit_and_grazing():
    te, tm = oracle.fresnel(1.0, 1e12, 1e9, 0.6)
    assert abs(te + 1) < 1e-6 and abs(tm - 1) < 1e-6
    te, tm = oracle.fresnel(5.31, 0.48, 28e9, 1e-9)
    assert abs(te + 1) < 1e-8 and abs(tm + 1) < 1e-7


def test_roughness_factor():
    # Eq. 6-7 in wavelengths: rho = exp(-8 pi^2 sigma_h^2 cos^2 / lambda^2)
    for h, f, c in [(0.0, 3e11, 0.7), (1e-4, 3e11, 1.0), (3e-4, 1e11, 0.3), (5e-5, 3.5e11, 0.9)]:
        lam = C0 / f
        ref = np.exp(-8 * np.pi ** 2 * h ** 2 * c ** 2 / lam ** 2)
        assert abs(oracle.roughness(h, f, c) - ref) < 1e-14
    assert oracle.roughness(0.0, 1e12, 1.0) == 1.0
    assert oracle.roughness(3e-4, 3e11, 0.0) == 1.0
    r = [oracle.roughness(2e-4, 3e11, c) for c in np.linspace(0.0, 1.0, 11)]
    assert all(0 < x <= 1 for x in r) and all(np.diff(r) < 0)
