"""Pins of the oracle's carrier statistics and contact potentials (no GPU).

Each pin comes from outside the oracle: the paper's stated error bounds
(tests/golden/paper_values.json), the defining integrals evaluated by adaptive
quadrature, textbook limits, and the charge-neutrality roots the closed forms
are derived from.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import physics as P

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_fd_half_approx_within_paper_bound():
    # Sec. II.A.1: Bednarczyk approximation error < 0.4 % for all x.
    xs = np.concatenate([np.linspace(-60, 20, 161), np.linspace(20, 200, 19)])
    exact = np.array([P.fd_half_integral(x) for x in xs])
    rel = np.abs(P.fd_half(xs) - exact) / exact
    assert rel.max() < GOLD["fd_half_approx_max_rel_error"]["value"]
    # the bound is nearly attained (0.379 % near x = 3.5): a dropped term would show
    assert rel.max() > 0.003


def test_fd_half_limits_and_clamp():
    # x -> -inf: F -> e^x (MB limit); x -> +inf: F -> 4 x^(3/2) / (3 sqrt(pi))
    for x in (-40.0, -49.0, -51.0, -300.0):
        assert abs(P.fd_half(x) / math.exp(x) - 1.0) < 1e-15
    for x in (1e3, 1e4):
        assert abs(P.fd_half(x) / (4.0 * x ** 1.5 / (3.0 * math.sqrt(math.pi))) - 1.0) < 1e-6
    # the clamp at -50 joins the two branches continuously
    c = GOLD["fd_half_clamp_x"]["value"]
    assert P.FD_CLAMP_X == c
    assert abs(P.fd_half(c - 1e-12) / P.fd_half(c + 1e-12) - 1.0) < 1e-10
    # no overflow far into the degenerate or non-degenerate tails
    assert np.all(np.isfinite(P.fd_half(np.array([-1e5, -745.0, 1e5]))))


def test_fd_half_derivative():
    xs = np.linspace(-55, 80, 271)
    d = P.fd_half_deriv(xs)
    h = 1e-5 * np.maximum(1.0, np.abs(xs))
    fd = (P.fd_half(xs + h) - P.fd_half(xs - h)) / (2 * h)
    assert np.max(np.abs(fd - d) / np.abs(d)) < 1e-7
    # the exact derivative of F_1/2 is F_-1/2: the approximation's slope tracks it
    for x in (-10.0, -1.0, 0.0, 2.0, 5.0, 30.0):
        assert abs(P.fd_half_deriv(x) / P.fd_mhalf_integral(x) - 1.0) < 0.015


def test_fd_half_inverse_within_paper_bound():
    from scipy import optimize
    worst = 0.0
    for u in np.logspace(-8, 4, 61):
        eta = optimize.brentq(lambda e: P.fd_half_integral(e) - u, -40, 2000, xtol=1e-13)
        worst = max(worst, abs(P.fd_half_inverse(u) - eta) / max(1.0, abs(eta)))
    assert worst < GOLD["fd_half_inverse_max_error"]["value"]
    assert abs(P.fd_half_inverse(1.0) - P.fd_half_inverse(1.0 + 1e-9)) < 1e-8


def test_effective_dos_textbook_values():
    # Si at 300 K: N_C ~ 2.8e19 cm^-3, N_V ~ 1.04e19 cm^-3 (standard tables); 1 cm^-3 = 1e-21 nm^-3
    NC, NV = P.band_params(W.SI, 300.0)
    assert abs(NC / 2.8e-2 - 1.0) < 0.02
    assert abs(NV / 1.04e-2 - 1.0) < 0.03
    assert abs(P.q_over_eps0() - 18.0951) < 1e-3
    assert abs(P.hbar2_over_2m0() - 0.0380998) < 1e-6


@pytest.mark.parametrize("T", [300.0, 4.0])
def test_phi_ref_is_intrinsic_level(T):
    # q phi_ref = E_0 - E_i(Si): at phi = 0 and E_F = 0 the MB electron and hole densities are equal
    mat = dict(W.SI, N_A=0.0, N_D=0.0)
    pr = P.phi_ref(mat, T)
    t = P.carrier_terms(np.array([0.0]), mat, T, pr, 0.0, statistics=0, incomplete=0)
    if T > 100:
        assert abs(t["n"][0] / t["p"][0] - 1.0) < 1e-12
    else:
        # at 4 K both underflow; compare logarithms of the exponent arguments instead
        kT = P.kT_eV(T)
        NC, NV = P.band_params(mat, T)
        ln_n = math.log(NC) + (0.0 - pr + mat["chi"]) / kT
        ln_p = math.log(NV) + (pr - mat["chi"] - mat["Eg"]) / kT
        assert abs(ln_n - ln_p) < 1e-9 * abs(ln_n)


@pytest.mark.parametrize("T", [300.0, 50.0, 4.0, 0.5])
@pytest.mark.parametrize("ntype", [False, True])
def test_ohmic_contacts_are_neutral_roots(T, ntype):
    mat = dict(W.SI, N_A=0.0, N_D=1e-6) if ntype else dict(W.SI)
    pr = P.phi_ref(mat, T)
    kT = P.kT_eV(T)
    # MB, complete ionization: exact root of n + NA = p + ND (minority carriers negligible)
    r = P.neutral_root(mat, T, pr, 0.0, statistics=0, incomplete=0)
    assert abs(P.ohmic_potential(mat, T, pr, 0.0, statistics=0, incomplete=0) - r) < 1e-10
    # MB, incomplete ionization: the y_n / y_p closed form is the exact root (at this doping its
    # low-T log approximation below 50 K differs by far less than rounding; at 1e13 cm^-3 and 41 K
    # the approximation alone moves the contact by 0.7 mV)
    r = P.neutral_root(mat, T, pr, 0.0, statistics=0, incomplete=1)
    assert abs(P.ohmic_potential(mat, T, pr, 0.0, statistics=0, incomplete=1) - r) < 1e-10
    # FD, complete ionization: the root uses the Bednarczyk F_1/2 (0.4 % in F, about 0.7 % in
    # eta near eta = 0) while the closed form uses Nilsson's inverse (0.6 % in eta)
    r = P.neutral_root(mat, T, pr, 0.0, statistics=1, incomplete=0)
    v = P.ohmic_potential(mat, T, pr, 0.0, statistics=1, incomplete=0)
    eta = abs(r - (pr - mat["chi"] - (0.0 if ntype else mat["Eg"]))) / kT
    assert abs(v - r) <= (0.006 + 0.008) * max(1.0, eta) * kT
    # applied bias shifts the contact rigidly
    assert abs(P.ohmic_potential(mat, T, pr, 0.25, 1, 1) - P.ohmic_potential(mat, T, pr, 0.0, 1, 1) - 0.25) < 1e-14


def test_p_type_incomplete_sign_of_Ea():
    # The printed p-type incomplete-ionization contact carries -E_a; the derivation from y_p
    # (Eq. Yval4MBIncompIon) gives +E_a. The neutral root decides: the two differ by 2 E_a.
    mat = dict(W.SI)
    T = 300.0
    pr = P.phi_ref(mat, T)
    r = P.neutral_root(mat, T, pr, 0.0, statistics=0, incomplete=1)
    v = P.ohmic_potential(mat, T, pr, 0.0, statistics=0, incomplete=1)
    assert abs(v - r) < 1e-10
    assert abs((v - 2 * mat["E_a"]) - r) > 0.08


@pytest.mark.parametrize("T", [300.0, 4.0, 0.5])
@pytest.mark.parametrize("stat", [0, 1])
def test_charge_derivative_and_range_safety(T, stat):
    mat = dict(W.SI, N_D=3e-7)
    pr = P.phi_ref(mat, T)
    kT = P.kT_eV(T)
    if stat == 1:
        phis = np.linspace(-0.7, 1.5, 301)
    else:
        # MB has no overflow safeguard in the paper: stay within 600 kT beyond the band edges
        lo = pr - mat["chi"] - mat["Eg"] - 600 * kT
        hi = pr - mat["chi"] + 600 * kT
        phis = np.linspace(max(-0.7, lo), min(0.75, hi), 301)
    t = P.carrier_terms(phis, mat, T, pr, 0.0, stat, 1)
    for k in ("rho", "drho", "n", "p", "ND", "NA"):
        assert np.all(np.isfinite(t[k])), k
    # -rho' >= 0: the Jacobian's mass term is positive semidefinite
    assert np.all(t["drho"] <= 0.0)
    h = 1e-4 * kT
    tp = P.carrier_terms(phis + h, mat, T, pr, 0.0, stat, 1)
    tm = P.carrier_terms(phis - h, mat, T, pr, 0.0, stat, 1)
    fd = (tp["rho"] - tm["rho"]) / (2 * h)
    # compare where the variation over the step is resolvable against rho itself
    ok = np.abs(t["drho"]) * 2 * h > 1e-8 * np.abs(t["rho"])
    assert ok.sum() >= 10
    assert np.max(np.abs(fd[ok] - t["drho"][ok]) / np.abs(t["drho"][ok])) < 1e-5


def test_ionization_fractions():
    mat = dict(W.SI, N_D=1e-6)
    T = 300.0
    pr = P.phi_ref(mat, T)
    t = P.carrier_terms(np.array([-0.3, 0.0, 0.3]), mat, T, pr, 0.0, 1, 1)
    # g_A = 4, g_D = 2 (Sec. II.A.3): at E_F = E_A exactly one fifth of acceptors is ionized
    kT = P.kT_eV(T)
    phi_at_EA = pr - mat["chi"] - mat["Eg"] + mat["E_a"]  # E_A - E_F = 0
    tA = P.carrier_terms(np.array([phi_at_EA]), mat, T, pr, 0.0, 1, 1)
    assert abs(tA["NA"][0] / mat["N_A"] - 1.0 / 5.0) < 1e-14
    phi_at_ED = pr - mat["chi"] - mat["E_d"]  # E_F - E_D = 0
    tD = P.carrier_terms(np.array([phi_at_ED]), mat, T, pr, 0.0, 1, 1)
    assert abs(tD["ND"][0] / mat["N_D"] - 1.0 / 3.0) < 1e-14
    assert np.all(t["NA"] <= mat["N_A"]) and np.all(t["ND"] <= mat["N_D"])
