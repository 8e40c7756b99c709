"""The paper's printed constants (tests/golden/paper_printed_constants.json)
against the oracle and the derivations they come from."""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import sgpic_oracle as O

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_printed_constants.json")))


def test_appendix_b_constants_by_quadrature():
    h = 0.37
    S = lambda z: max(0.0, 1.0 - abs(z) / h) / h
    m2 = quad(lambda z: 0.5 * z * z * S(z), -h, h)[0]
    assert m2 / h ** 2 == pytest.approx(G["cic_second_moment"]["value"], rel=1e-12)
    s2 = quad(lambda z: S(z) ** 2, -h, h)[0]  # = (2/3)/h
    assert s2 * h == pytest.approx(G["noise_1d"]["value"], rel=1e-12)
    assert (s2 * h) ** 2 == pytest.approx(G["noise_2d"]["value"], rel=1e-12)
    assert (s2 * h) ** 3 == pytest.approx(G["noise_3d"]["value"], rel=1e-12)
    assert G["cic_second_moment"]["value"] ** 2 == pytest.approx(G["mixed_2d"]["value"], rel=1e-12)
    assert G["cic_second_moment"]["value"] ** 3 == pytest.approx(G["mixed_3d"]["value"], rel=1e-12)


def test_grid_constant_factors_from_derivation():
    """Section 4.3.3: two transfers plus the regular deposit give 3 x 1/12 on
    second derivatives, 2 x 1/144 and 2 x 1/1728 on the mixed terms."""
    assert 3 * G["cic_second_moment"]["value"] == pytest.approx(G["kappa_factor"]["value"])
    assert 2 * G["mixed_2d"]["value"] == pytest.approx(G["beta_factor"]["value"])
    assert 2 * G["mixed_3d"]["value"] == pytest.approx(G["gamma_factor"]["value"])


def test_oracle_uses_printed_factors():
    n, L = 5, 1.0
    N = 2 ** n
    X = np.meshgrid(np.arange(N) / N, np.arange(N) / N, np.arange(N) / N, indexing="ij")
    k = 2 * math.pi
    rho = -1.0 + 0.1 * np.cos(k * X[0]) * np.cos(k * X[1]) * np.cos(k * X[2])
    _, _, c = O.tau_estimator(rho, Np=1e6, L=L, alpha=0.0, pc_ref=1, Qe=-1.0)
    A = 0.1
    assert c["kappa"][0] == pytest.approx(G["kappa_factor"]["value"] * k ** 2 * A, rel=1e-9)
    assert c["beta"][0] == pytest.approx(G["beta_factor"]["value"] * k ** 4 * A, rel=1e-9)
    assert c["gamma"] == pytest.approx(G["gamma_factor"]["value"] * k ** 6 * A, rel=1e-8)
    assert c["sigma"] == pytest.approx(math.sqrt(G["noise_3d"]["value"] * 1.0 * 1.1), rel=1e-12)


def test_tau_range_printed():
    for n in range(4, 12):
        assert O.tau_range(2, n)[-1] == n - 3
        assert O.tau_range(3, n)[-1] == n - 2


def test_penning_workload_matches_printed_parameters():
    """The Penning-trap inputs (box, fields, charge, time step, the moments
    of the Gaussian bunch) against the values Section 5.2 prints."""
    import os
    from paper_2008_09441_gb300 import workloads
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "penning_trap_parameters.json")))
    wl = workloads.penning3d(n_particles=200000, n=6, seed=7)
    L = g["L"]["value"]
    assert wl.L == (L, L, L)
    assert list(wl.B) == g["B_ext"]["value"]
    assert np.allclose(wl.eext_lin, np.array(g["E_ext_linear"]["value"]) / L, rtol=0, atol=1e-15)
    assert wl.dt == g["dt"]["value"]
    assert abs(wl.q.sum() - g["Q_e"]["value"]) < 1e-9 and np.all(wl.q == wl.q[0])
    v = wl.v
    assert np.all(np.abs(v.mean(axis=0)) < 0.01) and np.all(np.abs(v.std(axis=0) - 1.0) < 0.01)
    # positions about the centre in units of L (the tails that wrap around the
    # box, beyond 2.5 standard deviations in z, change the moments by < 2%)
    x = wl.u - 0.5
    assert np.all(np.abs(x.mean(axis=0)) < 0.002)
    assert np.allclose(x.std(axis=0), g["position"]["std_over_L"], rtol=0.02, atol=0)
