"""Pins for the dense brute-force evolution (oracle/dense.py).

Every expected value here comes from mathematics independent of the oracle:
closed forms of commuting dynamics and the free-fermion solution of the chain.
"""
import numpy as np
import pytest

from oracle import dense
from tests.free_fermion import autocorrelation_xxz, autocorrelation_zzx_edge


@pytest.mark.parametrize("order", [1, 2])
def test_zzx_J0_is_cos_2ht(order):
    # exp(-i h dt X) rotates Z into Y: C(t) = cos(2 h t) for any step split.
    h, dt, n = 0.8, 0.05, 12
    r = dense.evolve(3, 2, 0.0, h, dt, order, n, (1, 1))
    t = np.arange(n + 1) * dt
    assert np.max(np.abs(r["C"] - np.cos(2 * h * t))) < 1e-12


def test_zzx_h0_is_one():
    r = dense.evolve(3, 3, 1.3, 0.0, 0.05, 1, 8, (1, 1))
    assert np.max(np.abs(r["C"] - 1.0)) < 1e-12


@pytest.mark.parametrize("obs,deg", [((1, 1), 4), ((1, 0), 3), ((0, 0), 2)])
def test_xxz_h0_is_cos_power_degree(obs, deg):
    # Paper convention: the deg XX bonds at the observable site commute and each
    # anticommutes with Z_c, so C(t) = cos(2 J t)^deg.
    J, dt, n = 1.0, 0.1, 10
    r = dense.evolve(3, 3, J, 0.0, dt, 2, n, obs, gateset="XX_Z")
    t = np.arange(n + 1) * dt
    assert np.max(np.abs(r["C"] - np.cos(2 * J * t) ** deg)) < 1e-12


def test_zzx_h0_edge_x_observable_cos_cubed():
    # X at an edge site under ZZ bonds only: cos(2 J t)^3, negative on (pi/4, 3 pi/4).
    J, dt, n = 1.0, 0.05, 24
    r = dense.evolve(3, 3, J, 0.0, dt, 1, n, (1, 0), obs_pauli="X")
    t = np.arange(n + 1) * dt
    ref = np.cos(2 * J * t) ** 3
    assert ref.min() < -0.05
    assert np.max(np.abs(r["C"] - ref)) < 1e-12


def test_norm_is_preserved():
    r = dense.evolve(3, 3, 0.7, 1.9, 0.07, 2, 6, (0, 2))
    assert np.max(np.abs(r["norm"] - 1.0)) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("j", [0, 2, 5])
def test_xxz_chain_matches_free_fermions(order, j):
    N, J, h, dt, n = 6, 0.9, 1.3, 0.1, 15
    r = dense.evolve(N, 1, J, h, dt, order, n, (j, 0), gateset="XX_Z")
    ff = autocorrelation_xxz(N, j, J, h, dt, order, n)
    assert np.max(np.abs(r["C"] - ff)) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_zzx_chain_edge_matches_free_fermions(order):
    N, J, h, dt, n = 7, 1.0, 0.6, 0.1, 20
    r = dense.evolve(N, 1, J, h, dt, order, n, (0, 0))
    ff = autocorrelation_zzx_edge(N, J, h, dt, order, n)
    assert np.max(np.abs(r["C"] - ff)) < 1e-12
    # the same chain laid out vertically
    r2 = dense.evolve(1, N, J, h, dt, order, n, (0, 0))
    assert np.max(np.abs(r2["C"] - ff)) < 1e-12
