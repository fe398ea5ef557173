"""Pins of the oracle's Cahn-Hilliard step (Sec. 4)."""
import numpy as np
import pytest

from oracle import apply as ap
from oracle import ch
from synth_inputs import manufactured


@pytest.mark.parametrize("ndim,n,eps,dt", [(2, 32, 0.01, 1e-6), (2, 24, 0.05, 1e-4), (3, 12, 0.02, 1e-6)])
def test_cg_step_matches_dft_closed_form(ndim, n, eps, dt):
    """The periodic operators are diagonal in the DFT basis, so the IMEX step
    has the closed form of ch.step_fft; the CG solve must agree."""
    h = 1.0 / n
    u = manufactured.ch_uniform(n, ndim, seed=7)
    chem = ("cubic",)
    un, it, res, ok = ch.step(u, h, dt, 1.0, eps * eps, chem, rtol=1e-13)
    uf = ch.step_fft(u, h, dt, 1.0, eps * eps, chem)
    assert ok
    assert np.max(np.abs(un - uf)) <= 1e-10 * np.max(np.abs(uf))


def test_laplacian_matches_symbol():
    n = 20
    h = 1.0 / n
    lap_w, _ = ch.operators(2, h)
    v = manufactured.ch_uniform(n, 2, seed=3)
    direct = ap.apply(lap_w, v, "periodic")
    spec = np.real(np.fft.ifftn(ch.lap_symbol(v.shape, h) * np.fft.fftn(v)))
    assert np.allclose(direct, spec, rtol=0, atol=1e-9 * np.max(np.abs(direct)))


def test_mass_is_conserved_and_energy_decreases():
    n, eps, dt = 64, 0.02, 2e-6
    h = 1.0 / n
    u = manufactured.ch_uniform(n, 2, seed=11, amp=0.5)
    m0 = ch.mass(u)
    s0 = np.sum(np.abs(u))
    E = [ch.free_energy(u, h, eps * eps, ("cubic",))]
    for _ in range(3):
        u, it, res, ok = ch.step(u, h, dt, 1.0, eps * eps, ("cubic",), rtol=1e-12)
        assert ok
        assert abs(ch.mass(u) - m0) / s0 <= 1e-12
        E.append(ch.free_energy(u, h, eps * eps, ("cubic",)))
    assert all(E[i + 1] < E[i] for i in range(3)), E


def test_double_well_matches_closed_form():
    """The benchmark free energy of Sec. 4.1 (rho = 5, ca = 0.3, cb = 0.7,
    kappa = 2, M = 5) on the cosine initial data, one step."""
    n, L = 50, 200.0
    h = L / n
    c = manufactured.ch_spinodal_ic(n, 2, L)
    chem = ("double_well", 5.0, 0.3, 0.7)
    cn, it, res, ok = ch.step(c, h, 0.05, 5.0, 2.0, chem, rtol=1e-13)
    cf = ch.step_fft(c, h, 0.05, 5.0, 2.0, chem)
    assert ok and np.max(np.abs(cn - cf)) < 1e-10
    # f' of the double well vanishes at the wells and the barrier top
    assert np.allclose(ch.fprime(np.array([0.3, 0.5, 0.7]), chem), 0.0)
