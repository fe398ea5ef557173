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


def _chem_sum_cos_mode(A, N, chem):
    """sum_i f(A cos(2 pi k i / N)) for a mode with k, 2k, 3k, 4k all nonzero
    mod N, from sum cos = sum cos^3 = 0, sum cos^2 = N/2, sum cos^4 = 3N/8."""
    s2, s4 = N / 2.0, 3.0 * N / 8.0
    if chem[0] == "cubic":  # (u^4 - 2u^2 + 1) / 4
        return (A ** 4 * s4 - 2.0 * A ** 2 * s2 + N) / 4.0
    _, rho, ca, cb = chem  # rho ((u^2 - (ca+cb) u + ca cb))^2, odd powers drop
    return rho * (A ** 4 * s4 + ((ca + cb) ** 2 + 2.0 * ca * cb) * A ** 2 * s2 + (ca * cb) ** 2 * N)


@pytest.mark.parametrize("chem", [("cubic",), ("double_well", 5.0, 0.3, 0.7)])
def test_free_energy_of_constant_fields(chem):
    """A constant field has no gradient energy: F = h^d N^d f(c), with f known
    at its wells and elsewhere by hand (cubic: f(0) = 1/4, f(+-1) = 0,
    f(2) = 9/4; double well rho 5, ca .3, cb .7: f(ca) = f(cb) = 0,
    f(0.5) = 5 * 0.2^4, f(0) = 5 * 0.09 * 0.49)."""
    if chem[0] == "cubic":
        table = {0.0: 0.25, 1.0: 0.0, -1.0: 0.0, 2.0: 2.25}
    else:
        table = {0.3: 0.0, 0.7: 0.0, 0.5: 5 * 0.2 ** 4, 0.0: 5 * 0.09 * 0.49}
    for ndim, n, h in [(2, 12, 0.37), (3, 6, 2.5)]:
        for c, f in table.items():
            u = np.full((n,) * ndim, c)
            F = ch.free_energy(u, h, 1.7, chem)
            assert abs(F - h ** ndim * n ** ndim * f) <= 1e-13 * max(1.0, h ** ndim * n ** ndim * f), (c, F)


@pytest.mark.parametrize("chem", [("cubic",), ("double_well", 5.0, 0.3, 0.7)])
@pytest.mark.parametrize("ndim,n,k,h,kappa,A", [(2, 16, 3, 0.25, 2.0, 0.8), (3, 10, 1, 1.5, 0.3, 1.3)])
def test_free_energy_of_a_fourier_mode(chem, ndim, n, k, h, kappa, A):
    """u = A cos(2 pi k i / N) along one axis at a time: the forward-difference
    gradient sum is N^(d-1) A^2 N (2 sin(pi k / N) / h)^2 / 2, so
    F = h^d [ (kappa/2) N^(d-1) A^2 N (2 sin(pi k/N)/h)^2 / 2 + N^(d-1) sum_i f ]
    with sum_i f from the power sums of cos.  A kappa-for-kappa/2 slip, a
    missing h^d or a backward/central difference all break it."""
    grad = n ** (ndim - 1) * A ** 2 * n * (2.0 * np.sin(np.pi * k / n) / h) ** 2 / 2.0
    chem_sum = n ** (ndim - 1) * _chem_sum_cos_mode(A, n, chem)
    expect = h ** ndim * (0.5 * kappa * grad + chem_sum)
    i = np.arange(n)
    for ax in range(ndim):
        shape = [1] * ndim
        shape[ax] = n
        u = np.broadcast_to((A * np.cos(2 * np.pi * k * i / n)).reshape(shape), (n,) * ndim).copy()
        F = ch.free_energy(u, h, kappa, chem)
        assert abs(F - expect) <= 1e-12 * abs(expect), (ax, F, expect)



def test_sbdf1_is_the_first_order_step():
    """SBDF of order one is the first-order IMEX step of Sec. 4.1."""
    u = manufactured.ch_uniform(24, 2, seed=4, amp=0.4)
    a = ch.step_sbdf_fft([u], 1.0 / 24, 2e-5, 1.0, 0.05 ** 2, ("cubic",), 1)
    b = ch.step_fft(u, 1.0 / 24, 2e-5, 1.0, 0.05 ** 2, ("cubic",))
    assert np.allclose(a, b, rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_sbdf_temporal_order_on_a_linear_model(order):
    """With f'(u) = c u every Fourier mode obeys du/dt = M (c lam - kappa lam^2) u
    exactly (lam the discrete Laplacian's symbol); started from exact history,
    the SBDF error at a fixed time falls by 2^order when dt halves."""
    n, h, M, kappa, cc, T = 16, 1.0, 1.0, 0.5, -0.3, 1.0
    rng = np.random.default_rng(0)
    u0 = rng.normal(size=(n, n)) * 0.1
    lam = ch.lap_symbol((n, n), h)
    rate = M * (cc * lam - kappa * lam * lam)
    # keep only the modes whose exact evolution is resolved by the time steps
    keep = np.abs(rate) <= 1.0
    u0 = np.real(np.fft.ifftn(np.fft.fftn(u0) * keep))
    exact = lambda t: np.real(np.fft.ifftn(np.fft.fftn(u0) * np.exp(rate * t)))
    errs = []
    for dt in (0.1, 0.05, 0.025):
        hist = [exact(-j * dt) for j in range(order)]
        for _ in range(int(round(T / dt))):
            new = ch.step_sbdf_fft(hist, h, dt, M, kappa, ("linear", cc), order)
            hist = [new] + hist[:-1]
        errs.append(np.max(np.abs(hist[0] - exact(T))))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) <= 0.2 for r in rates), (errs, rates)


def test_sbdf_conserves_mass():
    """Sum al_j = 1 and the periodic operators annihilate constants: a step
    keeps the (common) mass of its history."""
    u = manufactured.ch_uniform(20, 2, seed=8, amp=0.3)
    hist = [u, np.roll(u, 1, axis=0), np.roll(u, 3, axis=1)]
    for order in (2, 3):
        new = ch.step_sbdf_fft(hist[:order], 1.0 / 20, 1e-5, 1.0, 0.03 ** 2, ("cubic",), order)
        assert abs(new.sum() - u.sum()) <= 1e-12 * np.abs(u).sum()
