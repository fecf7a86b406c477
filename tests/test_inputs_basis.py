"""Pins of the shared input generator (radial grid, hydrogenic functions, wave-packet pseudostates,
state lists, z-grids) against textbook closed forms and invariants.

Parity between the oracle and the CUDA path does not depend on these inputs (both read the same
tables); these tests fix that the tables are what the workloads say they are: the sinh-mapped grid
integrates the hydrogenic functions to their textbook moments, each l-block of a centre is orthonormal
on the grid, the pseudostate energies are the bin averages of k^2/2 and the state counts follow the
all-m rule.
"""
import math

import numpy as np
import pytest

import wpccc_inputs as wi


@pytest.fixture(scope="module")
def grid():
    return wi.radial_grid(2000)


def test_hydrogenic_functions_have_textbook_norm_and_mean_radius(grid):
    # <r> = (3 n^2 - l (l + 1)) / (2 Z): a moment the Laguerre form does not contain explicitly. The grid
    # starts at r_1 ~ 0.01 (the trapezoid rule's r = 0 end carries a zero integrand): the 1s density of
    # charge Z loses ~1e-9 Z^3 there
    wr2 = grid.w * grid.r ** 2
    for Z in (1.0, 2.0):
        for n in range(1, 5):
            for l in range(n):
                R = wi.hydrogenic_radial(n, l, Z, grid.r)
                assert abs(np.sum(wr2 * R * R) - 1.0) < 1e-7, (n, l, Z)
                assert abs(np.sum(wr2 * grid.r * R * R) - (3 * n * n - l * (l + 1)) / (2 * Z)) < 1e-7
                # the radial equation's node count: n - l - 1 sign changes inside the bulk
                bulk = R[grid.r < 4.0 * n * n / Z]
                assert np.count_nonzero(np.diff(np.sign(bulk[np.abs(bulk) > 1e-12])) != 0) == n - l - 1


def _energy(grid, f, l, Z):
    """<f|H|f> with H = -1/2 d^2/dr^2 + l(l+1)/(2 r^2) - Z/r acting on u = r f, in the symmetric form
    1/2 |u'|^2 + V u^2, by the trapezoid rule in the grid's mapped variable with the origin (u = 0)
    added; u' by second-order differences in the mapped variable and the chain rule."""
    Nr = grid.r.size
    x = np.arange(Nr + 1, dtype=np.float64) / Nr
    jac = grid.rmax * grid.alpha * np.cosh(grid.alpha * x) / math.sinh(grid.alpha)
    w = jac / Nr
    w[0] *= 0.5
    w[-1] *= 0.5
    r = np.concatenate([[0.0], grid.r])
    u = np.concatenate([[0.0], grid.r * f])
    du = np.gradient(u, x, edge_order=2) / jac
    V = np.zeros_like(r)
    V[1:] = l * (l + 1) / (2.0 * r[1:] ** 2) - Z / r[1:]
    return float(np.sum(w * (0.5 * du * du + V * u * u)))


def test_centre_blocks_are_orthonormal_with_their_energies(grid):
    nmax, lmax, nbins, kmax = 4, 3, 8, 2.0
    c = wi.make_centre(1.0, nmax, lmax, nbins, kmax, grid)
    wr2 = grid.w * grid.r ** 2
    edges = np.linspace(0.0, kmax, nbins + 1)
    for l in range(lmax + 1):
        sel = np.nonzero(c.rad_l == l)[0]
        assert sel.size == max(nmax - l, 0) + nbins
        G = (c.f[sel] * wr2) @ c.f[sel].T
        assert np.abs(G - np.eye(sel.size)).max() < 1e-8, l
    for i in range(c.n_rad):
        l, n, e = int(c.rad_l[i]), int(c.rad_n[i]), float(c.rad_eps[i])
        got = _energy(grid, c.f[i], l, 1.0)
        if n < 100:
            assert e == -0.5 / (n * n)
            assert abs(got - e) < 5e-4 * abs(e), (n, l, got, e)
        else:
            # the bin's average of k^2/2 over [k_j, k_j+1] (the wave packet is the bin's average of the
            # delta-normalised Coulomb waves, so <H> is that average up to the grid's cut at r_max)
            j = n - 100
            avg = (edges[j + 1] ** 3 - edges[j] ** 3) / (6.0 * (edges[j + 1] - edges[j]))
            assert e == pytest.approx(avg, rel=1e-14)
            assert abs(got - e) < 1.5e-3 * max(e, 1.0), (j, l, got, e)
    # states: every radial function once per m = -l..l, in order
    for i in range(c.n_rad):
        ms = c.st_m[c.st_rad == i]
        l = int(c.rad_l[i])
        assert list(ms) == list(range(-l, l + 1))
        assert np.all(c.st_eps[c.st_rad == i] == c.rad_eps[i])


def _count(nmax, lmax, nbins):
    # all-m counting: (bound states n = l+1..nmax plus the packets) x (2l + 1) per l
    return sum((max(nmax - l, 0) + nbins) * (2 * l + 1) for l in range(lmax + 1))


def test_workload_state_counts():
    assert _count(3, 2, 5) == 59
    assert _count(4, 3, 10) == 190
    assert _count(6, 5, 20) == 811
    assert _count(10, 10, 32) == 4257
    b1, _ = wi.config_inputs("p_H_1c_n3l2", Nr=400)
    assert b1.P is None and b1.N == 59
    b2, p2 = wi.config_inputs("p_H_2c_n4l3", Nr=400)
    assert b2.T.N == b2.P.N == 190 and b2.N == 380
    assert p2.n_paths == 32 and p2.z[0].size == 1001 and np.all(p2.v == 1.5)
    for name, c in wi.CONFIGS.items():
        n = _count(c["nmax"], c["lmax"], c["nbins"])
        assert n * (2 if c["two_centre"] else 1) in (59, 380, 1622, 4257), name


def test_geometric_zgrid_of_section_two():
    # the z-grid with the typical parameters the paper states: z_min = 1e-3, n_z = 500, z_max = 100
    z = wi.geometric_zgrid(1e-3, 100.0, 500)
    assert z.size == 1001 and z[500] == 0.0
    assert np.all(np.diff(z) > 0) and np.array_equal(z[:500], -z[:500:-1])
    assert z[501] == pytest.approx(1e-3 * 1e5 ** (1 / 500), rel=1e-14)
    assert z[-1] == pytest.approx(100.0, rel=1e-14) and z[502] / z[501] == pytest.approx(z[-1] / z[-2], rel=1e-12)


def test_observable_and_cross_section_weights():
    # capture = every bound projectile state, 2p excitation = the target's 2p states (all m)
    b = wi.make_basis(1.0, 1.0, 2, 1, 2, 2.0, True, Nr=300, Geta=8, Gtau=8)
    g = wi.observable_weights(b)
    T, P = b.T, b.P
    assert g.shape == (2, b.N) and set(np.unique(g)) <= {0.0, 1.0}
    assert g[0, :T.N].sum() == 0 and g[0, T.N:].sum() == 2 + 3          # projectile 1s, 2s, 2p(m = -1, 0, 1)
    assert g[1, T.N:].sum() == 0 and g[1, :T.N].sum() == 3              # target 2p(m = -1, 0, 1)
    assert np.all(T.st_l[g[1, :T.N] == 1] == 1)
    # sigma = 2 pi int b P(b) db: exact for P linear in b on [0, b_max] by the trapezoid rule with b = 0
    bs = np.linspace(0.5, 6.0, 12)
    wts = wi.cross_section_weights(bs)
    assert np.isclose(wts @ np.ones_like(bs), np.pi * bs[-1] ** 2)   # P = 1: pi b_max^2 (b P linear)
    # and b P(b) = 0 at the added node b = 0: for P = b the rule's error is the trapezoid's on b^2
    h = np.diff(np.concatenate([[0.0], bs]))
    assert np.isclose(wts @ bs, 2.0 * np.pi * (bs[-1] ** 3 / 3.0 + np.sum(h ** 3) / 6.0))


def test_model_potential_parameters_are_seeded_within_five_percent():
    a0, b0 = wi.li_parameters(0)
    assert (a0, b0) == wi.li_parameters(0)
    for seed in range(20):
        a, b = wi.li_parameters(seed)
        assert abs(a / 3.0 - 1.0) < 0.05 and abs(b / 1.5 - 1.0) < 0.05
    assert wi.li_parameters(1) != (a0, b0)
