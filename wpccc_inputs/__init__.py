"""Seeded / deterministic input generators shared by the oracle and the CUDA path.

This module builds the *inputs* of the close-coupling calculation and nothing
of the method itself: the radial grid with its integration weights, the
radial basis functions tabulated on that grid (hydrogenic bound states and
Coulomb wave-packet pseudostates), their energies, the state list, the
Gauss-Laguerre / Gauss-Legendre quadrature rules used in the two-centre
integrals, and the straight-line paths (impact parameters, velocity, z-grid).

None of the method's arithmetic (Eq. 6-9 matrix elements, Eq. 4 solve,
Algorithm 1 propagation) lives here; the oracle and the CUDA library each
implement that on their own and only consume what is built here.

The basis functions themselves are defined in the WP-CCC literature the paper
cites (its Sec. II refers to earlier work for the formalism); the reading used
here is: bound states are the closed-form hydrogenic radial functions, and a
wave-packet pseudostate of angular momentum l on the k-bin [k_i, k_{i+1}] is
(k_{i+1}-k_i)^(-1/2) * integral over the bin of the delta(k-k')-normalised
regular Coulomb function u_kl(r)/r, with energy (k_i^2 + k_i k_{i+1} +
k_{i+1}^2)/6.  Pseudostates are then orthonormalised on the grid against the
lower states of the same l (Gram-Schmidt), so the tabulated basis is
orthonormal under the grid's own quadrature (the lowest state of each l
keeps its closed form; higher bound states are orthonormalised as well, since
the grid's end at r_max cuts their tails).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import special
from scipy.interpolate import CubicSpline

__all__ = [
    "RadialGrid", "Centre", "Basis", "Quadrature", "Paths",
    "radial_grid", "hydrogenic_radial", "coulomb_bins", "make_centre",
    "make_basis", "make_quadrature", "uniform_zgrid", "geometric_zgrid", "piecewise_zgrid",
    "make_paths", "CONFIGS", "config_inputs", "CentreTangent", "box_centre", "li_model_potential",
    "li_basis", "li_parameters", "observable_weights", "cross_section_weights", "li_inputs",
]


# --------------------------------------------------------------------------
# radial grid (Sec. II: r-grid from 0 to ~100 a.u., denser near the origin)
# --------------------------------------------------------------------------
@dataclass
class RadialGrid:
    r: np.ndarray        # [Nr] strictly increasing, r[0] > 0, r[-1] = rmax
    w: np.ndarray        # [Nr] integration weights: sum_i w_i g(r_i) ~ int_0^rmax g dr
    rmax: float
    alpha: float


def radial_grid(Nr: int = 2000, rmax: float = 100.0, alpha: float = 3.5) -> RadialGrid:
    """sinh-mapped grid r_i = rmax sinh(alpha i/Nr)/sinh(alpha), i = 1..Nr.

    Weights are the trapezoid rule in the mapped variable x = i/Nr times the
    Jacobian dr/dx (the x = 0 end point, r = 0, is dropped: every integrand the
    method forms carries a factor r^2 there).  The trapezoid rule is used
    because its weights stay a valid rule for any split of the range at a grid
    node, which the min(r,R)/max(r,R) kernel of Eq. 7 requires.
    """
    i = np.arange(1, Nr + 1, dtype=np.float64)
    x = i / Nr
    r = rmax * np.sinh(alpha * x) / math.sinh(alpha)
    jac = rmax * alpha * np.cosh(alpha * x) / math.sinh(alpha)
    w = jac / Nr
    w[-1] *= 0.5
    r[-1] = rmax
    return RadialGrid(r=r, w=w, rmax=float(rmax), alpha=float(alpha))


# --------------------------------------------------------------------------
# radial functions
# --------------------------------------------------------------------------
def hydrogenic_radial(n: int, l: int, Z: float, r: np.ndarray) -> np.ndarray:
    """Closed-form hydrogenic R_nl(r), normalised so int r^2 R^2 dr = 1."""
    rho = 2.0 * Z * r / n
    norm = math.sqrt((2.0 * Z / n) ** 3 * math.factorial(n - l - 1)
                     / (2.0 * n * math.factorial(n + l)))
    return norm * np.exp(-rho / 2.0) * rho ** l * special.eval_genlaguerre(n - l - 1, 2 * l + 1, rho)


def _coulomb_regular(Z: float, l: int, ks: np.ndarray, rmatch: float, dr: float):
    """delta(k-k')-normalised regular Coulomb functions u_kl(r) on a uniform grid.

    Outward Numerov for u'' = (l(l+1)/r^2 - 2Z/r - k^2) u from a power-series
    start, normalised to the local WKB amplitude sqrt(2k/(pi*kappa(r))) over the
    last few wavelengths before rmatch.
    """
    n = int(math.ceil(rmatch / dr))
    ru = dr * np.arange(n + 1)
    k2 = ks[None, :] ** 2
    u = np.zeros((n + 1, ks.size))
    # series u = r^{l+1} (1 + a1 r + a2 r^2 + a3 r^3)
    a1 = -Z / (l + 1)
    a2 = (-2.0 * Z * a1 - k2) / (2.0 * (2 * l + 3))
    a3 = (-2.0 * Z * a2 - k2 * a1) / (3.0 * (2 * l + 4))
    for i in (1, 2):
        x = ru[i]
        u[i] = x ** (l + 1) * (1.0 + a1 * x + a2 * x * x + a3 * x ** 3)
    h2 = dr * dr / 12.0

    def g(i):
        x = ru[i]
        return l * (l + 1) / (x * x) - 2.0 * Z / x - k2[0]

    gm, g0 = g(1), g(2)
    for i in range(2, n):
        gp = g(i + 1)
        u[i + 1] = (2.0 * (1.0 + 5.0 * h2 * g0) * u[i] - (1.0 - h2 * gm) * u[i - 1]) / (1.0 - h2 * gp)
        gm, g0 = g0, gp
    # amplitude match over the tail
    tail = slice(int(0.8 * n), n)
    rt = ru[tail]
    du = (u[2:] - u[:-2])[tail.start - 1:tail.stop - 1] / (2.0 * dr)
    kap = np.sqrt(k2 + 2.0 * Z / rt[:, None] - l * (l + 1) / rt[:, None] ** 2)
    amp2 = u[tail] ** 2 + (du / kap) ** 2
    want = 2.0 * ks[None, :] / (np.pi * kap)
    scale = np.sqrt(np.mean(want, axis=0) / np.mean(amp2, axis=0))
    return ru, u * scale[None, :]


def coulomb_bins(Z: float, l: int, kmax: float, nbins: int, r: np.ndarray,
                 nk: int = 16, rmatch: float = 200.0, dr: float = 0.01):
    """Wave-packet pseudostates on uniform k-bins of (0, kmax]; returns (f[nbins, Nr], eps[nbins])."""
    edges = np.linspace(0.0, kmax, nbins + 1)
    xg, wg = np.polynomial.legendre.leggauss(nk)
    ks, wk, owner = [], [], []
    for i in range(nbins):
        a, b = edges[i], edges[i + 1]
        ks.append(0.5 * (b - a) * xg + 0.5 * (a + b))
        wk.append(0.5 * (b - a) * wg)
        owner.append(np.full(nk, i))
    ks, wk, owner = np.concatenate(ks), np.concatenate(wk), np.concatenate(owner)
    ru, u = _coulomb_regular(Z, l, ks, max(rmatch, r[-1] + 10.0), dr)
    spl = CubicSpline(ru, u, axis=0)
    ur = spl(r)                                    # [Nr, nk*nbins]
    f = np.zeros((nbins, r.size))
    for i in range(nbins):
        sel = owner == i
        dk = edges[i + 1] - edges[i]
        f[i] = (ur[:, sel] * wk[sel][None, :]).sum(axis=1) / r / math.sqrt(dk)
    eps = (edges[:-1] ** 2 + edges[:-1] * edges[1:] + edges[1:] ** 2) / 6.0
    return f, eps


# --------------------------------------------------------------------------
# one centre's basis and the two-centre basis
# --------------------------------------------------------------------------
@dataclass
class Centre:
    Z: float                 # nuclear charge of this centre
    rad_l: np.ndarray        # [n_rad] int, angular momentum of each radial function
    rad_n: np.ndarray        # [n_rad] int, principal number (bound) or 100+bin index (pseudostate)
    f: np.ndarray            # [n_rad, Nr] radial functions on the grid
    rad_eps: np.ndarray      # [n_rad] energies
    st_rad: np.ndarray       # [N] radial index of each state
    st_l: np.ndarray         # [N]
    st_m: np.ndarray         # [N]
    st_eps: np.ndarray       # [N]

    @property
    def n_rad(self) -> int:
        return int(self.rad_l.size)

    @property
    def N(self) -> int:
        return int(self.st_rad.size)


def _orthonormalise(funcs: list, grid: RadialGrid, fixed: int) -> list:
    """Gram-Schmidt under the grid inner product; the first `fixed` functions are kept as they are."""
    wr2 = grid.w * grid.r ** 2
    out = list(funcs[:fixed])
    for f in funcs[fixed:]:
        g = f.copy()
        for _ in range(2):
            for q in out:
                g -= (np.sum(wr2 * q * g) / np.sum(wr2 * q * q)) * q
        g /= math.sqrt(np.sum(wr2 * g * g))
        out.append(g)
    return out


def make_centre(Z: float, nmax: int, lmax: int, nbins: int, kmax: float,
                grid: RadialGrid, all_m: bool = True) -> Centre:
    """Bound hydrogenic n<=nmax and `nbins` Coulomb pseudostates per l<=lmax, on a centre of charge Z.

    Radial functions are ordered by l, then bound states by n, then bins by k.
    States are ordered by radial function, then m = -l..l (all_m) or 0..l.
    """
    rad_l, rad_n, f, eps = [], [], [], []
    for l in range(lmax + 1):
        fl, el, nl = [], [], []
        for n in range(l + 1, nmax + 1):
            fl.append(hydrogenic_radial(n, l, Z, grid.r))
            el.append(-Z * Z / (2.0 * n * n))
            nl.append(n)
        nbound = len(fl)
        if nbins > 0:
            fb, eb = coulomb_bins(Z, l, kmax, nbins, grid.r)
            fl.extend(list(fb))
            el.extend(list(eb))
            nl.extend([100 + i for i in range(nbins)])
        # the lowest function of each l is kept as it is; the rest (higher bound states, whose tails the
        # finite grid cuts, and the pseudostates) are orthonormalised on the grid in order
        fl = _orthonormalise(fl, grid, 1)
        rad_l += [l] * len(fl)
        rad_n += nl
        f += fl
        eps += el
    rad_l = np.array(rad_l, dtype=np.int32)
    st_rad, st_l, st_m = [], [], []
    for i, l in enumerate(rad_l):
        for m in (range(-l, l + 1) if all_m else range(0, l + 1)):
            st_rad.append(i)
            st_l.append(int(l))
            st_m.append(m)
    eps = np.array(eps, dtype=np.float64)
    st_rad = np.array(st_rad, dtype=np.int32)
    return Centre(Z=float(Z), rad_l=rad_l, rad_n=np.array(rad_n, dtype=np.int32),
                  f=np.ascontiguousarray(np.array(f, dtype=np.float64)), rad_eps=eps,
                  st_rad=st_rad, st_l=np.array(st_l, dtype=np.int32),
                  st_m=np.array(st_m, dtype=np.int32), st_eps=eps[st_rad].copy())


def centre_from_functions(Z: float, rad_l, rad_n, f, eps, all_m: bool = True) -> Centre:
    """A centre from explicitly given radial functions (used for tiny test bases)."""
    rad_l = np.asarray(rad_l, dtype=np.int32)
    eps = np.asarray(eps, dtype=np.float64)
    st_rad, st_l, st_m = [], [], []
    for i, l in enumerate(rad_l):
        for m in (range(-l, l + 1) if all_m else range(0, l + 1)):
            st_rad.append(i)
            st_l.append(int(l))
            st_m.append(m)
    st_rad = np.array(st_rad, dtype=np.int32)
    return Centre(Z=float(Z), rad_l=rad_l, rad_n=np.asarray(rad_n, dtype=np.int32),
                  f=np.ascontiguousarray(np.asarray(f, dtype=np.float64)), rad_eps=eps,
                  st_rad=st_rad, st_l=np.array(st_l, dtype=np.int32),
                  st_m=np.array(st_m, dtype=np.int32), st_eps=eps[st_rad].copy())


# --------------------------------------------------------------------------
# box eigenstates of a general central potential, with parameter tangents
# (the Li-like model-potential target of the differentiation workload)
# --------------------------------------------------------------------------
def li_model_potential(c: float, a: float, b: float, Z_as: float = 1.0):
    """V(r) = -[Z_as + c e^{-a r}(1 + b r)]/r and its derivatives with respect to (c, a, b)."""
    def V(r):
        return -(Z_as + c * np.exp(-a * r) * (1.0 + b * r)) / r

    def dV_dc(r):
        return -np.exp(-a * r) * (1.0 + b * r) / r

    def dV_da(r):
        return c * np.exp(-a * r) * (1.0 + b * r)

    def dV_db(r):
        return -c * np.exp(-a * r)
    return V, (dV_dc, dV_da, dV_db)


@dataclass
class CentreTangent:
    """Derivatives of one centre's radial functions and energies with respect to n_par parameters."""
    df: np.ndarray           # [n_par, n_rad, Nr]
    deps: np.ndarray         # [n_par, n_rad]


def box_centre(V, dVs, nmax: int, lmax: int, nbins: int, kmax: float, grid: RadialGrid,
               skip_lowest_s: bool = False, all_m: bool = True, Z: float = 1.0):
    """Bound states and wave packets of -1/2 u'' + (l(l+1)/(2r^2) + V(r)) u = E u in the box (0, r_max].

    The radial equation is discretised on the grid itself: kinetic energy from the difference quotients
    (u_i - u_{i-1})/(r_i - r_{i-1}) with u_0 = u(0) = 0 and u(r_max) = 0, potential and norm from the
    grid's own weights w_i.  The discrete eigenvectors are therefore orthonormal under the rule every
    matrix element uses.  Kept states of each l:
      * bound states with principal number n <= nmax (n = l + 1 + index of the eigenvalue; with
        skip_lowest_s the lowest s state, the Pauli-blocked core orbital of a Li-like target, is
        dropped, so the s series starts at n = 2);
      * `nbins` wave packets on uniform k-bins of (0, kmax]: the normalised sum of the box states whose
        k = sqrt(2E) lies in the bin (each signed so that u > 0 next to the origin), with the bin's
        mean box energy as its energy.
    Tangents (one per entry of dVs, the potential's derivative functions) are the exact derivatives
    of the discrete eigenpairs (first-order perturbation theory over all box states).
    Returns (Centre, CentreTangent)."""
    r, w = grid.r, grid.w
    n = r.size - 1                                  # unknowns u_1 .. u_{Nr-1}; u_{Nr} = 0
    ri, wi = r[:n], w[:n]
    h = np.diff(np.concatenate([[0.0], r]))         # h_i = r_i - r_{i-1}, i = 1..Nr
    kin_d = 0.5 * (1.0 / h[:n] + 1.0 / h[1:n + 1])
    kin_e = -0.5 / h[1:n]
    sw = np.sqrt(wi)
    off = kin_e / (sw[:-1] * sw[1:])
    edges = np.linspace(0.0, kmax, nbins + 1)
    npar = len(dVs)
    dVv = [dv(ri) for dv in dVs]
    rad_l, rad_n, f, eps, df, deps = [], [], [], [], [], []
    from scipy.linalg import eigh_tridiagonal
    for l in range(lmax + 1):
        diag = kin_d / wi + l * (l + 1) / (2.0 * ri * ri) + V(ri)
        E, Y = eigh_tridiagonal(diag, off)
        Y = Y * np.where(Y[0] < 0.0, -1.0, 1.0)[None, :]
        first = 1 if (skip_lowest_s and l == 0) else 0
        groups = []                                 # (label, member indices)
        for idx in range(first, n):
            nq = l + 1 + idx
            if nq > nmax or E[idx] >= 0.0:
                break
            groups.append((nq, [idx]))
        if nbins > 0:
            pos = np.nonzero(E > 0.0)[0]
            k = np.sqrt(2.0 * E[pos])
            for ib in range(nbins):
                sel = pos[(k > edges[ib]) & (k <= edges[ib + 1])]
                if sel.size == 0:
                    raise ValueError(f"k-bin {ib} of l={l} holds no box state; widen the bins")
                groups.append((100 + ib, list(sel)))
            kk = np.sqrt(2.0 * E[pos[k <= kmax * 1.0001]])
            clear = np.min(np.abs(kk[:, None] - edges[None, 1:]))
            if clear < 1e-7:
                raise ValueError("a box state lies on a k-bin edge; its bin is not well defined")
        # derivatives of every kept eigenpair: dE_s = y_s.dV y_s, dy_s = sum_{t != s} y_t (y_t.dV y_s)/(E_s - E_t)
        keep = sorted({i for _, mem in groups for i in mem})
        dE = {}
        dY = {}
        for p in range(npar):
            C = Y.T @ (dVv[p][:, None] * Y[:, keep])             # [n, len(keep)]
            for col, s in enumerate(keep):
                den = E[s] - E
                den[s] = np.inf
                dY[p, s] = Y @ (C[:, col] / den)
                dE[p, s] = C[s, col]
        for label, mem in groups:
            norm = 1.0 / math.sqrt(len(mem))
            y = Y[:, mem].sum(axis=1) * norm
            fu = np.zeros(r.size)
            fu[:n] = y / sw / ri
            rad_l.append(l)
            rad_n.append(label)
            f.append(fu)
            eps.append(float(np.mean(E[mem])))
            dfp = np.zeros((npar, r.size))
            dep = np.zeros(npar)
            for p in range(npar):
                dy = sum(dY[p, s] for s in mem) * norm
                dfp[p, :n] = dy / sw / ri
                dep[p] = float(np.mean([dE[p, s] for s in mem]))
            df.append(dfp)
            deps.append(dep)
    centre = centre_from_functions(Z, rad_l, rad_n, np.array(f), np.array(eps), all_m)
    tangent = CentreTangent(df=np.ascontiguousarray(np.transpose(np.array(df), (1, 0, 2))),
                            deps=np.ascontiguousarray(np.array(deps).T))
    return centre, tangent


@dataclass
class Quadrature:
    """Gauss-Laguerre in s (eta = 1 + s/(gamma R)) and Gauss-Legendre in tau (Eq. 9)."""
    s: np.ndarray           # [Geta] Laguerre nodes
    ws: np.ndarray          # [Geta] Laguerre weights times e^{s} (computed in log space)
    tau: np.ndarray         # [Gtau]
    wtau: np.ndarray        # [Gtau]
    gamma: float            # eta scale

    @property
    def G(self) -> int:
        return int(self.s.size * self.tau.size)


def make_quadrature(Geta: int = 48, Gtau: int = 48, gamma: float = 0.5) -> Quadrature:
    s, w = special.roots_laguerre(Geta)
    with np.errstate(divide="ignore"):   # weights that underflow (very large rules) drop their nodes
        ws = np.exp(np.log(w) + s)
    tau, wtau = np.polynomial.legendre.leggauss(Gtau)
    return Quadrature(s=s.astype(np.float64), ws=ws, tau=tau, wtau=wtau, gamma=float(gamma))


@dataclass
class Basis:
    grid: RadialGrid
    T: Centre
    P: Centre | None              # None in one-centre mode
    quad: Quadrature | None
    Z_T: float                    # charge of the target nucleus (asymptotic charge of a model potential)
    Z_P: float                    # charge of the projectile nucleus
    # short-range part of a Li-like target potential: V_T(r) = -[Z_T + mp_c e^{-mp_a r}(1 + mp_b r)]/r
    mp_c: float = 0.0
    mp_a: float = 0.0
    mp_b: float = 0.0
    # parameter tangents of the differentiation workload (None otherwise): derivatives of both
    # centres' functions and energies, and of (Z_P, mp_c, mp_a, mp_b), with respect to each parameter
    tangent_T: CentreTangent | None = None
    tangent_P: CentreTangent | None = None
    dexplicit: np.ndarray | None = None    # [n_par, 4]: d(Z_P, mp_c, mp_a, mp_b)/d theta_p
    theta_names: tuple = ()

    @property
    def n_centres(self) -> int:
        return 1 if self.P is None else 2

    @property
    def N(self) -> int:
        return self.T.N + (0 if self.P is None else self.P.N)


def make_basis(Z_T: float, Z_P: float, nmax, lmax, nbins, kmax, two_centre: bool,
               Nr: int = 2000, rmax: float = 100.0, alpha: float = 3.5,
               Geta: int = 48, Gtau: int = 48, gamma: float = 0.5, all_m: bool = True) -> Basis:
    """nmax/lmax/nbins/kmax may be scalars (same on both centres) or (target, projectile) pairs."""
    def pair(x):
        return (x, x) if np.isscalar(x) else tuple(x)
    nmax, lmax, nbins, kmax = pair(nmax), pair(lmax), pair(nbins), pair(kmax)
    grid = radial_grid(Nr, rmax, alpha)
    T = make_centre(Z_T, nmax[0], lmax[0], nbins[0], kmax[0], grid, all_m)
    P = make_centre(Z_P, nmax[1], lmax[1], nbins[1], kmax[1], grid, all_m) if two_centre else None
    quad = make_quadrature(Geta, Gtau, gamma) if two_centre else None
    return Basis(grid=grid, T=T, P=P, quad=quad, Z_T=float(Z_T), Z_P=float(Z_P))


def li_basis(Z_p: float = 1.0, a: float = 3.0, b: float = 1.5, c: float = 2.0, nmax: int = 4, lmax: int = 3,
             nbins: int = 10, kmax: float = 3.0, Nr: int = 2000, rmax: float = 100.0, alpha: float = 3.5,
             Geta: int = 48, Gtau: int = 48, gamma: float = 0.5, all_m: bool = True) -> Basis:
    """Bare projectile of charge Z_p on a one-electron Li-like target with the model potential
    V(r) = -[1 + c e^{-a r}(1 + b r)]/r.  Both centres' states are box eigenstates on the grid
    (box_centre); the target's lowest s state (the core orbital) is left out, so its first state is
    the valence 2s.  The tangents are with respect to theta = (Z_p, a, b)."""
    grid = radial_grid(Nr, rmax, alpha)
    V_T, (dV_dc, dV_da, dV_db) = li_model_potential(c, a, b)
    zero = lambda r: np.zeros_like(r)
    T, tT = box_centre(V_T, [zero, dV_da, dV_db], nmax, lmax, nbins, kmax, grid, skip_lowest_s=True,
                       all_m=all_m, Z=1.0)
    P, tP = box_centre(lambda r: -Z_p / r, [lambda r: -1.0 / r, zero, zero], nmax, lmax, nbins, kmax, grid,
                       all_m=all_m, Z=Z_p)
    dexp = np.array([[1.0, 0.0, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]])
    return Basis(grid=grid, T=T, P=P, quad=make_quadrature(Geta, Gtau, gamma), Z_T=1.0, Z_P=float(Z_p),
                 mp_c=float(c), mp_a=float(a), mp_b=float(b), tangent_T=tT, tangent_P=tP, dexplicit=dexp,
                 theta_names=("Z_p", "a", "b"))


def li_parameters(seed: int = 0, spread: float = 0.05):
    """Model-potential parameters a = 3.0 (1 + U), b = 1.5 (1 + U), U uniform in (-spread, spread)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-spread, spread, size=2)
    return 3.0 * (1.0 + u[0]), 1.5 * (1.0 + u[1])


def observable_weights(basis: Basis):
    """0/1 weights g of two observables P = sum_i g_i |c_i|^2: electron capture (every bound
    projectile state) and 2p excitation (the target's 2p states, all m)."""
    N, NT = basis.N, basis.T.N
    cap = np.zeros(N)
    P = basis.P
    cap[NT:] = (P.rad_n[P.st_rad] < 100).astype(np.float64)
    ex = np.zeros(N)
    T = basis.T
    ex[:NT] = ((T.rad_n[T.st_rad] == 2) & (T.st_l == 1)).astype(np.float64)
    return np.stack([cap, ex])


def cross_section_weights(bs) -> np.ndarray:
    """sigma = 2 pi int_0^inf b P(b) db by the trapezoid rule on the impact parameters plus b = 0
    (where b P(b) = 0): per-path weights 2 pi b_j w_j."""
    bs = np.asarray(bs, dtype=np.float64)
    nodes = np.concatenate([[0.0], bs])
    w = np.zeros(nodes.size)
    d = np.diff(nodes)
    w[:-1] += 0.5 * d
    w[1:] += 0.5 * d
    return 2.0 * np.pi * bs * w[1:]


# --------------------------------------------------------------------------
# paths
# --------------------------------------------------------------------------
def uniform_zgrid(z0: float, z1: float, h: float) -> np.ndarray:
    n = int(round((z1 - z0) / h))
    return z0 + h * np.arange(n + 1, dtype=np.float64)


def geometric_zgrid(zmin: float = 1e-3, zmax: float = 100.0, nz: int = 500) -> np.ndarray:
    """Sec. II z-grid: zgrid[i] = zmin (zmax/zmin)^(i/nz), zgrid[0] = 0, zgrid[-i] = -zgrid[i]."""
    i = np.arange(1, nz + 1, dtype=np.float64)
    pos = zmin * (zmax / zmin) ** (i / nz)
    return np.concatenate([-pos[::-1], [0.0], pos])


# Segments of the C6+ + H z-grid: (end of the |z| range, largest step in it).  The step bound in each
# range is 2 / omega_max at the range's start, where omega_max = max |lambda(H, S)| / v of the workload's
# basis at its smallest impact parameter b = 0.5 (FP64 oracle: 984 at |z| = 0.3, 514 at 2, 123 at 4,
# 40 at 6, 13.4 at 8, 2.6 at 12, 0.22 at 50); RK4 is stable on the imaginary axis for h omega < 2.83.
C6_ZGRID_SEGMENTS = ((2.0, 2.0e-3), (4.0, 3.9e-3), (6.0, 0.016), (8.0, 0.05), (12.0, 0.15), (50.0, 0.5))


def piecewise_zgrid(segments) -> np.ndarray:
    """Symmetric z-grid, uniform within each |z| range: segments = ((z_1, h_1), (z_2, h_2), ...) cover
    [0, z_1], [z_1, z_2], ... with ceil((z_k - z_{k-1}) / h_k) equal steps each, mirrored to z < 0."""
    pos = [0.0]
    z0 = 0.0
    for z1, h in segments:
        n = int(math.ceil((z1 - z0) / h - 1e-9))
        pos.extend(z0 + (z1 - z0) * np.arange(1, n + 1, dtype=np.float64) / n)
        z0 = z1
    pos = np.asarray(pos)
    return np.concatenate([-pos[:0:-1], pos])


@dataclass
class Paths:
    b: np.ndarray                     # [n_paths]
    v: np.ndarray                     # [n_paths]
    z: list = field(default_factory=list)   # n_paths arrays of z nodes (ascending)

    @property
    def n_paths(self) -> int:
        return int(self.b.size)


def make_paths(bs, v, zgrid) -> Paths:
    bs = np.asarray(bs, dtype=np.float64)
    vs = np.broadcast_to(np.asarray(v, dtype=np.float64), bs.shape).copy()
    return Paths(b=bs, v=vs, z=[np.asarray(zgrid, dtype=np.float64).copy() for _ in bs])


# --------------------------------------------------------------------------
# the workloads (synthetic stand-ins for the paper's p + H calculations)
# --------------------------------------------------------------------------
CONFIGS = {
    # one-centre p + H, direct elements only
    "p_H_1c_n3l2": dict(Z_T=1.0, Z_P=1.0, nmax=3, lmax=2, nbins=5, kmax=2.0, two_centre=False,
                        v=1.0, b=(0.5, 8.0, 8), z=(-40.0, 40.0, 0.1)),
    # one-centre p + H at the paper's large angular momentum: n <= 10, l <= 10, 32 packets per l
    # (N = 385 + 32 x 121 = 4257), v = 2 a.u. (100 keV)
    "p_H_1c_n10l10": dict(Z_T=1.0, Z_P=1.0, nmax=10, lmax=10, nbins=32, kmax=2.0, two_centre=False,
                          v=2.0, b=(0.5, 8.0, 8), z=(-40.0, 40.0, 0.1)),
    # two-centre p + H with electron capture
    "p_H_2c_n4l3": dict(Z_T=1.0, Z_P=1.0, nmax=4, lmax=3, nbins=10, kmax=3.0, two_centre=True,
                        v=1.5, b=(0.2, 12.0, 32), z=(-50.0, 50.0, 0.1)),
    # two-centre bare C6+ on H (projectile charge 6), the mixed-precision workload.  128 eta nodes: the
    # compact C5+ orbitals and the k <= 4 packets need them for a positive-definite S (sigma_max(K) at
    # b = 0.5, z = 0: 1.56 with 48 nodes, 1.28 with 72, 1.06 with 96, 0.99847 with 128, 0.99846 with
    # 160 x 64).  z-grid: steps bounded by the basis' stiffness (C6_ZGRID_SEGMENTS, 3562 RK4 steps); the
    # paper's geometric grid of Sec. II takes steps of 0.022 |z|, which RK4 cannot follow where
    # omega_max ~ 1e3 (0.1 < |z| < 6 at b = 0.5: the amplitudes overflow)
    "C6_H_2c_n6l5": dict(Z_T=1.0, Z_P=6.0, nmax=6, lmax=5, nbins=20, kmax=4.0, two_centre=True,
                         v=2.0, b=(0.5, 15.0, 16), z=("piecewise", C6_ZGRID_SEGMENTS), Geta=128, Gtau=48),
}


BATCH_SPEEDS = (0.5, 0.8, 1.2, 2.0, 3.0, 4.0)


def batch_inputs(n_b: int = 64, speeds=BATCH_SPEEDS, **over):
    """Two-centre p + H at several speeds: pseudostates per l scaled with v (round(8 + 8 (v - 0.5)/3.5),
    i.e. 8..16 for v = 0.5..4), hydrogenic n <= 4, l <= 3, k <= 3; n_b impact parameters uniform in
    [0.2, 12]; z in [-50, 50] with h = 0.1 v / 1.5 (step count proportional to 1/v).
    The two-centre quadrature has 72 eta nodes (x 48 tau): with 48, the overlaps of the slow-speed bases
    at R ~ 0.2 come out with sigma_max(K) up to 1.23, i.e. an indefinite S that no set of functions has;
    72 gives 0.9991, within 5e-6 of 96 nodes.
    Returns a list of (v, basis, paths)."""
    out = []
    for v in speeds:
        nb = int(round(8 + 8 * (v - 0.5) / 3.5))
        basis = make_basis(1.0, 1.0, over.get("nmax", 4), over.get("lmax", 3), over.get("nbins", nb),
                           over.get("kmax", 3.0), True, Nr=over.get("Nr", 2000), Geta=over.get("Geta", 72),
                           Gtau=over.get("Gtau", 48))
        h = 0.1 * v / 1.5
        paths = make_paths(np.linspace(0.2, 12.0, n_b), v, uniform_zgrid(-50.0, 50.0, h))
        out.append((v, basis, paths))
    return out


def config_inputs(name: str, **over):
    """(basis, paths) of a named workload; keyword overrides shrink it for tests."""
    c = dict(CONFIGS[name])
    c.update(over)
    basis = make_basis(c["Z_T"], c["Z_P"], c["nmax"], c["lmax"], c["nbins"], c["kmax"],
                       c["two_centre"], Nr=c.get("Nr", 2000), rmax=c.get("rmax", 100.0),
                       Geta=c.get("Geta", 48), Gtau=c.get("Gtau", 48), gamma=c.get("gamma", 0.5))
    b0, b1, nb = c["b"]
    if c["z"][0] == "geometric":
        zgrid = geometric_zgrid(*c["z"][1:])
    elif c["z"][0] == "piecewise":
        zgrid = piecewise_zgrid(c["z"][1])
    else:
        zgrid = uniform_zgrid(*c["z"])
    paths = make_paths(np.linspace(b0, b1, nb), c["v"], zgrid)
    return basis, paths


def li_inputs(seed: int = 0, n_b: int = 32, **over):
    """The differentiation workload: p + Li-like model-potential target with a, b drawn within 5 % of
    (3.0, 1.5) from `seed`; hydrogen-like projectile, n <= 4, l <= 3, 10 wave packets per l on (0, 3];
    v = 1.5; n_b impact parameters uniform in [0.2, 12]; z in [-50, 50], h = 0.1 (1000 steps).
    Keyword overrides shrink it for tests.  Returns (basis, paths)."""
    a, b = li_parameters(seed)
    kw = dict(Z_p=1.0, a=a, b=b)
    kw.update({k: v for k, v in over.items() if k not in ("v", "b_range", "z", "h")})
    basis = li_basis(**kw)
    b0, b1 = over.get("b_range", (0.2, 12.0))
    z0, z1 = over.get("z", (-50.0, 50.0))
    paths = make_paths(np.linspace(b0, b1, n_b), over.get("v", 1.5), uniform_zgrid(z0, z1, over.get("h", 0.1)))
    return basis, paths
