"""Plain FP64 CPU oracle of the WP-CCC hot path.  TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
leg may import this module.  The product library never calls it, and it
shares no code with the CUDA path: it reads the generated inputs of
`wpccc_inputs` (grid, radial tables, energies, quadrature rules, paths) and
computes everything else itself, following the paper's equations in order:

* Eq. 7  radial multipole integrals F_{n'l'nl lambda}(R) on the r-grid,
         5-point Lagrange interpolation at off-grid R (Sec. II, last part);
* Eq. 6  direct elements D_T (and D_P, the same expansion about the projectile);
* Eq. 9  molecular-frame two-centre integrals on the Gauss-Laguerre x
         Gauss-Legendre (eta, tau) rule, with the ETF phase and J_{q-q'};
* Eq. 8  rotation to the collision frame with Wigner d^l(theta);
* Eq. 1  assembly of S = [[I, K], [K^+, I]] and H = [[D_T, Q], [Q~, D_P]];
* Eq. 4  M = -(i/v) S^{-1} H through a linear solve (LAPACK zgesv, as the
         paper does), Eq. 5 (one-centre: M = -(i/v) D_T, no solve);
* Algorithm 1  RK4 along the z-grid, then probabilities |c_i|^2;
* differentiation form: derivatives of S, H and of the probabilities with
  respect to the projectile charge and the parameters of a Li-like target
  model potential V_T(r) = -[Z_T + c e^{-a r}(1 + b r)]/r, in forward mode
  (every line of Algorithm 1 differentiated alongside it).

Model-potential target (the paper treats bare Coulomb centres only; these
are the readings used for it): the transfer integral Q carries V_T(r_T) in
place of -Z_T/r_T; between projectile states the target's Coulomb part
keeps the Eq. 6 multipole form and its short-range part is integrated on
the Eq. 9 (eta, tau) rule, where only equal-q pairs couple.

Readings of garbled or silent passages (each pinned by a test in
tests/test_oracle_pins.py):
* Eq. 6: the square-root prefactor is sqrt((2l+1)/(2l'+1)) * sqrt((lam-mu)!/(lam+mu)!)
  and the element carries the charge of the other nucleus, -Z * sum(...);
  Legendre functions carry the Condon-Shortley phase.  D_P has the other
  nucleus at -R, which multiplies each multipole by (-1)^lam.
* Eq. 8/9: the molecular axis points from the target (at zeta = -R/2) to the
  projectile; beta is the target state, alpha the projectile state; the
  rotation uses d^{l_alpha}_{m_alpha q} (second index q, not q'); with the
  projectile at azimuth 0 (b along +x) the phi integral gives
  2 pi (-i)^(q-q') J_{q-q'}(v b/2 sqrt((eta^2-1)(1-tau^2))).
* Eq. 1 lower-left block: Q^+, as printed.  H is then Hermitian and
  S^-1 H has a real spectrum, so the propagation cannot grow; the exact
  reverse-transfer integral <P| -Z_P/r_P |T> differs from Q^+ for a
  finite pseudostate basis and gives growing modes (tests/test_oracle_pins.py).
* Energy phases: every element between states i and j carries
  exp(i (eps_i - eps_j) z / v) (interaction picture, t = z/v).
* Eq. 5: M = -(i/v) D_T (the -i/v of Eq. 4 with S = I).
* eta = 1 + s/(gamma R) maps the Laguerre variable s onto [1, inf).
* 5-point interpolation: nodes j-2..j+2 with r_j <= x < r_{j+1}, clamped at
  the grid ends; radial functions vanish beyond the last grid point, so for
  R beyond it F_lam(R) is the multipole moment times R^-(lam+1).
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np
from scipy import special

# ---------------------------------------------------------------------------
# angular-momentum algebra
# ---------------------------------------------------------------------------


@lru_cache(maxsize=None)
def clebsch_gordan(j1: int, m1: int, j2: int, m2: int, J: int, M: int) -> float:
    """<j1 m1 j2 m2 | J M> for integer angular momenta, from Racah's closed formula (exact rationals)."""
    if m1 + m2 != M or abs(m1) > j1 or abs(m2) > j2 or abs(M) > J:
        return 0.0
    if J < abs(j1 - j2) or J > j1 + j2:
        return 0.0
    f = math.factorial
    pre = Fraction((2 * J + 1) * f(J + j1 - j2) * f(J - j1 + j2) * f(j1 + j2 - J), f(j1 + j2 + J + 1))
    pre *= f(J + M) * f(J - M) * f(j1 - m1) * f(j1 + m1) * f(j2 - m2) * f(j2 + m2)
    s = Fraction(0)
    for k in range(0, j1 + j2 - J + 1):
        den = [k, j1 + j2 - J - k, j1 - m1 - k, j2 + m2 - k, J - j2 + m1 + k, J - j1 - m2 + k]
        if min(den) < 0:
            continue
        term = Fraction(1, math.prod(f(d) for d in den))
        s += -term if k % 2 else term
    val = s * s * pre
    return math.copysign(math.sqrt(float(val)), float(s)) if s != 0 else 0.0


def wigner_d(j: int, mp: int, m: int, beta: float) -> float:
    """Wigner small d^j_{m'm}(beta) = <j m'| exp(-i beta J_y) |j m>, Wigner's explicit sum."""
    f = math.factorial
    c, s = math.cos(beta / 2.0), math.sin(beta / 2.0)
    pre = math.sqrt(f(j + mp) * f(j - mp) * f(j + m) * f(j - m))
    tot = 0.0
    for k in range(0, 2 * j + 1):
        a, b, cc, d = j + m - k, k, mp - m + k, j - mp - k
        if min(a, b, cc, d) < 0:
            continue
        term = pre / (f(a) * f(b) * f(cc) * f(d))
        term *= c ** (2 * j + m - mp - 2 * k) * s ** (mp - m + 2 * k)
        tot += -term if (mp - m + k) % 2 else term
    return tot


def assoc_legendre(l: int, m: int, x):
    """P_l^m(x) with the Condon-Shortley phase; negative m through P_l^{-m} = (-1)^m (l-m)!/(l+m)! P_l^m."""
    x = np.asarray(x, dtype=np.float64)
    if abs(m) > l:
        return np.zeros_like(x)
    p = special.lpmv(abs(m), l, x)
    if m < 0:
        p = p * ((-1) ** m * math.factorial(l + m) / math.factorial(l - m))
    return p


def norm_legendre(l: int, q: int, x):
    """Theta_lq(x) = sqrt((2l+1)/2 * (l-q)!/(l+q)!) P_l^q(x), so Y_lq = Theta_lq e^{iq phi}/sqrt(2 pi)."""
    return math.sqrt((2 * l + 1) / 2.0 * math.factorial(l - q) / math.factorial(l + q)) * assoc_legendre(l, q, x)


# ---------------------------------------------------------------------------
# 5-point interpolation on the r-grid (Sec. II)
# ---------------------------------------------------------------------------


def interp5(r: np.ndarray, table: np.ndarray, x) -> np.ndarray:
    """Lagrange interpolation of table[..., Nr] at x on nodes j-2..j+2 (r_j <= x < r_{j+1}), clamped;
    zero beyond the last grid point."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    Nr = r.size
    j = np.searchsorted(r, x, side="right") - 1
    s = np.clip(j - 2, 0, Nr - 5)
    nodes = s[:, None] + np.arange(5)[None, :]           # [nx, 5]
    rn = r[nodes]
    L = np.ones((x.size, 5))
    for a in range(5):
        for b in range(5):
            if a != b:
                L[:, a] *= (x - rn[:, b]) / (rn[:, a] - rn[:, b])
    vals = np.einsum("...xk,xk->...x", table[..., nodes], L)
    return np.where(x > r[-1], 0.0, vals)


# ---------------------------------------------------------------------------
# Eq. 7: radial multipole integrals
# ---------------------------------------------------------------------------


def radial_F_at_nodes(grid, fa: np.ndarray, fb: np.ndarray, lam: int, idx: np.ndarray) -> np.ndarray:
    """F_lam(R) = int r^2 fa fb min(r,R)^lam / max(r,R)^(lam+1) dr on the grid's own rule, at R = r[idx].

    fa, fb: [npair, Nr]; returns [npair, len(idx)]."""
    r, w = grid.r, grid.w
    R = r[idx]
    rmin = np.minimum(r[:, None], R[None, :])
    rmax = np.maximum(r[:, None], R[None, :])
    kern = rmin ** lam / rmax ** (lam + 1)                # [Nr, nidx]
    return (fa * fb * (w * r * r)[None, :]) @ kern


def radial_F(grid, fa, fb, lam: int, R: float) -> np.ndarray:
    """F_lam at an off-grid R: table values on the 5 stencil nodes, then 5-point interpolation.

    Beyond the last grid point every radial function vanishes, so the whole charge
    distribution lies inside R and F_lam(R) = F_lam(r_max) (r_max / R)^(lam+1)."""
    r = grid.r
    if R > r[-1]:
        return radial_F_at_nodes(grid, fa, fb, lam, np.array([r.size - 1]))[:, 0] * (r[-1] / R) ** (lam + 1)
    j = np.searchsorted(r, R, side="right") - 1
    s = int(np.clip(j - 2, 0, r.size - 5))
    idx = np.arange(s, s + 5)
    Fn = radial_F_at_nodes(grid, fa, fb, lam, idx)        # [npair, 5]
    full = np.zeros((fa.shape[0], r.size))
    full[:, idx] = Fn
    return interp5(r, full, R)[:, 0]


# ---------------------------------------------------------------------------
# Eq. 6: direct elements
# ---------------------------------------------------------------------------


def _direct_angular(centre) -> np.ndarray:
    """z-independent part of Eq. 6 for every (a', a, lam):
    sqrt((2l_a+1)/(2l_a'+1)) sqrt((lam-mu)!/(lam+mu)!) C^{l_a' 0}_{lam 0 l_a 0} C^{l_a' m_a'}_{lam mu l_a m_a}.
    It depends on the states' (l', m', l, m) only: tabulated over those, then gathered per state pair."""
    key = "_oracle_direct_angular"
    if hasattr(centre, key):
        return getattr(centre, key)
    lmax = int(centre.rad_l.max())
    nl, L = 2 * lmax + 1, lmax
    tab = np.zeros((lmax + 1, 2 * lmax + 1, lmax + 1, 2 * lmax + 1, nl))
    for lp in range(lmax + 1):
        for mp in range(-lp, lp + 1):
            for l in range(lmax + 1):
                for m in range(-l, l + 1):
                    mu = mp - m
                    for lam in range(abs(lp - l), lp + l + 1):
                        if (lp + l + lam) % 2 or abs(mu) > lam:
                            continue
                        a = math.sqrt((2 * l + 1) / (2 * lp + 1)) * math.sqrt(
                            math.factorial(lam - mu) / math.factorial(lam + mu))
                        tab[lp, mp + L, l, m + L, lam] = (
                            a * clebsch_gordan(lam, 0, l, 0, lp, 0) * clebsch_gordan(lam, mu, l, m, lp, mp))
    sl, sm = centre.st_l, centre.st_m + L
    ang = tab[sl[:, None], sm[:, None], sl[None, :], sm[None, :], :]
    setattr(centre, key, ang)
    return ang


def direct_block(grid, centre, Z_other: float, R: float, cos_theta: float, other_at_minus_R: bool,
                 f_left=None, f_right=None) -> np.ndarray:
    """D[a', a] = -Z sum_lam sqrt((2l_a+1)/(2l_a'+1)) sqrt((lam-mu)!/(lam+mu)!)
    C^{l_a' 0}_{lam 0 l_a 0} C^{l_a' m_a'}_{lam mu l_a m_a} P_lam^mu(cos Theta) F_{a'a lam}(R), mu = m_a' - m_a.

    The other nucleus sits at +R (azimuth 0) from this centre, or at -R for the projectile
    centre (other_at_minus_R), which multiplies the lam-th multipole by (-1)^lam.
    f_left / f_right replace the bra's / ket's radial tables in Eq. 7 (the element is bilinear in them;
    the differentiation form passes derivative tables here)."""
    lmax = int(centre.rad_l.max())
    nl = 2 * lmax + 1
    ang = _direct_angular(centre)
    nrad = centre.n_rad
    # F_{a'a lam}(R) for every radial pair (zero where the pair cannot couple through lam)
    Ftab = np.zeros((nrad, nrad, nl))
    la = centre.rad_l
    for lam in range(nl):
        ok = (np.abs(la[:, None] - la[None, :]) <= lam) & (la[:, None] + la[None, :] >= lam) \
            & ((la[:, None] + la[None, :] + lam) % 2 == 0)
        pa, pb = np.nonzero(ok)
        if pa.size:
            fl = centre.f if f_left is None else f_left
            fr = centre.f if f_right is None else f_right
            Ftab[pa, pb, lam] = radial_F(grid, fl[pa], fr[pb], lam, R)
    # P_lam^mu(cos Theta) for -lam <= mu <= lam
    Pv = np.zeros((nl, 2 * nl + 1))
    for lam in range(nl):
        for mu in range(-lam, lam + 1):
            Pv[lam, mu + nl] = float(assoc_legendre(lam, mu, cos_theta))
    sign = np.array([(-1.0) ** lam if other_at_minus_R else 1.0 for lam in range(nl)])
    mu = centre.st_m[:, None] - centre.st_m[None, :]                          # [N, N]
    Pl = Pv[np.arange(nl)[None, None, :], (mu + nl)[:, :, None]]              # [N, N, nl]
    Fl = Ftab[centre.st_rad[:, None], centre.st_rad[None, :], :]              # [N, N, nl]
    return -Z_other * np.sum(ang * Pl * Fl * sign[None, None, :], axis=2)


# ---------------------------------------------------------------------------
# Eq. 9 (molecular frame) and Eq. 8 (rotation): S_TP, Q and Q~'
# ---------------------------------------------------------------------------


def target_sr_potential(basis, r):
    """Short-range part of a Li-like target potential, -c e^{-a r}(1 + b r)/r (zero for a bare nucleus)."""
    return -basis.mp_c * np.exp(-basis.mp_a * r) * (1.0 + basis.mp_b * r) / r


def target_potential(basis, r):
    """V_T(r) = -Z_T/r plus the short-range part of a model potential."""
    if basis.mp_c == 0.0:
        return -basis.Z_T / r
    return -basis.Z_T / r + target_sr_potential(basis, r)


def _nodes(basis, b: float, v: float, z: float):
    """(eta, tau) rule of Eq. 9 at one position: node radii and cosines about both centres, the
    Bessel argument, and the weights (R^3/8) w (eta^2 - tau^2) with and without the ETF phase."""
    qd = basis.quad
    R = math.sqrt(b * b + z * z)
    gR = qd.gamma * R
    eta = 1.0 + qd.s / gR                                   # [Ge]
    weta = qd.ws / gR
    E, Tt = np.meshgrid(eta, qd.tau, indexing="ij")         # [Ge, Gt]
    W0 = np.outer(weta, qd.wtau)
    E, Tt, W0 = E.ravel(), Tt.ravel(), W0.ravel()
    rT = 0.5 * R * (E + Tt)
    rP = 0.5 * R * (E - Tt)
    cT = (E * Tt + 1.0) / (E + Tt)
    cP = (E * Tt - 1.0) / (E - Tt)
    x = 0.5 * v * b * np.sqrt((E * E - 1.0) * (1.0 - Tt * Tt))
    vol = (R ** 3 / 8.0) * W0 * (E * E - Tt * Tt)
    base = vol * np.exp(0.5j * v * z * E * Tt)
    return dict(rT=rT, rP=rP, cT=cT, cP=cP, x=x, base=base, vol=vol)


def _state_tables(centre, ftab, rnode, cnode, r):
    """A[i, g] = f_{a_i}(r_g) Theta_{l_i q_i}(c_g) for every state, with m read as the frame's q."""
    fn = interp5(r, ftab, rnode)
    return np.array([fn[centre.st_rad[i]] * norm_legendre(int(centre.st_l[i]), int(centre.st_m[i]), cnode)
                     for i in range(centre.N)])


def molecular_integrals(basis, b: float, v: float, z: float, reverse: bool = False, fT=None, fP=None,
                        factors=None):
    """Molecular-frame integrals for every (target state in frame q', projectile state in frame q):
    X[i, j] = (R^3/8) sum_{eta,tau} w (eta^2 - tau^2) e^{i v z eta tau / 2} (-i)^{q-q'} J_{q-q'}(x)
              f_i(r_T) Theta_{l_i q'}(c_T) f_j(r_P) Theta_{l_j q}(c_P) * u(eta, tau)
    with u = 1 (overlap K) and V_T(r_T) (transfer Q: -Z_T/r_T for a bare target); with reverse=True
    also -Z_P/r_P (the reverse-transfer integral, before conjugation, used only to show why Q^+ is
    taken instead).  Rows/columns use the centres' own state lists with m read as the molecular-frame q.
    fT / fP replace the radial tables and `factors` (callables of (r_T, r_P)) the list of u; each
    integral is linear in each of them (the differentiation form uses that)."""
    T, P = basis.T, basis.P
    nd = _nodes(basis, b, v, z)
    rT, rP, x, base = nd["rT"], nd["rP"], nd["x"], nd["base"]
    r = basis.grid.r
    AT = _state_tables(T, T.f if fT is None else fT, rT, nd["cT"], r)
    AP = _state_tables(P, P.f if fP is None else fP, rP, nd["cP"], r)
    dmax = int(T.st_l.max() + P.st_l.max())
    Wd = {}
    for d in range(-dmax, dmax + 1):
        Wd[d] = base * ((-1j) ** d) * special.jv(d, x)
    if factors is None:
        factors = [lambda a, c: np.ones_like(a), lambda a, c: target_potential(basis, a)]
        if reverse:
            factors.append(lambda a, c: -basis.Z_P / c)
    out = []
    for fac in factors:
        u = fac(rT, rP)
        X = np.zeros((T.N, P.N), dtype=np.complex128)
        for q in sorted(set(int(m) for m in P.st_m)):
            cols = np.nonzero(P.st_m == q)[0]
            # row i gets W_{q - q'_i}: a per-row choice of the Delta q weight
            Wrow = np.array([Wd[q - int(T.st_m[i])] for i in range(T.N)]) * u[None, :]
            At = AT * Wrow
            X[:, cols] = At.real @ AP[cols].T + 1j * (At.imag @ AP[cols].T)
        out.append(X)
    return out


def sr_direct_mol(basis, b: float, z: float, f_left=None, f_right=None, Vs=None) -> np.ndarray:
    """Short-range part of the target potential between projectile states, in the molecular frame:
    D[i, j] = delta_{q_i q_j} (R^3/8) sum_{eta,tau} w (eta^2 - tau^2) V_s(r_T) f_i(r_P) Theta_{l_i q}(c_P)
              f_j(r_P) Theta_{l_j q}(c_P)
    on the (eta, tau) rule of Eq. 9 (the potential is symmetric about the molecular axis, so the phi
    integral only couples equal q; both states sit on the projectile, so no ETF phase remains).
    Vs (a callable of r_T) defaults to the basis's own short-range potential."""
    P = basis.P
    nd = _nodes(basis, b, 1.0, z)
    r = basis.grid.r
    AL = _state_tables(P, P.f if f_left is None else f_left, nd["rP"], nd["cP"], r)
    AR = AL if (f_left is None and f_right is None) else \
        _state_tables(P, P.f if f_right is None else f_right, nd["rP"], nd["cP"], r)
    u = nd["vol"] * (target_sr_potential(basis, nd["rT"]) if Vs is None else Vs(nd["rT"]))
    D = (AL * u[None, :]) @ AR.T
    return D * (P.st_m[:, None] == P.st_m[None, :])


def rotate(centre_T, centre_P, Xmol: np.ndarray, theta: float) -> np.ndarray:
    """Eq. 8: K[beta, alpha] = sum_{q', q} d^{l_b}_{m_b q'}(theta) d^{l_a}_{m_a q}(theta) Xmol[(b, q'), (a, q)]."""
    return rotation_matrix(centre_T, theta) @ Xmol @ rotation_matrix(centre_P, theta).T


def rotation_matrix(c, theta: float) -> np.ndarray:
    """D[i, k] = d^{l}_{m_i m_k}(theta) between the states of one radial function (zero otherwise)."""
    Dm = np.zeros((c.N, c.N))
    for i in range(c.N):
        for k in range(c.N):
            if c.st_rad[i] == c.st_rad[k]:
                Dm[i, k] = wigner_d(int(c.st_l[i]), int(c.st_m[i]), int(c.st_m[k]), theta)
    return Dm


# ---------------------------------------------------------------------------
# Eq. 1 assembly, Eq. 4/5 solve, Algorithm 1
# ---------------------------------------------------------------------------


def phases(eps_row: np.ndarray, eps_col: np.ndarray, z: float, v: float) -> np.ndarray:
    return np.exp(1j * np.subtract.outer(eps_row, eps_col) * z / v)


def assemble(basis, b: float, v: float, z: float):
    """S and H (N x N complex) at projectile position z on the path (b, v)."""
    T, P = basis.T, basis.P
    R = math.sqrt(b * b + z * z)
    cth = z / R
    DT = direct_block(basis.grid, T, basis.Z_P, R, cth, other_at_minus_R=False)
    if P is None:
        S = np.eye(T.N, dtype=np.complex128)
        H = DT * phases(T.st_eps, T.st_eps, z, v)
        return S, H
    DP = direct_block(basis.grid, P, basis.Z_T, R, cth, other_at_minus_R=True)
    theta = math.acos(cth)
    if basis.mp_c != 0.0:
        DRP = rotation_matrix(P, theta)
        DP = DP + DRP @ sr_direct_mol(basis, b, z) @ DRP.T
    Smol, Qmol = molecular_integrals(basis, b, v, z)
    ph = phases(T.st_eps, P.st_eps, z, v)
    K = rotate(T, P, Smol, theta) * ph
    Q = rotate(T, P, Qmol, theta) * ph
    NT, N = T.N, basis.N
    S = np.eye(N, dtype=np.complex128)
    S[:NT, NT:] = K
    S[NT:, :NT] = K.conj().T
    H = np.zeros((N, N), dtype=np.complex128)
    H[:NT, :NT] = DT * phases(T.st_eps, T.st_eps, z, v)
    H[:NT, NT:] = Q
    H[NT:, :NT] = Q.conj().T          # Eq. 1: the lower-left block is Q^+
    H[NT:, NT:] = DP * phases(P.st_eps, P.st_eps, z, v)
    return S, H


def solve(S: np.ndarray, H: np.ndarray) -> np.ndarray:
    """X = S^{-1} H by LU with partial pivoting and N right-hand sides (LAPACK zgesv)."""
    return np.linalg.solve(S, H)


def coupling_M(basis, b: float, v: float, z: float) -> np.ndarray:
    """Eq. 4 (two-centre) or Eq. 5 (one-centre): M = -(i/v) S^{-1} H."""
    S, H = assemble(basis, b, v, z)
    if basis.P is None:
        return (-1j / v) * H
    return (-1j / v) * solve(S, H)


def rk4_path(Mfun, zgrid: np.ndarray, c0: np.ndarray) -> np.ndarray:
    """Algorithm 1: X advanced from zgrid[0] to zgrid[-1]; M evaluated at z_mid and z_new each step."""
    X = np.array(c0, dtype=np.complex128)
    Mnew = Mfun(zgrid[0])
    for i in range(zgrid.size - 1):
        z, znew = zgrid[i], zgrid[i + 1]
        zmid = (z + znew) / 2.0
        h = znew - z
        h2, h6 = h / 2.0, h / 6.0
        Mz = Mnew
        Mmid = Mfun(zmid)
        Mnew = Mfun(znew)
        K1 = Mz @ X
        K2 = Mmid @ X + h2 * (Mmid @ K1)
        K3 = Mmid @ X + h2 * (Mmid @ K2)
        K4 = Mnew @ X + h * (Mnew @ K3)
        X = X + h6 * (K1 + 2.0 * K2 + 2.0 * K3 + K4)
    return X


def initial_state(basis) -> np.ndarray:
    """Algorithm 1's start: all amplitudes zero but the first (the target ground state)."""
    c = np.zeros(basis.N, dtype=np.complex128)
    c[0] = 1.0
    return c


def propagate(basis, b: float, v: float, zgrid: np.ndarray, c0=None) -> np.ndarray:
    """Amplitudes at the end of one straight-line path."""
    if c0 is None:
        c0 = initial_state(basis)
    return rk4_path(lambda z: coupling_M(basis, b, v, z), zgrid, c0)


def probabilities(c: np.ndarray) -> np.ndarray:
    """P_i = |c_i|^2 at the end of the path."""
    return (c.conj() * c).real


# ---------------------------------------------------------------------------
# differentiation form: derivatives of S, H and the probabilities with respect to the parameters
# theta (projectile charge, model-potential parameters), forward mode
# ---------------------------------------------------------------------------


def _sr_potential_tangent(basis, p: int):
    """d V_s / d theta_p as a callable of r, through d(c, a, b)/d theta_p."""
    _, dc, da, db = basis.dexplicit[p]
    c, a, bb = basis.mp_c, basis.mp_a, basis.mp_b

    def dVs(r):
        e = np.exp(-a * r)
        return dc * (-e * (1.0 + bb * r) / r) + da * (c * e * (1.0 + bb * r)) + db * (-c * e)
    return dVs


def assemble_with_tangents(basis, b: float, v: float, z: float):
    """S, H at one position and their derivatives dS[p], dH[p] with respect to every parameter.

    Each block is multilinear in the radial tables of its bra and ket, the nuclear charge and the
    target potential, so its derivative is the sum of the same integrals with one ingredient replaced
    by its derivative (basis.tangent_T/P, basis.dexplicit).  The energy phases e^{i(eps_i - eps_j)z/v}
    contribute (i z/v)(d eps_i - d eps_j) times the element."""
    T, P, grid = basis.T, basis.P, basis.grid
    S, H = assemble(basis, b, v, z)
    NT, N = T.N, basis.N
    R = math.sqrt(b * b + z * z)
    cth = z / R
    theta = math.acos(cth)
    DRT, DRP = rotation_matrix(T, theta), rotation_matrix(P, theta)
    eps = np.concatenate([T.st_eps, P.st_eps])
    npar = basis.dexplicit.shape[0]
    dS, dH = [], []
    for p in range(npar):
        dZP = basis.dexplicit[p][0]
        dfT, dfP = basis.tangent_T.df[p], basis.tangent_P.df[p]
        dVs = _sr_potential_tangent(basis, p)
        # phase-free element derivatives
        dDT = (direct_block(grid, T, dZP, R, cth, False)
               + direct_block(grid, T, basis.Z_P, R, cth, False, f_left=dfT)
               + direct_block(grid, T, basis.Z_P, R, cth, False, f_right=dfT))
        dDP = (direct_block(grid, P, basis.Z_T, R, cth, True, f_left=dfP)
               + direct_block(grid, P, basis.Z_T, R, cth, True, f_right=dfP))
        dsr = (sr_direct_mol(basis, b, z, f_left=dfP) + sr_direct_mol(basis, b, z, f_right=dfP)
               + sr_direct_mol(basis, b, z, Vs=dVs))
        dDP = dDP + DRP @ dsr @ DRP.T
        one = lambda a, c: np.ones_like(a)
        VT = lambda a, c: target_potential(basis, a)
        dK1, dQ1 = molecular_integrals(basis, b, v, z, fT=dfT, factors=[one, VT])
        dK2, dQ2 = molecular_integrals(basis, b, v, z, fP=dfP, factors=[one, VT])
        dQ3, = molecular_integrals(basis, b, v, z, factors=[lambda a, c: dVs(a)])
        dK = DRT @ (dK1 + dK2) @ DRP.T
        dQ = DRT @ (dQ1 + dQ2 + dQ3) @ DRP.T
        ph = phases(eps, eps, z, v)
        deps = np.concatenate([basis.tangent_T.deps[p][T.st_rad], basis.tangent_P.deps[p][P.st_rad]])
        dph = (1j * z / v) * np.subtract.outer(deps, deps)
        # d(S), d(H): element derivative times the phase plus element times the phase derivative
        Sd = np.zeros((N, N), dtype=np.complex128)
        Sd[:NT, NT:] = dK * ph[:NT, NT:] + S[:NT, NT:] * dph[:NT, NT:]
        Sd[NT:, :NT] = Sd[:NT, NT:].conj().T
        Hd = np.zeros((N, N), dtype=np.complex128)
        Hd[:NT, :NT] = dDT * ph[:NT, :NT] + H[:NT, :NT] * dph[:NT, :NT]
        Hd[:NT, NT:] = dQ * ph[:NT, NT:] + H[:NT, NT:] * dph[:NT, NT:]
        Hd[NT:, :NT] = Hd[:NT, NT:].conj().T
        Hd[NT:, NT:] = dDP * ph[NT:, NT:] + H[NT:, NT:] * dph[NT:, NT:]
        dS.append(Sd)
        dH.append(Hd)
    return S, H, dS, dH


def coupling_M_with_tangents(basis, b: float, v: float, z: float):
    """M = -(i/v) S^{-1} H and dM[p] = -(i/v) S^{-1} (dH[p] - dS[p] S^{-1} H)."""
    S, H, dS, dH = assemble_with_tangents(basis, b, v, z)
    X = solve(S, H)
    return (-1j / v) * X, [(-1j / v) * solve(S, dH[p] - dS[p] @ X) for p in range(len(dS))]


def gradient(basis, b: float, v: float, zgrid: np.ndarray, g: np.ndarray, c0=None):
    """Observables P_o = sum_i g[o, i] |c_i|^2 at the end of one path and dP_o/d theta_p.

    Forward mode: every line of Algorithm 1 is differentiated alongside it (dK1 = dM_z X + M_z dX, ...),
    so the result is the exact derivative of the discrete RK4 propagation.  Returns (P [n_obs],
    dP [n_obs, n_par], c at the end)."""
    if c0 is None:
        c0 = initial_state(basis)
    npar = basis.dexplicit.shape[0]
    X = np.array(c0, dtype=np.complex128)
    dX = np.zeros((npar, X.size), dtype=np.complex128)
    Mnew, dMnew = coupling_M_with_tangents(basis, b, v, zgrid[0])
    for i in range(zgrid.size - 1):
        z, znew = zgrid[i], zgrid[i + 1]
        zmid = (z + znew) / 2.0
        h = znew - z
        h2, h6 = h / 2.0, h / 6.0
        Mz, dMz = Mnew, dMnew
        Mmid, dMmid = coupling_M_with_tangents(basis, b, v, zmid)
        Mnew, dMnew = coupling_M_with_tangents(basis, b, v, znew)
        K1 = Mz @ X
        K2 = Mmid @ X + h2 * (Mmid @ K1)
        K3 = Mmid @ X + h2 * (Mmid @ K2)
        K4 = Mnew @ X + h * (Mnew @ K3)
        for p in range(npar):
            dK1 = dMz[p] @ X + Mz @ dX[p]
            dK2 = dMmid[p] @ X + Mmid @ dX[p] + h2 * (dMmid[p] @ K1 + Mmid @ dK1)
            dK3 = dMmid[p] @ X + Mmid @ dX[p] + h2 * (dMmid[p] @ K2 + Mmid @ dK2)
            dK4 = dMnew[p] @ X + Mnew @ dX[p] + h * (dMnew[p] @ K3 + Mnew @ dK3)
            dX[p] = dX[p] + h6 * (dK1 + 2.0 * dK2 + 2.0 * dK3 + dK4)
        X = X + h6 * (K1 + 2.0 * K2 + 2.0 * K3 + K4)
    g = np.atleast_2d(np.asarray(g, dtype=np.float64))
    Pobs = g @ probabilities(X)
    dP = 2.0 * np.real(g @ (X.conj()[:, None] * dX.T))
    return Pobs, dP, X
