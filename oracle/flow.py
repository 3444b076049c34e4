"""Explicit multiphase terms that feed the pressure solve (ORACLE, test use only).

Volume-fraction advection with the compressive Petrov-Galerkin diffusion (Sections 2.3.1 and
2.3.5-2.3.6; Eqs. Petrov-C, Petrov-Cs, a_psi, efficient-kabs, Sx-lin, negativek, normalisation,
positivek, alpha_min_and_max, transport-indicator-1) and the lumped-mass total of C used by the
mass diagnostic of Section 3.  Every step is written out in the paper's order and notation with
the assembled Q1 filters of ``fem``.

Readings where the paper is silent (see also the module docstring of ``mg``):
  * Psi_d inside the Petrov-Galerkin and interface formulas is the pointwise gradient
    m_i^-1 f(Psi; w_d), m_i the lumped nodal volume (h_x h_y h_z inside, halved per boundary);
    the residual terms use the raw filters and the update divides by m_i.
  * The advection velocity of Stage 4 is u^{n+1} throughout.
  * The VOF diffusion is k^d of the compressive scheme with k^{d+} = 3 k_abs (general-spacing
    k_abs), clamped to [-k_min, k_max]; the oscillation detector uses the copy-halo of Section
    2.3.3 at walls (so S = 0 there) and the linear (3x3x3) form.
  * "w_m / m_l - E" in Eq. a_psi divides by the lumped nodal volume m_i.
Parity status: the mass sum is pinned by exact quadrature identities.  The VOF step is pinned
by closed forms of every intermediate (gradient, a_C, k_abs, detectors with the override, w+ and
w-, u*, k^-, the clamped k^d) on a separable cubic field with anisotropic spacing, derived by
Taylor expansion, and by invariants (uniform field, linear profile weights, 1D-invariant
advection, mass conservation in a divergence-free flow, mirror and axis-exchange symmetry, the
printed constants).  The momentum predictor is pinned by closed forms of a, k_abs, k_square,
k_max and k_Psi (each branch of the min reached), the exact advection of a linear velocity
field, mirror symmetry and the hydrostatic rest state; the surface tension by a plane interface
(no force) and by the curvature 2/r of a sphere; the pressure right-hand sides and the velocity
correction by the hydrostatic column, a divergence-free uniform-density field and a linear
pressure.  tests/test_oracle_flow.py plants nineteen slips in a copy of this module and checks
that each one fails a pin.
"""

from dataclasses import dataclass

import numpy as np

from . import fem


@dataclass(frozen=True)
class VOFParams:
    """Constants of Sections 2.3.5-2.3.6 (values as printed)."""
    alpha_a: float = 2.0           # Eq. a_psi
    p: int = 1                     # polynomial order of the linear filters
    eps_k: float = 1e-7            # Eq. k-abs
    K_plus: float = 300.0          # weights w+, w-
    K_minus: float = 300.0
    beta: float = 0.1              # Eq. negativek
    eps_x: float = 1e-4            # Eqs. negativek, normalisation
    K_pos: float = 3.0             # Eq. positivek
    alpha_min: float = 1e-4        # Eq. alpha_min_and_max
    alpha_max: float = 0.05
    detect_hi: float = 0.95        # detector override thresholds
    detect_lo: float = 0.05

    @property
    def alpha_kabs(self):
        return 1.0 / (8.0 * 2 ** self.p)


def mass_sum(shape, h, C):
    """Total volume fraction sum_i m_i C_i (lumped nodal volume m_i); the C(t) of the mass
    diagnostic, computed in FP64."""
    return float((fem.lumped_mass(shape, h) * np.asarray(C, dtype=np.float64)).sum())


def _detector(C, axis):
    """S = (C_i - C_{i-1})(C_{i+1} - C_i) along `axis` with the copy-halo (C_{-1} = C_0)."""
    Cp = np.concatenate([np.take(C, [0], axis=axis), C, np.take(C, [-1], axis=axis)], axis=axis)
    n = C.shape[axis]
    lo = np.take(Cp, np.arange(0, n), axis=axis)
    mid = np.take(Cp, np.arange(1, n + 1), axis=axis)
    hi = np.take(Cp, np.arange(2, n + 2), axis=axis)
    return (mid - lo) * (hi - mid)


def vof_step(shape, h, C, u, v, w, dt, prm=VOFParams()):
    """One Stage-4 update; returns (s_C, C_next, parts) with parts the intermediate fields.

    Arrays are indexed [z, y, x]; h = (hx, hy, hz); (u, v, w) = q^{n+1}.
    """
    C = np.asarray(C, dtype=np.float64)
    vel = [np.asarray(u, dtype=np.float64), np.asarray(v, dtype=np.float64), np.asarray(w, dtype=np.float64)]
    ei = fem.element_integrals(h)
    m = fem.lumped_mass(shape, h)
    f_d = [fem.apply_assembled(ei["grad"][d], C) for d in range(3)]       # f(C; w_d)
    Cd = [f_d[d] / m for d in range(3)]                                    # pointwise gradient
    # advection residual, Eq. a_psi: alpha_a f(u.grad C; w_m/m - E)
    g_adv = vel[0] * Cd[0] + vel[1] * Cd[1] + vel[2] * Cd[2]
    a_C = prm.alpha_a * (fem.apply_assembled(ei["mass"], g_adv) / m - g_adv)
    # first residual-based coefficient, general spacing, Eq. efficient-kabs
    absd = [np.abs(c) for c in Cd]
    sum_abs = absd[0] + absd[1] + absd[2]
    k_abs = (prm.alpha_kabs * np.abs(a_C) * (h[0] * absd[0] + h[1] * absd[1] + h[2] * absd[2])
             / (prm.eps_k + sum_abs ** 2 / 3.0))
    # oscillation detectors, Eqs. Sx-lin..Sz-lin, with the 0.95 / 0.05 override
    over = (C > prm.detect_hi) | (C < prm.detect_lo)
    S = []
    for d, axis in enumerate((2, 1, 0)):
        s = _detector(C, axis)
        S.append(np.where(over, -1.0, s))
    w_plus = [-np.maximum(-1.0, np.minimum(0.0, prm.K_plus * s)) for s in S]
    w_minus = [np.minimum(1.0, np.maximum(0.0, prm.K_minus * s)) for s in S]
    # negative diffusion, Eqs. negativek and normalisation
    gradsq = Cd[0] ** 2 + Cd[1] ** 2 + Cd[2] ** 2
    proj = (vel[0] * Cd[0] + vel[1] * Cd[1] + vel[2] * Cd[2]) / (prm.eps_x + gradsq)
    ustar = [Cd[d] * proj for d in range(3)]
    speed2 = vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2
    k_neg = -prm.beta * speed2 / (prm.eps_x + gradsq * (np.abs(ustar[0]) + np.abs(ustar[1]) + np.abs(ustar[2])) / 3.0)
    # directional coefficients, positive part (Eq. positivek), combination and clamp
    k_min = prm.alpha_min * max(h) ** 2 / dt
    k_max = prm.alpha_max * min(h) ** 2 / dt
    kd = []
    for d in range(3):
        k_plus = prm.K_pos * k_abs
        k_minus = k_neg / h[d]
        k = w_plus[d] * k_plus + w_minus[d] * k_minus
        kd.append(np.maximum(-k_min, np.minimum(k_max, k)))
    # Eq. Petrov-Cs: advection with raw filters plus directional PG diffusion (Eq. k-Txx)
    s_C = vel[0] * f_d[0] + vel[1] * f_d[1] + vel[2] * f_d[2]
    for d in range(3):
        D = ei["dd"][d]
        s_C = s_C + 0.5 * (fem.apply_assembled(D, kd[d] * C) + kd[d] * fem.apply_assembled(D, C)
                           - C * fem.apply_assembled(D, kd[d]))
    # Eq. transport-indicator-1: C^{n+1} = C^n - dt m^-1 s_C
    C_next = C - dt * s_C / m
    parts = {"grad": Cd, "a_C": a_C, "k_abs": k_abs, "S": S, "w_plus": w_plus, "w_minus": w_minus,
             "k_neg": k_neg, "k": kd}
    return s_C, C_next, parts


# ---------------------------------------------------------------- Navier-Stokes terms

@dataclass(frozen=True)
class FlowParams:
    """Physical constants of one run (Sections 2.1, 2.3.2, 2.3.5) and the momentum scheme's."""
    rho_l: float = 1000.0
    rho_g: float = 1.0
    mu_l: float = 1e-3
    mu_g: float = 1.8e-5
    sigma_t: float = 0.07          # surface tension coefficient
    g: float = 9.81                # gravity magnitude, acting along -z
    alpha_a: float = 2.0           # Eq. a_psi
    p: int = 1
    eps_k: float = 1e-7            # Eqs. k-abs, h_Psi, k-square

    @property
    def alpha_kabs(self):
        return 1.0 / (8.0 * 2 ** self.p)

    @property
    def alpha_ksquare(self):
        return 8.0 / 2 ** self.p


def density(C, prm):
    """Eq. density-n: rho = rho_l C + rho_g (1 - C)."""
    return prm.rho_l * C + prm.rho_g * (1.0 - C)


def viscosity(C, prm):
    """mu = mu_l C + mu_g (1 - C) (reading: the paper's scalar mu, made two-phase)."""
    return prm.mu_l * C + prm.mu_g * (1.0 - C)


def _filters(shape, h):
    ei = fem.element_integrals(h)
    m = fem.lumped_mass(shape, h)
    return ei, m


def pointwise_gradient(shape, h, f):
    """m^-1 f(f; w_d), d = x, y, z."""
    ei, m = _filters(shape, h)
    return [fem.apply_assembled(ei["grad"][d], f) / m for d in range(3)]


def surface_tension(shape, h, C, prm):
    """Eqs. surface-tension-k and surface-tension-uvw: n = grad C / (eps_t + |grad C|),
    kappa = m^-1 sum_d f(n_d; w_d) (the printed w_v of the z term read as w_z),
    s_t = sigma_t kappa grad C; eps_t = 1e-7 / h with h the smallest spacing (reading)."""
    ei, m = _filters(shape, h)
    Cd = pointwise_gradient(shape, h, C)
    eps_t = 1e-7 / min(h)
    norm = np.sqrt(Cd[0] ** 2 + Cd[1] ** 2 + Cd[2] ** 2)
    nd = [Cd[d] / (eps_t + norm) for d in range(3)]
    kappa = sum(fem.apply_assembled(ei["grad"][d], nd[d]) for d in range(3)) / m
    return [prm.sigma_t * kappa * Cd[d] for d in range(3)], kappa


def pressure_rhs_hydrostatic(shape, h, C, prm, dirichlet_mask=None):
    """Stage 1 (Eq. hydro-pressure / Eq. ph_disc): the weak form int grad N . (s_q + s_t) with
    s_q = -rho g e_z, i.e. b = sum_d G_d^T s_d (G_d the assembled first-derivative filter w_d).
    With A the weak -laplacian this gives dp/dn = s.n on natural faces (the bottom condition
    dp_hs/dz = -rho g of Section 2.3.3)."""
    ei, _ = _filters(shape, h)
    st, _ = surface_tension(shape, h, C, prm)
    s = [st[0], st[1], st[2] - prm.g * density(C, prm)]
    b = sum(fem.apply_assembled(ei["grad"][d].T, s[d]) for d in range(3))
    if dirichlet_mask is not None:
        b = np.where(dirichlet_mask, 0.0, b)
    return b


def pressure_rhs_correction(shape, h, rho, ut, dt, dirichlet_mask=None):
    """Stage 3 (Eq. ph_disc2): b = -(1/dt) [ sum_d f(rho u~_d; w_d) - sum_d u~_d f(rho; w_d) ]."""
    ei, _ = _filters(shape, h)
    b = np.zeros(shape)
    for d in range(3):
        G = ei["grad"][d]
        b -= (fem.apply_assembled(G, rho * ut[d]) - ut[d] * fem.apply_assembled(G, rho)) / dt
    if dirichlet_mask is not None:
        b = np.where(dirichlet_mask, 0.0, b)
    return b


def velocity_correction(shape, h, rho, dp, dt, wall_mask=None):
    """Eq. vel-cor: du_d = -dt m^-1 f(dp; w_d) / rho (zero on no-slip walls)."""
    ei, m = _filters(shape, h)
    out = []
    for d in range(3):
        du = -dt * fem.apply_assembled(ei["grad"][d], dp) / (m * rho)
        if wall_mask is not None:
            du = np.where(wall_mask, 0.0, du)
        out.append(du)
    return out


def momentum_predict(shape, h, C, un, uh, p_total, dt, prm, wall_mask=None, parts=None):
    """One Stage-2 iteration (Eqs. Petrov-u/v/w, k_Psi-n, k-abs, k-square, max-k, velocity-1).

    un: velocity at level n; uh: the current u^{n+1/2}; p_total = p_hs + p_nh.  For each component
    Psi:  s~ = rho (u.grad_raw Psi) + f^lap(Psi, k_Psi; w_lap) + f(p; w_d) - f(s_Psi + s_tPsi; w_m),
    with k_Psi = rho min(k_max, k_abs, k_square) + mu computed from u^{n+1/2} (reading), then
    Psi~ = Psi^n - dt s~ / (m rho) (sigma = 0).  Returns (u~, u^{n+1/2} = (u^n + u~) / 2).
    If ``parts`` is a dict it receives the per-component intermediate fields (lists over the
    component c): "a" (Eq. a_psi), "k_abs", "k_square", "k" (Eq. k_Psi-n) and "k_max" (Eq. max-k).
    """
    ei, m = _filters(shape, h)
    rho = density(C, prm)
    mu = viscosity(C, prm)
    st, _ = surface_tension(shape, h, C, prm)
    src = [st[0], st[1], st[2] - prm.g * rho]          # s_Psi + s_tPsi (buoyancy on w only)
    L = ei["stiff"]
    kmax = h[0] * np.abs(uh[0]) + h[1] * np.abs(uh[1]) + h[2] * np.abs(uh[2])   # Eq. max-k
    ut = []
    rec = {"a": [], "k_abs": [], "k_square": [], "k": [], "k_max": kmax}
    for c in range(3):
        psi = uh[c]
        raw = [fem.apply_assembled(ei["grad"][d], psi) for d in range(3)]
        pd = [raw[d] / m for d in range(3)]
        gpsi = uh[0] * pd[0] + uh[1] * pd[1] + uh[2] * pd[2]
        a = prm.alpha_a * (fem.apply_assembled(ei["mass"], gpsi) / m - gpsi)        # Eq. a_psi
        ab = [np.abs(q) for q in pd]
        sab = ab[0] + ab[1] + ab[2]
        hsum = h[0] * ab[0] + h[1] * ab[1] + h[2] * ab[2]
        k_abs = prm.alpha_kabs * np.abs(a) * hsum / (prm.eps_k + sab ** 2 / 3.0)   # Eq. efficient-kabs
        h_psi = hsum / (prm.eps_k + sab)                                             # Eq. h_Psi
        k_sq = (prm.alpha_ksquare * a * a * h_psi /
                (prm.eps_k + (np.abs(uh[0] * pd[0]) + np.abs(uh[1] * pd[1]) + np.abs(uh[2] * pd[2]))
                 * (pd[0] ** 2 + pd[1] ** 2 + pd[2] ** 2) / 3.0))                   # Eq. k-square
        k = rho * np.minimum(kmax, np.minimum(k_abs, k_sq)) + mu                     # Eq. k_Psi-n
        for key, val in (("a", a), ("k_abs", k_abs), ("k_square", k_sq), ("k", k)):
            rec[key].append(val)
        s = rho * (uh[0] * raw[0] + uh[1] * raw[1] + uh[2] * raw[2])
        s = s + 0.5 * (fem.apply_assembled(L, k * psi) + k * fem.apply_assembled(L, psi)
                       - psi * fem.apply_assembled(L, k))                            # Eq. k-T
        s = s + fem.apply_assembled(ei["grad"][c], p_total)
        s = s - fem.apply_assembled(ei["mass"], src[c])
        u_new = un[c] - dt * s / (m * rho)                                           # Eq. velocity-1
        if wall_mask is not None:
            u_new = np.where(wall_mask, 0.0, u_new)
        ut.append(u_new)
    if parts is not None:
        parts.update(rec)
    return ut, [0.5 * (un[c] + ut[c]) for c in range(3)]
