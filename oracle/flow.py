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
Parity status: the mass sum is pinned by exact quadrature identities; the VOF step is pinned by
the invariants in tests/test_oracle_flow.py (uniform field, linear profile weights, 1D-invariant
advection, the printed constants) and is otherwise "parity unpinned" (no printed example).
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
