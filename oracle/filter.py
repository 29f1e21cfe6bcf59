"""Adaptive modal filter (oracle, FP64; Sec. 3.3, the paragraph on the optional filter).

Between time steps every coefficient whose normalised mode index
    zeta(n, m, k) = max(n / (Nc - 1), m / (M - 1), |k| / (Kz - 1))     (a term is 0 when its
                                                                        truncation keeps one index)
lies above the cutoff zeta_c is multiplied by
    sigma = exp(-eps ((zeta - zeta_c) / (1 - zeta_c))^8),
and the amplitude eps follows the fraction f of the field's spectral energy
(sum of |shat|^2 with multiplicity 2 for m >= 1) carried by those coefficients:
    eps* = eps_max * min(1, max(0, (f - tau) / tau))     (inactive below tau, saturated at 2 tau)
    eps  <- eps + beta (eps* - eps)                      (relaxed across steps, bounded by eps_max)
with f measured on the field before it is filtered; every field has its own eps.

The paper fixes the form of sigma, the tail-fraction rule and tau = 2e-2 (2 % of the
spectral energy) as the default, and says the response is bounded and relaxed
across steps.  Readings where it is silent: zeta normalised by the last retained
index (sigma = exp(-eps) at the truncation edge), zeta_c = 2/3, eps_max = 36
(exp(-36) ~ 2e-16: at saturation the edge mode is removed to round-off), a linear
ramp between tau and 2 tau, beta = 1/4, eps starting at 0.

Pins (tests/test_oracle_filter.py): sigma = 1 at the cutoff and exp(-eps) at the
edge; the tail fraction against a brute-force enumeration of the modes; a field
below the target passes unchanged; the relaxation's closed form
eps_j = eps_max (1 - (1 - beta)^j) at a saturated tail; the damping of each mode
against the formula.
"""

import math

import numpy as np

DEFAULTS = dict(zeta_c=2.0 / 3.0, tau=2e-2, eps_max=36.0, relax=0.25)


def zeta(g, m, kidx):
    """zeta over the n = m..Nc-1 coefficients of block (m, k)."""
    n = np.arange(m, g.nc, dtype=np.float64)
    zn = n / (g.nc - 1) if g.nc > 1 else 0.0 * n
    zm = m / (g.M - 1) if g.M > 1 else 0.0
    zk = abs(int(g.kz[kidx])) / (g.Kz - 1) if g.Kz > 1 else 0.0
    return np.maximum(np.maximum(zn, zm), zk)


def tail_fraction(g, spec, zeta_c):
    tail = tot = 0.0
    for m in range(g.M):
        w = 1.0 if m == 0 else 2.0
        for kk in range(g.K):
            e = np.abs(spec[m][kk]) ** 2
            tot += w * float(np.sum(e))
            tail += w * float(np.sum(e[zeta(g, m, kk) > zeta_c]))
    return tail / tot if tot > 0 else 0.0


def sigma(z, eps, zeta_c):
    """The filter's multiplier for normalised index z (1 at and below the cutoff)."""
    q = np.clip((np.asarray(z, dtype=np.float64) - zeta_c) / (1.0 - zeta_c), 0.0, None)
    return np.exp(-eps * q ** 8)


def update_eps(eps, f, tau, eps_max, relax):
    target = eps_max * min(1.0, max(0.0, (f - tau) / tau))
    return min(eps_max, max(0.0, eps + relax * (target - eps)))


def apply(g, spec, eps, params=None):
    """One filter step on one field: returns (filtered spec, new eps, tail fraction)."""
    p = dict(DEFAULTS, **(params or {}))
    f = tail_fraction(g, spec, p["zeta_c"])
    eps = update_eps(eps, f, p["tau"], p["eps_max"], p["relax"])
    out = []
    for m in range(g.M):
        blk = spec[m].copy()
        for kk in range(g.K):
            z = zeta(g, m, kk)
            above = z > p["zeta_c"]
            blk[kk, above] = blk[kk, above] * sigma(z[above], eps, p["zeta_c"])
        out.append(blk)
    return out, eps, f


class FieldFilter:
    """Filter state of a state with nfields fields (blocks [field 0 m-blocks..., field 1 ...])."""

    def __init__(self, g, nfields=1, params=None):
        self.g, self.nf = g, nfields
        self.params = dict(DEFAULTS, **(params or {}))
        self.eps = [0.0] * nfields
        self.tail = [0.0] * nfields

    def __call__(self, state):
        g = self.g
        out = []
        for f in range(self.nf):
            blk, self.eps[f], self.tail[f] = apply(g, state[f * g.M:(f + 1) * g.M], self.eps[f], self.params)
            out += blk
        return out
