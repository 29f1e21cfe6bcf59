"""Semi-implicit time integration of Eq. (10) (oracle, FP64).

ds/dt = A(s, t) + L s with L of Eq. (11), applied per harmonic (m, k).

* FE-BE:  (I - dt L) s^{j+1} = s^j + dt A^j
* AB-CN:  (I - dt/2 L) s^{j+1} = (I + dt/2 L) s^j + dt/2 (3 A^j - A^{j-1})   (Eq. (12))
* Start-up (Sec. 3.3: "Richardson extrapolation from FE-BE substeps"):
      s^1 = 2 FEBE_{dt/2}(FEBE_{dt/2}(s^0)) - FEBE_dt(s^0),
  and A^0 = A(s^0) serves as A^{j-1} in the first AB-CN step.  This reading
  reproduces every digit of the paper's Table 2.

The implicit matrices depend on (m, kappa^2) only, so one LU factorisation per
(m, |k|) is made (scipy.linalg.lu_factor, LAPACK getrf with partial pivoting) and
reused by every step through lu_solve.  The complex right-hand side is solved as
two real right-hand sides (the matrices are real).

Fisher-KPP (Eq. (17)): A(s) = gamma u (1 - u) with u = backward(s), formed at the
collocation nodes and forward-transformed; the storage truncation is the
two-thirds mask of Sec. 3.3 when the grid uses that chop policy.
Its linear regime is pinned by Eq. (18). Its nonlinear evolution is pinned in one
reduction: a uniform state follows the logistic closed form to second order in dt.
Other nonlinear FKPP evolutions are "parity unpinned" (oracle only).
"""

import numpy as np
import scipy.linalg as sla

from .operators import linear_operator
from .transform import backward, forward, serial


def fkpp_nonlinear(g, gamma):
    def A(spec):
        u = backward(g, spec)
        return forward(g, gamma * u * (1.0 - u))
    return A


class Stepper:
    def __init__(self, g, nu, dt, nu_h=0.0, p=8, nonlinear=None, post=None):
        """post: optional map applied to the state after every completed step (the
        modal filter of Sec. 3.3 is applied between steps)."""
        self.g, self.dt = g, float(dt)
        self.nonlinear = nonlinear
        self.post = post
        self.L = {}
        self.lu_half = {}
        self.lu_full = {}
        with serial():
            for m in range(g.M):
                for kabs in range(g.Kz):
                    kappa = 2.0 * np.pi * kabs / g.lz
                    L = linear_operator(m, kappa, g.nc, g.ell, nu, nu_h, p)
                    I = np.eye(L.shape[0])
                    self.L[(m, kabs)] = L
                    self.lu_half[(m, kabs)] = sla.lu_factor(I - 0.5 * self.dt * L)
                    self.lu_full[(m, kabs)] = sla.lu_factor(I - self.dt * L)

    def _kabs(self, kidx):
        return abs(int(self.g.kz[kidx]))

    def A(self, s):
        if self.nonlinear is None:
            return [np.zeros_like(b) for b in s]
        return self.nonlinear(s)

    def _solve(self, lus, rhs):
        with serial():
            return self._solve_blocks(lus, rhs)

    def _solve_blocks(self, lus, rhs):
        # a state may hold several fields: block j belongs to order m = j mod M
        out = []
        for j, blk in enumerate(rhs):
            m = j % self.g.M
            res = np.empty_like(blk)
            for kidx in range(self.g.K):
                lu = lus[(m, self._kabs(kidx))]
                b = np.stack([blk[kidx].real, blk[kidx].imag], axis=1)
                x = sla.lu_solve(lu, b)
                res[kidx] = x[:, 0] + 1j * x[:, 1]
            out.append(res)
        return out

    def apply_L(self, s):
        with serial():
            return self._apply_L_blocks(s)

    def _apply_L_blocks(self, s):
        out = []
        for j, blk in enumerate(s):
            m = j % self.g.M
            res = np.empty_like(blk)
            for kidx in range(self.g.K):
                res[kidx] = self.L[(m, self._kabs(kidx))] @ blk[kidx]
            out.append(res)
        return out

    def febe(self, s, half, A=None):
        """One FE-BE step of size dt/2 (half=True) or dt (half=False)."""
        h = 0.5 * self.dt if half else self.dt
        if A is None:
            A = self.A(s)
        rhs = [s[m] + h * A[m] for m in range(len(s))]
        return self._solve(self.lu_half if half else self.lu_full, rhs)

    def abcn(self, s, A, A_prev):
        Ls = self.apply_L(s)
        rhs = [s[m] + 0.5 * self.dt * Ls[m] + 0.5 * self.dt * (3.0 * A[m] - A_prev[m])
               for m in range(len(s))]
        return self._solve(self.lu_half, rhs)

    def start(self, s0):
        """Richardson start-up; returns (s1, A0)."""
        A0 = self.A(s0)
        y = self.febe(s0, True, A0)
        z = self.febe(y, True)
        v = self.febe(s0, False, A0)
        s1 = [2.0 * z[m] - v[m] for m in range(len(s0))]
        if self.post is not None:
            s1 = self.post(s1)
        return s1, A0

    def run_abcn(self, s0, nsteps, callback=None):
        """nsteps of AB-CN (the first by the Richardson start).  Returns (s, A_prev)."""
        if nsteps <= 0:
            return s0, None
        s, A_prev = self.start(s0)
        if callback:
            callback(1, s)
        for j in range(1, nsteps):
            A = self.A(s)
            s = self.abcn(s, A, A_prev)
            if self.post is not None:
                s = self.post(s)
            A_prev = A
            if callback:
                callback(j + 1, s)
        return s, A_prev

    def run_abcn_from(self, s, A_prev, nsteps):
        """Continue AB-CN from (s^j, A^{j-1}); returns (s^{j+nsteps}, A^{j+nsteps-1})."""
        for _ in range(nsteps):
            A = self.A(s)
            s = self.abcn(s, A, A_prev)
            if self.post is not None:
                s = self.post(s)
            A_prev = A
        return s, A_prev

    def run_febe(self, s0, nsteps):
        s = s0
        for _ in range(nsteps):
            s = self.febe(s, False)
        return s
