"""Free-boundary driver (Sec. 4.3 Algorithm, Steps 0-3): per time step, the
level-set step of every species, then the embedded-boundary operator on the
new domain, then one ETD2 step per species.

Readings for what the Algorithm leaves open:
  * u after an ETD step holds the new values at computational points and 0
    at every other node (ghost points are not unknowns; u = 0 on the
    complement of the domain, Eq. free).
  * F_{n-1} is kept on the grid from the previous step's computational
    points; where a point was not computational at the previous step
    F_{n-1} := F_n there (locally ETD1, as for the first step).
  * Two species: F of species s is evaluated at its computational points
    with its own extended field and the other species' field masked to the
    other's computational points.
  * Reinitialisation after the level-set advection of steps k with
    (k + 1) % reinit_every == 0 (k counted from 0), and once at t = 0 when
    requested.
"""
import numpy as np

from . import etd, levelset
from .eb import EBOperator


class Species:
    def __init__(self, phi, u, beta, mu):
        self.phi = phi
        self.u = u
        self.beta = beta
        self.mu = mu
        self.F_prev = None
        self.prev_comp = None
        self.comp = None


class FreeBoundary:
    def __init__(self, grid, species, reaction, rparams, tol, m_max, reinit_every=5, reinit_at_start=False):
        self.grid = grid
        self.sp = species
        self.reaction = reaction
        self.rparams = rparams
        self.tol = tol
        self.m_max = m_max
        self.reinit_every = reinit_every
        self.k = 0
        self.traces = []
        h = grid.h
        for s in self.sp:
            s.phi = levelset.clamp(np.asarray(s.phi, dtype=np.float64), h)
            if reinit_at_start:
                s.phi = levelset.reinit(s.phi, h)
            inside = s.phi < 0
            s.u = np.where(inside, s.u, 0.0)
            s.comp = EBOperator(grid, s.phi, s.beta).comp

    def step(self, dt, forced_traces=None):
        """One free-boundary step.  forced_traces: None, or per species a
        Krylov decision trace to replay (None for a species: decide)."""
        g = self.grid
        do_reinit = self.reinit_every > 0 and (self.k + 1) % self.reinit_every == 0
        exts = []
        for s in self.sp:
            phi_new, u_ext, _ = levelset.levelset_advance(s.phi, s.u, s.comp, g, dt, s.mu, do_reinit)
            s.phi = phi_new
            exts.append(u_ext)
        ops = [EBOperator(g, s.phi, s.beta) for s in self.sp]
        fields = []
        for i, s in enumerate(self.sp):
            fields.append(exts[i])
        F_grid = self._reaction_on_grid(fields, ops)
        new_u = []
        traces = []
        for i, (s, op) in enumerate(zip(self.sp, ops)):
            u_n = op.from_grid(exts[i])
            F_n = op.from_grid(F_grid[i])
            if s.F_prev is None:
                F_p = F_n
            else:
                was = s.prev_comp.ravel()[op.index]
                F_p = np.where(was, s.F_prev.ravel()[op.index], F_n)
            ft = None if forced_traces is None else forced_traces[i]
            u_new, tr = etd.etd2_step(op, u_n, F_n, F_p, dt, tol=self.tol, m_max=self.m_max, forced_trace=ft)
            traces.append(tr)
            new_u.append(op.to_grid(u_new))
            s.F_prev = op.to_grid(F_n)
            s.prev_comp = op.comp
            s.comp = op.comp
        for s, u in zip(self.sp, new_u):
            s.u = u
        self.traces.append(traces)
        self.k += 1
        return ops

    def _reaction_on_grid(self, fields, ops):
        if len(fields) == 1:
            return etd.reaction(self.reaction, self.rparams, fields)
        # two species: own extended field, other species masked to its own points
        u_ext, v_ext = fields
        u_phys = np.where(ops[0].comp, u_ext, 0.0)
        v_phys = np.where(ops[1].comp, v_ext, 0.0)
        Fu = etd.reaction(self.reaction, self.rparams, [u_ext, v_phys])[0]
        Fv = etd.reaction(self.reaction, self.rparams, [u_phys, v_ext])[1]
        return [Fu, Fv]
