"""Rigid-water trajectories through the library: the minimal integrator of row f3.

Every step runs in the library's kernels; this module only orders the calls (an MD step is
one integrator call under the forces, paper Sec. 1.1):

  ap_md_kick_drift (half kick, drift, SHAKE) -> [neighbour blocks, every `rebuild_every`
  steps] -> permanent_field -> initial guess -> induced_dipoles_pcg ->
  polarization_energy_forces -> ap_lj_forces (added) -> ap_md_kick (half kick, RATTLE,
  optional Berendsen scale).

The list is rebuilt on a fixed interval, chosen well inside half the list buffer: thermal
atoms of water at 300 K move < 0.03 A/fs, so 10 steps of 2 fs stay below 0.6 A against
buffer / 2 = 1 A (the library's default configuration). Water only: atoms 3k, 3k+1, 3k+2
are the O, H, H of molecule k.
"""
from __future__ import annotations

import numpy as np

from . import binding

MASS_O, MASS_H = 15.999, 1.008
LJ_O = (0.1521, 3.1507)          # eps (kcal/mol), sigma (A) between oxygens
KB = 0.0019872041                # kcal/mol/K


class RigidWaterMD:
    """Holds the integrator's device arrays for a water-only Context."""

    def __init__(self, ctx: "binding.Context", sysobj, dt: float = 2.0, rebuild_every: int = 10,
                 tol: float = 1e-5, max_iter: int = 200, lj=LJ_O):
        t = ctx.torch
        self.ctx, self.t, self.dt = ctx, t, float(dt)
        self.rebuild_every, self.tol, self.max_iter = int(rebuild_every), float(tol), int(max_iter)
        n = sysobj.n
        if n % 3:
            raise ValueError("water-only systems: n must be a multiple of 3")
        dev = ctx.device
        self.n_mol = n // 3
        self.mol = t.arange(n, dtype=t.int32, device=dev).reshape(-1, 3).contiguous()
        d = np.asarray(sysobj.xyz[:3], np.float64)
        self.lengths = (float(np.linalg.norm(d[1] - d[0])), float(np.linalg.norm(d[2] - d[0])),
                        float(np.linalg.norm(d[2] - d[1])))
        m = np.full(n, MASS_H)
        m[0::3] = MASS_O
        self.mass = t.tensor(m, device=dev)
        p = np.zeros((n, 2))
        p[:, 1] = 1.0
        p[0::3] = lj
        self.lj = t.tensor(p, device=dev)
        self.vel = t.zeros((n, 3), dtype=t.float64, device=dev)
        self.forces = t.zeros((n, 3), dtype=t.float64, device=dev)
        self.e_lj = t.zeros(1, dtype=t.float64, device=dev)
        self.kinetic = t.zeros(1, dtype=t.float64, device=dev)
        self.status = t.zeros(1, dtype=t.int32, device=dev)
        self.zero = t.zeros((n, 3), dtype=t.float64, device=dev)
        self.dof = 6 * self.n_mol - 3
        self.step_count = 0
        self.iterations = []

    def start(self, v):
        """Initial velocities and the forces at the context's current positions (lists built)."""
        self.set_velocities(v)
        return self.compute_forces(rebuild=True)

    def set_velocities(self, v):
        """Initial velocities (A/fs), projected onto the constraints by a kick with zero force."""
        self.vel.copy_(self.t.as_tensor(np.asarray(v, np.float64)))
        binding.ap_md_kick(self.mol, self.lengths, self.mass, self.dt, self.zero, self.ctx.xyz, self.vel,
                           self.kinetic, self.status)

    def compute_forces(self, guess=None, rebuild=False):
        """Total forces at the context's current positions into self.forces; returns the
        solve's info."""
        c = self.ctx
        if rebuild:
            c.build()
        c.permanent_field(out=False)
        info = c.solve(tol=self.tol, max_iter=self.max_iter, guess=guess)
        binding.polarization_energy_forces(c.ctx, c.mu, c.energy, self.forces)
        binding.ap_lj_forces(c.ctx, self.lj, self.e_lj, self.forces)
        return info

    def temperature(self):
        return 2.0 * float(self.kinetic.item()) / (self.dof * KB)

    def step(self, target_temperature=None, tau_fs=100.0, guess=None):
        """One velocity-Verlet step (NVE, or Berendsen towards target_temperature with
        coupling time tau_fs, its factor from the previous step's kinetic energy)."""
        c = self.ctx
        binding.ap_md_kick_drift(self.mol, self.lengths, self.mass, self.dt, self.forces, c.xyz, self.vel,
                                 self.status)
        self.step_count += 1
        info = self.compute_forces(guess=guess, rebuild=self.step_count % self.rebuild_every == 0)
        self.iterations.append(info.iterations)
        scale = 1.0
        if target_temperature is not None:
            T = self.temperature()
            if T > 0:
                scale = float(np.sqrt(max(0.5, min(2.0, 1.0 + self.dt / tau_fs * (target_temperature / T - 1.0)))))
        binding.ap_md_kick(self.mol, self.lengths, self.mass, self.dt, self.forces, c.xyz, self.vel, self.kinetic,
                           self.status, scale=scale)
        return info

    def potential(self):
        return float(self.ctx.energy.item()) + float(self.e_lj.item())

    def total_energy(self):
        return self.potential() + float(self.kinetic.item())

    def check(self):
        """Raises if SHAKE or RATTLE failed to converge in any step so far."""
        st = int(self.status.item())
        if st:
            raise binding.ApError(f"constraint iterations did not converge (status {st})")
