"""Geometry optimisation and molecular dynamics on the adjoint forces.

The paper's stated use of the sparse SCF is energies and, beyond them, forces
along trajectories (Introduction; Section "Summary and future work"). Every
energy and force here comes from libsscf: the SCF (sscf_run, or
sscf_run_from_current after a restart) and the adjoint (sscf_gradients). This
module only moves the atoms: between geometries it carries the converged MOs
over (sscf_get_C_tiles / sscf_set_C_tiles) as the start of the next SCF, the
MO groups staying those of the first geometry, so that every later geometry
runs the user stage alone from MOs that are already nearly converged.

Units: bohr, hartree, electron masses, atomic time units (1 a.u. = 0.0242 fs).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from ._lib import SSCF_FP64, Context

AMU = 1822.888486            # electron masses per dalton
MASS = (15.999 * AMU, 1.008 * AMU)   # O, H


def masses(species) -> np.ndarray:
    return np.where(np.asarray(species) == 0, MASS[0], MASS[1])


@dataclasses.dataclass
class Point:
    energy: float
    forces: np.ndarray      # (n_atoms, 3), -dE/dxyz
    converged: bool
    restarted: bool


class Surface:
    """Energies and forces of one system at successive geometries."""

    def __init__(self, system, params: dict, precision: int = SSCF_FP64, stream: int | None = None,
                 restart: bool = True):
        self.system, self.params = system, params
        self.precision, self.stream, self.restart = precision, stream, restart
        self._ck = None

    def __call__(self, xyz: np.ndarray) -> Point:
        s = self.system
        ctx = Context(s.species, np.asarray(xyz, dtype=np.float64), s.group_of_mol, self.params,
                      precision=self.precision, stream=self.stream,
                      cluster_of_mol=getattr(s, "cluster_of_mol", None))
        try:
            restarted = self.restart and self._ck is not None
            if restarted:
                ctx.set_C_tiles(*self._ck)
                out = ctx.run_from_current(allow_not_converged=True)
            else:
                out = ctx.run(allow_not_converged=True)
            g, _ = ctx.gradients()
            if self.restart:
                self._ck = ctx.get_C_tiles()
        finally:
            ctx.close()
        return Point(energy=out["energy"], forces=-g, converged=out["converged"], restarted=restarted)


def velocity_verlet(surface: Surface, xyz0: np.ndarray, v0: np.ndarray, dt: float, n_steps: int):
    """NVE trajectory: positions, velocities, potential and kinetic energy per step."""
    m = masses(surface.system.species)[:, None]
    x = np.array(xyz0, dtype=np.float64).reshape(-1, 3)
    v = np.array(v0, dtype=np.float64).reshape(-1, 3)
    pt = surface(x)
    out = {"x": [x.copy()], "v": [v.copy()], "epot": [pt.energy], "ekin": [0.5 * float((m * v * v).sum())],
           "converged": [pt.converged]}
    a = pt.forces / m
    for _ in range(n_steps):
        x = x + dt * v + 0.5 * dt * dt * a
        pt = surface(x)
        a_new = pt.forces / m
        v = v + 0.5 * dt * (a + a_new)
        a = a_new
        out["x"].append(x.copy())
        out["v"].append(v.copy())
        out["epot"].append(pt.energy)
        out["ekin"].append(0.5 * float((m * v * v).sum()))
        out["converged"].append(pt.converged)
    return {k: np.array(val) for k, val in out.items()}


def steepest_descent(surface: Surface, xyz0: np.ndarray, step: float, n_steps: int, max_move: float = 0.1):
    """Geometry optimisation: x <- x + step * F (each atom's move capped at
    max_move bohr); the step is halved and retried whenever the energy rises."""
    x = np.array(xyz0, dtype=np.float64).reshape(-1, 3)
    pt = surface(x)
    energies, fmax = [pt.energy], [float(np.abs(pt.forces).max())]
    for _ in range(n_steps):
        while True:
            d = step * pt.forces
            norm = np.linalg.norm(d, axis=1, keepdims=True)
            d = np.where(norm > max_move, d * (max_move / np.maximum(norm, 1e-300)), d)
            trial = surface(x + d)
            if trial.energy <= pt.energy or step < 1e-6:
                break
            step *= 0.5
        x, pt = x + d, trial
        energies.append(pt.energy)
        fmax.append(float(np.abs(pt.forces).max()))
    return x, np.array(energies), np.array(fmax)
