"""Geometry optimisation and molecular dynamics on the GPU adjoint forces.

A 4-molecule cluster whose atom pairs all stay far (> 0.7 bohr) from the
10-bohr hard cut-off, so that the energy surface is smooth along the paths
below. FP64, cut-off 1e-8, converged to 1e-9 e and 1e-11 Ha.

* A restart from the converged MOs of a nearby geometry (sscf_set_C_tiles +
  sscf_run_from_current) reaches the same state as a run from the guess.
* Velocity-Verlet dynamics conserves the total energy to a small fraction of
  the kinetic energy it exchanges with the potential (forces consistent with
  the energy), every step after the first restarting from the last MOs.
* Steepest descent lowers the energy at every accepted step and the largest
  force with it.
"""
import numpy as np
import pytest

from gpu_common import library
from synth import default_params, lattice_water

pytestmark = pytest.mark.gpu

PT = default_params(eps_mo=1e-8, dq_tol=1e-9, e_tol=1e-11)


def _system():
    return lattice_water(4, seed=37, displace_sigma_A=0.1)


def test_restart_reaches_the_state_of_a_fresh_run():
    library()
    from paper_1402_2880_gb300 import dynamics
    s = _system()
    rng = np.random.default_rng(1)
    x1 = s.xyz + 0.02 * rng.standard_normal(s.xyz.shape)
    warm = dynamics.Surface(s, PT)
    warm(s.xyz)
    p_restart = warm(x1)
    p_fresh = dynamics.Surface(s, PT, restart=False)(x1)
    assert p_restart.restarted and not p_fresh.restarted
    assert p_restart.converged and p_fresh.converged
    assert abs(p_restart.energy - p_fresh.energy) < 1e-9
    assert np.abs(p_restart.forces - p_fresh.forces).max() < 1e-6 * np.abs(p_fresh.forces).max()


def test_velocity_verlet_conserves_energy():
    library()
    from paper_1402_2880_gb300 import dynamics
    s = _system()
    m = dynamics.masses(s.species)[:, None]
    kT = 300.0 * 3.166811563e-6                      # 300 K in hartree
    v0 = np.random.default_rng(2).standard_normal(s.xyz.shape) * np.sqrt(kT / m)
    v0 -= (m * v0).sum(axis=0) / m.sum()            # no drift of the centre of mass
    tr = dynamics.velocity_verlet(dynamics.Surface(s, PT), s.xyz, v0, dt=10.0, n_steps=30)
    assert tr["converged"].all()
    etot = tr["epot"] + tr["ekin"]
    exchange = tr["ekin"].max() - tr["ekin"].min()
    drift = np.abs(etot - etot[0]).max()
    assert exchange > 1e-4
    assert drift < 0.02 * exchange
    d = np.sqrt(((tr["x"][:, :, None, :] - tr["x"][:, None, :, :]) ** 2).sum(-1))
    assert np.abs(d - 10.0).min() > 0.3                 # stayed clear of the cut-off


def test_steepest_descent_lowers_energy_and_forces():
    library()
    from paper_1402_2880_gb300 import dynamics
    s = _system()
    x, e, fmax = dynamics.steepest_descent(dynamics.Surface(s, PT), s.xyz, step=0.5, n_steps=8)
    assert np.all(np.diff(e) <= 1e-12)
    assert e[-1] < e[0] - 1e-4
    assert fmax[-1] < 0.5 * fmax[0]
