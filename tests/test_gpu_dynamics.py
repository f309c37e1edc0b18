"""Geometry optimisation and molecular dynamics on the GPU adjoint forces.

A 4-molecule cluster whose atom pairs all stay far (> 0.7 bohr) from the
10-bohr hard cut-off, so that the energy surface is smooth along the paths
below. FP64, cut-off 1e-8, converged to 1e-9 e and 1e-11 Ha.

* A restart from the converged MOs of a nearby geometry (sscf_set_C_tiles +
  sscf_run_from_current) reaches the same state as a run from the guess.
* Velocity-Verlet dynamics has a total-energy error of second order in the
  time step (forces consistent with the energy), every step after the first
  restarting from the last MOs.
* Steepest descent lowers the energy at every accepted step.
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


def test_velocity_verlet_error_is_second_order():
    """Over the same 40 a.u. from the same start, halving the time step cuts
    the largest total-energy deviation about fourfold (velocity Verlet is
    second order only when the forces are the energy's exact gradient), and
    it stays a small fraction of the energy exchanged with the kinetic term.
    (The model's rigid-water start is far from a minimum: forces of ~0.1
    Ha/bohr, so the steps are short.)"""
    library()
    from paper_1402_2880_gb300 import dynamics
    s = _system()
    m = dynamics.masses(s.species)[:, None]
    kT = 300.0 * 3.166811563e-6                      # 300 K in hartree
    v0 = np.random.default_rng(2).standard_normal(s.xyz.shape) * np.sqrt(kT / m)
    v0 -= (m * v0).sum(axis=0) / m.sum()            # no drift of the centre of mass
    drift, exchange = [], []
    for dt, n in ((4.0, 10), (2.0, 20)):
        tr = dynamics.velocity_verlet(dynamics.Surface(s, PT), s.xyz, v0, dt=dt, n_steps=n)
        assert tr["converged"].all()
        etot = tr["epot"] + tr["ekin"]
        drift.append(float(np.abs(etot - etot[0]).max()))
        exchange.append(float(tr["ekin"].max() - tr["ekin"].min()))
        d = np.sqrt(((tr["x"][:, :, None, :] - tr["x"][:, None, :, :]) ** 2).sum(-1))
        assert np.abs(d - 10.0).min() > 0.3             # stayed clear of the cut-off
    assert exchange[1] > 1e-3
    assert drift[1] < 0.4 * drift[0]
    assert drift[1] < 0.05 * exchange[1]


def test_steepest_descent_lowers_the_energy():
    library()
    from paper_1402_2880_gb300 import dynamics
    s = _system()
    x, e, fmax = dynamics.steepest_descent(dynamics.Surface(s, PT), s.xyz, step=0.5, n_steps=8)
    assert np.all(np.diff(e) <= 1e-12)
    assert e[-1] < e[0] - 1e-3
