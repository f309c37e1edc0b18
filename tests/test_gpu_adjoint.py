"""GPU adjoint (sscf_gradients) against the oracle's analytic gradients.

Both sides contract the same converged MOs: the oracle takes P = 2 C_o C_o^T
and dq from the GPU state, so the comparison isolates the adjoint kernels
(W = 1/2 P H P via F_oo and Z = C_o F_oo, the Slater-Koster derivative
blocks, the gamma forces, the parameter partials). The oracle's gradients
themselves are pinned against finite differences in test_oracle_adjoint.
"""
import numpy as np
import pytest

from gpu_common import P, context, water
from oracle import adjoint, model

pytestmark = pytest.mark.gpu


def _state(ctx, s):
    C = ctx.get_C()
    Co = C[:, :ctx.n_occ]
    Pm = 2.0 * Co @ Co.T
    q, dq, Q = ctx.get_charges()
    return Pm, dq


@pytest.mark.parametrize("n,prec,tol", [(32, 0, 1e-9), (8, 0, 1e-9), (32, 1, 2e-5)])
def test_gradients_match_oracle(n, prec, tol):
    s = water(n, seed=2, sigma=0.1)
    ctx = context(s, precision=prec)
    out = ctx.run(allow_not_converged=True)
    g, gp = ctx.gradients()
    Pm, dq = _state(ctx, s)
    # the GPU's charges must be those of its MOs
    H0, S = model.build_h0_s(s, P)
    _, atom_of_ao, _ = model.ao_layout(s.species)
    q = model.mulliken(Pm, S, atom_of_ao, s.n_atoms)
    assert np.abs(q - model.reference_population(s, P) - dq).max() < (1e-5 if prec else 1e-9)
    rg, rgp = adjoint.gradients(s, P, Pm, dq)
    assert np.abs(g - rg).max() <= tol * np.abs(rg).max()
    assert np.abs(gp - rgp).max() <= tol * np.abs(rgp).max()
    # net force vanishes (translation invariance of the energy)
    assert np.abs(g.sum(axis=0)).max() < 1e-6 * np.abs(g).max() + (1e-4 if prec else 1e-8)


def test_autograd_function_backward():
    import torch

    from gpu_common import library
    library()
    from paper_1402_2880_gb300.autograd import scc_energy
    s = water(8, seed=3, sigma=0.1)
    xyz = torch.tensor(s.xyz, dtype=torch.float64, requires_grad=True)
    V0 = torch.tensor(P["V0"], dtype=torch.float64, requires_grad=True)
    S0 = torch.tensor(P["S0"], dtype=torch.float64, requires_grad=True)
    E = scc_energy(s, xyz, V0, S0, P)
    (2.0 * E).backward()
    ctx = context(s)
    ctx.run(allow_not_converged=True)
    g, gp = ctx.gradients()
    assert np.allclose(xyz.grad.numpy(), 2.0 * g, rtol=0, atol=1e-9 * np.abs(g).max())
    assert np.allclose(V0.grad.numpy(), 2.0 * gp[:4], rtol=1e-9, atol=0)
    assert np.allclose(S0.grad.numpy(), 2.0 * gp[4:], rtol=1e-9, atol=0)
    # finite differences through the function itself (FP64 path) on a smooth,
    # tightly converged energy: cut-off 1e-9, charges to 1e-10 e, energy to
    # 1e-12 Ha (an SCF error of 1e-12 Ha is 5e-9 Ha/bohr at h = 1e-4 bohr);
    # no atom pair of the displaced atom within 2h of the 10-bohr hard cut-off
    from paper_1402_2880_gb300 import Context
    from synth import default_params
    pt = default_params(eps_mo=1e-9, dq_tol=1e-10, e_tol=1e-12)
    x0 = xyz.detach()
    h = 1e-4
    d = np.sqrt(((s.xyz[:, None, :] - s.xyz[None, :, :]) ** 2).sum(-1))
    c = Context.from_system(s, pt)
    assert c.run()["converged"]
    g_t, _ = c.gradients()
    c.close()
    gmax = np.abs(g_t).max()
    for k in np.argsort(-np.abs(g_t).ravel())[:3]:
        a, ax = divmod(int(k), 3)
        assert np.abs(d[a] - 10.0).min() > 2 * h
        xp = x0.clone()
        xm = x0.clone()
        xp[a, ax] += h
        xm[a, ax] -= h
        fd = (scc_energy(s, xp, V0.detach(), S0.detach(), pt) - scc_energy(s, xm, V0.detach(), S0.detach(), pt)) / (2 * h)
        assert abs(float(fd) - g_t[a, ax]) < 1e-5 * gmax
