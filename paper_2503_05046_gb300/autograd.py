"""torch.autograd binding of a differentiable rollout.

`rollout(sim, n_steps, x0, v0, E, nu, mu, solver, body_v=..., bodies=...)` runs
`n_steps` rigid time steps of the context held by `sim` (native.Sim) from the
particle positions x0 and velocities v0 (C = 0, F = I), with Young's modulus E
and Poisson ratio nu per particle group, friction coefficient mu and linear
velocity body_v per rigid body, and returns the final positions and
velocities. The bodies start from `bodies` (default: the context's current
ones, which a previous rollout has moved) and keep the dynamics set on `sim`
(Sim.set_dynamics). Its backward pass is the library's
hand-written adjoint (mpm_backward: checkpoints per step, the adjoints of
G2P, the contact solve by implicit differentiation, the grid update and
P2G); nothing is traced or taped by torch.
"""
import numpy as np
import torch

from . import native


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim, n_steps, solver, eps_r, bodies, x0, v0, E, nu, mu, body_v):
        n = sim.n
        for gi, g in enumerate(sim.scene["groups"]):
            m = dict(g["material"], E=float(E[gi]), nu=float(nu[gi]))
            native.mpm_set_material(sim.ctx, gi, m)
        bodies = [dict(b) for b in (sim.bodies() if bodies is None else bodies)]
        for b, mb in zip(bodies, mu.detach().cpu().numpy()):
            b["mu"] = float(mb)
        for b, vb in zip(bodies, body_v.detach().cpu().numpy().reshape(-1, 3)):
            b["v"] = np.asarray(vb, np.float64)
        dynamics = dict(sim.dynamics)
        sim.set_bodies(bodies)  # clears the dynamics: set them again
        for i, d in sorted(dynamics.items()):
            sim.set_dynamics(i, d)
        x = x0.detach().to(torch.float32).cpu().numpy().reshape(n, 3)
        v = v0.detach().to(torch.float32).cpu().numpy().reshape(n, 3)
        Cm = np.zeros((n, 3, 3), np.float32)
        F = np.tile(np.eye(3, dtype=np.float32), (n, 1, 1))
        sim.set_particles(x, v, Cm, F)
        sim.tape_begin()
        for _ in range(int(n_steps)):
            sim.step(solver=solver)
        sim.tape_end()
        out = sim.get_particles()
        ctx.sim = sim
        ctx.eps_r = eps_r
        ctx.like = [(a.device, a.dtype) for a in (x0, v0, E, nu, mu, body_v)]
        xf = torch.from_numpy(out["x"]).to(x0.device)
        vf = torch.from_numpy(out["v"]).to(x0.device)
        return xf, vf

    @staticmethod
    def backward(ctx, gx, gv):
        sim = ctx.sim
        g = sim.backward(x_bar=None if gx is None else gx.detach().cpu().numpy(),
                         v_bar=None if gv is None else gv.detach().cpu().numpy(), eps_r=ctx.eps_r)
        grads = [np.asarray(g[k]) for k in ("x", "v", "E", "nu", "mu", "body_v")]
        out = [torch.as_tensor(a, dtype=dt, device=dev) for a, (dev, dt) in zip(grads, ctx.like)]
        return (None, None, None, None, None, *out)


def rollout(sim, n_steps, x0, v0, E, nu, mu, solver=None, eps_r=1e-6, body_v=None, bodies=None):
    """Differentiable rollout (see the module docstring). x0, v0: [n, 3]
    tensors; E, nu: [n_groups] tensors; mu: [n_bodies] tensor; body_v:
    optional [n_bodies, 3] tensor of the bodies' linear velocities (default:
    those of the starting bodies); bodies: optional list of body dicts to
    start from (default: the context's current bodies). Returns the final
    (x, v)."""
    start = sim.bodies() if bodies is None else bodies
    if body_v is None:
        body_v = torch.tensor(np.array([b["v"] for b in start], np.float64).reshape(-1, 3))
    return _Rollout.apply(sim, n_steps, solver, eps_r, start, x0, v0, E, nu, mu, body_v)
