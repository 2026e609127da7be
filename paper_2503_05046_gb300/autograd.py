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
P2G); nothing is traced or taped by torch. Particle states and their
adjoints move between torch and the library in device memory
(MPM_MEM_DEVICE).
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
        # the state goes to and comes from the context's device memory
        # directly (no host round trip)
        dev = sim.device
        x = x0.detach().to(device=dev, dtype=torch.float32).reshape(n, 3).contiguous()
        v = v0.detach().to(device=dev, dtype=torch.float32).reshape(n, 3).contiguous()
        Cm = torch.zeros((n, 3, 3), dtype=torch.float32, device=dev)
        F = torch.eye(3, dtype=torch.float32, device=dev).expand(n, 3, 3).contiguous()
        sim.set_particles(x, v, Cm, F)
        sim.tape_begin()
        for _ in range(int(n_steps)):
            sim.step(solver=solver)
        sim.tape_end()
        xf = torch.empty((n, 3), dtype=torch.float32, device=dev)
        vf = torch.empty((n, 3), dtype=torch.float32, device=dev)
        sim.read_particles(x=xf, v=vf)
        ctx.sim = sim
        ctx.eps_r = eps_r
        ctx.dev = dev
        ctx.like = [(a.device, a.dtype) for a in (x0, v0, E, nu, mu, body_v)]
        return xf.to(x0.device), vf.to(x0.device)

    @staticmethod
    def backward(ctx, gx, gv):
        sim = ctx.sim

        def on_dev(t):
            return None if t is None else t.detach().to(device=ctx.dev, dtype=torch.float32).contiguous()

        g = sim.backward(x_bar=on_dev(gx), v_bar=on_dev(gv), eps_r=ctx.eps_r)
        out = []
        for k, (dev, dt) in zip(("x", "v", "E", "nu", "mu", "body_v"), ctx.like):
            a = g[k]
            out.append(a.to(device=dev, dtype=dt) if torch.is_tensor(a)
                       else torch.as_tensor(np.asarray(a), dtype=dt, device=dev))
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
