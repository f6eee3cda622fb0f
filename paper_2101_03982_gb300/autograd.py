"""torch.autograd.Function around the step and its adjoint.

``SimFunction.apply(rho0, u0, sim, nsteps, every)`` initialises ``sim`` with
the equilibrium of (rho0, u0), runs ``nsteps`` isothermal steps and returns
the density and velocity fields (rho_T, u_T) of the final state.  Its backward
pass gives dJ/drho0 and dJ/du0 for any scalar J(rho_T, u_T) computed with
torch, with every vector-Jacobian product evaluated by the library's kernels:

* forward: the compact state is saved every ``every`` steps (checkpoints);
* backward: the adjoint seed from (dJ/drho_T, dJ/du_T) at the final state
  (olb_moments_vjp); then, from the last checkpoint back to the first, the
  segment is recomputed onto the device tape (olb_tape_record) and swept back
  (olb_tape_adjoint); finally the gradient through the initial equilibrium
  (olb_equilibrium_vjp).

Memory: nsteps/every compact checkpoints plus `every` tape slots (four values
per node each: the moments of one step's pulled populations).
The recomputation costs one extra forward pass in total.
"""
import torch


class SimFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, u0, sim, nsteps, every):
        if every < 1 or nsteps < 1:
            raise ValueError("nsteps and every must be positive")
        rho0 = rho0.detach().contiguous()
        u0 = u0.detach().contiguous()
        sim.init_fields(rho0, u0)
        nb = sim.state_bytes()
        ckpts = []
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            buf = torch.empty(nb, dtype=torch.uint8, device=rho0.device)
            sim.get_state(buf)
            ckpts.append((buf, k))
            sim.step(k)
            done += k
        final = torch.empty(nb, dtype=torch.uint8, device=rho0.device)
        sim.get_state(final)
        rho = torch.empty_like(rho0)
        u = torch.empty_like(u0)
        sim.moments(rho, u)
        ctx.sim, ctx.ckpts, ctx.final, ctx.every = sim, ckpts, final, every
        ctx.save_for_backward(rho0, u0)
        return rho, u

    @staticmethod
    def backward(ctx, g_rho, g_u):
        sim = ctx.sim
        rho0, u0 = ctx.saved_tensors
        dev = rho0.device
        sim.set_state(ctx.final)
        lam = torch.empty((sim.Q,) + tuple(rho0.shape), dtype=getattr(torch, sim.adjoint_dtype), device=dev)
        gr = g_rho.contiguous() if g_rho is not None else None
        gu = g_u.contiguous() if g_u is not None else None
        sim.moments_vjp(gr, gu, lam)
        sim.tape_reserve(ctx.every)
        for buf, k in reversed(ctx.ckpts):
            sim.set_state(buf)
            sim.tape_record(k)
            sim.tape_adjoint(lam, k)
        grad_rho0 = torch.empty_like(rho0)
        grad_u0 = torch.empty_like(u0)
        sim.equilibrium_vjp(rho0, u0, lam, grad_rho0, grad_u0)
        return grad_rho0, grad_u0, None, None, None
