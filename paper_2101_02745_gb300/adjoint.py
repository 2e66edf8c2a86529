"""Gradients of the particle step: a torch.autograd.Function around the
library's hand-written discrete adjoint.

`Evolve.apply(n_nu, n_nubar, f_nu, f_nubar, sim)` initialises the particles of
`sim.box` from per-cell densities (nz,) and fluxes (nz, 3) (Eq. 8, with the
Eq. 9 perturbations of sim.alpha, sim.seed), takes sim.nsteps RK4 steps at
the fixed step sim.dt (Sec. 2.3) and returns the final moments (72, nz) as
emu_moments lays them out (Eq. 5: n, f_x, f_y, f_z of the neutrinos, then of
the antineutrinos, 9 packed reals each).  Any torch loss of those moments
can then be differentiated with respect to the four species inputs.  For a
batch of boxes the inputs and the moments cover all cells of the batch
(boxes concatenated), sim.dt, sim.alpha and sim.seed are per box, and one
backward pass gives the gradients of every box.

Forward keeps a checkpoint of the evolving state (z, rho, rhobar) every
sim.every steps.  Backward seeds the adjoint from dL/d(moments), then walks
the segments last to first: it restores a segment's checkpoint, recomputes
the segment's step-start states forward, and runs one adjoint step per step
backward (emu_adjoint_step, which recomputes the step's forward stages).
With sim.record the recomputation writes each step's record (stage states,
weights, potentials; emu_adjoint_record_step) and the adjoint steps read it
(emu_adjoint_step_recorded), so the forward stages run once instead of
twice; the library replays both calls as CUDA graphs per record slot.  The
default records whenever a segment's records fit in half the free device
memory.  The accumulated
dL/dN, dL/dNbar go through Eq. 8 to the species inputs
(emu_weight_gradient).  Every arithmetic step runs in the CUDA library; this
module only marshals buffers.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from .emu import Box


@dataclass
class Simulation:
    """Settings of one differentiable run on a box or a batch of boxes (then
    dt, alpha and seed are sequences with one entry per box)."""
    box: Box
    nsteps: int
    dt: object
    every: int = 20
    alpha: object = 1e-6
    seed: object = 0
    dirs: np.ndarray | None = None
    record: bool | None = None

    @property
    def batched(self) -> bool:
        return self.box.nbox > 1

    def step_dt(self) -> float:
        """The dt argument of the step calls: the step size, or 0 for a batch
        (each box's own size, set on the box)."""
        return 0.0 if self.batched else float(self.dt)

    def use_record(self) -> bool:
        """Whether backward keeps per-step records (see the module notes)."""
        if self.record is not None:
            return bool(self.record)
        import torch
        free, _ = torch.cuda.mem_get_info(self.box.device)
        return min(self.every, max(self.nsteps, 1)) * self.box.record_stride() <= free // 2


def _host(t: torch.Tensor, shape) -> np.ndarray:
    return np.ascontiguousarray(t.detach().to("cpu", torch.float64).numpy().reshape(shape))


class Evolve(torch.autograd.Function):
    """Species inputs -> final moments, with the library's adjoint as backward."""

    @staticmethod
    def forward(ctx, n_nu, n_nubar, f_nu, f_nubar, sim: Simulation):
        from . import emu as E
        box = sim.box
        dts = np.atleast_1d(np.asarray(sim.dt, float))
        if len(dts) != box.nbox or not np.all(dts > 0) or sim.nsteps < 0 or sim.every < 1:
            raise ValueError("need one dt > 0 per box, nsteps >= 0, every >= 1")
        nz = box.nz
        host = (_host(n_nu, (nz,)), _host(n_nubar, (nz,)), _host(f_nu, (nz, 3)), _host(f_nubar, (nz, 3)))
        if sim.batched:
            alpha = np.broadcast_to(np.asarray(sim.alpha, float), (box.nbox,)).copy()
            seed = np.broadcast_to(np.asarray(sim.seed, np.uint64), (box.nbox,)).copy()
            dirs = None if sim.dirs is None else np.ascontiguousarray(sim.dirs, float).reshape(-1)
            E.emu_batch_init_particles(box.box, host[0], host[1], host[2].reshape(-1), host[3].reshape(-1), dirs,
                                       alpha, seed)
            box.batch_set_dt(dts)
        else:
            box.init(*host, sim.dirs, sim.alpha, sim.seed)
        checkpoints = []
        done = 0
        while done < sim.nsteps:
            checkpoints.append(box.save_state())
            k = min(sim.every, sim.nsteps - done)
            _steps(sim, k)
            done += k
        final = box.save_state()
        mom = box.moments()
        ctx.sim = sim
        ctx.checkpoints = checkpoints
        ctx.final = final
        ctx.dev = n_nu.device
        return mom.to(n_nu.device)

    @staticmethod
    def backward(ctx, dmom):
        sim: Simulation = ctx.sim
        box = sim.box
        lam, gN, gNbar = box.adjoint_buffers()
        box.load_state(ctx.final)
        box.adjoint_seed(dmom, lam, gN, gNbar)
        nseg = len(ctx.checkpoints)
        dt = sim.step_dt()
        rec = box.record_buffer(min(sim.every, sim.nsteps)) if nseg and sim.use_record() else None
        for seg in range(nseg - 1, -1, -1):
            start = seg * sim.every
            k = min(sim.every, sim.nsteps - start)
            box.load_state(ctx.checkpoints[seg])
            starts = [box.save_state()]
            for j in range(k - 1):
                if rec is None:
                    _steps(sim, 1)
                else:
                    box.adjoint_record_step(dt, rec, j)
                starts.append(box.save_state())
            if rec is not None:
                box.adjoint_record_step(dt, rec, k - 1)
            for j in range(k - 1, -1, -1):
                box.load_state(starts[j])
                if rec is None:
                    box.adjoint_step(dt, lam, gN, gNbar)
                else:
                    box.adjoint_step_recorded(dt, rec, j, lam, gN, gNbar)
        box.load_state(ctx.final)
        g = box.weight_gradient(gN, gNbar).to(ctx.dev)
        return g[0], g[1], g[2:5].T.contiguous(), g[5:8].T.contiguous(), None


def _steps(sim: Simulation, k: int):
    if sim.batched:
        sim.box.batch_step(k)
    else:
        sim.box.step(k, float(sim.dt))


def objectives(mom: torch.Tensor) -> torch.Tensor:
    """(<n_ee>, log <|n_emu|>) of moments laid out as emu_moments returns them:
    the final nu_e abundance and the growth measure of Eq. 10."""
    nee = mom[0]
    nem = torch.hypot(mom[3], mom[4])
    return torch.stack([nee.mean(), torch.log(nem.mean())])
