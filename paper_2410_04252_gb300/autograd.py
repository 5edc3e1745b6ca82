"""torch.autograd.Function over sv_grad: E(theta) = <psi0|U^dagger H U|psi0>
(Eqs. vqe, vqe_qsu, vqe_evc) with its adjoint gradient computed by the
library in the same call.  backward() returns grad_output * dE/dtheta.
"""
from __future__ import annotations

import numpy as np
import torch

from . import sv as _sv


class VQEEnergy(torch.autograd.Function):
    """forward(params, sim, circ, ham, schedule, init_index) -> energy (0-d).

    params: 1-D tensor of circuit parameters (any device, float dtype).
    sim: sv.StateVector; circ: workloads.Circuit; ham: workloads.Hamiltonian
    or a (paulis, coeffs) pair of arrays; schedule: sv.LAZY or sv.EAGER.
    The state is reset to |init_index> before the forward pass.
    """

    @staticmethod
    def forward(ctx, params, sim, circ, ham, schedule, init_index):
        p = params.detach().to("cpu", torch.float64).numpy()
        sim.reset(init_index)
        if isinstance(ham, tuple):
            e, g = sim.grad(circ, p, paulis=ham[0], coeffs=ham[1], schedule=schedule)
        else:
            e, g = sim.grad(circ, p, ham, schedule=schedule)
        ctx.save_for_backward(torch.from_numpy(np.ascontiguousarray(g)).to(params.device, params.dtype))
        return params.new_tensor(e)

    @staticmethod
    def backward(ctx, grad_output):
        (g,) = ctx.saved_tensors
        return grad_output * g, None, None, None, None, None


def vqe_energy(params, sim, circ, ham, schedule: int = _sv.LAZY, init_index: int = 0):
    return VQEEnergy.apply(params, sim, circ, ham, schedule, init_index)
