"""torch.autograd.Function over the adjoint kernel: the final energy (or fidelity)
as a differentiable function of the Fourier schedule amplitudes a_m.

The schedule is s(t) = t/T + sum_{m=1..M} a_m sin(m pi t / T), sampled at step
midpoints t_k = (k - 1/2) dt (dt = T / N).  Forward runs the Trotterised evolution
from |+>^n and the reverse sweep in one qs_adjoint_grad call; backward applies the
chain rule dV/da_m = sum_k dV/ds_k sin(m pi t_k / T).
"""
from __future__ import annotations

import math

import numpy as np
import torch


def fourier_schedule(a: np.ndarray, T: float, n_steps: int):
    """(s_k, ds_k/da_m) for the midpoints of n_steps equal steps over [0, T]."""
    dt = T / n_steps
    t = (np.arange(1, n_steps + 1) - 0.5) * dt
    m = np.arange(1, len(a) + 1)
    jac = np.sin(np.outer(m, t) * math.pi / T)          # (M, N)
    return t / T + np.asarray(a, dtype=np.float64) @ jac, jac


class ScheduleValue(torch.autograd.Function):
    """value = V(psi_N(a)); V = final energy <H1> or fidelity |<phi|psi_N>|^2."""

    @staticmethod
    def forward(ctx, a, sim, couplings, T, n_steps, order=2, target="energy", ref_state=None):
        a_np = a.detach().to("cpu", torch.float64).numpy()
        s, jac = fourier_schedule(a_np, T, n_steps)
        sim.init_plus()
        val, g = sim.adjoint_grad(couplings, s, T / n_steps, order, target, ref_state)
        ctx.save_for_backward(torch.from_numpy(jac @ g[0]).to(a.dtype))
        return torch.tensor(val[0], dtype=a.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (dv_da,) = ctx.saved_tensors
        return grad_out * dv_da, None, None, None, None, None, None, None


def schedule_value(a, sim, couplings, T, n_steps, order=2, target="energy", ref_state=None):
    return ScheduleValue.apply(a, sim, couplings, T, n_steps, order, target, ref_state)
