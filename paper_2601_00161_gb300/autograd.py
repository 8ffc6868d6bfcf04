"""Automatic differentiation of the ESP long-range energy (positions and cell).

``long_range_energy(plan, pos, cell, q)`` returns U = U_F + U_self + U_bg as a 0-d
float64 tensor (Sec. 3: Fourier part, self term of eq. (selfen), background of eq. (Corr)).
Its backward pass uses the library's kernels only:

* d U / d r_i = -F_i, the forces of the same step (the gather kernel, Appendix C eq. (AD));
* d U / d h at fixed Cartesian positions = -W h^{-T} + sum_i F_i (h^{-1} r_i)^T, with
  W = W_F + U_bg I the virial of the scaling kernel (eqs. (PFfinal), (Corr)); this is the
  cell derivative behind the pressure tensor of eq. (instheta) once r = h s is
  differentiated too (``esp_cell_gradient``).

``cell`` is the 3 x 3 matrix h whose COLUMNS are the cell vectors, as in the C ABI.  The
charges are constants here (no gradient).  The forward pass synchronises the stream to
return the energy and raises if the step skipped atoms with non-finite input.
"""

from __future__ import annotations

import numpy as np
import torch

from . import (ESP_ACCUM_LEN, ESP_ERR_NONFINITE, ESPError, esp_cell_gradient,
               esp_result_from_accum, esp_step)


class LongRangeEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, cell, q, plan):
        h = cell.detach().to(torch.float64).cpu().numpy().reshape(3, 3)
        if not np.array_equal(plan.cell, h):
            plan.set_cell(h)  # NPT: the plan follows the cell it is given
        pos_c = pos.detach().to(device="cuda", dtype=plan.io_dtype).contiguous()
        q_c = q.detach().to(device="cuda", dtype=plan.io_dtype).contiguous()
        if pos_c.shape != (plan.n, 3) or q_c.shape != (plan.n,):
            raise ValueError("pos must be [n, 3] and q [n] for this plan")
        F = torch.empty_like(pos_c)
        acc = torch.zeros(ESP_ACCUM_LEN, dtype=torch.float64, device="cuda")
        esp_step(plan.handle, pos_c, q_c, F, acc)
        acc_h = acc.cpu().numpy()
        if acc_h[9] > 0:
            raise ESPError(ESP_ERR_NONFINITE, f"{int(acc_h[9])} atoms with non-finite input")
        r = esp_result_from_accum(plan.handle, acc_h)
        ctx.save_for_backward(pos_c, F, acc)
        ctx.plan, ctx.h = plan, h
        ctx.pos_dtype, ctx.cell_dtype = pos.dtype, cell.dtype
        U = r.energy_recip + r.energy_self + r.energy_bg
        return torch.tensor(U, dtype=torch.float64, device=pos.device)

    @staticmethod
    def backward(ctx, gU):
        pos_c, F, acc = ctx.saved_tensors
        plan = ctx.plan
        g_pos = g_cell = None
        if ctx.needs_input_grad[0]:
            g_pos = (F.to(torch.float64) * (-gU)).to(ctx.pos_dtype)
        if ctx.needs_input_grad[1]:
            if not np.array_equal(plan.cell, ctx.h):
                plan.set_cell(ctx.h)
            G = torch.empty(9, dtype=torch.float64, device="cuda")
            esp_cell_gradient(plan.handle, pos_c, F, acc, G)
            g_cell = (G.view(3, 3) * gU).to(ctx.cell_dtype)
        return g_pos, g_cell, None, None


def long_range_energy(plan, pos, cell, q):
    """U(pos, cell) = U_F + U_self + U_bg of the plan's parameters; differentiable in pos
    (N x 3, Cartesian) and cell (3 x 3, columns = cell vectors)."""
    return LongRangeEnergy.apply(pos, cell, q, plan)
