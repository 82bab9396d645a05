"""Two-output network (oracle, float64 torch).

Site energy, Eq. (U_i) of Sec. II.A:
    U_i = sum_mu w1E_mu tanh(sum_nu W0_{mu nu} D_nu - b0_mu) - b1E
and the charge node of Sec. II.B (the second output of the same hidden layer):
    q_i = sum_mu w1q_mu tanh(...) - b1q
Weights are those of the central atom's species (NEP4).  Biases are
subtracted, as printed in Eq. (U_i).
"""
from __future__ import annotations

import numpy as np
import torch


def site_energy_and_charge(d: torch.Tensor, types: np.ndarray, model):
    t = torch.as_tensor(types, dtype=torch.long)
    pre = torch.einsum("imn,in->im", model.w0[t], d) - model.b0[t]
    h = torch.tanh(pre)
    u = (model.w1e[t] * h).sum(1) - model.b1e[t]
    q = (model.w1q[t] * h).sum(1) - model.b1q[t]
    return u, q
