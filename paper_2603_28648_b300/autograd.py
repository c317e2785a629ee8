"""Energy of the two-site wavefunction as a torch.autograd.Function.

E(psi, h, V) = <psi| H_eff(h, V) |psi> / <psi|psi> at the context's centre.
Every quantity comes from one library call, qcdmrg_energy_grad: the energy
(FP64 H_eff psi), dE/dpsi = 2 (H_eff psi - E psi) / <psi|psi>, dE/dh_pq =
gamma_pq (the spin-summed one-particle density matrix) and 2 dE/dV_pqrs =
Gamma_pqrs (the spin-summed 2-RDM averaged over the 8 permutations of
(pq|rs), the gradient for an 8-fold symmetric V) -- the quantities CASSCF
orbital gradients are built from. This module only moves arrays and applies
the chain rule (scaling by the incoming gradient).
"""

import torch


class DMRGEnergy(torch.autograd.Function):
    """apply(psi, h, V, context).

    psi: CUDA float64 tensor of the context's psi size; h, V: the integrals the
    context's environment was built from (tensors; only their gradient slots
    are used). Forward stores psi as the context's wavefunction (so that the
    density matrices belong to the same state); gradients w.r.t. h need the
    context's centre at (L-2, L-1).
    """

    @staticmethod
    def forward(fctx, psi, h, V, context):
        context.set_psi(psi.detach().cpu().numpy())
        L = h.shape[0]
        want_h, want_V = fctx.needs_input_grad[1], fctx.needs_input_grad[2]
        E, dpsi, g1, g2 = context.energy_grad(L, dpsi=True, gamma1=want_h, gamma2=want_V)
        fctx.dpsi = torch.as_tensor(dpsi, dtype=torch.float64, device=psi.device)
        fctx.g1 = None if g1 is None else torch.as_tensor(g1, dtype=torch.float64)
        fctx.g2 = None if g2 is None else torch.as_tensor(g2, dtype=torch.float64)
        return torch.tensor(E, dtype=torch.float64, device=psi.device)

    @staticmethod
    def backward(fctx, gE):
        dpsi = dh = dV = None
        if fctx.needs_input_grad[0]:
            dpsi = fctx.dpsi * gE
        g = gE.detach().cpu()
        if fctx.needs_input_grad[1]:
            dh = fctx.g1 * g
        if fctx.needs_input_grad[2]:
            dV = fctx.g2 * (0.5 * g)   # the library returns Gamma = 2 dE/dV
        return dpsi, dh, dV, None
