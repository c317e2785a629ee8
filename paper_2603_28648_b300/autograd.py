"""Energy of the two-site wavefunction as a torch.autograd.Function.

E(psi, h, V) = <psi| H_eff(h, V) |psi> / <psi|psi> at the context's centre.
Backward: dE/dpsi = 2 (H_eff psi - E psi) / <psi|psi> (one H_eff psi in the
library), dE/dh_pq = gamma_pq, the spin-summed one-particle density matrix
of the state (qcdmrg_rdm1), and dE/dV_pqrs = 1/2 Gamma_pqrs, the spin-summed
2-RDM averaged over the 8 permutations of (pq|rs) (the gradient for an 8-fold
symmetric V) -- the quantities CASSCF orbital gradients are built from. Gamma
comes from qcdmrg_rdm2 (one environment build per permutation orbit) up to
PROBE_MAX_L orbitals and from the centre walk of qcdmrg_rdm2_sweep beyond.
"""

import torch

from . import FP64

PROBE_MAX_L = 10
_AXES = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
         (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]


class DMRGEnergy(torch.autograd.Function):
    """apply(psi, h, V, context, precision=FP64).

    psi: CUDA float64 tensor of the context's psi size; h, V: the integrals the
    context's environment was built from (tensors; only their gradient slots
    are used). Gradients w.r.t. h need the context's centre at (L-2, L-1) and
    its stored wavefunction equal to psi (context.set_psi).
    """

    @staticmethod
    def forward(fctx, psi, h, V, context, precision=FP64):
        sig = torch.empty_like(psi)
        stream = torch.cuda.current_stream()
        context.apply_heff_dev(psi.data_ptr(), sig.data_ptr(), stream.cuda_stream, precision)
        nn = torch.dot(psi, psi)
        E = torch.dot(psi, sig) / nn
        fctx.save_for_backward(psi, sig, E, nn)
        fctx.context = context
        fctx.L = h.shape[0]
        return E

    @staticmethod
    def backward(fctx, gE):
        psi, sig, E, nn = fctx.saved_tensors
        dpsi = dh = dV = None
        if fctx.needs_input_grad[0]:
            dpsi = 2.0 * (sig - E * psi) / nn * gE
        if fctx.needs_input_grad[1]:
            g = fctx.context.rdm1(fctx.L)
            dh = torch.as_tensor(g, dtype=torch.float64) * gE.detach().cpu()
        if fctx.needs_input_grad[2]:
            if fctx.L <= PROBE_MAX_L:
                G = fctx.context.rdm2(fctx.L)
            else:
                G1 = fctx.context.rdm2_sweep(fctx.L)
                G = sum(G1.transpose(a) for a in _AXES) / 8.0
            dV = 0.5 * torch.as_tensor(G, dtype=torch.float64) * gE.detach().cpu()
        return dpsi, dh, dV, None, None
