"""Algorithm-1 sweeps assembled around a library FFT, kept as a comparison of
the fused passes: the polarization (bfcs_polarize, Eq. 5.7) and the Green step
(bfcs_green_apply, Eq. 5.9) are the library's own kernels, the 3D real
transforms (Eqs. 4.3-4.4) are torch.fft's (cuFFT on the GPU), and the strain is
kept in real space between sweeps.  Not a product path: bench.py times it next
to the fused sweep and the tests check it against the oracle.
"""
from __future__ import annotations

import torch


class LibFftSweeps:
    """State of one solve (strain, d_prev, residual numerator) on a plan of any
    precision except the mixed ladder's."""

    def __init__(self, plan, phase, phases, c0, b, E=(0.0,) * 6):
        nx, ny, nz = plan.dims
        self.plan, self.phase, self.phases, self.c0, self.E = plan, phase, phases, c0, E
        self.dims = (nz, ny, nx)
        cdt = torch.complex64 if plan.dtype == torch.float32 else torch.complex128
        self.b_hat = torch.fft.rfftn(b, dim=(-3, -2, -1))
        self.spec = torch.zeros((6, nz, ny, nx // 2 + 1), dtype=cdt, device=b.device)
        self.d_prev = torch.zeros((3, nz, ny, nx // 2 + 1), dtype=cdt, device=b.device)
        self.num = torch.zeros(1, dtype=torch.float64, device=b.device)
        self.tau = torch.empty((6, nz, ny, nx), dtype=plan.dtype, device=b.device)
        self.eps = torch.empty_like(self.tau)
        # eps^0 = eps^{b(0)} + E: the Green step of a zero polarization
        plan.green_apply(c0, self.b_hat, self.spec, E)
        torch.fft.irfftn(self.spec, s=self.dims, dim=(-3, -2, -1), out=self.eps)

    def sweep(self):
        """tau^s = L1 eps^s, tau_hat^s, eps_hat^{s+1} (with the residual numerator of
        eps^s in self.num), eps^{s+1}."""
        self.plan.polarize(self.phase, self.phases, self.c0, self.eps, tau=self.tau)
        torch.fft.rfftn(self.tau, dim=(-3, -2, -1), out=self.spec)
        self.plan.green_apply(self.c0, self.b_hat, self.spec, self.E, self.d_prev, self.num)
        torch.fft.irfftn(self.spec, s=self.dims, dim=(-3, -2, -1), out=self.eps)
        return self.eps
