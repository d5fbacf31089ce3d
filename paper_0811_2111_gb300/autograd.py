"""d<O>/dbeta of Monte Carlo averages through torch.autograd.

``XYChain.apply(beta, L, seed, therm, meas)`` runs one chain per entry of the
1-d tensor ``beta`` (a batch of L x L lattices, no exchange): ``therm``
thermalisation sweeps, then ``meas`` measured sweeps whose per-sweep records
stay in device memory.  It returns the averages <e> and <Upsilon> per beta.
Its backward launches the library's FP64 series kernel on those device
records and returns sum_O grad_O * d<O>/dbeta with
    d<e>/dbeta = -cov(e_s, E_s),
    d<Upsilon>/dbeta = -cov(Upsilon_s, E_s) - J^2 <Ix^2 + Iy^2> / (2N),
so the specific heat c_v = -beta^2 d<e>/dbeta comes out of backward.
"""
import torch

from .lattice import Batch


class XYChain(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta, L, seed, therm, meas, sweeps_per_round=100, sincos="accurate",
                J=1.0, lattice_id0=0):
        b = beta.detach().to(torch.float64).cpu()
        n = b.numel()
        if therm % sweeps_per_round or meas % sweeps_per_round:
            raise ValueError("therm and meas must be multiples of sweeps_per_round")
        dev = torch.device("cuda", torch.cuda.current_device())
        batch = Batch([int(L)] * n, b.tolist(), seed, J=J, sincos=sincos,
                      lattice_id0=lattice_id0, sweeps_per_round=sweeps_per_round, device=dev)
        batch.reserve((therm + meas) // sweeps_per_round)
        batch.run((therm + meas) // sweeps_per_round)
        stats = batch.series_stats(therm, meas)
        ctx.batch = batch                      # the device-resident series for backward
        ctx.window = (therm, meas)
        ctx.beta_device = beta.device
        e = stats[:, 0].clone()
        u = stats[:, 1].clone()
        return e.to(beta.device), u.to(beta.device)

    @staticmethod
    def backward(ctx, grad_e, grad_u):
        first, count = ctx.window
        stats = ctx.batch.series_stats(first, count)     # the backward kernel
        dev = stats.device
        g = torch.zeros(stats.shape[0], dtype=torch.float64, device=dev)
        if grad_e is not None:
            g = g + grad_e.to(dev, torch.float64) * stats[:, 3]
        if grad_u is not None:
            g = g + grad_u.to(dev, torch.float64) * stats[:, 4]
        return g.to(ctx.beta_device), None, None, None, None, None, None, None, None


def chain_averages(beta, L, seed, therm, meas, sweeps_per_round=100, sincos="accurate", J=1.0,
                   lattice_id0=0):
    """(<e>, <Upsilon>) per beta with gradients attached (see XYChain)."""
    return XYChain.apply(beta, L, seed, therm, meas, sweeps_per_round, sincos, J, lattice_id0)
