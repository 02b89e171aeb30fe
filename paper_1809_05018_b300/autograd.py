"""torch.autograd.Function around the vertex pseudo-log-likelihood and its
hand-written FP64 adjoint (pmrf_pll / pmrf_pll_grad).

    pll = PLL.apply(mu, sigma, beta, graph, labels)   # [S] per-slice PLL
    pll.sum().backward()                              # grads of mu [S,L], sigma [S,L], beta []
"""
from __future__ import annotations

import torch


class PLL(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, sigma, beta, graph, labels):
        mu_c = mu.detach().contiguous()
        sg_c = sigma.detach().contiguous()
        L = mu_c.shape[-1]
        b = float(beta.detach().item()) if isinstance(beta, torch.Tensor) else float(beta)
        out = graph.pll(L, labels, mu_c, sg_c, b)
        ctx.graph = graph
        ctx.L = L
        ctx.beta = b
        ctx.beta_is_tensor = isinstance(beta, torch.Tensor)
        ctx.save_for_backward(mu_c, sg_c, labels)
        return out

    @staticmethod
    def backward(ctx, gout):
        mu_c, sg_c, labels = ctx.saved_tensors
        gmu, gsg, gb = ctx.graph.pll_grad(ctx.L, labels, mu_c, sg_c, ctx.beta, gout.contiguous().to(torch.float64))
        gbeta = gb.reshape(()) if ctx.beta_is_tensor else None
        return gmu, gsg, gbeta, None, None


def fit_beta(graph, labels, mu, sigma, beta0=0.2, steps=30, lr=1.0):
    """Gradient ascent on the pseudo-log-likelihood in beta (mu, sigma held
    fixed): beta <- max(0, beta + lr * dPLL/dbeta / V).  Returns the beta
    trajectory (a list of floats, starting with beta0)."""
    beta = torch.tensor(float(beta0), dtype=torch.float64, device=mu.device, requires_grad=True)
    traj = [float(beta0)]
    V = max(1, graph.V)
    for _ in range(steps):
        if beta.grad is not None:
            beta.grad = None
        pll = PLL.apply(mu, sigma, beta, graph, labels).sum()
        pll.backward()
        with torch.no_grad():
            beta += lr * beta.grad / V
            beta.clamp_(min=0.0)
        traj.append(float(beta.detach()))
    return traj
