"""Relaxed (fractional) objective in float64 PyTorch on the CPU.

Test infrastructure only: ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library; gradients come from torch autograd of this plain formula.

The objective is Eq. 14's scenario-averaged discounted cash flow with the
extraction decision x_{b,t} relaxed from {0, 1} to [0, 1] (a block may be
spread over periods; row sums are not forced) and the mill-deviation penalty
smoothed so that it has a derivative everywhere:

    ore[b,s]  = (g[b,s] * price) * recovery > proc_cost      (FP64, strict;
                a step in g, so it carries no gradient)
    v[b,s]    = ore ? m_b ((g price) recovery - proc_cost) - m_b mining_cost
                    : -m_b mining_cost
    O[t,s]    = sum_b x[b,t] m_b ore[b,s]          ore tonnes sent to the mill
    V[t,s]    = sum_b x[b,t] v[b,s]                undiscounted block value
    P_t(O)    = a m_ref sp((Q_t - O) / m_ref) + e m_ref sp((O - Q_t) / m_ref)
    sp(z)     = log(1 + exp(beta z)) / beta        (softplus, beta = 10)
    NPV_s     = sum_t d_t (V[t,s] - P_t(O[t,s])),  d_t = (1 + r)^-t
    J         = mean_s NPV_s - lambda std_s NPV_s  (population std; its
                gradient is taken as 0 where all NPV_s are equal)

As beta grows, m_ref sp(z / m_ref) tends to max(0, z) (the gap is at most
m_ref log(2) / beta), so the relaxed objective of a 0/1 schedule tends to the
discrete one of the C oracle.  The matrix products are library primitives
(torch.matmul); everything else is written out as above.
"""

from __future__ import annotations

import math

import torch

BETA = 10.0
M_REF = 10_000.0


def softplus(z: torch.Tensor, beta: float = BETA) -> torch.Tensor:
    """log(1 + exp(beta z)) / beta, evaluated without overflow:
    max(beta z, 0) + log1p(exp(-|beta z|)), divided by beta."""
    bz = beta * z
    return (torch.clamp(bz, min=0.0) + torch.log1p(torch.exp(-torch.abs(bz)))) / beta


def ore_mask(g: torch.Tensor, price: float, recovery: float, proc_cost: float) -> torch.Tensor:
    """Ore flag per (b, s) from float64 grades, in the order (g * price) * recovery."""
    return ((g.detach().to(torch.float64) * price) * recovery) > proc_cost


def contractions(x: torch.Tensor, g: torch.Tensor, mass, p):
    """ore, v, O = x^T (m ore), V = x^T v (float64, autograd-able)."""
    x = x.to(torch.float64)
    g = g.to(torch.float64)
    m = torch.as_tensor(mass, dtype=torch.float64).reshape(-1, 1)
    ore = ore_mask(g, p.price, p.recovery, p.proc_cost)
    oref = ore.to(torch.float64)
    v = torch.where(ore, m * ((g * p.price) * p.recovery - p.proc_cost) - m * p.mining_cost,
                    -m * p.mining_cost + 0.0 * g)
    O = x.t() @ (m * oref)            # [T][S]
    V = x.t() @ v                     # [T][S]
    return ore, v, O, V


def objective_from(O: torch.Tensor, V: torch.Tensor, target, p, beta: float = BETA, m_ref: float = M_REF):
    """pen, NPV_s, mean, std and J from the per-period contractions O, V [T][S]."""
    T = O.shape[0]
    Q = torch.as_tensor(target, dtype=torch.float64).reshape(-1, 1)
    pen = p.shortfall_pen * m_ref * softplus((Q - O) / m_ref, beta) \
        + p.excess_pen * m_ref * softplus((O - Q) / m_ref, beta)
    d = torch.tensor([(1.0 + p.discount_rate) ** (-t) for t in range(T)], dtype=torch.float64).reshape(-1, 1)
    npv = (d * (V - pen)).sum(dim=0)  # [S]
    mean = npv.mean()
    var = ((npv - mean) ** 2).mean()
    # std is not differentiable where every NPV_s is equal (var = 0); its
    # gradient is taken as 0 there (S = 1 always)
    pos = var > 0
    std = torch.where(pos, torch.sqrt(torch.where(pos, var, torch.ones_like(var))), torch.zeros_like(var))
    J = mean - p.lam * std
    return dict(pen=pen, npv=npv, mean=mean, std=std, J=J, d=d.reshape(-1))


def relaxed_parts(x: torch.Tensor, g: torch.Tensor, mass, target, p, beta: float = BETA, m_ref: float = M_REF):
    """All intermediate quantities of the relaxed objective (float64, autograd-able).

    x [B][T], g [B][S] float64 tensors; mass [B], target [T] (tonnes); p is a
    Problem (or any object with the economics attributes)."""
    ore, v, O, V = contractions(x, g, mass, p)
    return dict(ore=ore, v=v, O=O, V=V, **objective_from(O, V, target, p, beta, m_ref))


def relaxed_objective(x, g, mass, target, p, beta: float = BETA, m_ref: float = M_REF) -> torch.Tensor:
    """J (a float64 scalar tensor)."""
    return relaxed_parts(x, g, mass, target, p, beta, m_ref)["J"]


def relaxed_grads(x_np, g_np, mass, target, p, beta: float = BETA, m_ref: float = M_REF):
    """J, dJ/dx [B][T] and dJ/dg [B][S] by float64 autograd, plus the parts."""
    x = torch.tensor(x_np, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(g_np, dtype=torch.float64, requires_grad=True)
    parts = relaxed_parts(x, g, mass, target, p, beta, m_ref)
    J = parts["J"]
    gx, gg = torch.autograd.grad(J, (x, g))
    return dict(J=float(J.detach()), gx=gx.numpy(), gg=gg.numpy(),
                **{k: (v.detach().numpy() if torch.is_tensor(v) else v) for k, v in parts.items() if k != "J"})


def central_difference_x(x, g, mass, target, p, b: int, t: int, h: float = 1e-3, beta: float = BETA,
                         m_ref: float = M_REF) -> float:
    """Central difference of J in x[b][t].  O and V are linear in x, so the
    perturbed contractions are O, V plus or minus h times block b's row in
    period t; J is then evaluated from them with objective_from."""
    with torch.no_grad():
        ore, v, O, V = contractions(torch.as_tensor(x), torch.as_tensor(g), mass, p)
        dO = float(mass[b]) * ore[b].to(torch.float64)
        out = []
        for sgn in (1.0, -1.0):
            O2, V2 = O.clone(), V.clone()
            O2[t] += sgn * h * dO
            V2[t] += sgn * h * v[b]
            out.append(float(objective_from(O2, V2, target, p, beta, m_ref)["J"]))
    return (out[0] - out[1]) / (2.0 * h)


def central_difference_g(x, g, mass, target, p, b: int, s: int, h: float = 1e-3, beta: float = BETA,
                         m_ref: float = M_REF) -> float:
    """Central difference of J in g[b][s] for a grade at least h away (in value
    terms) from the ore threshold: the ore flags do not change, O is fixed and
    V[:, s] moves by the change of v[b][s] times x[b][:]."""
    with torch.no_grad():
        x = torch.as_tensor(x, dtype=torch.float64)
        ore, v, O, V = contractions(x, torch.as_tensor(g), mass, p)
        out = []
        for sgn in (1.0, -1.0):
            gb = float(g[b][s]) + sgn * h
            vb = float(mass[b]) * ((gb * p.price) * p.recovery - p.proc_cost) - float(mass[b]) * p.mining_cost \
                if bool(ore[b, s]) else -float(mass[b]) * p.mining_cost
            V2 = V.clone()
            V2[:, s] += (vb - float(v[b, s])) * x[b]
            out.append(float(objective_from(O, V2, target, p, beta, m_ref)["J"]))
    return (out[0] - out[1]) / (2.0 * h)


def central_difference(fn, base: torch.Tensor, index, h: float = 1e-3) -> float:
    """(f(base + h e_i) - f(base - h e_i)) / (2 h) for one coordinate."""
    up = base.clone()
    dn = base.clone()
    up[index] += h
    dn[index] -= h
    return (float(fn(up)) - float(fn(dn))) / (2.0 * h)


def discount(T: int, r: float):
    return [math.pow(1.0 + r, -t) for t in range(T)]
