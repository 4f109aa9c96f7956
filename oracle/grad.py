"""Gradient oracle (test infrastructure only): the render written again in
PyTorch FP64 on the CPU, differentiated by autograd.

It follows the same steps as conegs_oracle.c, in the paper's order, but is an
independent implementation: whitening (Sec. 3), t* and q (Eq. 2), half-edge
vectors (Eq. 6), footprint covariance (Eq. 8), floor (Eq. 10), the marginal
rule in its literal 3x3 form with an eigen-decomposition (Eq. 12), the
closed-form response (Eq. 9) and thresholded front-to-back compositing
(Eq. 4).  Rays (d, delta_x, delta_y) come from the C oracle's inverse mapping
and the per-ray depth order from the FP32 depth key; neither is
differentiated.  The loss is L = sum_p w_rgb[p] . C[p] + w_T[p] T[p].

Pins (tests/test_grad_oracle.py): forward equal to the C oracle; gradient
equal to FP64 central finite differences of the C oracle.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import rays as _rays

_ALPHA_MIN, _ALPHA_MAX, _T_STOP, _T_NEAR = 1.0 / 255.0, 0.99, 1e-4, 0.01


def _sh_basis(v: torch.Tensor, deg: int) -> torch.Tensor:
    """Real SH (positive constants, l-major, m = -l..l) of unit vectors v [..., 3]."""
    x, y, z = v[..., 0], v[..., 1], v[..., 2]
    pi = math.pi
    out = [torch.full_like(x, 0.5 * math.sqrt(1 / pi))]
    if deg >= 1:
        c1 = math.sqrt(3 / (4 * pi))
        out += [c1 * y, c1 * z, c1 * x]
    if deg >= 2:
        a, b, c = 0.5 * math.sqrt(15 / pi), 0.25 * math.sqrt(5 / pi), 0.25 * math.sqrt(15 / pi)
        out += [a * x * y, a * y * z, b * (3 * z * z - 1), a * x * z, c * (x * x - y * y)]
    if deg >= 3:
        a = 0.25 * math.sqrt(35 / (2 * pi))
        b = 0.5 * math.sqrt(105 / pi)
        c = 0.25 * math.sqrt(21 / (2 * pi))
        d = 0.25 * math.sqrt(7 / pi)
        e = 0.25 * math.sqrt(105 / pi)
        out += [a * y * (3 * x * x - y * y), b * x * y * z, c * y * (5 * z * z - 1), d * z * (5 * z * z - 3),
                c * x * (5 * z * z - 1), e * z * (x * x - y * y), a * x * (x * x - 3 * y * y)]
    return torch.stack(out, -1)


def _rotation(q: torch.Tensor) -> torch.Tensor:
    q = q / q.norm(dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def _fp32_key(means: np.ndarray, o: np.ndarray) -> np.ndarray:
    v = means.astype(np.float32) - o.astype(np.float32)
    return np.sqrt((v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2]).astype(np.float64)


def _isotropic_differentials(cam, d: np.ndarray, dx: np.ndarray, dy: np.ndarray, footprint: str):
    """Isotropic footprint variants: the half-edge differentials become a b1, a b2,
    (b1, b2) orthonormal across d (built here from d x (a coordinate axis), a
    different basis from the C oracle's: the footprint does not depend on it);
    a^2 = (|dx_perp|^2 + |dy_perp|^2)/2 ('iso') or a = |<d, z_cam>|/(2 f_x) ('zf')."""
    if footprint == "own":
        return dx, dy
    if footprint == "iso":
        px = dx - (d * dx).sum(1, keepdims=True) * d
        py = dy - (d * dy).sum(1, keepdims=True) * d
        a = np.sqrt(0.5 * ((px * px).sum(1) + (py * py).sum(1)))
    else:
        zc = cam.cam_to_world[:, 2].astype(np.float64)
        a = np.abs(d @ zc) / (2.0 * float(cam.fx))
    axis = np.eye(3)[np.argmax(np.abs(d), 1)]          # the axis most aligned with d
    b1 = np.cross(d, np.roll(axis, 1, axis=1))
    b1 /= np.linalg.norm(b1, axis=1, keepdims=True)
    b2 = np.cross(d, b1)
    b2 /= np.linalg.norm(b2, axis=1, keepdims=True)
    return a[:, None] * b1, a[:, None] * b2


def render_torch(cam, params: dict, deg: int, rho2: torch.Tensor, pix: np.ndarray, filter_on: bool = True,
                 additive: bool = False, footprint: str = "own"):
    """Differentiable FP64 render of pixels ``pix``.  params: means [n,3], log_scales
    [n,3], quats [n,4], logits [n], sh [n,K,3] (FP64 tensors).  Returns rgb [P,3], T [P]."""
    o = torch.as_tensor(cam.cam_to_world[:, 3].astype(np.float64))
    means, ls, q, logit, sh = (params[k] for k in ("means", "log_scales", "quats", "logits", "sh"))
    n = means.shape[0]
    R = _rotation(q)                                        # [n,3,3]
    s = torch.exp(ls)
    s_eff = torch.sqrt(s * s + rho2[:, None])               # Eq. 10
    sig = torch.sigmoid(logit)
    sig_eff = sig * torch.prod(s / s_eff, -1)
    W = R.transpose(-1, -2) / s_eff[:, :, None]             # W = S_eff^-1 R^T
    Winv = R * s_eff[:, None, :]
    v = means - o
    L = v.norm(dim=-1)
    u = v / L[:, None]
    col = torch.clamp((sh * _sh_basis(u, deg)[:, :, None]).sum(1) + 0.5, min=0.0)
    key = _fp32_key(means.detach().numpy(), o.numpy())
    order = np.lexsort((np.arange(n), key))               # depth order, ties by index

    xs = (pix % cam.width) + 0.5
    ys = (pix // cam.width) + 0.5
    d, dx, dy, valid = _rays(cam, xs, ys)
    # pixels outside the valid domain contribute nothing (masked below); give them a
    # harmless unit ray so that no NaN enters the batched linear algebra
    d[~valid] = (0.0, 0.0, 1.0)
    dx[~valid] = (1e-3, 0.0, 0.0)
    dy[~valid] = (0.0, 1e-3, 0.0)
    dx, dy = _isotropic_differentials(cam, d, dx, dy, footprint)
    d, dx, dy = (torch.as_tensor(a) for a in (d, dx, dy))
    W_o, Winv_o, sig_o, col_o, rho2_o = W[order], Winv[order], sig_eff[order], col[order], rho2[order]
    ou = torch.einsum("nab,nb->na", W_o, (o - means[order]))   # o_u = W (o - mu)
    du = torch.einsum("nab,pb->pna", W_o, d)                    # d_u = W d
    nn = (du * du).sum(-1)
    ts = -(ou[None] * du).sum(-1) / nn                          # Eq. 2
    Mp = torch.eye(3, dtype=torch.float64) - du[..., :, None] * du[..., None, :] / nn[..., None, None]
    qv = torch.einsum("pnab,nb->pna", Mp, ou)                   # q = M_perp o_u
    if filter_on:
        MW = torch.einsum("pnab,nbc->pnac", Mp, W_o)
        ex = ts[..., None] * torch.einsum("pnab,pb->pna", MW, dx)   # Eq. 6
        ey = ts[..., None] * torch.einsum("pnab,pb->pna", MW, dy)
        Sfp = (ex[..., :, None] * ex[..., None, :] + ey[..., :, None] * ey[..., None, :]) / 3.0   # Eq. 8
        if additive:
            Sr = Sfp
        else:                                                   # Eq. 12, literal 3x3 form
            F = torch.einsum("nab,pnbc,ndc->pnad", Winv_o, Sfp, Winv_o) - \
                rho2_o[None, :, None, None] * torch.eye(3, dtype=torch.float64)
            F = 0.5 * (F + F.transpose(-1, -2))
            lam, V = torch.linalg.eigh(F)
            Fp = torch.einsum("pnab,pnb,pncb->pnac", V, torch.clamp(lam, min=0.0), V)
            Sr = torch.einsum("nab,pnbc,ndc->pnad", W_o, Fp, W_o)
        A = torch.eye(3, dtype=torch.float64) + Sr
        Qf = (qv * torch.linalg.solve(A, qv[..., None])[..., 0]).sum(-1)
        T = sig_o[None] / torch.sqrt(torch.linalg.det(A)) * torch.exp(-0.5 * Qf)   # Eq. 9
    else:
        T = sig_o[None] * torch.exp(-0.5 * (qv * qv).sum(-1))
    # compositing (Eq. 4): skip t* <= 0.01 and alpha < 1/255, stop before T_acc (1 - a) < 1e-4
    alpha = torch.clamp(T, max=_ALPHA_MAX)
    ok = (ts > _T_NEAR) & (alpha >= _ALPHA_MIN) & torch.as_tensor(valid)[:, None]
    a_eff = torch.where(ok, alpha, torch.zeros_like(alpha))
    one = torch.ones_like(a_eff[:, :1])
    T_before = torch.cumprod(torch.cat([one, 1 - a_eff[:, :-1]], 1), 1)
    stop = ok & (T_before * (1 - a_eff) < _T_STOP)
    first_stop = torch.where(stop.any(1), stop.float().argmax(1), torch.full_like(stop[:, 0], stop.shape[1],
                                                                                 dtype=torch.long))
    keep = ok & (torch.arange(stop.shape[1])[None, :] < first_stop[:, None])
    w = torch.where(keep, a_eff * T_before, torch.zeros_like(a_eff))
    rgb = torch.einsum("pn,nc->pc", w, col_o)
    a_keep = torch.where(keep, a_eff, torch.zeros_like(a_eff))
    Tfin = torch.prod(1 - a_keep, 1)
    return rgb, Tfin


def loss_and_grad(cam, scene, pix, w_rgb: np.ndarray, w_T: np.ndarray, filter_on: bool = True,
                  additive: bool = False, chunk: int = 256, footprint: str = "own"):
    """L = sum w_rgb . rgb + w_T . T over ``pix``; returns (L, grads dict of numpy FP64)."""
    params = {
        "means": torch.tensor(scene.means.astype(np.float64), requires_grad=True),
        "log_scales": torch.tensor(scene.log_scales.astype(np.float64), requires_grad=True),
        "quats": torch.tensor(scene.quats.astype(np.float64), requires_grad=True),
        "logits": torch.tensor(np.asarray(scene.opacity_logits, np.float64), requires_grad=True),
        "sh": torch.tensor(scene.sh.astype(np.float64), requires_grad=True),
    }
    rho2 = torch.as_tensor(scene.rho2.astype(np.float64))
    pix = np.asarray(pix)
    total = 0.0
    for s0 in range(0, pix.size, chunk):
        sl = slice(s0, s0 + chunk)
        rgb, T = render_torch(cam, params, scene.sh_degree, rho2, pix[sl], filter_on, additive, footprint)
        l = (rgb * torch.as_tensor(w_rgb[sl])).sum() + (T * torch.as_tensor(w_T[sl])).sum()
        l.backward()
        total += float(l.detach())
    return total, {k: p.grad.numpy().copy() for k, p in params.items()}
