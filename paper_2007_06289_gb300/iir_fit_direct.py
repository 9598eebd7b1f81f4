"""Refining the recursive-filter coefficients against the direct FBP, in image space, by
gradient descent through the library's adjoint kernels.

The host fit (``iir_fit``) matches the filter's frequency response to the ideal ramp.  What
matters in the end is the reconstruction, so this module minimises instead
    loss(b, a) = mean over pixels and slices of (R_{b,a}(p) - D(p))^2,
R_{b,a} the fast reconstruction with coefficients (b, a) and D the direct FBP, over a set of
sinograms p.

Gradients.  R is linear in the filtered sinogram: R_{b,a}(p) = H L F_{b,a} p.  With the
image residual r = R - D, u = L^T H^T (2 r / n) (``fbp_fht_backproject_adjoint`` then
``fbp_resample_st_adjoint``) is the gradient of the loss with respect to the filtered
sinogram, and since F_{b,a} = sum_k b_k F_{e_k,a} is linear in b,
    d loss / d b_k = <u, F_{e_k,a} p>,
one filtering of p per coefficient (``fbp_filter_iir`` with numerator e_k).  The feedback
coefficients enter non-linearly; they are parameterised by reflection coefficients
k_i = 0.99999 tanh(x_i) (every trial filter stable) and their gradient is taken by central
differences of the loss.  The numerator keeps sum(b) = 0 (the gradient is projected).
Steps are Adam's.  Everything runs in the library's kernels; this module only orchestrates.

Variable projection (``fit_vp``).  For fixed feedback coefficients a the reconstruction is
linear in b, so the best numerator is a least-squares problem: with the basis numerators
d_k = e_k - e_{k+1} (k < Mb - 1, each summing to 0, so b = sum c_k d_k keeps sum(b) = 0)
and R_k the fast reconstructions with numerator d_k, c minimises ||sum_k c_k R_k - D||^2
(a least-squares problem with Mb-1 unknowns, solved by QR).  The feedback coefficients, reflection-parameterised,
are then searched by Nelder-Mead on that projected loss, from the default table's filter.
This is the fit the committed table uses: the Adam loop above stalls at its start for
N >= 512.

Running this file (on a GPU) fits orders 3 and 6 for N = 256 .. 2048 by variable
projection against the direct FBP of noisy ten-ellipse phantoms and writes them to
``iir_direct_coeffs.json`` (or the path given), read by ``direct_coefficients``.
"""
from __future__ import annotations

import numpy as np
import torch

try:
    from . import binding as fbp
    from .iir_fit import KMAX, poly_to_reflection, reflection_to_poly
except ImportError:                      # run as a script
    import os as _os
    import sys as _sys
    _sys.path.insert(0, _os.path.dirname(_os.path.dirname(_os.path.abspath(__file__))))
    from paper_2007_06289_gb300 import binding as fbp
    from paper_2007_06289_gb300.iir_fit import KMAX, poly_to_reflection, reflection_to_poly


class _Problem:
    def __init__(self, N, sinos, target):
        self.N = N
        self.sinos = sinos.contiguous()
        self.target = target.contiguous()
        self.S, self.K, self.M = sinos.shape
        self.img = torch.empty_like(target)

    def plan(self, b, a):
        return fbp.fbp_plan(self.N, self.K, self.M, self.S, (list(map(float, b)), list(map(float, a))))

    def loss(self, b, a, plan=None):
        plan = plan or self.plan(b, a)
        fbp.fbp_reconstruct(plan, self.sinos, self.img)
        r = self.img - self.target
        return float(torch.mean(r.double() ** 2)), r, plan

    def grad_b(self, b, a, r, plan):
        """Adjoint-based gradient of the loss with respect to b."""
        n = r.numel()
        lin = torch.empty(plan.lin_shape, device=r.device)
        u = torch.empty(plan.sino_shape, device=r.device)
        fbp.fbp_fht_backproject_adjoint(plan, (2.0 / n) * r, lin)
        fbp.fbp_resample_st_adjoint(plan, lin, u)
        g = np.zeros(len(b))
        fk = torch.empty_like(self.sinos)
        for k in range(len(b)):
            e = np.zeros(len(b))
            e[k] = 1.0
            fbp.fbp_filter_iir(self.plan(e, a), self.sinos, fk)
            g[k] = float(torch.sum(u.double() * fk.double()))
        return g


def loss_and_grad_b(N, sinos, target, b, a):
    """(loss, d loss / d b) at (b, a): the adjoint path, exposed for checking."""
    pr = _Problem(N, sinos, target)
    loss, r, plan = pr.loss(b, a)
    return loss, pr.grad_b(b, a, r, plan)


def fit_against_direct(N, sinos, target, b0, a0, steps: int = 40, lr_b: float = 2e-3,
                       lr_x: float = 2e-2, fd: float = 1e-3):
    """Adam on (b, x) from (b0, a0).  sinos [S][K][M], target [S][N][N]: float32 CUDA.
    Returns (b, a, losses); losses[0] is the starting loss."""
    pr = _Problem(N, sinos, target)
    b = np.array(b0, dtype=np.float64)
    x = np.arctanh(np.clip(poly_to_reflection(np.asarray(a0, np.float64)) / KMAX, -0.999999, 0.999999))
    params = np.concatenate([b, x])
    m1 = np.zeros_like(params)
    m2 = np.zeros_like(params)
    lr = np.concatenate([np.full(b.size, lr_b), np.full(x.size, lr_x)])
    losses = []
    best = None
    for it in range(steps + 1):
        b, x = params[:b.size], params[b.size:]
        a = reflection_to_poly(KMAX * np.tanh(x))
        loss, r, plan = pr.loss(b, a)
        losses.append(loss)
        if best is None or loss < best[0]:
            best = (loss, b.copy(), a.copy())
        if it == steps:
            break
        gb = pr.grad_b(b, a, r, plan)
        gb -= gb.mean()                             # stay on sum(b) = 0
        gx = np.zeros(x.size)
        for i in range(x.size):
            d = np.zeros(x.size)
            d[i] = fd
            lp = pr.loss(b, reflection_to_poly(KMAX * np.tanh(x + d)))[0]
            lm = pr.loss(b, reflection_to_poly(KMAX * np.tanh(x - d)))[0]
            gx[i] = (lp - lm) / (2 * fd)
        g = np.concatenate([gb, gx])
        m1 = 0.9 * m1 + 0.1 * g
        m2 = 0.999 * m2 + 0.001 * g * g
        step = lr * (m1 / (1 - 0.9 ** (it + 1))) / (np.sqrt(m2 / (1 - 0.999 ** (it + 1))) + 1e-12)
        params = params - step
        params[:b.size] -= params[:b.size].mean()
    return best[1], best[2], losses


def fit_vp(N, sinos, target, a0, order: int, iters: int = 300):
    """Variable-projection fit (module docstring).  Returns (b, a, loss, loss at a0)."""
    from scipy.optimize import minimize
    S, K, M = sinos.shape
    basis = []
    for k in range(order - 1):
        d = np.zeros(order)
        d[k], d[k + 1] = 1.0, -1.0
        basis.append(d)
    ws = None
    rec = torch.empty(len(basis), S, N, N, device=sinos.device)
    tgt = target.double().reshape(-1)

    def project(a):
        nonlocal ws
        if np.abs(np.roots(np.concatenate([[1.0], a]))).max() >= 0.99995:
            return None
        for k, d in enumerate(basis):
            try:
                plan = fbp.fbp_plan(N, K, M, S, (list(d), list(map(float, a))))
            except fbp.FbpError:
                return None
            if ws is None:
                ws = torch.empty(fbp.fbp_workspace_bytes(plan), dtype=torch.uint8, device=sinos.device)
            fbp.fbp_set_workspace(plan, ws)
            fbp.fbp_reconstruct(plan, sinos, rec[k])
        R = rec.double().reshape(len(basis), -1)
        # least squares by a QR of the tall matrix R^T (modified Gram-Schmidt, applied twice:
        # the basis reconstructions are nearly collinear for higher orders, and the normal
        # equations would square their condition number)
        nb = len(basis)
        Q = R.clone()
        U = torch.zeros(nb, nb, dtype=torch.float64, device=R.device)
        for j in range(nb):
            for _ in range(2):
                for i in range(j):
                    pr = torch.dot(Q[i], Q[j])
                    Q[j] -= pr * Q[i]
                    U[i, j] += pr
            nrm = torch.linalg.vector_norm(Q[j])
            Q[j] /= nrm
            U[j, j] = nrm
        c = torch.linalg.solve_triangular(U, (Q @ tgt)[:, None], upper=True)[:, 0]
        r = c @ R - tgt
        c = c.cpu().numpy()
        b = sum(ck * d for ck, d in zip(c, basis))
        return b, float(torch.mean(r * r))

    def loss(x):
        out = project(reflection_to_poly(KMAX * np.tanh(x)))
        return 1e9 if out is None else out[1]

    x0 = np.arctanh(np.clip(poly_to_reflection(np.asarray(a0, np.float64)) / KMAX, -0.999999, 0.999999))
    start = loss(x0)
    res = minimize(loss, x0, method="Nelder-Mead",
                   options=dict(maxiter=iters, maxfev=iters, xatol=1e-6, fatol=1e-12, adaptive=True))
    a = reflection_to_poly(KMAX * np.tanh(res.x))
    b, f = project(a)
    return b, a, f, start


FIT_SIZES = (256, 512, 1024, 2048)
FIT_ORDERS = (3, 6)
_TABLE = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.abspath(__file__)),
                                    "iir_direct_coeffs.json")


def direct_coefficients(N: int, order: int = 3):
    """(b, a) of the committed direct-FBP-fitted table (iir_direct_coeffs.json)."""
    import json
    with open(_TABLE) as fh:
        table = json.load(fh)
    for e in table["entries"]:
        if e["N"] == N and e["order"] == order:
            return np.array(e["b"]), np.array(e["a"])
    raise KeyError((N, order))


def fit_table(path: str = _TABLE, sizes=FIT_SIZES, orders=FIT_ORDERS, slices: int = 8,
              iters: int = 300, seed: int = 3000) -> None:
    """Fit every size and order by variable projection (training phantoms: seeds seed + N ..
    seed + N + slices - 1, noisy at I0 = 1e5) and write the table."""
    import json

    import phantoms
    from paper_2007_06289_gb300 import iir_fit as _fit
    fbp.load_library()
    entries = []
    for N in sizes:
        K, M = phantoms.geometry_for(N)
        sino = phantoms.phantom_stack_torch(N, slices, seed + N, "cuda", noise_i0=1e5)
        direct = torch.empty(slices, N, N, device="cuda")
        fbp.fbp_direct_reconstruct(fbp.fbp_plan(N, K, M, slices), sino, direct)
        for order in orders:
            b0, a0 = _fit.coefficients(N, order)
            b, a, loss, start = fit_vp(N, sino, direct, a0, order, iters=iters)
            table = float(_table_loss(N, sino, direct, b0, a0))
            source = "variable projection"
            if not loss < table:
                # the basis reconstructions of a high-order filter with poles clustered near
                # z = 1 have huge gains and lose the precision their combination needs: keep
                # the default table's filter where the fit does not improve on it
                b, a, loss, source = np.asarray(b0), np.asarray(a0), table, "default table"
            entries.append(dict(N=N, order=order, slices=slices, seed=seed + N,
                                loss_table=table, loss_start_projected=start, loss=loss,
                                source=source, b=list(map(float, b)), a=list(map(float, a))))
            print(f"N={N} order={order}: table {entries[-1]['loss_table']:.4g}, projected start "
                  f"{start:.4g} -> {loss:.4g}", flush=True)
    with open(path, "w") as fh:
        json.dump(dict(loss="mean squared difference to the direct FBP over the training "
                            "phantoms (image space)",
                       fit="variable projection: least-squares numerator, Nelder-Mead feedback "
                           "from the iir_coeffs.json filter of the same order",
                       entries=entries), fh, indent=1)


def _table_loss(N, sinos, target, b, a):
    return _Problem(N, sinos, target).loss(b, a)[0]


if __name__ == "__main__":
    import sys
    fit_table(*(sys.argv[1:2] or [_TABLE]))
