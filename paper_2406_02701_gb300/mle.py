"""Maximum-likelihood fit of a Matérn covariance on the GPU (the paper's MLE
workload, Sec. 6.2: an optimiser that calls the negative log-likelihood of
(log range, log variance) many times with the locations and the data fixed).

The optimiser is the Nelder-Mead simplex method (Nelder & Mead, The Computer
Journal 7, 1965; the default method of R's `optim`, which the paper uses),
with the usual coefficients: reflection 1, expansion 2, contraction 1/2,
shrink 1/2.  Evaluations are issued in batches: the initial simplex, every
shrink, and -- with `speculative=True` -- the four candidate points of an
iteration (reflection, expansion, outside and inside contraction) go out
together, and the method then takes exactly the decisions it takes when it
evaluates them one at a time.

`MaternMLE` keeps `lanes` tiled matrices of one layout, each on its own CUDA
stream, and the Morton-ordered points and data on the device; a batch of
parameter vectors is spread over the lanes and runs concurrently (generation,
factorisation and log-likelihood with FP64 refinement for each).
"""
from __future__ import annotations

import math

import numpy as np

ALPHA, GAMMA, RHO, SIGMA = 1.0, 2.0, 0.5, 0.5


REL_TOL = 1.490116119384765625e-08   # sqrt of the double epsilon, R optim's reltol


def nelder_mead(f_batch, x0, step=0.5, max_iter=200, reltol=REL_TOL, xtol=None, speculative=False):
    """Minimises f over R^d.  f_batch maps a list of points (1-D arrays) to a
    list of values.  Stops when the spread of f over the simplex is at most
    reltol (|f(x0)| + reltol), the tolerance fixed once from the value at
    the starting point (R optim's rule), or, with xtol, when every vertex
    lies within xtol of the best one.  Returns dict(x, f, iters, evals,
    simplex, fvals, rounds, converged) -- rounds counts the calls of
    f_batch (sequential round trips); converged is False when max_iter, not
    a stopping rule, ended the search."""
    x0 = np.asarray(x0, dtype=np.float64)
    d = x0.size
    simplex = [x0.copy()]
    for i in range(d):
        x = x0.copy()
        x[i] += step
        simplex.append(x)
    stats = {"evals": 0, "rounds": 0}

    def ev(points):
        stats["evals"] += len(points)
        stats["rounds"] += 1
        # a value that is not a number ranks as the worst possible
        return [float(v) if not math.isnan(v) else math.inf for v in f_batch(points)]

    fv = ev(simplex)
    convtol = reltol * (abs(fv[0]) + reltol) if math.isfinite(fv[0]) else math.inf
    it = 0
    converged = False
    while True:
        order = np.argsort(fv, kind="stable")
        simplex = [simplex[k] for k in order]
        fv = [fv[k] for k in order]
        if fv[-1] - fv[0] <= convtol:
            converged = True
            break
        if xtol is not None and max(np.max(np.abs(x - simplex[0])) for x in simplex[1:]) <= xtol:
            converged = True
            break
        if it >= max_iter:
            break
        it += 1
        xo = np.mean(simplex[:-1], axis=0)
        xw = simplex[-1]
        xr = xo + ALPHA * (xo - xw)
        xe = xo + GAMMA * (xr - xo)
        xc = xo + RHO * (xr - xo)        # outside contraction
        xcc = xo + RHO * (xw - xo)       # inside contraction
        if speculative:
            fr, fe, fc, fcc = ev([xr, xe, xc, xcc])
        else:
            fr, = ev([xr])
            fe = fc = fcc = None
        if fv[0] <= fr < fv[-2]:
            simplex[-1], fv[-1] = xr, fr
            continue
        if fr < fv[0]:
            if fe is None:
                fe, = ev([xe])
            if fe < fr:
                simplex[-1], fv[-1] = xe, fe
            else:
                simplex[-1], fv[-1] = xr, fr
            continue
        if fr < fv[-1]:
            if fc is None:
                fc, = ev([xc])
            if fc <= fr:
                simplex[-1], fv[-1] = xc, fc
                continue
        else:
            if fcc is None:
                fcc, = ev([xcc])
            if fcc < fv[-1]:
                simplex[-1], fv[-1] = xcc, fcc
                continue
        # shrink towards the best point
        shrunk = [simplex[0] + SIGMA * (x - simplex[0]) for x in simplex[1:]]
        fs = ev(shrunk)
        simplex = [simplex[0]] + shrunk
        fv = [fv[0]] + fs
    k = int(np.argmin(fv))
    return dict(x=simplex[k], f=fv[k], iters=it, evals=stats["evals"], rounds=stats["rounds"],
                simplex=np.array(simplex), fvals=np.array(fv), converged=converged)


class MaternMLE:
    """Negative log-likelihood of (log range, log sigma^2) for fixed nu and
    nugget, evaluated on the GPU; `fit` runs Nelder-Mead on it."""

    def __init__(self, ctx, locs, z, b, nu, nugget=1e-4, pmap=None, lanes=4, refine_iters=20,
                 ozaki=True):
        import torch
        from . import mpchol
        self.ctx, self.nu, self.nugget, self.refine = ctx, float(nu), float(nugget), refine_iters
        locs = np.ascontiguousarray(np.asarray(locs, dtype=np.float64))
        z = np.asarray(z, dtype=np.float64).reshape(-1)
        n = locs.shape[0]
        assert z.shape[0] == n
        dev = torch.device("cuda", ctx.device)
        dl = torch.from_numpy(locs).to(dev)
        # points in Morton order (the tiles' locality), data permuted alike
        self.locs, perm = ctx.morton_order(dl)
        zp = torch.from_numpy(z).to(dev)[perm]
        self.zt = zp.reshape(1, n).contiguous()
        torch.cuda.synchronize()
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(lanes)]
        self.mats = [mpchol.TiledMatrix(ctx, n, b, pmap, keep_sigma=refine_iters > 0, stream=s,
                                        ozaki=ozaki) for s in self.streams]
        self.out = [(torch.empty(1, dtype=torch.float64, device=dev),
                     torch.empty(1, dtype=torch.float64, device=dev),
                     torch.empty(1, dtype=torch.int32, device=dev)) for _ in range(lanes)]
        self.evals = 0

    def loglik(self, thetas):
        """Log-likelihoods at the parameter vectors (range, sigma^2) in
        `thetas`, lanes at a time; -inf where the matrix is not SPD or the
        FP64 refinement of the solve did not converge within its iteration
        cap (far from the data's scale the condition number grows until the
        refinement with the lower-precision factor no longer contracts; such
        a value is not the log-likelihood)."""
        import torch
        res = []
        lanes = len(self.mats)
        for c0 in range(0, len(thetas), lanes):
            chunk = thetas[c0:c0 + lanes]
            infos = []
            for (rng, s2), T, s, (ll, q, it) in zip(chunk, self.mats, self.streams, self.out):
                with torch.cuda.stream(s):
                    T.generate(self.locs, float(s2), float(rng), self.nu, self.nugget)
                    info, _ = T.chol()
                    T.loglik(self.zt, refine_iters=self.refine, ll=ll, quad=q, iters=it)
                    infos.append(info)
            for s in self.streams[:len(chunk)]:
                s.synchronize()
            for info, (ll, _, it) in zip(infos, self.out):
                ok = int(info.item()) == 0 and (self.refine == 0 or int(it.item()) < self.refine)
                res.append(float(ll.item()) if ok else -math.inf)
            self.evals += len(chunk)
        return res

    def nll_log(self, points):
        """Negative log-likelihood at points (log range, log sigma^2)."""
        ll = self.loglik([(math.exp(p[0]), math.exp(p[1])) for p in points])
        return [-v if math.isfinite(v) else math.inf for v in ll]

    def fit(self, range0, sigma2_0, step=0.5, max_iter=200, reltol=REL_TOL, speculative=True):
        r = nelder_mead(self.nll_log, [math.log(range0), math.log(sigma2_0)], step=step,
                        max_iter=max_iter, reltol=reltol, speculative=speculative)
        r["range"], r["sigma2"] = math.exp(r["x"][0]), math.exp(r["x"][1])
        r["loglik"] = -r["f"]
        return r

    def close(self):
        for T in self.mats:
            T.close()
        self.mats = []
