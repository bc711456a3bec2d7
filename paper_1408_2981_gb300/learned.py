"""Training of the learned form (include/tpmg_learned.h) from solves of the method.

Data: seeded smooth right-hand sides -- random combinations of the real
spherical harmonics up to degree ``l_max`` times vertical cosines, as cell
integrals -- each solved by plain TPMG-PCG (the mixed-precision form).  Each
solve gives

* WARM pairs: the network inputs of a seeded random subset of fine columns of f
  and the targets u / s of the same columns;
* COARSE pairs: the right-hand sides that the coarsest level received in the
  solve's V-cycles (recorded by the library) and their coarsest-level
  solutions (the V-cycle's coarse solve run to convergence), over all coarse
  columns.

Training: Adam on minibatches (``Net.train_step``: forward, loss, backward and
update in the library's kernels), learning rate decayed by a cosine from
``lr`` to ``lr / 100``, a fresh seeded permutation of the rows every epoch.

torch holds the device buffers and assembles minibatches (a gather of rows);
it also forms each smooth field as the product of the precomputed basis with
the pair's seeded coefficients.  The solves, features, targets and all of the
network's arithmetic run in the library.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import binding, inputs


def init_params(sizes, seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, from the seeded stream."""
    parts = []
    for l, (i, o) in enumerate(zip(sizes[:-1], sizes[1:])):
        bound = math.sqrt(6.0 / i) if l < len(sizes) - 2 else math.sqrt(3.0 / i)
        parts.append(inputs.uniform_pm1(seed + 7919 * l, o * i) * bound)
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


class SmoothFields:
    """Seeded smooth right-hand sides on the finest level of a solver:

        f_Tk = |T| v_k sum_{l <= l_max, |m| <= l, n <= n_max} c_lmn Y_lm(c_T) cos(n pi z_k / H) / (1 + l)^decay,

    c uniform[-1, 1] from the seed (inputs.smooth_field's ordering), built on
    the device as (Y C) V^T."""

    def __init__(self, solver, l_max: int = 16, n_max: int = 3, decay: float = 1.0):
        import torch

        mesh = solver.export_mesh()
        c, r = mesh["centres"], mesh["r_faces"]
        H = r[-1] - r[0]
        zmid = 0.5 * (r[:-1] + r[1:]) - r[0]
        Y = np.stack([inputs.real_sph_harm(l, m, c) / (1.0 + l) ** decay
                      for l in range(l_max + 1) for m in range(-l, l + 1)], axis=1)
        V = np.stack([np.cos(n * math.pi * zmid / H) for n in range(n_max + 1)], axis=1)
        dr = r[1:] - r[:-1]
        vol = dr * (r[1:] ** 2 + r[1:] * r[:-1] + r[:-1] ** 2) / 3.0   # factored: r^3 differences cancel
        self.n_coef = Y.shape[1] * (n_max + 1)
        self.shape = (Y.shape[1], n_max + 1)
        self.Y = torch.from_numpy(Y).cuda()
        self.V = torch.from_numpy(V).cuda()
        self.w = torch.from_numpy(np.outer(mesh["areas"], vol)).cuda()
        self.N = solver.N

    def field(self, seed: int):
        import torch

        C = torch.from_numpy(inputs.uniform_pm1(seed, self.n_coef).reshape(self.shape)).cuda()
        return ((self.Y @ C) @ self.V.T * self.w).reshape(-1).contiguous()


def generate(solver, fields: SmoothFields, n_pairs: int, seed: int, cells_per_pair: int = 512,
             coarse_per_pair: int = 4, coarse_sweeps: int = 16, rtol: float = 1e-6, max_iter: int = 200,
             log=None) -> dict:
    """(x, t) training rows for the WARM and COARSE networks from n_pairs plain
    solves of seeded smooth fields.  ``solver`` must be a mixed-precision
    Solver with graphs=0 (the coarse recording follows the host-driven loop)."""
    import torch

    n_r = solver.n_r
    n_fine = solver.n_cells
    n0 = solver.query(0)[0]
    M = min(cells_per_pair, n_fine)
    xw = torch.empty((n_pairs * M, 2 * n_r), dtype=torch.float32, device="cuda")
    tw = torch.empty((n_pairs * M, n_r), dtype=torch.float32, device="cuda")
    K = coarse_per_pair
    xc = torch.empty((n_pairs * K * n0, 2 * n_r), dtype=torch.float32, device="cuda") if K else None
    tc = torch.empty((n_pairs * K * n0, n_r), dtype=torch.float32, device="cuda") if K else None
    rec_cap = 64
    rec = torch.zeros(rec_cap * n0 * n_r, dtype=torch.float64, device="cuda") if K else None
    u0 = torch.zeros(n0 * n_r, dtype=torch.float64, device="cuda")
    iters, n_coarse = [], 0
    t0 = time.perf_counter()
    for p in range(n_pairs):
        f = fields.field(seed + p)
        u = torch.zeros_like(f)
        if K:
            solver.record_coarse(rec, rec_cap)
        st, it, rel, _ = solver.solve(f, u, rtol=rtol, max_iter=max_iter)
        iters.append(it)
        cells = (inputs.splitmix64(seed + 1000003 + p, M) % np.uint64(n_fine)).astype(np.int32)
        cells_t = torch.from_numpy(cells).cuda()
        solver.net_features(solver.n_levels - 1, f, xw[p * M:(p + 1) * M], cells=cells_t)
        solver.net_targets(solver.n_levels - 1, f, u, tw[p * M:(p + 1) * M], cells=cells_t)
        if K:
            got = solver.record_count()
            solver.record_coarse(None)
            # the first K recorded right-hand sides (the V-cycles of the first iterations)
            for j in range(min(K, got)):
                f0 = rec[j * n0 * n_r:(j + 1) * n0 * n_r]
                solver.coarse_solve(f0, u0, coarse_sweeps)
                rows = slice(n_coarse * n0, (n_coarse + 1) * n0)
                solver.net_features(0, f0, xc[rows])
                solver.net_targets(0, f0, u0, tc[rows])
                n_coarse += 1
        if log and (p + 1) % max(1, n_pairs // 10) == 0:
            log(f"  pairs {p + 1}/{n_pairs}: {time.perf_counter() - t0:.1f} s, solve iterations {it}")
    torch.cuda.synchronize()
    out = dict(xw=xw, tw=tw, iters=iters, seconds=time.perf_counter() - t0)
    if K:
        out["xc"], out["tc"] = xc[:n_coarse * n0], tc[:n_coarse * n0]
    return out


def train(net, x, t, steps: int, seed: int, batch: int = 4096, lr: float = 2e-3, log=None) -> dict:
    """Adam on (x, t) for `steps` minibatches; returns the loss history
    (loss before the step, every steps // 20 steps) and the final full-set loss."""
    import torch

    rows = x.shape[0]
    batch = min(batch, rows)
    per_epoch = max(1, rows // batch)
    hist = []
    t0 = time.perf_counter()
    perm = None
    for s in range(steps):
        e, b = divmod(s, per_epoch)
        if b == 0:
            key = inputs.splitmix64(seed + e, rows)
            perm = torch.from_numpy(np.argsort(key, kind="stable").astype(np.int64)).cuda()
            xs, ts = x.index_select(0, perm), t.index_select(0, perm)
        sl = slice(b * batch, (b + 1) * batch)
        rate = lr * (0.01 + 0.99 * 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps))))
        want = s % max(1, steps // 20) == 0
        loss = net.train_step(xs[sl], ts[sl], rate, want_loss=want)
        if want:
            hist.append((s, loss))
            if log:
                log(f"  step {s}: loss {loss:.3e}")
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    return dict(history=hist, seconds=seconds, final=full_loss(net, x, t))


def full_loss(net, x, t, chunk: int = 1 << 18) -> float:
    """Mean squared error of the network over all rows (forward in the library)."""
    import torch

    total, n = 0.0, 0
    for i in range(0, x.shape[0], chunk):
        xs, ts = x[i:i + chunk], t[i:i + chunk]
        y = torch.empty_like(ts)
        net.forward(xs.contiguous(), y)
        total += float(((y.double() - ts.double()) ** 2).sum())
        n += ts.numel()
    return total / max(n, 1)
