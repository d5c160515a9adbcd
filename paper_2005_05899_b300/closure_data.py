"""Training data and a-priori evaluation for the learned eddy-viscosity closure.

The network stands in for the Vreman closure (section 2.1); the paper has no
learned model, so this module defines the data pipeline:

1. **Fine runs of the plain method.**  A Taylor-Green vortex (nu = 1/1600) on
   an n_f^3 periodic Kuhn tet mesh, advanced by the three RK3 stages of
   Algorithm 1 with the library's element assembly (mixed precision, Vreman
   closure) for the momentum RHS.  Two ways to keep it divergence-free:
   `projection="library"` runs Algorithm 1 itself, the library's pressure
   projection (Jacobi-PCG on the Galerkin Laplacian) once per step after the
   stages, which use the frozen pressure; `projection="spectral"` makes the
   velocity divergence-free after every stage by a spectral (Leray)
   projection on the periodic node grid, which needs no iteration (the
   training sets of large fine meshes, where the CG solve would take
   thousands of iterations per step).
2. **Box filter** of the fine nodal velocity to a coarse grid of n_f / r
   cells per direction (trapezoidal top-hat of width r fine cells, periodic),
   for r in `ratios` (several filter widths give the network the range of
   Delta it is later applied to).
3. **Samples per coarse TET04 element**: the FE gradient G of the filtered
   velocity, Delta = V_e^(1/3), the subgrid stress tau = bar(u u) - bar(u)
   bar(u) averaged over the element's vertices, and the least-squares eddy
   viscosity nu_t* = max(0, -tau^d : S / (2 S : S)), S = (G + G^T)/2.
4. **Features** exactly as the kernels compute them, dimensionless so that a
   network fitted on one flow transfers to other scales: the invariants of S
   and O = (G - G^T)/2 over powers of g = |G|, and the element Reynolds
   number log(Delta^2 g / nu).  The network's target is the coefficient
   C* = nu_t* / (Delta^2 g) (the closure evaluates nu_t = C Delta^2 g).

All GPU work uses the library (assembly, fold, lumped mass, MLP training and
inference); torch supplies device memory, FFTs and elementwise data plumbing.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence

import numpy as np
import torch

from . import fea
from . import meshgen as mg


@dataclasses.dataclass
class Snapshot:
    t: float
    u: torch.Tensor          # fine master-grid velocity [3, n, n, n] (index order k, j, i), float64, cuda


def _master_grid(mesh: mg.Mesh, n: int):
    """Node index of every master grid point (i, j, k) of an unsorted tgv_mesh, and
    the master of every stored node (as grid-flat index k*n*n + j*n + i)."""
    g = np.arange(n)
    k, j, i = np.meshgrid(g, g, g, indexing="ij")
    nid = (i + (n + 1) * (j + (n + 1) * k)).ravel()
    gi = np.arange((n + 1) ** 3)
    ii, jj, kk = gi % (n + 1), (gi // (n + 1)) % (n + 1), gi // (n + 1) ** 2
    flat = (kk % n) * n * n + (jj % n) * n + (ii % n)
    return torch.as_tensor(nid, device="cuda"), torch.as_tensor(flat, device="cuda")


def _leray(ug: torch.Tensor) -> torch.Tensor:
    """Divergence-free projection of a periodic velocity [3, n, n, n] on (2 pi)^3."""
    n = ug.shape[-1]
    k = torch.fft.fftfreq(n, d=1.0 / n, device=ug.device, dtype=torch.float64)
    kz, ky, kx = torch.meshgrid(k, k, k, indexing="ij")
    kk = torch.stack([kx, ky, kz])
    k2 = (kk * kk).sum(0)
    k2[0, 0, 0] = 1.0
    uh = torch.fft.fftn(ug, dim=(1, 2, 3))
    div = (kk * uh).sum(0)
    uh = uh - kk * (div / k2)[None]
    return torch.fft.ifftn(uh, dim=(1, 2, 3)).real


def fine_tgv_run(ctx: fea.Context, n_f: int, t_snap: Sequence[float], nu: float = 1.0 / 1600.0,
                 c_vreman: float = 0.07, cfl: float = 0.3, log=None, projection: str = "spectral",
                 stats: Dict = None) -> List[Snapshot]:
    """Fine LES of the Taylor-Green vortex; returns master-grid snapshots at
    t_snap.  projection: "spectral" (Leray projection of every stage) or
    "library" (the library's RK3 stages and pressure projection per step,
    Algorithm 1); stats, if given, receives the CG iteration counts."""
    mesh = mg.tgv_mesh(n_f, sfc=False)
    field = mg.tgv_field(mesh, nu=nu, c_vreman=c_vreman)
    dm = ctx.upload_mesh(mesh)
    N = dm.n_nodes
    node_of, master_flat = _master_grid(mesh, n_f)
    mass = torch.empty(N, dtype=torch.float64, device="cuda")
    dm.lumped_mass(mass)
    dm.fold(mass)
    minv = 1.0 / mass
    u = torch.tensor(np.ascontiguousarray(field.u.T), device="cuda")
    p0 = torch.zeros(N, dtype=torch.float64, device="cuda")
    R = torch.empty((3, N), dtype=torch.float64, device="cuda")

    def to_grid(v):
        return v[:, node_of].reshape(3, n_f, n_f, n_f)

    def from_grid(g):
        return g.reshape(3, -1)[:, master_flat].contiguous()

    def L(v):
        dm.upload_field(v, p0, nu, c_vreman)
        dm.assemble(R, prec="mixed", closure="vreman")
        dm.fold(R)
        return R * minv

    h = 2 * math.pi / n_f
    dt = cfl * h          # |u| <= 1 for this flow
    t = 0.0
    out = []
    targets = sorted(t_snap)
    ti = 0
    if projection == "library":
        dm.upload_field(u, torch.tensor(field.p, device="cuda"), nu, c_vreman)
        dm.poisson_setup()
        state = torch.empty((3, N), dtype=torch.float64, device="cuda")
        iters = []
        while ti < len(targets):
            step = min(dt, targets[ti] - t)
            if step <= 1e-12:
                dm.state(state)
                torch.cuda.synchronize()
                out.append(Snapshot(t, to_grid(state).clone()))
                ti += 1
                continue
            for k in range(3):
                dm.rk_stage(k, step, prec="mixed", closure="vreman")
            it, rr = dm.project(step, rtol=1e-8, max_iter=20000)
            iters.append(it)
            t += step
            if log and abs(t - round(t)) < 0.5 * dt:
                log(f"fine run (library projection) t={t:.2f} CG iterations {it} residual {rr:.1e}")
        if stats is not None:
            stats["cg_iterations"] = iters
        ctx.sync_status()
        return out
    while ti < len(targets):
        step = min(dt, targets[ti] - t)
        if step <= 1e-12:
            out.append(Snapshot(t, to_grid(u).clone()))
            ti += 1
            continue
        un = u
        u1 = from_grid(_leray(to_grid(un + step * L(un))))
        u2 = from_grid(_leray(to_grid(0.75 * un + 0.25 * (u1 + step * L(u1)))))
        u = from_grid(_leray(to_grid(un / 3.0 + 2.0 / 3.0 * (u2 + step * L(u2)))))
        t += step
        if log and abs(t - round(t)) < 0.5 * dt:
            log(f"fine run t={t:.2f} max|u|={u.abs().max().item():.3f}")
    ctx.sync_status()
    return out


def _box(g: torch.Tensor, r: int) -> torch.Tensor:
    """Periodic trapezoidal top-hat of width r cells along the last three axes."""
    w = torch.ones(r + 1, dtype=g.dtype, device=g.device)
    w[0] = w[-1] = 0.5
    w /= r
    out = g
    for ax in (-1, -2, -3):
        acc = torch.zeros_like(out)
        for q, wq in zip(range(-r // 2, r // 2 + 1), w):
            acc = acc + wq * torch.roll(out, shifts=-q, dims=ax)
        out = acc
    return out


@dataclasses.dataclass
class CoarseSet:
    n_c: int
    mesh: mg.Mesh
    u_nodes: np.ndarray       # (N, 3) filtered velocity at the coarse mesh's stored nodes
    feats: np.ndarray         # (E, 6) raw (dimensionless) features per element
    target: np.ndarray        # (E,) nu_t*
    coef: np.ndarray          # (E,) the network's target C* = nu_t* / (Delta^2 |G|) (NaN where G = 0)
    tau_d: np.ndarray         # (E, 3, 3) deviatoric subgrid stress per element (None: training only)
    grad_n: np.ndarray        # (E, 4, 3) shape-function gradients (None: training only)
    vol: np.ndarray           # (E,)


def _features(G: torch.Tensor, delta: torch.Tensor, nu: float):
    """The closure's dimensionless inputs (the library's and the oracle's
    definition): invariants of S and O over powers of g = |G|, and
    log(Delta^2 g / nu); returns (features (E, 6), g (E,))."""
    S = 0.5 * (G + G.transpose(1, 2))
    O = 0.5 * (G - G.transpose(1, 2))
    S2, O2 = S @ S, O @ O

    def tr(a):
        return a.diagonal(dim1=1, dim2=2).sum(-1)

    g2 = (G * G).sum((1, 2))
    g = g2.sqrt()
    some = g2 > 0
    safe = torch.where(some, g, torch.ones_like(g))
    inv = [tr(S2), tr(O2), tr(S2 @ S), tr(S @ O2), tr(S2 @ O2)]
    deg = [2.0, 2.0, 3.0, 3.0, 4.0]
    cols = [torch.where(some, v / safe ** d, torch.zeros_like(v)) for v, d in zip(inv, deg)]
    cols.append(torch.where(some, torch.log(delta * delta * safe / nu), torch.zeros_like(g)))
    return torch.stack(cols, dim=1), g


def coarse_samples(snap: Snapshot, r: int, keep_stress: bool = True, nu: float = 1.0 / 1600.0) -> CoarseSet:
    """Filtered coarse field, features and targets at filter ratio r; the
    per-element stresses and gradients are kept for the a-priori comparison
    only when keep_stress."""
    n_f = snap.u.shape[-1]
    n_c = n_f // r
    ub = _box(snap.u, r)[:, ::r, ::r, ::r].contiguous()                  # [3, n_c^3]
    prods = {}
    for a in range(3):
        for b in range(a, 3):
            prods[(a, b)] = _box(snap.u[a] * snap.u[b], r)[::r, ::r, ::r]
    tau = torch.empty((3, 3) + ub.shape[1:], dtype=torch.float64, device="cuda")
    for (a, b), v in prods.items():
        tau[a, b] = v - ub[a] * ub[b]
        tau[b, a] = tau[a, b]
    mesh = mg.tgv_mesh(n_c, sfc=False)
    node_of, master_flat = _master_grid(mesh, n_c)
    u_nodes = ub.reshape(3, -1)[:, master_flat].T.contiguous()          # (N, 3)
    tau_nodes = tau.reshape(3, 3, -1)[:, :, master_flat].permute(2, 0, 1)  # (N, 3, 3)
    conn = torch.as_tensor(mesh.conn[mg.TET04].astype(np.int64), device="cuda")
    X = torch.as_tensor(mesh.xyz, device="cuda")[conn]                  # (E, 4, 3)
    E = torch.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], dim=1)
    vol = torch.linalg.det(E) / 6.0
    grads = torch.linalg.inv(E).transpose(1, 2)                          # rows: grad of N_1..N_3
    gN = torch.cat([-grads.sum(1, keepdim=True), grads], dim=1)         # (E, 4, 3)
    U = u_nodes[conn]                                                    # (E, 4, 3)
    G = torch.einsum("eai,eaj->eij", U, gN)                              # G_ij = sum_a u_a,i dN_a/dx_j
    S = 0.5 * (G + G.transpose(1, 2))
    te = tau_nodes[conn].mean(1)
    td = te - torch.eye(3, device="cuda", dtype=torch.float64) * (te.diagonal(dim1=1, dim2=2).sum(-1) / 3.0)[:, None, None]
    ss = (S * S).sum((1, 2))
    target = torch.clamp(-(td * S).sum((1, 2)) / (2.0 * ss + 1e-300), min=0.0)
    delta = vol.abs() ** (1.0 / 3.0)
    feats, g = _features(G, delta, nu)
    coef = torch.where(g > 0, target / (delta * delta * torch.where(g > 0, g, torch.ones_like(g))),
                       torch.full_like(g, float("nan")))
    return CoarseSet(n_c=n_c, mesh=mesh, u_nodes=u_nodes.cpu().numpy(), feats=feats.cpu().numpy(),
                     target=target.cpu().numpy(), coef=coef.cpu().numpy(),
                     tau_d=td.cpu().numpy() if keep_stress else None,
                     grad_n=gN.cpu().numpy() if keep_stress else None, vol=vol.cpu().numpy())


def generate(ctx: fea.Context, n_f: int = 96, ratios=(4, 8), t_snap=(3.0, 4.0, 5.0, 6.0, 7.0, 8.0), log=None,
             t_stress=None, projection: str = "spectral", stats: Dict = None):
    """Fine run + filtered samples: {t: [CoarseSet per ratio]}; stresses kept
    at the times in t_stress (all when None)."""
    snaps = fine_tgv_run(ctx, n_f, t_snap, log=log, projection=projection, stats=stats)
    return {s.t: [coarse_samples(s, r, keep_stress=t_stress is None or s.t in t_stress) for r in ratios]
            for s in snaps}


@dataclasses.dataclass
class TrainedClosure:
    theta: np.ndarray
    mean: np.ndarray
    std: np.ndarray
    scale: float
    losses: List[float]       # batch losses every 100 steps (units of scale^2; targets C* / scale)
    fit_mse: float = float("nan")      # full training set, same units
    n_samples: int = 0
    env_lo: np.ndarray = None          # training envelope (raw features), set in the context
    env_hi: np.ndarray = None
    target_var: float = float("nan")   # variance of the normalised target (the best constant's MSE)


def train(ctx: fea.Context, sets: Sequence[CoarseSet], steps: int = 2000, batch: int = 65536, lr: float = 2e-3,
          seed: int = 0, max_per_set: int = 2_000_000, envelope_q: float = 1e-4) -> TrainedClosure:
    """Fits the network to the coefficient C* = nu_t* / (Delta^2 |G|) on the
    GPU (the library's training step).
    Each set contributes at most max_per_set seeded random samples, so fine
    filter widths (many coarse elements) do not swamp the coarse ones.  The
    per-feature [q, 1 - q] quantiles of the training features, widened by 5 %
    of their range, become the closure's envelope (Vreman outside it)."""
    rng = np.random.default_rng(seed)
    xs, ys = [], []
    for c in sets:
        take = np.arange(c.target.size)
        if take.size > max_per_set:
            take = np.sort(rng.choice(take.size, max_per_set, replace=False))
        xs.append(c.feats[take])
        ys.append(c.coef[take])
    x = np.concatenate(xs).astype(np.float32)
    y = np.concatenate(ys)
    keep = np.all(np.isfinite(x), axis=1) & np.isfinite(y)
    x, y = x[keep], y[keep]
    mean = x.mean(axis=0)
    std = x.std(axis=0) + 1e-6
    scale = float(np.mean(y)) + 1e-12
    theta = np.zeros(fea.MLP_NPARAM, np.float32)
    off = 0
    for n_out, n_in in ((64, 6), (64, 64), (64, 64), (1, 64)):
        lim = math.sqrt(6.0 / (n_in + n_out))
        theta[off:off + n_out * n_in] = rng.uniform(-lim, lim, n_out * n_in)
        off += n_out * n_in + n_out
    ctx.mlp_load(theta, mean.astype(np.float32), std.astype(np.float32), scale)
    xt = torch.tensor(x, device="cuda")
    yt = torch.tensor((y / scale).astype(np.float32), device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    losses = []
    n = x.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    for step in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), device="cuda", generator=g)
        lr_s = lr * (0.1 ** (step / max(steps, 1)))
        ctx.mlp_train_step(xt[idx].contiguous(), yt[idx].contiguous(), lr_s, loss_out=loss)
        if step % 100 == 0 or step == steps - 1:
            torch.cuda.synchronize()
            losses.append(loss.item())
    ctx.sync_status()
    # fit on the whole training set with the trained weights (inference kernel)
    pred = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.mlp_forward(xt, pred)
    ctx.sync_status()
    ys = yt.double()
    mse = float(((pred.double() / scale - ys) ** 2).mean())
    var = float(ys.var(unbiased=False))
    lo = np.quantile(x, envelope_q, axis=0)
    hi = np.quantile(x, 1.0 - envelope_q, axis=0)
    # widen by 5 % of each range: a feature that takes few distinct values (log
    # Delta on a uniform grid) must not fail the test by the rounding of the
    # kernel's own evaluation
    pad = 0.05 * (hi - lo)
    lo = (lo - pad).astype(np.float32)
    hi = (hi + pad).astype(np.float32)
    ctx.mlp_set_envelope(lo, hi)
    return TrainedClosure(theta=ctx.mlp_get(), mean=mean, std=std, scale=scale, losses=losses,
                          fit_mse=mse, target_var=var, n_samples=n, env_lo=lo, env_hi=hi)


def apriori_errors(ctx: fea.Context, cs: CoarseSet, nu: float = 1.0 / 1600.0, c_vreman: float = 0.07) -> Dict:
    """nu_t and subgrid-force errors of no model, Vreman and the loaded MLP on
    one filtered coarse field.  Subgrid force: R_a = sum_e V_e tau_ij d_j N_a
    (true, from the filtered stresses) against the library's assembly with
    only the subgrid term (closure Vreman or MLP); both folded."""
    mesh = cs.mesh
    dm = ctx.upload_mesh(mesh)
    dm.upload_field(cs.u_nodes, np.zeros(mesh.n_nodes), nu, c_vreman)
    N = dm.n_nodes
    conn = mesh.conn[mg.TET04].astype(np.int64)
    true = np.zeros((N, 3))
    contrib = cs.vol[:, None, None] * np.einsum("eij,eaj->eai", cs.tau_d, cs.grad_n)
    for a in range(4):
        np.add.at(true, conn[:, a], contrib[:, a])
    true_t = torch.tensor(np.ascontiguousarray(true.T), device="cuda")
    dm.fold(true_t)
    masters = np.unique(mesh.periodic_master)
    tnorm = np.linalg.norm(true_t.cpu().numpy()[:, masters])
    u_m = cs.u_nodes[masters].T
    true_m = true_t.cpu().numpy()[:, masters]
    diss_true = float((u_m * true_m).sum())          # sum_e V_e tau^d : G_e, the subgrid energy transfer
    out = {"none": {"nut": 1.0, "rhs": 1.0, "diss": 1.0}, "diss_true": diss_true}
    R = torch.empty((3, N), dtype=torch.float64, device="cuda")
    nut = torch.empty(dm.n_gauss_total, dtype=torch.float32, device="cuda")
    tgt = cs.target
    for name in ("vreman", "mlp"):
        if name == "mlp":
            ctx.mlp_fallback_read(reset=True)
        dm.assemble(R, prec="mixed", closure=name, mask=fea.TERM_SGS, nut_out=nut)
        dm.fold(R)
        ctx.sync_status()
        if name == "mlp":
            out["fallback_frac"] = ctx.mlp_fallback_read(reset=True) / dm.n_gauss_total
        r = R.cpu().numpy()[:, masters]
        nt = nut.cpu().numpy().reshape(-1, 4)[:, 0]
        diss = float((u_m * r).sum())
        out[name] = {"nut": float(np.linalg.norm(nt - tgt) / np.linalg.norm(tgt)),
                     "rhs": float(np.linalg.norm(r - true_m) / tnorm),
                     "nut_corr": float(np.corrcoef(nt, tgt)[0, 1]),
                     "diss": abs(diss - diss_true) / abs(diss_true), "diss_model": diss}
    return out


def run(n_f: int = 96, ratios=(4, 8), t_train=(3.0, 4.0, 5.0, 7.0, 8.0), t_test=(6.0,), steps: int = 2000,
        save: str = "", log=print, ctx: fea.Context = None, projection: str = "spectral") -> Dict:
    """Fine run, filtering, GPU training and the a-priori comparison on held-out times.

    Returns a JSON-able dict plus the key "model" (the TrainedClosure, left
    loaded in the context when one is passed in)."""
    import time
    own = ctx is None
    if own:
        ctx = fea.Context(0)
    t0 = time.time()
    stats: Dict = {}
    data = generate(ctx, n_f=n_f, ratios=ratios, t_snap=sorted(set(t_train) | set(t_test)), log=log,
                    t_stress=set(t_test), projection=projection, stats=stats)
    t_gen = time.time() - t0
    train_sets = [c for t in t_train for c in data[t]]
    test_sets = [c for t in t_test for c in data[t]]
    t0 = time.time()
    model = train(ctx, train_sets, steps=steps)
    t_train_s = time.time() - t0
    if save:
        np.savez(save, theta=model.theta, mean=model.mean, std=model.std, scale=model.scale, env_lo=model.env_lo,
                 env_hi=model.env_hi)
    res = {"n_f": n_f, "ratios": list(ratios), "projection": projection, "samples_train": int(model.n_samples),
           "generate_s": t_gen, "train_s": t_train_s, "loss_first": model.losses[0], "loss_last": model.losses[-1],
           "fit_mse": model.fit_mse, "target_var": model.target_var, "test": []}
    if stats.get("cg_iterations"):
        its = stats["cg_iterations"]
        res["cg_iterations"] = {"steps": len(its), "mean": float(np.mean(its)), "max": int(np.max(its))}
    for c in test_sets:
        e = apriori_errors(ctx, c)
        e["n_c"] = c.n_c
        res["test"].append(e)
    res["model"] = model
    if own:
        ctx.close()
    return res


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-f", type=int, default=96)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--save", default="")
    ap.add_argument("--projection", choices=["spectral", "library"], default="spectral")
    a = ap.parse_args()
    r = run(n_f=a.n_f, steps=a.steps, save=a.save, projection=a.projection)
    r.pop("model")
    print(json.dumps(r), flush=True)
