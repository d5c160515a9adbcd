"""GPU MLP closure kernels (tensor cores) against the FP64 oracle.

Tolerances.  Training: the GPU rounds weights W1..W3 and every hidden
activation to BF16 (8 significant bits, relative 2^-9 per rounding) and
accumulates in FP32; the gradient is compared at 5e-2 relative in the L2
norm against the oracle with the same BF16-rounded weights and inputs.
Inference (batched forward and the fused closure, on the tcgen05 tensor
cores): the same BF16 weight values held as FP16 operands, FP16 normalised
inputs, FP16 hidden activations from a tanh-form SiLU and FP16 hidden-layer
accumulators, an FP32 output layer; compared at rel 2e-2 (+ a floor of 1e-3
of the largest value) against the oracle on the BF16-rounded weights and the
FP16-rounded inputs.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2005_05899_b300 import fea

pytestmark = pytest.mark.gpu

H, I = 64, 6


def bf16_round(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def split(theta):
    off = 0
    out = {}
    for name, n in (("w1", H * I), ("b1", H), ("w2", H * H), ("b2", H), ("w3", H * H), ("b3", H), ("w4", H),
                    ("b4", 1)):
        out[name] = theta[off:off + n]
        off += n
    return out


def f16_round(a):
    return np.asarray(a, dtype=np.float64).astype(np.float16).astype(np.float64)


def gpu_rounded_theta(theta):
    """theta as the GPU evaluates it: W1..W3 in BF16, the rest FP32."""
    t = theta.astype(np.float32).copy()
    p = split(t)
    for name in ("w1", "w2", "w3"):
        p[name][:] = bf16_round(p[name])
    return t.astype(np.float64)


@pytest.fixture(scope="module")
def ctx():
    c = fea.Context(0)
    yield c
    c.close()


def sample_features(rng, n, nu=1e-3):
    G = rng.standard_normal((n, 3, 3)) * rng.uniform(0.1, 3.0, (n, 1, 1))
    delta = rng.uniform(0.005, 0.05, n)
    return np.stack([O.mlp_features(G[k], delta[k], nu) for k in range(n)]).astype(np.float32)


def test_forward_matches_oracle(ctx):
    rng = np.random.default_rng(0)
    theta = (0.3 * rng.standard_normal(fea.MLP_NPARAM)).astype(np.float32)
    x = sample_features(rng, 3000)
    mean = x.mean(axis=0).astype(np.float32)
    std = (x.std(axis=0) + 1e-3).astype(np.float32)
    scale = 2e-4
    ctx.mlp_load(theta, mean, std, scale)
    xt = torch.tensor(x, device="cuda")
    out = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    ctx.mlp_forward(xt, out)
    ctx.sync_status()
    got = out.cpu().numpy().astype(np.float64)
    # oracle on the GPU's BF16 weight values and FP16 normalised inputs
    xn = f16_round((x - mean) / std)
    mlp = O.MLPParams(gpu_rounded_theta(theta), np.zeros(6), np.ones(6), scale)
    ref = O.mlp_forward(mlp, xn)
    assert np.all(np.abs(got - ref) <= 2e-2 * np.abs(ref) + 1e-3 * np.abs(ref).max())
    assert np.corrcoef(got, ref)[0, 1] > 0.999


def test_gradient_matches_oracle_and_adam_step(ctx):
    rng = np.random.default_rng(1)
    theta = (0.3 * rng.standard_normal(fea.MLP_NPARAM)).astype(np.float32)
    B = 4099                       # ragged: not a multiple of the 64-row CTA tile
    x = sample_features(rng, B)
    mean = x.mean(axis=0).astype(np.float32)
    std = (x.std(axis=0) + 1e-3).astype(np.float32)
    y = rng.uniform(0.0, 2.0, B).astype(np.float32)
    ctx.mlp_load(theta, mean, std, 1.0)
    xt = torch.tensor(x, device="cuda")
    yt = torch.tensor(y, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    grad = torch.zeros(fea.MLP_NPARAM, dtype=torch.float32, device="cuda")
    lr = 1e-3
    ctx.mlp_train_step(xt, yt, lr, loss_out=loss, grad_out=grad)
    ctx.sync_status()
    g = grad.cpu().numpy().astype(np.float64)
    xn = bf16_round((x - mean) / std).astype(np.float64)
    ref_loss, ref_g = O.mlp_loss_grad(gpu_rounded_theta(theta), xn, y.astype(np.float64))
    assert abs(loss.item() - ref_loss) <= 2e-2 * ref_loss
    assert np.linalg.norm(g - ref_g) <= 5e-2 * np.linalg.norm(ref_g)
    for name_range in ((0, H * I), (H * I + H, H * I + H + H * H)):   # w1 and w2 blocks separately
        a, b = name_range
        assert np.linalg.norm(g[a:b] - ref_g[a:b]) <= 5e-2 * np.linalg.norm(ref_g[a:b])
    # Adam on the GPU gradient, against the oracle's Adam
    th = theta.astype(np.float64).copy()
    m1 = np.zeros_like(th)
    m2 = np.zeros_like(th)
    O.adam_step(th, g, m1, m2, lr, 0.9, 0.999, 1e-8, 1)
    new = ctx.mlp_get().astype(np.float64)
    assert np.abs(new - th).max() <= 1e-6


def test_training_reduces_loss(ctx):
    rng = np.random.default_rng(2)
    B = 16384
    x = sample_features(rng, B)
    mean = x.mean(axis=0).astype(np.float32)
    std = (x.std(axis=0) + 1e-3).astype(np.float32)
    # smooth synthetic target in out_scale units
    xn = (x - mean) / std
    y = np.log1p(np.exp(0.8 * xn[:, 0] - 0.5 * xn[:, 1] + 0.3 * xn[:, 5])).astype(np.float32)
    theta = (0.1 * rng.standard_normal(fea.MLP_NPARAM)).astype(np.float32)
    ctx.mlp_load(theta, mean, std, 1.0)
    xt = torch.tensor(x, device="cuda")
    yt = torch.tensor(y, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    first = None
    for step in range(300):
        ctx.mlp_train_step(xt, yt, 3e-3, loss_out=loss)
        if step == 0:
            torch.cuda.synchronize()
            first = loss.item()
    torch.cuda.synchronize()
    ctx.sync_status()
    assert loss.item() < 0.1 * first, (first, loss.item())


# ---------------------------------------------------------------------------
# the MLP closure fused into the assembly kernels

from paper_2005_05899_b300 import meshgen as mg  # noqa: E402


def closure_model(rng, mesh, field):
    """An MLP whose nu_t = C Delta^2 |G| is of the size of Vreman's (Vreman's
    nu_t / (Delta^2 |G|) is c sqrt(B / (G:G)) / |G| <= c / sqrt(2): the
    coefficient scale 0.03 with softplus of order one)."""
    theta = (0.2 * rng.standard_normal(fea.MLP_NPARAM)).astype(np.float32)
    scale = 0.03
    x = sample_features(rng, 2000, field.nu)
    mean = x.mean(axis=0).astype(np.float32)
    std = (x.std(axis=0) + 1e-3).astype(np.float32)
    return theta, mean, std, scale


@pytest.mark.parametrize("prec,scatter", [("mixed", "chunk"), ("mixed", "atomic"), ("fp64", "atomic")])
def test_assembly_with_mlp_closure_matches_oracle(ctx, prec, scatter):
    rng = np.random.default_rng(5)
    m = mg.channel_mesh(nx=10, ny=12, nz=8, seed=21, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=5, nu=1e-3)
    theta, mean, std, scale = closure_model(rng, m, f)
    ctx.mlp_load(theta, mean, std, scale)
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    nut = torch.empty(dm.n_gauss_total, dtype=torch.float32, device="cuda")
    dm.assemble(out, prec=prec, closure="mlp", scatter=scatter, nut_out=nut)
    ctx.sync_status()
    got = out.cpu().numpy().T
    mlp = O.MLPParams(gpu_rounded_theta(theta), mean.astype(np.float64), std.astype(np.float64), scale)
    om = O.OracleMesh.of(m)
    ref, nref = O.assemble_rhs(om, f.u, f.p, f.nu, f.c_vreman, "mlp", mlp=mlp, want_nut=True)
    ref_sgs = O.assemble_rhs(om, f.u, f.p, f.nu, f.c_vreman, "mlp", mask=O.TERM_SGS, mlp=mlp)
    nr = np.concatenate([nref[t].ravel() for t in range(4) if t in nref])
    ng = nut.cpu().numpy()
    assert np.all(np.abs(ng - nr) <= 3e-2 * np.abs(nr) + 2e-3 * np.abs(nr).max())
    err = np.linalg.norm(got - ref)
    assert err <= 3e-2 * np.linalg.norm(ref_sgs) + 2e-5 * np.linalg.norm(ref), (err, np.linalg.norm(ref_sgs))


def test_batched_assembly_with_mlp_closure(ctx):
    rng = np.random.default_rng(6)
    batch = mg.batch_meshes(count=4, seed=3, e_min=2e3, e_max=2e4)
    theta, mean, std, scale = closure_model(rng, *batch[0])
    ctx.mlp_load(theta, mean, std, scale)
    dms, outs = [], []
    for m, f in batch:
        dm = ctx.upload_mesh(m)
        dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
        dms.append(dm)
        outs.append(torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda"))
    ctx.assemble_batched(dms, outs, prec="mixed", closure="mlp")
    ctx.sync_status()
    single = torch.empty_like(outs[0])
    for dm, o in zip(dms, outs):
        single = torch.empty_like(o)
        dm.assemble(single, prec="mixed", closure="mlp", scatter="chunk")
        ctx.sync_status()
        a, b = o.cpu().numpy(), single.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


# ---------------------------------------------------------------------------
# Vreman as the network's fallback outside the training envelope

def oracle_gp_features(mesh, field):
    """Raw features of every Gauss point, per element type (E, ng, 6), from
    the oracle's geometry and feature functions."""
    out = {}
    for t, conn in mesh.conn.items():
        ng = O.NGAUSS[t]
        F = np.zeros((conn.shape[0], ng, 6))
        for e in range(conn.shape[0]):
            _, d, W, _ = O.element_geometry(t, mesh.xyz[conn[e]])
            U = field.u[conn[e]]
            delta = W.sum() ** (1.0 / 3.0)
            for g in range(ng):
                F[e, g] = O.mlp_features(U.T @ d[g], delta, field.nu)
        out[t] = F
    return out


def test_mlp_envelope_falls_back_to_vreman(ctx):
    rng = np.random.default_rng(8)
    m = mg.channel_mesh(nx=10, ny=12, nz=8, seed=21, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=5, nu=1e-3)
    theta, mean, std, scale = closure_model(rng, m, f)
    ctx.mlp_load(theta, mean, std, scale)
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    N, NG = dm.n_nodes, dm.n_gauss_total

    def run(closure):
        out = torch.empty((3, N), dtype=torch.float64, device="cuda")
        nut = torch.empty(NG, dtype=torch.float32, device="cuda")
        dm.assemble(out, prec="mixed", closure=closure, scatter="chunk", nut_out=nut)
        ctx.sync_status()
        return out.cpu().numpy(), nut.cpu().numpy()

    r_mlp, n_mlp = run("mlp")
    r_vre, n_vre = run("vreman")
    ctx.mlp_fallback_read(reset=True)
    # an envelope that holds everything changes nothing and counts nothing
    ctx.mlp_set_envelope(np.full(6, -1e30), np.full(6, 1e30))
    r, n = run("mlp")
    assert np.array_equal(r, r_mlp) and np.array_equal(n, n_mlp)
    assert ctx.mlp_fallback_read(reset=True) == 0
    # an empty envelope gives the Vreman assembly at every Gauss point (up
    # to FP32 rounding: the Vreman path's TET04 kernel works on coordinates
    # relative to the chunks of its own tables, whose origins differ from
    # the fused kernel's, hence 1e-5 and not bitwise)
    ctx.mlp_set_envelope(np.full(6, 1e30), np.full(6, -1e30))
    r, n = run("mlp")
    assert ctx.mlp_fallback_read(reset=True) == NG
    assert np.all(np.abs(n - n_vre) <= 1e-5 * np.abs(n_vre) + 1e-12)
    assert np.linalg.norm(r - r_vre) <= 1e-6 * np.linalg.norm(r_vre)
    # a partial envelope on the first feature: each point takes the network's
    # or Vreman's value according to its own (oracle) feature
    feats = oracle_gp_features(m, f)
    x0 = np.concatenate([feats[t][:, :, 0].ravel() for t in range(4) if t in feats])
    lo0, hi0 = np.quantile(x0, [0.15, 0.85])
    lo = np.full(6, -1e30)
    hi = np.full(6, 1e30)
    lo[0], hi[0] = lo0, hi0
    ctx.mlp_set_envelope(lo, hi)
    _, n = run("mlp")
    count = ctx.mlp_fallback_read(reset=True)
    inside = (x0 >= lo0) & (x0 <= hi0)
    clear = np.minimum(np.abs(x0 - lo0), np.abs(x0 - hi0)) > 1e-4 * np.abs(x0).max()
    assert abs(count - int((~inside).sum())) <= int((~clear).sum())
    a, b = clear & inside, clear & ~inside
    assert np.all(np.abs(n[a] - n_mlp[a]) <= 1e-6 * np.abs(n_mlp[a]) + 1e-12)
    assert np.all(np.abs(n[b] - n_vre[b]) <= 1e-5 * np.abs(n_vre[b]) + 1e-12)
    assert 0.2 * NG < count < 0.4 * NG
    ctx.mlp_set_envelope(None, None)
