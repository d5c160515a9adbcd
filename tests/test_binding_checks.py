"""The Python binding's buffer checks, on the CPU.

The C ABI sees only addresses, so the binding checks every buffer's element
type, size, contiguity and (where the entry point takes device memory) its
device before the call.  Here the library is a stub that records the calls,
and CPU tensors stand in for device tensors: well-formed buffers reach the
stub, wrong ones raise ValueError and never reach it.
"""
import numpy as np
import pytest
import torch

from paper_2005_05899_b300 import fea

N = 7
N_ELEM = [2, 0, 1, 0]          # TET04 x 2, PEN06 x 1
N_GAUSS = 2 * 4 + 6


class StubLib:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if not name.startswith("fea_"):
            raise AttributeError(name)

        def f(*args):
            self.calls.append(name)
            return 0
        return f


@pytest.fixture
def env(monkeypatch):
    monkeypatch.setattr(fea, "_on_device", lambda t: True)     # CPU tensors stand in for CUDA ones
    monkeypatch.setattr(fea, "_stream", lambda s: 0)
    ctx = fea.Context.__new__(fea.Context)
    ctx._lib = StubLib()
    ctx.handle = None
    dm = fea.DeviceMesh(ctx, 0, N, N_ELEM)
    yield ctx, dm
    ctx.handle = None


def f64(*shape):
    return torch.zeros(shape, dtype=torch.float64)


def f32(*shape):
    return torch.zeros(shape, dtype=torch.float32)


def test_well_formed_buffers_reach_the_library(env):
    ctx, dm = env
    dm.upload_field(np.zeros((N, 3)), np.zeros(N), 0.1)
    dm.upload_field(f32(3, N), f32(N), 0.1)
    dm.assemble(f64(3, N))
    dm.assemble(f64(3, N), nut_out=f32(N_GAUSS))
    dm.lumped_mass(f64(N))
    dm.fold(f64(N))
    dm.fold(f64(2, N))
    dm.wall_assemble(f64(3, N))
    dm.poisson_solve(f64(N), f64(N))
    dm.divergence(f64(3, N), f64(N))
    dm.gradient(f64(N), f64(3, N))
    dm.rk_stage_noalloc(0, 1e-3, f64(3, N), f64(3, N), f64(N), f64(3, N), 0.1)
    dm.state(f64(3, N))
    dm.state(np.zeros((3, N)))                     # host memory is allowed here
    ctx.assemble_batched([dm, dm], [f64(3, N), f64(3, N)])
    ctx.mlp_load(np.zeros(fea.MLP_NPARAM, np.float32), np.zeros(6), np.ones(6), 1.0)
    ctx.mlp_forward(f32(5, 6), f32(5))
    ctx.mlp_forward(f32(0, 6), f32(0))
    ctx.mlp_train_step(f32(5, 6), f32(5), 1e-3, loss_out=f32(1), grad_out=np.zeros(fea.MLP_NPARAM, np.float32))
    loc = torch.zeros(3, dtype=torch.int64)
    ctx.interface_pack(f64(3, N), loc, loc, f64(3, 2))
    ctx.interface_unpack(f64(3, 2), loc, loc, f64(3, N))
    assert len(ctx._lib.calls) == 21


@pytest.mark.parametrize("call", [
    lambda ctx, dm: dm.assemble(f32(3, N)),                              # element type
    lambda ctx, dm: dm.assemble(f64(3, N + 1)),                          # size
    lambda ctx, dm: dm.assemble(f64(N, 3).t()),                          # not contiguous
    lambda ctx, dm: dm.assemble(np.zeros((3, N))),                       # host memory for a device output
    lambda ctx, dm: dm.assemble(f64(3, N), nut_out=f32(N_GAUSS - 1)),
    lambda ctx, dm: dm.assemble(f64(3, N), nut_out=f64(N_GAUSS)),
    lambda ctx, dm: dm.lumped_mass(f64(3, N)),
    lambda ctx, dm: dm.fold(f64(2, N - 1)),
    lambda ctx, dm: dm.wall_assemble(f64(N)),
    lambda ctx, dm: dm.poisson_solve(f64(N), f64(N + 1)),
    lambda ctx, dm: dm.divergence(f64(N), f64(N)),
    lambda ctx, dm: dm.gradient(f64(N), f64(N)),
    lambda ctx, dm: dm.rk_stage_noalloc(0, 1e-3, f64(3, N), f64(3, N), f64(3, N), f64(3, N), 0.1),
    lambda ctx, dm: dm.state(f32(3, N)),
    lambda ctx, dm: dm.upload_field(f64(3, N), f32(N), 0.1),            # p's type differs from u's
    lambda ctx, dm: dm.upload_field(f64(3, N - 1), f64(N - 1), 0.1),
    lambda ctx, dm: dm.upload_field(torch.zeros((3, N), dtype=torch.int32), f64(N), 0.1),
    lambda ctx, dm: ctx.assemble_batched([dm, dm], [f64(3, N)]),
    lambda ctx, dm: ctx.assemble_batched([dm], [f64(3, N - 1)]),
    lambda ctx, dm: ctx.mlp_load(np.zeros(10, np.float32), np.zeros(6), np.ones(6), 1.0),
    lambda ctx, dm: ctx.mlp_forward(f32(5, 5), f32(5)),
    lambda ctx, dm: ctx.mlp_forward(f32(5, 6), f32(4)),
    lambda ctx, dm: ctx.mlp_train_step(f32(5, 6), f32(5), 1e-3, grad_out=f32(10)),
    lambda ctx, dm: ctx.interface_pack(f64(3, N), torch.zeros(3, dtype=torch.int64),
                                       torch.zeros(2, dtype=torch.int64), f64(3, 2)),
    lambda ctx, dm: ctx.interface_pack(f64(2, N), torch.zeros(3, dtype=torch.int64),
                                       torch.zeros(3, dtype=torch.int64), f64(3, 2)),
    lambda ctx, dm: ctx.interface_unpack(f64(3, 2), torch.zeros(3, dtype=torch.int32),
                                         torch.zeros(3, dtype=torch.int32), f64(3, N)),
])
def test_wrong_buffers_are_rejected_before_the_call(env, call):
    ctx, dm = env
    with pytest.raises(ValueError):
        call(ctx, dm)
    assert ctx._lib.calls == []


def test_device_memory_is_required_where_the_entry_point_takes_it(env, monkeypatch):
    ctx, dm = env
    monkeypatch.setattr(fea, "_on_device", lambda t: False)
    with pytest.raises(ValueError, match="device memory"):
        dm.assemble(f64(3, N))
    dm.state(f64(3, N))                   # host or device
    dm.upload_field(f64(3, N), f64(N), 0.1)
    assert ctx._lib.calls == ["fea_state_download", "fea_field_upload"]
