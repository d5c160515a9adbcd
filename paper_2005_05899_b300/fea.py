"""Python binding of libfea (include/fea.h): argument marshalling only.

Every step of the assembly runs in the CUDA library; this module converts
torch tensors / numpy arrays to pointers, checks return codes and raises
FeaError with the library's message.  There is no CPU fallback: if the
shared library is missing or no CUDA device is usable, the calls fail.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfea.so")

OK, EINVAL, ENOMEM, ECUDA, EMESH, ENUMERIC, ETIMEOUT, ESTATE, ENOTFOUND = range(9)
STATUS_NAMES = ("OK", "EINVAL", "ENOMEM", "ECUDA", "EMESH", "ENUMERIC", "ETIMEOUT", "ESTATE", "ENOTFOUND")
TET04, PYR05, PEN06, HEX08 = 0, 1, 2, 3
NNODE = (4, 5, 6, 8)
NGAUSS = (4, 8, 6, 8)
PREC = {"fp64": 0, "mixed": 1}
CLOSURE = {"none": 0, "vreman": 1, "mlp": 2}
SCATTER = {"auto": 0, "atomic": 1, "chunk": 2, "colour": 3, "warp": 4}
TERM_CONV, TERM_VISC, TERM_SGS, TERM_PRES, TERM_ALL = 1, 2, 4, 8, 15

EXPORTED = (
    "fea_create", "fea_destroy", "fea_last_error", "fea_version", "fea_mesh_upload", "fea_mesh_info",
    "fea_lumped_mass", "fea_field_upload", "fea_assemble_rhs", "fea_assemble_rhs_batched", "fea_periodic_fold",
    "fea_rk_stage", "fea_rk_step_graph", "fea_state_download", "fea_get_plan", "fea_set_plan", "fea_autotune",
    "fea_sync_status", "fea_launch_count", "fea_profile_enable", "fea_profile_read", "fea_rk_stage_noalloc",
    "fea_mlp_load", "fea_mlp_get", "fea_mlp_forward", "fea_mlp_train_step", "fea_mlp_set_envelope",
    "fea_mlp_fallback_read", "fea_sfc_order", "fea_partition_sfc", "fea_interface_pack", "fea_interface_unpack",
    "fea_poisson_setup", "fea_poisson_solve", "fea_divergence", "fea_gradient", "fea_project",
    "fea_balance_update", "fea_set_model", "fea_wall_setup", "fea_wall_assemble", "fea_autotune_batched",
    "fea_colour_elements", "fea_set_wait_limit", "fea_fp32_peak",
)
MLP_NPARAM = 8833
NOALLOC_MAX_NODES = 262144


def mesh_desc(mesh):
    """fea_mesh_desc of a meshgen.Mesh-like object; returns (desc, the arrays
    it points to (keep them alive), elements per type)."""
    xyz = np.ascontiguousarray(np.asarray(mesh.xyz, dtype=np.float64).T)
    keep = [xyz]
    d = MeshDesc()
    d.n_nodes = xyz.shape[1]
    d.xyz = xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    n_elem = [0, 0, 0, 0]
    for t in range(4):
        c = mesh.conn.get(t)
        if c is not None and len(c):
            c = np.ascontiguousarray(c, dtype=np.int32)
            keep.append(c)
            d.conn[t] = c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            d.n_elem[t] = c.shape[0]
            n_elem[t] = c.shape[0]
        f = getattr(mesh, "fp64_flag", {}).get(t) if getattr(mesh, "fp64_flag", None) else None
        if f is not None and len(f):
            f = np.ascontiguousarray(f, dtype=np.uint8)
            keep.append(f)
            d.fp64_jac[t] = f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    if getattr(mesh, "periodic_master", None) is not None:
        pm = np.ascontiguousarray(mesh.periodic_master, dtype=np.int32)
        keep.append(pm)
        d.periodic_master = pm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    if getattr(mesh, "dirichlet", None) is not None:
        dm = np.ascontiguousarray(mesh.dirichlet, dtype=np.uint8)
        keep.append(dm)
        d.dirichlet = dm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    return d, keep, n_elem


def balance_update(Lambda_hist, times_hist) -> np.ndarray:
    """New correction coefficients from the history of cumulative coefficients
    Lambda [k][P+1] and measured per-part times [k][P] (host)."""
    L = np.ascontiguousarray(Lambda_hist, dtype=np.float64)
    T = np.ascontiguousarray(times_hist, dtype=np.float64)
    k, P = T.shape
    assert L.shape == (k, P + 1)
    out = np.zeros(P)
    st = lib().fea_balance_update(int(P), int(k), L.ctypes.data_as(ctypes.c_void_p), T.ctypes.data_as(ctypes.c_void_p),
                                  out.ctypes.data_as(ctypes.c_void_p))
    if st:
        raise FeaError(st, "fea_balance_update failed")
    return out


def sfc_order(xyz, level: int = 10) -> np.ndarray:
    """Hilbert-curve order of points xyz (N, 3) binned on a 2^level grid (host)."""
    x = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).T)
    n = x.shape[1]
    out = np.empty(n, np.int64)
    st = lib().fea_sfc_order(n, x.ctypes.data_as(ctypes.c_void_p), int(level), out.ctypes.data_as(ctypes.c_void_p))
    if st:
        raise FeaError(st, "fea_sfc_order failed")
    return out


def colour_elements(conn, n_nodes: int):
    """Greedy colouring of the elements conn (E, n_en) (host, no device):
    returns (colour per element (E,) int32, number of colours)."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    col = np.zeros(conn.shape[0], np.int32)
    nc = ctypes.c_int32(0)
    st = lib().fea_colour_elements(int(n_nodes), int(conn.shape[1]), int(conn.shape[0]), conn.ctypes.data,
                                   col.ctypes.data, ctypes.byref(nc))
    if st:
        raise FeaError(st, "fea_colour_elements failed")
    return col, nc.value

def partition_sfc(mesh, nparts: int, level: int = 10, lam=None) -> dict:
    """SFC partition of the elements: {etype: part id per element} (host);
    lam: optional correction coefficients [nparts] (target shares)."""
    d, keep, n_elem = mesh_desc(mesh)
    parts = {t: np.zeros(n_elem[t], np.int32) for t in range(4)}
    ptrs = (ctypes.c_void_p * 4)(*[parts[t].ctypes.data if n_elem[t] else None for t in range(4)])
    lam_a = None if lam is None else np.ascontiguousarray(lam, dtype=np.float64)
    st = lib().fea_partition_sfc(ctypes.byref(d), int(nparts), int(level),
                                 None if lam_a is None else lam_a.ctypes.data_as(ctypes.c_void_p), ptrs)
    if st:
        raise FeaError(st, "fea_partition_sfc failed")
    return {t: parts[t] for t in range(4) if n_elem[t]}


class FeaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"FEA_{name}: {msg}")
        self.status = status


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("n_elem", ctypes.c_int64 * 4), ("conn", ctypes.POINTER(ctypes.c_int32) * 4),
                ("periodic_master", ctypes.POINTER(ctypes.c_int32)), ("dirichlet", ctypes.POINTER(ctypes.c_uint8)),
                ("fp64_jac", ctypes.POINTER(ctypes.c_uint8) * 4)]


class WallDesc(ctypes.Structure):
    _fields_ = [("n_tri", ctypes.c_int64), ("tri", ctypes.c_void_p), ("tri_exch", ctypes.c_void_p),
                ("n_quad", ctypes.c_int64), ("quad", ctypes.c_void_p), ("quad_exch", ctypes.c_void_p),
                ("kappa", ctypes.c_double), ("c_plus", ctypes.c_double)]


class Plan(ctypes.Structure):
    _fields_ = [("scatter", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("chunk_elems", ctypes.c_int32), ("chunk_acc", ctypes.c_int32)]

    def as_dict(self):
        return {"scatter": self.scatter, "threads_per_block": self.threads_per_block,
                "chunk_elems": self.chunk_elems, "chunk_acc": self.chunk_acc}


_lib = None


def lib() -> ctypes.CDLL:
    """Loads libfea.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FeaError(ECUDA, f"{LIB_PATH} is missing: run paper_2005_05899_b300/build.py (no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
        L.fea_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp)]
        L.fea_destroy.argtypes = [vp]
        L.fea_destroy.restype = None
        L.fea_last_error.argtypes = [vp]
        L.fea_last_error.restype = ctypes.c_char_p
        L.fea_version.restype = ctypes.c_char_p
        L.fea_launch_count.argtypes = [vp]
        L.fea_launch_count.restype = i64
        L.fea_mesh_upload.argtypes = [vp, ctypes.POINTER(MeshDesc), vp, ctypes.POINTER(i32)]
        L.fea_mesh_info.argtypes = [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.fea_lumped_mass.argtypes = [vp, i32, vp, vp]
        L.fea_field_upload.argtypes = [vp, i32, vp, vp, ctypes.c_int, dbl, dbl, vp]
        L.fea_assemble_rhs.argtypes = [vp, i32, ctypes.c_int, ctypes.c_int, u32, ctypes.c_int, vp, vp, vp]
        L.fea_assemble_rhs_batched.argtypes = [vp, ctypes.POINTER(i32), i32, ctypes.c_int, ctypes.c_int, u32,
                                               ctypes.POINTER(vp), vp]
        L.fea_periodic_fold.argtypes = [vp, i32, vp, i32, vp]
        L.fea_rk_stage.argtypes = [vp, i32, i32, dbl, ctypes.c_int, ctypes.c_int, vp]
        L.fea_rk_step_graph.argtypes = [vp, i32, dbl, ctypes.c_int, ctypes.c_int, vp]
        L.fea_state_download.argtypes = [vp, i32, vp, vp]
        L.fea_get_plan.argtypes = [vp, i32, ctypes.POINTER(Plan)]
        L.fea_set_plan.argtypes = [vp, i32, ctypes.POINTER(Plan)]
        L.fea_autotune.argtypes = [vp, i32, ctypes.c_int, ctypes.c_int, ctypes.c_char_p]
        L.fea_sync_status.argtypes = [vp, vp]
        L.fea_set_wait_limit.argtypes = [vp, ctypes.c_uint32]
        L.fea_fp32_peak.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp]
        L.fea_profile_enable.argtypes = [vp, ctypes.c_int]
        L.fea_mlp_load.argtypes = [vp, vp, vp, vp, dbl, vp]
        L.fea_mlp_get.argtypes = [vp, vp, vp]
        L.fea_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
        L.fea_mlp_train_step.argtypes = [vp, vp, vp, i64, ctypes.c_float, vp, vp, vp]
        L.fea_mlp_set_envelope.argtypes = [vp, vp, vp, vp]
        L.fea_sfc_order.argtypes = [i64, vp, i32, vp]
        L.fea_colour_elements.argtypes = [i64, i32, i64, vp, vp, ctypes.POINTER(i32)]
        L.fea_poisson_setup.argtypes = [vp, i32, vp, vp]
        L.fea_poisson_solve.argtypes = [vp, i32, vp, dbl, vp, dbl, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl), vp]
        L.fea_divergence.argtypes = [vp, i32, vp, vp, vp]
        L.fea_gradient.argtypes = [vp, i32, vp, vp, vp]
        L.fea_project.argtypes = [vp, i32, dbl, dbl, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl), vp]
        L.fea_partition_sfc.argtypes = [ctypes.POINTER(MeshDesc), i32, i32, vp, ctypes.c_void_p * 4]
        L.fea_balance_update.argtypes = [i32, i32, vp, vp, vp]
        L.fea_set_model.argtypes = [vp, i32, i32, i32]
        L.fea_wall_setup.argtypes = [vp, i32, ctypes.POINTER(WallDesc)]
        L.fea_wall_assemble.argtypes = [vp, i32, vp, vp]
        L.fea_autotune_batched.argtypes = [vp, ctypes.POINTER(i32), i32, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(Plan)]
        L.fea_interface_pack.argtypes = [vp, vp, i64, vp, vp, i64, vp, i64, vp]
        L.fea_interface_unpack.argtypes = [vp, vp, i64, vp, vp, i64, vp, i64, vp]
        L.fea_mlp_fallback_read.argtypes = [vp, ctypes.POINTER(i64), ctypes.c_int]
        L.fea_rk_stage_noalloc.argtypes = [vp, i32, i32, dbl, ctypes.c_int, ctypes.c_int, dbl, dbl, vp, vp, vp, vp,
                                           vp]
        L.fea_profile_read.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(dbl), ctypes.POINTER(i64),
                                       ctypes.c_int]
        for name in EXPORTED:
            f = getattr(L, name)
            if f.restype is ctypes.c_int and name not in ("fea_destroy",):
                f.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(t) -> int:
    """Address of a torch tensor (any device) or a numpy array (host)."""
    if t is None:
        return 0
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return t.ctypes.data
    assert t.is_contiguous(), "tensor must be contiguous"
    return t.data_ptr()


def _on_device(t) -> bool:
    return bool(t.is_cuda)


_NP_DT = {"f64": np.float64, "f32": np.float32, "i64": np.int64}


def _buf(t, name: str, dtype: str, numel: int, device: bool = True, optional: bool = False):
    """Checks a buffer before its address goes to the C ABI, which cannot see
    its size: a contiguous torch tensor (a CUDA tensor where the entry point
    takes device memory) or, where host memory is allowed, also a numpy
    array, of the given element type ("f64", "f32", "i64") and exactly
    `numel` elements.  Raises ValueError, so that a wrong buffer never reaches
    a kernel."""
    if t is None:
        if optional:
            return
        raise ValueError(f"{name}: a buffer is required")
    if isinstance(t, np.ndarray):
        if device:
            raise ValueError(f"{name}: device memory required, got a numpy array")
        ok, contiguous, n = t.dtype == np.dtype(_NP_DT[dtype]), t.flags.c_contiguous, t.size
    else:
        import torch
        if device and not _on_device(t):
            raise ValueError(f"{name}: device memory required, got a tensor on {t.device}")
        want = {"f64": torch.float64, "f32": torch.float32, "i64": torch.int64}[dtype]
        ok, contiguous, n = t.dtype == want, t.is_contiguous(), t.numel()
    if not ok:
        raise ValueError(f"{name}: element type {dtype} required, got {t.dtype}")
    if not contiguous:
        raise ValueError(f"{name}: must be contiguous")
    if n != numel:
        raise ValueError(f"{name}: {numel} elements required, got {n}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _rows6(x) -> int:
    """Rows of a float32 device feature array [B][6]."""
    if getattr(x, "dim", lambda: -1)() != 2 or x.shape[1] != 6:
        raise ValueError("x: a [B][6] array of raw features required")
    B = int(x.shape[0])
    _buf(x, "x", "f32", 6 * B)
    return B


def _iface_check(v, loc, cls, packed, vname: str, pname: str):
    """Interface buffers: v [3][n] and the packed [3][n_class] float64, loc /
    cls int64 [m], all device; the sizes handed on are read from them."""
    for t, name in ((v, vname), (packed, pname)):
        if getattr(t, "dim", lambda: -1)() != 2 or t.shape[0] != 3:
            raise ValueError(f"{name}: a [3][n] array required")
        _buf(t, name, "f64", 3 * int(t.shape[1]))
    m = int(loc.numel()) if hasattr(loc, "numel") else -1
    _buf(loc, "loc", "i64", m)
    _buf(cls, "cls", "i64", m)


class Context:
    """One libfea context on one CUDA device."""

    def __init__(self, device: int = 0):
        self._lib = lib()
        h = ctypes.c_void_p()
        st = self._lib.fea_create(device, ctypes.byref(h))
        if st != OK:
            raise FeaError(st, f"fea_create(device={device}) failed (no usable CUDA device?)")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            self._lib.fea_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int):
        if st != OK:
            raise FeaError(st, self._lib.fea_last_error(self.handle).decode())

    @property
    def launch_count(self) -> int:
        return int(self._lib.fea_launch_count(self.handle))

    def profile(self, on: bool = True):
        self.check(self._lib.fea_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self, etype: int, fp64_jac: int = 0, reset: bool = False):
        """(summed kernel ms, launches) of one category since the last reset."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self.check(self._lib.fea_profile_read(self.handle, etype, fp64_jac, ctypes.byref(ms), ctypes.byref(n),
                                              1 if reset else 0))
        return ms.value, n.value

    # ---- learned closure ----
    def mlp_load(self, theta, feat_mean, feat_std, out_scale: float, stream=None):
        """theta [8833], feat_mean [6], feat_std [6]: float32 numpy (host) or torch tensors."""
        arrs = [np.ascontiguousarray(a, dtype=np.float32) if not hasattr(a, "data_ptr") else a
                for a in (theta, feat_mean, feat_std)]
        for a, name, n in zip(arrs, ("theta", "feat_mean", "feat_std"), (MLP_NPARAM, 6, 6)):
            _buf(a, name, "f32", n, device=False)
        self._mlp_keep = arrs
        self.check(self._lib.fea_mlp_load(self.handle, _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]),
                                          float(out_scale), _stream(stream)))

    # ---- interface exchange of a partitioned mesh ----
    def interface_pack(self, v, loc, cls, out, stream=None):
        """v: float64 device [3][n]; loc, cls: int64 device [m]; out: float64
        device [3][n_class] (zeroed, then the class sums of this part)."""
        _iface_check(v, loc, cls, out, "v", "out")
        self.check(self._lib.fea_interface_pack(self.handle, _ptr(v), int(v.shape[1]), _ptr(loc), _ptr(cls),
                                                int(loc.shape[0]), _ptr(out), int(out.shape[1]), _stream(stream)))
        return out

    def interface_unpack(self, buf, loc, cls, v, stream=None):
        """v[:, loc[k]] = buf[:, cls[k]] (all device)."""
        _iface_check(v, loc, cls, buf, "v", "buf")
        self.check(self._lib.fea_interface_unpack(self.handle, _ptr(buf), int(buf.shape[1]), _ptr(loc), _ptr(cls),
                                                  int(loc.shape[0]), _ptr(v), int(v.shape[1]), _stream(stream)))
        return v

    def mlp_set_envelope(self, lo=None, hi=None, stream=None):
        """Raw-feature bounds lo [6], hi [6] (None, None: no envelope); outside
        them the fused closure uses Vreman's nu_t."""
        if (lo is None) != (hi is None):
            raise ValueError("give both bounds or neither")
        if lo is None:
            self.check(self._lib.fea_mlp_set_envelope(self.handle, None, None, _stream(stream)))
            return
        a = np.ascontiguousarray(lo, dtype=np.float32)
        b = np.ascontiguousarray(hi, dtype=np.float32)
        self.check(self._lib.fea_mlp_set_envelope(self.handle, _ptr(a), _ptr(b), _stream(stream)))

    def mlp_fallback_read(self, reset: bool = False) -> int:
        """Gauss-point evaluations that fell back to Vreman since load / last reset."""
        n = ctypes.c_int64()
        self.check(self._lib.fea_mlp_fallback_read(self.handle, ctypes.byref(n), 1 if reset else 0))
        return n.value

    def mlp_get(self) -> np.ndarray:
        out = np.zeros(MLP_NPARAM, np.float32)
        self.check(self._lib.fea_mlp_get(self.handle, _ptr(out), _stream(None)))
        import torch
        torch.cuda.current_stream().synchronize()
        return out

    def mlp_forward(self, x, out, stream=None):
        """x: float32 device tensor [B][6] of raw features; out: float32 device [B]."""
        B = _rows6(x)
        _buf(out, "out", "f32", B)
        self.check(self._lib.fea_mlp_forward(self.handle, _ptr(x), int(x.shape[0]), _ptr(out), _stream(stream)))
        return out

    def mlp_train_step(self, x, y, lr: float, loss_out=None, grad_out=None, stream=None):
        """x: float32 device [B][6]; y: float32 device [B]; loss_out (1) and
        grad_out (MLP_NPARAM): optional float32, host or device."""
        B = _rows6(x)
        _buf(y, "y", "f32", B)
        _buf(loss_out, "loss_out", "f32", 1, device=False, optional=True)
        _buf(grad_out, "grad_out", "f32", MLP_NPARAM, device=False, optional=True)
        self.check(self._lib.fea_mlp_train_step(self.handle, _ptr(x), _ptr(y), int(x.shape[0]), float(lr),
                                                _ptr(loss_out), _ptr(grad_out), _stream(stream)))

    def sync_status(self, stream=None):
        self.check(self._lib.fea_sync_status(self.handle, _stream(stream)))

    def fp32_peak(self, stream=None):
        """Measured FP32 peak (TFLOP/s) as (scalar FFMA, paired FFMA2)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self.check(self._lib.fea_fp32_peak(self.handle, ctypes.byref(a), ctypes.byref(b), _stream(stream)))
        return a.value, b.value

    def set_wait_limit(self, polls: int):
        """Poll limit of the TET04 kernel's bounded device waits (0: default)."""
        if not 0 <= int(polls) < 2 ** 32:
            raise ValueError("polls must fit in 32 bits")
        self.check(self._lib.fea_set_wait_limit(self.handle, int(polls)))

    def upload_mesh(self, mesh, stream=None) -> "DeviceMesh":
        """mesh: meshgen.Mesh-like object (xyz (N,3), conn dict, optional
        periodic_master, dirichlet, fp64_flag).  Host arrays only."""
        d, keep, n_elem = mesh_desc(mesh)
        xyz = keep[0]
        mid = ctypes.c_int32(-1)
        self.check(self._lib.fea_mesh_upload(self.handle, ctypes.byref(d), _stream(stream), ctypes.byref(mid)))
        return DeviceMesh(self, mid.value, xyz.shape[1], n_elem)

    def assemble_batched(self, meshes: Sequence["DeviceMesh"], outs, prec="mixed", closure="vreman",
                         mask=TERM_ALL, stream=None):
        n = len(meshes)
        if len(outs) != n:
            raise ValueError(f"{n} meshes but {len(outs)} output buffers")
        for k, (m, o) in enumerate(zip(meshes, outs)):
            _buf(o, f"outs[{k}]", "f64", 3 * m.n_nodes)
        ids = (ctypes.c_int32 * n)(*[m.id for m in meshes])
        ptrs = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
        self.check(self._lib.fea_assemble_rhs_batched(self.handle, ids, n, PREC[prec], CLOSURE[closure], mask,
                                                      ptrs, _stream(stream)))


    def autotune_batched(self, meshes: Sequence["DeviceMesh"], prec="mixed", closure="vreman") -> Plan:
        """Chooses between the persistent batched launch (chunk size) and
        per-mesh launches (atomic / warp / colour) for assemble_batched."""
        n = len(meshes)
        ids = (ctypes.c_int32 * n)(*[m.id for m in meshes])
        p = Plan()
        self.check(self._lib.fea_autotune_batched(self.handle, ids, n, PREC[prec], CLOSURE[closure], ctypes.byref(p)))
        return p


class DeviceMesh:
    def __init__(self, ctx: Context, mid: int, n_nodes: int, n_elem):
        self.ctx = ctx
        self.id = mid
        self.n_nodes = n_nodes
        self.n_elem = list(n_elem)

    @property
    def n_elem_total(self) -> int:
        return sum(self.n_elem)

    @property
    def n_gauss_total(self) -> int:
        return sum(e * g for e, g in zip(self.n_elem, NGAUSS))

    def _L(self):
        return self.ctx._lib

    def upload_field(self, u, p, nu: float, c_vreman: float = 0.07, stream=None):
        """u: [3][n] (or (n,3) numpy, transposed here), p: [n]; float64 or float32;
        torch tensor (any device) or numpy (host)."""
        if isinstance(u, np.ndarray) and u.ndim == 2 and u.shape == (self.n_nodes, 3):
            u = np.ascontiguousarray(u.T)
        dtype = 0
        if isinstance(u, np.ndarray):
            u = np.ascontiguousarray(u, dtype=np.float32 if u.dtype == np.float32 else np.float64)
            p = np.ascontiguousarray(p, dtype=u.dtype)
            dtype = 0 if u.dtype == np.float64 else 1
        else:
            import torch
            if u.dtype not in (torch.float64, torch.float32):
                raise ValueError(f"u: float64 or float32 required, got {u.dtype}")
            dtype = 0 if u.dtype == torch.float64 else 1
        kind = "f64" if dtype == 0 else "f32"
        _buf(u, "u", kind, 3 * self.n_nodes, device=False)
        _buf(p, "p", kind, self.n_nodes, device=False)
        self._keep = (u, p)
        self.ctx.check(self._L().fea_field_upload(self.ctx.handle, self.id, _ptr(u), _ptr(p), dtype, float(nu),
                                                  float(c_vreman), _stream(stream)))

    def assemble(self, out, prec="mixed", closure="vreman", mask=TERM_ALL, scatter="auto", nut_out=None,
                 stream=None):
        """out: float64 device tensor [3][n] (overwritten); nut_out: optional
        float32 device tensor [n_gauss_total]."""
        _buf(out, "out", "f64", 3 * self.n_nodes)
        _buf(nut_out, "nut_out", "f32", self.n_gauss_total, optional=True)
        self.ctx.check(self._L().fea_assemble_rhs(self.ctx.handle, self.id, PREC[prec], CLOSURE[closure], mask,
                                                  SCATTER[scatter], _ptr(out), _ptr(nut_out), _stream(stream)))
        return out

    def lumped_mass(self, out, stream=None):
        _buf(out, "out", "f64", self.n_nodes)
        self.ctx.check(self._L().fea_lumped_mass(self.ctx.handle, self.id, _ptr(out), _stream(stream)))
        return out

    def fold(self, v, stream=None):
        ncomp = 1 if v.dim() == 1 else v.shape[0]
        _buf(v, "v", "f64", ncomp * self.n_nodes)
        self.ctx.check(self._L().fea_periodic_fold(self.ctx.handle, self.id, _ptr(v), ncomp, _stream(stream)))
        return v

    def set_model(self, conv="gu", delta="volume"):
        """Convective form "gu" | "emac"; Vreman filter width "volume" | "axes"."""
        self.ctx.check(self._L().fea_set_model(self.ctx.handle, self.id, {"gu": 0, "emac": 1}[conv],
                                               {"volume": 0, "axes": 1}[delta]))

    # ---- boundary assembly: wall model ----
    def wall_setup(self, tri=None, tri_exch=None, quad=None, quad_exch=None, kappa=0.41, c_plus=7.8):
        """Wall-model faces (host int arrays (F, 3) / (F, 4) of node ids and their
        exchange nodes, normals out of the fluid); no faces clears them."""
        keep = []

        def arr(a, nv):
            if a is None or len(a) == 0:
                return 0, None
            a = np.ascontiguousarray(a, dtype=np.int32)
            assert a.ndim == 2 and a.shape[1] == nv
            keep.append(a)
            return a.shape[0], a.ctypes.data

        d = WallDesc()
        d.n_tri, d.tri = arr(tri, 3)
        n2, d.tri_exch = arr(tri_exch, 3)
        d.n_quad, d.quad = arr(quad, 4)
        n4, d.quad_exch = arr(quad_exch, 4)
        assert n2 == d.n_tri and n4 == d.n_quad, "faces and exchange nodes differ in length"
        d.kappa, d.c_plus = float(kappa), float(c_plus)
        self.ctx.check(self._L().fea_wall_setup(self.ctx.handle, self.id, ctypes.byref(d)))

    def wall_assemble(self, rhs, stream=None):
        """rhs [3][n] (device float64) += the wall-model term at the current field."""
        _buf(rhs, "rhs", "f64", 3 * self.n_nodes)
        self.ctx.check(self._L().fea_wall_assemble(self.ctx.handle, self.id, _ptr(rhs), _stream(stream)))
        return rhs

    # ---- pressure projection ----
    def poisson_setup(self, pinned=None, stream=None):
        """Laplacian over periodic classes; pinned: optional host bool/uint8 [n]."""
        pin = None if pinned is None else np.ascontiguousarray(pinned, dtype=np.uint8)
        self.ctx.check(self._L().fea_poisson_setup(self.ctx.handle, self.id, _ptr(pin), _stream(stream)))

    def poisson_solve(self, b, x, scale=1.0, rtol=1e-10, max_iter=2000, stream=None):
        """K x = scale fold(b) (device float64 [n]); x: initial guess / solution.
        Returns (iterations, ||r|| / ||b||)."""
        _buf(b, "b", "f64", self.n_nodes)
        _buf(x, "x", "f64", self.n_nodes)
        it, rr = ctypes.c_int32(0), ctypes.c_double(0.0)
        self.ctx.check(self._L().fea_poisson_solve(self.ctx.handle, self.id, _ptr(b), float(scale), _ptr(x),
                                                   float(rtol), int(max_iter), ctypes.byref(it), ctypes.byref(rr),
                                                   _stream(stream)))
        return it.value, rr.value

    def divergence(self, u, out, stream=None):
        _buf(u, "u", "f64", 3 * self.n_nodes)
        _buf(out, "out", "f64", self.n_nodes)
        self.ctx.check(self._L().fea_divergence(self.ctx.handle, self.id, _ptr(u), _ptr(out), _stream(stream)))
        return out

    def gradient(self, p, out, stream=None):
        _buf(p, "p", "f64", self.n_nodes)
        _buf(out, "out", "f64", 3 * self.n_nodes)
        self.ctx.check(self._L().fea_gradient(self.ctx.handle, self.id, _ptr(p), _ptr(out), _stream(stream)))
        return out

    def project(self, dt: float, rtol=1e-10, max_iter=2000, stream=None):
        """Projection step on the state; returns (iterations, ||r|| / ||b||)."""
        it, rr = ctypes.c_int32(0), ctypes.c_double(0.0)
        self.ctx.check(self._L().fea_project(self.ctx.handle, self.id, float(dt), float(rtol), int(max_iter),
                                             ctypes.byref(it), ctypes.byref(rr), _stream(stream)))
        return it.value, rr.value

    def rk_stage(self, stage: int, dt: float, prec="mixed", closure="vreman", stream=None):
        self.ctx.check(self._L().fea_rk_stage(self.ctx.handle, self.id, stage, float(dt), PREC[prec],
                                              CLOSURE[closure], _stream(stream)))

    def rk_stage_noalloc(self, stage: int, dt: float, un, uk, p, out, nu: float, c_vreman: float = 0.07,
                         prec="mixed", closure="vreman", stream=None):
        """One RK stage from caller arrays (device, [3][n] / [n] FP64) into `out`,
        through the entry point that allocates nothing (static device scratch)."""
        for t, name in ((un, "un"), (uk, "uk"), (out, "out")):
            _buf(t, name, "f64", 3 * self.n_nodes)
        _buf(p, "p", "f64", self.n_nodes)
        self.ctx.check(self._L().fea_rk_stage_noalloc(self.ctx.handle, self.id, stage, float(dt), PREC[prec],
                                                      CLOSURE[closure], float(nu), float(c_vreman), _ptr(un),
                                                      _ptr(uk), _ptr(p), _ptr(out), _stream(stream)))
        return out

    def rk_step_graph(self, dt: float, prec="mixed", closure="vreman", stream=None):
        self.ctx.check(self._L().fea_rk_step_graph(self.ctx.handle, self.id, float(dt), PREC[prec],
                                                   CLOSURE[closure], _stream(stream)))

    def state(self, out, stream=None):
        """out: float64 [3][n], host (numpy, pinned or pageable torch) or device."""
        _buf(out, "out", "f64", 3 * self.n_nodes, device=False)
        self.ctx.check(self._L().fea_state_download(self.ctx.handle, self.id, _ptr(out), _stream(stream)))
        return out

    def get_plan(self) -> Plan:
        p = Plan()
        self.ctx.check(self._L().fea_get_plan(self.ctx.handle, self.id, ctypes.byref(p)))
        return p

    def set_plan(self, scatter="chunk", threads_per_block=256, chunk_elems=512, chunk_acc=0):
        p = Plan(SCATTER[scatter], threads_per_block, chunk_elems, chunk_acc)
        self.ctx.check(self._L().fea_set_plan(self.ctx.handle, self.id, ctypes.byref(p)))

    def autotune(self, prec="mixed", closure="vreman", cache_path: Optional[str] = None):
        self.ctx.check(self._L().fea_autotune(self.ctx.handle, self.id, PREC[prec], CLOSURE[closure],
                                              cache_path.encode() if cache_path else None))
        return self.get_plan()
