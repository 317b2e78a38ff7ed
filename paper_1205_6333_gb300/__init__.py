"""GB300-native leading-order Stokesian dynamics (Kopp & Hoefling, arXiv:1205.6333).

Python binding of the C ABI in include/sd.h.  Every step of the computation
runs in the CUDA kernels of libsd_gb300.so; this module only marshals
arguments (numpy arrays and torch tensors -> pointers, torch's current stream
and caching allocator -> the handle's stream and allocator callbacks).

Two layers:
  * the C names (``sd_create``, ``sd_set_positions``, ``sd_mobility_apply``,
    ``sd_step``, ``sd_step_batched``, ``sd_adjoint``, ...), taking the same
    arguments as in C (pointers as ints) and raising SDError on a non-OK status;
  * ``System`` and ``Batch``, which accept numpy arrays (host memory) or torch
    tensors (CUDA tensors are passed as device pointers, no copy).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L
from ._lib import (SD_TENSOR_RPY, SD_TENSOR_RP, SD_TENSOR_OSEEN, SD_PREC_FP32C, SD_PREC_FP64, SD_PREC_FP32,
                   SD_DTYPE_F32, SD_DTYPE_F64, SD_KERNEL_DENSE, SD_KERNEL_EPILOGUE, SD_KERNEL_CELLS,
                   SD_KERNEL_FORCES, SD_KERNEL_BATCHED, SD_KERNEL_VJP, SD_KERNEL_NEAR, sd_config)

TENSORS = {"rpy": SD_TENSOR_RPY, "rp": SD_TENSOR_RP, "oseen": SD_TENSOR_OSEEN}
PRECISIONS = {"fp32c": SD_PREC_FP32C, "fp64": SD_PREC_FP64, "fp32": SD_PREC_FP32}
DENSE_KERNELS = {"auto": L.SD_DENSE_AUTO, "directed": L.SD_DENSE_DIRECTED, "symmetric": L.SD_DENSE_SYMMETRIC}


class SDError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.status_name = L.STATUS_NAMES[status] if 0 <= status < len(L.STATUS_NAMES) else str(status)
        super().__init__("%s: %s (%s)" % (where, self.status_name, message))


def _check(st: int, where: str):
    if st != 0:
        raise SDError(st, where, L.load().sd_last_error().decode())


def lib():
    return L.load()


# ---------------------------------------------------------------- C names

def sd_config_init() -> sd_config:
    cfg = sd_config()
    lib().sd_config_init(ctypes.byref(cfg))
    return cfg


def sd_create(cfg: sd_config) -> int:
    h = ctypes.c_void_p()
    _check(lib().sd_create(ctypes.byref(cfg), ctypes.byref(h)), "sd_create")
    return h.value


def sd_destroy(h: int):
    lib().sd_destroy(h)


def sd_set_positions(h, xyz_ptr, on_device):
    _check(lib().sd_set_positions(h, xyz_ptr, on_device), "sd_set_positions")


def sd_get_positions(h, xyz_ptr, on_device):
    _check(lib().sd_get_positions(h, xyz_ptr, on_device), "sd_get_positions")


def sd_set_forces(h, f_ptr, on_device):
    _check(lib().sd_set_forces(h, f_ptr, on_device), "sd_set_forces")


def sd_mobility_apply(h, F_ptr, V_ptr, dtype, on_device):
    _check(lib().sd_mobility_apply(h, F_ptr, V_ptr, dtype, on_device), "sd_mobility_apply")


def sd_step(h, dt, nsteps):
    _check(lib().sd_step(h, float(dt), int(nsteps)), "sd_step")


def sd_mobility_apply_rows(h, F_ptr, V_ptr, dtype, on_device, row0, row1):
    _check(lib().sd_mobility_apply_rows(h, F_ptr, V_ptr, int(dtype), int(on_device), int(row0), int(row1)),
           "sd_mobility_apply_rows")


def sd_step_rows(h, dt, row0, row1):
    _check(lib().sd_step_rows(h, float(dt), int(row0), int(row1)), "sd_step_rows")


def sd_mobility_apply_part(h, F_ptr, dtype, on_device, shard, nshards, P_ptr):
    _check(lib().sd_mobility_apply_part(h, F_ptr, int(dtype), int(on_device), int(shard), int(nshards), P_ptr),
           "sd_mobility_apply_part")


def sd_mobility_apply_combine(h, Pall_ptr, nparts, V_ptr, dtype, on_device):
    _check(lib().sd_mobility_apply_combine(h, Pall_ptr, int(nparts), V_ptr, int(dtype), int(on_device)),
           "sd_mobility_apply_combine")


def sd_step_part(h, shard, nshards, P_ptr):
    _check(lib().sd_step_part(h, int(shard), int(nshards), P_ptr), "sd_step_part")


def sd_step_combine(h, dt, Pall_ptr, nparts):
    _check(lib().sd_step_combine(h, float(dt), Pall_ptr, int(nparts)), "sd_step_combine")


def sd_synchronize(h):
    _check(lib().sd_synchronize(h), "sd_synchronize")


def sd_mobility_vjp(h, F_ptr, W_ptr, gX_ptr, gF_ptr, dtype, on_device):
    _check(lib().sd_mobility_vjp(h, F_ptr, W_ptr, gX_ptr, gF_ptr, dtype, on_device), "sd_mobility_vjp")


def sd_adjoint(h, dt, nsteps, ckpt_every, gxT_ptr, gx0_ptr, gF_ptr, on_device):
    _check(lib().sd_adjoint(h, float(dt), int(nsteps), int(ckpt_every), gxT_ptr, gx0_ptr, gF_ptr, on_device),
           "sd_adjoint")


def sd_batch_create(cfg: sd_config, offsets) -> int:
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    b = ctypes.c_void_p()
    _check(lib().sd_batch_create(ctypes.byref(cfg), off.ctypes.data, off.size - 1, ctypes.byref(b)),
           "sd_batch_create")
    return b.value


def sd_batch_destroy(b):
    lib().sd_batch_destroy(b)


def sd_batch_set_positions(b, ptr, on_device):
    _check(lib().sd_batch_set_positions(b, ptr, on_device), "sd_batch_set_positions")


def sd_batch_get_positions(b, ptr, on_device):
    _check(lib().sd_batch_get_positions(b, ptr, on_device), "sd_batch_get_positions")


def sd_batch_set_forces(b, ptr, on_device):
    _check(lib().sd_batch_set_forces(b, ptr, on_device), "sd_batch_set_forces")


def sd_step_batched(b, dt, nsteps):
    _check(lib().sd_step_batched(b, float(dt), int(nsteps)), "sd_step_batched")


def sd_batch_autotune(b) -> int:
    c = ctypes.c_int32(-1)
    _check(lib().sd_batch_autotune(b, ctypes.byref(c)), "sd_batch_autotune")
    return c.value


def sd_mobility_apply_noalloc(x_ptr, F_ptr, V_ptr, n, a=1.0, eta=1.0, tensor="rpy", stream=None):
    """V = mu(x) F without any GPU allocation (device pointers only; see include/sd.h).
    For callers that must not allocate, e.g. while a CUDA graph is being captured."""
    t = TENSORS[tensor] if isinstance(tensor, str) else int(tensor)
    _check(lib().sd_mobility_apply_noalloc(x_ptr, F_ptr, V_ptr, int(n), float(a), float(eta), t, stream),
           "sd_mobility_apply_noalloc")


ACCESS_ALGOS = {"naive": 0, "tiling": 1, "smalltiling": 2, "bulk": 3}
ACCESS_MAPS = {"linear": 0, "strided": 1, "unordered": 2}


def sd_access_run(algo, map, vec4, n, block, in_ptr, out_ptr, stream=None):
    """One kernel of the App. A memory-access study (device pointers; see include/sd.h)."""
    a = ACCESS_ALGOS[algo] if isinstance(algo, str) else int(algo)
    m = ACCESS_MAPS[map] if isinstance(map, str) else int(map)
    _check(lib().sd_access_run(a, m, int(bool(vec4)), int(n), int(block), in_ptr, out_ptr, stream),
           "sd_access_run")


def sd_access_status():
    _check(lib().sd_access_status(), "sd_access_status")


def access_study(algo, map, data, block=128, out=None):
    """Run one study kernel on a CUDA float32 tensor of shape (n,) (float) or (n, 4)
    (float4) on torch's current stream; returns the output tensor (same shape)."""
    import torch
    if not (_is_torch(data) and data.is_cuda and data.dtype == torch.float32 and data.is_contiguous()):
        raise TypeError("access_study needs a contiguous CUDA float32 tensor")
    if data.dim() == 2 and data.shape[1] == 4:
        vec4 = True
    elif data.dim() == 1:
        vec4 = False
    else:
        raise ValueError("data must have shape (n,) or (n, 4)")
    if out is None:
        out = torch.empty_like(data)
    elif out.shape != data.shape or out.dtype != data.dtype or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must match data")
    st = torch.cuda.current_stream(data.device).cuda_stream
    sd_access_run(algo, map, vec4, data.shape[0], block, data.data_ptr(), out.data_ptr(), st)
    return out


def sd_last_error() -> str:
    return lib().sd_last_error().decode()


def sd_version() -> str:
    return lib().sd_version().decode()


# ---------------------------------------------------------------- array helpers

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _as_arg(x, dtype, asynchronous=False):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor of n x 3 values.
    With `asynchronous`, a page-locked CPU tensor is passed as on_device = 2 (copied
    on the stream without a host synchronisation)."""
    if _is_torch(x):
        import torch
        want = torch.float64 if dtype == np.float64 else torch.float32
        t = x.detach()
        if t.dtype != want or not t.is_contiguous():
            if asynchronous:
                raise ValueError("an asynchronous copy needs a contiguous tensor of the right dtype")
            t = t.to(want).contiguous()
        if t.is_cuda:
            return t.data_ptr(), 1, t
        return t.data_ptr(), 2 if (asynchronous and t.is_pinned()) else 0, t
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    return a.ctypes.data, 0, a


def _out_like(x, n, dtype):
    if _is_torch(x):
        import torch
        want = torch.float64 if dtype == np.float64 else torch.float32
        t = torch.empty((n, 3), dtype=want, device=x.device)
        return t.data_ptr(), int(t.is_cuda), t
    a = np.empty((n, 3), dtype=dtype)
    return a.ctypes.data, 0, a


def _dtype_of(x):
    if _is_torch(x):
        import torch
        return np.float32 if x.dtype == torch.float32 else np.float64
    return np.float32 if np.asarray(x).dtype == np.float32 else np.float64


def _torch_allocator(device: int):
    """Allocator callbacks backed by torch's CUDA caching allocator."""
    import torch

    def _alloc(nbytes, ctx):
        try:
            s = torch.cuda.current_stream(device)
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, s)
        except Exception:
            return None

    def _free(ptr, ctx):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    return L.ALLOC_FN(_alloc), L.FREE_FN(_free)


def _make_config(n=0, a=1.0, eta=1.0, tensor="rpy", prec="fp32c", r_near=None, rep_eps=0.0, rep_rc=None,
                 gravity=(0.0, 0.0, 0.0), device=0, stream=None, torch_allocator=False, dense="auto",
                 lubrication=False, box=None, verlet_skin=None):
    cfg = sd_config_init()
    cfg.verlet_skin = 0.5 * float(a) if verlet_skin is None else float(verlet_skin)
    cfg.lubrication = int(bool(lubrication))
    if box is not None:
        for d in range(3):
            cfg.box[d] = float(box[d])
    cfg.dense_kernel = DENSE_KERNELS[dense] if isinstance(dense, str) else int(dense)
    cfg.n = int(n)
    cfg.a = float(a)
    cfg.eta = float(eta)
    cfg.tensor = TENSORS[tensor] if isinstance(tensor, str) else int(tensor)
    cfg.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    cfg.r_near = float(r_near) if r_near else 2.5 * float(a)
    cfg.rep_eps = float(rep_eps)
    cfg.rep_rc = float(rep_rc) if rep_rc else 2.5 * float(a)
    for d in range(3):
        cfg.gravity[d] = float(gravity[d])
    cfg.device = int(device)
    keep = ()
    if stream == "torch":
        import torch
        cfg.stream = torch.cuda.current_stream(device).cuda_stream
    elif stream is not None:
        cfg.stream = int(stream)
    if torch_allocator:
        fa, ff = _torch_allocator(int(device))
        cfg.alloc, cfg.free = fa, ff
        keep = (fa, ff)
    return cfg, keep


# ---------------------------------------------------------------- System

class System:
    """A system of n spheres: positions (FP64 state), per-particle forces, and the
    all-pairs mobility on the GPU.  Arrays are n x 3; numpy arrays are host
    memory, CUDA torch tensors device memory."""

    def __init__(self, n, a=1.0, eta=1.0, tensor="rpy", prec="fp32c", r_near=None, rep_eps=0.0, rep_rc=None,
                 gravity=(0.0, 0.0, 0.0), device=0, stream=None, torch_allocator=False, dense="auto",
                 lubrication=False, box=None, verlet_skin=None):
        """verlet_skin: neighbour-list skin of the steps (None: 0.5a; <= 0: no list reuse)."""
        if verlet_skin is not None and verlet_skin <= 0:
            verlet_skin = -1.0
        self.cfg, self._keep = _make_config(n, a, eta, tensor, prec, r_near, rep_eps, rep_rc, gravity, device,
                                            stream, torch_allocator, dense, lubrication, box, verlet_skin)
        self.n = int(n)
        self.h = sd_create(self.cfg)

    def close(self):
        if getattr(self, "h", None):
            sd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_positions(self, x, asynchronous=False):
        """Positions from a numpy array, a CUDA tensor or (asynchronous=True: copied on
        the stream, no host synchronisation) a page-locked CPU tensor."""
        p, dev, _k = _as_arg(x, np.float64, asynchronous)
        sd_set_positions(self.h, p, dev)

    def get_positions(self, out=None, asynchronous=False):
        if out is None:
            out = np.empty((self.n, 3))
        p, dev, _k = _as_arg(out, np.float64, asynchronous)
        sd_get_positions(self.h, p, dev)
        return out

    def set_forces(self, f, asynchronous=False):
        p, dev, _k = _as_arg(f, np.float64, asynchronous)
        sd_set_forces(self.h, p, dev)

    def mobility_apply(self, F):
        dt = _dtype_of(F)
        pf, dev, _kf = _as_arg(F, dt)
        pv, devv, V = _out_like(F, self.n, dt)
        sd_mobility_apply(self.h, pf, pv, SD_DTYPE_F32 if dt == np.float32 else SD_DTYPE_F64, dev)
        return V

    def step(self, dt, nsteps=1):
        sd_step(self.h, dt, nsteps)

    def mobility_apply_rows(self, F, row0, row1):
        """Rows row0 .. row1-1 of mu(x) F (F: all n forces); a shard of mobility_apply."""
        dt = _dtype_of(F)
        pf, dev, _kf = _as_arg(F, dt)
        pv, _, V = _out_like(F, int(row1) - int(row0), dt)
        sd_mobility_apply_rows(self.h, pf, pv, SD_DTYPE_F32 if dt == np.float32 else SD_DTYPE_F64, dev, row0, row1)
        return V

    def step_rows(self, dt, row0, row1):
        """One Euler step in which only rows row0 .. row1-1 advance."""
        sd_step_rows(self.h, dt, row0, row1)

    def synchronize(self):
        sd_synchronize(self.h)

    def _part_buffer(self, P):
        import torch
        if P is None:
            P = torch.empty((self.n, 3), dtype=torch.float64, device="cuda:%d" % self.cfg.device)
        if not (P.is_cuda and P.dtype == torch.float64 and P.is_contiguous() and tuple(P.shape) == (self.n, 3)):
            raise ValueError("P must be a contiguous CUDA float64 tensor of shape (n, 3)")
        return P

    @staticmethod
    def _parts(Pall):
        import torch
        if not (Pall.is_cuda and Pall.dtype == torch.float64 and Pall.is_contiguous() and Pall.dim() == 3):
            raise ValueError("Pall must be a contiguous CUDA float64 tensor of shape (nparts, n, 3)")
        return Pall.data_ptr(), Pall.shape[0]

    def mobility_apply_part(self, F, shard, nshards, P=None):
        """This shard's raw share of the all-pairs sum for forces F (a CUDA float64
        tensor P of shape (n, 3) is returned); see sd_mobility_apply_part."""
        dt = _dtype_of(F)
        pf, dev, _kf = _as_arg(F, dt)
        P = self._part_buffer(P)
        sd_mobility_apply_part(self.h, pf, SD_DTYPE_F32 if dt == np.float32 else SD_DTYPE_F64, dev, shard, nshards,
                               P.data_ptr())
        return P

    def mobility_apply_combine(self, Pall, like=None, dtype=np.float64):
        """V = mu(x) F from the shards' results Pall (nparts, n, 3), added in shard
        order.  The output is a CUDA tensor, or a numpy array when `like` is numpy."""
        pp, k = self._parts(Pall)
        import torch
        if like is not None and not _is_torch(like):
            pv, dev, V = _out_like(like, self.n, dtype)
        else:
            V = torch.empty((self.n, 3), dtype=torch.float64 if dtype == np.float64 else torch.float32,
                            device=Pall.device)
            pv, dev = V.data_ptr(), 1
        sd_mobility_apply_combine(self.h, pp, k, pv, SD_DTYPE_F32 if dtype == np.float32 else SD_DTYPE_F64, dev)
        return V

    def step_part(self, shard, nshards, P=None):
        """This shard's raw share of one Euler step's all-pairs sum (P returned)."""
        P = self._part_buffer(P)
        sd_step_part(self.h, shard, nshards, P.data_ptr())
        return P

    def step_combine(self, dt, Pall):
        """Finish the Euler step from the shards' results Pall (nparts, n, 3)."""
        pp, k = self._parts(Pall)
        sd_step_combine(self.h, dt, pp, k)

    def vjp(self, F, W):
        dt = _dtype_of(F)
        pf, dev, _kf = _as_arg(F, dt)
        pw, _, _kw = _as_arg(W, dt)
        pgx, _, gX = _out_like(F, self.n, dt)
        pgf, _, gF = _out_like(F, self.n, dt)
        sd_mobility_vjp(self.h, pf, pw, pgx, pgf, SD_DTYPE_F32 if dt == np.float32 else SD_DTYPE_F64, dev)
        return gX, gF

    def adjoint(self, dt, nsteps, ckpt_every, gxT):
        pg, dev, _kg = _as_arg(gxT, np.float64)
        p0, _, gx0 = _out_like(gxT, self.n, np.float64)
        pF, _, gF = _out_like(gxT, self.n, np.float64)
        sd_adjoint(self.h, dt, nsteps, ckpt_every, pg, p0, pF, dev)
        return gx0, gF

    def profile(self, on=True):
        _check(lib().sd_profile(self.h, int(on)), "sd_profile")

    def profile_read(self, kernel):
        ms = ctypes.c_double()
        cnt = ctypes.c_int64()
        _check(lib().sd_profile_read(self.h, int(kernel), ctypes.byref(ms), ctypes.byref(cnt)), "sd_profile_read")
        return ms.value, cnt.value

    def launch_count(self) -> int:
        return int(lib().sd_launch_count(self.h))

    def dense_kernel(self) -> str:
        """'directed' or 'symmetric': the all-pairs kernel this system runs."""
        k = int(lib().sd_dense_kernel_used(self.h))
        return {v: k2 for k2, v in DENSE_KERNELS.items()}[k]

    def set_watchdog(self, iterations):
        _check(lib().sd_set_watchdog(self.h, int(iterations)), "sd_set_watchdog")

    def inject_stall(self, on=True):
        """Test hook: make the all-pairs kernels' bounded waits run out (SD_ERR_TIMEOUT)."""
        _check(lib().sd_inject_stall(self.h, int(bool(on))), "sd_inject_stall")


class Batch:
    """Independent clusters (CSR offsets, sizes 0..256) stepped by one persistent
    kernel launch per Euler step."""

    def __init__(self, offsets, a=1.0, eta=1.0, tensor="rpy", prec="fp32c", gravity=(0.0, 0.0, 0.0), device=0,
                 stream=None, torch_allocator=False):
        self.cfg, self._keep = _make_config(0, a, eta, tensor, prec, None, 0.0, None, gravity, device, stream,
                                            torch_allocator)
        self.offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
        self.P = int(self.offsets[-1]) if self.offsets.size else 0
        self.b = sd_batch_create(self.cfg, self.offsets)

    def close(self):
        if getattr(self, "b", None):
            sd_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_positions(self, x):
        p, dev, _k = _as_arg(x, np.float64)
        sd_batch_set_positions(self.b, p, dev)

    def get_positions(self, out=None):
        if out is None:
            out = np.empty((self.P, 3))
        p, dev, _k = _as_arg(out, np.float64)
        sd_batch_get_positions(self.b, p, dev)
        return out

    def set_forces(self, f):
        p, dev, _k = _as_arg(f, np.float64)
        sd_batch_set_forces(self.b, p, dev)

    def step(self, dt, nsteps=1):
        sd_step_batched(self.b, dt, nsteps)

    def autotune(self) -> int:
        return sd_batch_autotune(self.b)

    def shapes(self):
        """The candidate launch shapes: dicts of threads per CTA, resident CTAs per SM and
        targets per thread, indexed as autotune() and set_shape() count them."""
        out = []
        for k in range(lib().sd_batch_shape_count(self.b)):
            t, c, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
            _check(lib().sd_batch_shape_info(self.b, k, ctypes.byref(t), ctypes.byref(c), ctypes.byref(r)),
                   "sd_batch_shape_info")
            out.append({"threads": t.value, "ctas_per_sm": c.value, "targets_per_thread": r.value})
        return out

    def set_shape(self, k: int):
        _check(lib().sd_batch_set_shape(self.b, int(k)), "sd_batch_set_shape")

    def synchronize(self):
        _check(lib().sd_batch_synchronize(self.b), "sd_batch_synchronize")

    def profile(self, on=True):
        _check(lib().sd_batch_profile(self.b, int(on)), "sd_batch_profile")

    def profile_read(self, kernel=SD_KERNEL_BATCHED):
        ms = ctypes.c_double()
        cnt = ctypes.c_int64()
        _check(lib().sd_batch_profile_read(self.b, int(kernel), ctypes.byref(ms), ctypes.byref(cnt)),
               "sd_batch_profile_read")
        return ms.value, cnt.value

    def launch_count(self) -> int:
        return int(lib().sd_batch_launch_count(self.b))
