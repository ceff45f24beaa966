"""Python binding of libvga, the sm_103a implementation of the voxel-graph diffusion-transformation
method of arXiv 2406.04177.

This module only marshals arguments: every function named `vga_*` calls the C entry point of the
same name declared in include/vga.h, and every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if libvga.so is missing or cannot be loaded the first call
raises, on purpose.  Build it with `paper_2406_04177_gb300.build.build()` (or the repository's
`__graft_entry__.build()`).

Arrays: host data are numpy arrays; device data are torch CUDA tensors (their data_ptr() is passed
with on_device = 1).  Streams are torch.cuda.Stream objects or raw cudaStream_t integers.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvga.so")

VGA_OK = 0
STATUS_NAMES = {0: "VGA_OK", -1: "VGA_ERR_INVALID_ARG", -2: "VGA_ERR_OOM", -3: "VGA_ERR_CUDA",
                -4: "VGA_ERR_UNSTABLE_DT", -5: "VGA_ERR_NOT_CONVERGED", -6: "VGA_ERR_TIMEOUT",
                -7: "VGA_ERR_NONFINITE", -8: "VGA_ERR_UNSUPPORTED"}
VGA_KEEP_LARGEST_COMPONENT = 1
VGA_IMAGE_ON_DEVICE = 2
VGA_SCHEME_EXPLICIT = 0
VGA_SCHEME_IMPLICIT_PCG = 1
VGA_TRANSFORM_SYNC = 0
VGA_TRANSFORM_ASYNC = 1
VGA_STATE_COMPENSATED = 0
VGA_STATE_F32 = 1
VGA_SOLVER_FP64_PCG = 0
VGA_SOLVER_MIXED_REFINEMENT = 1
VGA_SOLVER_MIXED_HOST_LOOP = 2


class VgaError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, "VGA_ERR_UNKNOWN")
        super().__init__(f"{where}: {self.name}: {detail}")


class vga_params(C.Structure):
    _fields_ = [("D", C.c_double), ("dt", C.c_double), ("rho", C.c_double), ("mu", C.c_double),
                ("beta", C.c_double), ("v_som", C.c_double), ("v_fom", C.c_double),
                ("v_dom", C.c_double), ("K_dom", C.c_double), ("scheme", C.c_int32),
                ("transform", C.c_int32), ("cg_rtol", C.c_double), ("cg_maxit", C.c_int32),
                ("state_precision", C.c_int32), ("dt_transform", C.c_double)]


class vga_tune_entry(C.Structure):
    _fields_ = [("variant", C.c_int32), ("chunk", C.c_int32), ("depth", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("ms_per_step", C.c_double)]


class vga_tune_result(C.Structure):
    _fields_ = [("count", C.c_int32), ("best", C.c_int32), ("entries", vga_tune_entry * 16)]


class vga_batch_stats(C.Structure):
    _fields_ = [("instances", C.c_int32), ("grid_blocks", C.c_int32), ("total_nodes", C.c_int64),
                ("steps_per_launch", C.c_int32), ("capture_failed", C.c_int32), ("kernel_launches", C.c_int64),
                ("graph_replays", C.c_int64), ("steps_done", C.c_int64)]


class vga_batch_tune_entry(C.Structure):
    _fields_ = [("steps_per_launch", C.c_int32), ("blocks_per_sm", C.c_int32), ("grid_blocks", C.c_int32),
                ("pad", C.c_int32), ("ms_per_step", C.c_double)]


class vga_batch_tune(C.Structure):
    _fields_ = [("count", C.c_int32), ("best", C.c_int32), ("entries", vga_batch_tune_entry * 16)]


class vga_sim_stats(C.Structure):
    _fields_ = [("steps_done", C.c_int64), ("cg_iterations", C.c_int64),
                ("cg_last_relres", C.c_double), ("kernel_launches", C.c_int64), ("graph_launches", C.c_int64),
                ("active_nodes", C.c_int64), ("blocked_passes", C.c_int64), ("negative_reports", C.c_int64)]


VGA_KERNEL_KINDS = 8
KERNEL_KIND_NAMES = ("fused_step", "transform", "diffuse", "totals", "pcg_stencil", "pcg_vector", "adjoint",
                     "other")


class vga_kernel_timing(C.Structure):
    _fields_ = [("ms", C.c_double * VGA_KERNEL_KINDS), ("launches", C.c_int64 * VGA_KERNEL_KINDS)]


_P, _I32, _I64, _U32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
# name -> argtypes (every function returns int32 vga_status unless listed in _RESTYPES)
_SIGNATURES = {
    "vga_strerror": [C.c_int],
    "vga_last_error": [],
    "vga_version": [],
    "vga_graph_build": [_P, _I32, _I32, _I32, _U32, _P, _P],
    "vga_graph_info": [_P, _P, _P, _P],
    "vga_graph_export": [_P, _P, _P, _P],
    "vga_graph_free": [_P],
    "vga_sim_create": [_P, _P, _P, _P],
    "vga_sim_set_params": [_P, _P],
    "vga_sim_set_block_conductances": [_P, _I32, _P, _I64],
    "vga_sim_set_block_conductances_device": [_P, _I32, _P, _I64],
    "vga_sim_clear_conductances": [_P],
    "vga_sim_set_masses": [_P, _P, _I32],
    "vga_sim_get_masses": [_P, _P, _I32],
    "vga_sim_set_state_f32": [_P, _P, _I32],
    "vga_sim_get_state_f32": [_P, _P, _I32],
    "vga_sim_state_bytes": [_P, _P],
    "vga_sim_save_state": [_P, _P, _I64],
    "vga_sim_load_state": [_P, _P, _I64],
    "vga_sim_step": [_P, _I64],
    "vga_sim_totals": [_P, _P],
    "vga_sim_sync": [_P],
    "vga_sim_get_stats": [_P, _P],
    "vga_adjoint_forward": [_P, _I64, _I32],
    "vga_adjoint_backward": [_P, _P, _I32, _P, _P, _P],
    "vga_adjoint_grad_theta": [_P, _P, _I32, _I64],
    "vga_loss_block_mass": [_P, _I32, _U32, _P, _P, _P, _P],
    "vga_sgd_block_conductances": [_P, C.c_double, C.c_double, C.c_double],
    "vga_sim_get_block_conductances": [_P, _P, _I64],
    "vga_sim_set_kernel": [_P, _I32, _I32],
    "vga_sim_set_solver": [_P, _I32],
    "vga_sim_set_activity_skip": [_P, _I32],
    "vga_batch_set_activity_skip": [_P, _I32],
    "vga_sim_set_wavefront": [_P, _I32, _I32, _I32],
    "vga_sim_autotune": [_P, _I32, _P],
    "vga_sim_enable_timing": [_P, _I32],
    "vga_sim_read_timing": [_P, _P, _I32],
    "vga_sim_free": [_P],
    "vga_batch_create": [_P, _P, _I32, _P],
    "vga_batch_info": [_P, _P, _P],
    "vga_batch_set_masses": [_P, _I32, _P],
    "vga_batch_get_masses": [_P, _I32, _P],
    "vga_batch_step": [_P, _I64],
    "vga_batch_set_launch": [_P, _I32, _I32, _I32],
    "vga_batch_get_stats": [_P, _P],
    "vga_batch_autotune": [_P, _I32, _P],
    "vga_batch_free": [_P],
    "vga_state_totals_noalloc": [_P, _P, _I64, _I64, _P, _P],
    "vga_batch_set_wait_test": [_P, _I32, C.c_uint32],
    "vga_sim_set_face_conductances": [_P, _P],
    "vga_pngm_create": [_P, _P, _I32, _I32, _P, _P],
    "vga_pngm_get_info": [_P, _P],
    "vga_pngm_export": [_P, _P, _P, _P, _P, _P, _P, _P],
    "vga_pngm_set_theta": [_P, _P, _I32],
    "vga_pngm_get_theta": [_P, _P, _I32],
    "vga_pngm_restrict": [_P, _P, _I32, _P],
    "vga_pngm_step": [_P, _P, _I64, _I32, C.c_double, C.c_double, C.c_double, _I32],
    "vga_pngm_objective": [_P, _I32, _P, _I64, _P, _I32, C.c_double, C.c_double, _I32, _P, _P],
    "vga_pngm_sgd_step": [_P, _I32, _P, _I64, _P, _I32, C.c_double, C.c_double, C.c_double, C.c_double, _I32, _P],
    "vga_pngm_free": [_P],
}
_RESTYPES = {"vga_strerror": C.c_char_p, "vga_last_error": C.c_char_p, "vga_version": C.c_int32}

_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None):
    """Loads libvga.so (raises if it is missing: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_2406_04177_gb300.build.build() "
                               "(nvcc for sm_103a); no CPU fallback exists")
        lib = C.CDLL(p)
        for name, args in _SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = _RESTYPES.get(name, C.c_int32)
        _lib = lib
        return lib


def declared_symbols() -> list[str]:
    return list(_SIGNATURES)


def _check(status: int, where: str):
    if status != VGA_OK:
        detail = load_library().vga_last_error().decode(errors="replace")
        raise VgaError(int(status), where, detail)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _host_ptr(a: np.ndarray, dtype, shape_n: int | None = None):
    if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous):
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    if shape_n is not None and a.size != shape_n:
        raise ValueError(f"expected {shape_n} elements, got {a.size}")
    return a.ctypes.data_as(C.c_void_p)


def _dev_ptr(t, dtype_name: str, count: int | None = None) -> int:
    import torch

    want = {"float64": torch.float64, "float32": torch.float32, "uint8": torch.uint8}[dtype_name]
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == want and t.is_contiguous()):
        raise TypeError(f"expected a contiguous CUDA tensor of {want}")
    if count is not None and t.numel() != count:
        raise ValueError(f"expected {count} elements, got {t.numel()}")
    return t.data_ptr()


# ---- one Python function per C entry point (argument marshalling only) -------------------------
def vga_strerror(status: int) -> str:
    return load_library().vga_strerror(int(status)).decode()


def vga_last_error() -> str:
    return load_library().vga_last_error().decode(errors="replace")


def vga_version() -> int:
    return int(load_library().vga_version())


def vga_graph_build(img, flags: int = VGA_KEEP_LARGEST_COMPONENT, stream=None) -> C.c_void_p:
    """img: uint8 [nz, ny, nx] numpy array (host) or CUDA tensor (device); 0 = pore."""
    lib = load_library()
    nz, ny, nx = (int(s) for s in img.shape)
    if isinstance(img, np.ndarray):
        img = np.ascontiguousarray(img, dtype=np.uint8)  # kept alive until the call returns
        ptr = _host_ptr(img, np.uint8)
        flags &= ~VGA_IMAGE_ON_DEVICE
    else:
        ptr = _dev_ptr(img, "uint8")
        flags |= VGA_IMAGE_ON_DEVICE
    out = C.c_void_p()
    _check(lib.vga_graph_build(ptr, nx, ny, nz, flags, _stream_ptr(stream), C.byref(out)), "vga_graph_build")
    return out


def vga_graph_info(g) -> tuple[int, int, int]:
    n, nc, lg = C.c_int64(), C.c_int32(), C.c_int32()
    _check(load_library().vga_graph_info(g, C.byref(n), C.byref(nc), C.byref(lg)), "vga_graph_info")
    return n.value, nc.value, lg.value


def vga_graph_export(g, labels=None, voxel_of_node=None, nbr=None):
    lib = load_library()
    _check(lib.vga_graph_export(g, None if labels is None else _host_ptr(labels, np.int32),
                                None if voxel_of_node is None else _host_ptr(voxel_of_node, np.int64),
                                None if nbr is None else _host_ptr(nbr, np.int32)), "vga_graph_export")


def vga_graph_free(g):
    _check(load_library().vga_graph_free(g), "vga_graph_free")


def make_params(p: dict) -> vga_params:
    return vga_params(D=p["D"], dt=p["dt"], rho=p["rho"], mu=p["mu"], beta=p["beta"], v_som=p["v_som"],
                      v_fom=p["v_fom"], v_dom=p["v_dom"], K_dom=p["K_dom"], scheme=int(p.get("scheme", 0)),
                      transform=int(p.get("transform", 0)), cg_rtol=float(p.get("cg_rtol", 1e-8)),
                      cg_maxit=int(p.get("cg_maxit", 500)), state_precision=int(p.get("state_precision", 0)),
                      dt_transform=float(p.get("dt_transform", 0.0)))


def vga_sim_create(g, params: dict, stream=None) -> C.c_void_p:
    out = C.c_void_p()
    pp = make_params(params)
    _check(load_library().vga_sim_create(g, C.byref(pp), _stream_ptr(stream), C.byref(out)), "vga_sim_create")
    return out


def vga_sim_set_params(s, params: dict):
    pp = make_params(params)
    _check(load_library().vga_sim_set_params(s, C.byref(pp)), "vga_sim_set_params")


def vga_sim_set_block_conductances(s, block_side: int, theta: np.ndarray):
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    _check(load_library().vga_sim_set_block_conductances(s, int(block_side), _host_ptr(theta, np.float32),
                                                         theta.size), "vga_sim_set_block_conductances")


def vga_sim_set_block_conductances_device(s, block_side: int, d_theta):
    """d_theta: contiguous CUDA float32 tensor (checked on the device)."""
    _check(load_library().vga_sim_set_block_conductances_device(s, int(block_side), _dev_ptr(d_theta, "float32"),
                                                                d_theta.numel()),
           "vga_sim_set_block_conductances_device")


def vga_sim_clear_conductances(s):
    _check(load_library().vga_sim_clear_conductances(s), "vga_sim_clear_conductances")


def vga_sim_set_masses(s, x, n: int):
    if isinstance(x, np.ndarray):
        _check(load_library().vga_sim_set_masses(s, _host_ptr(x, np.float64, 5 * n), 0), "vga_sim_set_masses")
    else:
        _check(load_library().vga_sim_set_masses(s, _dev_ptr(x, "float64", 5 * n), 1), "vga_sim_set_masses")


def vga_sim_get_masses(s, out, n: int):
    if isinstance(out, np.ndarray):
        _check(load_library().vga_sim_get_masses(s, _host_ptr(out, np.float64, 5 * n), 0), "vga_sim_get_masses")
    else:
        _check(load_library().vga_sim_get_masses(s, _dev_ptr(out, "float64", 5 * n), 1), "vga_sim_get_masses")


def vga_sim_set_state_f32(s, x, n: int):
    if isinstance(x, np.ndarray):
        _check(load_library().vga_sim_set_state_f32(s, _host_ptr(x, np.float32, 5 * n), 0), "vga_sim_set_state_f32")
    else:
        _check(load_library().vga_sim_set_state_f32(s, _dev_ptr(x, "float32", 5 * n), 1), "vga_sim_set_state_f32")


def vga_sim_get_state_f32(s, out, n: int):
    if isinstance(out, np.ndarray):
        _check(load_library().vga_sim_get_state_f32(s, _host_ptr(out, np.float32, 5 * n), 0), "vga_sim_get_state_f32")
    else:
        _check(load_library().vga_sim_get_state_f32(s, _dev_ptr(out, "float32", 5 * n), 1), "vga_sim_get_state_f32")


def vga_sim_state_bytes(s) -> int:
    v = C.c_int64()
    _check(load_library().vga_sim_state_bytes(s, C.byref(v)), "vga_sim_state_bytes")
    return v.value


def vga_sim_save_state(s) -> bytes:
    nb = vga_sim_state_bytes(s)
    buf = (C.c_char * nb)()
    _check(load_library().vga_sim_save_state(s, buf, nb), "vga_sim_save_state")
    return bytes(buf)


def vga_sim_load_state(s, data: bytes):
    buf = C.create_string_buffer(data, len(data))
    _check(load_library().vga_sim_load_state(s, buf, len(data)), "vga_sim_load_state")


def vga_sim_step(s, n_steps: int):
    _check(load_library().vga_sim_step(s, int(n_steps)), "vga_sim_step")


def vga_sim_totals(s) -> np.ndarray:
    out = np.zeros(5, dtype=np.float64)
    _check(load_library().vga_sim_totals(s, out.ctypes.data_as(C.c_void_p)), "vga_sim_totals")
    return out


def vga_sim_sync(s):
    _check(load_library().vga_sim_sync(s), "vga_sim_sync")


def vga_sim_get_stats(s) -> dict:
    st = vga_sim_stats()
    _check(load_library().vga_sim_get_stats(s, C.byref(st)), "vga_sim_get_stats")
    return {k: getattr(st, k) for k, _ in vga_sim_stats._fields_}


GRAD_NAMES = ("D", "rho", "mu", "beta", "v_som", "v_fom", "v_dom", "K_dom")


def vga_adjoint_forward(s, n_steps: int, ckpt_every: int):
    _check(load_library().vga_adjoint_forward(s, int(n_steps), int(ckpt_every)), "vga_adjoint_forward")


def vga_adjoint_backward(s, dL_dXN, n: int, dL_dX0=None, n_theta: int = 0):
    """Returns (grad dict, grad_theta numpy array or None); fills dL_dX0 if given (same memory
    space as dL_dXN)."""
    grad = np.zeros(8, dtype=np.float64)
    gth = np.zeros(max(n_theta, 1), dtype=np.float64) if n_theta > 0 else None
    if isinstance(dL_dXN, np.ndarray):
        src = _host_ptr(dL_dXN, np.float64, 5 * n)
        dst = None if dL_dX0 is None else _host_ptr(dL_dX0, np.float64, 5 * n)
        dev = 0
    else:
        src = _dev_ptr(dL_dXN, "float64", 5 * n)
        dst = None if dL_dX0 is None else _dev_ptr(dL_dX0, "float64", 5 * n)
        dev = 1
    _check(load_library().vga_adjoint_backward(s, src, dev, dst, grad.ctypes.data_as(C.c_void_p),
                                               None if gth is None else gth.ctypes.data_as(C.c_void_p)),
           "vga_adjoint_backward")
    return dict(zip(GRAD_NAMES, grad.tolist())), gth


def vga_adjoint_grad_theta(s, out):
    """Conductance gradient of the last backward sweep into `out` (numpy float64 array, or CUDA
    float64 tensor), whose size is the number of conductances."""
    if isinstance(out, np.ndarray):
        ptr, dev, n = _host_ptr(out, np.float64), 0, out.size
    else:
        ptr, dev, n = _dev_ptr(out, "float64"), 1, out.numel()
    _check(load_library().vga_adjoint_grad_theta(s, ptr, dev, int(n)), "vga_adjoint_grad_theta")
    return out


def vga_loss_block_mass(s, block_side: int, comp_mask: int, target: np.ndarray, n: int, dL_dX=None,
                        want_mass: bool = False):
    """Returns (loss, block masses or None); writes dL/dX into the CUDA tensor dL_dX if given."""
    target = np.ascontiguousarray(target, dtype=np.float64)
    loss = C.c_double()
    mass = np.empty_like(target) if want_mass else None
    _check(load_library().vga_loss_block_mass(s, int(block_side), int(comp_mask), _host_ptr(target, np.float64),
                                              C.byref(loss), None if mass is None else _host_ptr(mass, np.float64),
                                              None if dL_dX is None else _dev_ptr(dL_dX, "float64", 5 * n)),
           "vga_loss_block_mass")
    return loss.value, mass


def vga_sim_set_kernel(s, variant: int, chunk: int):
    _check(load_library().vga_sim_set_kernel(s, int(variant), int(chunk)), "vga_sim_set_kernel")


def vga_sim_set_solver(s, solver: int):
    _check(load_library().vga_sim_set_solver(s, int(solver)), "vga_sim_set_solver")


def vga_sim_set_activity_skip(s, on: bool):
    _check(load_library().vga_sim_set_activity_skip(s, 1 if on else 0), "vga_sim_set_activity_skip")


def vga_batch_set_activity_skip(b, on: bool):
    _check(load_library().vga_batch_set_activity_skip(b, 1 if on else 0), "vga_batch_set_activity_skip")


def vga_sim_set_wavefront(s, chunk: int, depth: int, ctas_per_sm: int = 0):
    _check(load_library().vga_sim_set_wavefront(s, int(chunk), int(depth), int(ctas_per_sm)), "vga_sim_set_wavefront")


def vga_sim_autotune(s, trial_steps: int = 20) -> dict:
    r = vga_tune_result()
    _check(load_library().vga_sim_autotune(s, int(trial_steps), C.byref(r)), "vga_sim_autotune")
    entries = [dict(variant=r.entries[k].variant, chunk=r.entries[k].chunk, depth=r.entries[k].depth,
                    ctas_per_sm=r.entries[k].ctas_per_sm, ms_per_step=r.entries[k].ms_per_step)
               for k in range(r.count)]
    return dict(best=entries[r.best] if r.best >= 0 else None, entries=entries)


def vga_sgd_block_conductances(s, lr: float, theta_min: float, theta_max: float):
    _check(load_library().vga_sgd_block_conductances(s, float(lr), float(theta_min), float(theta_max)),
           "vga_sgd_block_conductances")


def vga_sim_get_block_conductances(s, n_theta: int) -> np.ndarray:
    out = np.empty(n_theta, dtype=np.float32)
    _check(load_library().vga_sim_get_block_conductances(s, _host_ptr(out, np.float32), n_theta),
           "vga_sim_get_block_conductances")
    return out


def vga_sim_enable_timing(s, on: bool = True):
    _check(load_library().vga_sim_enable_timing(s, 1 if on else 0), "vga_sim_enable_timing")


def vga_sim_read_timing(s, reset: bool = False) -> dict:
    """{kind name: (total ms, launches)} of the kernels timed since the last reset."""
    kt = vga_kernel_timing()
    _check(load_library().vga_sim_read_timing(s, C.byref(kt), 1 if reset else 0), "vga_sim_read_timing")
    return {KERNEL_KIND_NAMES[k]: (kt.ms[k], int(kt.launches[k])) for k in range(VGA_KERNEL_KINDS)}


def vga_sim_free(s):
    _check(load_library().vga_sim_free(s), "vga_sim_free")


def vga_sim_set_face_conductances(s, g_face: np.ndarray):
    """g_face: (n, 6) float32 host array, slot order -x, +x, -y, +y, -z, +z; symmetric across edges."""
    g = np.ascontiguousarray(g_face, dtype=np.float32)
    _check(load_library().vga_sim_set_face_conductances(s, g.ctypes.data_as(C.c_void_p)), "vga_sim_set_face_conductances")


def vga_batch_set_wait_test(b, skip_block: int, spin_limit: int = 0):
    """Bounded-wait test hook of the batched launches; skip_block = -1 switches it off."""
    _check(load_library().vga_batch_set_wait_test(b, int(skip_block), int(spin_limit)), "vga_batch_set_wait_test")


def vga_state_totals_noalloc(values, residuals, n: int, row_stride: int, totals, stream=None):
    """values / residuals / totals are CUDA tensors (float32; 16-bit residual bits or None;
    float64 with at least 5 entries), contiguous; compartment c occupies
    [c * row_stride, c * row_stride + n) of values (and residuals).  The call allocates nothing.
    Sizes and layout are checked here, before any device access: the kernel itself has no bounds
    to check against."""
    import torch

    n, row_stride = int(n), int(row_stride)
    if n < 0 or row_stride < n:
        raise ValueError(f"need 0 <= n <= row_stride (n = {n}, row_stride = {row_stride})")
    need = 4 * row_stride + n if n > 0 else 0
    for name, t in (("values", values), ("residuals", residuals), ("totals", totals)):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        want = 5 if name == "totals" else need
        if t.numel() < want:
            raise ValueError(f"{name} holds {t.numel()} elements, the call reads or writes {want}")
    if not (isinstance(values, torch.Tensor) and values.is_cuda and values.dtype == torch.float32):
        raise TypeError("values must be a CUDA float32 tensor")
    if residuals is not None and not (isinstance(residuals, torch.Tensor) and residuals.is_cuda
                                      and residuals.element_size() == 2):
        raise TypeError("residuals must be a CUDA tensor of 16-bit elements")
    if not (isinstance(totals, torch.Tensor) and totals.is_cuda and totals.dtype == torch.float64):
        raise TypeError("totals must be a CUDA float64 tensor")
    _check(load_library().vga_state_totals_noalloc(values.data_ptr(), None if residuals is None else residuals.data_ptr(),
                                                   int(n), int(row_stride), totals.data_ptr(), _stream_ptr(stream)),
           "vga_state_totals_noalloc")


def vga_batch_create(graph_handles, params_list) -> C.c_void_p:
    count = len(graph_handles)
    arr = (C.c_void_p * count)(*[g.value if isinstance(g, C.c_void_p) else g for g in graph_handles])
    parr = (vga_params * count)(*[make_params(p) for p in params_list])
    out = C.c_void_p()
    _check(load_library().vga_batch_create(arr, parr, count, C.byref(out)), "vga_batch_create")
    return out


def vga_batch_info(b, count: int):
    tot = C.c_int64()
    offs = np.zeros(count, dtype=np.int64)
    _check(load_library().vga_batch_info(b, C.byref(tot), offs.ctypes.data_as(C.c_void_p)), "vga_batch_info")
    return tot.value, offs


def vga_batch_set_masses(b, instance: int, x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float64)
    _check(load_library().vga_batch_set_masses(b, int(instance), x.ctypes.data_as(C.c_void_p)), "vga_batch_set_masses")


def vga_batch_get_masses(b, instance: int, out: np.ndarray):
    _check(load_library().vga_batch_get_masses(b, int(instance), _host_ptr(out, np.float64)), "vga_batch_get_masses")


def vga_batch_step(b, n_steps: int):
    _check(load_library().vga_batch_step(b, int(n_steps)), "vga_batch_step")


def vga_batch_set_launch(b, steps_per_launch: int, blocks_per_sm: int = 0, use_graph: bool = True):
    _check(load_library().vga_batch_set_launch(b, int(steps_per_launch), int(blocks_per_sm), 1 if use_graph else 0),
           "vga_batch_set_launch")


def vga_batch_get_stats(b) -> dict:
    st = vga_batch_stats()
    _check(load_library().vga_batch_get_stats(b, C.byref(st)), "vga_batch_get_stats")
    return {k: getattr(st, k) for k, _ in vga_batch_stats._fields_}


def vga_batch_autotune(b, trial_steps: int = 50) -> dict:
    r = vga_batch_tune()
    _check(load_library().vga_batch_autotune(b, int(trial_steps), C.byref(r)), "vga_batch_autotune")
    entries = [dict(steps_per_launch=r.entries[k].steps_per_launch, blocks_per_sm=r.entries[k].blocks_per_sm,
                    grid_blocks=r.entries[k].grid_blocks, ms_per_step=r.entries[k].ms_per_step) for k in range(r.count)]
    return dict(best=entries[r.best] if r.best >= 0 else None, entries=entries)


def vga_batch_free(b):
    _check(load_library().vga_batch_free(b), "vga_batch_free")


# ---- handle classes (ownership only) ------------------------------------------------------------
class vga_pngm_info(C.Structure):
    _fields_ = [("q", C.c_int32), ("n_slots", C.c_int32), ("n_nodes", C.c_int64), ("cross_faces", C.c_int64),
                ("symmetric", C.c_int32), ("last_cg_iterations", C.c_int64), ("last_cg_relres", C.c_double)]


def _pairs_array(pairs) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    if a.shape[0] < 1:
        raise ValueError("need at least one pair")
    return a


class Graph:
    """Owns a vga_graph handle."""

    def __init__(self, img, keep_largest: bool = True, stream=None):
        self.shape = tuple(int(s) for s in img.shape)
        self.handle = vga_graph_build(img, VGA_KEEP_LARGEST_COMPONENT if keep_largest else 0, stream)
        self.n, self.n_components, self.largest = vga_graph_info(self.handle)

    def export(self, labels: bool = True, voxel_of_node: bool = True, nbr: bool = True) -> dict:
        nvox = int(np.prod(self.shape))
        out = {}
        if labels:
            out["labels"] = np.empty(nvox, dtype=np.int32)
        if voxel_of_node:
            out["voxel_of_node"] = np.empty(max(self.n, 0), dtype=np.int64)
        if nbr:
            out["nbr"] = np.empty(6 * max(self.n, 0), dtype=np.int32)
        vga_graph_export(self.handle, out.get("labels"), out.get("voxel_of_node"), out.get("nbr"))
        if labels:
            out["labels"] = out["labels"].reshape(self.shape)
        if nbr:
            out["nbr"] = out["nbr"].reshape(-1, 6)
        return out

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None  # never freed twice, even if the free reports an error
            vga_graph_free(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sim:
    """Owns a vga_sim handle on a Graph (which must stay alive)."""

    def __init__(self, graph: Graph, params: dict, stream=None):
        self.graph = graph
        self.n = graph.n
        self._base_params = dict(params)
        self.handle = vga_sim_create(graph.handle, params, stream)

    def set_params(self, params: dict):
        vga_sim_set_params(self.handle, params)
        self._base_params = dict(params)

    def set_block_conductances(self, block_side: int, theta):
        """theta: numpy array (host), or CUDA float32 tensor (device form)."""
        if isinstance(theta, np.ndarray):
            vga_sim_set_block_conductances(self.handle, block_side, theta)
        else:
            vga_sim_set_block_conductances_device(self.handle, block_side, theta)

    def clear_conductances(self):
        vga_sim_clear_conductances(self.handle)

    def set_face_conductances(self, g_face):
        """Per-face conductances, (n, 6) float32 in the slot order of Graph.export's nbr."""
        g = np.ascontiguousarray(g_face, dtype=np.float32)
        if g.shape != (self.n, 6):
            raise ValueError(f"g_face must have shape ({self.n}, 6)")
        vga_sim_set_face_conductances(self.handle, g)

    def set_masses(self, x):
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
        vga_sim_set_masses(self.handle, x, self.n)

    def get_masses(self, out=None) -> np.ndarray:
        if out is None:
            out = np.empty((5, self.n), dtype=np.float64)
        vga_sim_get_masses(self.handle, out, self.n)
        return out

    def set_state_f32(self, x):
        vga_sim_set_state_f32(self.handle, x, self.n)

    def get_state_f32(self, out=None):
        if out is None:
            out = np.empty((5, self.n), dtype=np.float32)
        vga_sim_get_state_f32(self.handle, out, self.n)
        return out

    def step(self, n_steps: int):
        vga_sim_step(self.handle, n_steps)

    def save_state(self) -> bytes:
        return vga_sim_save_state(self.handle)

    def load_state(self, data: bytes):
        vga_sim_load_state(self.handle, data)

    def totals(self) -> np.ndarray:
        return vga_sim_totals(self.handle)

    def sync(self):
        vga_sim_sync(self.handle)

    def stats(self) -> dict:
        return vga_sim_get_stats(self.handle)

    def set_kernel(self, variant: int, chunk: int):
        vga_sim_set_kernel(self.handle, variant, chunk)

    def set_solver(self, solver: int):
        vga_sim_set_solver(self.handle, solver)

    def set_activity_skip(self, on: bool):
        vga_sim_set_activity_skip(self.handle, on)

    def set_wavefront(self, chunk: int, depth: int, ctas_per_sm: int = 0):
        vga_sim_set_wavefront(self.handle, chunk, depth, ctas_per_sm)

    def autotune(self, trial_steps: int = 20) -> dict:
        return vga_sim_autotune(self.handle, trial_steps)

    def adjoint_forward(self, n_steps: int, ckpt_every: int = 100):
        vga_adjoint_forward(self.handle, n_steps, ckpt_every)

    def adjoint_backward(self, dL_dXN, dL_dX0=None, n_theta: int = 0):
        return vga_adjoint_backward(self.handle, dL_dXN, self.n, dL_dX0, n_theta)

    def adjoint_grad_theta(self, out):
        return vga_adjoint_grad_theta(self.handle, out)

    def loss_block_mass(self, block_side: int, comp_mask: int, target, dL_dX=None, want_mass: bool = False):
        return vga_loss_block_mass(self.handle, block_side, comp_mask, target, self.n, dL_dX, want_mass)

    def sgd_block_conductances(self, lr: float, theta_min: float, theta_max: float):
        vga_sgd_block_conductances(self.handle, lr, theta_min, theta_max)

    def get_block_conductances(self, n_theta: int) -> np.ndarray:
        return vga_sim_get_block_conductances(self.handle, n_theta)

    def enable_timing(self, on: bool = True):
        vga_sim_enable_timing(self.handle, on)

    def read_timing(self, reset: bool = False) -> dict:
        return vga_sim_read_timing(self.handle, reset)

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None
            vga_sim_free(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns a vga_batch handle over several Graphs (which must stay alive)."""

    def __init__(self, graphs, params_list):
        self.graphs = list(graphs)
        self.sizes = [g.n for g in self.graphs]
        self.handle = vga_batch_create([g.handle for g in self.graphs], params_list)
        self.total_nodes, self.offsets = vga_batch_info(self.handle, len(self.graphs))

    def set_masses(self, k: int, x):
        vga_batch_set_masses(self.handle, k, x)

    def get_masses(self, k: int) -> np.ndarray:
        out = np.empty((5, self.sizes[k]), dtype=np.float64)
        vga_batch_get_masses(self.handle, k, out)
        return out

    def step(self, n_steps: int):
        vga_batch_step(self.handle, n_steps)

    def set_activity_skip(self, on: bool):
        vga_batch_set_activity_skip(self.handle, on)

    def set_launch(self, steps_per_launch: int, blocks_per_sm: int = 0, use_graph: bool = True):
        vga_batch_set_launch(self.handle, steps_per_launch, blocks_per_sm, use_graph)

    def stats(self) -> dict:
        return vga_batch_get_stats(self.handle)

    def set_wait_test(self, skip_block: int, spin_limit: int = 0):
        """Bounded-wait test hook (vga_batch_set_wait_test); skip_block = -1 switches it off."""
        vga_batch_set_wait_test(self.handle, skip_block, spin_limit)

    def autotune(self, trial_steps: int = 50) -> dict:
        return vga_batch_autotune(self.handle, trial_steps)

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None
            vga_batch_free(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



# ---- coarse primitive-graph model (Sec. V.A) ----------------------------------------------------
def vga_pngm_create(g, labels, q: int, n: int, stream=None):
    """labels: int32 numpy array (host) or contiguous int32 CUDA tensor of n entries."""
    if isinstance(labels, np.ndarray):
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        if lab.size != n:
            raise ValueError("labels must have one entry per node")
        ptr, on_dev = lab.ctypes.data, 0
    else:
        import torch

        if not (isinstance(labels, torch.Tensor) and labels.is_cuda and labels.dtype == torch.int32
                and labels.is_contiguous() and labels.numel() == n):
            raise TypeError("labels must be an int32 numpy array or contiguous CUDA tensor of n entries")
        ptr, on_dev = labels.data_ptr(), 1
    h = C.c_void_p()
    _check(load_library().vga_pngm_create(g, ptr, on_dev, int(q), _stream_ptr(stream), C.byref(h)), "vga_pngm_create")
    return h


def vga_pngm_get_info(h) -> dict:
    st = vga_pngm_info()
    _check(load_library().vga_pngm_get_info(h, C.byref(st)), "vga_pngm_get_info")
    return {k: getattr(st, k) for k, _ in vga_pngm_info._fields_}


def vga_pngm_export(h, q: int, n_slots: int) -> dict:
    out = dict(vol=np.empty(q), centroid=np.empty((q, 3)), row_ptr=np.empty(q + 1, dtype=np.int32),
               col=np.empty(n_slots, dtype=np.int32), rev=np.empty(n_slots, dtype=np.int32), S=np.empty(n_slots),
               dist=np.empty(n_slots))
    _check(load_library().vga_pngm_export(h, out["vol"].ctypes.data, out["centroid"].ctypes.data,
                                          out["row_ptr"].ctypes.data, out["col"].ctypes.data, out["rev"].ctypes.data,
                                          out["S"].ctypes.data, out["dist"].ctypes.data), "vga_pngm_export")
    return out


def vga_pngm_set_theta(h, theta, n_slots: int):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.size != n_slots:
        raise ValueError(f"theta needs {n_slots} entries")
    _check(load_library().vga_pngm_set_theta(h, th.ctypes.data, 0), "vga_pngm_set_theta")


def vga_pngm_get_theta(h, n_slots: int) -> np.ndarray:
    out = np.empty(n_slots)
    _check(load_library().vga_pngm_get_theta(h, out.ctypes.data, 0), "vga_pngm_get_theta")
    return out


def vga_pngm_restrict(h, sim, comp: int, out, q: int):
    _check(load_library().vga_pngm_restrict(h, sim, int(comp), _dev_ptr(out, "float64", q)), "vga_pngm_restrict")
    return out


def vga_pngm_step(h, m, q: int, n_steps: int, scheme: int, D: float, dt: float, cg_rtol: float = 1e-12,
                  cg_maxit: int = 10000):
    _check(load_library().vga_pngm_step(h, _dev_ptr(m, "float64", q), int(n_steps), int(scheme), float(D), float(dt),
                                        float(cg_rtol), int(cg_maxit)), "vga_pngm_step")
    return m


def _pngm_data(data, q: int) -> int:
    if data.dim() != 2 or data.shape[1] != q:
        raise ValueError(f"data must be (records, {q})")
    return _dev_ptr(data, "float64")


def vga_pngm_objective(h, q: int, n_slots: int, kind: int, data, pairs, D: float, dt: float, tied: bool = False,
                       grad=None) -> float:
    p = _pairs_array(pairs)
    loss = C.c_double(0.0)
    _check(load_library().vga_pngm_objective(h, int(kind), _pngm_data(data, q), int(data.shape[0]), p.ctypes.data,
                                             p.shape[0], float(D), float(dt), 1 if tied else 0, C.byref(loss),
                                             None if grad is None else _dev_ptr(grad, "float64", n_slots)),
           "vga_pngm_objective")
    return loss.value


def vga_pngm_sgd_step(h, q: int, kind: int, data, pairs, D: float, dt: float, lr: float, tied: bool = False,
                      theta_min: float = -np.inf) -> float:
    p = _pairs_array(pairs)
    loss = C.c_double(0.0)
    _check(load_library().vga_pngm_sgd_step(h, int(kind), _pngm_data(data, q), int(data.shape[0]), p.ctypes.data,
                                            p.shape[0], float(D), float(dt), float(lr), float(theta_min),
                                            1 if tied else 0, C.byref(loss)), "vga_pngm_sgd_step")
    return loss.value


def vga_pngm_free(h):
    _check(load_library().vga_pngm_free(h), "vga_pngm_free")


class Pngm:
    """Owns a vga_pngm handle: the coarse primitive graph of a node partition on a Graph (which
    must stay alive).  Device vectors (masses, data, gradients) are torch CUDA float64 tensors."""

    def __init__(self, graph: Graph, labels, q: int, stream=None):
        self.graph = graph
        self.handle = vga_pngm_create(graph.handle, labels, q, graph.n, stream)
        self.q = int(q)
        self.n_slots = self.info()["n_slots"]

    def info(self) -> dict:
        return vga_pngm_get_info(self.handle)

    def export(self) -> dict:
        return vga_pngm_export(self.handle, self.q, self.n_slots)

    def get_theta(self) -> np.ndarray:
        return vga_pngm_get_theta(self.handle, self.n_slots)

    def set_theta(self, theta):
        vga_pngm_set_theta(self.handle, theta, self.n_slots)

    def restrict(self, sim: "Sim", comp: int, out):
        return vga_pngm_restrict(self.handle, sim.handle, comp, out, self.q)

    def step(self, m, n_steps: int, scheme: int, D: float, dt: float, cg_rtol: float = 1e-12, cg_maxit: int = 10000):
        return vga_pngm_step(self.handle, m, self.q, n_steps, scheme, D, dt, cg_rtol, cg_maxit)

    def objective(self, kind: int, data, pairs, D: float, dt: float, tied: bool = False, grad=None) -> float:
        return vga_pngm_objective(self.handle, self.q, self.n_slots, kind, data, pairs, D, dt, tied, grad)

    def sgd_step(self, kind: int, data, pairs, D: float, dt: float, lr: float, tied: bool = False,
                 theta_min: float = -np.inf) -> float:
        return vga_pngm_sgd_step(self.handle, self.q, kind, data, pairs, D, dt, lr, tied, theta_min)

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None
            vga_pngm_free(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
