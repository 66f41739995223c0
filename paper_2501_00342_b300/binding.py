"""ctypes binding of the C ABI in include/sgs.h (argument marshalling only).

Every function here forwards to ``libsgs.so``; all arithmetic runs in its CUDA kernels.
Loading fails loudly when the library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsgs.so")

MAX_VIEWS = 64

SGS_OK = 0
SGS_ERR_INVALID = 1
SGS_ERR_CAPACITY = 2
SGS_ERR_TIMEOUT = 4
SGS_ERR_CUDA = 8

REGION = dict(STATUS=0, REC0=1, REC1=2, REC2=3, RECT=4, TILES=5, OFFSETS=6, KEYS=7, VALS=8,
              KEYS_IN=9, VALS_IN=10, RANGES=11, PIX_T=12, PIX_LAST=13, GRAD2D=14,
              PIX_COUNT=15)

# every symbol include/sgs.h declares
EXPORTS = ("sgs_workspace_size", "sgs_preprocess", "sgs_bin_sort", "sgs_render",
           "sgs_render_backward", "sgs_read_device_status", "sgs_region_info",
           "sgs_sort_temp_bytes", "sgs_sort_pairs", "sgs_l1_loss", "sgs_status_string",
           "sgs_abi_sizes", "sgs_set_events", "sgs_sort_pairs_noalloc", "sgs_selftest_lookback",
           "sgs_sort_pairs32", "sgs_adam_step", "sgs_alu_probe_size", "sgs_alu_probe", "sgs_l1_loss_scaled")

SORT_NOALLOC_MAX_PAIRS = 1 << 18

# probe points of sgs_set_events (sgs_event_point)
EVENTS = ("PRE_BEGIN", "PRE_END", "BIN_BEGIN", "SCAN_END", "DUP_END", "HIST_END", "SORT_END",
          "RANGES_END", "BLEND_BEGIN", "BLEND_END", "BWD_BEGIN", "BWD_ZERO_END", "BWD_BLEND_END",
          "BWD_PRE_END")


class Camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 12), ("campos", C.c_float * 3), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("near_plane", C.c_float)]


class Gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("stride", C.c_int64), ("sh_degree", C.c_int32),
                ("num_lobes", C.c_int32), ("axis_mode", C.c_int32)] + \
               [(f, C.c_void_p) for f in ("mean", "scale", "rot", "opacity", "sh", "sg_amp",
                                          "sg_axis", "sg_sharp")] + \
               [("sh_adaptive", C.c_int32), ("sh_radius", C.c_float * 2)]


class Grads(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in ("mean", "scale", "rot", "opacity", "sh", "sg_amp",
                                          "sg_axis", "sg_sharp")]


GROUPS = ("MEAN", "SCALE", "ROT", "OPACITY", "SH_DC", "SH_REST", "SG")  # sgs_param_group


class AdamConfig(C.Structure):
    _fields_ = [("lr", C.c_float * len(GROUPS)), ("step", C.c_int32 * len(GROUPS)), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float)]


class Settings(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("batch_depth", C.c_int32),
                ("digit_bits", C.c_int32), ("memory_mode", C.c_int32), ("bg", C.c_float * 3),
                ("fwd_pixels", C.c_int32), ("bwd_pixels", C.c_int32), ("count_pairs", C.c_int32),
                ("persistent", C.c_int32)]


class Plan(C.Structure):
    _fields_ = [("n", C.c_int64), ("stride", C.c_int64), ("sh_degree", C.c_int32),
                ("num_lobes", C.c_int32), ("axis_mode", C.c_int32), ("B", C.c_int32),
                ("settings", Settings), ("cams", Camera * MAX_VIEWS),
                ("tiles_x", C.c_int32 * MAX_VIEWS), ("tiles_y", C.c_int32 * MAX_VIEWS),
                ("tile_base", C.c_int64 * (MAX_VIEWS + 1)), ("pixel_base", C.c_int64 * (MAX_VIEWS + 1)),
                ("num_records", C.c_int64), ("num_tiles", C.c_int64), ("num_pixels", C.c_int64),
                ("instance_capacity", C.c_int64), ("key_bits", C.c_int32), ("sort_passes", C.c_int32),
                ("stage", C.c_int32), ("events", C.c_void_p), ("offsets", C.c_size_t * 40),
                ("workspace_bytes", C.c_size_t), ("workspace", C.c_void_p)]


class SgsError(RuntimeError):
    def __init__(self, call, code, instances=None):
        super().__init__(f"{call} failed: {status_string(code)} (status {code})")
        self.code = code
        self.instances = instances  # the instance count an overflowing bin_sort needed


_lib = None


def lib():
    """Loads libsgs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2501_00342_b300/build.py")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, st = C.c_void_p, C.c_int32, C.c_int64, C.c_int
        P = C.POINTER
        L.sgs_workspace_size.argtypes = [P(Gaussians), P(Camera), i32, P(Settings), i64, P(Plan), P(C.c_size_t)]
        L.sgs_preprocess.argtypes = [P(Plan), P(Gaussians), vp, C.c_size_t, vp]
        L.sgs_bin_sort.argtypes = [P(Plan), P(C.c_int64), vp]
        L.sgs_render.argtypes = [P(Plan), vp, vp, vp]
        L.sgs_render_backward.argtypes = [P(Plan), P(Gaussians), vp, P(Grads), vp]
        L.sgs_read_device_status.argtypes = [P(Plan), P(C.c_int32), vp]
        L.sgs_region_info.argtypes = [P(Plan), i32, P(C.c_size_t), P(C.c_size_t)]
        L.sgs_sort_temp_bytes.argtypes = [i64, i32, i32, P(C.c_size_t)]
        L.sgs_sort_pairs.argtypes = [vp, vp, i64, i32, i32, vp, C.c_size_t, vp]
        L.sgs_l1_loss.argtypes = [vp, vp, i64, vp, vp, vp]
        L.sgs_status_string.argtypes = [C.c_int]
        L.sgs_status_string.restype = C.c_char_p
        L.sgs_abi_sizes.argtypes = [P(C.c_size_t)]
        L.sgs_set_events.argtypes = [P(Plan), vp]
        L.sgs_set_events.restype = st
        L.sgs_sort_pairs_noalloc.argtypes = [vp, vp, i64, i32, i32, vp]
        L.sgs_sort_pairs_noalloc.restype = st
        L.sgs_sort_pairs32.argtypes = [vp, vp, i64, i32, i32, vp, C.c_size_t, vp]
        L.sgs_sort_pairs32.restype = st
        L.sgs_adam_step.argtypes = [P(Gaussians), P(Grads), P(Grads), P(Grads), P(Grads), P(Grads), P(AdamConfig), vp]
        L.sgs_adam_step.restype = st
        L.sgs_selftest_lookback.argtypes = [vp, i64, vp, vp, vp]
        L.sgs_selftest_lookback.restype = st
        L.sgs_l1_loss_scaled.argtypes = [vp, vp, i64, C.c_float, vp, vp, vp]
        L.sgs_l1_loss_scaled.restype = st
        L.sgs_alu_probe_size.argtypes = [P(C.c_int64)]
        L.sgs_alu_probe_size.restype = st
        L.sgs_alu_probe.argtypes = [i32, i32, vp, P(C.c_double), vp]
        L.sgs_alu_probe.restype = st
        for f in ("sgs_workspace_size", "sgs_preprocess", "sgs_bin_sort", "sgs_render",
                  "sgs_render_backward", "sgs_read_device_status", "sgs_region_info",
                  "sgs_sort_temp_bytes", "sgs_sort_pairs", "sgs_l1_loss"):
            getattr(L, f).restype = st
        sizes = (C.c_size_t * 6)()
        L.sgs_abi_sizes(sizes)
        want = (C.sizeof(Plan), C.sizeof(Camera), C.sizeof(Gaussians), C.sizeof(Settings), C.sizeof(AdamConfig),
                C.sizeof(Grads))
        if tuple(sizes) != want:
            raise RuntimeError(f"sgs ABI mismatch: library {tuple(sizes)} vs binding {want}")
        _lib = L
    return _lib


def set_events(plan, handles):
    """Attaches a ctypes array of cudaEvent_t handles (len(EVENTS), 0 = unused) to the plan,
    or detaches with None.  The caller keeps the array alive."""
    check("sgs_set_events", lib().sgs_set_events(C.byref(plan), None if handles is None else C.cast(handles, C.c_void_p)))


def status_string(code: int) -> str:
    return lib().sgs_status_string(code).decode()


def check(call: str, code: int):
    if code != SGS_OK:
        raise SgsError(call, code)


def camera_struct(cam) -> Camera:
    """From paper_2501_00342_b300.inputs.Camera."""
    c = Camera()
    for k in range(12):
        c.viewmat[k] = float(cam.viewmat[k])
    for k in range(3):
        c.campos[k] = float(cam.campos[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.near_plane = int(cam.width), int(cam.height), float(cam.near)
    return c


def cameras_struct(cams):
    arr = (Camera * len(cams))()
    for k, cam in enumerate(cams):
        arr[k] = camera_struct(cam)
    return arr


def ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


def workspace_size(g: Gaussians, cams, settings: Settings, capacity: int):
    plan = Plan()
    nbytes = C.c_size_t(0)
    arr = cameras_struct(cams)
    check("sgs_workspace_size",
          lib().sgs_workspace_size(C.byref(g), arr, len(cams), C.byref(settings), int(capacity),
                                   C.byref(plan), C.byref(nbytes)))
    return plan, nbytes.value


def preprocess(plan, g, workspace, nbytes, stream):
    check("sgs_preprocess", lib().sgs_preprocess(C.byref(plan), C.byref(g), workspace, nbytes, stream))


def bin_sort(plan, stream, sync: bool):
    """Returns the instance count when ``sync``; raises SgsError(CAPACITY) on overflow."""
    if sync:
        m = C.c_int64(0)
        code = lib().sgs_bin_sort(C.byref(plan), C.byref(m), stream)
        if code == SGS_ERR_CAPACITY:
            # raised without a local name: a local holding the exception would form a cycle
            # with its traceback and keep the caller's workspace alive until a collection
            raise SgsError("sgs_bin_sort", code, instances=m.value)
        check("sgs_bin_sort", code)
        return m.value
    check("sgs_bin_sort", lib().sgs_bin_sort(C.byref(plan), None, stream))
    return None


def render(plan, out_rgb, out_T, stream):
    check("sgs_render", lib().sgs_render(C.byref(plan), out_rgb, out_T, stream))


def render_backward(plan, g, dL_drgb, grads: Grads, stream):
    check("sgs_render_backward",
          lib().sgs_render_backward(C.byref(plan), C.byref(g), dL_drgb, C.byref(grads), stream))


def read_device_status(plan, stream) -> int:
    v = C.c_int32(0)
    check("sgs_read_device_status", lib().sgs_read_device_status(C.byref(plan), C.byref(v), stream))
    return v.value


def region_info(plan, name: str):
    off, nb = C.c_size_t(0), C.c_size_t(0)
    check("sgs_region_info", lib().sgs_region_info(C.byref(plan), REGION[name], C.byref(off), C.byref(nb)))
    return off.value, nb.value


def sort_temp_bytes(m, key_bits, digit_bits) -> int:
    nb = C.c_size_t(0)
    check("sgs_sort_temp_bytes", lib().sgs_sort_temp_bytes(int(m), int(key_bits), int(digit_bits), C.byref(nb)))
    return nb.value


def sort_pairs(keys_ptr, vals_ptr, m, key_bits, digit_bits, temp_ptr, temp_bytes, stream):
    check("sgs_sort_pairs", lib().sgs_sort_pairs(keys_ptr, vals_ptr, int(m), int(key_bits), int(digit_bits),
                                                 temp_ptr, int(temp_bytes), stream))


def sort_pairs32(keys_ptr, vals_ptr, m, key_bits, digit_bits, temp_ptr, temp_bytes, stream):
    check("sgs_sort_pairs32", lib().sgs_sort_pairs32(keys_ptr, vals_ptr, int(m), int(key_bits), int(digit_bits),
                                                     temp_ptr, int(temp_bytes), stream))


def sort_pairs_noalloc(keys_ptr, vals_ptr, m, key_bits, digit_bits, stream):
    """In-place sort with the library's own fixed scratch (no allocation anywhere)."""
    check("sgs_sort_pairs_noalloc",
          lib().sgs_sort_pairs_noalloc(keys_ptr, vals_ptr, int(m), int(key_bits), int(digit_bits), stream))


def adam_step(layout, raw, act, grad, m, v, cfg, stream):
    check("sgs_adam_step", lib().sgs_adam_step(C.byref(layout), C.byref(raw), C.byref(act), C.byref(grad),
                                               C.byref(m), C.byref(v), C.byref(cfg), stream))


# slot flags of sgs_selftest_lookback
LOOKBACK_AGGREGATE = 1 << 62
LOOKBACK_INCLUSIVE = 2 << 62


def selftest_lookback(slots_ptr, num_slots, sum_ptr, status_ptr, stream):
    check("sgs_selftest_lookback", lib().sgs_selftest_lookback(slots_ptr, int(num_slots), sum_ptr,
                                                               status_ptr, stream))


def l1_loss(img_ptr, target_ptr, count, loss_ptr, grad_ptr, stream):
    check("sgs_l1_loss", lib().sgs_l1_loss(img_ptr, target_ptr, int(count), loss_ptr, grad_ptr, stream))


def l1_loss_scaled(img_ptr, target_ptr, count, scale, loss_ptr, grad_ptr, stream):
    check("sgs_l1_loss_scaled",
          lib().sgs_l1_loss_scaled(img_ptr, target_ptr, int(count), float(scale), loss_ptr, grad_ptr, stream))


def alu_probe_size() -> int:
    n = C.c_int64()
    check("sgs_alu_probe_size", lib().sgs_alu_probe_size(C.byref(n)))
    return n.value


def alu_probe(packed: bool, iters: int, out_ptr, stream) -> float:
    """Enqueues the FP32 throughput probe; returns the FP32 operations it performs."""
    ops = C.c_double()
    check("sgs_alu_probe", lib().sgs_alu_probe(int(packed), int(iters), out_ptr, C.byref(ops), stream))
    return ops.value
