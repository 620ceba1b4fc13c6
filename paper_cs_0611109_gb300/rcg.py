"""Python binding of librcg (include/rcg.h): ctypes argument marshalling only.

Every function here has the name and the semantics of the C call it wraps;
all stripe arithmetic runs in the CUDA kernels of librcg.so.  Device buffers
are passed as PyTorch CUDA tensors (their data_ptr) or raw integer addresses;
streams as torch.cuda.Stream, a raw cudaStream_t integer, or None for the
current PyTorch stream.  There is no CPU fallback: if librcg.so has not been
built, importing the library raises.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

RCG_OK, RCG_EINVAL, RCG_ENOMEM, RCG_ECUDA, RCG_ETIMEOUT, RCG_EBUSY, RCG_EUNSUPPORTED, RCG_EDEVICE = range(8)
RCG_DEV_TIMEOUT, RCG_DEV_BADPAIR, RCG_DEV_BADJOB = 1, 2, 4
RCG_OP_ENCODE, RCG_OP_RECOVER, RCG_OP_DEGRADED_READ, RCG_OP_UPDATE = range(4)
RCG_COPY_AUTO, RCG_COPY_ROWS = 0, 1
RCG_SOLVE_CHAIN, RCG_SOLVE_TABLE = 0, 1
RCG_NOALLOC_MAX_JOBS = 256
RCG_SHAPE_AUTO, RCG_SHAPE_WIDE, RCG_SHAPE_PAIR = 0, 1, 2
RCG_SCHED_STATIC, RCG_SCHED_DYNAMIC = 0, 1
RCG_COLUMN_AUTO, RCG_COLUMN_OFF = 0, 1
RCG_TABLES_AUTO, RCG_TABLES_DEVICE = 0, 1
RCG_RING_FIXED, RCG_RING_BYTES = 0, 1

_u32, _u64, _vp, _int = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int


class RcgError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = "%s: %s (status %d)" % (what, rcg_status_str(status), status)
        if status == RCG_ECUDA:
            msg += " [%s]" % rcg_last_error()
        super().__init__(msg)
        self.status = status


class rcg_layout(ctypes.Structure):
    _fields_ = [("base", _vp), ("p", _u32), ("n_data", _u32), ("row_bytes", _u64),
                ("row_stride", _u64), ("strip_stride", _u64), ("stripe_stride", _u64)]


class rcg_job(ctypes.Structure):
    _fields_ = [("layout", rcg_layout), ("first_stripe", _u64), ("n_stripes", _u64), ("op", _u32),
                ("i", _u32), ("j", _u32), ("aux", _vp), ("aux_row_stride", _u64),
                ("aux_stripe_stride", _u64)]


class rcg_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", _u64), ("max_inflight_jobs", _u32), ("max_batch_jobs", _u32),
                ("per_job_launches", _u32), ("max_inflight_batches", _u32)]


class rcg_serve_request(ctypes.Structure):
    _fields_ = [("job", rcg_job), ("arrival_ns", _u64), ("footprint_bytes", _u64)]


class rcg_serve_result(ctypes.Structure):
    _fields_ = [("id", _u64), ("arrival_ns", _u64), ("admit_ns", _u64), ("launch_ns", _u64),
                ("complete_ns", _u64), ("status", _u32), ("batch", _u32)]


class rcg_serve_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", _u64), ("completed", _u64), ("conflict_waits", _u64),
                ("max_inflight_launches", _u32), ("max_inflight_jobs", _u32)]


class rcg_plan_info(ctypes.Structure):
    _fields_ = [("tile_bytes", _u32), ("tiles_per_stripe", _u32), ("slot_bytes", _u32), ("n_slots", _u32),
                ("max_items", _u32), ("smem_bytes", _u32), ("ctas_per_sm", _u32), ("shape", _u32)]


class rcg_hlayout(ctypes.Structure):
    _fields_ = [("base", _vp), ("p", _u32), ("n_data", _u32), ("strip_bytes", _u64),
                ("strip_stride", _u64), ("stripe_stride", _u64)]


class rcg_batch_tuning(ctypes.Structure):
    _fields_ = [("shape", _u32), ("schedule", _u32), ("item_bytes", _u64), ("tile_div", _u32),
                ("ring", _u32), ("ms", ctypes.c_float), ("reserved", _u32)]


class rcg_prime_info_t(ctypes.Structure):
    _fields_ = [("ord2", _u32), ("is_field", _u32), ("extends", _u32), ("max_data", _u32)]


EXPORTS = {
    "rcg_create": (_int, [_int, ctypes.POINTER(_vp)]),
    "rcg_destroy": (_int, [_vp]),
    "rcg_set_timeout": (_int, [_vp, _u64]),
    "rcg_set_copy_mode": (_int, [_vp, _int]),
    "rcg_set_dd_solve": (_int, [_vp, _int]),
    "rcg_set_engine_shape": (_int, [_vp, _int]),
    "rcg_set_host_chunk": (_int, [_vp, _u64]),
    "rcg_set_batch_schedule": (_int, [_vp, _int]),
    "rcg_last_device_status": (_int, [_vp, ctypes.POINTER(_u32)]),
    "rcg_status_str": (ctypes.c_char_p, [_int]),
    "rcg_abi_version": (_u32, []),
    "rcg_last_error": (ctypes.c_char_p, []),
    "rcg_encode": (_int, [_vp, ctypes.POINTER(rcg_layout), _u64, _u64, _vp]),
    "rcg_recover": (_int, [_vp, ctypes.POINTER(rcg_layout), _u64, _u32, _u32, _vp]),
    "rcg_recover_many": (_int, [_vp, ctypes.POINTER(rcg_layout), _u64, _u64, _vp, _vp]),
    "rcg_update": (_int, [_vp, ctypes.POINTER(rcg_layout), _u64, _u32, _vp, _u64, _vp]),
    "rcg_degraded_read": (_int, [_vp, ctypes.POINTER(rcg_layout), _u64, _u32, _vp, _u64, _vp]),
    "rcg_encode_host": (_int, [_vp, ctypes.POINTER(rcg_layout), _u64, _u64, _vp]),
    "rcg_recover_many_host": (_int, [_vp, ctypes.POINTER(rcg_layout), _u64, _u64, _vp, _vp]),
    "rcg_batch_submit": (_int, [_vp, ctypes.POINTER(rcg_job), _u32, _vp, ctypes.POINTER(_u64)]),
    "rcg_batch_wait": (_int, [_vp, _u64, _u64]),
    "rcg_batch_prepare": (_int, [_vp, ctypes.POINTER(rcg_job), _u32, ctypes.POINTER(_vp)]),
    "rcg_batch_launch": (_int, [_vp, _vp, _vp, ctypes.POINTER(_u64)]),
    "rcg_batch_free": (_int, [_vp]),
    "rcg_serve_create": (_int, [_vp, ctypes.POINTER(rcg_serve_config), ctypes.POINTER(_vp)]),
    "rcg_serve_submit": (_int, [_vp, ctypes.POINTER(rcg_serve_request), _u32, ctypes.POINTER(_u64)]),
    "rcg_serve_start": (_int, [_vp]),
    "rcg_serve_drain": (_int, [_vp, _u64]),
    "rcg_serve_results": (_int, [_vp, ctypes.POINTER(rcg_serve_result), _u64, ctypes.POINTER(_u64)]),
    "rcg_serve_get_stats": (_int, [_vp, ctypes.POINTER(rcg_serve_stats)]),
    "rcg_serve_destroy": (_int, [_vp]),
    "rcg_batch_submit_noalloc": (_int, [ctypes.POINTER(rcg_job), _u32, _vp, _vp]),
    "rcg_fill_random": (_int, [_vp, _u64, _u64, _u64, _vp]),
    "rcg_selftest_wait_timeout": (_int, [_vp, _u64, _vp]),
    "rcg_inverse_table": (_int, [_u32, ctypes.POINTER(_u64)]),
    "rcg_plan": (_int, [_u32, _u64, ctypes.POINTER(rcg_plan_info)]),
    "rcg_prime_info": (_int, [_u32, ctypes.POINTER(rcg_prime_info_t)]),
    "rcg_set_column_kernel": (_int, [_vp, _int]),
    "rcg_set_batch_tables": (_int, [_vp, _int]),
    "rcg_batch_autotune": (_int, [_vp, _vp, _u32, _vp, ctypes.POINTER(rcg_batch_tuning)]),
    "rcg_set_batch_tuning": (_int, [_vp, ctypes.POINTER(rcg_batch_tuning)]),
    "rcg_h_encode": (_int, [_vp, ctypes.POINTER(rcg_hlayout), _u64, _u64, _vp]),
    "rcg_h_recover": (_int, [_vp, ctypes.POINTER(rcg_hlayout), _u64, _u32, _u32, _vp]),
    "rcg_h_recover_many": (_int, [_vp, ctypes.POINTER(rcg_hlayout), _u64, _u64, _vp, _vp]),
    "rcg_ring_inverse": (_int, [_u32, _u64, ctypes.POINTER(_u64)]),
}

_lib: ctypes.CDLL | None = None


def lib(path: str | None = None) -> ctypes.CDLL:
    """Load librcg.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        path = path or LIB
        if not os.path.exists(path):
            raise ImportError("librcg.so is not built (%s); run paper_cs_0611109_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != RCG_OK:
        raise RcgError(st, what)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def make_layout(base, p: int, n_data: int, row_bytes: int, row_stride: int = 0,
                strip_stride: int = 0, stripe_stride: int = 0) -> rcg_layout:
    """Describe stripes at device address `base` (tensor or int); zero strides = packed."""
    return rcg_layout(_ptr(base), p, n_data, row_bytes, row_stride, strip_stride, stripe_stride)


def make_hlayout(base, p: int, n_data: int, strip_bytes: int, strip_stride: int = 0,
                 stripe_stride: int = 0) -> rcg_hlayout:
    """Describe stripes in the horizontal representation (one ring element per
    (p-1)-bit field) at device address `base`; zero strides = packed."""
    return rcg_hlayout(_ptr(base), p, n_data, strip_bytes, strip_stride, stripe_stride)


# ------------------------------------------------------------- the C calls

def rcg_status_str(st: int) -> str:
    try:
        return lib().rcg_status_str(st).decode()
    except ImportError:
        return "status %d" % st


def rcg_last_error() -> str:
    try:
        return lib().rcg_last_error().decode()
    except ImportError:
        return ""


def rcg_abi_version() -> int:
    return int(lib().rcg_abi_version())


def rcg_create(device: int = 0) -> int:
    h = _vp()
    _check(lib().rcg_create(device, ctypes.byref(h)), "rcg_create")
    return h.value


def rcg_destroy(ctx: int):
    _check(lib().rcg_destroy(ctx), "rcg_destroy")


def rcg_set_timeout(ctx: int, timeout_ns: int):
    _check(lib().rcg_set_timeout(ctx, timeout_ns), "rcg_set_timeout")


def rcg_set_copy_mode(ctx: int, mode: int):
    _check(lib().rcg_set_copy_mode(ctx, mode), "rcg_set_copy_mode")


def rcg_set_dd_solve(ctx: int, solve: int):
    _check(lib().rcg_set_dd_solve(ctx, solve), "rcg_set_dd_solve")


def rcg_set_engine_shape(ctx: int, shape: int):
    _check(lib().rcg_set_engine_shape(ctx, shape), "rcg_set_engine_shape")


def rcg_batch_autotune(ctx: int, jobs, stream=None) -> dict:
    """Tune the batch layout on a real job list (see include/rcg.h) and apply it."""
    arr = (rcg_job * len(jobs))(*jobs)
    t = rcg_batch_tuning()
    _check(lib().rcg_batch_autotune(ctx, arr, len(jobs), _stream(stream), ctypes.byref(t)), "rcg_batch_autotune")
    return {f: (float(getattr(t, f)) if f == "ms" else int(getattr(t, f))) for f, _ in rcg_batch_tuning._fields_
            if f != "reserved"}


def rcg_set_batch_tuning(ctx: int, tuning: dict | None):
    if tuning is None:
        _check(lib().rcg_set_batch_tuning(ctx, None), "rcg_set_batch_tuning")
        return
    t = rcg_batch_tuning(tuning["shape"], tuning["schedule"], tuning["item_bytes"], tuning["tile_div"],
                         tuning.get("ring", RCG_RING_FIXED), tuning.get("ms", 0.0), 0)
    _check(lib().rcg_set_batch_tuning(ctx, ctypes.byref(t)), "rcg_set_batch_tuning")


def tuning_key(device: int = 0) -> str:
    """Cache key of a tuning: the GPU model and its SM count."""
    import torch
    prop = torch.cuda.get_device_properties(device)
    return "%s/%d" % (prop.name, prop.multi_processor_count)


def save_tuning(path: str, tuning: dict, device: int = 0):
    """Store a tuning in a JSON file under this GPU's key (other keys kept)."""
    import json
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    cache[tuning_key(device)] = tuning
    with open(path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)


def load_tuning(path: str, device: int = 0) -> dict | None:
    """The tuning stored for this GPU's key, or None."""
    import json
    try:
        with open(path) as f:
            return json.load(f).get(tuning_key(device))
    except (OSError, ValueError):
        return None


def rcg_set_column_kernel(ctx: int, mode: int):
    _check(lib().rcg_set_column_kernel(ctx, mode), "rcg_set_column_kernel")


def rcg_set_batch_tables(ctx: int, mode: int):
    _check(lib().rcg_set_batch_tables(ctx, mode), "rcg_set_batch_tables")


def rcg_set_host_chunk(ctx: int, nbytes: int):
    _check(lib().rcg_set_host_chunk(ctx, nbytes), "rcg_set_host_chunk")


def rcg_set_batch_schedule(ctx: int, schedule: int):
    _check(lib().rcg_set_batch_schedule(ctx, schedule), "rcg_set_batch_schedule")


def rcg_last_device_status(ctx: int) -> int:
    """Synchronise, return and clear the device status word (RCG_DEV_* bits)."""
    code = _u32(0)
    st = lib().rcg_last_device_status(ctx, ctypes.byref(code))
    if st not in (RCG_OK, RCG_EDEVICE):
        _check(st, "rcg_last_device_status")
    return int(code.value)


def rcg_encode(ctx: int, layout: rcg_layout, first_stripe: int, n_stripes: int, stream=None):
    _check(lib().rcg_encode(ctx, ctypes.byref(layout), first_stripe, n_stripes, _stream(stream)),
           "rcg_encode")


def rcg_recover(ctx: int, layout: rcg_layout, stripe: int, i: int, j: int, stream=None):
    _check(lib().rcg_recover(ctx, ctypes.byref(layout), stripe, i, j, _stream(stream)), "rcg_recover")


def rcg_recover_many(ctx: int, layout: rcg_layout, first_stripe: int, n_stripes: int, pairs,
                     stream=None):
    """pairs: device uint8 tensor [n_stripes, 2] (or address) of per-stripe (i, j)."""
    _check(lib().rcg_recover_many(ctx, ctypes.byref(layout), first_stripe, n_stripes, _ptr(pairs),
                                  _stream(stream)), "rcg_recover_many")


def rcg_update(ctx: int, layout: rcg_layout, stripe: int, i: int, new_strip, new_row_stride: int = 0,
               stream=None):
    _check(lib().rcg_update(ctx, ctypes.byref(layout), stripe, i, _ptr(new_strip), new_row_stride,
                            _stream(stream)), "rcg_update")


def rcg_degraded_read(ctx: int, layout: rcg_layout, stripe: int, j: int, out, out_row_stride: int = 0,
                      stream=None):
    _check(lib().rcg_degraded_read(ctx, ctypes.byref(layout), stripe, j, _ptr(out), out_row_stride,
                                   _stream(stream)), "rcg_degraded_read")


def rcg_encode_host(ctx: int, layout: rcg_layout, first_stripe: int, n_stripes: int, stream=None):
    """rcg_encode for stripes in page-locked host memory (layout.base = host address)."""
    _check(lib().rcg_encode_host(ctx, ctypes.byref(layout), first_stripe, n_stripes, _stream(stream)),
           "rcg_encode_host")


def rcg_recover_many_host(ctx: int, layout: rcg_layout, first_stripe: int, n_stripes: int, pairs,
                          stream=None):
    """rcg_recover_many for stripes in page-locked host memory; pairs is a HOST
    uint8 array (numpy or CPU tensor) of shape [n_stripes, 2]."""
    if hasattr(pairs, "ctypes"):
        ptr = pairs.ctypes.data
    else:
        ptr = _ptr(pairs)
    _check(lib().rcg_recover_many_host(ctx, ctypes.byref(layout), first_stripe, n_stripes, ptr,
                                       _stream(stream)), "rcg_recover_many_host")


def make_job(layout: rcg_layout, first_stripe: int, n_stripes: int, op: int, i: int = 0, j: int = 0,
             aux=None, aux_row_stride: int = 0, aux_stripe_stride: int = 0) -> rcg_job:
    return rcg_job(layout, first_stripe, n_stripes, op, i, j, _ptr(aux), aux_row_stride,
                   aux_stripe_stride)


def rcg_batch_submit(ctx: int, jobs, stream=None) -> int:
    arr = (rcg_job * len(jobs))(*jobs)
    ticket = _u64(0)
    _check(lib().rcg_batch_submit(ctx, arr, len(jobs), _stream(stream), ctypes.byref(ticket)),
           "rcg_batch_submit")
    return int(ticket.value)


def rcg_batch_prepare(ctx: int, jobs) -> int:
    """Host half of rcg_batch_submit: returns an opaque prepared-batch handle."""
    arr = (rcg_job * max(1, len(jobs)))(*jobs)
    h = _vp()
    _check(lib().rcg_batch_prepare(ctx, arr, len(jobs), ctypes.byref(h)), "rcg_batch_prepare")
    return h.value


def rcg_batch_launch(ctx: int, batch: int, stream=None) -> int:
    ticket = _u64(0)
    _check(lib().rcg_batch_launch(ctx, batch, _stream(stream), ctypes.byref(ticket)), "rcg_batch_launch")
    return int(ticket.value)


def rcg_batch_free(batch: int):
    _check(lib().rcg_batch_free(batch), "rcg_batch_free")


def rcg_serve_create(ctx: int, hbm_budget_bytes=0, max_inflight_jobs=0, max_batch_jobs=0,
                     per_job_launches=False, max_inflight_batches=0) -> int:
    cfg = rcg_serve_config(hbm_budget_bytes, max_inflight_jobs, max_batch_jobs, 1 if per_job_launches else 0,
                           max_inflight_batches)
    h = _vp()
    _check(lib().rcg_serve_create(ctx, ctypes.byref(cfg), ctypes.byref(h)), "rcg_serve_create")
    return h.value


def rcg_serve_submit(server: int, jobs, arrivals_ns, footprints=None) -> int:
    n = len(jobs)
    arr = (rcg_serve_request * max(1, n))()
    for k in range(n):
        arr[k] = rcg_serve_request(jobs[k], int(arrivals_ns[k]), int(footprints[k]) if footprints is not None else 0)
    first = _u64(0)
    _check(lib().rcg_serve_submit(server, arr, n, ctypes.byref(first)), "rcg_serve_submit")
    return int(first.value)


def rcg_serve_start(server: int):
    _check(lib().rcg_serve_start(server), "rcg_serve_start")


def rcg_serve_drain(server: int, timeout_ns: int = 60 * 10 ** 9):
    _check(lib().rcg_serve_drain(server, timeout_ns), "rcg_serve_drain")


def rcg_serve_results(server: int, n: int):
    """Timings of the first n requests as a list of dicts."""
    arr = (rcg_serve_result * max(1, n))()
    got = _u64(0)
    _check(lib().rcg_serve_results(server, arr, n, ctypes.byref(got)), "rcg_serve_results")
    return [{f: int(getattr(arr[k], f)) for f, _ in rcg_serve_result._fields_} for k in range(int(got.value))]


def rcg_serve_get_stats(server: int) -> dict:
    """Kernel launches issued, requests completed, conflict waits, and the most
    launches / requests in flight at once."""
    st = rcg_serve_stats()
    _check(lib().rcg_serve_get_stats(server, ctypes.byref(st)), "rcg_serve_get_stats")
    return {f: int(getattr(st, f)) for f, _ in rcg_serve_stats._fields_}


def rcg_serve_destroy(server: int):
    _check(lib().rcg_serve_destroy(server), "rcg_serve_destroy")


def rcg_batch_submit_noalloc(jobs, status_dev=None, stream=None):
    """rcg_batch_submit without a context and without allocating device memory
    (scratch in a fixed device array; at most RCG_NOALLOC_MAX_JOBS jobs).
    status_dev: optional caller-owned device uint32 that receives RCG_DEV_* bits."""
    arr = (rcg_job * max(1, len(jobs)))(*jobs)
    _check(lib().rcg_batch_submit_noalloc(arr, len(jobs), _ptr(status_dev), _stream(stream)),
           "rcg_batch_submit_noalloc")


def rcg_batch_wait(ctx: int, ticket: int, timeout_ns: int = 10 ** 10) -> bool:
    """True when the batch finished, False on RCG_ETIMEOUT."""
    st = lib().rcg_batch_wait(ctx, ticket, timeout_ns)
    if st == RCG_ETIMEOUT:
        return False
    _check(st, "rcg_batch_wait")
    return True


def rcg_fill_random(dev, nbytes: int, seed: int, byte_offset: int = 0, stream=None):
    _check(lib().rcg_fill_random(_ptr(dev), nbytes, seed, byte_offset, _stream(stream)),
           "rcg_fill_random")


def rcg_selftest_wait_timeout(ctx: int, timeout_ns: int, stream=None):
    _check(lib().rcg_selftest_wait_timeout(ctx, timeout_ns, _stream(stream)), "rcg_selftest_wait_timeout")


def rcg_inverse_table(p: int) -> list[int]:
    masks = (_u64 * p)()
    _check(lib().rcg_inverse_table(p, masks), "rcg_inverse_table")
    return [int(m) for m in masks]


def rcg_h_encode(ctx: int, layout: rcg_hlayout, first_stripe: int, n_stripes: int, stream=None):
    _check(lib().rcg_h_encode(ctx, ctypes.byref(layout), first_stripe, n_stripes, _stream(stream)), "rcg_h_encode")


def rcg_h_recover(ctx: int, layout: rcg_hlayout, stripe: int, i: int, j: int, stream=None):
    _check(lib().rcg_h_recover(ctx, ctypes.byref(layout), stripe, i, j, _stream(stream)), "rcg_h_recover")


def rcg_h_recover_many(ctx: int, layout: rcg_hlayout, first_stripe: int, n_stripes: int, pairs, stream=None):
    _check(lib().rcg_h_recover_many(ctx, ctypes.byref(layout), first_stripe, n_stripes, _ptr(pairs),
                                    _stream(stream)), "rcg_h_recover_many")


def rcg_prime_info(p: int) -> dict:
    """ord2 (Lemma 3.3.1), is_field, extends (Theorem 3.3.3) and max_data for p."""
    info = rcg_prime_info_t()
    _check(lib().rcg_prime_info(p, ctypes.byref(info)), "rcg_prime_info")
    return {f: int(getattr(info, f)) for f, _ in rcg_prime_info_t._fields_}


def rcg_ring_inverse(p: int, a: int) -> int:
    """Inverse of a (bit m = coefficient of x^m) in F2[x]/(1 + ... + x^(p-1))."""
    inv = _u64()
    _check(lib().rcg_ring_inverse(p, a, ctypes.byref(inv)), "rcg_ring_inverse")
    return int(inv.value)


def rcg_plan(p: int, row_bytes: int) -> dict:
    info = rcg_plan_info()
    _check(lib().rcg_plan(p, row_bytes, ctypes.byref(info)), "rcg_plan")
    return {f: int(getattr(info, f)) for f, _ in rcg_plan_info._fields_}


class Context:
    """Owns an rcg_ctx; methods forward to the C calls above."""

    def __init__(self, device: int = 0):
        self.handle = rcg_create(device)

    def close(self):
        if self.handle:
            rcg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def encode(self, layout, first_stripe, n_stripes, stream=None):
        rcg_encode(self.handle, layout, first_stripe, n_stripes, stream)

    def recover(self, layout, stripe, i, j, stream=None):
        rcg_recover(self.handle, layout, stripe, i, j, stream)

    def recover_many(self, layout, first_stripe, n_stripes, pairs, stream=None):
        rcg_recover_many(self.handle, layout, first_stripe, n_stripes, pairs, stream)

    def encode_host(self, layout, first_stripe, n_stripes, stream=None):
        rcg_encode_host(self.handle, layout, first_stripe, n_stripes, stream)

    def recover_many_host(self, layout, first_stripe, n_stripes, pairs, stream=None):
        rcg_recover_many_host(self.handle, layout, first_stripe, n_stripes, pairs, stream)

    def update(self, layout, stripe, i, new_strip, new_row_stride=0, stream=None):
        rcg_update(self.handle, layout, stripe, i, new_strip, new_row_stride, stream)

    def h_encode(self, layout, first_stripe, n_stripes, stream=None):
        rcg_h_encode(self.handle, layout, first_stripe, n_stripes, stream)

    def h_recover(self, layout, stripe, i, j, stream=None):
        rcg_h_recover(self.handle, layout, stripe, i, j, stream)

    def h_recover_many(self, layout, first_stripe, n_stripes, pairs, stream=None):
        rcg_h_recover_many(self.handle, layout, first_stripe, n_stripes, pairs, stream)

    def degraded_read(self, layout, stripe, j, out, out_row_stride=0, stream=None):
        rcg_degraded_read(self.handle, layout, stripe, j, out, out_row_stride, stream)

    def batch_submit(self, jobs, stream=None) -> int:
        return rcg_batch_submit(self.handle, jobs, stream)

    def batch_wait(self, ticket, timeout_ns=10 ** 10) -> bool:
        return rcg_batch_wait(self.handle, ticket, timeout_ns)

    def batch_prepare(self, jobs) -> int:
        return rcg_batch_prepare(self.handle, jobs)

    def batch_launch(self, batch, stream=None) -> int:
        return rcg_batch_launch(self.handle, batch, stream)

    def set_timeout(self, timeout_ns):
        rcg_set_timeout(self.handle, timeout_ns)

    def set_copy_mode(self, mode):
        rcg_set_copy_mode(self.handle, mode)

    def set_dd_solve(self, solve):
        rcg_set_dd_solve(self.handle, solve)

    def set_engine_shape(self, shape):
        rcg_set_engine_shape(self.handle, shape)

    def set_host_chunk(self, nbytes):
        rcg_set_host_chunk(self.handle, nbytes)

    def batch_autotune(self, jobs, stream=None) -> dict:
        return rcg_batch_autotune(self.handle, jobs, stream)

    def set_batch_tuning(self, tuning):
        rcg_set_batch_tuning(self.handle, tuning)

    def set_column_kernel(self, mode):
        rcg_set_column_kernel(self.handle, mode)

    def set_batch_tables(self, mode):
        rcg_set_batch_tables(self.handle, mode)

    def set_batch_schedule(self, schedule):
        rcg_set_batch_schedule(self.handle, schedule)

    def last_device_status(self) -> int:
        return rcg_last_device_status(self.handle)
