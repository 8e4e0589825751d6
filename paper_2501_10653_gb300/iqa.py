"""Thin ctypes binding of ``libiqa.so`` (declared in ``include/iqa.h``).

Argument marshalling only: every step of the map computation runs in the
library's CUDA kernels.  Functions keep the C names.  Pointer arguments accept
an int address or any object with ``data_ptr()`` (a torch tensor); stream
arguments accept an int handle, ``None`` (legacy default stream) or an object
with a ``cuda_stream`` attribute (``torch.cuda.Stream``).  A non-OK status
raises ``IqaError`` carrying the status and ``iqa_last_error``.

The library must have been built (``paper_2501_10653_gb300.build.build()``);
there is no fallback: loading fails loudly if it is missing.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# IQA_LIBRARY selects another build of the same ABI (the tests use it for the
# bounds-checked libiqa_checked.so); the default is the product library.
LIB_PATH = os.environ.get("IQA_LIBRARY") or os.path.join(_HERE, "libiqa.so")

IQA_OK = 0
IQA_PENDING = 1
IQA_ERR_INVALID_ARG = -1
IQA_ERR_NOMEM = -2
IQA_ERR_CUDA = -3
IQA_ERR_TIMEOUT = -4
IQA_ERR_BUSY = -5
IQA_ERR_UNSUPPORTED = -6

IQA_F32 = 0
IQA_F16 = 1
IQA_BF16 = 2

MAPS_LISI = 1
MAPS_AUGLISI = 2
MAPS_BOTH = 3

STATUS_NAMES = {
    0: "IQA_OK", 1: "IQA_PENDING", -1: "IQA_ERR_INVALID_ARG", -2: "IQA_ERR_NOMEM",
    -3: "IQA_ERR_CUDA", -4: "IQA_ERR_TIMEOUT", -5: "IQA_ERR_BUSY",
    -6: "IQA_ERR_UNSUPPORTED",
}


class IqaError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))


class iqa_params(ctypes.Structure):
    _fields_ = [("C1", ctypes.c_double), ("C2", ctypes.c_double),
                ("C", ctypes.c_double), ("D", ctypes.c_double)]

    def as_dict(self):
        return {"C1": self.C1, "C2": self.C2, "C": self.C, "D": self.D}


class iqa_launch_config(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("threads", ctypes.c_int),
                ("ilp", ctypes.c_int), ("tiles_across", ctypes.c_int),
                ("split", ctypes.c_int), ("vector", ctypes.c_int),
                ("stages", ctypes.c_int), ("stage_kb", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("unit_kpx", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class iqa_pair(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("N", ctypes.c_int),
                ("NT", ctypes.c_int), ("lisi_map", ctypes.c_void_p),
                ("aug_map", ctypes.c_void_p), ("sums", ctypes.c_void_p)]


class iqa_host_pair(ctypes.Structure):
    _fields_ = [("hx", ctypes.c_void_p), ("hy", ctypes.c_void_p), ("N", ctypes.c_int),
                ("NT", ctypes.c_int), ("lisi_map", ctypes.c_void_p),
                ("aug_map", ctypes.c_void_p), ("sums", ctypes.c_void_p)]


class iqa_catalog(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("nsrc", ctypes.c_int),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("flux", ctypes.c_void_p),
                ("half", ctypes.c_void_p), ("profile_off", ctypes.c_void_p),
                ("profile", ctypes.c_void_p), ("nprofile", ctypes.c_int),
                ("noise_sigma", ctypes.c_float)]


class iqa_server_config(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("max_pairs_per_step", ctypes.c_int),
                ("max_inflight_steps", ctypes.c_int), ("pool_bytes", ctypes.c_size_t),
                ("one_pair_per_launch", ctypes.c_int), ("simulate", ctypes.c_int),
                ("sim_bytes_per_s", ctypes.c_double), ("step_timeout_ms", ctypes.c_double),
                ("max_step_bytes", ctypes.c_ulonglong), ("params", iqa_params),
                ("generator_blocks_per_sm", ctypes.c_int), ("map_ctas_per_sm", ctypes.c_int),
                ("time_kernels", ctypes.c_int)]


class iqa_request(ctypes.Structure):
    _fields_ = [("ref_id", ctypes.c_int), ("NT", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("ndrop", ctypes.c_int),
                ("drop", ctypes.c_int * 8), ("add_src", ctypes.c_int),
                ("add_x", ctypes.c_int), ("add_y", ctypes.c_int),
                ("add_flux", ctypes.c_float)]


class iqa_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("pending", ctypes.c_longlong),
                ("inflight", ctypes.c_longlong), ("steps", ctypes.c_longlong),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("pairs_per_s", ctypes.c_double), ("input_gb_per_s", ctypes.c_double),
                ("mean_pairs_per_step", ctypes.c_double),
                ("pool_bytes", ctypes.c_ulonglong), ("pool_peak_bytes", ctypes.c_ulonglong),
                ("p50_queue_ms", ctypes.c_double), ("p50_launch_ms", ctypes.c_double),
                ("p50_device_ms", ctypes.c_double),
                ("mean_step_generator_ms", ctypes.c_double),
                ("mean_step_map_ms", ctypes.c_double),
                ("generator_ms_per_pair", ctypes.c_double),
                ("map_ms_per_pair", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class iqa_plan_stats(ctypes.Structure):
    _fields_ = [("npairs", ctypes.c_int), ("total_units", ctypes.c_longlong),
                ("grid", ctypes.c_int), ("input_bytes", ctypes.c_ulonglong),
                ("graph", ctypes.c_int), ("config", iqa_launch_config)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "config"}
        d["config"] = self.config.as_dict()
        return d


IQA_PLAN_GRAPH = 1
IQA_PLAN_INDEPENDENT = 2
IQA_NOALLOC_MAX_PAIRS = 64
IQA_OPT_WAIT_TIMEOUT_US = 1
IQA_OPT_INJECT_STALL = 2
IQA_OPT_INDEPENDENT_CALLS = 3

_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_sz = ctypes.c_size_t
_st = ctypes.c_int


def _declare(lib):
    P = ctypes.POINTER
    sig = {
        "iqa_version": ([], ctypes.c_char_p),
        "iqa_default_params": ([P(iqa_params)], _st),
        "iqa_create": ([P(_vp), _i, _sz], _st),
        "iqa_destroy": ([_vp], None),
        "iqa_last_error": ([_vp], ctypes.c_char_p),
        "iqa_lisi": ([_vp, _vp, _vp, _i, _i, _i, P(iqa_params), _vp, _vp, _vp], _st),
        "iqa_auglisi": ([_vp, _vp, _vp, _i, _i, _i, P(iqa_params), _vp, _vp, _vp], _st),
        "iqa_both": ([_vp, _vp, _vp, _i, _i, _i, P(iqa_params), _vp, _vp, _vp, _vp], _st),
        "iqa_both_host": ([_vp, _vp, _vp, _i, _i, _i, P(iqa_params), _vp, _vp, _vp], _st),
        "iqa_get_config": ([_vp, _i, _i, _i, _i, P(iqa_launch_config)], _st),
        "iqa_set_config": ([_vp, _i, _i, _i, _i, P(iqa_launch_config)], _st),
        "iqa_wait": ([_vp, _vp, _i], _st),
        "iqa_debug_violations": ([P(ctypes.c_ulonglong)], _st),
        "iqa_set_option": ([_vp, _i, ctypes.c_longlong], _st),
        "iqa_plan_create": ([_vp, P(iqa_pair), _i, _i, P(iqa_params), _i, P(_vp)], _st),
        "iqa_plan_launch": ([_vp, _vp], _st),
        "iqa_plan_destroy": ([_vp], None),
        "iqa_plan_info": ([_vp, P(iqa_plan_stats)], _st),
        "iqa_plan_autotune": ([_vp, _vp, _i, P(iqa_launch_config)], _st),
        "iqa_plan_set_config": ([_vp, P(iqa_launch_config)], _st),
        "iqa_plan_unit_shape": ([_i, _i, _i, P(iqa_launch_config), P(ctypes.c_int),
                                 P(ctypes.c_int), P(ctypes.c_longlong)], _st),
        "iqa_batch_noalloc": ([P(iqa_pair), _i, _i, P(iqa_params), _vp], _st),
        "iqa_merge": ([_vp, _vp, _i, _i, P(iqa_params), _vp, _vp, _vp, _vp], _st),
        "iqa_both_host_many": ([_vp, P(iqa_host_pair), _i, _i, P(iqa_params)], _st),
        "iqa_server_create": ([_vp, P(iqa_server_config), P(_vp)], _st),
        "iqa_server_add_reference": ([_vp, _i, P(iqa_catalog), ctypes.c_ulonglong], _st),
        "iqa_server_reference_image": ([_vp, _i, _vp], _st),
        "iqa_submit": ([_vp, P(iqa_request), P(ctypes.c_ulonglong)], _st),
        "iqa_poll": ([_vp, ctypes.c_ulonglong, _i], _st),
        "iqa_result": ([_vp, ctypes.c_ulonglong, _vp, _vp, P(ctypes.c_double)], _st),
        "iqa_server_get_stats": ([_vp, P(iqa_server_stats)], _st),
        "iqa_server_destroy": ([_vp], None),
        "iqa_server_run_trace": ([_vp, P(iqa_request), P(ctypes.c_double), _i,
                                  ctypes.c_double], _st),
        "iqa_render_epoch": ([_vp, P(iqa_catalog), ctypes.c_ulonglong, P(_i), _i, _i, _i,
                              _i, ctypes.c_float, _i, _vp], _st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "libiqa.so is not built (expected at %s); run "
                "paper_2501_10653_gb300.build.build() -- there is no CPU fallback"
                % LIB_PATH)
        _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def _ptr(p):
    if p is None:
        return None
    if isinstance(p, int):
        return p
    if hasattr(p, "data_ptr"):
        return p.data_ptr()
    if hasattr(p, "ctypes"):  # numpy array (host path)
        return p.ctypes.data
    raise TypeError("expected an address, a tensor or an array, got %r" % type(p))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(ctx, status):
    if status != IQA_OK:
        msg = lib().iqa_last_error(ctx)
        raise IqaError(status, msg.decode() if msg else "")
    return status


def _params(p):
    if p is None:
        return None
    if isinstance(p, iqa_params):
        return ctypes.byref(p)
    if isinstance(p, dict):
        return ctypes.byref(iqa_params(p.get("C1", 1e-6), p.get("C2", 1e-6),
                                       p.get("C", 1e-6), p.get("D", 0.0)))
    raise TypeError("params must be iqa_params, a dict or None")


def iqa_version():
    return lib().iqa_version().decode()


def iqa_default_params():
    p = iqa_params()
    _check(None, lib().iqa_default_params(ctypes.byref(p)))
    return p


def iqa_create(device=0, hbm_budget_bytes=0):
    h = _vp()
    _check(None, lib().iqa_create(ctypes.byref(h), int(device), int(hbm_budget_bytes)))
    return h.value


def iqa_destroy(ctx):
    lib().iqa_destroy(ctx)


def iqa_last_error(ctx):
    m = lib().iqa_last_error(ctx)
    return m.decode() if m else ""


def iqa_lisi(ctx, x, y, dtype, N, NT, params, map, sums=None, stream=None):
    return _check(ctx, lib().iqa_lisi(ctx, _ptr(x), _ptr(y), dtype, N, NT,
                                      _params(params), _ptr(map), _ptr(sums),
                                      _stream(stream)))


def iqa_auglisi(ctx, x, y, dtype, N, NT, params, map, sums=None, stream=None):
    return _check(ctx, lib().iqa_auglisi(ctx, _ptr(x), _ptr(y), dtype, N, NT,
                                         _params(params), _ptr(map), _ptr(sums),
                                         _stream(stream)))


def iqa_both(ctx, x, y, dtype, N, NT, params, lisi_map, aug_map, sums=None,
             stream=None):
    return _check(ctx, lib().iqa_both(ctx, _ptr(x), _ptr(y), dtype, N, NT,
                                      _params(params), _ptr(lisi_map),
                                      _ptr(aug_map), _ptr(sums), _stream(stream)))


def iqa_both_host(ctx, hx, hy, dtype, N, NT, params, lisi_map, aug_map, sums=None):
    return _check(ctx, lib().iqa_both_host(ctx, _ptr(hx), _ptr(hy), dtype, N, NT,
                                           _params(params), _ptr(lisi_map),
                                           _ptr(aug_map), _ptr(sums)))


def iqa_get_config(ctx, dtype, N, NT, maps):
    c = iqa_launch_config()
    _check(ctx, lib().iqa_get_config(ctx, dtype, N, NT, maps, ctypes.byref(c)))
    return c


def iqa_set_config(ctx, dtype, N, NT, maps, cfg):
    if cfg is None:
        ref = None
    else:
        if isinstance(cfg, dict):
            full = {"variant": 0, "threads": 256, "ilp": 4, "tiles_across": 1,
                    "split": 1, "vector": 1, "stages": 8, "stage_kb": 8,
                    "ctas_per_sm": 1, "unit_kpx": 16}
            full.update(cfg)
            cfg = iqa_launch_config(**full)
        ref = ctypes.byref(cfg)
    return _check(ctx, lib().iqa_set_config(ctx, dtype, N, NT, maps, ref))


def iqa_debug_violations():
    """Failed bounds checks since the last call (checked build only)."""
    n = ctypes.c_ulonglong(0)
    _check(None, lib().iqa_debug_violations(ctypes.byref(n)))
    return n.value


def iqa_wait(ctx, stream=None, timeout_us=-1):
    return _check(ctx, lib().iqa_wait(ctx, _stream(stream), int(timeout_us)))


def iqa_set_option(ctx, option, value):
    return _check(ctx, lib().iqa_set_option(ctx, int(option), int(value)))


def make_pair(x, y, N, NT, lisi_map=None, aug_map=None, sums=None):
    """An iqa_pair from tensors / addresses (marshalling helper)."""
    return iqa_pair(_ptr(x), _ptr(y), int(N), int(NT), _ptr(lisi_map), _ptr(aug_map),
                    _ptr(sums))


class _Plan:
    """Owner of an iqa_plan handle; keeps the pair array alive."""

    def __init__(self, ctx, handle, pairs):
        self.ctx = ctx
        self.handle = handle
        self._pairs = pairs

    def __int__(self):
        return self.handle


def iqa_plan_create(ctx, pairs, dtype, params=None, flags=IQA_PLAN_GRAPH):
    arr = (iqa_pair * len(pairs))(*pairs)
    h = _vp()
    _check(ctx, lib().iqa_plan_create(ctx, arr, len(pairs), int(dtype), _params(params),
                                      int(flags), ctypes.byref(h)))
    return _Plan(ctx, h.value, arr)


def iqa_plan_launch(plan, stream=None):
    return _check(plan.ctx, lib().iqa_plan_launch(plan.handle, _stream(stream)))


def iqa_plan_destroy(plan):
    if plan.handle:
        lib().iqa_plan_destroy(plan.handle)
        plan.handle = None


def iqa_plan_info(plan):
    st = iqa_plan_stats()
    _check(plan.ctx, lib().iqa_plan_info(plan.handle, ctypes.byref(st)))
    return st


def iqa_plan_set_config(plan, cfg):
    """Variant 1 shape for the plan (an iqa_launch_config, or a dict of its
    fields: threads, stages, stage_kb, ctas_per_sm, unit_kpx)."""
    if isinstance(cfg, dict):
        full = {"variant": 1, "threads": 128, "ilp": 0, "tiles_across": 0, "split": 1,
                "vector": 1, "stages": 2, "stage_kb": 16, "ctas_per_sm": 3, "unit_kpx": 16}
        full.update(cfg)
        cfg = iqa_launch_config(**full)
    _check(plan.ctx, lib().iqa_plan_set_config(plan.handle, ctypes.byref(cfg)))


def iqa_plan_unit_shape(dtype, N, NT, cfg):
    """(tiles_across, tile_rows, units) of one pair in a plan of shape cfg (an
    iqa_launch_config, or a dict of its variant 1 fields); host-only."""
    if isinstance(cfg, dict):
        full = {"variant": 1, "threads": 128, "ilp": 0, "tiles_across": 0, "split": 1,
                "vector": 1, "stages": 2, "stage_kb": 16, "ctas_per_sm": 3, "unit_kpx": 32}
        full.update(cfg)
        cfg = iqa_launch_config(**full)
    tx, rh, units = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check(None, lib().iqa_plan_unit_shape(int(dtype), int(N), int(NT), ctypes.byref(cfg),
                                           ctypes.byref(tx), ctypes.byref(rh),
                                           ctypes.byref(units)))
    return tx.value, rh.value, units.value


def iqa_plan_autotune(plan, stream=None, iters=5):
    best = iqa_launch_config()
    _check(plan.ctx, lib().iqa_plan_autotune(plan.handle, _stream(stream), int(iters),
                                             ctypes.byref(best)))
    return best


def iqa_batch_noalloc(pairs, dtype, params=None, stream=None):
    """Batched launch that allocates no device memory (see include/iqa.h)."""
    arr = (iqa_pair * len(pairs))(*pairs)
    return _check(None, lib().iqa_batch_noalloc(arr, len(pairs), int(dtype),
                                                _params(params), _stream(stream)))


def iqa_merge(ctx, sums, T, m, params, merged_lisi, merged_aug, merged_sums=None,
              stream=None):
    return _check(ctx, lib().iqa_merge(ctx, _ptr(sums), int(T), int(m), _params(params),
                                       _ptr(merged_lisi), _ptr(merged_aug),
                                       _ptr(merged_sums), _stream(stream)))


def make_host_pair(hx, hy, N, NT, lisi_map=None, aug_map=None, sums=None):
    return iqa_host_pair(_ptr(hx), _ptr(hy), int(N), int(NT), _ptr(lisi_map),
                         _ptr(aug_map), _ptr(sums))


def iqa_both_host_many(ctx, pairs, dtype, params=None):
    arr = (iqa_host_pair * len(pairs))(*pairs)
    return _check(ctx, lib().iqa_both_host_many(ctx, arr, len(pairs), int(dtype),
                                                _params(params)))


# --- serving loop --------------------------------------------------------------

class _Server:
    """Owner of an iqa_server handle (and of the context it reports errors on)."""

    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.handle = handle


def iqa_server_create(ctx, dtype=IQA_F16, max_pairs_per_step=16, max_inflight_steps=2,
                      pool_bytes=8 << 30, one_pair_per_launch=0, simulate=0,
                      sim_bytes_per_s=1e12, step_timeout_ms=0.0, max_step_bytes=0,
                      params=None, generator_blocks_per_sm=0, map_ctas_per_sm=0,
                      time_kernels=0):
    p = iqa_params(1e-6, 1e-6, 1e-6, 0.0) if params is None else params
    if isinstance(p, dict):
        p = iqa_params(p.get("C1", 1e-6), p.get("C2", 1e-6), p.get("C", 1e-6), p.get("D", 0.0))
    cfg = iqa_server_config(int(dtype), int(max_pairs_per_step), int(max_inflight_steps),
                            int(pool_bytes), int(one_pair_per_launch), int(simulate),
                            float(sim_bytes_per_s), float(step_timeout_ms),
                            int(max_step_bytes), p, int(generator_blocks_per_sm),
                            int(map_ctas_per_sm), int(time_kernels))
    h = _vp()
    _check(ctx, lib().iqa_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h)))
    return _Server(ctx, h.value)


def _catalog(cat):
    """An iqa_catalog over a dict as made by synth.serving_catalog; returns the
    struct and the arrays it points into (keep both alive for the call)."""
    import numpy as np
    arrs = {k: np.ascontiguousarray(cat[k], dtype=np.int32 if k in ("x", "y", "half",
                                                                      "profile_off")
                                    else np.float32)
            for k in ("x", "y", "half", "profile_off", "flux", "profile")}
    c = iqa_catalog(int(cat["N"]), len(arrs["x"]), arrs["x"].ctypes.data,
                    arrs["y"].ctypes.data, arrs["flux"].ctypes.data, arrs["half"].ctypes.data,
                    arrs["profile_off"].ctypes.data, arrs["profile"].ctypes.data,
                    len(arrs["profile"]), float(cat["noise_sigma"]))
    return c, arrs


def iqa_server_add_reference(srv, ref_id, cat, seed):
    """cat: a dict as made by synth.serving_catalog (numpy arrays)."""
    c, _keep = _catalog(cat)
    return _check(srv.ctx, lib().iqa_server_add_reference(srv.handle, int(ref_id),
                                                          ctypes.byref(c), int(seed)))


def iqa_render_epoch(ctx, cat, seed, out, dtype=IQA_F32, drop=(), add=None):
    """Render one epoch of `cat` on the device into `out` (N*N elements)."""
    c, _keep = _catalog(cat)
    d = [int(v) for v in drop]
    arr = (ctypes.c_int * max(1, len(d)))(*(d or [0]))
    a = add if add is not None else (-1, 0, 0, 0.0)
    return _check(ctx, lib().iqa_render_epoch(ctx, ctypes.byref(c), int(seed), arr, len(d),
                                              int(a[0]), int(a[1]), int(a[2]), float(a[3]),
                                              int(dtype), _ptr(out)))


def iqa_server_reference_image(srv, ref_id, host_out):
    return _check(srv.ctx, lib().iqa_server_reference_image(srv.handle, int(ref_id),
                                                            _ptr(host_out)))


def make_request(ref_id, NT, seed, drop=(), add=None):
    """An iqa_request; more than 8 drops are passed on as such (the library
    rejects them)."""
    d = [int(v) for v in drop]
    head = d[:8]
    arr = (ctypes.c_int * 8)(*(head + [-1] * (8 - len(head))))
    a = add if add is not None else (-1, 0, 0, 0.0)
    return iqa_request(int(ref_id), int(NT), int(seed), len(d), arr, int(a[0]), int(a[1]),
                       int(a[2]), float(a[3]))


def iqa_submit(srv, req):
    h = ctypes.c_ulonglong()
    _check(srv.ctx, lib().iqa_submit(srv.handle, ctypes.byref(req), ctypes.byref(h)))
    return h.value


def iqa_poll(srv, h, timeout_us=0):
    """Returns the status (IQA_OK, IQA_PENDING or an error code); no raise."""
    return lib().iqa_poll(srv.handle, int(h), int(timeout_us))


def iqa_result(srv, h, lisi_map=None, aug_map=None):
    lat = ctypes.c_double()
    _check(srv.ctx, lib().iqa_result(srv.handle, int(h), _ptr(lisi_map), _ptr(aug_map),
                                     ctypes.byref(lat)))
    return lat.value


def iqa_server_get_stats(srv):
    st = iqa_server_stats()
    _check(srv.ctx, lib().iqa_server_get_stats(srv.handle, ctypes.byref(st)))
    return st


def iqa_server_destroy(srv):
    if srv.handle:
        lib().iqa_server_destroy(srv.handle)
        srv.handle = None


def iqa_server_run_trace(srv, reqs, arrival_s, timeout_s=600.0):
    """Native load generator: submits reqs[i] at arrival_s[i] s, waits for all."""
    arr = (iqa_request * len(reqs))(*reqs)
    t = (ctypes.c_double * len(reqs))(*[float(v) for v in arrival_s])
    return _check(srv.ctx, lib().iqa_server_run_trace(srv.handle, arr, t, len(reqs),
                                                      float(timeout_s)))
