"""Thin ctypes binding of libeat's C ABI (include/eat.h), with the same names.

Only argument marshalling happens here: every step of a query runs in libeat's
CUDA kernels.  Buffers may be torch tensors (CPU or CUDA) or numpy arrays; the
binding passes their raw pointers and never copies or computes results itself.
If libeat.so is missing this module raises ImportError: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeat.so")

EAT_INF = 2**31 - 1
EAT_OK, EAT_ERR_INVALID, EAT_ERR_OOM, EAT_ERR_CUDA = 0, 1, 2, 3
EAT_ERR_NO_CONVERGENCE, EAT_ERR_NO_DEVICE, EAT_ERR_WORKSPACE = 4, 5, 6
EAT_MODE_AUTO, EAT_MODE_CTA, EAT_MODE_CLUSTER, EAT_MODE_ASYNC, EAT_MODE_PAIR = 0, 1, 2, 3, 4
EAT_MODE_EDGE = 5
EAT_ORDER_AUTO, EAT_ORDER_BY_TIME, EAT_ORDER_AS_GIVEN = 0, 1, 2
EAT_PLACE_AUTO, EAT_PLACE_SHARED, EAT_PLACE_GLOBAL_ARR, EAT_PLACE_GLOBAL = 0, 1, 2, 3
EAT_SUBTRIPS_NONE, EAT_SUBTRIPS_SQRT_K, EAT_SUBTRIPS_SQRT_MEAN = 0, 1, 2
EAT_ADMIT_RING, EAT_ADMIT_BATCH = 0, 1
EAT_MAX_NETS = 128
EAT_VAR_CONNECTION, EAT_VAR_TYPE, EAT_VAR_TYPE_AP = 1, 2, 3
EAT_VAR_CLUSTER_AP, EAT_VAR_EDGE, EAT_VAR_WARP = 4, 5, 6

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libeat.so not found at {LIB_PATH}: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)

_i32p = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p


class eat_connections(ctypes.Structure):
    _fields_ = [("n_stops", ctypes.c_int32), ("n_conn", ctypes.c_int64),
                ("u", _vp), ("v", _vp), ("dep", _vp), ("dur", _vp), ("trip", _vp)]


class eat_build_opts(ctypes.Structure):
    _fields_ = [("cluster_width", ctypes.c_int32), ("t0", ctypes.c_int32),
                ("device", ctypes.c_int32), ("subtrips", ctypes.c_int32)]


class eat_csr_input(ctypes.Structure):
    _fields_ = [("n_stops", ctypes.c_int32), ("n_types", ctypes.c_int32),
                ("n_clusters", ctypes.c_int64), ("n_aps", ctypes.c_int64),
                ("row_ptr", _vp), ("type_v", _vp), ("type_dur", _vp), ("type_cl_ptr", _vp),
                ("cl_k", _vp), ("cl_ap_ptr", _vp), ("ap_first", _vp), ("ap_step", _vp),
                ("ap_count", _vp)]


class eat_stats(ctypes.Structure):
    _fields_ = [("n_stops", ctypes.c_int32), ("n_types", ctypes.c_int32),
                ("n_edges", ctypes.c_int32), ("cluster_width", ctypes.c_int32),
                ("t0", ctypes.c_int32), ("max_clusters", ctypes.c_int32),
                ("max_out_types", ctypes.c_int32), ("device", ctypes.c_int32),
                ("n_conn", ctypes.c_int64), ("n_ap", ctypes.c_int64),
                ("n_cl", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("k_min", ctypes.c_int32), ("y", ctypes.c_int32), ("n_ap_extra", ctypes.c_int64),
                ("n_shortcuts", ctypes.c_int64)]


class eat_net_view(ctypes.Structure):
    _fields_ = [("row_ptr", _vp), ("type_rec", _vp), ("type_cl", _vp), ("cl", _vp),
                ("ap", _vp), ("cluster_entries", _vp), ("ap_extra", _vp), ("type_records", _vp)]


class eat_counters(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("vertices", ctypes.c_int64),
                ("types", ctypes.c_int64), ("evals", ctypes.c_int64),
                ("lookups", ctypes.c_int64), ("aps", ctypes.c_int64),
                ("relaxed", ctypes.c_int64)]


COUNTER_FIELDS = ("rounds", "vertices", "types", "evals", "lookups", "aps", "relaxed")


class eat_query_opts(ctypes.Structure):
    _fields_ = [("max_rounds", ctypes.c_int32), ("block", ctypes.c_int32),
                ("vwarp", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("placement", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("order", ctypes.c_int32), ("idle_cap", ctypes.c_int32),
                ("horizon", ctypes.c_int32), ("status", _vp), ("counters", _vp)]


class eat_server_opts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("batch_wait_us", ctypes.c_int32), ("admission", ctypes.c_int32),
                ("mem_budget", ctypes.c_int64)]


class eat_server_result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("net", ctypes.c_int32),
                ("latency_ns", ctypes.c_int64)]


class eat_server_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "submitted", "completed", "pending", "batches", "batched_queries", "max_batch_seen",
        "max_inflight_seen", "max_pending_seen", "slots", "slot_bytes", "last_error",
        "admitted_running", "base_bytes")]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("eat_last_error", ctypes.c_char_p, [])
_sig("eat_version", ctypes.c_int32, [])
_sig("eat_build", ctypes.c_int, [ctypes.POINTER(eat_connections), ctypes.POINTER(eat_build_opts),
                                 ctypes.POINTER(_vp)])
_sig("eat_build_csr", ctypes.c_int, [ctypes.POINTER(eat_csr_input), ctypes.POINTER(eat_build_opts),
                                     ctypes.POINTER(_vp)])
_sig("eat_free", None, [_vp])
_sig("eat_get_stats", ctypes.c_int, [_vp, ctypes.POINTER(eat_stats)])
_sig("eat_net_host_view", ctypes.c_int, [_vp, ctypes.POINTER(eat_net_view)])
_sig("eat_query", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp])
_sig("eat_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(_vp), ctypes.c_int32,
                                              ctypes.c_int32, ctypes.POINTER(eat_query_opts)])
_sig("eat_launch_shape", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(eat_query_opts), ctypes.POINTER(eat_query_opts)])
_sig("eat_query_batch", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, _vp, _vp, ctypes.c_size_t,
                                       ctypes.POINTER(eat_query_opts), _vp])
_sig("eat_query_batch_multi", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, _vp, _vp, _vp,
                                             ctypes.c_int32, _vp, _vp, _vp, ctypes.c_size_t,
                                             ctypes.POINTER(eat_query_opts), _vp])
_sig("eat_next_departure", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, _vp, _vp])
_sig("eat_query_batch_noalloc", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, _vp,
                                               ctypes.POINTER(eat_query_opts), _vp])

_sig("eat_autotune", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.POINTER(eat_query_opts), _vp])
_sig("eat_autotune_multi", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, _vp, _vp, _vp,
                                          ctypes.c_int32, ctypes.POINTER(eat_query_opts), _vp])
_sig("eat_server_create", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32,
                                         ctypes.POINTER(eat_server_opts), ctypes.POINTER(_vp)])
_sig("eat_server_submit", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp,
                                         ctypes.c_uint64])
_sig("eat_server_poll", ctypes.c_int32, [_vp, ctypes.POINTER(eat_server_result), ctypes.c_int32,
                                         ctypes.c_int32])
_sig("eat_server_get_stats", ctypes.c_int, [_vp, ctypes.POINTER(eat_server_stats)])
_sig("eat_server_destroy", None, [_vp])


class eat_ladder_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("flag_reads", ctypes.c_int32)]


class eat_ladder_view(ctypes.Structure):
    _fields_ = [("n_types", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("n_dep", ctypes.c_int64), ("n_ap", ctypes.c_int64),
                ("type_uvl", _vp), ("dep_ptr", _vp), ("dep", _vp), ("ap_ptr", _vp), ("ap", _vp),
                ("edge_ptr", _vp)]


_sig("eat_ladder_build", ctypes.c_int, [ctypes.POINTER(eat_connections),
                                        ctypes.POINTER(eat_build_opts), ctypes.POINTER(_vp)])
_sig("eat_ladder_free", None, [_vp])
_sig("eat_ladder_query", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, _vp,
                                        ctypes.POINTER(eat_ladder_stats)])
_sig("eat_ladder_host_view", ctypes.c_int, [_vp, ctypes.POINTER(eat_ladder_view)])

EXPORTED = ("eat_autotune", "eat_autotune_multi", "eat_server_create", "eat_server_submit", "eat_server_poll", "eat_server_get_stats",
            "eat_server_destroy", "eat_last_error", "eat_version", "eat_build", "eat_build_csr", "eat_free", "eat_get_stats",
            "eat_net_host_view", "eat_query", "eat_workspace_bytes", "eat_launch_shape", "eat_query_batch",
            "eat_query_batch_multi", "eat_next_departure", "eat_query_batch_noalloc",
            "eat_ladder_build", "eat_ladder_free", "eat_ladder_query", "eat_ladder_host_view")


class EatError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.eat_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {code}: {msg}")


def _check(rc, where):
    if rc != EAT_OK:
        raise EatError(rc, where)


def _ptr(x):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("buffers must be contiguous")
        return x.ctypes.data
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Net:
    """Owning handle of an eat_net (released by eat_free on close or garbage collection)."""

    def __init__(self, handle, keep=None):
        self._h = _vp(handle)
        self._keep = keep

    @property
    def handle(self):
        if not self._h:
            raise ValueError("network already freed")
        return self._h

    def close(self):
        if self._h:
            _lib.eat_free(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stats(self):
        return eat_get_stats(self)


def eat_build(n_stops, u, v, dep, dur, cluster_width=0, t0=0, device=0, trip=None,
              subtrips=EAT_SUBTRIPS_NONE) -> Net:
    """Preprocess connections (host int32 arrays) into a device-resident network."""
    u, v, dep, dur = _i32(u), _i32(v), _i32(dep), _i32(dur)
    n = u.shape[0]
    if not (v.shape[0] == dep.shape[0] == dur.shape[0] == n):
        raise ValueError("connection arrays differ in length")
    tr = None if trip is None else _i32(trip)
    if tr is not None and tr.shape[0] != n:
        raise ValueError("trip array differs in length")
    c = eat_connections(int(n_stops), int(n), u.ctypes.data, v.ctypes.data, dep.ctypes.data,
                        dur.ctypes.data, None if tr is None else tr.ctypes.data)
    o = eat_build_opts(int(cluster_width), int(t0), int(device), int(subtrips))
    h = _vp()
    _check(_lib.eat_build(ctypes.byref(c), ctypes.byref(o), ctypes.byref(h)), "eat_build")
    return Net(h.value)


def eat_build_csr(n_stops, row_ptr, type_v, type_dur, type_cl_ptr, cl_k, cl_ap_ptr, ap_first,
                  ap_step, ap_count, cluster_width=0, t0=0, device=0) -> Net:
    """Build from pre-encoded connection types, clusters and AP runs (see eat.h)."""
    i64 = lambda a: np.ascontiguousarray(a, dtype=np.int64)
    arrs = [_i32(row_ptr), _i32(type_v), _i32(type_dur), i64(type_cl_ptr), _i32(cl_k),
            i64(cl_ap_ptr), _i32(ap_first), _i32(ap_step), _i32(ap_count)]
    c = eat_csr_input(int(n_stops), int(arrs[1].shape[0]), int(arrs[4].shape[0]),
                      int(arrs[6].shape[0]), *[a.ctypes.data for a in arrs])
    o = eat_build_opts(int(cluster_width), int(t0), int(device), 0)
    h = _vp()
    _check(_lib.eat_build_csr(ctypes.byref(c), ctypes.byref(o), ctypes.byref(h)), "eat_build_csr")
    return Net(h.value, keep=arrs)


def eat_free(net: Net) -> None:
    net.close()


def eat_get_stats(net: Net) -> dict:
    s = eat_stats()
    _check(_lib.eat_get_stats(net.handle, ctypes.byref(s)), "eat_get_stats")
    return {f: getattr(s, f) for f, _ in eat_stats._fields_}


def eat_net_host_view(net: Net) -> dict:
    """Copies of the built arrays: row_ptr, type_rec [T, 4], type_cl, cl, ap [A, 2]."""
    st = eat_get_stats(net)
    view = eat_net_view()
    _check(_lib.eat_net_host_view(net.handle, ctypes.byref(view)), "eat_net_host_view")

    def arr(ptr, n, dt):
        if n == 0:
            return np.zeros(0, dtype=dt)
        buf = (ctypes.c_char * (n * np.dtype(dt).itemsize)).from_address(ptr)
        return np.frombuffer(buf, dtype=dt).copy()

    T, V = st["n_types"], st["n_stops"]
    return {
        "row_ptr": arr(view.row_ptr, V + 1, np.int32),
        "type_rec": arr(view.type_rec, 4 * T, np.int32).reshape(T, 4),
        "type_cl": arr(view.type_cl, T, np.int32),
        "cl": arr(view.cl, st["n_cl"], np.int32),
        "ap": arr(view.ap, 2 * st["n_ap"], np.uint32).reshape(-1, 2),
        # stored cluster-major; returned as [type, cluster, 8]
        "cluster_entries": arr(view.cluster_entries, 8 * T * st["y"], np.int32)
        .reshape(st["y"], T, 8).transpose(1, 0, 2).copy(),
        "ap_extra": arr(view.ap_extra, 2 * st["n_ap_extra"], np.uint32).reshape(-1, 2),
        "type_records": arr(view.type_records, 4 * T, np.int32).reshape(T, 4),
    }


def _opts(max_rounds=0, block=0, vwarp=0, mode=0, placement=0, cluster=0, order=0, idle_cap=0,
          horizon=0, status=None, counters=None):
    return eat_query_opts(int(max_rounds), int(block), int(vwarp), int(mode), int(placement),
                          int(cluster), int(order), int(idle_cap), int(horizon), _ptr(status),
                          _ptr(counters))


def eat_query(net: Net, s: int, t_s: int, out=None, counters: bool = False):
    """One blocking query; `out` may be a host/device buffer of n_stops int32 (allocated as
    numpy when None).  Returns out, or (out, counters dict) if counters=True."""
    if out is None:
        out = np.empty(eat_get_stats(net)["n_stops"], dtype=np.int32)
    c = eat_counters()
    _check(_lib.eat_query(net.handle, int(s), int(t_s), _ptr(out), ctypes.byref(c)), "eat_query")
    if counters:
        return out, {f: getattr(c, f) for f in COUNTER_FIELDS}
    return out


def eat_workspace_bytes(nets, n, **opts) -> int:
    if isinstance(nets, Net):
        nets = [nets]
    arr = (_vp * len(nets))(*[x.handle.value for x in nets])
    o = _opts(**opts)
    return int(_lib.eat_workspace_bytes(arr, len(nets), int(n), ctypes.byref(o)))


def eat_launch_shape(nets, n, **opts) -> dict:
    """Launch shape a batch of n queries would run with: block, vwarp, mode, cluster, order,
    horizon (-1 = none)."""
    if isinstance(nets, Net):
        nets = [nets]
    arr = (_vp * len(nets))(*[x.handle.value for x in nets])
    o = _opts(**opts)
    shape = eat_query_opts()
    _check(_lib.eat_launch_shape(arr, len(nets), int(n), ctypes.byref(o), ctypes.byref(shape)),
           "eat_launch_shape")
    return {"block": shape.block, "vwarp": shape.vwarp, "mode": shape.mode, "cluster": shape.cluster,
            "order": shape.order, "horizon": shape.horizon}


def eat_query_batch(net: Net, sources, times, out, workspace=None, workspace_bytes=None,
                    stream=None, **opts):
    """n queries on one network.  sources/times/out: torch tensors or numpy arrays, host or
    device; out holds n * n_stops int32.  Asynchronous when every buffer is on the device."""
    n = int(sources.shape[0])
    o = _opts(**opts)
    wb = workspace_bytes if workspace_bytes is not None else (
        workspace.numel() * workspace.element_size() if workspace is not None else 0)
    _check(_lib.eat_query_batch(net.handle, _ptr(sources), _ptr(times), n, _ptr(out),
                                _ptr(workspace), int(wb), ctypes.byref(o),
                                _stream_handle(stream)), "eat_query_batch")
    return out


def eat_query_batch_multi(nets, net_idx, sources, times, out, arr_offsets, workspace=None,
                          workspace_bytes=None, stream=None, **opts):
    """n queries over several networks in one launch (see eat.h)."""
    arr = (_vp * len(nets))(*[x.handle.value for x in nets])
    n = int(sources.shape[0])
    o = _opts(**opts)
    wb = workspace_bytes if workspace_bytes is not None else (
        workspace.numel() * workspace.element_size() if workspace is not None else 0)
    _check(_lib.eat_query_batch_multi(arr, len(nets), _ptr(net_idx), _ptr(sources), _ptr(times),
                                      n, _ptr(out), _ptr(arr_offsets), _ptr(workspace), int(wb),
                                      ctypes.byref(o), _stream_handle(stream)),
           "eat_query_batch_multi")
    return out


def eat_query_batch_noalloc(net: Net, sources, times, out, stream=None, **opts):
    """eat_query_batch for callers that cannot allocate device memory: no workspace argument,
    the library's fixed 16 MiB scratch holds the frontier queues instead.  All buffers must be
    device memory; calls that overlap on the GPU must be serialised (they share the scratch)."""
    o = _opts(**opts)
    _check(_lib.eat_query_batch_noalloc(net.handle, _ptr(sources), _ptr(times),
                                        int(sources.shape[0]), _ptr(out), ctypes.byref(o),
                                        _stream_handle(stream)), "eat_query_batch_noalloc")
    return out


def eat_autotune(net: Net, sources, times, stream=None) -> dict:
    """Time the candidate launch shapes on a sample batch (device int32 arrays) and keep the
    fastest for this network and batch size; returns {"block", "vwarp", "mode", "horizon"}
    (horizon -1 = none)."""
    o = eat_query_opts()
    _check(_lib.eat_autotune(net.handle, _ptr(sources), _ptr(times), int(sources.shape[0]),
                             ctypes.byref(o), _stream_handle(stream)), "eat_autotune")
    return {"block": o.block, "vwarp": o.vwarp, "mode": o.mode, "horizon": o.horizon}


def eat_autotune_multi(nets, net_idx, sources, times, stream=None) -> dict:
    """Time the candidate launch shapes and start orders of a batch over several networks
    (device int32 arrays); returns {"block", "vwarp", "mode", "order", "horizon"} to pass
    as the options of eat_query_batch_multi."""
    arr = (_vp * len(nets))(*[x.handle.value for x in nets])
    o = eat_query_opts()
    _check(_lib.eat_autotune_multi(arr, len(nets), _ptr(net_idx), _ptr(sources), _ptr(times),
                                   int(sources.shape[0]), ctypes.byref(o), _stream_handle(stream)),
           "eat_autotune_multi")
    return {"block": o.block, "vwarp": o.vwarp, "mode": o.mode, "order": o.order,
            "horizon": o.horizon}


def eat_next_departure(net: Net, types, times, out, stream=None):
    """out[i] = least departure >= times[i] of type types[i] (device int32 buffers)."""
    _check(_lib.eat_next_departure(net.handle, _ptr(types), _ptr(times), int(types.shape[0]),
                                   _ptr(out), _stream_handle(stream)), "eat_next_departure")
    return out


def eat_version() -> int:
    return int(_lib.eat_version())


def eat_last_error() -> str:
    return _lib.eat_last_error().decode(errors="replace")


class Server:
    """Continuous-batching request loop over resident networks (eat_server_* in eat.h);
    admission EAT_ADMIT_RING (default) or EAT_ADMIT_BATCH."""

    def __init__(self, nets, max_batch=0, max_inflight=0, batch_wait_us=0, mem_budget=0,
                 admission=0):
        self._nets = list(nets)
        arr = (_vp * len(self._nets))(*[x.handle.value for x in self._nets])
        o = eat_server_opts(int(max_batch), int(max_inflight), int(batch_wait_us), int(admission),
                            int(mem_budget))
        h = _vp()
        _check(_lib.eat_server_create(arr, len(self._nets), ctypes.byref(o), ctypes.byref(h)),
               "eat_server_create")
        self._h = h
        self._buf = (eat_server_result * 4096)()

    def submit(self, net, s, t_s, out, tag):
        """Queue a query; `out` is a host int32 buffer of the network's n_stops (kept alive
        by the caller until its result is polled)."""
        _check(_lib.eat_server_submit(self._h, int(net), int(s), int(t_s), _ptr(out), int(tag)),
               "eat_server_submit")

    def poll(self, timeout_us=1000, max_results=4096):
        n = _lib.eat_server_poll(self._h, self._buf, min(int(max_results), 4096), int(timeout_us))
        return [(r.tag, r.status, r.net, r.latency_ns) for r in self._buf[:n]]

    def stats(self):
        st = eat_server_stats()
        _check(_lib.eat_server_get_stats(self._h, ctypes.byref(st)), "eat_server_get_stats")
        return {f: getattr(st, f) for f, _ in eat_server_stats._fields_}

    def close(self):
        if self._h:
            _lib.eat_server_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ladder:
    """Owning handle of an eat_ladder (released by eat_ladder_free)."""

    def __init__(self, handle):
        self._h = _vp(handle)

    @property
    def handle(self):
        if not self._h:
            raise ValueError("ladder already freed")
        return self._h

    def close(self):
        if self._h:
            _lib.eat_ladder_free(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eat_ladder_build(n_stops, u, v, dep, dur, cluster_width=0, t0=0, device=0) -> Ladder:
    """The topology-driven variants' arrays (see eat.h); device=-1 builds host arrays only."""
    u, v, dep, dur = _i32(u), _i32(v), _i32(dep), _i32(dur)
    n = u.shape[0]
    if not (v.shape[0] == dep.shape[0] == dur.shape[0] == n):
        raise ValueError("connection arrays differ in length")
    c = eat_connections(int(n_stops), int(n), u.ctypes.data, v.ctypes.data, dep.ctypes.data,
                        dur.ctypes.data, None)
    o = eat_build_opts(int(cluster_width), int(t0), int(device), 0)
    h = _vp()
    _check(_lib.eat_ladder_build(ctypes.byref(c), ctypes.byref(o), ctypes.byref(h)),
           "eat_ladder_build")
    return Ladder(h.value)


def eat_ladder_query(ladder: Ladder, variant, s, t_s, out=None, flag_every=1, graph=False,
                     n_stops=None):
    """One blocking query with a topology-driven variant; returns (out, stats dict)."""
    if out is None:
        if n_stops is None:
            raise ValueError("pass `out` or `n_stops`")
        out = np.empty(int(n_stops), dtype=np.int32)
    st = eat_ladder_stats()
    _check(_lib.eat_ladder_query(ladder.handle, int(variant), int(s), int(t_s), int(flag_every),
                                 int(bool(graph)), _ptr(out), ctypes.byref(st)),
           "eat_ladder_query")
    return out, {"rounds": st.rounds, "flag_reads": st.flag_reads}


def eat_ladder_host_view(ladder: Ladder) -> dict:
    """Copies of the variants' host arrays: type_uvl [T, 3], dep_ptr, dep, ap_ptr, ap [A, 3],
    edge_ptr."""
    vw = eat_ladder_view()
    _check(_lib.eat_ladder_host_view(ladder.handle, ctypes.byref(vw)), "eat_ladder_host_view")
    T, E = vw.n_types, vw.n_edges

    def arr(p, n):
        if n == 0:
            return np.zeros(0, dtype=np.int32)
        return np.ctypeslib.as_array(ctypes.cast(p, _i32p), shape=(n,)).copy()

    return {"type_uvl": arr(vw.type_uvl, 3 * T).reshape(T, 3), "dep_ptr": arr(vw.dep_ptr, T + 1),
            "dep": arr(vw.dep, vw.n_dep), "ap_ptr": arr(vw.ap_ptr, T + 1),
            "ap": arr(vw.ap, 3 * vw.n_ap).reshape(-1, 3), "edge_ptr": arr(vw.edge_ptr, E + 1)}
