"""Python binding of the C ABI in include/hoph.h (argument marshalling only).

Every function keeps the C name and argument order.  Device buffers may be
passed as torch CUDA tensors or raw integer addresses; ``stream`` may be a
torch.cuda.Stream, a raw handle, or None for torch's current stream.  All
work runs in libhoph.so; if the library is missing this module raises
instead of falling back to anything else.

On top of the raw calls, ``Plan`` bundles a plan with torch-allocated
buffers for the common sequence sketch -> query -> read pairs.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhoph.so")

HOPH_OK = 0
HOPH_ERR_PARAM = -1
HOPH_ERR_ID_RANGE = -2
HOPH_ERR_CAPACITY = -3
HOPH_ERR_TIMEOUT = -4
HOPH_ERR_CUDA = -5
HOPH_ERR_NOMEM = -6
HOPH_ERR_UNSUPPORTED = -7
HOPH_ERR_TOO_LARGE = -8
HOPH_ERR_CAPTURE = -9

HOPH_MODE_OPH_FULL = 0
HOPH_MODE_GOPH = 1
HOPH_MODE_HOPH = 2
HOPH_MODE_MINWISE_FULL = 3
MODES = {"oph_full": 0, "goph": 1, "hoph": 2, "minwise_full": 3}

HOPH_PERM_TABLE = 0
HOPH_PERM_HASH61 = 1
HOPH_EMPTY_BOTH = 0
HOPH_EMPTY_EITHER = 1
HOPH_EMPTY_NONE = 2
RULES = {"both": 0, "either": 1, "none": 2}
HOPH_WEIGHT_SPACE = 0
HOPH_WEIGHT_LITERAL = 1
HOPH_MAX_GROUPS = 16
HOPH_EMPTY_VALUE = 0xFFFFFFFF
HOPH_EMPTY_VALUE16 = 0xFFFF


class hoph_params(ctypes.Structure):
    _fields_ = [("universe_D", ctypes.c_uint64), ("k", ctypes.c_uint32),
                ("k_group", ctypes.c_uint32), ("a", ctypes.c_uint32), ("b", ctypes.c_uint32),
                ("perm_kind", ctypes.c_uint32), ("minwise_k", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("thr_num", ctypes.c_uint32),
                ("thr_den", ctypes.c_uint32), ("epsilon", ctypes.c_double),
                ("empty_rule", ctypes.c_uint32), ("weighting", ctypes.c_uint32)]


class hoph_pair(ctypes.Structure):
    _fields_ = [("row", ctypes.c_int64), ("query", ctypes.c_uint32),
                ("groups", ctypes.c_uint16), ("matches", ctypes.c_uint16)]


PAIR_DTYPE = np.dtype([("row", "<i8"), ("query", "<u4"), ("groups", "<u2"), ("matches", "<u2")])


class hoph_stats(ctypes.Structure):
    _fields_ = [("entering", ctypes.c_int64 * HOPH_MAX_GROUPS),
                ("accepted", ctypes.c_int64 * HOPH_MAX_GROUPS),
                ("rejected", ctypes.c_int64 * HOPH_MAX_GROUPS),
                ("sketch_bytes", ctypes.c_int64), ("join_hits", ctypes.c_int64),
                ("strategy", ctypes.c_int64), ("rows_counted", ctypes.c_int64)]


STATS_WORDS = ctypes.sizeof(hoph_stats) // 8


class hoph_plan_info(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_uint32), ("key_bits", ctypes.c_uint32),
                ("upper_limit", ctypes.c_int64), ("lower_limit", ctypes.c_int64),
                ("group_size", ctypes.c_uint64 * HOPH_MAX_GROUPS),
                ("max_bin_width", ctypes.c_uint64)]


class hoph_exec(ctypes.Structure):
    _fields_ = [("strategy", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
                ("consumer_warps", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("lanes_per_row", ctypes.c_int32),
                ("sketch_cta_bits", ctypes.c_int32), ("join_lanes", ctypes.c_int32)]


class HophError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, hoph_status_string(code), code))


_lib = None
_EXPORTS = ["hoph_plan_create", "hoph_plan_create_with_perm", "hoph_plan_destroy",
            "hoph_plan_get_info", "hoph_plan_set_exec", "oph_build_sketches",
            "minwise_build_sketches", "hoph_query_batch", "hoph_pair_counts", "hoph_synth_ids",
            "hoph_sync_status", "hoph_status_string", "hoph_plan_enable_timing",
            "hoph_plan_read_timing", "oph_build_sketches_static", "hoph_plan_peek_timing",
            "hoph_check_bounded_wait", "hoph_synth_sketch", "oph_build_sketches16",
            "hoph_query_batch16", "hoph_self_join", "hoph_self_join16", "hoph_self_join_part",
            "hoph_small_probability_limits",
            "hoph_int_probe"]


def load(path=LIB_PATH):
    """Load libhoph.so (raises OSError if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libhoph.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P, i64, u64, u32, i32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                             ctypes.c_int)
    pp = ctypes.POINTER(ctypes.c_void_p)
    lib.hoph_plan_create.argtypes = [ctypes.POINTER(hoph_params), pp]
    lib.hoph_plan_create.restype = i32
    lib.hoph_plan_create_with_perm.argtypes = [ctypes.POINTER(hoph_params), P, pp]
    lib.hoph_plan_create_with_perm.restype = i32
    lib.hoph_plan_destroy.argtypes = [P]
    lib.hoph_plan_destroy.restype = None
    lib.hoph_plan_get_info.argtypes = [P, ctypes.POINTER(hoph_plan_info)]
    lib.hoph_plan_get_info.restype = i32
    lib.hoph_plan_set_exec.argtypes = [P, ctypes.POINTER(hoph_exec)]
    lib.hoph_plan_set_exec.restype = i32
    lib.hoph_small_probability_limits.argtypes = [u32, u32, u32, ctypes.c_double, P, P]
    lib.hoph_small_probability_limits.restype = i32
    lib.hoph_int_probe.argtypes = [u32, i64, P, P]
    lib.hoph_int_probe.restype = i32
    lib.oph_build_sketches.argtypes = [P, P, P, i64, P, P]
    lib.oph_build_sketches.restype = i32
    lib.oph_build_sketches_static.argtypes = [P, P, P, i64, P, P]
    lib.oph_build_sketches_static.restype = i32
    lib.minwise_build_sketches.argtypes = [P, P, P, i64, P, P]
    lib.minwise_build_sketches.restype = i32
    lib.hoph_query_batch.argtypes = [P, u32, P, i64, P, i64, P, i64, P, P, P]
    lib.hoph_query_batch.restype = i32
    lib.hoph_self_join.argtypes = [P, u32, P, i64, i64, P, i64, P, P, P]
    lib.hoph_self_join.restype = i32
    lib.hoph_self_join16.argtypes = [P, u32, P, i64, i64, P, i64, P, P, P]
    lib.hoph_self_join16.restype = i32
    lib.hoph_self_join_part.argtypes = [P, u32, P, u32, i64, i64, i64, i64, P, i64, P, P, P]
    lib.hoph_self_join_part.restype = i32
    lib.oph_build_sketches16.argtypes = [P, P, P, i64, P, P]
    lib.oph_build_sketches16.restype = i32
    lib.hoph_query_batch16.argtypes = [P, u32, P, i64, P, i64, P, i64, P, P, P]
    lib.hoph_query_batch16.restype = i32
    lib.hoph_pair_counts.argtypes = [P, P, i64, P, i64, P, P]
    lib.hoph_pair_counts.restype = i32
    lib.hoph_synth_ids.argtypes = [u64, i64, i64, u64, u32, P, i64, P, P]
    lib.hoph_synth_ids.restype = i32
    lib.hoph_sync_status.argtypes = [P, P]
    lib.hoph_sync_status.restype = i32
    lib.hoph_plan_enable_timing.argtypes = [P, i32]
    lib.hoph_plan_enable_timing.restype = i32
    lib.hoph_plan_read_timing.argtypes = [P, P, P, P]
    lib.hoph_plan_read_timing.restype = i32
    lib.hoph_synth_sketch.argtypes = [P, u64, u64, P, i64, P, P]
    lib.hoph_synth_sketch.restype = i32
    lib.hoph_check_bounded_wait.argtypes = [P, u64, P]
    lib.hoph_check_bounded_wait.restype = i32
    lib.hoph_plan_peek_timing.argtypes = [P, P]
    lib.hoph_plan_peek_timing.restype = i32
    lib.hoph_status_string.argtypes = [i32]
    lib.hoph_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("expected a tensor, ndarray or address, got %r" % type(x))


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, where):
    if rc != HOPH_OK:
        raise HophError(rc, where)
    return rc


# ---- the C entry points, same names and argument order ---------------------

def hoph_status_string(status):
    return load().hoph_status_string(int(status)).decode()


def make_params(D, k, k_group, a=0, b=0, perm_kind=HOPH_PERM_TABLE, minwise_k=0, seed=1,
                thr=(7, 10), epsilon=1e-4, empty_rule="both", weighting=HOPH_WEIGHT_SPACE):
    return hoph_params(D, k, k_group, a, b, perm_kind, minwise_k, seed, thr[0], thr[1],
                       float(epsilon), RULES.get(empty_rule, empty_rule), weighting)


def hoph_plan_create(params):
    h = ctypes.c_void_p()
    _check(load().hoph_plan_create(ctypes.byref(params), ctypes.byref(h)), "hoph_plan_create")
    return h.value


def hoph_plan_create_with_perm(params, host_perm):
    perm = np.ascontiguousarray(host_perm, dtype=np.uint32)
    h = ctypes.c_void_p()
    _check(load().hoph_plan_create_with_perm(ctypes.byref(params), perm.ctypes.data,
                                             ctypes.byref(h)), "hoph_plan_create_with_perm")
    return h.value


def hoph_plan_destroy(plan):
    load().hoph_plan_destroy(plan)


def hoph_plan_get_info(plan):
    info = hoph_plan_info()
    _check(load().hoph_plan_get_info(plan, ctypes.byref(info)), "hoph_plan_get_info")
    return info


def hoph_plan_set_exec(plan, exec_=None):
    _check(load().hoph_plan_set_exec(plan, ctypes.byref(exec_) if exec_ is not None else None),
           "hoph_plan_set_exec")


def hoph_small_probability_limits(k_group, thr_num, thr_den, epsilon):
    """(U, L) of Definition 1, exact (host only; no device needed)."""
    U = ctypes.c_int64()
    L = ctypes.c_int64()
    _check(load().hoph_small_probability_limits(int(k_group), int(thr_num), int(thr_den),
                                                float(epsilon), ctypes.addressof(U),
                                                ctypes.addressof(L)),
           "hoph_small_probability_limits")
    return U.value, L.value


def oph_build_sketches(plan, d_ids, d_offsets, n_sets, d_planes, stream=None):
    return _check(load().oph_build_sketches(plan, _ptr(d_ids), _ptr(d_offsets), int(n_sets),
                                            _ptr(d_planes), _stream(stream)), "oph_build_sketches")


def oph_build_sketches_static(plan, d_ids, d_offsets, n_sets, d_planes, stream=None):
    """oph_build_sketches with its work list in the library's fixed device
    array (no device allocation; at most 262,144 sets per call)."""
    return _check(load().oph_build_sketches_static(plan, _ptr(d_ids), _ptr(d_offsets),
                                                   int(n_sets), _ptr(d_planes), _stream(stream)),
                  "oph_build_sketches_static")


def minwise_build_sketches(plan, d_ids, d_offsets, n_sets, d_sketches, stream=None):
    return _check(load().minwise_build_sketches(plan, _ptr(d_ids), _ptr(d_offsets), int(n_sets),
                                                _ptr(d_sketches), _stream(stream)),
                  "minwise_build_sketches")


def hoph_query_batch(plan, mode, d_query_planes, n_queries, d_coll_planes, n_rows, d_out,
                     out_capacity, d_out_count, d_stats=None, stream=None):
    return _check(load().hoph_query_batch(plan, MODES.get(mode, mode), _ptr(d_query_planes),
                                          int(n_queries), _ptr(d_coll_planes), int(n_rows),
                                          _ptr(d_out), int(out_capacity), _ptr(d_out_count),
                                          _ptr(d_stats), _stream(stream)), "hoph_query_batch")


def hoph_self_join(plan, mode, d_planes, n_rows, batch, d_out, out_capacity, d_out_count,
                   d_stats=None, stream=None):
    return _check(load().hoph_self_join(plan, MODES.get(mode, mode), _ptr(d_planes), int(n_rows),
                                        int(batch), _ptr(d_out), int(out_capacity),
                                        _ptr(d_out_count), _ptr(d_stats), _stream(stream)),
                  "hoph_self_join")


def hoph_self_join_part(plan, mode, d_planes, n_rows, batch, part, parts, d_out, out_capacity,
                        d_out_count, d_stats=None, stream=None):
    """Blocks part, part + parts, ... of the self-join (uint32 or compact
    uint16 planes, told apart by the tensor's element size)."""
    return _check(load().hoph_self_join_part(plan, MODES.get(mode, mode), _ptr(d_planes),
                                             int(d_planes.element_size()), int(n_rows),
                                             int(batch), int(part), int(parts), _ptr(d_out),
                                             int(out_capacity), _ptr(d_out_count),
                                             _ptr(d_stats), _stream(stream)),
                  "hoph_self_join_part")


def hoph_self_join16(plan, mode, d_planes, n_rows, batch, d_out, out_capacity, d_out_count,
                     d_stats=None, stream=None):
    return _check(load().hoph_self_join16(plan, MODES.get(mode, mode), _ptr(d_planes),
                                          int(n_rows), int(batch), _ptr(d_out),
                                          int(out_capacity), _ptr(d_out_count), _ptr(d_stats),
                                          _stream(stream)), "hoph_self_join16")


def oph_build_sketches16(plan, d_ids, d_offsets, n_sets, d_planes, stream=None):
    """Compact (uint16) sketches; d_planes int16/uint16 [G][n_sets][k']."""
    return _check(load().oph_build_sketches16(plan, _ptr(d_ids), _ptr(d_offsets), int(n_sets),
                                              _ptr(d_planes), _stream(stream)),
                  "oph_build_sketches16")


def hoph_query_batch16(plan, mode, d_query_planes, n_queries, d_coll_planes, n_rows, d_out,
                       out_capacity, d_out_count, d_stats=None, stream=None):
    return _check(load().hoph_query_batch16(plan, MODES.get(mode, mode), _ptr(d_query_planes),
                                            int(n_queries), _ptr(d_coll_planes), int(n_rows),
                                            _ptr(d_out), int(out_capacity), _ptr(d_out_count),
                                            _ptr(d_stats), _stream(stream)), "hoph_query_batch16")


def hoph_pair_counts(plan, d_query_planes, n_queries, d_coll_planes, n_rows, d_counts,
                     stream=None):
    return _check(load().hoph_pair_counts(plan, _ptr(d_query_planes), int(n_queries),
                                          _ptr(d_coll_planes), int(n_rows), _ptr(d_counts),
                                          _stream(stream)), "hoph_pair_counts")


def hoph_int_probe(kind, iters, d_sink, stream=None):
    return _check(load().hoph_int_probe(int(kind), int(iters), _ptr(d_sink), _stream(stream)),
                  "hoph_int_probe")


def hoph_synth_ids(seed, first, n_ids, D, kind, d_cdf, n_cdf, d_ids, stream=None):
    return _check(load().hoph_synth_ids(int(seed), int(first), int(n_ids), int(D), int(kind),
                                        _ptr(d_cdf), int(n_cdf), _ptr(d_ids), _stream(stream)),
                  "hoph_synth_ids")


def hoph_plan_enable_timing(plan, enable=True):
    return _check(load().hoph_plan_enable_timing(plan, int(bool(enable))),
                  "hoph_plan_enable_timing")


def hoph_plan_read_timing(plan):
    """Returns ([index_ms, stream_ms, count_ms, tail_ms], calls, launches)
    summed over the recorded calls, and resets."""
    ms = (ctypes.c_double * 4)()
    calls = ctypes.c_int64()
    launches = ctypes.c_int64()
    _check(load().hoph_plan_read_timing(plan, ctypes.addressof(ms), ctypes.addressof(calls),
                                        ctypes.addressof(launches)), "hoph_plan_read_timing")
    return list(ms), calls.value, launches.value


def hoph_plan_peek_timing(plan):
    """Phase times (ms) of the most recently recorded call, no reset."""
    ms = (ctypes.c_double * 4)()
    _check(load().hoph_plan_peek_timing(plan, ctypes.addressof(ms)), "hoph_plan_peek_timing")
    return list(ms)


def hoph_synth_sketch(plan, seed, D, d_offsets, n_sets, d_planes, stream=None):
    return _check(load().hoph_synth_sketch(plan, int(seed), int(D), _ptr(d_offsets), int(n_sets),
                                           _ptr(d_planes), _stream(stream)), "hoph_synth_sketch")


def hoph_check_bounded_wait(plan, limit_ns, stream=None):
    return _check(load().hoph_check_bounded_wait(plan, int(limit_ns), _stream(stream)),
                  "hoph_check_bounded_wait")


def hoph_sync_status(plan, stream=None):
    """Synchronise and return (and clear) the plan's device status word."""
    return load().hoph_sync_status(plan, _stream(stream))


# ---- convenience wrapper ---------------------------------------------------

class Plan:
    """A plan plus torch-allocated buffers for sketch / query round trips."""

    def __init__(self, D, k, k_group, a=0, b=0, perm_kind=HOPH_PERM_TABLE, minwise_k=0, seed=1,
                 thr=(7, 10), epsilon=1e-4, empty_rule="both", host_perm=None,
                 weighting=HOPH_WEIGHT_SPACE):
        self.params = make_params(D, k, k_group, a, b, perm_kind, minwise_k, seed, thr, epsilon,
                                  empty_rule, weighting)
        if host_perm is not None:
            self.handle = hoph_plan_create_with_perm(self.params, host_perm)
        else:
            self.handle = hoph_plan_create(self.params)
        self.info = hoph_plan_get_info(self.handle)
        self.exec_kwargs = dict(strategy=-1)
        self.G = self.info.groups
        self.k = k
        self.kg = k_group
        self.minwise_k = minwise_k

    def close(self):
        if self.handle:
            hoph_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_exec(self, strategy=-1, tile_rows=0, consumer_warps=0, ctas_per_sm=0, stages=0,
                 lanes_per_row=0, sketch_cta_bits=0, join_lanes=0):
        """Replace all execution knobs (kept in self.exec_kwargs)."""
        hoph_plan_set_exec(self.handle, hoph_exec(strategy, tile_rows, consumer_warps,
                                                  ctas_per_sm, stages, lanes_per_row,
                                                  sketch_cta_bits, join_lanes))
        self.exec_kwargs = dict(strategy=strategy, tile_rows=tile_rows,
                                consumer_warps=consumer_warps, ctas_per_sm=ctas_per_sm,
                                stages=stages, lanes_per_row=lanes_per_row,
                                sketch_cta_bits=sketch_cta_bits, join_lanes=join_lanes)

    def update_exec(self, **knobs):
        """Change some execution knobs, keeping the others."""
        self.set_exec(**{**self.exec_kwargs, **knobs})

    def check(self, stream=None):
        rc = hoph_sync_status(self.handle, stream)
        if rc != HOPH_OK:
            raise HophError(rc, "device status")

    def sketch(self, d_ids, d_offsets, n_sets, out=None, stream=None):
        """OPH/HOPH planes [G][n_sets][k'] (int32 storage of uint32 values)."""
        import torch
        if out is None:
            out = torch.empty((self.G, n_sets, self.kg), dtype=torch.int32,
                              device=d_offsets.device)
        oph_build_sketches(self.handle, d_ids, d_offsets, n_sets, out, stream)
        return out

    def sketch16(self, d_ids, d_offsets, n_sets, out=None, stream=None):
        """Compact sketches, int16 tensor [G][n_sets][k'] (0xFFFF = empty)."""
        import torch
        if out is None:
            out = torch.empty((self.G, n_sets, self.kg), dtype=torch.int16, device=d_offsets.device)
        oph_build_sketches16(self.handle, d_ids, d_offsets, n_sets, out, stream)
        return out

    def minwise(self, d_ids, d_offsets, n_sets, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((n_sets, self.minwise_k), dtype=torch.int32, device=d_offsets.device)
        minwise_build_sketches(self.handle, d_ids, d_offsets, n_sets, out, stream)
        return out

    def query(self, mode, q_planes, n_queries, c_planes, n_rows, capacity=1 << 16, stream=None,
              stats=False, check=True):
        """Run hoph_query_batch; returns (pairs structured ndarray, count, stats)."""
        import torch
        dev = c_planes.device
        out = torch.empty((max(capacity, 1), 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(STATS_WORDS, dtype=torch.int64, device=dev) if stats else None
        call = hoph_query_batch16 if c_planes.element_size() == 2 else hoph_query_batch
        call(self.handle, mode, q_planes, n_queries, c_planes, n_rows, out, capacity, cnt, st,
             stream)
        if check:
            rc = hoph_sync_status(self.handle, stream)
            if rc not in (HOPH_OK, HOPH_ERR_CAPACITY):
                raise HophError(rc, "hoph_query_batch (device)")
        n = int(cnt.item())
        pairs = out[:min(n, capacity)].cpu().numpy().view(PAIR_DTYPE).reshape(-1)
        st_out = None
        if stats:
            s = hoph_stats.from_buffer_copy(st.cpu().numpy().tobytes())
            st_out = s
        return pairs, n, st_out

    def self_join(self, mode, planes, n_rows, batch=1536, capacity=1 << 16, stream=None,
                  stats=False, check=True, part=0, parts=1):
        """Run hoph_self_join (hoph_self_join16 for compact 16-bit planes) over
        one collection's planes; returns (pairs structured ndarray with
        query < row, count, stats).  parts > 1: only blocks part, part +
        parts, ... (hoph_self_join_part)."""
        import torch
        dev = planes.device
        out = torch.empty((max(capacity, 1), 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(STATS_WORDS, dtype=torch.int64, device=dev) if stats else None
        if parts > 1:
            hoph_self_join_part(self.handle, mode, planes, n_rows, batch, part, parts, out,
                                capacity, cnt, st, stream)
        else:
            call = hoph_self_join16 if planes.element_size() == 2 else hoph_self_join
            call(self.handle, mode, planes, n_rows, batch, out, capacity, cnt, st, stream)
        if check:
            rc = hoph_sync_status(self.handle, stream)
            if rc not in (HOPH_OK, HOPH_ERR_CAPACITY):
                raise HophError(rc, "hoph_self_join (device)")
        n = int(cnt.item())
        pairs = out[:min(n, capacity)].cpu().numpy().view(PAIR_DTYPE).reshape(-1)
        st_out = hoph_stats.from_buffer_copy(st.cpu().numpy().tobytes()) if stats else None
        return pairs, n, st_out
