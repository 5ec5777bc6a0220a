"""ctypes loader for the plain C oracle (oracle/hoph_oracle.c).

TEST INFRASTRUCTURE ONLY (tests/, __graft_entry__.smoke(), bench.py's CPU
baseline legs).  ``build()`` compiles the library with gcc into this folder;
``load()`` compiles it on first use if it is missing.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hoph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MODE = {"oph_full": 0, "goph": 1, "hoph": 2, "minwise_full": 3}
RULE = {"both": 0, "either": 1, "none": 2}


def build(force=False):
    """Compile the oracle with gcc (-O2, pthreads).  Plain C, no CUDA."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class QueryParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("rule", ctypes.c_uint32),
                ("k", ctypes.c_uint32), ("kg", ctypes.c_uint32),
                ("tn", ctypes.c_uint32), ("td", ctypes.c_uint32),
                ("eps", ctypes.c_double), ("z", ctypes.POINTER(ctypes.c_uint64)),
                ("weighting", ctypes.c_uint32), ("a", ctypes.c_uint32), ("b", ctypes.c_uint32)]


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, u64, u32, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        lib.or_permutation.argtypes = [u64, u64, P]
        lib.or_permutation.restype = i32
        lib.or_hash_params.argtypes = [u64, P, P]
        lib.or_hash_psi.argtypes = [u64, u64, u64]
        lib.or_hash_psi.restype = u32
        lib.or_layout.argtypes = [u64, u32, u32, u32, u32, P]
        lib.or_layout.restype = i32
        lib.or_sketch.argtypes = [P, P, i64, P, u64, u64, u64, P, u32, P, i32]
        lib.or_sketch.restype = i32
        lib.or_minwise.argtypes = [P, P, i64, P, u64, u32, P, i32]
        lib.or_minwise.restype = i32
        lib.or_tails_double.argtypes = [u32, u32, u32, P, P]
        lib.or_tails_double.restype = i32
        lib.or_limits.argtypes = [u32, u32, u32, ctypes.c_double, P, P]
        lib.or_limits.restype = i32
        lib.or_query.argtypes = [ctypes.POINTER(QueryParams), P, i64, P, i64, P, P, P, P, i64,
                                 P, i32]
        lib.or_query.restype = i64
        lib.or_pair_counts.argtypes = [P, i64, P, i64, u32, u32, P]
        lib.or_jaccard_pairs.argtypes = [P, P, P, P, P, P, i64, P, P, i32]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def default_threads():
    return os.cpu_count() or 1


def permutation(D, seed):
    out = np.empty(D, dtype=np.uint32)
    if load().or_permutation(D, seed, _p(out)):
        raise ValueError("bad D")
    return out


def hash_params(seed):
    a = ctypes.c_uint64()
    b = ctypes.c_uint64()
    load().or_hash_params(seed, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def layout(D, k, kg, a=0, b=0):
    lo = np.empty(k + 1, dtype=np.uint64)
    if load().or_layout(D, k, kg, a, b, _p(lo)):
        raise ValueError("invalid layout")
    return lo


def sketch(ids, offsets, lo, perm=None, D=None, hash_ab=(0, 0), threads=None):
    """OPH/HOPH sketches [n][k] (bins in psi-space order)."""
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    k = len(lo) - 1
    n = len(offsets) - 1
    out = np.empty((n, k), dtype=np.uint32)
    if perm is not None:
        perm = np.ascontiguousarray(perm, dtype=np.uint32)
        D = len(perm)
    rc = load().or_sketch(_p(ids), _p(offsets), n, _p(perm), D, hash_ab[0], hash_ab[1],
                          _p(lo), k, _p(out), threads or default_threads())
    if rc:
        raise ValueError("ID out of range")
    return out


def minwise(ids, offsets, perms, threads=None):
    """MinWise sketches [n][k] from k permutation tables perms[k][D]."""
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    perms = np.ascontiguousarray(perms, dtype=np.uint32)
    k, D = perms.shape
    n = len(offsets) - 1
    out = np.empty((n, k), dtype=np.uint32)
    rc = load().or_minwise(_p(ids), _p(offsets), n, _p(perms), D, k, _p(out),
                           threads or default_threads())
    if rc:
        raise ValueError("ID out of range")
    return out


def tails(kg, tn, td):
    low = np.empty(kg + 2)
    up = np.empty(kg + 2)
    if load().or_tails_double(kg, tn, td, _p(low), _p(up)):
        raise ValueError("bad T")
    return low, up


def limits(kg, tn, td, eps):
    """(U, L) from the oracle's exact tail tests (Definition 1)."""
    U = ctypes.c_int64()
    L = ctypes.c_int64()
    if load().or_limits(kg, tn, td, float(eps), ctypes.byref(U), ctypes.byref(L)):
        raise ValueError("bad tail parameters")
    return U.value, L.value


def query(mode, qs, rs, kg, tn, td, eps, rule="both", z=None, per_pair=False,
          acc_cap=None, threads=None, weighting="space", ab=(0, 0)):
    """All-pairs comparison.  Returns dict with 'accepted' [n][4] int64
    (q, r, groups, matched) sorted by (q, r), 'count', 'hist' [G+1][3] and,
    if per_pair, 'dec', 'groups', 'msum' arrays [Q][N].  weighting='literal'
    takes HOPH's remaining requirement from Algorithm 2's recursion with
    r = a/(a+b), ab = (a, b)."""
    qs = np.ascontiguousarray(qs, dtype=np.uint32)
    rs = np.ascontiguousarray(rs, dtype=np.uint32)
    Q, k = qs.shape
    N = rs.shape[0]
    G = k // kg if MODE[mode] in (1, 2) else 1
    zz = np.ascontiguousarray(z if z is not None else np.zeros(max(G, 1)), dtype=np.uint64)
    p = QueryParams(MODE[mode], RULE[rule], k, kg, tn, td, float(eps),
                    zz.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                    {"space": 0, "literal": 1}[weighting], ab[0], ab[1])
    dec = grp = ms = None
    if per_pair:
        dec = np.empty((Q, N), dtype=np.int8)
        grp = np.empty((Q, N), dtype=np.uint8)
        ms = np.empty((Q, N), dtype=np.uint16)
    cap = acc_cap if acc_cap is not None else max(1024, Q * 64)
    acc = np.empty((cap, 4), dtype=np.int64)
    hist = np.zeros((G + 1, 3), dtype=np.int64)
    n = load().or_query(ctypes.byref(p), _p(qs), Q, _p(rs), N, _p(dec), _p(grp), _p(ms),
                        _p(acc), cap, _p(hist), threads or default_threads())
    if n < 0:
        raise ValueError("oracle query failed (%d)" % n)
    if n > cap:
        return query(mode, qs, rs, kg, tn, td, eps, rule, z, per_pair, n, threads, weighting, ab)
    out = {"accepted": acc[:n].copy(), "count": int(n), "hist": hist}
    if per_pair:
        out.update(dec=dec, groups=grp, msum=ms)
    return out


def pair_counts(qs, rs, kg):
    qs = np.ascontiguousarray(qs, dtype=np.uint32)
    rs = np.ascontiguousarray(rs, dtype=np.uint32)
    Q, k = qs.shape
    N = rs.shape[0]
    out = np.empty((Q, N, k // kg, 3), dtype=np.uint16)
    load().or_pair_counts(_p(qs), Q, _p(rs), N, k, kg, _p(out))
    return out


def jaccard_pairs(a_ids, a_off, b_ids, b_off, pa, pb, threads=None):
    """(|A n B|, |A u B|) for each pair (a set pa[i], b set pb[i])."""
    a_ids = np.ascontiguousarray(a_ids, dtype=np.uint32)
    b_ids = np.ascontiguousarray(b_ids, dtype=np.uint32)
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    b_off = np.ascontiguousarray(b_off, dtype=np.int64)
    pa = np.ascontiguousarray(pa, dtype=np.int64)
    pb = np.ascontiguousarray(pb, dtype=np.int64)
    inter = np.empty(len(pa), dtype=np.int64)
    uni = np.empty(len(pa), dtype=np.int64)
    load().or_jaccard_pairs(_p(a_ids), _p(a_off), _p(b_ids), _p(b_off), _p(pa), _p(pb),
                            len(pa), _p(inter), _p(uni), threads or default_threads())
    return inter, uni
