"""Shared helpers of the GPU parity tests: build the libraries, move inputs
to the device, reshape GPU planes for comparison with the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle_c as oc  # noqa: E402
from paper_1805_11254_gb300 import build_lib, hoph  # noqa: E402

_built = False


def device():
    global _built
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not _built:
        build_lib.build()
        oc.build()
        hoph.load()
        _built = True
    return torch.device("cuda:0")


def to_dev(a, dev):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(dev)


def planes_to_rows(planes):
    """[G][n][k'] device planes -> [n][k] uint32 numpy (bins in psi order)."""
    p = planes.cpu().numpy().view(np.uint32)
    G, n, kg = p.shape
    return np.ascontiguousarray(p.transpose(1, 0, 2).reshape(n, G * kg))


def rows_to_planes(rows, kg, dev):
    """[n][k] uint32 numpy -> [G][n][k'] device planes."""
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    n, k = rows.shape
    G = k // kg
    p = np.ascontiguousarray(rows.reshape(n, G, kg).transpose(1, 0, 2))
    return to_dev(p, dev)


def pairs_tuples(pairs):
    return [(int(p["query"]), int(p["row"]), int(p["groups"]), int(p["matches"])) for p in pairs]


def oracle_tuples(res):
    return [tuple(int(v) for v in row) for row in res["accepted"]]


_perm_cache = {}


def oracle_rows(ids, off, D, k, kg, ab=(0, 0), seed=1, hashed=False):
    """The oracle's own sketches ([n][k] uint32, bins in psi order) of the
    sets (ids, off): its layout (Sec. 3.2 / 4.1) and its own psi (explicit
    Fisher-Yates table, or the 2-universal hash), nothing from the GPU."""
    lo = oc.layout(D, k, kg, *ab)
    if hashed:
        return oc.sketch(ids, off, lo, D=D, hash_ab=oc.hash_params(seed))
    key = (D, seed)
    if key not in _perm_cache:
        _perm_cache.clear()
        _perm_cache[key] = oc.permutation(D, seed)
    return oc.sketch(ids, off, lo, perm=_perm_cache[key])


def oracle_z(D, k, kg, ab=(0, 0)):
    """Group sizes z_g (values of V per group) from the oracle's layout."""
    lo = oc.layout(D, k, kg, *ab)
    return np.diff(lo[::kg]).astype(np.uint64)
