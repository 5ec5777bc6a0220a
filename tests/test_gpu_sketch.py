"""GPU sketches (oph_build_sketches, minwise_build_sketches, hoph_synth_ids)
against the CPU oracle, bit for bit, through the C ABI."""
import json
import os

import numpy as np
import pytest

from gpu_helpers import device, planes_to_rows, to_dev, torch  # noqa: F401
from oracle import oracle_c as oc
from paper_1805_11254_gb300 import hoph, synth

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gpu_sketch(plan, ids, off, dev):
    d_ids = to_dev(ids if len(ids) else np.zeros(1, np.uint32), dev)
    d_off = to_dev(off, dev)
    planes = plan.sketch(d_ids, d_off, len(off) - 1)
    plan.check()
    return planes_to_rows(planes)


@pytest.fixture(scope="module")
def small():
    return synth.small_parity_workload()


@pytest.mark.parametrize("ab,kg", [((0, 0), 32), ((1, 1), 32), ((1, 2), 16), ((2, 1), 64)])
def test_oph_hoph_sketch_parity_small_workload(small, ab, kg):
    dev = device()
    D, k = small["D"], 128
    with hoph.Plan(D, k, kg, *ab, seed=1) as plan:
        got = _gpu_sketch(plan, small["ids"], small["off"], dev)
    perm = oc.permutation(D, 1)
    want = oc.sketch(small["ids"], small["off"], oc.layout(D, k, kg, *ab), perm=perm)
    assert np.array_equal(got, want)
    qgot = None
    with hoph.Plan(D, k, kg, *ab, seed=1) as plan:
        qgot = _gpu_sketch(plan, small["q_ids"], small["q_off"], dev)
    qwant = oc.sketch(small["q_ids"], small["q_off"], oc.layout(D, k, kg, *ab), perm=perm)
    assert np.array_equal(qgot, qwant)


def test_ragged_sizes_unaligned_offsets_and_empty_sets():
    dev = device()
    D, k, kg = 1 << 12, 64, 16
    rng = np.random.default_rng(3)
    sizes = [0, 1, 2, 3, 4, 5, 7, 31, 32, 33, 127, 128, 129, 130, 1000, 0, 4095, 20000, 9]
    sets = [rng.integers(0, D, s).astype(np.uint32) for s in sizes]  # duplicates allowed
    ids, off = synth.pack_sets(sets)
    perm = oc.permutation(D, 5)
    for ab in ((0, 0), (1, 1)):
        with hoph.Plan(D, k, kg, *ab, seed=5) as plan:
            got = _gpu_sketch(plan, ids, off, dev)
        want = oc.sketch(ids, off, oc.layout(D, k, kg, *ab), perm=perm)
        assert np.array_equal(got, want)
        assert (got[0] == hoph.HOPH_EMPTY_VALUE).all()


def test_size_sorted_work_list_path():
    """Enough sets to switch on the size-bucket work list (> 2 per resident warp)."""
    dev = device()
    D, k, kg = 1 << 20, 256, 64
    n = 60000
    sizes = synth.lognormal_sizes(n, 60, 1.0, 1, 3000, 21)
    off = synth.offsets_from_sizes(sizes)
    cdf = synth.zipf_cdf(D, 1.1)
    ids = synth.counter_zipf_ids(7, 0, int(off[-1]), cdf)
    perm = oc.permutation(D, 1)
    with hoph.Plan(D, k, kg, 1, 2, seed=1) as plan:
        got = _gpu_sketch(plan, ids, off, dev)
    want = oc.sketch(ids, off, oc.layout(D, k, kg, 1, 2), perm=perm)
    assert np.array_equal(got, want)


def test_id_out_of_range_is_flagged_and_skipped():
    dev = device()
    D, k, kg = 1000, 8, 8
    ids = np.asarray([5, 999, 1000, 77, 123456], dtype=np.uint32)
    off = np.asarray([0, 2, 5], dtype=np.int64)
    with hoph.Plan(D, k, kg, seed=2) as plan:
        planes = plan.sketch(to_dev(ids, dev), to_dev(off, dev), 2)
        assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_ERR_ID_RANGE
        assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_OK  # cleared
    got = planes_to_rows(planes)
    ok_ids = np.asarray([5, 999, 77], dtype=np.uint32)
    want = oc.sketch(ok_ids, np.asarray([0, 2, 3]), oc.layout(D, k, kg), perm=oc.permutation(D, 2))
    assert np.array_equal(got, want)


def test_hash_permutation_sketch_parity():
    """D = 2^32 through psi(x) = ((a x + b) mod 2^61-1) >> 29, (2:1)HOPH, k = 512."""
    dev = device()
    D, k, kg = 1 << 32, 512, 128
    rng = np.random.default_rng(4)
    sizes = [0, 1, 1000, 2345, 50000, 7, 100000]
    sets = [rng.integers(0, 1 << 32, s, dtype=np.uint64).astype(np.uint32) for s in sizes]
    ids, off = synth.pack_sets(sets)
    with hoph.Plan(D, k, kg, 2, 1, perm_kind=hoph.HOPH_PERM_HASH61, seed=1) as plan:
        got = _gpu_sketch(plan, ids, off, dev)
    want = oc.sketch(ids, off, oc.layout(D, k, kg, 2, 1), D=D, hash_ab=oc.hash_params(1))
    assert np.array_equal(got, want)


def test_minwise_parity():
    dev = device()
    D, mk = 1 << 12, 64
    rng = np.random.default_rng(6)
    sets = [rng.choice(D, s, replace=False).astype(np.uint32) for s in (0, 1, 40, 300, 33)]
    ids, off = synth.pack_sets(sets)
    with hoph.Plan(D, 64, 64, minwise_k=mk, seed=3) as plan:
        got = plan.minwise(to_dev(ids, dev), to_dev(off, dev), len(sets))
        plan.check()
    perms = np.stack([oc.permutation(D, 3 + t) for t in range(mk)])
    want = oc.minwise(ids, off, perms)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), want)


def test_paper_examples_on_gpu():
    """Sec. 3.2 and Sec. 4.1 worked examples with psi = identity."""
    dev = device()
    g = json.load(open(os.path.join(GOLD, "worked_examples.json")))
    sets = g["oph_example"]["sets"]
    ids, off = synth.pack_sets([np.asarray(s, dtype=np.uint32) for s in sets])
    ident = np.arange(16, dtype=np.uint32)
    E = hoph.HOPH_EMPTY_VALUE
    with hoph.Plan(16, 4, 4, host_perm=ident) as plan:
        got = _gpu_sketch(plan, ids, off, dev)
    want = [[E if v is None else v for v in s] for s in g["oph_example"]["sketches"]]
    assert got.tolist() == want
    with hoph.Plan(16, 6, 2, 1, 1, host_perm=ident) as plan:
        got = _gpu_sketch(plan, ids, off, dev)
    printed = g["hoph_example"]["sketches_printed"]
    for row, p in zip(got.tolist(), printed):
        flat = [E if v is None else v for grp in p for v in grp]
        assert row == flat


@pytest.mark.parametrize("kind", [0, 1])
def test_synth_ids_match_host_twin(kind):
    dev = device()
    n, first, seed = 100003, 12345, 99
    D = 1 << 20
    out = torch.empty(n, dtype=torch.int32, device=dev)
    if kind == 0:
        hoph.hoph_synth_ids(seed, first, n, D, 0, None, 0, out)
        want = synth.counter_ids(seed, first, n, D)
    else:
        cdf = synth.zipf_cdf(D, 1.1)
        d_cdf = torch.from_numpy(cdf).to(dev)
        hoph.hoph_synth_ids(seed, first, n, D, 1, d_cdf, len(cdf), out)
        want = synth.counter_zipf_ids(seed, first, n, cdf)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("bits", [0, 10, 13, 64])
@pytest.mark.parametrize("hash_perm", [False, True])
def test_large_sets_take_the_cta_path(hash_perm, bits):
    """With a work list (>= 64 sets), the large sets are sketched by a whole
    CTA (from 2,048 IDs by default, from 2^(bits-1) IDs with the
    sketch_cta_bits knob, never with 64); the result must not depend on which
    path a set took."""
    dev = device()
    rng = np.random.default_rng(12)
    big = [2047, 2048, 2049, 4096, 5000, 30001, 100000]
    sizes = big + list(rng.integers(0, 300, 90)) + [0, 1, 3]
    rng.shuffle(sizes)
    if hash_perm:
        D, k, kg, ab = 1 << 32, 512, 128, (2, 1)
        sets = [rng.integers(0, 1 << 32, s, dtype=np.uint64).astype(np.uint32) for s in sizes]
    else:
        D, k, kg, ab = 1 << 20, 256, 64, (1, 2)
        sets = [rng.integers(0, D, s).astype(np.uint32) for s in sizes]
    ids, off = synth.pack_sets(sets)
    kind = hoph.HOPH_PERM_HASH61 if hash_perm else hoph.HOPH_PERM_TABLE
    with hoph.Plan(D, k, kg, *ab, perm_kind=kind, seed=3) as plan:
        plan.update_exec(sketch_cta_bits=bits)  # which sets get a CTA: never the result
        got = _gpu_sketch(plan, ids, off, dev)
    lo = oc.layout(D, k, kg, *ab)
    if hash_perm:
        want = oc.sketch(ids, off, lo, D=D, hash_ab=oc.hash_params(3))
    else:
        want = oc.sketch(ids, off, lo, perm=oc.permutation(D, 3))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("hash_perm", [False, True])
def test_generated_sets_sketch_like_stored_ones(hash_perm):
    """hoph_synth_sketch (IDs generated in the kernel) equals the oracle's
    sketch of the host-regenerated IDs, through both the warp and CTA paths."""
    dev = device()
    rng = np.random.default_rng(21)
    sizes = np.concatenate([rng.integers(0, 3000, 150), [2048, 9000, 40000]]).astype(np.int64)
    off = synth.offsets_from_sizes(sizes) + 12345  # any element window of the stream
    if hash_perm:
        D, k, kg, ab, kind = 1 << 32, 512, 128, (2, 1), hoph.HOPH_PERM_HASH61
    else:
        D, k, kg, ab, kind = 1 << 20, 256, 64, (1, 2), hoph.HOPH_PERM_TABLE
    seed = 77
    with hoph.Plan(D, k, kg, *ab, perm_kind=kind, seed=5) as plan:
        planes = torch.empty((plan.G, len(sizes), kg), dtype=torch.int32, device=dev)
        hoph.hoph_synth_sketch(plan.handle, seed, D, to_dev(off, dev), len(sizes), planes)
        plan.check()
        got = planes_to_rows(planes)
    ids = synth.counter_ids(seed, int(off[0]), int(off[-1] - off[0]), D)
    lo = oc.layout(D, k, kg, *ab)
    if hash_perm:
        want = oc.sketch(ids, off - off[0], lo, D=D, hash_ab=oc.hash_params(5))
    else:
        want = oc.sketch(ids, off - off[0], lo, perm=oc.permutation(D, 5))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("ab,kg", [((0, 0), 32), ((1, 2), 64)])
def test_compact_sketches_are_the_offsets_in_16_bits(small, ab, kg):
    """oph_build_sketches16: the oracle's values, empty bins as 0xFFFF."""
    dev = device()
    D, k = small["D"], 128
    with hoph.Plan(D, k, kg, *ab, seed=1) as plan:
        assert plan.info.max_bin_width <= 0xFFFF
        d_ids, d_off = to_dev(small["ids"], dev), to_dev(small["off"], dev)
        got = plan.sketch16(d_ids, d_off, len(small["off"]) - 1)
        plan.check()
    want = oc.sketch(small["ids"], small["off"], oc.layout(D, k, kg, *ab),
                     perm=oc.permutation(D, 1))
    want16 = np.where(want == hoph.HOPH_EMPTY_VALUE, hoph.HOPH_EMPTY_VALUE16, want)
    rows = got.cpu().numpy().view(np.uint16).transpose(1, 0, 2).reshape(len(want), -1)
    assert np.array_equal(rows, want16.astype(np.uint16))


def test_compact_sketches_need_bins_of_at_most_65535_values():
    dev = device()
    with hoph.Plan(1 << 20, 8, 8, seed=1) as plan:  # bins of 131,072 values
        assert plan.info.max_bin_width == 1 << 17
        out = torch.empty((1, 1, 8), dtype=torch.int16, device=dev)
        off = to_dev(np.zeros(2, dtype=np.int64), dev)
        with pytest.raises(hoph.HophError) as e:
            hoph.oph_build_sketches16(plan.handle, off, off, 1, out)
        assert e.value.code == hoph.HOPH_ERR_UNSUPPORTED
        # the compact query and self-join refuse such a plan too
        pairs = torch.empty((4, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        planes = torch.full((1, 3, 8), -1, dtype=torch.int16, device=dev)
        with pytest.raises(hoph.HophError) as e:
            hoph.hoph_query_batch16(plan.handle, "oph_full", planes, 3, planes, 3, pairs, 4, cnt)
        assert e.value.code == hoph.HOPH_ERR_UNSUPPORTED
        with pytest.raises(hoph.HophError) as e:
            hoph.hoph_self_join16(plan.handle, "oph_full", planes, 3, 2, pairs, 4, cnt)
        assert e.value.code == hoph.HOPH_ERR_UNSUPPORTED


@pytest.mark.parametrize("n", [64, 4096, 4097, 16383, 16384])
def test_work_list_shapes_at_their_boundaries(n):
    """The work list in one CTA (<= 4,096 sets) or three kernels, one launch
    or two (>= 16,384 sets): the same sketches as the oracle either way."""
    dev = device()
    D, k, kg = 1 << 16, 128, 32
    rng = np.random.default_rng(n)
    sizes = rng.integers(0, 600, n)
    sizes[rng.integers(0, n, 3)] = [2048, 3000, 5000]
    off = synth.offsets_from_sizes(sizes)
    ids = synth.counter_ids(5, 0, int(off[-1]), D)
    with hoph.Plan(D, k, kg, 1, 1, seed=4) as plan:
        got = _gpu_sketch(plan, ids, off, dev)
    want = oc.sketch(ids, off, oc.layout(D, k, kg, 1, 1), perm=oc.permutation(D, 4))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("D,k", [(1 << 20, 256), (24, 8)])
def test_frequent_small_ids_take_the_bitmask_path(D, k):
    """IDs below 32 (the most frequent words of a frequency-ranked
    vocabulary) are collected as bits and applied once per set: sets made
    mostly of them, on the warp and the CTA paths and in a one-launch batch,
    give the oracle's sketches; with a universe smaller than 32 the IDs at or
    beyond it are still flagged and skipped."""
    dev = device()
    rng = np.random.default_rng(55)
    sizes = list(rng.integers(1, 200, 150)) + [5000, 12000, 0, 3]
    sets = []
    for s in sizes:
        x = rng.integers(0, 32, s)
        tail = rng.integers(0, min(D, 1 << 20), s)
        sets.append(np.where(rng.random(s) < 0.8, x, tail).astype(np.uint32))
    valid = [st[st < D] for st in sets]
    ids, off = synth.pack_sets(sets)
    vids, voff = synth.pack_sets(valid)
    for n_rep in (1, 130):  # one launch with a work list, then two launches
        ids_r, off_r = synth.pack_sets([st for st in sets for _ in range(1)] * n_rep)
        with hoph.Plan(D, k, k, seed=4) as plan:
            planes = plan.sketch(to_dev(ids_r, dev), to_dev(off_r, dev), len(off_r) - 1)
            rc = hoph.hoph_sync_status(plan.handle)
            assert rc == (hoph.HOPH_ERR_ID_RANGE if D < 32 else hoph.HOPH_OK)
            got = planes_to_rows(planes)
        want = oc.sketch(vids, voff, oc.layout(D, k, k), perm=oc.permutation(D, 4))
        assert np.array_equal(got, np.tile(want, (n_rep, 1)))
