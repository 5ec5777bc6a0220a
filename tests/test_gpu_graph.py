"""A sketch + query step captured in a CUDA graph and replayed gives the
oracle's accepted pairs, for both comparison strategies."""
import numpy as np
import pytest

from gpu_helpers import device, oracle_tuples, pairs_tuples, planes_to_rows, to_dev, torch  # noqa
from oracle import oracle_c as oc
from paper_1805_11254_gb300 import hoph, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("strategy", [0, 1])
def test_graph_replay_matches_oracle(strategy):
    dev = device()
    w = synth.small_parity_workload(n=3000, n_queries=40)
    D, k, kg = w["D"], 128, 32
    with hoph.Plan(D, k, kg, 1, 2, seed=1, thr=(7, 10), epsilon=1e-4) as plan:
        plan.set_exec(strategy=strategy)
        d_ids, d_off = to_dev(w["ids"], dev), to_dev(w["off"], dev)
        dq_ids, dq_off = to_dev(w["q_ids"], dev), to_dev(w["q_off"], dev)
        c = plan.sketch(d_ids, d_off, 3000)
        q = torch.empty((plan.G, 40, kg), dtype=torch.int32, device=dev)
        cap = 4096
        out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)

        def step(s):
            hoph.oph_build_sketches(plan.handle, dq_ids, dq_off, 40, q, s)
            hoph.hoph_query_batch(plan.handle, "hoph", q, 40, c, 3000, out, cap, cnt, None, s)

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step(side)  # warm: scratch and tables are sized outside the capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step(torch.cuda.current_stream())
        lo = oc.layout(D, k, kg, 1, 2)
        perm = oc.permutation(D, 1)
        want = oc.query("hoph", oc.sketch(w["q_ids"], w["q_off"], lo, perm=perm),
                        oc.sketch(w["ids"], w["off"], lo, perm=perm), kg, 7, 10, 1e-4,
                        z=np.diff(lo[::kg]).astype(np.uint64))
        for _ in range(2):
            out.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_OK
            n = int(cnt.item())
            got = out[:n].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
            assert pairs_tuples(got) == oracle_tuples(want) and n > 0


@pytest.mark.parametrize("strategy", [0, 1])
def test_two_batches_in_flight_match_the_oracle(strategy):
    """Two plans, each the whole step of one batch, as two stream branches of
    one graph (the benchmark's two-batches-in-flight schedule): both give the
    oracle's pairs, replay after replay."""
    dev = device()
    w = synth.small_parity_workload(n=3000, n_queries=40)
    D, k, kg = w["D"], 128, 32
    lo = oc.layout(D, k, kg, 1, 2)
    perm = oc.permutation(D, 1)
    want = oc.query("hoph", oc.sketch(w["q_ids"], w["q_off"], lo, perm=perm),
                    oc.sketch(w["ids"], w["off"], lo, perm=perm), kg, 7, 10, 1e-4,
                    z=np.diff(lo[::kg]).astype(np.uint64))
    plans = [hoph.Plan(D, k, kg, 1, 2, seed=1, thr=(7, 10), epsilon=1e-4) for _ in range(2)]
    try:
        d_ids, d_off = to_dev(w["ids"], dev), to_dev(w["off"], dev)
        dq_ids, dq_off = to_dev(w["q_ids"], dev), to_dev(w["q_off"], dev)
        c = plans[0].sketch(d_ids, d_off, 3000)
        lanes = []
        for p in plans:
            p.set_exec(strategy=strategy)
            lanes.append(dict(plan=p, q=torch.empty((p.G, 40, kg), dtype=torch.int32, device=dev),
                              out=torch.empty((4096, 2), dtype=torch.int64, device=dev),
                              cnt=torch.zeros(1, dtype=torch.int64, device=dev)))

        def step(lane, s):
            hoph.oph_build_sketches(lane["plan"].handle, dq_ids, dq_off, 40, lane["q"], s)
            hoph.hoph_query_batch(lane["plan"].handle, "hoph", lane["q"], 40, c, 3000,
                                  lane["out"], 4096, lane["cnt"], None, s)

        for lane in lanes:
            step(lane, torch.cuda.current_stream())  # size scratch outside the capture
        torch.cuda.synchronize()
        sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cs = torch.cuda.current_stream()
            sa.wait_stream(cs)
            sb.wait_stream(cs)
            step(lanes[0], sa)
            step(lanes[1], sb)
            cs.wait_stream(sa)
            cs.wait_stream(sb)
        for _ in range(3):
            for lane in lanes:
                lane["out"].zero_()
            g.replay()
            torch.cuda.synchronize()
            for lane in lanes:
                assert hoph.hoph_sync_status(lane["plan"].handle) == hoph.HOPH_OK
                n = int(lane["cnt"].item())
                got = lane["out"][:n].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
                assert n > 0 and pairs_tuples(got) == oracle_tuples(want)
    finally:
        for p in plans:
            p.close()


def test_capture_refuses_new_plan_memory_then_works_after_a_warm_call():
    """A query captured on a fresh plan would have to allocate its scratch and
    decision table inside the capture: the call returns HOPH_ERR_CAPTURE
    before enqueuing anything.  After one uncaptured call of the same shape
    the capture succeeds and its replay gives that call's pairs."""
    dev = device()
    w = synth.small_parity_workload()
    D, k, kg = w["D"], 128, 32
    with hoph.Plan(D, k, kg, 1, 1, seed=1, thr=(7, 10), epsilon=1e-4) as plan:
        c = plan.sketch(to_dev(w["ids"], dev), to_dev(w["off"], dev), 3000)
        q = plan.sketch(to_dev(w["q_ids"], dev), to_dev(w["q_off"], dev), 40)
        plan.check()
        cap = 4096
        out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        with hoph.Plan(D, k, kg, 1, 1, seed=1, thr=(7, 10), epsilon=1e-4) as fresh:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(side):
                with torch.cuda.graph(g, stream=side):
                    with pytest.raises(hoph.HophError) as e:
                        hoph.hoph_query_batch(fresh.handle, "hoph", q, 40, c, 3000, out, cap, cnt,
                                              None, side)
                    cnt.zero_()  # keep the capture non-empty
            assert e.value.code == hoph.HOPH_ERR_CAPTURE
            torch.cuda.synchronize()
            with torch.cuda.stream(side):
                hoph.hoph_query_batch(fresh.handle, "hoph", q, 40, c, 3000, out, cap, cnt, None,
                                      side)  # warm: scratch and table sized here
                side.synchronize()
                want = out[:int(cnt.item())].clone()
                g2 = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g2, stream=side):
                    hoph.hoph_query_batch(fresh.handle, "hoph", q, 40, c, 3000, out, cap, cnt,
                                          None, side)
            torch.cuda.synchronize()
            out.zero_()
            g2.replay()
            torch.cuda.synchronize()
            fresh.check()
            assert int(cnt.item()) == len(want) > 0
            assert torch.equal(out[:len(want)], want)
