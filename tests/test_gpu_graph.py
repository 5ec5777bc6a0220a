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
