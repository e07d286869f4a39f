"""Host-side logic of the serving loop: the batching decision and the request trace."""
import numpy as np

from paper_2409_06765_gb300 import serve


class _R:
    def __init__(self, rid, arrival, w=64, h=48):
        self.rid, self.arrival = rid, arrival
        self.camera = type("Cam", (), {"width": w, "height": h})()


def _est_per_request(bytes_each):
    return lambda sid, reqs: bytes_each * len(reqs)


def _ids(plan):
    return [(sid, [r.rid for r in reqs]) for sid, reqs in plan]


def test_oldest_scene_goes_first_and_takes_its_queue_in_order():
    q = {0: [_R(1, 0.5), _R(2, 0.6)], 1: [_R(3, 0.2), _R(4, 0.9), _R(5, 1.0)], 2: []}
    plan = serve.plan_batch(q, max_views=4, budget_free=10**9, estimate=_est_per_request(1))
    # scene 1 (oldest request) first, then scene 0 fills the batch in arrival order
    assert _ids(plan) == [(1, [3, 4, 5]), (0, [1])]


def test_a_batch_takes_several_scenes_while_it_has_room():
    q = {0: [_R(1, 0.5)], 1: [_R(2, 0.1)], 2: [_R(3, 0.3)], 3: []}
    plan = serve.plan_batch(q, max_views=8, budget_free=10**9, estimate=_est_per_request(1))
    assert _ids(plan) == [(1, [2]), (2, [3]), (0, [1])]
    assert _ids(serve.plan_batch(q, max_views=1, budget_free=10**9, estimate=_est_per_request(1))) == [(1, [2])]


def test_batch_is_capped_by_max_views():
    q = {0: [_R(i, 0.1 * i) for i in range(10)]}
    plan = serve.plan_batch(q, max_views=4, budget_free=10**9, estimate=_est_per_request(1))
    assert _ids(plan) == [(0, [0, 1, 2, 3])]


def test_batch_is_capped_by_free_memory():
    q = {0: [_R(i, 0.1 * i) for i in range(6)], 1: [_R(9, 0.05)]}
    plan = serve.plan_batch(q, max_views=8, budget_free=25, estimate=_est_per_request(10))
    assert _ids(plan) == [(0, [0, 1])]  # the third request of scene 0 does not fit: the batch ends
    q[1][0].arrival = -1.0
    plan = serve.plan_batch(q, max_views=8, budget_free=25, estimate=_est_per_request(10))
    assert _ids(plan) == [(1, [9]), (0, [0])]


def test_nothing_launches_when_the_oldest_request_does_not_fit():
    q = {0: [_R(0, 0.0)], 1: [_R(1, 0.5)]}
    est = lambda sid, reqs: 100 if sid == 0 else 1
    assert serve.plan_batch(q, max_views=8, budget_free=50, estimate=est) is None


def test_a_younger_scene_does_not_overtake_a_scene_that_does_not_fit():
    q = {0: [_R(0, 0.0)], 1: [_R(1, 0.5)], 2: [_R(2, 0.7)]}
    est = lambda sid, reqs: 100 if sid == 1 else 1
    assert _ids(serve.plan_batch(q, max_views=8, budget_free=50, estimate=est)) == [(0, [0])]


def test_a_group_rule_splits_a_scene_queue_across_batches():
    # at most 300 pixels' worth of views per scene group; a view alone is always allowed
    q = {0: [_R(0, 0.0, 10, 10), _R(1, 0.1, 10, 10), _R(2, 0.2, 10, 20), _R(3, 0.3, 10, 10)], 1: [_R(4, 0.15)]}
    ok = lambda sid, reqs: sum(r.camera.width * r.camera.height for r in reqs) <= 300
    plan = serve.plan_batch(q, max_views=8, budget_free=10**9, estimate=_est_per_request(1), group_ok=ok)
    # scene 0 takes its first two views (400 px would not pass), then scene 1 joins the batch
    assert _ids(plan) == [(0, [0, 1]), (1, [4])]
    big = {0: [_R(0, 0.0, 100, 100)]}
    assert _ids(serve.plan_batch(big, 8, 10**9, _est_per_request(1), group_ok=ok)) == [(0, [0])]


def test_empty_queues_plan_nothing():
    assert serve.plan_batch({0: [], 1: []}, 8, 10**9, _est_per_request(1)) is None


def test_poisson_trace_is_seeded_and_has_the_requested_rate():
    a = serve.poisson_trace(200.0, 20.0, 8, seed=5)
    b = serve.poisson_trace(200.0, 20.0, 8, seed=5)
    assert [(r.scene, r.arrival, r.camera.width) for r in a] == [(r.scene, r.arrival, r.camera.width) for r in b]
    assert abs(len(a) / 20.0 - 200.0) < 200.0 * 0.1
    assert all(0 <= r.scene < 8 for r in a)
    assert {(r.camera.width, r.camera.height) for r in a} == set(serve.SERVING_SIZES)
    gaps = np.diff([r.arrival for r in a])
    assert np.all(gaps > 0) and abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0


def test_latency_summary_percentiles():
    res = [serve.Result(i, i % 3, None, arrival=float(i), launched=float(i), done=float(i) + 0.001 * (i + 1),
                        batch_views=1, batch=i // 4) for i in range(100)]
    s = serve.latency_summary(res)
    assert s["requests"] == 100
    assert abs(s["p50_ms"] - 50.5) < 1.0 and abs(s["p99_ms"] - 99.01) < 0.1
    assert s["mean_views_per_batch"] == 4.0 and 2.0 < s["mean_scenes_per_batch"] <= 3.0
    s2 = serve.latency_summary(res, skip_before_s=50.0)
    assert s2["requests"] == 50
