"""Host logic of the serving loop's admission and batching (no GPU): which waiting requests one
launch takes (RenderServer._take), with the device memory of a launch given by a stand-in."""
import collections

from paper_2507_23006_gb300.serve import RenderServer, Request


def _server(budget, max_batch=8):
    s = object.__new__(RenderServer)  # no slots, contexts or streams: _take needs none
    s.memory_budget = budget
    s.max_batch = max_batch
    s.queue = collections.deque()
    s.mem_in_use = 0
    s.in_flight = 0
    s.max_in_flight = 0
    # stand-in for the library's workspace query: 10 bytes per rendered Gaussian, 100 per camera
    s._memory = lambda n_render, cams: 10 * int(n_render) + 100 * len(cams)
    return s


def _req(s, rid, scene, selection):
    """A waiting request whose selection lists (partition, level, begin, count)."""
    n = sum(c for *_, c in selection)
    r = Request(rid, scene, f"cam{rid}", 0.0, segments=[(b, c) for _, _, b, c in selection],
                selection=selection, n_selected=n, mem_bytes=s._memory(n, [f"cam{rid}"]))
    s.queue.append(r)
    return r


def test_batches_same_scene_views_by_the_union_of_their_selections():
    s = _server(budget=10_000)
    a = _req(s, 0, "city", [(0, 0, 0, 100), (1, 1, 500, 50)])
    b = _req(s, 1, "city", [(0, 0, 0, 100), (2, 0, 300, 40)])  # shares partition 0 at level 0
    other = _req(s, 2, "park", [(0, 0, 0, 10)])
    c = _req(s, 3, "city", [(1, 1, 500, 50)])
    batch, mem = s._take()
    assert [r.rid for r in batch] == [0, 1, 3]
    # the union counts (partition 0, level 0) once: 100 + 50 + 40 Gaussians, three cameras
    assert mem == 10 * 190 + 100 * 3
    assert s.mem_in_use == mem and s.in_flight == 3 and s.max_in_flight == 3
    assert list(s.queue) == [other]


def test_head_of_line_waits_for_memory_and_order_is_kept():
    s = _server(budget=1_500)
    s.mem_in_use = 1_000
    head = _req(s, 0, "city", [(0, 0, 0, 50)])  # needs 600: does not fit beside 1000 in use
    small = _req(s, 1, "city", [(1, 0, 50, 1)])
    assert s._take() is None
    assert list(s.queue) == [head, small]  # nothing overtakes the oldest request
    s.mem_in_use = 0
    batch, mem = s._take()
    assert [r.rid for r in batch] == [0, 1] and mem == 10 * 51 + 200


def test_a_view_that_would_overflow_the_batch_memory_stays_queued_in_order():
    s = _server(budget=1_000)
    _req(s, 0, "city", [(0, 0, 0, 40)])    # 500 alone
    big = _req(s, 1, "city", [(1, 0, 40, 60)])  # the union would need 1200
    fits = _req(s, 2, "city", [(0, 0, 0, 40)])  # adds a camera only: 600
    later = _req(s, 3, "city", [(2, 0, 100, 10)])  # 800 with it: 10 * 50 + 300
    batch, mem = s._take()
    assert [r.rid for r in batch] == [0, 2, 3] and mem == 10 * 50 + 300
    assert list(s.queue) == [big]


def test_max_batch_caps_the_launch():
    s = _server(budget=10 ** 9, max_batch=3)
    for k in range(5):
        _req(s, k, "city", [(k, 0, 10 * k, 10)])
    batch, _ = s._take()
    assert [r.rid for r in batch] == [0, 1, 2]
    assert [r.rid for r in s.queue] == [3, 4]
    batch, _ = s._take()
    assert [r.rid for r in batch] == [3, 4] and not s.queue
    assert s.in_flight == 5


def test_empty_queue_takes_nothing():
    assert _server(budget=100)._take() is None
