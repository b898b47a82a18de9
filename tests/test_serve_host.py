"""Host logic of the serving loop (no GPU): per-robot ordering, one scan in
flight per map, continuous batch formation within limits, and per-scan
admission by a device-memory budget (maps created on a robot's first scan,
robots waiting for memory retried when memory is released, idle maps given
back, oversized scans refused)."""
from paper_2109_13176_gb300.serve import Admission, FrontDoor, Request, Scheduler, map_bytes
from synth import MapSpec


def reqs(spec):
    return [Request(robot=r, n_points=n, arrival=t, seq=i) for i, (t, r, n) in enumerate(spec)]


def test_batches_take_oldest_scan_of_each_idle_robot():
    s = Scheduler(max_batch_maps=8, max_batch_points=10_000)
    for q in reqs([(0.0, 1, 100), (0.1, 2, 100), (0.2, 1, 100), (0.3, 3, 100)]):
        s.arrive(q)
    b = s.next_batch()
    assert [(q.robot, q.arrival) for q in b] == [(1, 0.0), (2, 0.1), (3, 0.3)]
    # robot 1's second scan waits while its first is on the GPU
    assert s.next_batch() == []
    s.finish(b)
    b2 = s.next_batch()
    assert [(q.robot, q.arrival) for q in b2] == [(1, 0.2)]
    assert s.pending() == 0


def test_limits_on_maps_and_points_keep_order():
    s = Scheduler(max_batch_maps=2, max_batch_points=250)
    for q in reqs([(0.0, 1, 100), (0.1, 2, 100), (0.2, 3, 100), (0.3, 4, 10)]):
        s.arrive(q)
    b = s.next_batch()
    assert [q.robot for q in b] == [1, 2]  # map limit
    b2 = s.next_batch()
    assert [q.robot for q in b2] == [3, 4]
    s.finish(b)
    s.finish(b2)
    s2 = Scheduler(max_batch_maps=8, max_batch_points=250)
    for q in reqs([(0.0, 1, 200), (0.1, 2, 100), (0.2, 3, 40)]):
        s2.arrive(q)
    b = s2.next_batch()
    assert [q.robot for q in b] == [1, 3]  # robot 2 does not fit; robot 3 does
    s2.finish(b)
    assert [q.robot for q in s2.next_batch()] == [2]


def test_per_robot_sequence_is_preserved_under_load():
    s = Scheduler(max_batch_maps=4, max_batch_points=1 << 30)
    seen = {}
    for i in range(40):
        s.arrive(Request(robot=i % 5, n_points=10, arrival=float(i), seq=i // 5))
    while s.pending():
        b = s.next_batch()
        assert len({q.robot for q in b}) == len(b)
        for q in b:
            assert seen.get(q.robot, -1) == q.seq - 1
            seen[q.robot] = q.seq
        s.finish(b)
    assert all(v == 7 for v in seen.values())


def test_admission_budget_holds_and_releases():
    a = Admission.from_free_memory(lambda: 10 << 30, reserve_bytes=1 << 30, extra_bytes=1 << 30)
    assert a.budget == 8 << 30
    big = map_bytes(MapSpec(512, 512, 64, 0.1))
    assert a.try_hold(1, big) and a.used == big
    assert a.try_hold(1, big) and a.used == big        # already held: no second charge
    b = Admission(big + big // 2)
    assert b.try_hold(1, big)
    assert not b.try_hold(2, big) and b.refusals == 1
    b.release(1)
    assert b.used == 0 and b.releases == 1
    assert b.try_hold(2, big)


class FakeGpu:
    def __init__(self):
        self.created, self.released = [], []


def door_with(budget, sizes, max_points=1000):
    gpu = FakeGpu()
    sched = Scheduler(max_batch_maps=8, max_batch_points=max_points)
    door = FrontDoor(Admission(budget), sched, lambda r: sizes[r], gpu.created.append, gpu.released.append,
                     max_points)
    return door, sched, gpu


def test_maps_are_created_on_a_robots_first_scan_within_the_budget():
    door, sched, gpu = door_with(budget=250, sizes={1: 100, 2: 100, 3: 100})
    assert door.offer(Request(1, 10, 0.0), 0.0) == "admitted"
    assert door.offer(Request(1, 10, 0.1, seq=1), 0.1) == "admitted"   # the map exists: no new charge
    assert door.offer(Request(2, 10, 0.2), 0.2) == "admitted"
    assert gpu.created == [1, 2] and door.adm.used == 200
    # robot 3 does not fit: its scans wait, in order, and nothing is created
    assert door.offer(Request(3, 10, 0.3, seq=0), 0.3) == "waiting"
    assert door.offer(Request(3, 10, 0.4, seq=1), 0.4) == "waiting"
    assert gpu.created == [1, 2] and door.pending() == 2
    assert [q.robot for q in sched.next_batch()] == [1, 2]
    # no memory was released: retrying changes nothing
    assert door.retry(0.5) == 0


def test_waiting_robot_is_admitted_when_an_idle_map_is_released():
    door, sched, gpu = door_with(budget=250, sizes={1: 100, 2: 100, 3: 100})
    door.offer(Request(1, 10, 0.0), 0.0)
    door.offer(Request(2, 10, 0.0), 0.0)
    door.offer(Request(3, 10, 0.1, seq=0), 0.1)
    door.offer(Request(3, 10, 0.2, seq=1), 0.2)
    b = sched.next_batch()
    assert [q.robot for q in b] == [1, 2]
    sched.finish([q for q in b if q.robot == 2])
    # robot 1 is still on the GPU: only robot 2, idle for 5 s, gives its map back
    assert door.release_idle(5.0, idle_s=1.0) == [2]
    assert gpu.released == [2]
    sched.finish([q for q in b if q.robot == 1])
    # the release lets robot 3 in, both of its scans in order
    assert door.retry(5.0) == 2 and gpu.created == [1, 2, 3]
    assert door.pending() == 0
    order = []
    while sched.pending():
        bb = sched.next_batch()
        order += [(q.robot, q.seq) for q in bb]
        sched.finish(bb)
    assert [x for x in order if x[0] == 3] == [(3, 0), (3, 1)]
    # a released robot that comes back gets a new map if it fits
    assert door.release_idle(20.0, idle_s=1.0) == [1, 3]
    assert door.offer(Request(2, 10, 21.0), 21.0) == "admitted" and gpu.created[-1] == 2


def test_oversized_scan_is_refused_not_queued():
    # a scan larger than a batch's staging would never be scheduled
    door, sched, gpu = door_with(budget=1000, sizes={1: 100}, max_points=500)
    assert door.offer(Request(1, 501, 0.0), 0.0) == "rejected"
    assert door.offer(Request(1, 500, 0.1), 0.1) == "admitted"
    assert len(door.rejected) == 1 and sched.pending() == 1
    assert [q.n_points for q in sched.next_batch()] == [500]


def test_a_map_larger_than_the_budget_never_blocks_others():
    door, sched, gpu = door_with(budget=150, sizes={1: 200, 2: 100})
    assert door.offer(Request(1, 10, 0.0), 0.0) == "waiting"
    assert door.offer(Request(2, 10, 0.0), 0.0) == "admitted"
    assert [q.robot for q in sched.next_batch()] == [2]
