"""Host logic of the serving loop (no GPU): per-robot ordering, one scan in
flight per map, continuous batch formation within limits, and admission by
device memory (with a fake memory probe)."""
from paper_2109_13176_gb300.serve import Admission, Request, Scheduler, map_bytes
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


def test_admission_by_free_memory():
    free = [10 << 30]
    a = Admission(lambda: free[0], reserve_bytes=1 << 30)
    big = map_bytes(MapSpec(512, 512, 64, 0.1))
    assert a.admit(1, big)
    free[0] -= big
    free[0] = (1 << 30) + big // 2
    assert not a.admit(2, big)
    assert a.refused == [2]
