"""The multi-user dispatch policy (Sec. 6.2, Algorithm 1, Eq. 13) on the host:
dispatch order by (frames in flight, target time), the ray budget of the
device, starved frames first, denial of new clients in the starvation state,
and the wait time w_i = 1/FPS_i - t_i with t_i a moving average of completion
times."""
import pytest

from paper_2303_04086_gb300 import build, inolf

MS = 1_000_000


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def test_loaded_viewers_wait_behind_idle_ones():
    s = inolf.Scheduler()
    for v in (1, 2):
        s.set_viewer(v, 10.0, 0)           # 100 ms frame period: nothing starves here
    assert s.admit(1, 11, 100, 0) == inolf.OK
    assert s.next(0) == 11                 # viewer 1 now has one frame in flight
    assert s.admit(1, 12, 100, 1 * MS) == inolf.OK
    assert s.admit(2, 21, 100, 2 * MS) == inolf.OK
    assert s.next(3 * MS) == 21            # viewer 2 (nothing in flight) first
    assert s.next(3 * MS) == 12
    assert s.next(3 * MS) is None


def test_ray_budget_and_break():
    s = inolf.Scheduler(max_rays_in_flight=100)
    s.set_viewer(1, 10.0, 0)
    s.set_viewer(2, 10.0, 0)
    assert s.admit(1, 1, 60, 0) == inolf.OK
    assert s.admit(2, 2, 60, 0) == inolf.OK
    assert s.next(0) == 1
    assert s.next(0) is None                 # 60 + 60 > 100: the device is full
    assert s.state(0)["rays_in_flight"] == 60
    s.complete(1, 5 * MS)
    assert s.next(5 * MS) == 2


def test_wait_time_is_period_minus_moving_average():
    s = inolf.Scheduler()
    s.set_viewer(7, 50.0, 0)                 # 20 ms period
    assert s.wait_ns(7)[0] == 20 * MS        # no history yet: w = 1/FPS
    s.admit(7, 1, 10, 0)
    assert s.next(0) == 1
    s.complete(1, 4 * MS)                    # t = 4 ms
    w, target = s.wait_ns(7)
    assert w == 16 * MS and target == 4 * MS + 16 * MS
    s.admit(7, 2, 10, 5 * MS)
    assert s.next(5 * MS) == 2
    s.complete(2, 13 * MS)                   # 8 ms; moving average 0.75 * 4 + 0.25 * 8 = 5 ms
    assert s.wait_ns(7)[0] == 15 * MS


def test_starvation_dispatches_first_and_denies_new_clients():
    s = inolf.Scheduler(max_rays_in_flight=100)
    s.set_viewer(1, 100.0, 0)                # 10 ms period, last frame at 0
    s.set_viewer(2, 10.0, 0)                 # 100 ms period
    assert s.admit(2, 20, 100, 0) == inolf.OK
    assert s.next(0) == 20                   # fills the budget
    assert s.admit(1, 10, 50, 1 * MS) == inolf.OK
    assert s.next(2 * MS) is None            # budget full, viewer 1 not starved yet
    assert not s.state(2 * MS)["starving"]
    # at 11 ms viewer 1's frame has waited past its target time: starved
    assert s.state(11 * MS)["starving"]
    assert s.admit(3, 30, 10, 11 * MS) == inolf.E_BUDGET   # new client denied
    assert s.state(11 * MS)["denied"] == 1
    assert s.admit(2, 21, 10, 11 * MS) == inolf.OK          # known clients still queue
    assert s.next(11 * MS) == 10             # starved frame goes first, over the budget
    assert not s.state(11 * MS)["starving"]
    assert s.admit(3, 31, 10, 12 * MS) == inolf.OK          # starvation resolved: admitted
    s.complete(20, 20 * MS)
    assert s.next(20 * MS) in (21, 31)


def test_starved_frames_in_target_time_order():
    s = inolf.Scheduler(max_rays_in_flight=1)
    for v, fps in ((1, 100.0), (2, 200.0), (3, 50.0)):
        s.set_viewer(v, fps, 0)
    for v in (1, 2, 3):
        assert s.admit(v, v, 10, 0) == inolf.OK
    # at 100 ms all three are starved; targets 10, 5 and 20 ms
    assert [s.next(100 * MS) for _ in range(3)] == [2, 1, 3]


def test_cancel_pending_and_unknown():
    s = inolf.Scheduler()
    s.set_viewer(1, 10.0, 0)
    s.admit(1, 5, 10, 0)
    assert s.cancel(5) == inolf.OK
    assert s.next(0) is None
    assert s.cancel(5) == inolf.E_UNKNOWN_TICKET
    with pytest.raises(inolf.InolfError):
        s.complete(99, 0)
