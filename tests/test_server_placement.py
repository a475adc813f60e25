"""Placement of independent solves across GPUs (bem_server_place), on the CPU
with a faked device list: a job goes to a device with an idle worker where its
device-memory footprint fits (after evicting idle cached handles), preferring
a device that already holds its influence spectrum, then the device with the
most budget left, then the lower index.  No GPU is needed: the policy is host
code exported through the C ABI."""
import numpy as np

import paper_1612_08395_gb300.inputs as I

GB = 1 << 30


def view(budget=10 * GB, used=0, evictable=0, cached_bytes=0, idle_workers=1, has_cached=0):
    return dict(budget=budget, used=used, evictable=evictable, cached_bytes=cached_bytes,
                idle_workers=idle_workers, has_cached=has_cached)


def test_most_room_left_wins(bem_mod):
    place = bem_mod.Server.place
    assert place([view(used=6 * GB), view(used=2 * GB), view(used=4 * GB)], GB) == 1
    # ties go to the lower index
    assert place([view(used=2 * GB), view(used=2 * GB)], GB) == 0


def test_cached_spectrum_preferred(bem_mod):
    place = bem_mod.Server.place
    devs = [view(used=1 * GB), view(used=5 * GB, has_cached=1, cached_bytes=2 * GB)]
    assert place(devs, 3 * GB) == 1
    # but not when the job cannot fit there even with its cached handle
    devs = [view(used=1 * GB), view(budget=4 * GB, used=4 * GB, has_cached=1, cached_bytes=1 * GB)]
    assert place(devs, 3 * GB) == 0


def test_busy_devices_are_skipped(bem_mod):
    place = bem_mod.Server.place
    assert place([view(idle_workers=0), view(used=8 * GB)], GB) == 1
    assert place([view(idle_workers=0), view(idle_workers=0)], GB) == -1


def test_idle_cached_handles_can_be_evicted(bem_mod):
    place = bem_mod.Server.place
    # device 0 is full of idle cached handles (evictable); device 1 has running jobs
    devs = [view(used=10 * GB, evictable=10 * GB), view(used=9 * GB)]
    assert place(devs, 4 * GB) == 0
    assert place([view(used=10 * GB, evictable=3 * GB)], 4 * GB) == -1


def test_nothing_fits(bem_mod):
    place = bem_mod.Server.place
    assert place([view(budget=2 * GB), view(budget=3 * GB)], 4 * GB) == -1
    assert place([], GB) == -1


def test_request_stream_spreads_over_devices(bem_mod):
    """The Poisson request mix (sides 64..2048) placed on four faked devices of
    40 GB, one worker each, holding every job until the end: no device exceeds
    its budget, and the bytes spread evenly (the policy fills the emptiest)."""
    place = bem_mod.Server.place
    reqs = I.serving_requests(64, seed=5)
    used = [0] * 4
    placed = []
    for r in reqs:
        need = bem_mod.Server.footprint(r["n"], r["n"])
        d = place([view(budget=40 * GB, used=u) for u in used], need)
        if d < 0:
            continue
        used[d] += need
        placed.append(d)
    assert all(u <= 40 * GB for u in used)
    assert len(set(placed)) == 4
    assert max(used) - min(used) <= max(bem_mod.Server.footprint(2048, 2048), 1)
    assert len(placed) >= 0.9 * len(reqs)
    assert np.bincount(placed).min() >= 0.15 * len(placed)
