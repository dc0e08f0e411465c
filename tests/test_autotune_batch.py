"""Host logic of the batch-level tuner (autotune.tune_batch) against a fake
library and a fake device clock: the chosen knobs are those of the fastest
timed candidate, changes within min_gain are reverted, and every width stays
in [2, 20] with the reduction chunk capped at c - 1."""
import types

import pytest

from paper_2501_03245_gb300 import autotune


class FakeLib:
    """ecc_msm_window / set_window / set_reduce_chunk over dictionaries."""

    def __init__(self, widths):
        self.w = dict(widths)
        self.chunk = {}

    def ecc_msm_window(self, curve, n):
        return self.w[n.bit_length() - 1]

    def ecc_msm_set_window(self, curve, l, c):
        assert 2 <= c <= 20
        self.w[l] = c

    def ecc_msm_set_reduce_chunk(self, curve, l, k):
        assert 1 <= k <= self.w[l] - 1
        self.chunk[l] = k


def fake_torch(clock):
    class Event:
        def __init__(self, enable_timing=True):
            self.t = None

        def record(self):
            self.t = clock[0]

        def elapsed_time(self, other):
            return other.t - self.t

    cuda = types.SimpleNamespace(Event=Event, synchronize=lambda: None)
    return types.SimpleNamespace(cuda=cuda)


def run_tuner(monkeypatch, widths, cost, **kw):
    lib = FakeLib(widths)
    monkeypatch.setattr(autotune, "ecc", lib)
    clock = [0.0]

    def run():
        clock[0] += cost(lib)

    out = autotune.tune_batch(0, sorted(widths), run, fake_torch(clock), **kw)
    return lib, out


def test_picks_the_fastest_shift_and_chunk(monkeypatch):
    widths = {10: 8, 11: 8, 14: 13, 17: 15}
    target = {10: 7, 11: 7, 14: 12, 17: 14}  # shift -1 is best

    def cost(lib):
        t = 100.0 + sum(abs(lib.w[l] - target[l]) for l in target)
        t += 0.5 * abs(lib.chunk.get(17, 4) - 5)
        return t

    lib, out = run_tuner(monkeypatch, widths, cost)
    assert out["shift"] == -1 and out["chunk_log2"] == 5
    assert lib.w == target
    assert all(lib.chunk[l] == min(5, lib.w[l] - 1) for l in widths)
    assert out["widths"] == target


def test_group_width_change_kept_only_above_min_gain(monkeypatch):
    widths = {10: 8, 14: 13, 17: 15}

    def cost(lib):
        # 15 -> 14 for the largest class gains 2%, 8 -> 9 gains 0.1%
        t = 100.0
        if lib.w[17] == 14:
            t -= 2.0
        if lib.w[10] == 9:
            t -= 0.1
        if lib.w[14] != 13 or lib.w[10] not in (8, 9) or lib.w[17] not in (14, 15):
            t += 10.0
        return t

    lib, out = run_tuner(monkeypatch, widths, cost, shifts=(0,), chunks=(4,))
    assert lib.w == {10: 8, 14: 13, 17: 14}
    assert out["widths"] == {10: 8, 14: 13, 17: 14}


@pytest.mark.parametrize("widths", [{10: 2, 11: 3}, {17: 20, 18: 19}])
def test_widths_stay_in_range(monkeypatch, widths):
    lib, out = run_tuner(monkeypatch, widths, lambda lib: 1.0, shifts=(-1, 0, 1))
    assert all(2 <= c <= 20 for c in lib.w.values())
