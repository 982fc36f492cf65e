"""Argument checks of the allocation-free level entry point that run before
it touches a device, so they are tested on the CPU: the windows of a call
must lie inside the stimulus, and a window must be shorter than 2^31 ps (all
times are int32 ps)."""
import ctypes

import paper_2203_06117_gb300 as gs


def _call(num_windows, first_window, window_cycles, num_cycles, cycle_ps):
    err = ctypes.create_string_buffer(256)
    dummy = 16  # never dereferenced: the checks come first
    a = gs.gatspi_level_args(*([dummy] * 11), 1 << 20, dummy, dummy, dummy, 4, 1, 0, 8,
                             num_windows, first_window, window_cycles, num_cycles, cycle_ps, 256,
                             ctypes.cast(err, ctypes.c_char_p))
    return gs.lib().gatspi_propagate_level_noalloc(ctypes.byref(a), None), err.value.decode()


def test_windows_past_the_stimulus_are_rejected():
    gs.build()
    # 100 cycles in windows of 3 -> 34 windows (the last one ragged)
    rc, msg = _call(num_windows=5, first_window=30, window_cycles=3, num_cycles=100, cycle_ps=1000)
    assert rc == gs.EINVAL and "first_window + num_windows" in msg
    rc, msg = _call(num_windows=1, first_window=34, window_cycles=3, num_cycles=100, cycle_ps=1000)
    assert rc == gs.EINVAL and "first_window + num_windows" in msg


def test_window_length_of_2_31_ps_is_rejected():
    gs.build()
    rc, msg = _call(num_windows=1, first_window=0, window_cycles=1 << 16, num_cycles=1 << 16, cycle_ps=1 << 15)
    assert rc == gs.EINVAL and "2^31" in msg
    # one picosecond less passes this check (and fails later only for want of a GPU)
    rc, msg = _call(num_windows=1, first_window=0, window_cycles=1, num_cycles=1, cycle_ps=(1 << 31) - 1)
    assert "2^31" not in msg and "first_window" not in msg
