"""The C ABI library loads and exports every entry point include/elsar.h declares;
host-side argument checks answer without touching a GPU."""
import ctypes

import pytest

import paper_2305_05671_b300 as elsar


def test_library_exports_every_declared_symbol():
    L = elsar.lib()
    names = elsar.declared_symbols()
    assert {"elsar_fit_model", "elsar_partition", "elsar_sort_partitions", "elsar_sort"} <= set(names)
    for name in names:
        assert hasattr(L, name), name


def test_defaults():
    p = elsar.default_params()
    assert p.num_partitions == 1024 and p.balance == elsar.BALANCE_REFINED and p.schedule == elsar.SCHED_PERSISTENT


def test_workspace_grows_with_n():
    p = elsar.Params()
    small, big = elsar.workspace_size(1000, p), elsar.workspace_size(10**8, p)
    assert 0 < small < big
    assert big >= 2 * 16 * 10**8  # two 16-byte pair arrays
    assert elsar.model_size(10**8, p) > 8 << 17


def _status(fn, *args):
    return fn(*args)


FAKE_WS = 1 << 20  # never dereferenced: every case below is rejected before any CUDA call


@pytest.mark.parametrize("field,value", [("num_partitions", 1000), ("num_partitions", 1 << 17), ("tile_pairs", 300),
                                         ("tile_pairs", 1 << 14), ("sample_size", 1 << 24), ("balance", 2),
                                         ("schedule", 5), ("model_kind", 9), ("fine_bins_log2", 23),
                                         ("skip_checks", 8), ("key_bytes", 11), ("wait_limit_cycles", 1 << 41)])
def test_bad_params_rejected(field, value):
    p = elsar.Params(**{field: value})
    rc = elsar.lib().elsar_sort(FAKE_WS, FAKE_WS * 2, 1000, ctypes.byref(p.c()), FAKE_WS, 1 << 40, None, None)
    assert rc == 1
    assert elsar.lib().elsar_last_error()


def test_sizes_and_buffers_rejected_on_host():
    L = elsar.lib()
    p = elsar.Params().c()
    assert L.elsar_sort(FAKE_WS, FAKE_WS * 2, 1 << 32, ctypes.byref(p), FAKE_WS, 1 << 60, None, None) == 5
    assert L.elsar_sort(FAKE_WS, FAKE_WS * 2, 1000, ctypes.byref(p), FAKE_WS, 10, None, None) == 2
    assert L.elsar_sort(FAKE_WS, FAKE_WS * 2, 1000, ctypes.byref(p), FAKE_WS + 8, 1 << 40, None, None) == 1
    assert L.elsar_sort(FAKE_WS + 1, FAKE_WS * 2, 1000, ctypes.byref(p), FAKE_WS, 1 << 40, None, None) == 1
    # overlapping input and output
    assert L.elsar_sort(FAKE_WS, FAKE_WS + 400, 1000, ctypes.byref(p), FAKE_WS, 1 << 40, None, None) == 1
    assert L.elsar_fit_model(FAKE_WS, 0, ctypes.byref(p), FAKE_WS, 1 << 30, FAKE_WS, 1 << 40, None) == 1
    # n == 0 is a no-op
    assert L.elsar_sort(None, None, 0, ctypes.byref(p), FAKE_WS, 1 << 40, None, None) == 0


def test_host_async_arguments_rejected_on_host():
    L = elsar.lib()
    p = elsar.Params().c()
    assert L.elsar_sort_host_async(None, None, 1000, ctypes.byref(p), FAKE_WS, FAKE_WS, FAKE_WS, 1 << 40, None) == 1
    assert L.elsar_sort_host_async(None, None, 0, ctypes.byref(p), FAKE_WS, FAKE_WS, FAKE_WS, 1 << 40, None) == 0


def test_wait_arguments_rejected_on_host():
    L = elsar.lib()
    assert L.elsar_wait(None, 1 << 20, None) == 1  # no workspace
    assert L.elsar_wait(FAKE_WS + 16, 1 << 20, None) == 1  # not 256-byte aligned
    assert L.elsar_wait(FAKE_WS, 64, None) == 1  # smaller than the control words
    assert L.elsar_last_error()


def test_status_strings():
    L = elsar.lib()
    for s in range(7):
        assert L.elsar_status_str(s)


def test_binding_raises():
    with pytest.raises(elsar.ElsarError):
        elsar._check(2)


def test_selftest_arguments_rejected_on_host():
    L = elsar.lib()
    res = (ctypes.c_uint32 * 3)()
    # limit out of range, unaligned source, null pointers: EINVAL before any CUDA call
    assert L.elsar_selftest_bounded_wait(FAKE_WS, FAKE_WS, 0, None, ctypes.byref(res)) == 1
    assert L.elsar_selftest_bounded_wait(FAKE_WS, FAKE_WS, 5_000_000_000, None, ctypes.byref(res)) == 1
    assert L.elsar_selftest_bounded_wait(FAKE_WS + 4, FAKE_WS, 1000, None, ctypes.byref(res)) == 1
    assert L.elsar_selftest_bounded_wait(None, FAKE_WS, 1000, None, ctypes.byref(res)) == 1
    assert L.elsar_selftest_bounded_wait(FAKE_WS, FAKE_WS, 1000, None, None) == 1


def test_ooc_arguments_rejected_on_host():
    L = elsar.lib()
    p = elsar.Params().c()
    assert L.elsar_sort_ooc(FAKE_WS, FAKE_WS, 1 << 32, ctypes.byref(p), FAKE_WS, 1 << 40, None, None) == 5
    assert L.elsar_sort_ooc(FAKE_WS, FAKE_WS, 1000, ctypes.byref(p), FAKE_WS + 8, 1 << 40, None, None) == 1
    assert L.elsar_sort_ooc(None, None, 0, ctypes.byref(p), FAKE_WS, 1 << 40, None, None) == 0
    assert elsar.ooc_min_workspace(10**9) > elsar.ooc_min_workspace(10**3) > 64 << 20


def test_mlp_adam_arguments_rejected_on_host():
    L = elsar.lib()
    assert L.elsar_mlp_adam(FAKE_WS, FAKE_WS, FAKE_WS, FAKE_WS, 0, 1e-3, None) == 1  # t starts at 1
    assert L.elsar_mlp_adam(None, FAKE_WS, FAKE_WS, FAKE_WS, 1, 1e-3, None) == 1


def test_params_struct_matches_header():
    """The binding's parameter and stats structs have the sizes the header's
    field lists give (8 u32 + 2 u64 + 2 u32 + 1 u64; 8 floats + 4 u32 + 2 u64 +
    6 u32 + 2 floats)."""
    assert ctypes.sizeof(elsar._Params) == 8 * 4 + 2 * 8 + 2 * 4 + 8
    assert ctypes.sizeof(elsar._Stats) == 8 * 4 + 4 * 4 + 2 * 8 + 6 * 4 + 2 * 4
