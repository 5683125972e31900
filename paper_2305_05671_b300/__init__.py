"""Python binding of libelsar (include/elsar.h): argument marshalling only.

Every step of the sort runs in the CUDA kernels of libelsar.so; this module
turns torch tensors into pointers, calls the C ABI and raises on errors.  It
refuses to run when the library is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass, fields

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libelsar.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "elsar.h")
RECORD = 100

MODEL_RMI, MODEL_MLP, MODEL_RADIX = 0, 1, 2
SKIP_BOUNDARY, SKIP_JUDGE, SKIP_IMBALANCE = 1, 2, 4
BALANCE_PAPER, BALANCE_REFINED = 0, 1
SCHED_PER_PARTITION, SCHED_PERSISTENT = 0, 1


class ElsarError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"elsar status {status}: {message}")
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("num_partitions", ctypes.c_uint32), ("fine_bins_log2", ctypes.c_uint32),
                ("leaf_target", ctypes.c_uint32), ("max_depth", ctypes.c_uint32), ("model_kind", ctypes.c_uint32),
                ("balance", ctypes.c_uint32), ("schedule", ctypes.c_uint32), ("tile_pairs", ctypes.c_uint32),
                ("sample_size", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("skip_checks", ctypes.c_uint32),
                ("key_bytes", ctypes.c_uint32), ("wait_limit_cycles", ctypes.c_uint64)]


class _Stats(ctypes.Structure):
    _fields_ = [("pass_ms", ctypes.c_float * 8), ("launches", ctypes.c_uint32), ("num_items", ctypes.c_uint32),
                ("oversize_items", ctypes.c_uint32), ("model_nodes", ctypes.c_uint32),
                ("max_partition", ctypes.c_uint64), ("max_bin", ctypes.c_uint64), ("model_used", ctypes.c_uint32),
                ("fallback_reason", ctypes.c_uint32), ("judge_buckets", ctypes.c_uint32),
                ("judge_rmi_max", ctypes.c_uint32), ("judge_mlp_max", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("F_first_knot", ctypes.c_float), ("F_last_knot", ctypes.c_float)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("tile_pairs", ctypes.c_uint32), ("records_per_bin_log2", ctypes.c_uint32 * 3),
                ("total_records", ctypes.c_uint64), ("total_bins", ctypes.c_uint64), ("sample_keys", ctypes.c_uint64),
                ("launches", ctypes.c_uint32), ("tuning_runs", ctypes.c_uint32), ("tuning_ms", ctypes.c_float * 16)]


class _OocStats(ctypes.Structure):
    _fields_ = [("phase_ms", ctypes.c_float * 4), ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
                ("chunks", ctypes.c_uint32), ("groups", ctypes.c_uint32), ("chunk_records", ctypes.c_uint64),
                ("group_records", ctypes.c_uint64), ("model_used", ctypes.c_uint32),
                ("fallback_reason", ctypes.c_uint32), ("max_partition", ctypes.c_uint64)]


@dataclass
class Params:
    """elsar_params; zero means "library default"."""

    num_partitions: int = 1024
    fine_bins_log2: int = 0
    leaf_target: int = 16
    max_depth: int = 32
    model_kind: int = MODEL_RMI
    balance: int = BALANCE_REFINED
    schedule: int = SCHED_PERSISTENT
    tile_pairs: int = 0
    sample_size: int = 0
    seed: int = 0x5EED
    skip_checks: int = 0
    key_bytes: int = 0
    wait_limit_cycles: int = 0

    def c(self) -> _Params:
        return _Params(*[getattr(self, f.name) for f in fields(self)])


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, U64, SZ = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t
        PP = ctypes.POINTER(_Params)
        sig = {
            "elsar_default_params": (None, [PP]),
            "elsar_workspace_size": (SZ, [U64, PP]),
            "elsar_model_size": (SZ, [U64, PP]),
            "elsar_fit_model": (ctypes.c_int, [P, U64, PP, P, SZ, P, SZ, P]),
            "elsar_partition": (ctypes.c_int, [P, P, U64, PP, P, P, P, P, SZ, P]),
            "elsar_sort_partitions": (ctypes.c_int, [P, U64, PP, P, P, P, P, SZ, P]),
            "elsar_sort": (ctypes.c_int, [P, P, U64, PP, P, SZ, P, ctypes.POINTER(_Stats)]),
            "elsar_sort_host": (ctypes.c_int, [P, P, U64, PP, P, P, P, SZ, P]),
            "elsar_wait": (ctypes.c_int, [P, SZ, P]),
            "elsar_sort_host_async": (ctypes.c_int, [P, P, U64, PP, P, P, P, SZ, P]),
            "elsar_sort_noalloc": (ctypes.c_int, [P, P, U64, PP, P]),
            "elsar_ooc_min_workspace": (SZ, [U64, PP]),
            "elsar_selftest_bounded_wait": (ctypes.c_int, [P, P, U64, P, ctypes.POINTER(ctypes.c_uint32 * 3)]),
            "elsar_sort_ooc": (ctypes.c_int, [P, P, U64, PP, P, SZ, P, ctypes.POINTER(_OocStats)]),
            "elsar_mlp_grad_workspace": (SZ, [U64]),
            "elsar_mlp_eval": (ctypes.c_int, [P, P, P, U64, P, P]),
            "elsar_mlp_grad": (ctypes.c_int, [P, P, P, P, U64, P, P, SZ, P]),
            "elsar_mlp_splitters": (ctypes.c_int, [P, P, ctypes.c_uint32, P, P]),
            "elsar_mlp_adam": (ctypes.c_int, [P, P, P, P, ctypes.c_uint32, ctypes.c_float, P]),
            "elsar_batch_workspace_size": (SZ, [P, ctypes.c_uint32, PP]),
            "elsar_batch_create": (ctypes.c_int, [P, P, P, ctypes.c_uint32, PP, P, SZ, P, ctypes.POINTER(P)]),
            "elsar_batch_run": (ctypes.c_int, [P, P]),
            "elsar_batch_wait": (ctypes.c_int, [P, P]),
            "elsar_batch_describe": (ctypes.c_int, [P, ctypes.POINTER(_BatchInfo)]),
            "elsar_batch_destroy": (None, [P]),
            "elsar_status_str": (ctypes.c_char_p, [ctypes.c_int]),
            "elsar_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_symbols() -> list[str]:
    """Function names declared in include/elsar.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(elsar_[a-z_]+)\s*\(", txt)))


def _check(rc: int):
    if rc != 0:
        L = lib()
        raise ElsarError(rc, f"{L.elsar_status_str(rc).decode()}: {L.elsar_last_error().decode()}")


def _ptr(t) -> int | None:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data  # numpy


def _stream(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _nbytes(t) -> int:
    return t.numel() * t.element_size() if hasattr(t, "numel") else t.nbytes


def default_params() -> Params:
    c = _Params()
    lib().elsar_default_params(ctypes.byref(c))
    return Params(*[getattr(c, f.name) for f in fields(Params)])


def workspace_size(n: int, p: Params | None = None) -> int:
    return int(lib().elsar_workspace_size(n, ctypes.byref((p or Params()).c())))


def model_size(n: int, p: Params | None = None) -> int:
    return int(lib().elsar_model_size(n, ctypes.byref((p or Params()).c())))


def alloc_workspace(n: int, p: Params | None = None, device="cuda"):
    import torch

    return torch.empty(max(256, workspace_size(n, p)), dtype=torch.uint8, device=device)


def fit_model(d_records, n: int, p: Params, d_model, ws, stream=None):
    _check(lib().elsar_fit_model(_ptr(d_records), n, ctypes.byref(p.c()), _ptr(d_model), _nbytes(d_model), _ptr(ws),
                                 _nbytes(ws), _stream(stream)))


def partition(d_model, d_records, n: int, p: Params, d_pairs, d_bin_offsets, d_part_offsets, ws, stream=None):
    _check(lib().elsar_partition(_ptr(d_model), _ptr(d_records), n, ctypes.byref(p.c()), _ptr(d_pairs),
                                 _ptr(d_bin_offsets), _ptr(d_part_offsets), _ptr(ws), _nbytes(ws), _stream(stream)))


def sort_partitions(d_records, n: int, p: Params, d_pairs, d_bin_offsets, d_out, ws, stream=None):
    _check(lib().elsar_sort_partitions(_ptr(d_records), n, ctypes.byref(p.c()), _ptr(d_pairs), _ptr(d_bin_offsets),
                                       _ptr(d_out), _ptr(ws), _nbytes(ws), _stream(stream)))


def sort(d_in, d_out, n: int, p: Params | None = None, ws=None, stream=None, stats: bool = False):
    """Sort n records of d_in into d_out (both CUDA uint8 tensors); returns a stats dict if asked.

    Without stats the call is asynchronous on `stream` (wait(ws) reports a device-side timeout); with a
    workspace of its own (ws None) it waits, so that the workspace outlives the work."""
    p = p or Params()
    own_ws = ws is None
    if own_ws:
        ws = alloc_workspace(n, p, device=d_in.device)
    st = _Stats() if stats else None
    _check(lib().elsar_sort(_ptr(d_in), _ptr(d_out), n, ctypes.byref(p.c()), _ptr(ws), _nbytes(ws), _stream(stream),
                            ctypes.byref(st) if st is not None else None))
    if own_ws and st is None and n:
        wait(ws, stream)
    if st is None:
        return None
    return dict(pass_ms=list(st.pass_ms)[:5], launches=st.launches, num_items=st.num_items,
                oversize_items=st.oversize_items, model_nodes=st.model_nodes, max_partition=st.max_partition,
                max_bin=st.max_bin, model_used=st.model_used, fallback_reason=st.fallback_reason,
                judge_buckets=st.judge_buckets, judge_rmi_max=st.judge_rmi_max, judge_mlp_max=st.judge_mlp_max,
                F_first_knot=st.F_first_knot, F_last_knot=st.F_last_knot)


def wait(ws, stream=None):
    """Wait for `stream`; raise ElsarError(ELSAR_ETIMEOUT) if a device-side wait gave up in an asynchronous
    sort on workspace ws since the last check."""
    _check(lib().elsar_wait(_ptr(ws), _nbytes(ws), _stream(stream)))


def sort_noalloc(d_in, d_out, n: int, p: Params | None = None, stream=None):
    """Sort without any workspace: the library's built-in scratch array (small n only)."""
    _check(lib().elsar_sort_noalloc(_ptr(d_in), _ptr(d_out), n, ctypes.byref((p or Params()).c()), _stream(stream)))


def sort_host(h_in, h_out, n: int, p: Params, d_in, d_out, ws, stream=None):
    """Host records in (pinned for async DMA), host records out; synchronises."""
    _check(lib().elsar_sort_host(_ptr(h_in), _ptr(h_out), n, ctypes.byref(p.c()), _ptr(d_in), _ptr(d_out), _ptr(ws),
                                 _nbytes(ws), _stream(stream)))


def sort_host_async(h_in, h_out, n: int, p: Params, d_in, d_out, ws, stream=None):
    """sort_host without waiting: copy in, sort and copy out enqueued on `stream`; wait(ws) waits and reports."""
    _check(lib().elsar_sort_host_async(_ptr(h_in), _ptr(h_out), n, ctypes.byref(p.c()), _ptr(d_in), _ptr(d_out),
                                       _ptr(ws), _nbytes(ws), _stream(stream)))


def ooc_min_workspace(n: int, p: Params | None = None) -> int:
    return int(lib().elsar_ooc_min_workspace(n, ctypes.byref((p or Params()).c())))


def sort_ooc(h_in, h_out, n: int, p: Params | None = None, ws=None, budget: int | None = None, stream=None):
    """Sort n records held in pinned host memory (h_in) into pinned h_out using at
    most `budget` bytes of device memory (or the given workspace); synchronises and
    returns the phase statistics."""
    import torch

    p = p or Params()
    if ws is None:
        ws = torch.empty(max(budget or 0, ooc_min_workspace(n, p)), dtype=torch.uint8, device="cuda")
    st = _OocStats()
    _check(lib().elsar_sort_ooc(_ptr(h_in), _ptr(h_out), n, ctypes.byref(p.c()), _ptr(ws), _nbytes(ws),
                                _stream(stream), ctypes.byref(st)))
    return dict(phase_ms=list(st.phase_ms), h2d_bytes=st.h2d_bytes, d2h_bytes=st.d2h_bytes, chunks=st.chunks,
                groups=st.groups, chunk_records=st.chunk_records, group_records=st.group_records,
                model_used=st.model_used, fallback_reason=st.fallback_reason, max_partition=st.max_partition)


def selftest_bounded_wait(d_src, d_word, limit_cycles: int, stream=None):
    """Run the bounded-wait self-test; returns (status, [flags, byte_sum, cycles_waited]).
    ELSAR_ETIMEOUT (4) is the expected status: the wait gave up as designed."""
    res = (ctypes.c_uint32 * 3)()
    rc = lib().elsar_selftest_bounded_wait(_ptr(d_src), _ptr(d_word), limit_cycles, _stream(stream),
                                           ctypes.byref(res))
    return rc, list(res)


def mlp_eval(d_w, d_knots, d_x, n: int, d_F, stream=None):
    _check(lib().elsar_mlp_eval(_ptr(d_w), _ptr(d_knots), _ptr(d_x), n, _ptr(d_F), _stream(stream)))


def mlp_grad(d_w, d_knots, d_x, d_y, n: int, d_grad, stream=None):
    import torch

    ws = torch.empty(lib().elsar_mlp_grad_workspace(n), dtype=torch.uint8, device=d_w.device)
    _check(lib().elsar_mlp_grad(_ptr(d_w), _ptr(d_knots), _ptr(d_x), _ptr(d_y), n, _ptr(d_grad), _ptr(ws),
                                _nbytes(ws), _stream(stream)))


def mlp_adam(d_w, d_grad, d_m, d_v, t: int, lr: float = 1e-3, stream=None):
    """One Adam step of the trainer (in place on d_w, d_m, d_v)."""
    _check(lib().elsar_mlp_adam(_ptr(d_w), _ptr(d_grad), _ptr(d_m), _ptr(d_v), t, lr, _stream(stream)))


def mlp_splitters(d_w, d_knots, log2B: int, d_t, stream=None):
    _check(lib().elsar_mlp_splitters(_ptr(d_w), _ptr(d_knots), log2B, _ptr(d_t), _stream(stream)))


class Batch:
    """A plan sorting many record sets with one CUDA-graph launch (elsar_batch_*)."""

    def __init__(self, d_ins, d_outs, p: Params | None = None, ws=None, stream=None):
        import numpy as np
        import torch

        self.p = p or Params()
        self.n = np.array([t.numel() // RECORD for t in d_ins], dtype=np.uint64)
        K = len(d_ins)
        self._ins = (ctypes.c_void_p * K)(*[t.data_ptr() for t in d_ins])
        self._outs = (ctypes.c_void_p * K)(*[t.data_ptr() for t in d_outs])
        self._keep = (d_ins, d_outs)
        need = lib().elsar_batch_workspace_size(self.n.ctypes.data, K, ctypes.byref(self.p.c()))
        self.ws = ws if ws is not None else torch.empty(max(256, need), dtype=torch.uint8, device=d_ins[0].device)
        h = ctypes.c_void_p()
        _check(lib().elsar_batch_create(self._ins, self._outs, self.n.ctypes.data, K, ctypes.byref(self.p.c()),
                                        _ptr(self.ws), _nbytes(self.ws), _stream(stream), ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        _check(lib().elsar_batch_run(self.handle, _stream(stream)))

    def wait(self, stream=None):
        _check(lib().elsar_batch_wait(self.handle, _stream(stream)))

    def info(self) -> dict:
        i = _BatchInfo()
        _check(lib().elsar_batch_describe(self.handle, ctypes.byref(i)))
        return dict(tile_pairs=i.tile_pairs, records_per_bin_log2=list(i.records_per_bin_log2),
                    total_records=i.total_records, total_bins=i.total_bins, sample_keys=i.sample_keys,
                    launches=i.launches, tuning_runs=i.tuning_runs,
                    tuning_ms=list(i.tuning_ms)[: min(16, i.tuning_runs)])

    def close(self):
        if self.handle:
            lib().elsar_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- device model buffer layout (read back for inspection and parity tests)
MLP_PARAMS = 1517  # the network's parameters (include/elsar.h gives the layout)
MODEL_HEADER_BYTES = 256
NODE_BYTES = 64


def read_model(d_model, p: Params, n: int):
    """Host copy of a fitted model: (header dict, nodes structured array, splitters uint64)."""
    import numpy as np

    buf = d_model.cpu().numpy()
    hdr = np.frombuffer(buf[:96].tobytes(), dtype=np.dtype([
        ("magic", "<u4"), ("kind", "<u4"), ("log2B", "<u4"), ("num_nodes", "<u4"), ("S", "<u8"), ("node_cap", "<u8"),
        ("nodes_off", "<u8"), ("splitters_off", "<u8"), ("bytes", "<u8"), ("T", "<u4"), ("Dmax", "<u4"),
        ("levels", "<u4"), ("fallback", "<u4"), ("lut_off", "<u8"), ("knots_off", "<u8"), ("weights_off", "<u8")]))[0]
    ndt = np.dtype([("s", "<u4"), ("e", "<u4"), ("base", "<u8"), ("child0", "<u4"), ("fanout", "<u4"),
                    ("shift", "<u4"), ("depth_set", "<u4"), ("a", "<f8"), ("b", "<f8"), ("c", "<f8"), ("h", "<f8")])
    nn = int(hdr["num_nodes"])
    off = int(hdr["nodes_off"])
    nodes = np.frombuffer(buf[off:off + nn * NODE_BYTES].tobytes(), dtype=ndt)
    so = int(hdr["splitters_off"])
    B = 1 << int(hdr["log2B"])
    spl = np.frombuffer(buf[so:so + 8 * B].tobytes(), dtype=np.uint64)
    h = {k: hdr[k].item() for k in hdr.dtype.names}
    ko, wo = int(hdr["knots_off"]), int(hdr["weights_off"])
    h["mlp_knots"] = np.frombuffer(buf[ko:ko + 104].tobytes(), dtype=np.uint64).copy()
    h["mlp_w"] = np.frombuffer(buf[wo:wo + MLP_PARAMS * 4].tobytes(), dtype=np.float32).copy()
    return h, nodes, spl
