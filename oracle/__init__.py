"""ctypes access to the ELSAR CPU oracle (oracle/elsar_oracle.cpp, oracle/mlp_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
bench's CPU-baseline leg, never by the product package.  Shares no code with
the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "libelsar_oracle.so")
_SRCS = ["elsar_oracle.cpp", "mlp_oracle.cpp"]
RECORD = 100

_lib = None

P = ctypes.c_void_p
U64 = ctypes.c_uint64
U32 = ctypes.c_uint32
I32 = ctypes.c_int


def build():
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                           "-o", _LIB] + srcs)


def lib():
    global _lib
    if _lib is None:
        srcs = [os.path.join(_HERE, s) for s in _SRCS]
        if not os.path.exists(_LIB) or any(os.path.getmtime(s) > os.path.getmtime(_LIB) for s in srcs):
            build()
        L = ctypes.CDLL(_LIB)
        sig = {
            "eo_encode9": (U64, [P]),
            "eo_set_key_bytes": (I32, [I32]),
            "eo_encode9_records": (None, [P, U64, P]),
            "eo_splitmix64_at": (U64, [U64, U64]),
            "eo_default_sample_size": (U64, [U64]),
            "eo_sample": (None, [P, U64, U64, U64, P]),
            "eo_rmi_fit": (U64, [P, U64, U32, U32, P]),
            "eo_rmi_export": (None, [I32, P, P, P]),
            "eo_rmi_eval": (None, [I32, P, U64, P, P]),
            "eo_rmi_release": (None, []),
            "eo_sort": (I32, [P, U64, U32, U32, U32, U32, U64, U64, I32, P, P, P, P, P, P]),
            "eo_classify": (I32, [P, U64, U32, U32, U32, U32, U64, U64, I32, P, P]),
            "eo_stable_sort": (None, [P, U64, P]),
            "eo_mlp_params": (I32, []),
            "eo_mlp_knots": (None, [P, U64, P]),
            "eo_mlp_init": (None, [P]),
            "eo_mlp_features": (None, [P, P, U64, P]),
            "eo_mlp_forward32": (None, [P, P, U64, P]),
            "eo_mlp_forward64": (None, [P, P, U64, P]),
            "eo_mlp_grad64": (None, [P, P, P, U64, P]),
            "eo_mlp_train64": (None, [P, P, P, U64, U32, U32, ctypes.c_double, ctypes.c_double, P]),
            "eo_mlp_lr_at": (ctypes.c_double, [U64, U64, ctypes.c_double, ctypes.c_double]),
            "eo_mlp_adam64": (None, [P, P, P, P, U64, ctypes.c_double]),
            "eo_radix_bins": (None, [P, U64, U32, P]),
            "eo_radix_splitters": (None, [U32, P]),
            "eo_sort_by_splitters": (I32, [P, U64, P, U32, U32, I32, P, P, P, P, P, P]),
            "eo_model_choice": (I32, [P, U64, U32, U32, U32, U32, U64, U64, I32, P, U32, P]),
            "eo_sort_threads": (I32, [P, U64, U32, U32, U32, U32, U64, U64, I32, P, U32]),
            "eo_mlp_splitters": (None, [P, P, U32, P]),
            "eo_bins_by_splitters": (None, [P, U32, P, U64, P]),
            "eo_validate": (I32, [P, P, U64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class key_bytes:
    """Context: the oracle's key is the first l bytes of each record (Sec. 4's
    variable-length keys, 0-padded); 10 (the whole key field) outside it."""

    def __init__(self, l: int):
        self.l = l

    def __enter__(self):
        if lib().eo_set_key_bytes(self.l) != self.l:
            raise ValueError("key length must be in [1, 10]")
        return self

    def __exit__(self, *a):
        lib().eo_set_key_bytes(10)


def encode9(key: bytes) -> int:
    buf = np.frombuffer(bytes(key[:10]).ljust(10, b" "), dtype=np.uint8).copy()
    return int(lib().eo_encode9(buf.ctypes.data))


def encode9_records(recs: np.ndarray) -> np.ndarray:
    n = recs.size // RECORD
    out = np.empty(n, dtype=np.uint64)
    lib().eo_encode9_records(_ptr(recs), n, _ptr(out))
    return out


def splitmix64_at(seed: int, k: int) -> int:
    return int(lib().eo_splitmix64_at(seed, k))


def default_sample_size(n: int) -> int:
    return int(lib().eo_default_sample_size(n))


LEAF_TARGET = 16  # T: sample keys per RMI node below which it stops splitting (a node splits above 2T)
MAX_DEPTH = 32  # Dmax


def default_fine_log2(n: int, P: int) -> int:
    """log2 of the fine-bin count: about 1024 records per bin, within [max(log2 P, 6), 20]."""
    lp = P.bit_length() - 1
    want = max(0, (max(n, 1) - 1).bit_length() - 10)
    return max(lp, min(20, max(6, want)))


def sample(recs: np.ndarray, S: int, seed: int) -> np.ndarray:
    n = recs.size // RECORD
    out = np.empty(S, dtype=np.uint64)
    lib().eo_sample(_ptr(recs), n, S, seed, _ptr(out))
    return out


class Rmi:
    """The oracle's fitted RMI, exported as breadth-first node arrays."""

    def __init__(self, sorted_sample: np.ndarray, T: int = LEAF_TARGET, Dmax: int = MAX_DEPTH):
        s = np.ascontiguousarray(sorted_sample, dtype=np.uint64)
        self.sample, self.S = s, s.size
        h = ctypes.c_int(-1)
        nn = int(lib().eo_rmi_fit(_ptr(s), s.size, T, Dmax, ctypes.byref(h)))
        if nn == 0:
            raise ValueError("eo_rmi_fit rejected the sample")
        self.handle = h.value
        self.nu64 = np.zeros((nn, 4), dtype=np.uint64)
        self.nu32 = np.zeros((nn, 3), dtype=np.uint32)
        self.nf64 = np.zeros((nn, 7))
        lib().eo_rmi_export(self.handle, _ptr(self.nu64), _ptr(self.nu32), _ptr(self.nf64))

    def __len__(self):
        return self.nu64.shape[0]

    s_ = property(lambda self: self.nu64[:, 0])
    e_ = property(lambda self: self.nu64[:, 1])
    base = property(lambda self: self.nu64[:, 2])
    child0 = property(lambda self: self.nu64[:, 3])
    shift = property(lambda self: self.nu32[:, 0])
    fanout = property(lambda self: self.nu32[:, 1])
    depth = property(lambda self: self.nu32[:, 2])
    gamma = property(lambda self: self.nf64[:, 0])
    delta = property(lambda self: self.nf64[:, 1])
    scale = property(lambda self: self.nf64[:, 2])
    g = property(lambda self: self.nf64[:, 3])
    d = property(lambda self: self.nf64[:, 4])
    lo = property(lambda self: self.nf64[:, 5])
    hi = property(lambda self: self.nf64[:, 6])

    def eval(self, xs: np.ndarray):
        """(F, leaf node index) at each key encoding."""
        xs = np.ascontiguousarray(xs, dtype=np.uint64)
        F = np.empty(xs.size)
        leaf = np.empty(xs.size, dtype=np.uint64)
        lib().eo_rmi_eval(self.handle, _ptr(xs), xs.size, _ptr(F), _ptr(leaf))
        return F, leaf


def sort(recs: np.ndarray, P: int, log2B: int, S: int, seed: int, balance: int = 1, want_detail=False,
         T: int = LEAF_TARGET, Dmax: int = MAX_DEPTH):
    """Run the whole oracle; returns out (and a dict of intermediate results)."""
    n = recs.size // RECORD
    out = np.empty_like(recs)
    B = 1 << log2B
    q = np.empty(n, dtype=np.uint32) if want_detail else None
    pid = np.empty(n, dtype=np.uint32) if want_detail else None
    off = np.empty(P + 1, dtype=np.uint64)
    counts = np.empty(B, dtype=np.uint64) if want_detail else None
    cuts = np.empty(P + 1, dtype=np.uint32) if want_detail else None
    rc = lib().eo_sort(_ptr(recs), n, P, log2B, T, Dmax, S, seed, balance, _ptr(out), _ptr(q), _ptr(pid), _ptr(off),
                       _ptr(counts), _ptr(cuts))
    if rc:
        raise ValueError(f"eo_sort rc={rc}")
    if want_detail:
        return out, dict(q=q, pid=pid, part_off=off, bin_counts=counts, cuts=cuts)
    return out


def classify(recs: np.ndarray, P: int, log2B: int, S: int, seed: int, balance: int = 1, T: int = LEAF_TARGET,
             Dmax: int = MAX_DEPTH):
    """Fine-bin counts and partition offsets of every record (no sort)."""
    n = recs.size // RECORD
    counts = np.empty(1 << log2B, dtype=np.uint64)
    off = np.empty(P + 1, dtype=np.uint64)
    rc = lib().eo_classify(_ptr(recs), n, P, log2B, T, Dmax, S, seed, balance, _ptr(counts), _ptr(off))
    if rc:
        raise ValueError(f"eo_classify rc={rc}")
    return counts, off


def stable_sort(recs: np.ndarray) -> np.ndarray:
    out = np.empty_like(recs)
    lib().eo_stable_sort(_ptr(recs), recs.size // RECORD, _ptr(out))
    return out


def validate(inp: np.ndarray, out: np.ndarray) -> int:
    return int(lib().eo_validate(_ptr(inp), _ptr(out), inp.size // RECORD))


# ---------------------------------------------------------------- monotone MLP CDF (mlp_oracle.cpp)
MLP_FEATURES, MLP_HIDDEN = 12, 32
MLP_PARAMS = 12 * 32 + 32 + 32 * 32 + 32 + 32 + 1 + 12  # 1517
MLP_SLICES = {"W1": (0, 384), "b1": (384, 416), "W2": (416, 1440), "b2": (1440, 1472), "w3": (1472, 1504),
              "b3": (1504, 1505), "v": (1505, 1517)}
MLP_WEIGHTS = ("W1", "W2", "w3", "v")  # projected onto >= 0
MLP_BIASES = ("b1", "b2", "b3")


def mlp_knots(sorted_sample: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(sorted_sample, dtype=np.uint64)
    T = np.empty(13, dtype=np.uint64)
    lib().eo_mlp_knots(_ptr(s), s.size, _ptr(T))
    return T


def mlp_init() -> np.ndarray:
    w = np.empty(MLP_PARAMS, dtype=np.float32)
    lib().eo_mlp_init(_ptr(w))
    return w


def mlp_features(T: np.ndarray, xs: np.ndarray) -> np.ndarray:
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    phi = np.empty((xs.size, 12), dtype=np.float32)
    lib().eo_mlp_features(_ptr(np.ascontiguousarray(T, dtype=np.uint64)), _ptr(xs), xs.size, _ptr(phi))
    return phi


def mlp_forward32(w: np.ndarray, phi: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float32)
    phi = np.ascontiguousarray(phi, dtype=np.float32)
    F = np.empty(phi.shape[0], dtype=np.float32)
    lib().eo_mlp_forward32(_ptr(w), _ptr(phi), phi.shape[0], _ptr(F))
    return F


def mlp_forward64(w: np.ndarray, phi: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    F = np.empty(phi.shape[0])
    lib().eo_mlp_forward64(_ptr(w), _ptr(phi), phi.shape[0], _ptr(F))
    return F


def mlp_grad64(w: np.ndarray, phi: np.ndarray, y: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    g = np.empty(MLP_PARAMS)
    lib().eo_mlp_grad64(_ptr(w), _ptr(phi), _ptr(y), y.size, _ptr(g))
    return g


def mlp_train64(w0: np.ndarray, phi: np.ndarray, y: np.ndarray, batch: int = 8192, steps: int = 400,
                lr: float = 1e-3, lr_min: float = 1e-5):
    w = np.array(w0, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    loss = ctypes.c_double(0)
    lib().eo_mlp_train64(_ptr(w), _ptr(phi), _ptr(y), y.size, batch, steps, lr, lr_min, ctypes.byref(loss))
    return w, loss.value


def mlp_lr_at(t: int, steps: int, lr: float = 1e-3, lr_min: float = 1e-5) -> float:
    return float(lib().eo_mlp_lr_at(t, steps, lr, lr_min))


def mlp_splitters(w: np.ndarray, T: np.ndarray, log2B: int) -> np.ndarray:
    t = np.empty(1 << log2B, dtype=np.uint64)
    lib().eo_mlp_splitters(_ptr(np.ascontiguousarray(w, dtype=np.float32)),
                           _ptr(np.ascontiguousarray(T, dtype=np.uint64)), log2B, _ptr(t))
    return t


def bins_by_splitters(t: np.ndarray, log2B: int, xs: np.ndarray) -> np.ndarray:
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    q = np.empty(xs.size, dtype=np.uint32)
    lib().eo_bins_by_splitters(_ptr(np.ascontiguousarray(t, dtype=np.uint64)), log2B, _ptr(xs), xs.size, _ptr(q))
    return q


def mlp_adam64(w, g, m, v, t: int, lr: float = 1e-3):
    """One Adam step (FP64) at step number t from state (m, v); returns new (w, m, v)."""
    w = np.array(w, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    lib().eo_mlp_adam64(_ptr(w), _ptr(g), _ptr(m), _ptr(v), t, lr)
    return w, m, v


# ---------------------------------------------------------------- radix partitioning, classifiers by splitters
def radix_bins(xs: np.ndarray, log2B: int) -> np.ndarray:
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    q = np.empty(xs.size, dtype=np.uint32)
    lib().eo_radix_bins(_ptr(xs), xs.size, log2B, _ptr(q))
    return q


def radix_splitters(log2B: int) -> np.ndarray:
    t = np.empty(1 << log2B, dtype=np.uint64)
    lib().eo_radix_splitters(log2B, _ptr(t))
    return t


def sort_by_splitters(recs: np.ndarray, t: np.ndarray, log2B: int, P: int, balance: int = 1, want_out: bool = True):
    """The method with a given classifier (splitters t): (out or None, detail dict)."""
    n = recs.size // RECORD
    B = 1 << log2B
    t = np.ascontiguousarray(t, dtype=np.uint64)
    out = np.empty_like(recs) if want_out else None
    q = np.empty(n, dtype=np.uint32)
    pid = np.empty(n, dtype=np.uint32)
    off = np.empty(P + 1, dtype=np.uint64)
    counts = np.empty(B, dtype=np.uint64)
    cuts = np.empty(P + 1, dtype=np.uint32)
    rc = lib().eo_sort_by_splitters(_ptr(recs), n, _ptr(t), log2B, P, balance, _ptr(out), _ptr(q), _ptr(pid),
                                    _ptr(off), _ptr(counts), _ptr(cuts))
    if rc:
        raise ValueError(f"eo_sort_by_splitters rc={rc}")
    return out, dict(q=q, pid=pid, part_off=off, bin_counts=counts, cuts=cuts)


MODEL_CHOICE_DIAG = ("rmi_max_bucket", "mlp_max_bucket", "J", "F_first_knot", "F_last_knot", "mlp_max_partition")


def model_choice(recs: np.ndarray, P: int, log2B: int, S: int, seed: int, balance: int, w: np.ndarray,
                 skip: int = 0, T: int = LEAF_TARGET, Dmax: int = MAX_DEPTH):
    """The network-or-RMI decision for given network weights: (reason, diagnostics dict)."""
    n = recs.size // RECORD
    w = np.ascontiguousarray(w, dtype=np.float32)
    diag = np.zeros(6)
    r = int(lib().eo_model_choice(_ptr(recs), n, P, log2B, T, Dmax, S, seed, balance, _ptr(w), skip, _ptr(diag)))
    if r < 0:
        raise ValueError("eo_model_choice rejected its arguments")
    return r, dict(zip(MODEL_CHOICE_DIAG, diag.tolist()))


def sort_threads(recs: np.ndarray, P: int, log2B: int, S: int, seed: int, balance: int = 1, threads: int = 1,
                 T: int = LEAF_TARGET, Dmax: int = MAX_DEPTH) -> np.ndarray:
    """eo_sort over `threads` host threads (classification ranges, partitions sorted in parallel)."""
    n = recs.size // RECORD
    out = np.empty_like(recs)
    rc = lib().eo_sort_threads(_ptr(recs), n, P, log2B, T, Dmax, S, seed, balance, _ptr(out), threads)
    if rc:
        raise ValueError(f"eo_sort_threads rc={rc}")
    return out
