"""Seeded synthetic 100-byte records shaped like the paper's benchmark data.

The paper (Sec. 7.1) sorts gensort files: 100-byte records, a 10-byte printable
ASCII key and a 90-byte payload, uniform or skewed.  gensort itself is not
available, so these generators stand in for it.  Both the oracle and the CUDA
path take their inputs from here; this module holds none of the sort's
arithmetic (no encoding, model, partitioning or ordering).

Definitions (identical in the C and CUDA implementations):

* ``h(i, pos, stream) = splitmix64(seed*0x9E3779B97F4A7C15 ^ (i*16+pos) ^ (stream<<60))``
* uniform key byte: ``0x20 + mulhi32(h(i,pos,0) >> 32, 95)``
* Zipf(s) key byte: rank ``r = #{k : cum[k] <= h(i,pos,2)}`` over a 94-entry
  fixed-point CDF table of ``r^-s`` (built here in FP64, shared as integers),
  then ``0x20 + perm[pos][r]`` with a per-position Fisher-Yates permutation
  drawn from stream 3
* prefix-skew key (the paper's skewed data, Sec. 7.1: a table of 128 6-byte
  entries, the key's leading bytes of record i replaced by entry
  ``log2(i) mod 128``): uniform bytes, then bytes 0-5 replaced by entry
  ``t = floor(log2 i) mod 128`` (record 0: entry 0) of a seed-drawn table whose
  byte p of entry t is ``0x20 + mulhi32(h(t,p,4) >> 32, 95)``
* variable-length key (Sec. 4: keys of different lengths, the longest l = 10,
  padded with 0): ``L = 1 + mulhi32(h(i,12,5) >> 32, 10)`` uniform bytes, then
  0x00 up to byte 10
* duplicates: with probability d (``h(i,10,1) < floor(d*2^64)``) the key is the
  base key of record ``mulhi64(h(i,11,1), n)``
* payload: 32 hex digits of i, 56 filler letters, CRLF
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

RECORD = 100
KEY = 10
_HERE = os.path.dirname(os.path.abspath(__file__))
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """splitmix64 finaliser on a counter (Steele, Lea, Flood 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def h(seed: int, i: int, pos: int, stream: int) -> int:
    return splitmix64(((seed * 0x9E3779B97F4A7C15) & _M64) ^ ((i * 16 + pos) & _M64) ^ ((stream << 60) & _M64))


@dataclass(frozen=True)
class KeySpec:
    """How the 10-byte keys of one record set are drawn."""

    kind: str = "uniform"  # "uniform" | "zipf" | "prefix" (the paper's table-of-prefixes skew) | "varlen"
    s: float = 1.1  # Zipf exponent (kind == "zipf")
    dup: float = 0.0  # fraction of exact-duplicate keys
    seed: int = 1

    def tables(self):
        """(cum[94] uint64, perm[10*95] uint8, dup_thr) shared by both generators."""
        if self.kind in ("uniform", "prefix", "varlen"):
            cum = np.full(94, _M64, dtype=np.uint64)
            perm = np.tile(np.arange(95, dtype=np.uint8), 10)
        elif self.kind == "zipf":
            w = [r ** (-self.s) for r in range(1, 96)]
            tot = math.fsum(w)
            acc = 0.0
            vals = []
            for k in range(94):
                acc += w[k]
                vals.append(min(_M64, int(math.floor(acc / tot * 2.0**64))))
            cum = np.array(vals, dtype=np.uint64)
            perm = np.zeros((10, 95), dtype=np.uint8)
            for pos in range(10):
                p = list(range(95))
                for k in range(94, 0, -1):
                    j = ((h(self.seed, k, pos, 3) >> 32) * (k + 1)) >> 32
                    p[k], p[j] = p[j], p[k]
                perm[pos] = p
            perm = perm.reshape(-1)
        else:
            raise ValueError(f"unknown key kind {self.kind!r}")
        thr = int(math.floor(self.dup * 2.0**64)) if self.dup > 0 else 0
        return cum, perm, min(thr, _M64)

    @property
    def kind_code(self) -> int:
        return {"uniform": 0, "zipf": 1, "prefix": 2, "varlen": 3}[self.kind]


_cpu = None
_gpu = None


def _load_cpu():
    global _cpu
    if _cpu is None:
        path = os.path.join(_HERE, "librecgen.so")
        if not os.path.exists(path):
            build_cpu()
        lib = ctypes.CDLL(path)
        lib.recgen_cpu.restype = ctypes.c_int
        lib.recgen_cpu.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_uint64, ctypes.c_int]
        lib.recgen_splitmix64.restype = ctypes.c_uint64
        lib.recgen_splitmix64.argtypes = [ctypes.c_uint64]
        _cpu = lib
    return _cpu


def _load_gpu():
    global _gpu
    if _gpu is None:
        path = os.path.join(_HERE, "librecgen_cuda.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} missing: run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        lib.recgen_gpu.restype = ctypes.c_int
        lib.recgen_gpu.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_uint64, ctypes.c_void_p]
        _gpu = lib
    return _gpu


def generate_cpu(n: int, spec: KeySpec, i0: int = 0, count: int | None = None, threads: int | None = None):
    """Records [i0, i0+count) of an n-record set as a flat uint8 array."""
    if count is None:
        count = n - i0
    out = np.empty(count * RECORD, dtype=np.uint8)
    cum, perm, thr = spec.tables()
    if threads is None:
        threads = os.cpu_count() or 1
    rc = _load_cpu().recgen_cpu(out.ctypes.data, n, i0, count, spec.seed, spec.kind_code, cum.ctypes.data,
                                perm.ctypes.data, thr, threads)
    if rc != 0:
        raise RuntimeError("recgen_cpu failed")
    return out


def generate_gpu(out_tensor, n: int, spec: KeySpec, i0: int = 0, count: int | None = None, stream: int = 0):
    """Fill a CUDA uint8 tensor (count*100 bytes) with records [i0, i0+count)."""
    if count is None:
        count = n - i0
    assert out_tensor.is_cuda and out_tensor.numel() >= count * RECORD
    cum, perm, thr = spec.tables()
    rc = _load_gpu().recgen_gpu(out_tensor.data_ptr(), n, i0, count, spec.seed, spec.kind_code,
                                cum.ctypes.data, perm.ctypes.data, thr, stream)
    if rc != 0:
        raise RuntimeError(f"recgen_gpu failed ({rc})")


def build_cpu():
    import subprocess

    src = os.path.join(_HERE, "recgen.c")
    dst = os.path.join(_HERE, "librecgen.so")
    subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", dst, src])


def build_gpu():
    import subprocess

    src = os.path.join(_HERE, "recgen_cuda.cu")
    dst = os.path.join(_HERE, "librecgen_cuda.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-shared",
                           "-Xcompiler", "-fPIC", "-o", dst, src])


# ---------------------------------------------------------------------------
# Workloads (the shapes of the paper's uniform and skewed data sets)

UNIFORM_1M = dict(name="uniform-1M", n=1_000_000, spec=KeySpec("uniform", seed=1), P=64)
UNIFORM_100M = dict(name="uniform-100M", n=100_000_000, spec=KeySpec("uniform", seed=2), P=1024)
ZIPF11_100M = dict(name="zipf1.1-dup5%-100M", n=100_000_000, spec=KeySpec("zipf", s=1.1, dup=0.05, seed=3), P=1024)
PREFIX_100M = dict(name="prefix-skew-100M", n=100_000_000, spec=KeySpec("prefix", seed=8), P=1024)
ZIPF13_500M = dict(name="zipf1.3-dup10%-500M", n=500_000_000, spec=KeySpec("zipf", s=1.3, dup=0.10, seed=5),
                   P=4096)


def batch_sizes(num_sets: int = 4096, lo: float = 1e3, hi: float = 1e6, seed: int = 4, cap_records: int = 400_000_000):
    """Log-uniform set sizes in [lo, hi], scaled down (floor, min lo) if their sum exceeds cap_records."""
    sizes = []
    for k in range(num_sets):
        u = (h(seed, k, 0, 0) >> 11) * (1.0 / 9007199254740992.0)
        sizes.append(int(math.floor(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))))
    tot = sum(sizes)
    if tot > cap_records:
        sizes = [max(int(lo), (s * cap_records) // tot) for s in sizes]
    return sizes


def batch_spec(k: int) -> KeySpec:
    """Set k of the batched workload: even sets uniform, odd sets Zipf(1.1) with 5% duplicates."""
    if k % 2 == 0:
        return KeySpec("uniform", seed=1000 + k)
    return KeySpec("zipf", s=1.1, dup=0.05, seed=1000 + k)
