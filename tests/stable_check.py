"""Property check of a sorted record set that holds at any size: sorted by
key, equal keys in input order (the record index rides in the payload), and
a permutation of the input byte for byte -- together they single out the
stable sort.  Used by the full-size GPU tests; pinned on the CPU against the
oracle's stable sort and planted faults."""
import torch

HEX = torch.tensor([0] * 48 + list(range(10)) + [0] * 7 + list(range(10, 16)) + [0] * 185, dtype=torch.int64)


def _record_index(rec: torch.Tensor) -> torch.Tensor:
    """Low 32 bits of the record index from its 32 hex digits (bytes 10..41)."""
    digits = HEX.to(rec.device)[rec[:, 34:42].long()]
    idx = torch.zeros(rec.shape[0], dtype=torch.int64, device=rec.device)
    for k in range(8):
        idx = idx * 16 + digits[:, k]
    return idx


def _key_words(rec: torch.Tensor, idx: torch.Tensor):
    """(bytes 0-6, bytes 7-9 << 32 | index): lexicographic order = key order, then input order."""
    b = rec[:, :10].long()
    a = torch.zeros(rec.shape[0], dtype=torch.int64, device=rec.device)
    for k in range(7):
        a = a * 256 + b[:, k]
    c = ((b[:, 7] * 256 + b[:, 8]) * 256 + b[:, 9]) * (1 << 32) + idx
    return a, c


def check_stable_sort(d_in: torch.Tensor, d_out: torch.Tensor, n: int, chunk: int = 25_000_000):
    inp = d_in.view(n, 100)
    out = d_out.view(n, 100)
    seen = torch.zeros(n, dtype=torch.bool, device=d_in.device)
    prev = None
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        rec = out[s:e]
        idx = _record_index(rec)
        assert int(idx.min()) >= 0 and int(idx.max()) < n
        seen[idx] = True
        assert torch.equal(inp[idx], rec), "output record differs from the input record it names"
        a, c = _key_words(rec, idx)
        if prev is not None:
            a = torch.cat([prev[0], a])
            c = torch.cat([prev[1], c])
        ok = (a[:-1] < a[1:]) | ((a[:-1] == a[1:]) & (c[:-1] < c[1:]))
        assert bool(ok.all()), "output not in (key, input position) order"
        prev = (a[-1:], c[-1:])
        del rec, idx, a, c, ok
    assert bool(seen.all()), "output is not a permutation of the input"
