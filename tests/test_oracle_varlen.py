"""Pins for variable-length keys (Sec. 4): keys of different lengths, padded
with ASCII 0 to the longest, and key fields shorter than the record's first 10
bytes.  The order is the one strncmp gives NUL-terminated strings -- a key
sorts before every longer key it is a prefix of -- with ties in input order,
which Python's sort of the unpadded byte strings reproduces independently."""
import numpy as np
import pytest

TOP = 95**9


def _records(keys):
    n = len(keys)
    recs = np.zeros((n, 100), dtype=np.uint8)
    for i, k in enumerate(keys):
        recs[i, :len(k)] = np.frombuffer(k, dtype=np.uint8)
        recs[i, 10:42] = np.frombuffer(f"{i:032X}".encode(), dtype=np.uint8)
        recs[i, 98:100] = [13, 10]
    return recs.reshape(-1)


def test_padded_encoding_closed_form(orc):
    # ASCII 0 past the end: every later digit encodes as 0 (the padding reading)
    assert orc.encode9(b"ab" + b"\0" * 8) == 65 * 95**8 + 66 * 95**7
    assert orc.encode9(b"\0" * 10) == 0
    # a space also encodes as digit 0: the byte order decides "ab" < "ab "
    assert orc.encode9(b"ab \0\0\0\0\0\0\0") == orc.encode9(b"ab" + b"\0" * 8)
    # a shorter key never encodes above a longer key it is a prefix of
    for k in (b"A", b"Zz", b"~~~~", b"hello w"):
        longer = k + b" "
        assert orc.encode9(k.ljust(10, b"\0")) <= orc.encode9(longer.ljust(10, b"\0"))


def test_variable_length_keys_sort_like_strncmp(orc, gen):
    n = 20_000
    recs = gen.generate_cpu(n, gen.KeySpec("varlen", seed=9))
    keys = [bytes(recs[i * 100:i * 100 + 10]).rstrip(b"\0") for i in range(n)]
    assert {len(k) for k in keys} == set(range(1, 11))
    order = sorted(range(n), key=lambda i: keys[i])  # Python's sort is stable
    want = recs.reshape(n, 100)[order].reshape(-1)
    assert np.array_equal(orc.stable_sort(recs), want)
    out = orc.sort(recs, 16, orc.default_fine_log2(n, 16), S=1000, seed=3)
    assert np.array_equal(out, want)
    assert orc.validate(recs, out) == 0


def test_brute_force_prefix_families(orc):
    """Every key over a 3-letter alphabet up to length 3 (with repeats), shuffled."""
    import itertools
    import random

    alpha = [b" ", b"A", b"~"]
    keys = [b""] if False else []
    for L in range(1, 4):
        keys += [b"".join(t) for t in itertools.product(alpha, repeat=L)]
    keys = keys * 3
    random.Random(4).shuffle(keys)
    recs = _records(keys)
    order = sorted(range(len(keys)), key=lambda i: keys[i])
    want = recs.reshape(-1, 100)[order].reshape(-1)
    for P in (1, 4, 16):
        assert np.array_equal(orc.sort(recs, P, orc.default_fine_log2(len(keys), P), S=1000, seed=1), want)


@pytest.mark.parametrize("l", [1, 4, 8, 9])
def test_key_field_shorter_than_ten_bytes(orc, gen, l):
    """key_bytes = l: only the first l bytes are the key; the rest of the key
    field is payload, never compared: ties on the l-byte key keep input order."""
    n = 30_000
    recs = gen.generate_cpu(n, gen.KeySpec("zipf", s=1.2, dup=0.05, seed=10))
    keys = [bytes(recs[i * 100:i * 100 + l]) for i in range(n)]
    order = sorted(range(n), key=lambda i: keys[i])
    want = recs.reshape(n, 100)[order].reshape(-1)
    with orc.key_bytes(l):
        assert np.array_equal(orc.stable_sort(recs), want)
        out = orc.sort(recs, 8, orc.default_fine_log2(n, 8), S=1000, seed=2)
        assert np.array_equal(out, want)
        assert orc.validate(recs, out) == 0
    # the setting ends with the context
    assert np.array_equal(orc.stable_sort(recs[:1000]), orc.sort(recs[:1000], 1, 6, S=1000, seed=2))


def test_key_bytes_out_of_range(orc):
    with pytest.raises(ValueError):
        with orc.key_bytes(11):
            pass
