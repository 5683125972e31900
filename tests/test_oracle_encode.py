"""Pins for the oracle's base-95 key encoding (Sec. 4 of the paper)."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_closed_form_extremes(orc):
    assert orc.encode9(b" " * 10) == 0
    assert orc.encode9(b"~" * 10) == 95**9 - 1  # sum_{i=1..9} 94*95^(9-i)
    # a single non-space character: (ASCII - 32) * 95^(9 - i) at 1-based position i
    assert orc.encode9(b"!" + b" " * 9) == 95**8
    assert orc.encode9(b" " * 8 + b"!" + b" ") == 1
    assert orc.encode9(b"A" + b" " * 9) == 33 * 95**8
    assert orc.encode9(b" " * 9 + b"~") == 0  # the tenth byte is not encoded


def test_hand_example(orc):
    key = b"Az~ 0!    "
    digits = [ord(c) - 32 for c in "Az~ 0!   "]
    want = 0
    for i, dgt in enumerate(digits, start=1):
        want += dgt * 95 ** (9 - i)
    assert orc.encode9(key) == want


def test_paper_constants_match_closed_forms():
    g = _golden("paper_encoding_constants.txt")
    s9 = sum(95**i for i in range(1, 10))
    s10 = sum(95**i for i in range(1, 11))
    assert round(math.log2(s9), 2) == g["log2_l9"]
    assert round(math.log2(s10), 2) == g["log2_l10"]
    assert f"{s9:.2e}" == f"{g['partitions']:.2e}"
    assert round(s9 * 10 / 1e15, 1) == g["petabytes"]
    # so 9 characters fit a 64-bit integer and 10 do not
    assert 95**9 - 1 < 2**64 <= 95**10 - 1


def test_monotone_all_two_char_prefixes(orc):
    chars = [bytes([c]) for c in range(32, 127)]
    keys = sorted(a + b + b"  " * 4 for a in chars for b in chars)
    enc = [orc.encode9(k) for k in keys]
    assert all(x < y for x, y in zip(enc, enc[1:]))
    assert enc[0] == 0 and enc[-1] == 94 * 95**8 + 94 * 95**7


def test_monotone_random_pairs_vs_memcmp(orc):
    rng = np.random.default_rng(7)
    keys = rng.integers(32, 127, size=(4000, 10), dtype=np.uint8)
    # give neighbours shared prefixes of random length so that ties and late differences occur
    for a in range(0, 4000, 2):
        k = int(rng.integers(0, 11))
        keys[a + 1, :k] = keys[a, :k]
    recs = np.zeros((4000, 100), dtype=np.uint8)
    recs[:, :10] = keys
    enc = orc.encode9_records(recs.reshape(-1))
    for a in range(0, 3999):
        ka, kb = bytes(keys[a][:9]), bytes(keys[a + 1][:9])
        if ka < kb:
            assert enc[a] < enc[a + 1]
        elif ka > kb:
            assert enc[a] > enc[a + 1]
        else:
            assert enc[a] == enc[a + 1]


def test_out_of_range_bytes_saturate(orc):
    assert orc.encode9(b"\x00" * 10) == 0
    assert orc.encode9(b"\xff" * 9 + b" ") == 95**9 - 1
    # after the first byte above 126 every digit is 94; after one below 32 every digit is 0
    assert orc.encode9(b"\x7f" + b" " * 9) == 95**9 - 1
    assert orc.encode9(b"A\x80" + b" " * 8) == 33 * 95**8 + 95**8 - 1
    assert orc.encode9(b"A~\x01~~~~~~~") == 33 * 95**8 + 94 * 95**7
    assert orc.encode9(b"\x1f" + b"~" * 9) == 0


def test_monotone_on_arbitrary_bytes(orc):
    """Eq. 1 needs the encoding monotone in memcmp order for every key, printable or not."""
    rng = np.random.default_rng(3)
    pool = np.array([0, 1, 31, 32, 33, 64, 125, 126, 127, 128, 200, 255], dtype=np.uint8)
    keys = np.where(rng.random((20000, 10)) < 0.5, rng.choice(pool, size=(20000, 10)),
                    rng.integers(0, 256, size=(20000, 10), dtype=np.uint8)).astype(np.uint8)
    keys[1::2, :4] = keys[0::2, :4]  # shared prefixes
    order = sorted(range(len(keys)), key=lambda i: bytes(keys[i]))
    recs = np.zeros((len(keys), 100), dtype=np.uint8)
    recs[:, :10] = keys[order]
    enc = orc.encode9_records(recs.reshape(-1))
    assert np.all(np.diff(enc.astype(np.float64)) >= 0) and np.all(enc[1:] >= enc[:-1])
