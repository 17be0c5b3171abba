"""Loading serialised functions, host side (no device needed).

mphf_load_info decodes a whole blob on the host: the header's sizes, both
Elias-Fano sequences, and every bucket's fixed parts and unary terminators
(Section 2.2, "Representation").  Blobs written from the oracle's arrays must
pass with the oracle's sizes; damaged blobs must be refused, because the
query kernel walks whatever structure it is given.
"""
import ctypes

import numpy as np
import pytest

from paper_2212_09562_b300 import build as B
from paper_2212_09562_b300 import mphf as M
from paper_2212_09562_b300 import workloads as W
from helpers import oracle_blob

CASES = [  # (leaf, bucket, leaf method, tree, key bytes, n)
    (8, 100, M.PLAIN, M.TREE_RECSPLIT, 8, 5000),
    (12, 1000, M.ROTATION, M.TREE_RECSPLIT, 16, 20000),
    (24, 2000, M.SHOCKHASH, M.TREE_FANOUT2, 8, 20000),
    (12, 300, M.SHOCKHASH, M.TREE_RECSPLIT, 8, 9000),
    (10, 500, M.PLAIN, M.TREE_FANOUT2, 16, 8000),
    (5, 1, M.ROTATION, M.TREE_RECSPLIT, 8, 50),  # empty and one-key buckets
    (8, 100, M.ROTATION, M.TREE_RECSPLIT, 8, 1),
    (8, 100, M.ROTATION, M.TREE_RECSPLIT, 8, 0),
]


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.lib()


def _built(orc, leaf, bucket, bij, tree, kb, n):
    keys = W.random_keys(n, kb, 17 * n + leaf)
    o = orc.build_mphf(keys, leaf, bucket, bij, threads=4, tree=tree)
    return o, oracle_blob(o, leaf, bucket, kb, bij, tree)


def _rc(lib, blob: bytes) -> int:
    info = M.Info()
    return lib.mphf_load_info(blob, len(blob), ctypes.byref(info))


@pytest.mark.parametrize("leaf,bucket,bij,tree,kb,n", CASES)
def test_oracle_blobs_load_with_the_oracle_sizes(lib, orc, leaf, bucket, bij, tree, kb, n):
    o, blob = _built(orc, leaf, bucket, bij, tree, kb, n)
    info = M.load_info(blob)
    assert (info.n, info.nb, info.n_nodes, info.gr_bits) == (o.n, o.nb, o.n_nodes, o.gr_bits)
    assert (info.leaf_size, info.bucket_size, info.key_bytes) == (leaf, bucket, kb)
    assert (info.leaf_bijection, info.tree_shape) == (bij, tree)
    assert (info.gr_words, info.ef_words) == (len(o.gr), len(o.ef))
    assert tuple(info.ef_low_bits) == o.ef_L
    sizes = np.diff(o.cum_keys.astype(np.int64))
    assert info.max_bucket == (int(sizes.max()) if len(sizes) else 0)
    # trailing bytes are ignored, and the buffer needs no alignment
    assert M.load_info(blob + b"\0" * 13).n_nodes == o.n_nodes
    shifted = ctypes.create_string_buffer(len(blob) + 8)
    ctypes.memmove(ctypes.addressof(shifted) + 3, blob, len(blob))
    out = M.Info()
    assert lib.mphf_load_info(ctypes.addressof(shifted) + 3, len(blob), ctypes.byref(out)) == M.OK
    assert out.n_nodes == o.n_nodes


def _with_word(blob: bytes, i: int, value: int) -> bytes:
    w = np.frombuffer(blob, np.uint64).copy()
    w[i] = value
    return w.tobytes()


def test_damaged_headers_are_refused(lib, orc):
    o, blob = _built(orc, 12, 1000, M.ROTATION, M.TREE_RECSPLIT, 16, 20000)
    assert _rc(lib, blob) == M.OK
    w = np.frombuffer(blob, np.uint64)
    for i, value in [(0, 0), (1, int(w[1]) + 1), (1, 1 << 32), (2, int(w[2]) + 1),
                     (3, 1), (3, 25), (3, 12 | (2 << 16)), (3, 12 | (1 << 32)), (4, 0), (4, 3001),
                     (5, 12), (6, 3), (7, int(w[7]) + 1), (7, int(w[7]) - 1),
                     (8, int(w[8]) + 1), (9, int(w[9]) - 1), (10, int(w[10]) + 1),
                     (11, int(w[11]) - 1), (12, int(w[12]) + 1), (13, int(w[13]) + 1),
                     (14, int(w[14]) - 1), (15, int(w[15]) + 1), (7, (1 << 64) - 1),
                     (8, (1 << 61)), (9, (1 << 61))]:
        assert _rc(lib, _with_word(blob, i, value)) == M.EINVAL, (i, value)
    for cut in (0, 8, 127, 128, len(blob) - 8, len(blob) - 1):
        assert _rc(lib, blob[:cut]) == M.EINVAL, cut
    assert lib.mphf_load_info(None, 0, ctypes.byref(M.Info())) == M.EINVAL
    assert lib.mphf_load_info(blob, len(blob), None) == M.EINVAL
    h = ctypes.c_void_p(5)
    assert lib.mphf_load(blob[:100], 100, None, None, ctypes.byref(h)) == M.EINVAL
    assert h.value is None  # refused before any device call


def _flip(blob: bytes, bit: int) -> bytes:
    b = bytearray(blob)
    b[bit >> 3] ^= 1 << (bit & 7)
    return bytes(b)


@pytest.mark.parametrize("bij,tree", [(M.ROTATION, M.TREE_RECSPLIT), (M.SHOCKHASH, M.TREE_FANOUT2)])
def test_flipped_bits_in_the_unary_parts_are_refused(lib, orc, bij, tree):
    """Every bit of a few buckets flipped in turn.  A bucket's code is its
    nodes' fixed parts, then their unary parts (Section 2.2,
    "Representation").  A flip in a unary part adds or removes a terminator
    and must be refused; a flip in a fixed part only changes a value and
    loads.  So in every bucket the accepted flips form a prefix of its bits,
    the refused ones the rest, and at least one refused bit per node."""
    leaf = 8 if tree == M.TREE_RECSPLIT else 24
    o, blob = _built(orc, leaf, 200, bij, tree, 8, 3000)
    head_bits = 16 * 64
    pos = o.bit_pos.astype(np.int64)
    nodes = np.diff(o.node_off.astype(np.int64))
    for b in (0, 1, o.nb // 2, o.nb - 1):
        codes = [_rc(lib, _flip(blob, head_bits + int(p))) for p in range(pos[b], pos[b + 1])]
        assert set(codes) <= {M.OK, M.EINVAL}
        first_refused = codes.index(M.EINVAL)
        assert all(v == M.OK for v in codes[:first_refused])
        assert all(v == M.EINVAL for v in codes[first_refused:])
        assert len(codes) - first_refused >= nodes[b]


def test_flipped_bits_in_the_elias_fano_high_vectors_are_refused(lib, orc):
    o, blob = _built(orc, 12, 300, M.ROTATION, M.TREE_RECSPLIT, 8, 9000)
    k = o.nb + 1
    start = 16 * 64 + 64 * len(o.gr)
    l0 = (k * o.ef_L[0] + 63) // 64
    h0 = ((o.n >> o.ef_L[0]) + k + 63) // 64
    l1 = (k * o.ef_L[1] + 63) // 64
    h1 = ((o.gr_bits >> o.ef_L[1]) + k + 63) // 64
    for first, count in ((start + 64 * l0, h0), (start + 64 * (l0 + h0 + l1), h1)):
        for bit in range(first, first + 64 * count):
            assert _rc(lib, _flip(blob, bit)) == M.EINVAL, bit


def test_random_damage_never_passes_unnoticed_as_a_different_shape(lib, orc):
    """Random bit flips anywhere: each blob is refused or loads with the
    original's sizes (a flip in a fixed part, or in a header field that the
    query does not use, such as b when ceil(n / b) is unchanged)."""
    o, blob = _built(orc, 16, 300, M.ROTATION, M.TREE_RECSPLIT, 8, 3000)
    rng = np.random.default_rng(11)
    ok = 0
    for bit in rng.integers(0, 8 * len(blob), 3000):
        damaged = _flip(blob, int(bit))
        info = M.Info()
        rc = lib.mphf_load_info(damaged, len(damaged), ctypes.byref(info))
        assert rc in (M.OK, M.EINVAL)
        if rc == M.OK:
            ok += 1
            assert (info.n, info.nb, info.n_nodes, info.gr_bits) == (o.n, o.nb, o.n_nodes, o.gr_bits)
    assert 0 < ok < 3000


def test_serialised_fixture_is_still_what_the_oracle_writes(lib, orc):
    """tests/golden/serialised_l8_rotation.txt pins the byte layout: the
    oracle today writes the same words and the same values, and the
    library's host decoder accepts them with the stored sizes."""
    from helpers import read_serialised_fixture
    p, blob, keys, values = read_serialised_fixture()
    assert len(keys) == p["n"]
    o = orc.build_mphf(keys, p["leaf"], p["bucket"], p["bijection"], tree=p["tree"])
    assert oracle_blob(o, p["leaf"], p["bucket"], p["key_bytes"], p["bijection"], p["tree"]) == blob
    assert np.array_equal(o.query(keys), values)
    assert np.array_equal(np.sort(values), np.arange(p["n"], dtype=np.uint64))
    info = M.load_info(blob)
    assert (info.n, info.nb, info.n_nodes) == (p["n"], 3, o.n_nodes)


def test_mutated_headers_and_lengths_never_crash_the_decoder(lib):
    """20,000 mutations of the golden blob (header words random or small,
    payload words random, lengths cut): the host decoder returns OK or
    EINVAL every time.  Each buffer holds exactly the given length, so a
    read far past it would crash the test; small over-reads are caught by
    reading the decoder's bounds, not here."""
    from helpers import read_serialised_fixture
    _, blob, _, _ = read_serialised_fixture()
    w0 = np.frombuffer(blob, np.uint64).copy()
    rng = np.random.default_rng(2212)
    seen = {M.OK: 0, M.EINVAL: 0}
    for it in range(20_000):
        w = w0.copy()
        kind = it % 4
        if kind == 0:
            w[rng.integers(1, 16)] = rng.integers(0, 2**63, dtype=np.uint64) >> np.uint64(rng.integers(0, 63))
        elif kind == 1:
            for i in rng.integers(1, 16, 3):
                w[i] = rng.integers(0, 300)
        elif kind == 2:
            for i in rng.integers(16, len(w), 3):
                w[i] = rng.integers(0, 2**63, dtype=np.uint64)
        b = w.tobytes()
        length = len(b) if kind != 3 else int(rng.integers(0, len(b) + 1))
        buf = ctypes.create_string_buffer(b[:length], length)  # exactly `length` bytes
        rc = lib.mphf_load_info(buf, length, ctypes.byref(M.Info()))
        seen[rc] += 1
    assert seen[M.OK] > 0 and seen[M.EINVAL] > 0
