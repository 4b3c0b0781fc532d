"""Index arithmetic of the row-task launch form, checked on the CPU (no GPU needed).

The kernels cut every search-cell row into 32-particle pieces (count: ceil(len / 32) a
row, exclusive scan, fill) into a buffer of ceil(n / 32) + rows entries, and block b of G
takes the runs of W consecutive pieces numbered b, b + G, b + 2G, ...: a warp's q-th grab
from its block's queue is piece (b + G (q // W)) W + q % W. These tests restate that
arithmetic and check what the kernels rely on: every particle lies in exactly one piece,
the buffer bound holds for any row lengths, and the queue mapping hands out every piece
exactly once across the blocks, in increasing order within a block (so a warp can stop at
its first index past the end)."""
import numpy as np


def pieces_of(row_len):
    cnt = (row_len + 31) // 32
    off = np.concatenate([[0], np.cumsum(cnt)])
    first = np.concatenate([[0], np.cumsum(row_len)])[:-1]
    out = np.zeros((int(off[-1]), 2), dtype=np.int64)
    for r, k_end in enumerate(cnt):
        for k in range(k_end):
            out[off[r] + k] = (first[r] + 32 * k, min(32, row_len[r] - 32 * k))
    return out


def test_pieces_cover_every_particle_once_and_fit_the_buffer():
    rng = np.random.default_rng(5)
    for trial in range(40):
        rows = int(rng.integers(1, 400))
        row_len = rng.integers(0, 300, rows) * (rng.random(rows) < 0.8)   # empty rows too
        n = int(row_len.sum())
        p = pieces_of(row_len)
        assert len(p) <= (n + 31) // 32 + rows                  # the allocated bound
        assert np.all((p[:, 1] >= 1) & (p[:, 1] <= 32))
        seen = np.zeros(n, dtype=np.int64)
        for first, count in p:
            seen[first:first + count] += 1
        assert np.all(seen == 1)
        # a piece never leaves its row
        ends = np.cumsum(row_len)
        for first, count in p:
            r = np.searchsorted(ends, first, side="right")
            assert first + count <= ends[r]


def test_queue_mapping_hands_out_every_piece_once():
    for G in (1, 3, 152):
        for W in (1, 7, 28):
            for total in (0, 1, W * G - 1, W * G, 5 * W * G + 3):
                got = []
                for b in range(G):
                    mine = []
                    q = 0
                    while True:
                        t = (b + G * (q // W)) * W + q % W
                        if t >= total:
                            break
                        mine.append(t)
                        q += 1
                    assert mine == sorted(mine)
                    # the first index past the end is past it for every later grab too
                    t_next = [(b + G * ((q + d) // W)) * W + (q + d) % W for d in range(3 * W)]
                    assert all(t >= total for t in t_next)
                    got += mine
                assert sorted(got) == list(range(total))
