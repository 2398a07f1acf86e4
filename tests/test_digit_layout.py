"""CPU pin of the packed-digit layout the throughput kernel shares between its
digit pass and its forward transforms (make_digits and the row loop in
br_kernel.cuh), restated from the kernel's index formulas.  Position k = r + 32e
of a 1024-coefficient polynomial (r = k mod 32) is stored in word 4 ((e / 4) XOR
(r mod 8)) + (e mod 4) of row r of a 32 x 32 word block.  The digit pass writes
16-byte chunks: work item it = tid + m T covers row r = it mod 32, chunk
j = (it / 32) mod 8, component c = it / 256, positions r + 32 (4j + i), i < 4.
Lane l of a warp reads chunk q of its row as the 16-byte word l 8 + (q XOR
(l mod 8)) and takes position l + 32 (4q + i) from its word i.

Checked here: every position of both components is written exactly once and read
back at the position it came from; a warp's 16-byte stores and loads touch 32
distinct banks in each group of 8 lanes (one shared-memory wavefront), and the
digit pass's reads of the accumulator (positions r + 32 (4j + i) and their
rotations) touch 32 distinct banks per warp instruction."""
import pytest

N = 1024


def store_word(c, r, j):
    """First 32-bit word of the 16-byte chunk the digit pass writes for (c, r, j)."""
    return c * N + 4 * (r * 8 + (j ^ (r & 7)))


def load_word(lane, q):
    return 4 * (lane * 8 + (q ^ (lane & 7)))


@pytest.mark.parametrize("threads", [64, 128, 192, 384])  # 64 H gate threads, H = 1, 2, 3, 6
def test_every_position_round_trips(threads):
    written = {}
    for tid in range(threads):
        for it in range(tid, 2 * 256, threads):
            r, j, c = it & 31, (it >> 5) & 7, it >> 8
            base = store_word(c, r, j)
            for i in range(4):
                k = r + 32 * (4 * j + i)
                assert (c, base + i) not in written
                written[(c, base + i)] = k
    assert len(written) == 2 * N
    for c in range(2):
        seen = set()
        for lane in range(32):
            for q in range(8):
                for i in range(4):
                    word = c * N + load_word(lane, q) + i
                    assert written[(c, word)] == lane + 32 * (4 * q + i)
                    seen.add(word)
        assert len(seen) == N


def banks_of_16_byte_accesses(words):
    """Banks per group of 8 lanes for 16-byte accesses starting at the given words."""
    groups = []
    for g in range(0, 32, 8):
        banks = []
        for w in words[g:g + 8]:
            banks += [(w + i) % 32 for i in range(4)]
        groups.append(banks)
    return groups


def test_stores_and_loads_are_conflict_free():
    for c in range(2):
        for j in range(8):
            # one warp of the digit pass: 32 consecutive items, rows 0..31, chunk j
            words = [store_word(c, r, j) for r in range(32)]
            for banks in banks_of_16_byte_accesses(words):
                assert len(set(banks)) == 32
    for q in range(8):
        words = [load_word(lane, q) for lane in range(32)]
        for banks in banks_of_16_byte_accesses(words):
            assert len(set(banks)) == 32


@pytest.mark.parametrize("a", [0, 1, 31, 32, 500, 1023, 1024, 1500, 2047])
def test_accumulator_reads_are_conflict_free(a):
    for j in range(8):
        for i in range(4):
            ks = [r + 32 * (4 * j + i) for r in range(32)]
            assert len({k % 32 for k in ks}) == 32  # A[k]
            assert len({((k - a) % 2048 % N) % 32 for k in ks}) == 32  # A[(k - a) mod 2N mod N]
