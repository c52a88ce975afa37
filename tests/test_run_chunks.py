"""How the multi-step schedule groups a batch into launches (host arithmetic
of the C ABI, no GPU): every lattice in one chunk, at most 32 lattices and
80 MiB of populations per chunk (a larger lattice alone), lattices taken
largest first, as few chunks as those limits allow, and the bytes spread
evenly over the chunks."""
import numpy as np
import pytest

import paper_1412_7228_gb300 as P

MIB = 1 << 20
LIMIT = 80 * MIB
MAX_INST = 32


def pop_bytes(nx, ny, prec):
    """Populations of both time levels of one lattice, from the documented
    layout: nine planes of (ny + 4) rows (two ghost rows each side) of a
    pitch that holds 32 bytes of ghost columns on the left, the row and two
    ghost columns on the right, rounded up to 32 bytes."""
    es = 4 if prec == P.LBM_FP32 else 8
    per32 = 32 // es
    pitch = -(-(32 // es + nx + 2) // per32) * per32
    return 2 * 9 * pitch * (ny + 4) * es


def plan(shapes, prec=P.LBM_FP32):
    nx = [s[0] for s in shapes]
    ny = [s[1] for s in shapes]
    chunk_of = P.lbm_run_chunk_plan(nx, ny, prec)
    n = max(chunk_of) + 1
    return [[i for i in range(len(shapes)) if chunk_of[i] == k] for k in range(n)]


def check_plan(shapes, prec=P.LBM_FP32):
    chunks = plan(shapes, prec)
    b = [pop_bytes(nx, ny, prec) for nx, ny in shapes]
    # a partition of the lattices into non-empty chunks
    assert sorted(i for c in chunks for i in c) == list(range(len(shapes)))
    assert all(c for c in chunks)
    for c in chunks:
        assert len(c) <= MAX_INST
        assert len(c) == 1 or sum(b[i] for i in c) <= LIMIT
    # largest first: nothing in a later chunk is larger than anything before it
    for k in range(len(chunks) - 1):
        assert min(b[i] for i in chunks[k]) >= max(b[i] for i in chunks[k + 1])
    # as few chunks as the limits allow: filling each chunk to its limits,
    # largest first, needs no fewer
    need, cur, cnt = 0, 0, 0
    for x in sorted(b, reverse=True):
        if cnt and (cnt == MAX_INST or cur + x > LIMIT):
            need, cur, cnt = need + 1, 0, 0
        cur, cnt = cur + x, cnt + 1
    need += 1
    assert len(chunks) == need
    return chunks, b


def test_sixty_equal_droplets_go_in_four_chunks_of_fifteen():
    chunks, b = check_plan([(256, 256)] * 60)
    assert [len(c) for c in chunks] == [15] * 4
    assert b[0] * 16 <= LIMIT < b[0] * 17      # sixteen would fit: evenness, not the limit, cuts at 15


def test_small_lattices_are_cut_at_32_and_spread_evenly():
    chunks, _ = check_plan([(64, 64)] * 70)
    assert sorted(len(c) for c in chunks) == [23, 23, 24]
    chunks, _ = check_plan([(64, 64)] * 32)
    assert [len(c) for c in chunks] == [32]


def test_a_lattice_larger_than_the_limit_is_a_chunk_of_its_own():
    chunks, b = check_plan([(128, 128), (4096, 4096), (256, 256)])
    assert b[1] > LIMIT and chunks == [[1], [0, 2]]


def test_the_batched_sweep_configuration():
    """64 droplets, L uniform over {128, 256, 512, 1024} (seed 7228): each
    1024^2 lattice alone (73 MiB), the 512^2 ones four to a chunk, the
    256^2 and 128^2 ones together."""
    from paper_1412_7228_gb300 import sweep as SW
    drops = SW.sweep_droplets(64, 7228)
    shapes = [(d.L, d.L) for d in drops]
    chunks, _ = check_plan(shapes)
    sizes = [sorted({shapes[i][0] for i in c}) for c in chunks]
    n1024 = sum(1 for s in shapes if s[0] == 1024)
    n512 = sum(1 for s in shapes if s[0] == 512)
    assert sizes[:n1024] == [[1024]] * n1024
    assert sizes[n1024:n1024 + -(-n512 // 4)] == [[512]] * -(-n512 // 4)
    assert sizes[-1] == [128, 256] and len(chunks) == n1024 + -(-n512 // 4) + 1


def test_equal_sizes_keep_index_order_and_fp64_doubles_the_bytes():
    chunks, _ = check_plan([(200, 100)] * 40)
    assert [i for c in chunks for i in c] == list(range(40))
    c32 = plan([(512, 512)] * 8, P.LBM_FP32)
    c64 = plan([(512, 512)] * 8, P.LBM_FP64)
    assert [len(c) for c in c32] == [4, 4] and [len(c) for c in c64] == [2, 2, 2, 2]


@pytest.mark.parametrize("seed", range(6))
def test_random_uneven_batches(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 120))
    shapes = [(int(rng.integers(2, 1500)), int(rng.integers(2, 1500))) for _ in range(n)]
    for prec in (P.LBM_FP32, P.LBM_FP64):
        check_plan(shapes, prec)


def test_bad_shapes_are_refused():
    with pytest.raises(P.LbmError):
        P.lbm_run_chunk_plan([1], [64], P.LBM_FP32)
    with pytest.raises(P.LbmError):
        P.lbm_run_chunk_plan([64], [64], 3)
    with pytest.raises(P.LbmError):
        P.lbm_run_chunk_plan([], [], P.LBM_FP32)
