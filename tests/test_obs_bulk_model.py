"""A CPU model of the bulk-copy observables kernel's copies and reads
(observables_bulk_kernel in k_field.cu, FP32 real fields): the tile-major
(tile, plane) runs of each block, the bytes each plane's cp.async.bulk
copies, and the shared-memory reads of every site.  For grids the kernel
accepts (planes of whole 16-byte units, a stage of tile + nz + 1 sites within
12 KB) it checks that every copy starts on a 16-byte boundary, moves a whole
number of 16-byte units and stays inside the field; that every read of a
site and of its +y and +z neighbours (where those links exist) falls inside
the copied bytes of its stage, and every read at all inside the stage; and
that every site of every plane is summed exactly once.  This checks the
indexing, not the kernel: tests/test_gpu_lines.py checks its results."""
import pytest

TILE, STAGES, STAGE_BYTES, THREADS, SPT, ELEM = 1024, 8, 12288, 256, 4, 4


def span_of(nz):
    return (TILE + nz + 1 + 3) // 4 * 4


def accepted(shape):
    nx, ny, nz = shape
    return (ny * nz) % 4 == 0 and span_of(nz) * ELEM <= STAGE_BYTES


def grid_of(shape, resident=304):
    nx, ny, nz = shape
    tiles = (ny * nz + TILE - 1) // TILE
    runs = (tiles * nx + 7) // 8
    return max(1, min(resident, runs))


def check(shape):
    nx, ny, nz = shape
    plane = ny * nz
    span = span_of(nz)
    tiles = (plane + TILE - 1) // TILE
    total = tiles * nx
    G = grid_of(shape)
    buf = nx * plane * ELEM
    seen = [0] * (nx * plane)
    for b in range(G):
        lo, hi = total * b // G, total * (b + 1) // G
        assert hi > lo
        r = lo
        while r < hi:
            tile, i0 = divmod(r, nx)
            i1 = min(nx, i0 + (hi - r))
            r += i1 - i0
            s0 = tile * TILE
            nbytes = min(span, plane - s0) * ELEM
            assert nbytes > 0 and nbytes % 16 == 0
            interior = s0 + span <= plane
            pf = i0 - 1 if i0 > 0 else 0
            for i in range(pf, i1):
                src = (i * plane + s0) * ELEM
                assert src % 16 == 0 and src + nbytes <= buf
                if i < i0:
                    continue
                for t in range(THREADS):
                    for m in range(SPT):
                        l = t + m * THREADS
                        s = s0 + l
                        if s >= plane:
                            assert not interior
                            continue
                        j, k = divmod(s, nz)
                        assert (l + 1) * ELEM <= nbytes
                        assert l + nz < span and l + 1 < span  # any read stays in the stage
                        if interior or j + 1 < ny:
                            if j + 1 < ny:
                                assert (l + nz + 1) * ELEM <= nbytes
                        if interior:
                            assert (l + nz + 1) * ELEM <= nbytes and (l + 2) * ELEM <= nbytes
                        elif k + 1 < nz:
                            assert (l + 2) * ELEM <= nbytes
                        seen[i * plane + s] += 1
    assert all(c == 1 for c in seen)
    assert STAGES * span * ELEM + 16 * STAGES <= STAGES * STAGE_BYTES + 16 * STAGES


@pytest.mark.parametrize("shape", [(70, 36, 50), (33, 52, 84), (4, 4, 2046), (6, 6, 1030), (16, 14, 32),
                                   (1, 64, 48), (7, 1, 36), (48, 34, 40), (30, 40, 160)])
def test_bulk_observables_indexing(shape):
    assert accepted(shape)
    check(shape)


@pytest.mark.parametrize("shape", [(4, 4, 2048), (41, 27, 37), (64, 1, 1)])
def test_bulk_observables_refuses(shape):
    assert not accepted(shape)
