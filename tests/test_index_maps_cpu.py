"""Host checks of the kernels' index maps (restated from solver_kernels.cuh): every tile walk
touches each element of its tile exactly once and stays inside its shared-memory allocation,
for every compiled grid size and precision. A walk that leaves its tile faults the GPU, so
these run on the CPU first."""

import pytest

SIZES = (8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 512, 1024)


def padp(p):
    return p + (p >> 4)


def padded_len(L):
    return L + L // 16 + 1


def pow2_part(n):
    r = 1
    while n % (r * 2) == 0:
        r *= 2
    return r


def odd_ld(lines):
    return lines if lines % 2 else lines + 1


def ycfg(N, cb, inv):
    tx = min(((128 if (inv or cb == 16) and N <= 512 else 64)) // cb, pow2_part(N))
    return tx, odd_ld(tx), padded_len(N) * odd_ld(tx)


def ywalk_row(r, cb, tx, N):
    if cb == 8 and tx == 8 and N % 16 == 0:
        t = r & 15
        u, q = t >> 2, t & 3
        return (r & ~15) | (2 * u + (q >> 1) + (q & 1) * 8)
    return r


@pytest.mark.parametrize("cb", [8, 16])
@pytest.mark.parametrize("inv", [0, 1])
@pytest.mark.parametrize("N", SIZES)
def test_y_tile_walk_is_a_bijection_inside_the_tile(N, cb, inv):
    tx, ld, tile = ycfg(N, cb, inv)
    seen = set()
    for e in range(tx * N):
        x, y = e % tx, ywalk_row(e // tx, cb, tx, N)
        assert 0 <= y < N
        pos = padp(y) * ld + x
        assert 0 <= pos < tile
        seen.add((y, x))
    assert len(seen) == tx * N


def test_z512_tile_walk_covers_the_tile_once():
    # k_zcross16p: kz = 32 g + TX kq + c (g < 8, c < TX, kq = lane / TX), padp(kz) = 34 g + padp(TX kq) + c
    M, TX = 256, 16
    LD = odd_ld(6 * TX)
    seen = set()
    for lane in range(32):
        tx, kq = lane % TX, lane // TX
        for g in range(M // 32):
            for c in range(TX):
                kz = 32 * g + TX * kq + c
                assert padp(kz) == 34 * g + padp(TX * kq) + c
                for f in range(6):
                    pos = padp(kz) * LD + f * TX + tx
                    assert pos < padded_len(M) * LD
                    seen.add((kz, f, tx))
    assert len(seen) == M * 6 * TX


def test_z512_c2r_partner_rows():
    # partner X_{M-k} of k = h + 16 m at padded row pb0 + 17 (15 - m)
    M = 256
    for h in range(16):
        pb0 = 17 if h == 0 else 16 - h
        for m in range(16):
            if h == 0 and m == 0:
                continue  # X_M = 0, not read
            assert padp(M - h - 16 * m) == pb0 + 17 * (15 - m)
            assert pb0 + 17 * (15 - m) < padded_len(M)


@pytest.mark.parametrize("cb", [8, 16])
@pytest.mark.parametrize("N", SIZES)
def test_x_stage_staged_rows_fit(N, cb):
    xls = padded_len(N)
    wide = ((6 * xls + 1) // 2 * 2 + 9 * N) * cb <= 64 * 1024
    xst = ((6 if wide else 3) * xls + 1) // 2 * 2
    pre = (xst + 9 * N) * cb <= 100 * 1024
    if not pre:
        return
    assert (xst * cb) % 16 == 0  # 16-byte cp.async destinations
    if not wide:
        # omega's padded work lines lie over the consumed U1 / U rows 3..8
        assert 3 * N + 3 * xls <= 9 * N


def test_z256_quarter_warp_maps():
    # k_zcross8q: tile walk kz = 32 g + TX kq + c (g < 4) over 16 x and 6 fields; quarter-warp qw of
    # warp group gi takes line 16 (gi >> 2) + 2 (gi & 3) + 8 (qw & 1) + (qw >> 1); lane h < 8 holds
    # k = h + 8 m; exchange at 17 h + k1 inside the padded line
    M, TX, NW = 128, 16, 12
    LD = odd_ld(6 * TX)
    tile = padded_len(M) * LD
    seen = set()
    for lane in range(32):
        tx, kq = lane % TX, lane // TX
        for g in range(M // 32):
            for c in range(TX):
                kz = 32 * g + TX * kq + c
                assert padp(kz) == 34 * g + padp(TX * kq) + c
                for f in range(6):
                    assert padp(kz) * LD + f * TX + tx < tile
                    seen.add((kz, f, tx))
    assert len(seen) == M * 6 * TX
    assert (6 * (M // 32) * TX) % NW == 0
    lines = [16 * (gi >> 2) + 2 * (gi & 3) + 8 * (qw & 1) + (qw >> 1) for gi in range(24) for qw in range(4)]
    assert sorted(lines) == list(range(6 * TX))
    assert sorted(lines[: 12 * 4]) == list(range(3 * TX))
    for h in range(8):
        for k1 in range(16):
            assert 17 * h + k1 < padded_len(M)
        for m in range(16):
            k = h + 8 * m
            if k:
                assert 0 < M - k < M
            # r2c partner Z_{M-k}: lane (8 - h) & 7, slot 15 - m (lane 0: slot (16 - m) & 15)
            src_h, src_m = ((8 - h) & 7, 15 - m) if h else (0, (16 - m) & 15)
            assert (src_h + 8 * src_m) % M == (M - k) % M


def _library_widths(N, cb, which):
    import ctypes

    from paper_1602_03638_gb300 import _lib
    from paper_1602_03638_gb300 import build as B

    B.build()
    buf = (ctypes.c_int * 8)()
    n = _lib.lib().dns_tile_widths(N, 0 if cb == 8 else 1, which, buf, 8)
    assert n >= 0, _lib.last_error()
    return list(buf[:n])


def _zbytes(N, t, cb):
    return padded_len(N // 2) * odd_ld(6 * t) * cb


@pytest.mark.parametrize("cb", [8, 16])
@pytest.mark.parametrize("N", [n for n in SIZES if n <= 128])
def test_offered_tile_widths_divide_the_grid_and_fit(N, cb):
    # the widths a tuner may pick (y-pass: x columns per block; z-pass: x per tile), as the
    # library offers them (dns_tile_widths needs no device), against the rule restated here
    y = _library_widths(N, cb, 0)
    z = _library_widths(N, cb, 1)
    assert y == [t for t in (4, 8, 16, 32) if pow2_part(N) % t == 0 and t * cb <= 256]
    assert z == [t for t in (4, 8, 16, 32) if pow2_part(N) % t == 0 and _zbytes(N, t, cb) <= 112 * 1024]
    for t in y:
        assert N % t == 0
        assert padded_len(N) * odd_ld(t) * cb <= 227 * 1024
        seen = set()
        for e in range(t * N):
            x, row = e % t, ywalk_row(e // t, cb, t, N)
            assert 0 <= row < N and padp(row) * odd_ld(t) + x < padded_len(N) * odd_ld(t)
            seen.add((row, x))
        assert len(seen) == t * N
    for t in z:
        assert N % t == 0
        # tile rows padp(k) (k < N/2) of 6 fields x t columns inside the allocation
        assert padp(N // 2 - 1) * odd_ld(6 * t) + 6 * t - 1 < padded_len(N // 2) * odd_ld(6 * t)


# ---------------------------------------------------------------- x-stage rows of a pruned state

def _kept_rows_map(NY, M, k3y, k3z):
    """The block -> row map of the x-stage launch over the rows inside the 2/3 box
    (xpass_body with compact = true, xpass_kept_ky, x_rows)."""
    R = min((k3y - 1) // 3, NY // 2 - 1)
    kcz = min(M, (k3z + 2) // 3)
    w = 2 * R + 1
    rows = []
    for bx in range(kcz * w):
        t = bx % w
        rows.append((bx // w) * NY + (t if t <= R else NY - w + t))
    return rows


@pytest.mark.parametrize("shape", [(n, n, n) for n in (8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 512, 1024)]
                         + [(32, 16, 24), (24, 48, 16), (1024, 512, 256)])
@pytest.mark.parametrize("variant", [0, 1])
def test_pruned_x_stage_rows_are_exactly_the_kept_rows(shape, variant):
    nx, ny, nz = shape
    M = nz // 2
    k3y, k3z = ny + 2 * variant, nz + 2 * variant
    rows = _kept_rows_map(ny, M, k3y, k3z)
    kept = []
    for kz in range(M):
        for ky in range(ny):
            kf = ky if ky < ny // 2 else ky - ny
            if 3 * kz < k3z and 3 * abs(kf) < k3y:
                kept.append(kz * ny + ky)
    assert sorted(rows) == kept  # a bijection onto the kept rows, in row order per plane
    assert all(0 <= r < M * ny for r in rows)
