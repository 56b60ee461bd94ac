"""CPU checks of the bench's byte models (bench.pass_bytes, bench.truncated_step_cv).

The closed forms are compared with counts made by enumerating the modes of the stored half
spectrum: the planes kz < N/2 of a field volume FV = N^2 N/2 complex values, the rows
(kz, ky) and columns kx kept by the 2/3 rule 3|k| < N, and the box modes of a
component-volume cv = N^2 (N/2 + 1).
"""

import numpy as np
import pytest

import bench


def _freqs(n):
    return np.where(np.arange(n) < n // 2, np.arange(n), np.arange(n) - n)


def _kept(n):
    return 3 * np.abs(_freqs(n)) < n


@pytest.mark.parametrize("N", [96, 256, 512, 1024])
def test_pass_bytes_match_enumerated_rows(N):
    b = 4
    M = N // 2
    fv = N * N * M * 2 * b
    kz_kept = int(np.sum(3 * np.arange(M) < N))  # planes kz < N/3 of the stored kz < N/2
    ky_kept = int(np.sum(_kept(N)))
    kx_kept = ky_kept
    zk, yk, xk = kz_kept / M, ky_kept / N, kx_kept / N
    rk_mean = (9 + 15 + 15 + 9) / 4.0  # RK state read + written per stage, stages 0 .. 3
    full = bench.pass_bytes(N, b)
    assert full["y_inverse"] == pytest.approx(12 * fv)
    assert full["z_pass"] == pytest.approx((6 + 3 * zk) * fv)
    assert full["y_forward"] == pytest.approx((3 * zk + 3 * zk * yk) * fv)
    assert full["x_stage"] == pytest.approx((3 * zk * yk + rk_mean + 6) * fv)
    pr = bench.pass_bytes(N, b, rows=True, box=True)
    assert pr["y_inverse"] == pytest.approx((6 * zk * yk + 6 * zk) * fv)
    assert pr["z_pass"] == pytest.approx(9 * zk * fv)
    assert pr["y_forward"] == pytest.approx(full["y_forward"])
    assert pr["x_stage"] == pytest.approx((3 + rk_mean * xk + 6) * zk * yk * fv)
    rows_only = bench.pass_bytes(N, b, rows=True)
    assert rows_only["x_stage"] == pytest.approx((3 + rk_mean + 6) * zk * yk * fv)
    assert all(pr[k] <= full[k] for k in full)


@pytest.mark.parametrize("N", [32, 256, 512, 1024])
def test_truncated_step_model_counts_the_box(N):
    # box modes of the half spectrum kz = 0 .. N/2, over cv = N^2 (N/2 + 1)
    kz = np.arange(N // 2 + 1)
    b3 = np.sum(3 * kz < N) * np.sum(_kept(N)) ** 2 / (N * N * (N // 2 + 1))
    zk = np.sum(3 * kz < N) / (N // 2 + 1)
    expect = 4 * (6 * b3 + 18 * zk) + 36 * b3
    assert bench.truncated_step_cv(N) == pytest.approx(expect)
    assert 60.0 < bench.truncated_step_cv(N) < 70.0 < bench.STEP_CV
